"""Pin of the oracle's Eq. 42 residual (the stopping quantity of the subspace
iteration, Sec. 2.6) against an explicit full-grid evaluation.

The reduced system of dim d (Eq. 42/43) is the Galerkin projection of A u = F onto the
test functions e_i (x) (x)_{e != d} U_e[:, m].  So its residual is, entry by entry,

    r_d[i, m] = (e_i (x)_{e != d} U_e[:, m])^T (A vec(u) - F),
    F_d[i, m] = (e_i (x)_{e != d} U_e[:, m])^T F,

with A and F assembled explicitly as Kronecker sums and u = sum_m (x)_d U_d[:, m] the
full tensor.  The oracle forms the same quantity from 1D Gram products and Hadamard
coefficients (no Kronecker product anywhere), so agreement to rounding pins its
normalisation (||F_d||, not ||F||), its norm (Frobenius, not max-abs), its coefficient
set (all other factors at their current values) and the index convention of the
coefficient matrices (test mode m, trial mode n), which matters once a G term makes
them nonsymmetric.  A copy of the oracle with one planted mistake must fail the pin.
"""
import numpy as np
import pytest

from oracle import taps_oracle as O
from paper_2503_13933_gb300 import workloads as W


def _projector(prob, U, d):
    """Columns e_i (x)_{e != d} U_e[:, m] in the order (i, m), i major (C order of the
    full tensor: the last dim fastest)."""
    n = prob.nfree
    M = U[0].shape[1]
    cols = []
    for i in range(n[d]):
        for m in range(M):
            v = np.ones(1)
            for e in range(prob.D):
                if e == d:
                    f = np.zeros(n[d])
                    f[i] = 1.0
                else:
                    f = U[e][:, m]
                v = np.kron(v, f)
            cols.append(v)
    return np.stack(cols, axis=1)


def _explicit_rho42(prob, U, per_dim=False):
    A = O.full_operator(prob)
    F = O.full_rhs(prob)
    res = A @ O.cp_full(U) - F
    out = []
    for d in range(prob.D):
        P = _projector(prob, U, d)
        out.append(np.linalg.norm(P.T @ res) / np.linalg.norm(P.T @ F))
    return out if per_dim else max(out)


def _rich_sources(desc, R=4, seed=7):
    """Replace the sources by R random separable nodal terms (U(-1, 1) values at all
    nodes), so that the right-hand side has rank > M and the sweeps keep the modes
    apart (a single smooth source makes fixed-M modes collinear)."""
    rng = np.random.default_rng(seed)
    desc = dict(desc)
    desc["sources"] = [(1.0, [("nodal", rng.uniform(-1.0, 1.0, dm["n"])) for dm in desc["dims"]])
                       for _ in range(R)]
    return desc


CASES = [
    ("poisson 3D, no G", lambda: _rich_sources(W.poisson_sin(8, D=3))),
    ("transient 2D + t (G term)", lambda: W.heat_transient(n_space=8, n_t=6, D_space=2, seed=3021)),
    ("space-parameter 4D", lambda: W.poisson_k(n_space=7, n_k=5, seed=2031)),
    ("transient 3D + t, convection face (G and B terms)",
     lambda: W.heat_transient(n_space=6, n_t=5, D_space=3, h_conv=1.5, seed=3022)),
]


def _states(prob, M=3, seed=11):
    """Random factors, and the factors after one and two sweeps (not a fixed point)."""
    U = O.init_factors(prob, M, "random", seed)
    out = [U]
    for _ in range(2):
        U, _ = O.sweep(prob, U)
        out.append(U)
    return out


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_eq42_residual_equals_explicit_projection(name, make):
    prob = O.problem_from_description(make())
    for U in _states(prob):
        a = O.als_residual(prob, U)
        b = _explicit_rho42(prob, U)
        assert b > 1e-8          # not at a fixed point: the comparison has digits
        assert abs(a - b) <= 1e-12 * b, (name, a, b)


def _mutant_full_norm(prob, U):
    """Planted mistake: normalised by ||F|| (full grid) instead of ||F_d||."""
    nF = np.linalg.norm(O.full_rhs(prob))
    worst = 0.0
    for d in range(prob.D):
        C, F = O.coefficients(prob, U, d)
        r = -F.copy()
        for op, Cop in C.items():
            r += prob.ops[d][op] @ U[d] @ Cop.T
        worst = max(worst, np.linalg.norm(r) / nF)
    return worst


def _mutant_max_abs(prob, U):
    """Planted mistake: max-abs entries instead of Frobenius norms."""
    worst = 0.0
    for d in range(prob.D):
        C, F = O.coefficients(prob, U, d)
        r = -F.copy()
        for op, Cop in C.items():
            r += prob.ops[d][op] @ U[d] @ Cop.T
        worst = max(worst, np.max(np.abs(r)) / np.max(np.abs(F)))
    return worst


def _mutant_transposed(prob, U):
    """Planted mistake: C_op instead of C_op^T (test and trial modes swapped)."""
    worst = 0.0
    for d in range(prob.D):
        C, F = O.coefficients(prob, U, d)
        r = -F.copy()
        for op, Cop in C.items():
            r += prob.ops[d][op] @ U[d] @ Cop
        worst = max(worst, np.linalg.norm(r) / np.linalg.norm(F))
    return worst


def _mutant_stale(prob, U):
    """Planted mistake: coefficients of dim d from the factors as they were before dim
    d's own update in a sweep (a residual that any ALS fixed point also zeroes)."""
    V = [u.copy() for u in U]
    V[0] = V[0] * 1.1      # stands in for an out-of-date factor of another dim
    worst = 0.0
    for d in range(1, prob.D):
        C, F = O.coefficients(prob, V, d)
        r = -F.copy()
        for op, Cop in C.items():
            r += prob.ops[d][op] @ U[d] @ Cop.T
        worst = max(worst, np.linalg.norm(r) / np.linalg.norm(F))
    return worst


@pytest.mark.parametrize("mutant", [_mutant_full_norm, _mutant_max_abs, _mutant_transposed, _mutant_stale],
                         ids=["norm_by_F", "max_abs", "transposed_C", "stale_coefficients"])
def test_planted_mistakes_fail_the_pin(mutant):
    """Each plausible mistake in the residual moves it well outside the pin's 1e-12 on
    at least one case (the transposed coefficients only show with a G term)."""
    worst = 0.0
    for _, make in CASES:
        prob = O.problem_from_description(make())
        for U in _states(prob)[1:]:
            b = _explicit_rho42(prob, U)
            worst = max(worst, abs(mutant(prob, U) - b) / b)
    assert worst > 1e-3, worst


def test_eq42_residual_tracks_full_residual_at_full_rank():
    """At a mode count that holds every grid function (D = 2, 6 free nodes per dim,
    M = 6) the subspace iteration reaches the full-grid solution, where the full
    residual and the Eq. 42 residual (a projection of it) both vanish to rounding."""
    prob = O.problem_from_description(_rich_sources(W.poisson_sin(8, D=2), R=6))
    r = O.solve(prob, M0=6, M_max=6, als_tol=1e-14, res_tol=-1.0, max_sweeps=200, init="random", seed=4)
    rho_full = O.residual_explicit(prob, r.U)
    assert rho_full < 1e-10
    assert O.als_residual(prob, r.U) < 1e-10
