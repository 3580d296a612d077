"""Pins of the oracle's weighted 1D operators and of the global-local iteration for
solution-dependent coefficients (App. A, Algorithm 2; Sec. 3.3)."""
import math

import numpy as np
import pytest

from oracle import taps_oracle as O
from paper_2503_13933_gb300 import workloads as W


@pytest.mark.parametrize("s,p", [(1, 1), (2, 2), (3, 3)])
def test_weighted_ops_with_unit_weight_are_the_plain_ops(s, p):
    dm = O.Dim(n=13, lo=-0.5, hi=1.5, s=s, p=p)
    full = O.assemble_full(dm)
    one = np.ones(dm.n)
    for base, op in (("K", O.OP_K), ("M", O.OP_M), ("G", O.OP_G)):
        A = O.assemble_weighted(dm, base, one)
        assert np.max(np.abs(A - full[op])) <= 1e-13 * np.max(np.abs(full[op])), base


def test_weighted_mass_reproduces_polynomial_weights():
    """C-HiDeNN reproduces polynomials up to order p: the nodal values of
    w = 1 + 2x - x^2 (p = 2) weight the mass exactly as the weight-polynomial operator
    W of the same w (an independent code path: w evaluated in closed form)."""
    dm = O.Dim(n=11, lo=0.0, hi=2.0, s=2, p=2, weight_poly=(1.0, 2.0, -1.0, 0.0))
    w = 1.0 + 2.0 * dm.x - dm.x ** 2
    A = O.assemble_weighted(dm, "M", w)
    Wm = O.assemble_full(dm)[O.OP_W]
    assert np.max(np.abs(A - Wm)) <= 1e-12 * np.max(np.abs(Wm))


@pytest.mark.parametrize("s,p", [(1, 1), (2, 2), (3, 3)])
def test_weighted_ops_sum_rules(s, p):
    """Partition of unity (sum_i N~_i = 1, sum_i B~_i = 0) with a random weight field:
    the columns of K^w sum to 0; the entries of M^w sum to int w; the columns of G^w
    sum to the boundary term w N~_j at the ends (int (w N~_j)' dx), i.e. w_n at the
    last node, -w_1 at the first (Kronecker delta) and 0 elsewhere."""
    rng = np.random.default_rng(4)
    dm = O.Dim(n=15, lo=0.0, hi=3.0, s=s, p=p)
    w = rng.uniform(0.5, 2.0, dm.n)
    K = O.assemble_weighted(dm, "K", w)
    Mw = O.assemble_weighted(dm, "M", w)
    G = O.assemble_weighted(dm, "G", w)
    scale = np.max(np.abs(K))
    assert np.max(np.abs(K.sum(axis=0))) <= 1e-12 * scale
    int_w = sum(wj * (np.asarray(N) @ w[np.array(ids)]) for pts in O.shape_tables(dm) for _, wj, ids, N, _ in pts)
    assert abs(Mw.sum() - int_w) <= 1e-13 * abs(int_w)
    expect = np.zeros(dm.n)
    expect[0], expect[-1] = -w[0], w[-1]
    assert np.max(np.abs(G.sum(axis=0) - expect)) <= 1e-12 * np.max(np.abs(G))


def test_manufactured_source_is_the_residual_of_the_exact_solution():
    """The manufactured nonlinear source as built (product-to-sum harmonics) matches
    d/dt[c(u) u] - d/dx(k(u) du/dx) of the exact solution by central differences."""
    desc = W.nonlinear_manufactured(8)
    m_c, n_c, m_k, n_k = W.NONLINEAR_LAW
    u = lambda x, t: W.nonlinear_exact(np.array([[x, t]]))[0]
    rng = np.random.default_rng(0)
    h = 1e-4
    for _ in range(6):
        x, t = rng.uniform(0.05, 0.95, 2)
        f = 0.0
        for beta, fac in desc["sources"]:
            v = beta
            for (kind, par), z in zip(fac, (x, t)):
                v *= par[0] if kind == "const" else math.sin(par[0] * z + par[1])
            f += v
        cu = lambda x, t: (m_c * u(x, t) + n_c) * u(x, t)
        flux = lambda y: (m_k * u(y, t) + n_k) * (u(y + h, t) - u(y - h, t)) / (2 * h)
        ref = (cu(x, t + h) - cu(x, t - h)) / (2 * h) - (flux(x + h) - flux(x - h)) / (2 * h)
        assert abs(f - ref) <= 1e-5 * (1.0 + abs(ref)), (x, t, f, ref)


def test_global_local_iteration_converges_to_the_exact_solution():
    """Algorithm 2 on the manufactured problem (s = p = 2, M = 3, 6 subspace iterations
    per global stage): the fixed point is reached (change <= 1e-7 within 15 global
    iterations) and its error against the exact solution falls at order >= 2.5 from
    12 to 24 nodes per dim (p + 1 = 3), below 1e-3 at 24."""
    errs = []
    X = np.random.default_rng(0).uniform(size=(3000, 2))
    for n in (12, 24):
        desc = W.nonlinear_manufactured(n)
        U, hist = O.nonlinear_solve(desc, W.NONLINEAR_LAW, M=3, sweeps=6, max_iters=15, tol=1e-7, seed=1)
        assert hist[-1] <= 1e-7, hist
        Po = O.problem_from_description(O.nonlinear_global_description(desc, W.NONLINEAR_LAW, None))
        got = O.eval_points(Po, U, X)
        ref = W.nonlinear_exact(X)
        errs.append(math.sqrt(np.sum((got - ref) ** 2) / np.sum(ref ** 2)))
    rate = math.log(errs[0] / errs[1]) / math.log(23 / 11)
    assert errs[1] < 1e-3 and rate > 2.5, (errs, rate)


def test_linear_laws_with_zero_slope_reduce_to_one_linear_solve():
    """m_c = m_k = 0: the global stage is the linear heat problem with c = n_c, k = n_k
    (no weighted operators), so the iteration stops after the second global stage with
    the linear solution."""
    desc = W.nonlinear_manufactured(10)
    law = (0.0, 1.3, 0.0, 0.7)
    g = O.nonlinear_global_description(desc, law, None)
    assert all(not wl for wl in g["weighted"]) and len(g["terms"]) == 2
    U, hist = O.nonlinear_solve(desc, law, M=3, sweeps=40, max_iters=5, tol=1e-9, seed=1)
    assert len(hist) <= 3


@pytest.mark.parametrize("D,M,law", [(2, 3, W.NONLINEAR_LAW), (4, 5, W.INCONEL_LAW), (3, 1, (0.0, 1.0, 0.2, 1.0)),
                                     (4, 2, (0.3, 1.0, 0.0, 2.0))])
def test_library_global_stage_terms_match_the_oracle_reading(D, M, law):
    """The library's global-stage term structure (host logic of nonlinear.py) equals the
    oracle's reading of Algorithm 2's weak form: the same terms in the same order and,
    per dim, the same weighted operators (base and mode) behind each 'w<j>' name."""
    from paper_2503_13933_gb300 import nonlinear as NL
    terms, wops = NL.global_terms(D, M, law)
    dims = [dict(n=6, dirichlet_lo=True, dirichlet_hi=True)] * D
    V = [np.tile(np.arange(1.0, M + 1.0), (6, 1)) * (d + 1) for d in range(D)]
    g = O.nonlinear_global_description(dict(dims=dims, sources=[]), law, V)
    assert g["terms"] == terms
    for d in range(D):
        assert [b for b, _ in g["weighted"][d]] == [b for b, _ in wops[d]]
        for (b, w), (b2, j) in zip(g["weighted"][d], wops[d]):
            assert np.array_equal(w, V[d][:, j])


def _expanded_change(U_new, U_old):
    """|a|^2 + |b|^2 - 2 <a, b> from Gram products (the form that cancels)."""
    A = [np.concatenate([a, b], axis=1) for a, b in zip(U_new, U_old)]
    G = np.ones((A[0].shape[1],) * 2)
    for a in A:
        G *= a.T @ a
    m = U_new[0].shape[1]
    c = np.concatenate([np.ones(m), -np.ones(U_old[0].shape[1])])
    return math.sqrt(max(float(c @ G @ c), 0.0) / float(np.sum(G[:m, :m])))


@pytest.mark.parametrize("rel", [1e-1, 1e-4, 1e-9])
def test_cp_change_equals_explicit_tensor_difference(rel):
    """The convergence check of Algorithm 2 against its plain definition: the norm of
    the difference of the two full nodal tensors (3 dims of 7, 6 and 5 nodes; 4 modes
    against 3, then a perturbation of relative size `rel` of the same 4 modes).  The
    telescoped form keeps ~1e-6 relative accuracy down to changes of 1e-9, where the
    expanded Gram form has lost every digit."""
    rng = np.random.default_rng(17)
    A = [rng.uniform(-1, 1, (n, 4)) for n in (7, 6, 5)]
    B3 = [a[:, :3] + 0.3 * rng.uniform(-1, 1, (a.shape[0], 3)) for a in A]
    a_full = O.cp_full(A)
    got = O.cp_change(A, B3)
    ref = np.linalg.norm(a_full - O.cp_full(B3)) / np.linalg.norm(a_full)
    assert abs(got - ref) <= 1e-12 * ref
    B = [a + rel * rng.uniform(-1, 1, a.shape) for a in A]
    got = O.cp_change(A, B)
    ref = np.linalg.norm(a_full - O.cp_full(B)) / np.linalg.norm(a_full)
    # the explicit difference itself carries ~eps / rel relative rounding
    assert abs(got - ref) <= max(1e-12, 1e-6 * 1e-9 / rel) * ref + 1e-15, (got, ref)
    assert O.cp_change(A, A) == 0.0
    if rel == 1e-9:   # the expanded form cannot resolve this change
        assert abs(_expanded_change(A, B) - ref) > 0.5 * ref
