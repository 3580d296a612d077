"""Solution-dependent coefficients on the GPU (App. A, Algorithm 2): the weighted 1D
operators element by element against the oracle, sweeps of a global stage with more
distinct operators per dim than the plain kinds, and the global-local iteration against
the oracle's and against the manufactured exact solution."""
import math

import numpy as np
import pytest

from oracle import taps_oracle as O
from paper_2503_13933_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_13933_gb300 import build, taps
    build.build()
    taps.lib()
    return taps


def to_band(A, hb):
    n = A.shape[0]
    out = np.zeros((n, 2 * hb + 1))
    for i in range(n):
        for k in range(2 * hb + 1):
            j = i + k - hb
            if 0 <= j < n:
                out[i, k] = A[i, j]
    return out


def _global(n, M, seed):
    """The global stage of the manufactured problem at random weights (modes of a
    seeded random u at all nodes, zero at the constrained ones)."""
    from paper_2503_13933_gb300 import nonlinear as NL
    desc = W.nonlinear_manufactured(n)
    terms, wops = NL.global_terms(2, M, W.NONLINEAR_LAW)
    rng = np.random.default_rng(seed)
    V = []
    for dm in desc["dims"]:
        v = rng.uniform(-1, 1, (dm["n"], M))
        if dm["dirichlet_lo"]:
            v[0] = 0.0
        if dm["dirichlet_hi"]:
            v[-1] = 0.0
        V.append(v)
    weighted = [[(b, V[d][:, j]) for b, j in wops[d]] for d in range(2)]
    return dict(desc, terms=terms, weighted=weighted)


@pytest.mark.parametrize("s,p", [(1, 1), (2, 2), (3, 3)])
def test_weighted_operator_bands_parity(T, s, p):
    """Every weighted operator of a global stage (K, M in space, G, M in time; random
    weights) against the oracle's assembly restricted to the free nodes, within the
    plain operators' assembly bound (5e-12 of the largest entry: the s = p = 3 shape
    functions carry ~1e-12 of the patch inverse's rounding)."""
    desc = _global(17, 3, seed=5)
    for dm in desc["dims"]:
        dm.update(s=s, p=p)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    for d in range(2):
        hb = P.dims[d].hb
        for j in range(len(desc["weighted"][d])):
            ref = to_band(Po.ops[d][O.OP_WEIGHTED + j], hb)
            got = P.op_band(d, f"w{j}")
            assert np.max(np.abs(got - ref)) <= 5e-12 * np.max(np.abs(ref)), (d, j)


def test_global_stage_sweeps_match_oracle(T):
    """8 distinct operators per dim (2 plain + 6 weighted), M = 3: three sweeps from the
    same factors give the oracle's normalised factors to 1e-10, and the Eq. 42 residual
    of the result matches."""
    desc = _global(20, 3, seed=6)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, 3, seed=7)
    U = P.factors(3)
    U.set(U0)
    P.sweep(U, 3, solver=T.SOLVER_BLOCK_LU)
    Uo = [u.copy() for u in U0]
    for _ in range(3):
        Uo, _ = O.sweep(Po, Uo)
    for d, (g, o) in enumerate(zip(U.get(), Uo)):
        assert np.max(np.abs(g - o)) < 1e-10 * np.max(np.abs(o)), d
    rho = P.residual(U, T.RES_ALS)
    assert abs(rho - O.als_residual(Po, U.get())) <= 1e-8 * max(rho, 1e-300)


def test_global_stage_many_operators_sweeps_match_oracle(T):
    """34 distinct operators per dim (2 plain + 32 weighted: a global stage at 16
    weight modes), M = 3: more operators than one CTA of the Gram chunk sums has warps,
    so each warp adds several operators' entries; three sweeps from the same factors give
    the oracle's normalised factors to 1e-10 and the Eq. 42 residual matches."""
    desc = _global(20, 16, seed=8)
    assert all(len(w) + 2 > 32 for w in desc["weighted"])
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, 3, seed=9)
    U = P.factors(3)
    U.set(U0)
    P.sweep(U, 3, solver=T.SOLVER_BLOCK_LU)
    Uo = [u.copy() for u in U0]
    for _ in range(3):
        Uo, _ = O.sweep(Po, Uo)
    for d, (g, o) in enumerate(zip(U.get(), Uo)):
        assert np.max(np.abs(g - o)) < 1e-10 * np.max(np.abs(o)), d
    rho = P.residual(U, T.RES_ALS)
    assert abs(rho - O.als_residual(Po, U.get())) <= 1e-8 * max(rho, 1e-300)


def test_weighted_ops_must_be_defined_before_a_sweep(T):
    from paper_2503_13933_gb300 import nonlinear as NL
    desc = W.nonlinear_manufactured(12)
    terms, _ = NL.global_terms(2, 2, W.NONLINEAR_LAW)
    P = T.Problem(dict(desc, terms=terms))
    U = P.factors(2)
    U.set(W.random_factors(desc, 2, seed=1))
    with pytest.raises(T.TapsError):
        P.sweep(U, 1)


def test_global_local_iteration_matches_oracle(T):
    """Algorithm 2 on the manufactured problem, 16 nodes per dim, M = 3, 6 subspace
    iterations per global stage, from the same factors: the GPU's fixed point is the
    oracle's (nodal fields to 1e-9) after the same number of global stages (+-1)."""
    from paper_2503_13933_gb300 import nonlinear as NL
    desc = W.nonlinear_manufactured(16)
    U0 = W.random_factors(dict(desc, terms=[]), 3, seed=11)
    gl = NL.GlobalLocal(desc, W.NONLINEAR_LAW, 3)
    U, hist = gl.solve(6, max_iters=20, tol=1e-7, U0=U0)
    Uo, ho = O.nonlinear_solve(desc, W.NONLINEAR_LAW, M=3, sweeps=6, max_iters=20, tol=1e-7, U0=U0)
    assert hist[-1] <= 1e-7 and ho[-1] <= 1e-7
    assert abs(len(hist) - len(ho)) <= 1, (hist, ho)
    ug, uo = O.cp_full(U), O.cp_full(Uo)
    assert np.max(np.abs(ug - uo)) <= 1e-9 * np.max(np.abs(uo))


def test_global_local_iteration_converges_to_exact_solution(T):
    """The GPU's fixed point against the exact solution at 24, 48 and 96 nodes per dim
    (s = p = 2, M = 3): error falling at order >= 2.5 (p + 1 = 3), from 8192 random
    points evaluated on the device."""
    from paper_2503_13933_gb300 import nonlinear as NL
    X = np.random.default_rng(3).uniform(size=(8192, 2))
    pts = torch.as_tensor(X, device="cuda")
    errs = []
    for n in (24, 48, 96):
        desc = W.nonlinear_manufactured(n)
        gl = NL.GlobalLocal(desc, W.NONLINEAR_LAW, 3)
        U, hist = gl.solve(6, max_iters=30, tol=1e-7, seed=2)
        assert hist[-1] <= 1e-7, hist
        u = gl.P.eval_points(gl.U, pts, torch.empty(len(X), dtype=torch.float64, device="cuda")).cpu().numpy()
        ref = W.nonlinear_exact(X)
        errs.append(math.sqrt(np.sum((u - ref) ** 2) / np.sum(ref ** 2)))
    assert errs[0] > errs[1] > errs[2], errs
    rate = math.log(errs[0] / errs[2]) / math.log(95 / 23)
    assert rate >= 2.5, (errs, rate)


def test_moving_source_track_matches_oracle(T):
    """The Sec. 3.3 moving-source plate at a small size (21 x 21 x 6 space, 21 time
    nodes, Inconel 718 laws, M = 4): eight global stages of four subspace iterations
    from the same factors give the oracle's temperature field to 1e-8 of its maximum
    (three space dims with 10 distinct operators each, the time dim with 10)."""
    from paper_2503_13933_gb300 import nonlinear as NL
    desc = W.nonlinear_track(n_xy=21, n_z=6, n_t=21)
    U0 = W.random_factors(dict(desc, terms=[]), 4, seed=3)
    gl = NL.GlobalLocal(desc, W.INCONEL_LAW, 4)
    U, hist = gl.solve(4, max_iters=8, tol=0.0, U0=U0)
    Uo, ho = O.nonlinear_solve(desc, W.INCONEL_LAW, M=4, sweeps=4, max_iters=8, tol=0.0, U0=U0)
    ug, uo = O.cp_full(U), O.cp_full(Uo)
    assert np.max(np.abs(ug - uo)) <= 1e-8 * np.max(np.abs(uo))
    assert np.allclose(hist[1:], ho[1:], rtol=1e-6)


def test_factor_copy_and_relative_change_match_oracle(T):
    """taps_factors_copy (device copy) and taps_factors_rel_change (Gram products on the
    device) against the oracle's |u_A - u_B| / |u_A| of random factor sets with
    different mode counts, and 0 for identical sets."""
    desc = _global(19, 3, seed=8)
    P = T.Problem(desc)
    A0 = W.random_factors(desc, 5, seed=9)
    B0 = [a[:, :3] + 0.1 * b for a, b in zip(A0, W.random_factors(desc, 3, seed=10))]
    A, B, C = P.factors(5), P.factors(5), P.factors(5)
    A.set(A0)
    B.set(B0)
    got = A.rel_change(B)
    ref = O.cp_change(A0, B0)
    assert abs(got - ref) <= 1e-9 * ref
    C.copy_from(A)
    assert C.M == 5 and all(np.array_equal(x, y) for x, y in zip(C.get(), A0))
    assert C.rel_change(A) == 0.0
    # small changes keep their digits: against the explicit difference of the full
    # nodal tensors (which itself carries ~eps / change relative rounding)
    rng = np.random.default_rng(12)
    a_full = O.cp_full(A0)
    for rel in (1e-4, 1e-7, 1e-10):
        B1 = [a + rel * rng.uniform(-1, 1, a.shape) for a in A0]
        B.set(B1)
        got = A.rel_change(B)
        ref = np.linalg.norm(a_full - O.cp_full(B1)) / np.linalg.norm(a_full)
        assert abs(got - ref) <= 1e-5 * ref, (rel, got, ref)


def test_global_local_stops_at_default_tolerance(T):
    """With the default tolerance (1e-8) the global-local iteration of the manufactured
    problem stops on its own, well before max_iters: the stage-to-stage change falls
    by ~5x per stage and is resolved down to rounding (the oracle's history on 16 nodes
    per dim reaches 1.5e-8 at stage 9 and 3e-11 at stage 13)."""
    from paper_2503_13933_gb300 import nonlinear as NL
    desc = W.nonlinear_manufactured(16)
    U0 = W.random_factors(dict(desc, terms=[]), 3, seed=11)
    gl = NL.GlobalLocal(desc, W.NONLINEAR_LAW, 3)
    U, hist = gl.solve(6, max_iters=40, U0=U0)
    assert hist[-1] <= 1e-8 and len(hist) < 20, hist
    _, ho = O.nonlinear_solve(desc, W.NONLINEAR_LAW, M=3, sweeps=6, max_iters=40, tol=1e-8, U0=U0)
    assert abs(len(hist) - len(ho)) <= 1, (hist, ho)
