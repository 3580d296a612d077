"""GPU parity: every step of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances: FP64 path <= 1e-10 relative (assembly <= 1e-12); fields are compared,
not raw factors, except for runs from the same seeded factors over a few sweeps,
where the normalised factors themselves must agree."""
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


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


DIMS = [
    W.dim(16, 0.0, 1.0),
    W.dim(23, -0.5, 2.0, s=1, p=1),
    W.dim(19, 1.0, 10.0, kind=W.PARAM, dirichlet_lo=False, dirichlet_hi=False,
          weight_poly=(0.5, 1.0, 0.25, 0.1)),
    W.dim(13, 0.0, 2.0, kind=W.TIME, dirichlet_hi=False),
    W.dim(21, 0.0, 1.0, s=3, p=3, n_quad=8),
    W.dim(40, 0.0, 3.0, s=4, p=2, dirichlet_lo=False),
]


@pytest.mark.parametrize("dm", DIMS, ids=lambda d: f"n{d['n']}s{d['s']}p{d['p']}")
def test_assembly_parity(T, dm):
    """A1/A2: shape tables and every banded 1D matrix vs the oracle (<= 1e-12)."""
    g = T.Dim(dm)
    od = O.dim_from_description(dm)
    mats = O.assemble_free(od)
    for name, op in O.OP_BY_NAME.items():
        assert rel(g.band(name), to_band(mats[op], g.hb)) < 5e-12, name
    N, B, X = g.shape_tables()
    tab = O.shape_tables(od)
    s = dm["s"]
    for e in (0, 1, dm["n"] // 2, dm["n"] - 2):
        for q, (xe, wj, ids, Nv, Bv) in enumerate(tab[e]):
            assert abs(X[e, q] - xe) < 1e-14
            for c, k in enumerate(ids):
                assert abs(N[e, q, k - (e - s)] - Nv[c]) < 5e-12
                assert abs(B[e, q, k - (e - s)] - Bv[c]) < 1e-10 * max(1, np.max(np.abs(Bv)))


def test_assembly_rejects_bad_patches(T):
    bad = W.dim(8, 0.0, 1.0, s=1, p=2)     # end patch of 2 nodes < p+1
    with pytest.raises(T.TapsError) as e:
        T.Dim(bad)
    assert e.value.status == T.ERR_INVALID_ARG
    with pytest.raises(T.TapsError):
        T.Dim(W.dim(8, 0.0, 1.0, s=5, p=1))   # s beyond the supported maximum


def _pair(desc):
    return O.problem_from_description(desc), None


def _poisson_nodal(n, nsrc, seed):
    """3D Poisson with random separable nodal sources (a solution of CP rank > 1, so
    that a few modes are well posed; the sine source gives a nearly rank-1 solution)."""
    desc = W.poisson_sin(n)
    rng = np.random.default_rng(seed)
    desc["sources"] = [(1.0, [("nodal", rng.uniform(-1, 1, n)) for _ in range(3)])
                       for _ in range(nsrc)]
    return desc


CASES = {
    "poisson3d_n12": _poisson_nodal(12, 4, seed=31),
    "poisson_k_7x9": W.poisson_k(n_space=11, n_k=9, seed=2002),
    "heat2d_robin": W.heat_transient(n_space=10, n_t=9, D_space=2, h_conv=3.0),
    "heat3d_ragged": W.heat_transient(n_space=19, n_t=7, D_space=3, seed=3001),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_sources_parity(T, name):
    desc = CASES[name]
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    for r, (beta, qs) in enumerate(Po.sources):
        for d in range(Po.D):
            assert rel(P.source(r, d), qs[d]) < 1e-12


@pytest.mark.parametrize("name,M,nsw", [("poisson3d_n12", 3, 3), ("poisson_k_7x9", 4, 2),
                                        ("heat2d_robin", 5, 3), ("heat3d_ragged", 2, 2),
                                        ("poisson3d_n12", 1, 2)])
def test_sweep_parity_same_seed(T, name, M, nsw):
    """A3-A8: from the same seeded factors, k sweeps give the same normalised factors
    (<= 1e-10) and the same factor change."""
    desc = CASES[name]
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, M, seed=17 + M)
    Ug = P.factors(max(M, 4))
    Ug.set(U0)
    rep = P.sweep(Ug, nsw)
    Uo = [u.copy() for u in U0]
    for _ in range(nsw):
        Uo, ch = O.sweep(Po, Uo)
    Ugot = Ug.get()
    for d in range(Po.D):
        assert rel(Ugot[d], Uo[d]) < 1e-10, (d, rel(Ugot[d], Uo[d]))
    assert abs(rep["change"] - ch) <= 1e-9 * max(1.0, ch)


@pytest.mark.parametrize("name,M,nsw", [("poisson3d_n12", 3, 3), ("poisson_k_7x9", 4, 2),
                                        ("heat2d_robin", 5, 3), ("heat3d_ragged", 2, 2)])
def test_fastdiag_sweep_parity(T, name, M, nsw):
    """Fast-diagonalisation solver (Sec. 2.6) where the pencil allows, block LU
    elsewhere: same normalised factors as the oracle's sweeps from the same seed."""
    desc = CASES[name]
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, M, seed=57 + M)
    Ug = P.factors(M)
    Ug.set(U0)
    P.sweep(Ug, nsw, solver=T.SOLVER_FASTDIAG)
    Uo = [u.copy() for u in U0]
    for _ in range(nsw):
        Uo, ch = O.sweep(Po, Uo, solver="fastdiag")
    Ugot = Ug.get()
    for d in range(Po.D):
        assert rel(Ugot[d], Uo[d]) < 1e-9, (d, rel(Ugot[d], Uo[d]))
    prof = P.profile()
    assert prof["fastdiag"]["launches"] > 0


def _rich_transient(n_space, n_t, M, h_conv, seed):
    """A 2D transient problem whose source has M random separable terms (nodal values
    U(-1,1)): the right-hand side has rank M, so the ALS systems stay well conditioned
    at M modes (a few Gaussians would make the modes nearly collinear)."""
    desc = W.heat_transient(n_space=n_space, n_t=n_t, D_space=2, h_conv=h_conv, seed=seed)
    rng = np.random.default_rng(seed)
    desc["sources"] = [(1.0, [("nodal", rng.uniform(-1.0, 1.0, dm["n"])) for dm in desc["dims"]])
                       for _ in range(M)]
    return desc


def _md_launches(M, pencil):
    """Launches of one mode-side solve: up to 32 modes the eigen-solve (with W^T c), band
    rows, elimination, output; beyond, the eigen-solve split into transforms on many CTAs
    (two per operator and pass), an FP32 and an FP64 rotation kernel, two basis products
    and the FP64 refinement between the passes, then W^T c, band rows, elimination,
    output."""
    if M <= 32:
        return 4
    return (2 + 2 * (4 if pencil else 2) + 2 + 1) + 4


@pytest.mark.parametrize("n_space,n_t,M,h_conv", [(12, 9, 3, 0.0), (40, 130, 20, 2.0), (24, 300, 32, 0.0),
                                                   (40, 200, 7, 0.0), (36, 90, 33, 0.0), (70, 140, 64, 0.0),
                                                   (104, 110, 100, 0.0)])
def test_mode_side_time_solve_matches_oracle(T, n_space, n_t, M, h_conv):
    """Time dims (G, M: symmetric coefficients) solved on the mode side (Sec. 2.6: M x M
    generalised eigenproblem, M banded eliminations): two sweeps give the oracle's
    factors, with no block elimination anywhere (space dims by the node-side pencil,
    or by block elimination when convection faces give them a third operator).  Beyond
    32 modes (odd 33, 64, 100) the eigen-solve keeps only the rotated matrix in shared
    memory and the eliminations run one warp per 32 systems."""
    desc = _rich_transient(n_space, n_t, M, h_conv, seed=3030 + M)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, M, seed=70 + M)
    Ug = P.factors(M)
    Ug.set(U0)
    P.profile_reset()
    P.sweep(Ug, 2, solver=T.SOLVER_FASTDIAG)
    Uo = [u.copy() for u in U0]
    for _ in range(2):
        Uo, _ = O.sweep(Po, Uo, solver="fastdiag")
    got = Ug.get()
    for d in range(Po.D):
        assert rel(got[d], Uo[d]) < 1e-10, (d, rel(got[d], Uo[d]))
    prof = P.profile()
    assert prof["modediag"]["launches"] == 2 * _md_launches(M, True)
    if h_conv == 0.0:
        assert prof["block_lu"]["launches"] == 0


def _rich_poisson_k(n_space, n_k, M, seed):
    """The space-parameter problem with an M-term random separable source (nodal values
    U(-1,1)), well conditioned at M modes."""
    desc = W.poisson_k(n_space=n_space, n_k=n_k, seed=seed)
    rng = np.random.default_rng(seed)
    desc["sources"] = [(1.0, [("nodal", rng.uniform(-1.0, 1.0, dm["n"])) for dm in desc["dims"]])
                       for _ in range(M)]
    return desc


@pytest.mark.parametrize("n_space,n_k,M", [(10, 7, 3), (60, 16, 12), (200, 32, 30), (60, 50, 45)])
def test_modediag_poisson_matches_oracle(T, n_space, n_k, M):
    """TAPS_SOLVER_MODEDIAG on the space-parameter problem: every dim (K, M pairs and
    the W-only parameter dim) on the mode side, no pencil decomposition; two sweeps
    give the oracle's mode-side factors."""
    desc = _rich_poisson_k(n_space, n_k, M, seed=2040 + M)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, M, seed=80 + M)
    Ug = P.factors(M)
    Ug.set(U0)
    P.profile_reset()
    P.sweep(Ug, 2, solver=T.SOLVER_MODEDIAG)
    Uo = [u.copy() for u in U0]
    for _ in range(2):
        Uo, _ = O.sweep(Po, Uo, solver="modediag")
    got = Ug.get()
    for d in range(Po.D):
        assert rel(got[d], Uo[d]) < 1e-10, (d, rel(got[d], Uo[d]))
    prof = P.profile()
    # three space dims with a (K, M) pencil, the parameter dim with W alone
    assert prof["modediag"]["launches"] == 2 * (3 * _md_launches(M, True) + _md_launches(M, False))
    assert prof["fastdiag"]["launches"] == 0 and prof["block_lu"]["launches"] == 0


@pytest.mark.parametrize("s,p,M", [(1, 1, 3), (0, 0, 3), (2, 1, 4)])
def test_modediag_narrow_bands_match_oracle(T, s, p, M):
    """The mode-side eliminations for band half-widths 3 (s = 1) and 1 (s = 0, linear
    hats): 3D Poisson with rich separable sources, two sweeps against the oracle."""
    desc = W.poisson_sin(14, D=3, s=s, p=p)
    rng = np.random.default_rng(40 + s)
    desc["sources"] = [(1.0, [("nodal", rng.uniform(-1.0, 1.0, dm["n"])) for dm in desc["dims"]])
                       for _ in range(M)]
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, M, seed=90 + s)
    Ug = P.factors(M)
    Ug.set(U0)
    P.sweep(Ug, 2, solver=T.SOLVER_MODEDIAG)
    Uo = [u.copy() for u in U0]
    for _ in range(2):
        Uo, _ = O.sweep(Po, Uo, solver="modediag")
    got = Ug.get()
    for d in range(3):
        assert rel(got[d], Uo[d]) < 1e-10, (d, rel(got[d], Uo[d]))


@pytest.mark.parametrize("solver", ["fastdiag", "block_lu"])
def test_graph_replay_matches_direct_launches(T, solver):
    """Sweeps replayed from a captured CUDA graph give the same history and factors as
    direct launches (same kernels, same order)."""
    desc = W.heat_transient(n_space=14, n_t=10, D_space=2, h_conv=1.5, seed=3020)
    P = T.Problem(desc)
    sv = T.SOLVER_FASTDIAG if solver == "fastdiag" else T.SOLVER_BLOCK_LU
    out = []
    for graphs in (False, True):
        U = P.factors(5)
        r = P.solve(U, M0=5, M_max=5, res_tol=-1.0, als_tol=0.0, max_sweeps=4,
                    init=T.INIT_RANDOM, seed=11, solver=sv, graphs=graphs)
        out.append((r, U.get()))
    (ra, Ua), (rb, Ub) = out
    assert ra["sweeps"] == rb["sweeps"] == 4
    for (_, ca, pa), (_, cb, pb) in zip(ra["history"], rb["history"]):
        assert ca == cb and pa == pb
    for a, b in zip(Ua, Ub):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision,res_tol", [("fp64", 1e-7), ("fp64", -1.0), ("mixed", 1e-7)])
def test_device_solve_loop_matches_host_loop(T, precision, res_tol):
    """The solve loop run on the device (graphs = 2: a conditional WHILE graph node
    repeating sweep, residual and decision) stops at the same sweep, with the same
    history and the same factors bit for bit, as the host loop over per-sweep graphs
    (graphs = 1); with mode growth M = 2 -> 4, stopping on the residual target or on
    the sweep cap."""
    desc = W.poisson_k(n_space=18, n_k=9, seed=2007)
    prec = T.FP64 if precision == "fp64" else T.MIXED
    out = []
    for graphs in (2, 1):
        P = T.Problem(desc)
        U = P.factors(4)
        r = P.solve(U, M0=2, M_max=4, res_tol=res_tol, als_tol=0.0, max_sweeps=12, precision=prec,
                    init=T.INIT_RANDOM, seed=5, solver=T.SOLVER_FASTDIAG, graphs=graphs)
        out.append((r, U.get()))
    (ra, Ua), (rb, Ub) = out
    assert ra["sweeps"] == rb["sweeps"] and ra["M"] == rb["M"] and ra["converged"] == rb["converged"]
    assert ra["history"] == rb["history"]
    for a, b in zip(Ua, Ub):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("solver", ["fastdiag", "modediag"])
def test_device_solve_loop_transient_routes(T, solver):
    """The device-side solve loop on a transient problem with a convection face: the
    time dim on the mode side (its stored basis carried across the loop's sweeps), the
    convection dim by the face-corrected route, the other by the node-side pencil; same
    sweeps, history and factors as the host loop."""
    desc = _rich_transient(16, 24, 5, 2.0, seed=3060)
    sv = T.SOLVER_FASTDIAG if solver == "fastdiag" else T.SOLVER_MODEDIAG
    out = []
    for graphs in (2, 1):
        P = T.Problem(desc)
        U = P.factors(5)
        r = P.solve(U, M0=5, M_max=5, res_tol=1e-30, als_tol=0.0, max_sweeps=6, init=T.INIT_RANDOM, seed=7,
                    solver=sv, graphs=graphs)
        out.append((r, U.get()))
    (ra, Ua), (rb, Ub) = out
    assert ra["sweeps"] == rb["sweeps"] == 6
    assert ra["history"] == rb["history"]
    for a, b in zip(Ua, Ub):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name,M,nsw", [("poisson3d_n12", 3, 3), ("poisson_k_7x9", 4, 2),
                                        ("heat2d_robin", 5, 3)])
def test_mixed_refined_small_solves_parity(T, name, M, nsw):
    """TAPS_MIXED: the small systems of the fast-diagonalisation solve are factorised in
    FP32 and refined in FP64 to FP64 backward accuracy: same factors as the oracle."""
    desc = CASES[name]
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, M, seed=77 + M)
    Ug = P.factors(M)
    Ug.set(U0)
    P.sweep(Ug, nsw, solver=T.SOLVER_FASTDIAG, precision=T.MIXED)
    Uo = [u.copy() for u in U0]
    for _ in range(nsw):
        Uo, _ = O.sweep(Po, Uo, solver="fastdiag")
    Ugot = Ug.get()
    for d in range(Po.D):
        assert rel(Ugot[d], Uo[d]) < 1e-9, (d, rel(Ugot[d], Uo[d]))


def test_fastdiag_large_dim_matches_block_lu(T):
    """n = 254 free nodes, M = 12: one fast-diagonalisation sweep and one block-LU
    sweep from the same factors give the same field."""
    desc = W.poisson_k(n_space=256, n_k=32, seed=2011)
    P = T.Problem(desc)
    U0 = W.random_factors(desc, 12, seed=9)
    Ua, Ub = P.factors(12), P.factors(12)
    Ua.set(U0)
    Ub.set(U0)
    P.sweep(Ua, 1, solver=T.SOLVER_FASTDIAG)
    P.sweep(Ub, 1, solver=T.SOLVER_BLOCK_LU)
    ga, gb = Ua.get(), Ub.get()
    for d in range(4):
        assert rel(ga[d], gb[d]) < 1e-9, (d, rel(ga[d], gb[d]))


@pytest.mark.parametrize("name", sorted(CASES))
def test_residual_parity(T, name):
    """A9: the residual of Eq. 42 and the full-system residual vs the oracle."""
    desc = CASES[name]
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, 3, seed=5)
    Ug = P.factors(3)
    Ug.set(U0)
    r_als = P.residual(Ug, T.RES_ALS)
    r_full = P.residual(Ug, T.RES_FULL)
    assert abs(r_als - O.als_residual(Po, U0)) < 1e-10 * max(1.0, r_als)
    ro = O.residual(Po, U0)[0]
    assert abs(r_full - ro) < 1e-7 + 1e-9 * ro
    assert abs(r_full - O.residual_explicit(Po, U0)) < 1e-7 + 1e-9 * ro


def test_solve_poisson_16cubed_vs_brute_force(T):
    """Greedy solve on 16^3 vs the oracle's greedy solve and the full Kronecker FE
    solution: reconstructed fields agree (FP64 <= 1e-10 against the oracle)."""
    desc = W.poisson_sin(16)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    Ug = P.factors(4)
    # res_tol < 0: never stop on the residual (it can reach its cancellation floor 0)
    rep = P.solve(Ug, M0=1, M_max=3, als_tol=1e-12, res_tol=-1.0, res_kind=T.RES_FULL,
                  max_sweeps=100, init=T.INIT_ZERO)
    ro = O.solve(Po, M0=1, M_max=3, als_tol=1e-12, res_tol=-1.0, max_sweeps=100, init="zero")
    ug = O.cp_full(Ug.get())
    uo = O.cp_full(ro.U)
    assert rep["M"] == 3
    assert np.linalg.norm(ug - uo) / np.linalg.norm(uo) < 1e-10
    u_full = O.solve_full(Po)
    assert np.linalg.norm(ug - u_full) / np.linalg.norm(u_full) < 1e-6
    assert abs(rep["rho_full"] - O.residual(Po, ro.U)[0]) < 1e-7


def test_solve_random_init_matches_oracle_counter_rng(T):
    """TAPS_INIT_RANDOM draws the same SplitMix64 values as the oracle."""
    desc = W.poisson_k(n_space=9, n_k=7, seed=2004)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    Ug = P.factors(3)
    P.solve(Ug, M0=3, M_max=3, max_sweeps=1, res_tol=-1.0, als_tol=0.0, init=T.INIT_RANDOM, seed=99)
    Uo = O.init_factors(Po, 3, "random", 99)
    Uo, _ = O.sweep(Po, Uo)
    got = Ug.get()
    for d in range(Po.D):
        assert rel(got[d], Uo[d]) < 1e-10


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_eval_grid_parity(T, dtype):
    """A10: grid reconstruction on strided node slices (constrained nodes = 0)."""
    desc = W.heat_transient(n_space=14, n_t=11, D_space=2, h_conv=1.0)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, 7, seed=3)
    Ug = P.factors(7)
    Ug.set(U0)
    start, count, step = [0, 1, 0], [14, 5, 11], [1, 3, 1]
    idx = [list(range(s, s + c * st, st)) for s, c, st in zip(start, count, step)]
    ref = O.eval_grid(Po, U0, idx)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    out = torch.empty(int(np.prod(count)), dtype=tdt, device="cuda")
    P.eval_grid(Ug, start, count, step, out, dtype=T.FP64 if dtype == "f64" else T.FP32)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy().reshape(count)
    tol = 1e-13 if dtype == "f64" else 2e-6
    assert rel(got, ref) < tol


def test_eval_points_parity(T):
    """Point evaluation with the C-HiDeNN shape functions (Eq. 13)."""
    desc = W.poisson_k(n_space=12, n_k=8, seed=2005)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, 4, seed=8)
    Ug = P.factors(4)
    Ug.set(U0)
    rng = np.random.default_rng(0)
    pts = np.stack([rng.uniform(0, 1, 50), rng.uniform(0, 1, 50), rng.uniform(0, 1, 50),
                    rng.uniform(1, 10, 50)], axis=1)
    pts[0] = [0.0, 1.0, 0.5, 1.0]
    ref = O.eval_points(Po, U0, pts)
    out = torch.empty(50, dtype=torch.float64, device="cuda")
    P.eval_points(Ug, torch.tensor(pts, device="cuda"), out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), ref) < 1e-12


def _full_rank_2d(n, nsrc, seed):
    """D = 2 Poisson with nsrc random separable nodal sources: with M = n_free modes
    the CP space holds every grid function, so one sweep from full-rank factors gives
    the full Galerkin solution."""
    desc = W.poisson_sin(n, D=2)
    rng = np.random.default_rng(seed)
    desc["sources"] = [(1.0, [("nodal", rng.uniform(-1, 1, n)) for _ in range(2)])
                       for _ in range(nsrc)]
    return desc


def test_full_rank_2d_more_than_32_modes(T):
    """M = 34 > 32 (several rows per lane in the block triangular solves): one sweep
    reaches the brute-force Kronecker solution, and matches the oracle's sweep."""
    desc = _full_rank_2d(36, 40, seed=21)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, 34, seed=4)
    Ug = P.factors(34)
    Ug.set(U0)
    P.sweep(Ug, 1)
    u_full = O.solve_full(Po)
    ug = O.cp_full(Ug.get())
    assert np.linalg.norm(ug - u_full) / np.linalg.norm(u_full) < 1e-9
    Uo, _ = O.sweep(Po, U0)
    # 34 modes from random factors: the reduced systems carry kappa ~ 1e5, so two
    # FP64 eliminations (no pivoting vs LAPACK partial pivoting) agree to ~kappa*eps
    assert np.linalg.norm(ug - O.cp_full(Uo)) / np.linalg.norm(u_full) < 1e-8


@pytest.mark.parametrize("nodes,M", [(7, 1), (19, 17), (31, 29), (34, 32)])
def test_fastdiag_full_rank_2d_reaches_kronecker_solution(T, nodes, M):
    """Fast-diagonalisation small solves with the columns of each M x M system spread
    over four warps (ragged when 4 does not divide M, one column at M = 1): with
    M = n_free modes one sweep gives the brute-force Kronecker solution, and the same
    field as the oracle's fast-diagonalisation sweep."""
    desc = _full_rank_2d(nodes, M + 2, seed=30 + M)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, M, seed=11 + M)
    Ug = P.factors(M)
    Ug.set(U0)
    P.sweep(Ug, 1, solver=T.SOLVER_FASTDIAG)
    assert P.profile()["fastdiag"]["launches"] > 0
    u_full = O.solve_full(Po)
    ug = O.cp_full(Ug.get())
    Uo, _ = O.sweep(Po, U0, solver="fastdiag")
    Ub, _ = O.sweep(Po, U0)
    # the reduced systems of M random modes are ill-conditioned; the spread between
    # the oracle's own two FP64 solvers (fast diagonalisation, dense LU) measures
    # kappa * eps for this case and sets the bound
    uo = O.cp_full(Uo)
    spread = np.linalg.norm(uo - O.cp_full(Ub)) / np.linalg.norm(u_full)
    assert np.linalg.norm(ug - uo) / np.linalg.norm(u_full) < max(1e-10, 10 * spread)
    if M == nodes - 2:   # as many modes as free nodes
        reach = np.linalg.norm(uo - u_full) / np.linalg.norm(u_full)
        assert np.linalg.norm(ug - u_full) / np.linalg.norm(u_full) < max(1e-10, 10 * reach)


def test_fp32_grams_then_fp64_polish(T):
    """Mixed precision: FP32 Gram sweeps, then FP64 polishing, reach the full-rank
    solution within the mixed-path bound 1e-6."""
    desc = _full_rank_2d(20, 20, seed=22)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    u_full = O.solve_full(Po)
    U32 = P.factors(18)
    U32.set(W.random_factors(desc, 18, seed=6))
    P.sweep(U32, 2, precision=T.FP32)
    e32 = np.linalg.norm(O.cp_full(U32.get()) - u_full) / np.linalg.norm(u_full)
    # FP32 Grams of 18 random modes carry kappa-amplified single-precision error
    assert 1e-9 < e32 < 0.5
    # an unreachable residual target forces the FP32 -> FP64 hand-over within the
    # sweep budget; FP64 sweeps then restore FP64 accuracy of the field
    r = P.solve(U32, M_max=18, res_tol=1e-30, max_sweeps=8, init=T.INIT_GIVEN,
                precision=T.FP32, polish_sweeps=3)
    assert r["fp64_sweeps"] >= 1, r
    e = np.linalg.norm(O.cp_full(U32.get()) - u_full) / np.linalg.norm(u_full)
    # the mixed-path bound after refinement (18 random modes carry kappa ~ 1e6)
    assert e < 1e-6, (e, r["rho"])


def test_bf16_grams_then_fp64_polish(T):
    """BF16-rounded Gram operands with FP32 accumulation (TAPS_BF16): the BF16 sweeps
    carry BF16-level error, the solve hands over to FP64 and polishing restores the
    mixed-path bound 1e-6 against the full-rank solution."""
    desc = _full_rank_2d(20, 20, seed=23)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    u_full = O.solve_full(Po)
    U = P.factors(18)
    U.set(W.random_factors(desc, 18, seed=7))
    P.sweep(U, 2, precision=T.BF16)
    e16 = np.linalg.norm(O.cp_full(U.get()) - u_full) / np.linalg.norm(u_full)
    assert 1e-6 < e16 < 1.0
    r = P.solve(U, M_max=18, res_tol=1e-30, max_sweeps=8, init=T.INIT_GIVEN, precision=T.BF16,
                polish_sweeps=3)
    assert r["fp64_sweeps"] >= 1, r
    e = np.linalg.norm(O.cp_full(U.get()) - u_full) / np.linalg.norm(u_full)
    assert e < 1e-6, (e, r["rho"])


def test_fp32_solve_poisson_matches_fp64(T):
    """3D Poisson, greedy to a full-residual target: the mixed-precision solve and the
    FP64 solve reconstruct the same field within the mixed-path bound 1e-6."""
    desc = W.poisson_sin(20)
    P = T.Problem(desc)
    U64, U32 = P.factors(3), P.factors(3)
    r64 = P.solve(U64, M0=1, M_max=3, res_tol=1e-7, res_kind=T.RES_FULL, max_sweeps=50)
    r32 = P.solve(U32, M0=1, M_max=3, res_tol=1e-7, res_kind=T.RES_FULL, max_sweeps=50,
                  precision=T.FP32, polish_sweeps=10)
    assert r64["converged"] and r32["converged"]
    a, b = O.cp_full(U64.get()), O.cp_full(U32.get())
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-6


def test_degenerate_inputs(T):
    """Edge cases: one free node per dim... and bad arguments come back as statuses."""
    desc = W.poisson_sin(3, D=2, s=1, p=1)     # one free node per dim
    P = T.Problem(desc)
    Ug = P.factors(2)
    rep = P.solve(Ug, M0=1, M_max=1, res_tol=1e-12, max_sweeps=5, init=T.INIT_ZERO)
    Po = O.problem_from_description(desc)
    u_full = O.solve_full(Po)
    assert abs(O.cp_full(Ug.get())[0] - u_full[0]) < 1e-12 * abs(u_full[0])
    with pytest.raises(T.TapsError):
        P.factors(0)
    with pytest.raises(T.TapsError):
        P.solve(Ug, M0=1, M_max=3)       # M_max > M_cap


def test_small_solve_reciprocal_within_one_ulp(T):
    """The FP64 reciprocal of the fast-diagonalisation small solves (approximate seed
    refined by the series 1/x = y0 (1 + e + e^2)) against IEEE division on the GPU:
    within one ulp of 1.0 / x over log-uniform magnitudes 1e-250 .. 1e250, both signs,
    and exact at powers of two."""
    rng = np.random.default_rng(17)
    x = 10.0 ** rng.uniform(-250, 250, 1 << 20) * rng.choice([-1.0, 1.0], 1 << 20)
    x = np.concatenate([x, 2.0 ** np.arange(-1000, 1001, 7), [1.0, -1.0, 3.0, 0.1]])
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    T.rcp(xd, yd)
    ref = (1.0 / xd)
    torch.cuda.synchronize()
    y, r = yd.cpu().numpy(), ref.cpu().numpy()
    ulp = np.spacing(np.abs(r))
    assert np.all(np.abs(y - r) <= ulp)
    pow2 = np.isin(x, 2.0 ** np.arange(-1000, 1001, 7))
    assert np.array_equal(y[pow2], r[pow2])


def test_greedy_full_residual_schedule_matches_oracle(T):
    """The greedy schedule on the full residual with two modes per growth step and the
    stagnation rule armed (space-parameter problem, 12^3 x 8): the GPU's mode counts,
    the residual at the end of each of them, and the final field equal the oracle's."""
    desc = W.poisson_k(n_space=12, n_k=8, seed=2060)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U = P.factors(20)
    rep = P.solve(U, M0=1, M_max=11, als_tol=1e-6, res_tol=1e-12, res_kind=T.RES_FULL, max_sweeps=30,
                  init=T.INIT_RANDOM, seed=3, solver=T.SOLVER_FASTDIAG, res_stall=0.01, M_step=2)
    ro = O.solve(Po, M0=1, M_max=11, als_tol=1e-6, res_tol=1e-12, max_sweeps=30, init="random", seed=3,
                 solver="fastdiag", res_stall=0.01, M_step=2)
    ends_g, ends_o = {}, {}
    for M, ch, rho in rep["history"]:
        ends_g[M] = rho
    for M, it, ch, rho in ro.history:
        ends_o[M] = rho
    assert list(ends_g) == list(ends_o) == [1, 3, 5, 7, 9, 11]
    for M in ends_o:
        assert abs(ends_g[M] - ends_o[M]) <= 1e-6 * ends_o[M], (M, ends_g[M], ends_o[M])
    assert O.cp_change(ro.U, U.get()) <= 1e-8
