"""Non-homogeneous Dirichlet data by lifting on the GPU (Sec. 2.5 weak form with
u = u_D + w): the all-node operator-vector sources element by element against the
oracle, and lifted solves against the oracle and against the full-grid solve with the
boundary values imposed directly."""
import numpy as np
import pytest

from oracle import taps_oracle as O
from paper_2503_13933_gb300 import boundary as B
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


def _scale(dm, fac):
    """Per-entry rounding scale of a source factor: for (Op v)[free], |Op| |v| (the
    assembled entries agree to ~1e-13 relative and the sum cancels); else max |q|."""
    kind, par = fac
    if kind == "opvecfull":
        A = np.abs(O.assemble_full(dm)[O.OP_BY_NAME[par[0]]])
        return (A @ np.abs(np.asarray(par[1])))[dm.free]
    return None


def _lifted_heat(seed):
    """Transient 3D heat (Robin faces, moving source) with rank-3 boundary data on
    every Dirichlet face: sources of every operator of the description."""
    desc = W.heat_transient(n_space=19, n_t=11, D_space=3, h_conv=2.0, seed=seed)
    rng = np.random.default_rng(seed)
    vecs = [rng.uniform(-1, 1, (dm["n"], 3)) for dm in desc["dims"]]
    return desc, vecs, np.array([1.0, -0.6, 0.3])


def test_lifting_sources_parity(T):
    """Every lifting source factor (each operator, each dim, ragged free-node sets)
    against the oracle's (Op v)[free], per entry within 1e-11 |Op| |v|."""
    desc, vecs, wts = _lifted_heat(41)
    lifted = B.lifted(desc, vecs, wts)
    P = T.Problem(lifted)
    Po = O.problem_from_description(lifted)
    n0 = len(desc["sources"])
    assert len(Po.sources) == n0 + len(desc["terms"]) * 3
    for r in range(n0, len(Po.sources)):
        for d in range(Po.D):
            ref = Po.sources[r][1][d]
            got = P.source(r, d)
            sc = _scale(Po.dims[d], lifted["sources"][r][1][d])
            assert np.all(np.abs(got - ref) <= 1e-11 * sc), (r, d)


@pytest.mark.parametrize("solver", ["block_lu", "fastdiag"])
def test_lifted_2d_solve_equals_direct_boundary_solve(T, solver):
    """2D Poisson on 6 x 6 nodes, random separable boundary data (rank 2 at all nodes)
    and sources: with M = 4 modes the GPU's u_D + w equals the full-grid solve with the
    boundary values imposed directly, and the oracle's lifted solve, to 1e-9; the
    device evaluation of u = w + u_D at points matches the interpolants to 1e-12."""
    rng = np.random.default_rng(12)
    desc = W.poisson_sin(6, D=2)
    desc["sources"] = [(1.0, [("nodal", rng.uniform(-1, 1, 6)), ("nodal", rng.uniform(-1, 1, 6))])
                       for _ in range(2)]
    vecs = [rng.uniform(-1, 1, (6, 2)), rng.uniform(-1, 1, (6, 2))]
    wts = np.array([0.7, -1.3])
    lifted = B.lifted(desc, vecs, wts)
    P = T.Problem(lifted)
    U = P.factors(4)
    sv = T.SOLVER_FASTDIAG if solver == "fastdiag" else T.SOLVER_BLOCK_LU
    P.solve(U, M0=4, M_max=4, als_tol=1e-14, res_tol=-1.0, max_sweeps=60, init=T.INIT_RANDOM,
            seed=3, solver=sv)
    w = O.cp_full(U.get()).reshape(4, 4)
    uD = np.einsum("im,jm,m->ij", vecs[0], vecs[1], wts)
    u = w + uD[1:-1, 1:-1]
    # the oracle's lifted solve
    Po = O.problem_from_description(lifted)
    ro = O.solve(Po, M0=4, M_max=4, als_tol=1e-14, res_tol=-1.0, max_sweeps=60, init="random", seed=3)
    wo = O.cp_full(ro.U).reshape(4, 4)
    assert np.max(np.abs(w - wo)) < 1e-9 * np.max(np.abs(wo))
    # the direct full-grid solve with the boundary rows imposed
    dm = O.dim_from_description(desc["dims"][0])
    mats = O.assemble_full(dm)
    K, Mm = mats[O.OP_K], mats[O.OP_M]
    A = np.kron(K, Mm) + np.kron(Mm, K)
    F = np.zeros(36)
    for beta, fl in desc["sources"]:
        F += beta * np.kron(Mm @ fl[0][1], Mm @ fl[1][1])
    inner = np.array([(i % 6 not in (0, 5)) and (i // 6 not in (0, 5)) for i in range(36)])
    ub = uD.reshape(-1)
    uI = np.linalg.solve(A[np.ix_(inner, inner)], F[inner] - A[np.ix_(inner, ~inner)] @ ub[~inner])
    assert np.max(np.abs(u.reshape(-1) - uI)) < 1e-9 * np.max(np.abs(uI))
    # u = w + u_D at arbitrary points on the device against the interpolants summed
    # point by point from the same factors (the lifting's at all nodes)
    rng2 = np.random.default_rng(5)
    X = rng2.uniform(0.0, 1.0, (64, 2))
    X[:4] = [[0.0, 0.3], [1.0, 0.7], [0.2, 0.0], [0.6, 1.0]]   # on the boundary: u = u_D
    got = B.LiftedField(lifted, vecs, wts).eval_points(
        P, U, torch.as_tensor(X, device="cuda"), torch.empty(64, dtype=torch.float64, device="cuda")).cpu().numpy()
    dims = [O.dim_from_description(dm) for dm in lifted["dims"]]
    V, c = O.lifted_field_factors(dims, U.get(), (vecs, wts))
    ref = np.zeros(64)
    for i, xp in enumerate(X):
        prod = np.array(c)
        for d, dm in enumerate(dims):
            e = O.locate(dm.x, xp[d])
            ids, N, _ = O.shape_functions(dm.x, dm.s, dm.a, dm.p, e, xp[d])
            prod = prod * (np.asarray(N) @ V[d][np.array(ids)])
        ref[i] = prod.sum()
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_lifted_transient_sweeps_match_oracle(T):
    """The lifted transient problem, 3 sweeps from the same seeded factors on both
    sides (FP64 block elimination): the same normalised factors to 1e-10."""
    desc, vecs, wts = _lifted_heat(43)
    lifted = B.lifted(desc, vecs, wts)
    P = T.Problem(lifted)
    Po = O.problem_from_description(lifted)
    U0 = W.random_factors(lifted, 3, seed=44)
    U = P.factors(3)
    U.set(U0)
    P.sweep(U, 3, solver=T.SOLVER_BLOCK_LU)
    Uo = [u.copy() for u in U0]
    for _ in range(3):
        Uo, _ = O.sweep(Po, Uo, solver="banded")
    for d, (g, o) in enumerate(zip(U.get(), Uo)):
        assert np.max(np.abs(g - o)) < 1e-10 * np.max(np.abs(o)), d
