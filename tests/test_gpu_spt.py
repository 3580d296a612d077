"""The eight-dimensional space-parameter-time problem of Sec. 3.2 on the GPU
(x, y, z, k, P, rho, c_p, t; lifted non-homogeneous Dirichlet data): sources and
sweeps element by element against the oracle, and the GPU solution's relative L2 error
against the closed-form exact solution: equal to the oracle's, falling at the rate of
the reproducing order under refinement, down to 450 nodes per dim (450^8 = 1.7e21
grid points in the equivalent full model)."""
import math

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
    """Per-entry rounding scale of a source factor: for (Op v)[free] and the nodal
    kind's (M v)[free], |Op| |v| (the assembled entries agree to ~1e-13 relative and
    the sum cancels); else None (max |q| applies)."""
    kind, par = fac
    if kind == "opvecfull":
        A = np.abs(O.assemble_full(dm)[O.OP_BY_NAME[par[0]]])
        return (A @ np.abs(np.asarray(par[1])))[dm.free]
    if kind == "nodal":
        return (np.abs(O.assemble_full(dm)[O.OP_M]) @ np.abs(np.asarray(par)))[dm.free]
    return None


def _case(n, s=2, p=2):
    desc, lift, ex = W.spt_manufactured(n, s=s, p=p)
    return B.lifted(desc, *lift), lift, ex


def _gpu_solve(T, n, s=2, p=2, M=6, sweeps=10):
    """Algorithm 1 with greedy enrichment: modes 1..M, each step up to `sweeps`
    subspace iterations (ALS change 1e-3)."""
    lifted, lift, ex = _case(n, s, p)
    P = T.Problem(lifted)
    U = P.factors(M)
    rep = P.solve(U, M0=1, M_max=M, als_tol=1e-3, res_tol=-1.0, max_sweeps=sweeps,
                  init=T.INIT_RANDOM, seed=3, solver=T.SOLVER_FASTDIAG)
    assert rep["M"] == M
    return lifted, lift, ex, P, U


def _gpu_error(T, n, s=2, p=2, M=6, sweeps=10):
    """The relative L2 error of u_D + w against u_ex by the oracle's per-dim Gauss rules
    (exact integration; a floor near 1e-7 from the expansion's cancellation)."""
    lifted, lift, ex, P, U = _gpu_solve(T, n, s, p, M, sweeps)
    dims = [O.dim_from_description(dm) for dm in lifted["dims"]]
    V, c = O.lifted_field_factors(dims, U.get(), lift)
    return O.relative_l2_error(dims, V, c, ex["sep"], ex["pair"], W.spt_exact_pair)


def _sampled_error(T, n, s=2, p=2, M=6, sweeps=10, n_pts=1 << 16, seed=9):
    """The relative L2 error estimated from n_pts uniform random points of the 8-dim
    box (no cancellation floor; sampling noise of a few percent): u = w + u_D evaluated
    on the GPU (w through the solved factors, u_D through the lifting's all-node factors
    on a copy of the dims with no constrained node), u_ex in closed form."""
    lifted, (vecs, wts), ex, P, U = _gpu_solve(T, n, s, p, M, sweeps)
    rng = np.random.default_rng(seed)
    lo = np.array([dm["lo"] for dm in lifted["dims"]])
    hi = np.array([dm["hi"] for dm in lifted["dims"]])
    X = lo + (hi - lo) * rng.uniform(size=(n_pts, 8))
    pts = torch.as_tensor(X, device="cuda")
    field = B.LiftedField(lifted, vecs, wts)
    u = field.eval_points(P, U, pts, torch.empty(n_pts, dtype=torch.float64, device="cuda")).cpu().numpy()
    uex = W.spt_exact(X)
    return math.sqrt(np.sum((u - uex) ** 2) / np.sum(uex ** 2))


def test_spt_sources_parity(T):
    """Every source factor of the lifted problem (Gaussian, nodal, polynomial, constant
    and all-node operator-vector kinds on all 8 dims) against the oracle: <= 1e-12 of
    the largest entry, per entry within 1e-11 |Op| |v| for the nodal and
    operator-vector kinds."""
    lifted, _, _ = _case(10)
    P = T.Problem(lifted)
    Po = O.problem_from_description(lifted)
    for r in range(len(Po.sources)):
        for d in range(Po.D):
            ref = Po.sources[r][1][d]
            got = P.source(r, d)
            sc = _scale(Po.dims[d], lifted["sources"][r][1][d])
            if sc is None:
                assert np.max(np.abs(got - ref)) <= 1e-12 * max(np.max(np.abs(ref)), 1e-300), (r, d)
            else:
                assert np.all(np.abs(got - ref) <= 1e-11 * sc), (r, d)


def _oracle_sweeps(Po, U0, solver, n):
    U = [u.copy() for u in U0]
    for _ in range(n):
        U, _ = O.sweep(Po, U, solver=solver)
    return U


@pytest.mark.parametrize("solver", ["block_lu", "fastdiag"])
def test_spt_sweeps_match_oracle(T, solver):
    """Three sweeps from the same seeded factors (M = 6, 10 nodes per dim): the same
    normalised factors as the oracle's block elimination / fast diagonalisation (node
    side, mode side for the time dim).  The 1D operators agree to 1e-12 relative (the
    assembly's parity bound) and the right-hand side near the boundary is a sum of 224
    lifting terms of alternating sign, so the bound is measured on the oracle itself:
    per dim, 10x the change of its own result under a random 1e-12 relative
    perturbation of every operator and source entry."""
    lifted, _, _ = _case(10)
    P = T.Problem(lifted)
    Po = O.problem_from_description(lifted)
    U0 = W.random_factors(lifted, 6, seed=61)
    U = P.factors(6)
    U.set(U0)
    sv = T.SOLVER_FASTDIAG if solver == "fastdiag" else T.SOLVER_BLOCK_LU
    P.sweep(U, 3, solver=sv)
    osv = "fastdiag" if solver == "fastdiag" else "banded"
    Uo = _oracle_sweeps(Po, U0, osv, 3)
    rng = np.random.default_rng(0)
    Pp = O.problem_from_description(lifted)
    for d in range(Pp.D):
        for k in Pp.ops[d]:
            Pp.ops[d][k] = Pp.ops[d][k] * (1 + 1e-12 * rng.uniform(-1, 1, Pp.ops[d][k].shape))
    for _, qs in Pp.sources:
        for d in range(Pp.D):
            qs[d] = qs[d] * (1 + 1e-12 * rng.uniform(-1, 1, qs[d].shape))
    Up = _oracle_sweeps(Pp, U0, osv, 3)
    for d, (g, o, q) in enumerate(zip(U.get(), Uo, Up)):
        sens = np.max(np.abs(q - o))
        assert np.max(np.abs(g - o)) <= 10 * sens + 1e-12 * np.max(np.abs(o)), (d, sens)


def test_spt_error_equals_oracle_error(T):
    """14 nodes per dim, modes 1..6: the GPU solution's L2 error against u_ex equals the
    oracle solution's (discretisation error dominates) to 1%, and the sampled
    estimator used at finer grids agrees with the exact integration to 10%."""
    err_g = _gpu_error(T, 14)
    # the sampled estimator agrees with the exact integration
    assert abs(_sampled_error(T, 14) - err_g) <= 0.1 * err_g
    lifted, lift, ex = _case(14)
    Po = O.problem_from_description(lifted)
    r = O.solve(Po, M0=1, M_max=6, als_tol=1e-3, res_tol=-1.0, max_sweeps=10, init="random", seed=3)
    V, c = O.lifted_field_factors(Po.dims, r.U, lift)
    err_o = O.relative_l2_error(Po.dims, V, c, ex["sep"], ex["pair"], W.spt_exact_pair)
    assert abs(err_g - err_o) <= 1e-2 * err_o, (err_g, err_o)


@pytest.mark.parametrize("s,p,order", [(1, 1, 1.6), (2, 2, 2.5), (3, 3, 2.5)])
def test_spt_convergence_rate(T, s, p, order):
    """Refinement 16 -> 32 -> 64 nodes per dim: the error falls at each step, at an
    observed order of at least `order` in h over the whole range (p + 1 in theory; the
    paper's own p = 3 rate is below 4 on meshes this coarse)."""
    errs = [_sampled_error(T, n, s, p) for n in (16, 32, 64)]
    assert errs[0] > errs[1] > errs[2], errs
    rate = math.log(errs[0] / errs[2]) / math.log(63 / 15)
    assert rate >= order, (errs, rate)


def test_spt_zetta_scale_450_nodes_per_dim(T):
    """450 nodes per dim in all 8 dims (1.7e21 grid points in the full model), s = p = 2,
    modes 1..8: the sampled error is below 1e-6 and below 1/20 of that at 64 nodes per
    dim (p + 1 = 3 predicts 1/360)."""
    err = _sampled_error(T, 450, M=8)
    err64 = _sampled_error(T, 64, M=8)
    assert err < min(err64 / 20, 1e-6), (err, err64)
