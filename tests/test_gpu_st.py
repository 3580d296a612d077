"""The space-time moving-source problem of Sec. 3.1 on the GPU (x, y, t; lifted
Dirichlet data; the (x, t)-coupled source as nodal SVD factors): sources against the
oracle, and the GPU solution's relative L2 error against the closed-form solution,
equal to the oracle's and falling with the number of modes and with refinement."""
import math

import numpy as np
import pytest

from oracle import taps_oracle as O
from paper_2503_13933_gb300 import boundary as B
from paper_2503_13933_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHORT = dict(x=(0.0, 10.0), y=(-4.0, 4.0), t=(0.0, 0.02))


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_13933_gb300 import build, taps
    build.build()
    taps.lib()
    return taps


def _case(n, s=1, p=1, ranges=None):
    desc, lift, ex = W.st_manufactured(n, s=s, p=p, ranges=ranges)
    return B.lifted(desc, *lift), lift, ex


def _gpu_error(T, n, s=1, p=1, M=8, sweeps=5, ranges=None, greedy=True):
    """Algorithm 1 and the error of u_D + w by exact integration.  greedy: modes 1..M,
    up to `sweeps` subspace iterations each (ALS change 1e-3); else Algorithm 1 as
    printed: M random modes, `sweeps` subspace iterations."""
    lifted, lift, ex = _case(n, s, p, ranges)
    P = T.Problem(lifted)
    U = P.factors(M)
    rep = P.solve(U, M0=1 if greedy else M, M_max=M, als_tol=1e-3 if greedy else 0.0, res_tol=-1.0,
                  max_sweeps=sweeps, init=T.INIT_RANDOM, seed=3, solver=T.SOLVER_FASTDIAG)
    assert rep["M"] == M
    dims = [O.dim_from_description(dm) for dm in lifted["dims"]]
    V, c = O.lifted_field_factors(dims, U.get(), lift)
    return O.relative_l2_error(dims, V, c, ex["sep"], ex["pair"], W.st_exact_pair)


def test_st_sources_parity(T):
    """Every source factor (nodal SVD factors, Gaussian, lifting operator-vectors)
    against the oracle: <= 1e-12 of the largest entry, or per entry within
    1e-11 |Op| |v| for the kinds that multiply an assembled operator."""
    lifted, _, _ = _case(30)
    P = T.Problem(lifted)
    Po = O.problem_from_description(lifted)
    for r in range(len(Po.sources)):
        for d in range(Po.D):
            ref = Po.sources[r][1][d]
            got = P.source(r, d)
            kind, par = lifted["sources"][r][1][d]
            if kind in ("nodal", "opvecfull"):
                op = O.OP_M if kind == "nodal" else O.OP_BY_NAME[par[0]]
                v = par if kind == "nodal" else par[1]
                sc = (np.abs(O.assemble_full(Po.dims[d])[op]) @ np.abs(np.asarray(v)))[Po.dims[d].free]
                assert np.all(np.abs(got - ref) <= 1e-11 * sc), (r, d)
            else:
                assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), (r, d)


def test_st_error_equals_oracle_error(T):
    """Shortened window, 48 nodes per dim, s = p = 1, modes 1..8: the GPU solution's
    error against u_ex equals the oracle solution's to 1%."""
    err_g = _gpu_error(T, 48, ranges=SHORT)
    lifted, lift, ex = _case(48, ranges=SHORT)
    Po = O.problem_from_description(lifted)
    r = O.solve(Po, M0=1, M_max=8, als_tol=1e-3, res_tol=-1.0, max_sweeps=5, init="random", seed=3)
    V, c = O.lifted_field_factors(Po.dims, r.U, lift)
    err_o = O.relative_l2_error(Po.dims, V, c, ex["sep"], ex["pair"], W.st_exact_pair)
    assert abs(err_g - err_o) <= 1e-2 * err_o, (err_g, err_o)


def test_st_error_falls_with_modes(T):
    """The full window at 100 nodes per dim, s = p = 1 (the paper's mode study
    configuration), Algorithm 1 as printed (M random modes, 3 subspace iterations):
    the error falls from 5 to 15 to 25 modes, where it is below 5e-3 (the paper reports
    2.5e-3 at 25 modes on its own, unstated, domain)."""
    errs = [_gpu_error(T, 100, M=M, sweeps=3, greedy=False) for M in (5, 15, 25)]
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 5e-3, errs


def test_st_three_iterations_suffice(T):
    """The paper's iteration study: at 25 modes, 3 subspace iterations give the error
    of 8 to within 5%."""
    e3 = _gpu_error(T, 100, M=25, sweeps=3, greedy=False)
    e8 = _gpu_error(T, 100, M=25, sweeps=8, greedy=False)
    assert abs(e3 - e8) <= 0.05 * e8, (e3, e8)


@pytest.mark.parametrize("s,p,order", [(1, 1, 1.8), (2, 2, 2.7), (3, 3, 3.5)])
def test_st_convergence_rate(T, s, p, order):
    """The paper's refinement study on the full window: Algorithm 1 as printed with
    30 modes and 4 subspace iterations, 100 -> 200 -> 400 nodes per dim: the error falls
    at each step at an observed order of at least `order` in h (p + 1 in theory)."""
    errs = [_gpu_error(T, n, s, p, M=30, sweeps=4, greedy=False) for n in (100, 200, 400)]
    assert errs[0] > errs[1] > errs[2], errs
    rate = math.log(errs[0] / errs[2]) / math.log(399 / 99)
    assert rate >= order, (errs, rate)
