"""The allocation-free reconstruction entry point, through the C ABI.

taps_eval_grid_noalloc serves callers that cannot allocate device memory when they
need a field; it takes its working memory from a fixed array the library reserves
at load time.  Here it must reproduce taps_eval_grid (same tolerance as the other
reconstruction tests) on two calls in a row -- the second call finds the first
call's data in the shared array -- and refuse a request larger than that array.
This file is collected last so that a failure here cannot hide other results."""
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
    import os
    if not os.path.exists(taps.LIB_PATH):
        build.build()
    taps.lib()
    return taps


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_matches_eval_grid_twice(T, dtype):
    desc = W.poisson_k(n_space=40, n_k=12, seed=2007)
    P = T.Problem(desc)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    code = T.FP32 if dtype == "f32" else T.FP64
    tol = 2e-6 if dtype == "f32" else 1e-13
    grids = [([0, 0, 0, 0], [40, 40, 40, 12], [1, 1, 1, 1]),
             ([1, 3, 0, 2], [19, 12, 40, 5], [2, 3, 1, 2])]
    for call, (seed, (start, count, step)) in enumerate(zip((41, 42), grids)):
        U = P.factors(9)
        U.set(W.random_factors(desc, 9, seed=seed))
        n = int(np.prod(count))
        ref = torch.empty(n, dtype=tdt, device="cuda")
        got = torch.full((n,), float("nan"), dtype=tdt, device="cuda")
        P.eval_grid(U, start, count, step, ref, dtype=code)
        P.eval_grid_noalloc(U, start, count, step, got, dtype=code)
        torch.cuda.synchronize()
        r, g = ref.double().cpu().numpy(), got.double().cpu().numpy()
        assert np.all(np.isfinite(g)), call
        assert np.max(np.abs(g - r)) <= tol * np.max(np.abs(r)), call


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_matches_oracle_eval_grid(T, dtype):
    """Against the FP64 oracle's reconstruction (Eq. 13 at the nodes: the factor
    entries, zero at constrained nodes) on a strided slice with a ragged last dim,
    two calls in a row with different factors and grids."""
    desc = W.poisson_k(n_space=23, n_k=9, seed=2009)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    code = T.FP32 if dtype == "f32" else T.FP64
    # FP32: the factors rounded to float and M = 7 products of D = 4 of them summed in
    # float, a few units of 2^-24 times the magnitude of the terms
    tol = 1e-5 if dtype == "f32" else 1e-13
    for seed, (start, count, step) in ((43, ([0, 2, 1, 0], [23, 7, 11, 9], [1, 3, 2, 1])),
                                       (44, ([21, 0, 5, 3], [1, 23, 6, 5], [1, 1, 3, 1]))):
        U0 = W.random_factors(desc, 7, seed=seed)
        U = P.factors(7)
        U.set(U0)
        n = int(np.prod(count))
        got = torch.full((n,), float("nan"), dtype=tdt, device="cuda")
        P.eval_grid_noalloc(U, start, count, step, got, dtype=code)
        torch.cuda.synchronize()
        ref = O.eval_grid(Po, U0, [range(a, a + b * c, c) for a, b, c in zip(start, count, step)])
        g = got.double().cpu().numpy().reshape(ref.shape)
        err = float(np.max(np.abs(g - ref)) / np.max(np.abs(ref)))
        print(f"noalloc vs oracle ({dtype}): max rel. diff {err:.2e}")
        assert err <= tol, err


def test_noalloc_rejects_requests_beyond_its_scratch(T):
    """(4096 + 4096 + 1 + 12) rows x 128 modes x 8 bytes = 8.4 MB of gathered rows, above
    the 4 MiB array: refused with TAPS_ERR_SCRATCH_LIMIT before any launch.  The output
    buffer is allocated at full size anyway, so no launch could write out of bounds."""
    desc = W.poisson_k(n_space=4096, n_k=12, seed=2008)
    P = T.Problem(desc)
    U = P.factors(128)
    U.set(W.random_factors(desc, 128, seed=4))
    count = [4096, 4096, 1, 12]
    assert sum(count) * 128 * 8 > T.NOALLOC_SCRATCH_BYTES
    out = torch.zeros(int(np.prod(count)), dtype=torch.float64, device="cuda")
    with pytest.raises(T.TapsError) as e:
        P.eval_grid_noalloc(U, [0, 0, 0, 0], count, [1, 1, 1, 1], out, dtype=T.FP64)
    assert e.value.status == T.ERR_SCRATCH_LIMIT
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0       # nothing was launched
