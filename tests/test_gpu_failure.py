"""Failure detection without a GPU fault: the library's bounded grid barrier is made to
wait for CTAs that never arrive; the wait runs out, the kernel records the timeout and
returns, the host reads TAPS_ERR_TIMEOUT, and the context stays usable."""
import time

import numpy as np
import pytest

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


def test_barrier_with_all_ctas_passes(T):
    assert T.barrier_test(8, 0, 1 << 20) == T.OK


def test_barrier_wait_runs_out_and_reports_timeout(T):
    t0 = time.perf_counter()
    st = T.barrier_test(4, 1, 1 << 14)     # one CTA never arrives; 2^14 polls per wait
    dt = time.perf_counter() - t0
    assert st == T.ERR_TIMEOUT
    assert dt < 5.0
    # the status word was reset and the context is usable: the next barrier passes and
    # a sweep runs
    assert T.barrier_test(4, 0, 1 << 20) == T.OK
    desc = W.poisson_sin(10)
    P = T.Problem(desc)
    U = P.factors(2)
    U.set(W.random_factors(desc, 2, seed=1))
    ch = P.sweep(U, 1)
    assert np.isfinite(ch["change"])


def test_barrier_test_rejects_bad_arguments(T):
    assert T.barrier_test(0, 0, 10) == T.ERR_INVALID_ARG
    assert T.barrier_test(4, 0, 0) == T.ERR_INVALID_ARG
