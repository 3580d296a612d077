"""Batched independent instances: one CUDA graph sweeping all instances gives exactly the
per-instance results, and an instance agrees with the oracle."""
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


def _instances(T, count, seed):
    descs, Ms = W.batch_instances(count=count, seed=seed, n_lo=10, n_hi=24, M_lo=2, M_hi=5)
    probs, facs, inits = [], [], []
    for i, (dsc, M) in enumerate(zip(descs, Ms)):
        P = T.Problem(dsc, stream=T.ctypes.c_void_p(torch.cuda.Stream().cuda_stream))
        U = P.factors(M)
        U0 = W.random_factors(dsc, M, seed=100 + i)
        U.set(U0)
        probs.append(P)
        facs.append(U)
        inits.append(U0)
    return descs, probs, facs, inits


@pytest.mark.parametrize("solver", ["fastdiag", "block_lu"])
def test_batched_graph_equals_per_instance(T, solver):
    sv = T.SOLVER_FASTDIAG if solver == "fastdiag" else T.SOLVER_BLOCK_LU
    descs, probs, facs, inits = _instances(T, 6, 4100)
    B = T.Batch(probs, facs, solver=sv)
    chg = B.sweep(3, graphs=True)
    got = [u.get() for u in facs]
    for P, U, U0 in zip(probs, facs, inits):
        U.set(U0)
    chg2 = T.Batch(probs, facs, solver=sv).sweep(3, graphs=False)
    ref = [u.get() for u in facs]
    for a, b in zip(got, ref):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert np.array_equal(chg, chg2)
    # one instance against the oracle
    Po = O.problem_from_description(descs[0])
    Uo = [u.copy() for u in inits[0]]
    for _ in range(3):
        Uo, _ = O.sweep(Po, Uo, solver="fastdiag" if solver == "fastdiag" else "banded")
    a, b = O.cp_full(got[0]), O.cp_full(Uo)
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)


@pytest.mark.parametrize("graphs", [True, False])
def test_batched_sweep_restarts_from_reset_factors(T, graphs):
    """Factors set between two calls on the same batch: the second call starts from the
    new factors (every instance's Grams are recomputed), so resetting to the initial
    factors repeats the first call bit for bit."""
    descs, probs, facs, inits = _instances(T, 5, 4200)
    B = T.Batch(probs, facs, solver=T.SOLVER_FASTDIAG)
    c1 = B.sweep(2, graphs=graphs)
    first = [u.get() for u in facs]
    for U, U0 in zip(facs, inits):
        U.set(U0)
    c2 = B.sweep(2, graphs=graphs)
    again = [u.get() for u in facs]
    for a, b in zip(first, again):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert np.array_equal(c1, c2)


def test_batched_auto_solver_choice_is_timed_and_kept(T):
    """TAPS_SOLVER_AUTO: the first graph sweep times one batch sweep with each solver
    (factors restored), keeps the faster, and gives exactly the factors of a batch made
    with that solver."""
    descs, probs, facs, inits = _instances(T, 6, 4300)
    B = T.Batch(probs, facs, solver=T.SOLVER_AUTO)
    c1 = B.sweep(2, graphs=True)
    chosen, trial = B.info()
    assert chosen in (T.SOLVER_FASTDIAG, T.SOLVER_MODEDIAG)
    assert trial[0] > 0 and trial[1] > 0
    assert (chosen == T.SOLVER_FASTDIAG) == (trial[0] <= trial[1])
    got = [u.get() for u in facs]
    for U, U0 in zip(facs, inits):
        U.set(U0)
    c2 = T.Batch(probs, facs, solver=chosen).sweep(2, graphs=True)
    for a, b in zip(got, [u.get() for u in facs]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert np.array_equal(c1, c2)


def test_batched_statuses_report_per_instance(T):
    """With statuses requested every instance runs all sweeps and reports its own
    status (all well posed here: zeros)."""
    descs, probs, facs, inits = _instances(T, 4, 4400)
    B = T.Batch(probs, facs, solver=T.SOLVER_MODEDIAG)
    ch, st = B.sweep(2, graphs=True, statuses=True)
    assert st.tolist() == [0, 0, 0, 0] and np.all(np.isfinite(ch))


def test_batched_instances_at_full_dim_sizes_match_oracle(T):
    """Four instances of the batched configuration's family at n_d in [256, 320] (three
    transient with a time dim on the mode side, one 6-dim Poisson; M = 4..6), swept
    three times as one CUDA graph, against the oracle's sweeps (fast diagonalisation)
    from the same factors.  The sources are M + 2 random separable nodal terms, so the
    right-hand sides have rank above M and the reduced systems stay well conditioned
    (with one or two Gaussians the fixed-M modes turn nearly collinear after a sweep,
    where even the oracle's two FP64 solvers disagree at 1e-9..1e-6).  Whole fields
    compared through the telescoped CP difference, and factors: both within 1e-10."""
    descs, Ms = W.batch_instances(count=4, seed=4500, n_lo=256, n_hi=320, M_lo=4, M_hi=8)
    probs, facs, inits = [], [], []
    for i, (dsc, M) in enumerate(zip(descs, Ms)):
        rng = np.random.default_rng(900 + i)
        dsc["sources"] = [(1.0, [("nodal", rng.uniform(-1, 1, dm["n"])) for dm in dsc["dims"]])
                          for _ in range(M + 2)]
        P = T.Problem(dsc, stream=T.ctypes.c_void_p(torch.cuda.Stream().cuda_stream))
        U = P.factors(M)
        U0 = W.random_factors(dsc, M, seed=100 + i)
        U.set(U0)
        probs.append(P)
        facs.append(U)
        inits.append(U0)
    B = T.Batch(probs, facs, solver=T.SOLVER_FASTDIAG)
    B.sweep(3, graphs=True)
    for i, (dsc, U, U0) in enumerate(zip(descs, facs, inits)):
        Po = O.problem_from_description(dsc)
        Uo = [u.copy() for u in U0]
        for _ in range(3):
            Uo, _ = O.sweep(Po, Uo, solver="fastdiag")
        got = U.get()
        field = O.cp_change(Uo, got)
        fac = max(np.linalg.norm(g - o) / np.linalg.norm(o) for g, o in zip(got, Uo))
        print(f"instance {i}: D = {len(dsc['dims'])}, n_d = {[dm['n'] for dm in dsc['dims']]}, "
              f"M = {Ms[i]}: field rel. diff {field:.2e}, factors {fac:.2e}")
        assert field <= 1e-10 and fac <= 1e-10, (i, field, fac)
