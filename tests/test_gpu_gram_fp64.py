"""The FP64 Gram refresh (Eq. 34: Gamma_o = U^T Op_o U, h_r = U^T q_r) through the C
ABI against the oracle's contraction, on both of its routes: a dim of many nodes with
more than 32 modes (banded products once, then the tiled contraction over the nodes
with its chunk reduction), and the fused per-chunk kernel elsewhere.  The device
assembles its own operators and source projections, which agree with the oracle's to
~1e-12 relative (the assembly and source parity tests), so the bound here is 5e-12 of
|U|^T |Op| |U| (resp. |U|^T |q|), not the contraction's own rounding."""
import numpy as np
import pytest

from paper_2503_13933_gb300 import workloads as W
from oracle import taps_oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_13933_gb300 import taps
    taps.lib()
    return taps


@pytest.mark.parametrize("case,M", [("poisson_k", 33), ("poisson_k", 100), ("transient", 64), ("poisson_k", 24)])
def test_fp64_gram_refresh_matches_oracle(T, case, M):
    if case == "poisson_k":
        desc = W.poisson_k(n_space=300, n_k=40, seed=2090)
    else:
        desc = W.heat_transient(n_space=270, n_t=70, D_space=2, seed=3090)
    rng = np.random.default_rng(11)
    # many source terms, so that the source columns span several output tiles
    desc["sources"] = desc["sources"] + [(1.0, [("nodal", rng.uniform(-1, 1, dm["n"])) for dm in desc["dims"]])
                                         for _ in range(40)]
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    U0 = W.random_factors(desc, M, seed=92)
    U = P.factors(M)
    U.set(U0)
    P.refresh_grams(U, T.FP64)
    worst = 0.0
    for d in range(len(desc["dims"])):
        g, h, ops = P.grams(d, M)
        for k, op in enumerate(ops):
            Op = Po.ops[d][op]
            ref = O.gram(U0[d], Op)
            scale = np.abs(U0[d]).T @ np.abs(Op) @ np.abs(U0[d])
            err = np.max(np.abs(g[k] - ref) / (scale + 1e-300))
            worst = max(worst, err)
            assert err < 5e-12, (d, op, err)
        for r, (beta, qs) in enumerate(Po.sources):
            ref = U0[d].T @ qs[d]
            scale = np.abs(U0[d]).T @ np.abs(qs[d])
            err = np.max(np.abs(h[r] - ref) / (scale + 1e-300))
            worst = max(worst, err)
            assert err < 5e-12, (d, r, err)
    print(f"{case} M={M}: worst |Gamma - ref| / (|U|^T |Op| |U|) = {worst:.2e}")
