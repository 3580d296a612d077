"""The Gram refresh on the tensor cores (tcgen05 kind::f16, BF16 operands, FP32
accumulation in tensor memory) through the C ABI: per dim (the TAPS_BF16 sweeps' path)
and batched (one persistent launch over every dim of every instance, with its tile
tuner), element by element against the FP64 contraction of the same bfloat16-rounded
operands (Eq. 34: Gamma_o = U^T Op_o U, h_r = U^T q_r)."""
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


def bf16(x):
    """FP64 -> FP32 -> bfloat16 (round to nearest even), as FP64 values."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def dense(band, hb):
    n = band.shape[0]
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(2 * hb + 1):
            j = i + k - hb
            if 0 <= j < n:
                A[i, j] = band[i, k]
    return A


def check_dim(T, P, U0, d, M, names):
    """The problem's current Grams of dim d against the FP64 contraction of the rounded
    operands; per entry within (2^-15 + (n + nb) 2^-23) sum_i |U_im| (|Op| |U|)_in (the
    split of the banded product and FP32 accumulation over n nodes)."""
    g, h, ops = P.grams(d, M)
    Ub = bf16(U0[d])
    n = Ub.shape[0]
    hb = P.dims[d].hb
    worst = 0.0
    for o, code in enumerate(ops):
        Ob = bf16(dense(P.op_band(d, names[code]), hb))
        ref = Ub.T @ (Ob @ Ub)
        mag = np.abs(Ub).T @ (np.abs(Ob) @ np.abs(Ub))
        bound = (2.0 ** -15 + (n + 2 * hb + 1) * 2.0 ** -23) * mag
        assert np.all(np.abs(g[o] - ref) <= bound), (d, o, np.max(np.abs(g[o] - ref) / bound))
        worst = max(worst, float(np.max(np.abs(g[o] - ref) / np.maximum(mag, 1e-300))))
    Q = np.stack([bf16(P.source(r, d)) for r in range(h.shape[0])], axis=0)
    href = Q @ Ub
    hmag = np.abs(Q) @ np.abs(Ub)
    assert np.all(np.abs(h - href) <= n * 2.0 ** -23 * hmag), (d, np.max(np.abs(h - href) / hmag))
    return worst


NAMES = {0: "K", 1: "M", 2: "G", 3: "W", 4: "Blo", 5: "Bhi"}


@pytest.mark.parametrize("case", ["poisson_k_M7", "poisson_k_M30", "transient_M20", "rich_M64"])
def test_tensor_core_grams_per_dim(T, case):
    """Space-parameter dims (K/M, W), a transient problem's time dim (G: nonsymmetric
    Grams, so a transposed operand shows), 64 modes and 40 source terms; ragged last
    chunks (nodes not a multiple of 64)."""
    if case == "poisson_k_M7":
        desc, M = W.poisson_k(n_space=50, n_k=12, seed=2050), 7
    elif case == "poisson_k_M30":
        desc, M = W.poisson_k(n_space=130, n_k=33, seed=2051), 30
    elif case == "transient_M20":
        desc, M = W.heat_transient(n_space=90, n_t=150, D_space=2, seed=3050), 20
    else:
        desc, M = W.heat_transient(n_space=100, n_t=70, D_space=2, seed=3051), 64
        rng = np.random.default_rng(7)
        desc["sources"] = [(1.0, [("nodal", rng.uniform(-1, 1, dm["n"])) for dm in desc["dims"]])
                           for _ in range(40)]
    P = T.Problem(desc)
    U0 = W.random_factors(desc, M, seed=91)
    U = P.factors(M)
    U.set(U0)
    P.refresh_grams(U, T.BF16)
    worst = max(check_dim(T, P, U0, d, M, NAMES) for d in range(P.D))
    print(f"{case}: worst |Gamma - ref| / (|U|^T |Op| |U|) = {worst:.2e}")


def test_batched_tensor_core_refresh(T):
    """Twelve instances of the batched configuration's family (D 3..6, n_d 32..700,
    M 4..32, Poisson or transient): one persistent launch refreshes every dim of every
    instance; each dim's Grams against the rounded-operand reference, the tuner's table
    filled with its choice the fastest, and the FP64 batched refresh equal bit for bit to
    each instance's own FP64 refresh."""
    descs, Ms = W.batch_instances(count=12, seed=4600, n_lo=32, n_hi=700, M_lo=4, M_hi=32)
    probs, facs, inits = [], [], []
    for i, (dsc, M) in enumerate(zip(descs, Ms)):
        P = T.Problem(dsc, stream=T.ctypes.c_void_p(torch.cuda.Stream().cuda_stream))
        U = P.factors(M)
        U0 = W.random_factors(dsc, M, seed=200 + i)
        U.set(U0)
        probs.append(P)
        facs.append(U)
        inits.append(U0)
    B = T.Batch(probs, facs, solver=T.SOLVER_FASTDIAG)
    ms, by = B.refresh_grams(T.BF16)
    rows, cps, table = B.gram_info()
    print(f"batched BF16 refresh: {ms:.3f} ms, {by / 1e6:.1f} MB, tile rows {rows}, CTAs/SM {cps}, table {table}")
    assert (rows, cps) in T.Batch.GRAM_TILES and ms > 0 and by > 0
    timed = [t for t in table if t > 0]
    assert timed and min(timed) == table[T.Batch.GRAM_TILES.index((rows, cps))]
    for P, U0, M in zip(probs, inits, Ms):
        for d in range(P.D):
            check_dim(T, P, U0, d, M, NAMES)
    # FP64: the batched call runs each instance's own FP64 refresh
    B.refresh_grams(T.FP64)
    got = [[P.grams(d, M)[0] for d in range(P.D)] for P, M in zip(probs, Ms)]
    for P, U, M, gl in zip(probs, facs, Ms, got):
        P.refresh_grams(U, T.FP64)
        for d in range(P.D):
            assert np.array_equal(P.grams(d, M)[0], gl[d])
