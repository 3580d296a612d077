"""Warm-start network on the GPU against the FP64 oracle (gradients <= 1e-4 relative in
FP32), training, and the profiles -> factors initialisation."""
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


def _rand_case(dims, B, seed):
    rng = np.random.default_rng(seed)
    n = sum(i * o + o for i, o in zip(dims[:-1], dims[1:]))
    p = rng.normal(0, 0.3, n).astype(np.float32)
    X = rng.normal(0, 1, (B, dims[0])).astype(np.float32)
    Tt = rng.normal(0, 1, (B, dims[-1])).astype(np.float32)
    return p, X, Tt


@pytest.mark.parametrize("dims,B", [([21, 32, 32, 32, 17], 9), ([5, 64, 3], 40), ([21, 256, 256, 256, 257], 33)])
def test_mlp_gradients_match_oracle(T, dims, B):
    p, X, Tt = _rand_case(dims, B, 3)
    net = T.MLP(dims[0], dims[1], len(dims) - 2, dims[-1])
    net.set_params(p)
    loss, g = net.grad(torch.tensor(X, device="cuda"), torch.tensor(Tt, device="cuda"))
    lo, go = O.mlp_loss_grad(p.astype(float), dims, X.astype(float), Tt.astype(float))
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    y = torch.empty((B, dims[-1]), dtype=torch.float32, device="cuda")
    net.forward(torch.tensor(X, device="cuda"), y)
    torch.cuda.synchronize()
    yo = O.mlp_forward(p.astype(float), dims, X.astype(float))[-1]
    assert np.max(np.abs(y.cpu().numpy() - yo)) <= 1e-5 * max(1.0, np.max(np.abs(yo)))


def test_mlp_adam_step_matches_oracle(T):
    dims, B = [6, 16, 4], 11
    p, X, Tt = _rand_case(dims, B, 4)
    net = T.MLP(6, 16, 1, 4)
    net.set_params(p)
    xd, td = torch.tensor(X, device="cuda"), torch.tensor(Tt, device="cuda")
    pp, m, v = p.astype(float), np.zeros(p.size), np.zeros(p.size)
    for t in (1, 2, 3):
        net.grad(xd, td, want_grad=False)
        net.adam(lr=1e-2)
        _, go = O.mlp_loss_grad(pp, dims, X.astype(float), Tt.astype(float))
        pp, m, v = O.adam_step(pp, go, m, v, t, lr=1e-2)
    assert np.max(np.abs(net.params() - pp)) < 2e-5


def test_mlp_training_fits_a_smooth_map(T):
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (256, 3)).astype(np.float32)
    Y = np.stack([np.sin(2 * X[:, 0]) * X[:, 1], np.cos(X[:, 2]) - X[:, 0] ** 2], axis=1).astype(np.float32)
    net = T.MLP(3, 64, 2, 2, seed=1)
    xd, yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    l0, _ = net.grad(xd, yd, want_grad=False)
    l1 = net.train(xd, yd, 1500, lr=3e-3)
    assert l1 < 0.02 * l0, (l0, l1)


def test_factors_from_profiles(T):
    desc = W.poisson_k(n_space=20, n_k=9, seed=2012)
    P = T.Problem(desc)
    U = P.factors(3)
    n_ref = 16
    rng = np.random.default_rng(6)
    prof = rng.uniform(-1, 1, (3, 4 * n_ref + 1)).astype(np.float32)
    U.from_profiles(torch.tensor(prof, device="cuda"), 3, n_ref, weight_scale=2.5)
    got = U.get()
    for d, dm in enumerate(desc["dims"]):
        xs = np.linspace(0, 1, dm["n"])
        off = 1 if dm["dirichlet_lo"] else 0
        nodes = xs[off:off + got[d].shape[0]]
        for m in range(3):
            ref = np.interp(nodes, np.linspace(0, 1, n_ref), prof[m, d * n_ref:(d + 1) * n_ref].astype(float))
            if d == 3:
                ref = ref * 2.5 * float(prof[m, -1])
            assert np.max(np.abs(got[d][:, m] - ref)) < 1e-6 * max(1.0, np.max(np.abs(ref)))


def test_warm_start_gain_over_random_init(T):
    """What the trained network gains over the method without it.  Trained on the
    converged factors of 8 seeded space-parameter instances (48^3 x 16, M = 24), it
    initialises 3 held-out instances.  After the first sweep the warm start's Eq. 42
    residual is more than 3x below the random start's, and at no later sweep of the
    first three is it more than 2x above it.  (From the second sweep on both starts
    are in the slow, oscillating phase of the subspace iteration, where the order of
    two nearby residuals is set by rounding; sweeps-to-target are reported by the
    benchmark, not asserted here.)"""
    from paper_2503_13933_gb300 import warmstart as WS
    M = 24
    X, Tt, _ = WS.training_set(range(2101, 2109), n_space=48, n_k=16, M=M, res_tol=1e-8, max_sweeps=40)
    ws = WS.WarmStart(M=M)
    ws.fit(X, Tt, steps=3000, lr=5e-4)
    for sd in (2200, 2201, 2202):
        desc = W.poisson_k(48, 16, seed=sd)
        P = T.Problem(desc)
        Ur, Um = P.factors(M), P.factors(M)
        rr = P.solve(Ur, M0=M, M_max=M, res_tol=-1.0, max_sweeps=3, init=T.INIT_RANDOM, seed=sd,
                     als_tol=0.0, solver=T.SOLVER_FASTDIAG)
        ws.init_factors(P, Um, desc)
        rm = P.solve(Um, M_max=M, res_tol=-1.0, max_sweeps=3, init=T.INIT_GIVEN, als_tol=0.0,
                     solver=T.SOLVER_FASTDIAG)
        hr = [h[2] for h in rr["history"]]
        hm = [h[2] for h in rm["history"]]
        print(f"seed {sd}: residual per sweep random {hr} vs warm {hm}")
        assert hm[0] * 3.0 < hr[0]
        assert all(a <= 2.0 * b for a, b in zip(hm, hr)), (hm, hr)
