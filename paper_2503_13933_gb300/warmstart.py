"""Learned warm start (A12/A13): a network trained on converged factors that the method
itself produces across parameter draws proposes every mode's initial factors.

Training data are built here on the host from factors the GPU solver returned (mode
order, peak normalisation, sampling on a reference grid: dataset preparation).  The
network is trained and evaluated by the library's own kernels (taps_mlp_*), and the
predicted profiles become factors on the device (taps_factors_from_profiles).

Features of a space-parameter instance (workloads.poisson_k): its four Gaussian
sources sorted by amplitude, each (A, sigma, c_x, c_y, c_z) scaled to [-1, 1], plus the
mode index scaled to [-1, 1].  Targets per mode: for every dim the factor column
divided by its largest magnitude, sampled at N_REF uniform points of the dim (all-node
coordinates, zero at Dirichlet ends), then the mode weight prod_d max|U_d[:, m]| with
the sign of the last dim, divided by a training-set scale.  Modes are ordered by
decreasing weight.
"""
from __future__ import annotations

import numpy as np

from . import taps

N_REF = 64


def features_conductivity(desc, M):
    """Features of an instance of the large moving-source family: its conductivity k
    (scaled to [-1, 1] over [10, 30] W/m/K) and the mode index scaled to [-1, 1]."""
    k = float(desc["params"]["k"])
    X = np.zeros((M, 2), dtype=np.float32)
    X[:, 0] = (k - 20.0) / 10.0
    X[:, 1] = np.array([2.0 * m / max(M - 1, 1) - 1.0 for m in range(M)], dtype=np.float32)
    return X


def features(desc, M):
    g = sorted(desc["params"], key=lambda t: -t[0])
    base = []
    for A, sig, c in g:
        base += [(A - 1.25) / 0.75, (sig - 0.125) / 0.075] + [(ci - 0.5) / 0.3 for ci in c]
    X = np.zeros((M, len(base) + 1), dtype=np.float32)
    for m in range(M):
        X[m, :-1] = base
        X[m, -1] = 2.0 * m / max(M - 1, 1) - 1.0
    return X


def _all_nodes(dm, col):
    full = np.zeros(dm["n"])
    off = 1 if dm["dirichlet_lo"] else 0
    full[off:off + len(col)] = col
    return full


def targets(desc, Us, n_ref=N_REF):
    """Converged factors -> (targets [M, D*n_ref + 1], raw weights [M])."""
    dims = desc["dims"]
    D, M = len(Us), Us[0].shape[1]
    prof = np.zeros((M, D, n_ref))
    w = np.ones(M)
    for d, dm in enumerate(dims):
        xs = np.linspace(0.0, 1.0, dm["n"])
        xr = np.linspace(0.0, 1.0, n_ref)
        for m in range(M):
            col = _all_nodes(dm, Us[d][:, m])
            k = int(np.argmax(np.abs(col)))
            peak = col[k]
            if peak == 0.0:
                w[m] = 0.0
                continue
            prof[m, d] = np.interp(xr, xs, col / abs(peak))
            w[m] *= abs(peak) if d < D - 1 else peak
    order = np.argsort(-np.abs(w), kind="stable")
    T = np.concatenate([prof[order].reshape(M, D * n_ref), w[order, None]], axis=1)
    return T.astype(np.float64), w[order]


class WarmStart:
    """A taps.MLP plus the weight scale of its training set.  `features(desc, M)` maps an
    instance to the network's inputs; profiles live on n_ref points per dim."""

    def __init__(self, n_in=21, M=30, D=4, hidden=256, layers=3, seed=7, n_ref=N_REF, features=features):
        self.M, self.D, self.n_ref, self.features = M, D, n_ref, features
        self.net = taps.MLP(n_in, hidden, layers, D * n_ref + 1, seed=seed)
        self.weight_scale = 1.0

    def fit(self, X, T, steps=3000, lr=1e-3):
        """X [S, n_in], T [S, D*N_REF+1] (raw weights in the last column)."""
        import torch
        T = np.array(T, dtype=np.float64)
        self.weight_scale = float(np.max(np.abs(T[:, -1]))) or 1.0
        T[:, -1] /= self.weight_scale
        xd = torch.tensor(np.asarray(X, dtype=np.float32), device="cuda")
        td = torch.tensor(T.astype(np.float32), device="cuda")
        return self.net.train(xd, td, steps, lr)

    def init_factors(self, P, U, desc):
        """Predict profiles for every mode of `desc` and write them into U (device)."""
        import torch
        X = torch.tensor(self.features(desc, self.M), device="cuda")
        prof = torch.empty((self.M, self.D * self.n_ref + 1), dtype=torch.float32, device="cuda")
        self.net.forward(X, prof)
        U.from_profiles(prof, self.M, self.n_ref, self.weight_scale)
        return U


def training_set(seeds, n_space=256, n_k=32, M=30, res_tol=1e-8, max_sweeps=80):
    """Converged factors of the space-parameter instances `seeds` (GPU FP64 solver with
    fast diagonalisation) -> stacked (X, T) and the per-instance sweep counts."""
    from . import workloads as W
    Xs, Ts, sweeps = [], [], []
    for sd in seeds:
        desc = W.poisson_k(n_space, n_k, seed=sd)
        P = taps.Problem(desc)
        U = P.factors(M)
        r = P.solve(U, M0=M, M_max=M, res_tol=res_tol, res_kind=taps.RES_ALS, max_sweeps=max_sweeps,
                    init=taps.INIT_RANDOM, seed=sd, als_tol=0.0, solver=taps.SOLVER_FASTDIAG)
        sweeps.append(r["sweeps"])
        T, _ = targets(desc, U.get())
        Xs.append(features(desc, M))
        Ts.append(T)
    return np.concatenate(Xs), np.concatenate(Ts), sweeps


def training_set_conductivity(base, ks, M=100, sweeps=12, n_ref=1536, dim_cache=None, seed=0):
    """Factors of the large moving-source family at the conductivities `ks` (the base
    description's other data shared), M modes after `sweeps` FP64 sweeps from the same
    seeded random factors -> stacked (X, T)."""
    from . import workloads as W
    Xs, Ts = [], []
    for j, k in enumerate(ks):
        desc = W.with_conductivity(base, k)
        P = taps.Problem(desc, dim_cache=dim_cache)
        U = P.factors(M)
        # one seed for every conductivity: the iterations of neighbouring k follow each
        # other, so their modes are comparable targets
        P.solve(U, M0=M, M_max=M, res_tol=-1.0, max_sweeps=sweeps, init=taps.INIT_RANDOM, seed=seed,
                als_tol=0.0, solver=taps.SOLVER_FASTDIAG)
        T, _ = targets(desc, U.get(), n_ref)
        Xs.append(features_conductivity(desc, M))
        Ts.append(T)
        del U, P
    return np.concatenate(Xs), np.concatenate(Ts)
