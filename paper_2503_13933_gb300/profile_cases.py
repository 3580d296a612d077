"""Small, seeded cases for kernel profiles (ncu captures stay small enough to end on
their own): run one or more by name, in the order given.

    python -m paper_2503_13933_gb300.profile_cases modediag convection images
    python -m paper_2503_13933_gb300.profile_cases pencil

modediag   : poisson_k 256^3 x 32, M = 30, two sweeps on the mode-side route
convection : a powder-bed-fusion slab at 128^2 x 32 space, M = 20, two sweeps
             (convection-face route on the space dims)
images     : the FP32 tensor-core reconstruction of poisson_k 160^3 x 32, M = 30
pencil     : poisson_k 256^3 x 32, M = 30, one node-side sweep (the pencil
             decomposition of the 254-node space dims runs first)
nonlinear  : the temperature-dependent moving-source plate at full size (101^2 x 11
             space, 113 time, M = 10): two global stages of two subspace iterations
"""
from __future__ import annotations

import sys


def _modediag(taps, W):
    d = W.poisson_k(256, 32, seed=2000)
    P = taps.Problem(d)
    U = P.factors(30)
    U.set(W.random_factors(d, 30, seed=1))
    P.sweep(U, 2, solver=taps.SOLVER_MODEDIAG)


def _convection(taps, W):
    d = W.lpbf_slab(n_xy=128, n_z=32, n_t=32, n_par=8)
    P = taps.Problem(d)
    U = P.factors(20)
    U.set(W.random_factors(d, 20, seed=2))
    P.sweep(U, 2, solver=taps.SOLVER_FASTDIAG)


def _images(taps, W):
    import torch
    d = W.poisson_k(160, 32, seed=2000)
    P = taps.Problem(d)
    U = P.factors(30)
    U.set(W.random_factors(d, 30, seed=3))
    out = torch.empty(160 ** 3 * 32, dtype=torch.float32, device="cuda")
    P.eval_grid(U, [0, 0, 0, 0], [160, 160, 160, 32], [1, 1, 1, 1], out)


def _pencil(taps, W):
    d = W.poisson_k(256, 32, seed=2000)
    P = taps.Problem(d)
    U = P.factors(30)
    U.set(W.random_factors(d, 30, seed=1))
    P.sweep(U, 1, solver=taps.SOLVER_FASTDIAG)


def _nonlinear(taps, W):
    from . import nonlinear as NL
    gl = NL.GlobalLocal(W.nonlinear_track(), W.INCONEL_LAW, 10)
    gl.solve(2, max_iters=2, tol=0.0, seed=5)


CASES = dict(modediag=_modediag, convection=_convection, images=_images, pencil=_pencil, nonlinear=_nonlinear)


def main(argv=None):
    import torch
    from . import taps, workloads as W
    names = (argv if argv is not None else sys.argv[1:]) or ["modediag", "convection", "images"]
    for nm in names:
        if nm not in CASES:
            raise SystemExit(f"unknown case {nm!r}; cases: {', '.join(CASES)}")
    taps.lib()
    for nm in names:
        CASES[nm](taps, W)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
