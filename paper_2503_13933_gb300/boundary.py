"""Non-homogeneous Dirichlet data by lifting (the Sec. 2.5 weak form with u = u_D + w).

The boundary data enter as a lifting u_D = sum_m weight[m] (x)_d V[d][:, m], each
V[d] given at ALL nodes of dim d (constrained ones included; only the values at the
constrained nodes fix the answer, the interior values only change how the work splits
between u_D and w).  The unknown w vanishes on the constrained nodes, so it is solved
with the homogeneous machinery; the lifting moves to the right-hand side as, per
operator term t with coefficient alpha_t and per lifting mode m, the separable source

    -alpha_t * weight[m] * (x)_d (Op_{t,d} V[d][:, m]) restricted to the free nodes,

which the library forms on the device (source kind "opvecfull").  The answer is
u = u_D + w: at the free nodes, w plus the lifting's values there.
"""
from __future__ import annotations

import numpy as np


def lifting_sources(desc, vecs, weights):
    """Source terms (description format) that carry the lifting (vecs, weights) of
    `desc`'s operator; append them to desc["sources"]."""
    weights = np.asarray(weights, dtype=float)
    D = len(desc["dims"])
    if len(vecs) != D:
        raise ValueError("one lifting factor per dim")
    for d in range(D):
        v = np.asarray(vecs[d])
        if v.ndim != 2 or v.shape != (desc["dims"][d]["n"], len(weights)):
            raise ValueError(f"dim {d}: lifting factor must be n x M (all nodes)")
    out = []
    for alpha, ops in desc["terms"]:
        for m, wm in enumerate(weights):
            out.append((-float(alpha) * float(wm),
                        [("opvecfull", (ops[d], np.ascontiguousarray(vecs[d][:, m], dtype=float)))
                         for d in range(D)]))
    return out


def lifted(desc, vecs, weights):
    """`desc` with the lifting's sources appended (a new description)."""
    return dict(desc, sources=list(desc["sources"]) + lifting_sources(desc, vecs, weights))


class LiftedField:
    """u = w + u_D at arbitrary points, both parts on the device: w through the solved
    factors of the lifted problem, u_D through the lifting's all-node factors on a copy
    of the dims with no constrained node (the same C-HiDeNN interpolation), in chunks of
    at most 128 lifting modes (the factor width limit)."""

    CHUNK = 128

    def __init__(self, desc, vecs, weights, stream=None):
        from . import taps
        weights = np.asarray(weights, dtype=float)
        free = dict(desc, dims=[dict(dm, dirichlet_lo=False, dirichlet_hi=False) for dm in desc["dims"]],
                    sources=[(1.0, [("const", (1.0,))] * len(desc["dims"]))])
        self._P = taps.Problem(free, stream=stream)
        self._U = []
        for a in range(0, len(weights), self.CHUNK):
            b = min(a + self.CHUNK, len(weights))
            U = self._P.factors(b - a)
            U.set([np.asarray(vecs[0][:, a:b], dtype=float) * weights[None, a:b]] +
                  [np.asarray(v[:, a:b], dtype=float) for v in vecs[1:]])
            self._U.append(U)

    def eval_points(self, P, U, pts, out):
        """out = w(pts) + u_D(pts); pts a CUDA float64 tensor [n, D], out CUDA float64 [n]."""
        import torch
        P.eval_points(U, pts, out)
        tmp = torch.empty_like(out)
        for UL in self._U:
            self._P.eval_points(UL, pts, tmp)
            out += tmp
        return out
