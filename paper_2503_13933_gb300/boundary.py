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
