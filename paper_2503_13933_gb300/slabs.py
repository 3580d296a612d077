"""Space-parameter-time slabs (Sec. 2.4, Eq. 16; App. B, Eq. 56): the initial condition
of slab T+1 is the state of slab T at its last time node.

With the lifting u = u_end (x) 1_t + w, w(t = 0) = 0, the next slab solves for w with
the same operator and a force that gains, for every operator term without a time
derivative and every mode m of u_end, the separable term
    -alpha_t * tau_m * (x)_{d != t} (Op_{t,d} U_d[:, m]) (x) (M_t 1),
where tau_m is mode m's time factor at t_max (the time derivative of the constant-in-
time lifting vanishes).  The end state of slab T+1 is u_end + w(., t_max): the modes
of both, concatenated; `compress` reduces them again (App. B: the L2 projection of the
end state onto fewer modes, solved by the same subspace iteration).
"""
from __future__ import annotations

import numpy as np


class EndState:
    """u_end(x) = sum_m weight[m] prod_{d != time} U[d][:, m] over the free nodes."""

    def __init__(self, U, weight, time_dim):
        self.U = U                # list over all dims; U[time_dim] is None
        self.weight = np.asarray(weight, dtype=float)
        self.time_dim = time_dim

    @property
    def M(self):
        return len(self.weight)


def end_state(Us, time_dim, previous=None):
    """End state of a slab from its factors (and the lifting of the previous slab)."""
    U = [None if d == time_dim else np.array(u) for d, u in enumerate(Us)]
    w = np.array(Us[time_dim][-1, :])
    if previous is not None and previous.M > 0:
        U = [None if d == time_dim else np.concatenate([previous.U[d], U[d]], axis=1)
             for d in range(len(U))]
        w = np.concatenate([previous.weight, w])
    return EndState(U, w, time_dim)


def lifting_sources(desc, state):
    """Extra source terms (description format) carrying the initial condition."""
    t = state.time_dim
    out = []
    for alpha, ops in desc["terms"]:
        if ops[t] == "G":
            continue
        if ops[t] != "M":
            raise ValueError("time operator of a term without time derivative must be 'M'")
        for m in range(state.M):
            facs = [("const", (1.0,)) if d == t else ("opvec", (ops[d], state.U[d][:, m]))
                    for d in range(len(ops))]
            out.append((-alpha * state.weight[m], facs))
    return out


def next_slab(desc, state, t_shift):
    """Description of the next slab: the time window moved by t_shift and the lifting
    sources appended."""
    nd = dict(desc)
    dims = [dict(dm) for dm in desc["dims"]]
    t = state.time_dim
    dims[t]["lo"] += t_shift
    dims[t]["hi"] += t_shift
    nd["dims"] = dims
    nd["sources"] = list(desc["sources"]) + lifting_sources(desc, state)
    return nd


def compression_description(desc, state):
    """The mode-compression problem of an end state (App. B): over the dims other than
    time, the operator (x)_d M_d and one source term per mode, w_m (x)_d M_d U_d[:, m]
    (the projection of u_end)."""
    t = state.time_dim
    keep = [d for d in range(len(desc["dims"])) if d != t]
    return dict(name="compress", dims=[desc["dims"][d] for d in keep], terms=[(1.0, ["M"] * len(keep))],
                sources=[(float(state.weight[m]), [("opvec", ("M", state.U[d][:, m])) for d in keep])
                         for m in range(state.M)])


def compress(desc, state, U0, sweeps, stream=None, dim_cache=None):
    """Compressed end state: `sweeps` subspace-iteration sweeps of the compression
    problem on the GPU from the initial factors U0 (one array per kept dim, M_new
    columns).  Weights are 1: the normalisation puts each mode's scale in the last dim.
    dim_cache: shared assembled dims (see taps.Problem)."""
    from . import taps
    cdesc = compression_description(desc, state)
    P = taps.Problem(cdesc, stream=stream, dim_cache=dim_cache)
    M_new = U0[0].shape[1]
    U = P.factors(M_new)
    U.set(U0)
    P.sweep(U, sweeps, solver=taps.SOLVER_FASTDIAG)
    got = U.get()
    keep = [d for d in range(len(desc["dims"])) if d != state.time_dim]
    out = [None] * len(desc["dims"])
    for j, d in enumerate(keep):
        out[d] = got[j]
    return EndState(out, np.ones(M_new), state.time_dim)
