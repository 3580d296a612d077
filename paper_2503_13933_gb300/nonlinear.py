"""Solution-dependent coefficients: the global-local iteration of App. A (Algorithm 2).

For rho c_p(u) and k(u) linear in u (the Sec. 3.3 setting), both coefficients are
separated fields with the modes of u plus a constant mode.  The global stage is the
linear weak form
    int du d/dt[c u] + int grad du . k grad u = int du f
with c and k frozen at the previous iterate: per mode j of c (coefficient m_c; n_c
for the constant mode) the term (x)_{space} M[v_j] (x) G[v_j], and per mode j of k and
space direction e the term K[v_j] in dim e, M[v_j] in the other space dims and M[v_j]
in time, X[v] the 1D operator weighted by the C-HiDeNN interpolant of the mode's
factor v (TAPS_OP_WEIGHTED operators, assembled on the device).  The local stage
updates c and k from the new u; with linear laws that is exact in the separated form
(the weights become the new factors).  The iteration stops when the relative change of
u falls below the tolerance (taps_factors_rel_change, on the device).  The problem and
its term structure are built once; each global stage re-assembles the weighted
operators and runs Algorithm 1.
"""
from __future__ import annotations

import numpy as np

from . import taps


def _free_index(dm):
    n = dm["n"]
    lo = 1 if dm["dirichlet_lo"] else 0
    hi = n - 1 if dm["dirichlet_hi"] else n
    return lo, hi


def global_terms(D, M, law):
    """Terms of the global stage (space dims 0..D-2, time dim D-1) and, per dim, the
    weighted operators they use as (base, mode j): 'w<i>' in a term is entry i."""
    m_c, n_c, m_k, n_k = law
    Ds = D - 1
    wops = [[] for _ in range(D)]

    def w(d, base, j):
        key = (base, j)
        if key not in wops[d]:
            wops[d].append(key)
        return f"w{wops[d].index(key)}"

    terms = [(n_c, ["M"] * Ds + ["G"])]
    terms += [(n_k, ["K" if d == e else "M" for d in range(Ds)] + ["M"]) for e in range(Ds)]
    for j in range(M):
        if m_c != 0.0:
            terms.append((m_c, [w(d, "M", j) for d in range(Ds)] + [w(Ds, "G", j)]))
        if m_k != 0.0:
            for e in range(Ds):
                terms.append((m_k, [w(d, "K" if d == e else "M", j) for d in range(Ds)] + [w(Ds, "M", j)]))
    return terms, wops


class GlobalLocal:
    """Algorithm 2 for a description `desc` (dims with time last, sources; its terms
    are replaced) and law = (m_c, n_c, m_k, n_k)."""

    def __init__(self, desc, law, M, stream=None):
        self.law = law
        self.M = M
        D = len(desc["dims"])
        terms, self.wops = global_terms(D, M, law)
        if len(terms) > taps.MAX_TERMS:
            raise ValueError(f"{len(terms)} operator terms for M = {M} exceed the library's {taps.MAX_TERMS}")
        self.desc = dict(desc, terms=terms)
        self.dims = desc["dims"]
        self.P = taps.Problem(self.desc, stream=stream)
        self.U = self.P.factors(M)
        self.U_old = self.P.factors(M)
        self._set_weights(None)

    def _set_weights(self, U):
        """Weighted operators from the factors of u (all nodes; zero before the first
        global stage, so that its terms vanish and the stage is the constant-coefficient
        problem)."""
        for d, ops in enumerate(self.wops):
            if not ops:
                continue
            n = self.dims[d]["n"]
            lo, hi = _free_index(self.dims[d])
            spec = []
            for base, j in ops:
                v = np.zeros(n)
                if U is not None:
                    v[lo:hi] = U[d][:, j]
                spec.append((base, v))
            self.P.set_weighted(d, spec)

    def solve(self, sweeps, max_iters=50, tol=1e-8, U0=None, seed=0, solver=taps.SOLVER_BLOCK_LU):
        """Global stages of `sweeps` subspace iterations each, from U0 (free-node factors
        per dim; default seeded U(-1, 1) values), until the relative change of u <= tol.
        Returns (factors of u, history of relative changes; the first is inf)."""
        if U0 is None:
            rng = np.random.default_rng(seed)
            U0 = [rng.uniform(-1.0, 1.0, (nf, self.M)) for nf in self.P.n_free]
        self.U.set(U0)
        self._set_weights(None)
        hist, U = [], None
        for it in range(max_iters):
            self.U_old.copy_from(self.U)
            self.P.sweep(self.U, sweeps, solver=solver)
            ch = self.U.rel_change(self.U_old) if it > 0 else float("inf")
            hist.append(ch)
            U = self.U.get()   # the new weights (host copies for the weighted-operator call)
            self._set_weights(U)
            if ch <= tol:
                break
        return U, hist
