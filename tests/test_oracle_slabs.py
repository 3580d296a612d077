"""Pin of the oracle's slab chaining (Eq. 16 continuity by lifting): under a
time-independent source, chained slabs approach the steady state, i.e. the solution of
the spatial finite-element problem K u = q alone."""
import numpy as np

from oracle import taps_oracle as O
from paper_2503_13933_gb300 import workloads as W


def test_chained_slabs_reach_the_steady_state():
    desc = W.heat_transient(n_space=12, n_t=9, D_space=1, T=1.0, k=1.0, rho_cp=1.0, seed=3030,
                            n_gauss=1)
    desc["sources"] = [(1.0, [("sin", (np.pi, 0.0)), ("const", (1.0,))])]
    state = None
    cur = desc
    for slab in range(4):
        P = O.problem_from_description(cur)
        r = O.solve(P, M0=1, M_max=1, als_tol=1e-13, res_tol=-1.0, max_sweeps=200, init="random",
                    seed=slab + 1)
        state = O.slab_end_state(r.U, 1, state)
        cur = O.slab_next_description(desc, state, 1, (slab + 1) * 1.0)
    facs, wts = state
    u_end = facs[0] @ wts
    dm = O.dim_from_description(desc["dims"][0])
    K = O.assemble_free(dm)[O.OP_K]
    q = O.project_source(dm, "sin", (np.pi, 0.0))
    steady = np.linalg.solve(K, q)
    assert np.max(np.abs(u_end - steady)) < 1e-6 * np.max(np.abs(steady))


def test_lifting_continues_the_full_grid_solution():
    """1D space x time with 5 free nodes each and 5 random separable sources: M = 5 modes
    hold every grid function, so each slab's TAPS solution is the full-grid one.  The
    two-slab solution by lifting, u = u_end (x) 1 + w on slab 2, must equal the
    full-grid solve of slab 2 with the initial condition imposed directly (the IC
    node kept and fixed to u_end)."""
    rng = np.random.default_rng(4)
    desc = W.heat_transient(n_space=7, n_t=6, D_space=1, T=0.5, seed=3031)
    desc["sources"] = [(1.0, [("nodal", rng.uniform(-1, 1, 7)), ("nodal", rng.uniform(-1, 1, 6))])
                       for _ in range(5)]
    P = O.problem_from_description(desc)
    u1 = O.solve_full(P).reshape(5, 5)               # free x nodes, free t nodes
    r = O.solve(P, M0=5, M_max=5, als_tol=1e-14, res_tol=-1.0, max_sweeps=50, init="random", seed=2)
    assert np.linalg.norm(O.cp_full(r.U).reshape(5, 5) - u1) < 1e-9 * np.linalg.norm(u1)
    state = O.slab_end_state(r.U, 1)
    u_end = state[0][0] @ state[1]
    assert np.allclose(u_end, u1[:, -1])
    d2 = O.slab_next_description(desc, state, 1, 0.5)
    P2 = O.problem_from_description(d2)
    r2 = O.solve(P2, M0=5, M_max=5, als_tol=1e-14, res_tol=-1.0, max_sweeps=50, init="random", seed=3)
    u2 = O.cp_full(r2.U).reshape(5, 5) + u_end[:, None]
    # direct: all time nodes of slab 2 (t in [0.5, 1]), the first fixed to u_end
    d2d = dict(d2)
    d2d["dims"] = [dict(dm) for dm in d2["dims"]]
    d2d["dims"][1]["dirichlet_lo"] = False
    d2d["sources"] = desc["sources"]
    Pd = O.problem_from_description(d2d)
    A = O.full_operator(Pd)                          # free x nodes x all 6 time nodes
    F = O.full_rhs(Pd)
    nt = 6
    idx_ic = [i * nt for i in range(5)]
    idx_in = [i for i in range(5 * nt) if i % nt != 0]
    ub = A[np.ix_(idx_in, idx_in)]
    rhs = F[idx_in] - A[np.ix_(idx_in, idx_ic)] @ u_end
    direct = np.linalg.solve(ub, rhs).reshape(5, 5)
    assert np.linalg.norm(u2 - direct) < 1e-9 * np.linalg.norm(direct)


def test_mode_compression_recovers_a_low_rank_end_state():
    """An end state of 8 modes whose field has rank 2 (two modes split into weighted
    copies, plus pairs that cancel) is compressed to 2 modes: the compressed field
    equals the end state's (App. B's projection reproduces a field it can represent)."""
    desc = W.heat_transient(n_space=9, n_t=5, D_space=2, seed=3033)
    rng = np.random.default_rng(5)
    n = 7
    a = [rng.uniform(-1, 1, (n, 2)) for _ in range(2)]
    cols = [[], []]
    w = []
    for m in range(2):                  # mode m as 0.3 + 0.7 of itself
        for f in (0.3, 0.7):
            for d in range(2):
                cols[d].append(a[d][:, m])
            w.append(f)
    b = [rng.uniform(-1, 1, n) for _ in range(2)]
    for sgn in (1.0, -1.0):             # two cancelling pairs
        for _ in range(2):
            for d in range(2):
                cols[d].append(b[d])
            w.append(sgn)
    facs = [np.stack(cols[0], axis=1), np.stack(cols[1], axis=1), None]
    state = (facs, np.array(w))
    u_end = np.einsum("im,jm,m->ij", facs[0], facs[1], np.array(w))
    U0 = W.random_factors(dict(dims=[desc["dims"][0], desc["dims"][1]]), 2, seed=6)
    cf, cw = O.slab_compress(desc, state, 2, U0, sweeps=60)
    u_c = np.einsum("im,jm,m->ij", cf[0], cf[1], cw)
    assert np.linalg.norm(u_c - u_end) <= 1e-9 * np.linalg.norm(u_end)
    assert cf[2] is None and len(cw) == 2
