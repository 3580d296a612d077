"""Pins of the oracle's subspace iteration (Algorithm 1, Eq. 43), residual and
evaluation against brute force, closed forms and manufactured solutions."""
import math

import numpy as np
import pytest

from oracle import taps_oracle as O
from paper_2503_13933_gb300 import workloads as W


def _poisson(n, D=3, p=2, s=2):
    return O.problem_from_description(W.poisson_sin(n, D=D, p=p, s=s))


def test_dense_and_block_banded_solves_agree():
    P = O.problem_from_description(W.heat_transient(n_space=9, n_t=8, D_space=2))
    U = O.init_factors(P, 3, "random", 5)
    for d in range(P.D):
        C, F = O.coefficients(P, U, d)
        Xd = O.solve_dense(O.reduced_matrix_dense(P, d, C), F)
        Xb = O.solve_block_banded(P, d, C, F)
        assert np.max(np.abs(Xd - Xb)) < 1e-10 * np.max(np.abs(Xd))


def test_fast_diagonalisation_agrees_with_dense():
    """The fast-diagonalisation route of Sec. 2.6 solves the same reduced system:
    Poisson dims (K, M pencil), the k dim (W alone), transient spatial dims (K, M with
    nonsymmetric coefficients from the time factor)."""
    for desc in (W.poisson_k(n_space=10, n_k=7, seed=2010),
                 W.heat_transient(n_space=9, n_t=8, D_space=2, seed=3010)):
        P = O.problem_from_description(desc)
        U = O.init_factors(P, 3, "random", 12)
        used = 0
        for d in range(P.D):
            C, F = O.coefficients(P, U, d)
            if O.fast_diag_pencil(P, d, C) is None:
                continue
            used += 1
            Xd = O.solve_dense(O.reduced_matrix_dense(P, d, C), F)
            Xf = O.solve_fast_diag(P, d, C, F)
            assert np.max(np.abs(Xd - Xf)) < 1e-10 * np.max(np.abs(Xd))
        assert used >= 2


def test_mode_side_diagonalisation_agrees_with_dense():
    """Diagonalisation on the mode side (the Sylvester form of Sec. 2.6, M x M
    generalised eigenproblem + banded n_d x n_d solves) solves the same reduced system
    as the dense Kronecker-assembled solve: transient time dims (G, M with symmetric
    coefficients), also with convection faces on the space dims, and Poisson space dims
    (K, M)."""
    cases = (W.heat_transient(n_space=9, n_t=8, D_space=2, seed=3010),
             W.heat_transient(n_space=8, n_t=7, D_space=2, h_conv=2.0, seed=3011),
             W.poisson_sin(9, D=3),
             W.poisson_k(n_space=8, n_k=6, seed=2012))
    used = {}
    for k, desc in enumerate(cases):
        P = O.problem_from_description(desc)
        U = O.init_factors(P, 4, "random", 21 + k)
        for d in range(P.D):
            C, F = O.coefficients(P, U, d)
            pair = O.mode_diag_pair(P, d, C)
            if pair is None:
                continue
            used[(k, d)] = pair
            Xd = O.solve_dense(O.reduced_matrix_dense(P, d, C), F)
            Xm = O.solve_mode_diag(P, d, C, F)
            assert np.max(np.abs(Xd - Xm)) < 1e-10 * np.max(np.abs(Xd)), (k, d)
    # every time dim (ops G, M: mass-like X = M) and every Poisson dim was covered
    assert used[(0, 2)] == (O.OP_M, O.OP_G) and used[(1, 2)] == (O.OP_M, O.OP_G)
    assert all((2, d) in used for d in range(3))
    # the parameter dim (W alone): one operator, W = L^-T
    assert used[(3, 3)] == (O.OP_W, None) and all((3, d) in used for d in range(3))
    # space dims of a transient problem carry the nonsymmetric time Gram: not eligible
    assert (0, 0) not in used and (1, 0) not in used


def test_mode_side_poisson_sweeps_follow_block_elimination():
    """The space-parameter problem swept on the mode side in every dim gives the
    factors of block elimination."""
    P = O.problem_from_description(W.poisson_k(n_space=9, n_k=7, seed=2013))
    U0 = O.init_factors(P, 4, "random", 6)
    Ua, Ub = [u.copy() for u in U0], [u.copy() for u in U0]
    for _ in range(2):
        Ua, ca = O.sweep(P, Ua, solver="modediag")
        Ub, cb = O.sweep(P, Ub, solver="banded")
    for a, b in zip(Ua, Ub):
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)


def test_mode_side_sweeps_follow_block_elimination():
    """Three sweeps with the mode-side solver where it applies give the factors of
    three block-elimination sweeps from the same start."""
    P = O.problem_from_description(W.heat_transient(n_space=8, n_t=9, D_space=2, seed=3012))
    U0 = O.init_factors(P, 3, "random", 4)
    Ua, Ub = [u.copy() for u in U0], [u.copy() for u in U0]
    for _ in range(3):
        Ua, ca = O.sweep(P, Ua, solver="modediag")
        Ub, cb = O.sweep(P, Ub, solver="banded")
    for a, b in zip(Ua, Ub):
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)
    assert abs(ca - cb) <= 1e-8 * max(cb, 1.0)


def test_reduced_system_is_the_galerkin_condition():
    """The reduced solve makes the dim-d Galerkin residual of the FULL system vanish:
    for every test direction dU (x) prod_{e!=d} U_e[:,m], <dU-test, F - A u> = 0."""
    P = O.problem_from_description(W.poisson_k(n_space=7, n_k=5, seed=2003))
    U = O.init_factors(P, 2, "random", 9)
    A = O.full_operator(P)
    F = O.full_rhs(P)
    for d in range(P.D):
        C, Fd = O.coefficients(P, U, d)
        U[d] = O.solve_dense(O.reduced_matrix_dense(P, d, C), Fd)
        r = F - A @ O.cp_full(U)
        for m in range(2):
            for i in range(P.nfree[d]):
                vecs = [U[e][:, m] if e != d else np.eye(P.nfree[d])[i] for e in range(P.D)]
                test = O.kron_all([v.reshape(-1, 1) for v in vecs]).reshape(-1)
                assert abs(test @ r) < 1e-10 * np.linalg.norm(F) * np.linalg.norm(test)


def test_gram_identity_terms_match_explicit():
    """||F||^2, F^T A u and ||A u||^2 of the Gram identity equal the explicit
    full-grid values (the residual is their combination)."""
    P = O.problem_from_description(W.heat_transient(n_space=8, n_t=6, D_space=2, h_conv=2.0))
    U = O.init_factors(P, 3, "random", 2)
    rho, nF2, fau, au2 = O.residual(P, U)
    A = O.full_operator(P)
    F = O.full_rhs(P)
    u = O.cp_full(U)
    assert abs(nF2 - F @ F) < 1e-12 * (F @ F)
    assert abs(fau - F @ (A @ u)) < 1e-12 * abs(F @ (A @ u))
    Au = A @ u
    assert abs(au2 - Au @ Au) < 1e-12 * (Au @ Au)
    assert abs(rho - O.residual_explicit(P, U)) < 1e-7


def test_exact_rank_recovered_2d():
    """D=2 with 6 free nodes per dim: CP rank <= 6, so M=6 reaches the full Galerkin
    solution (the u^{C-HiDeNN} of Eq. 44).  The source is a sum of 6 random
    separable nodal terms so that the discrete solution has full rank 6 (with the
    smooth sine source it is numerically rank-1 and M=6 would be degenerate)."""
    desc = W.poisson_sin(8, D=2)
    rng = np.random.default_rng(11)
    desc["sources"] = [(1.0, [("nodal", rng.uniform(-1, 1, 8)) for _ in range(2)])
                       for _ in range(6)]
    P = O.problem_from_description(desc)
    u_full = O.solve_full(P)
    U = O.init_factors(P, 6, "random", 3)
    for _ in range(200):
        U, ch = O.sweep(P, U)
        if ch < 1e-13:
            break
    err = np.linalg.norm(O.cp_full(U) - u_full) / np.linalg.norm(u_full)
    assert err < 1e-10


def test_brute_force_16cubed_and_galerkin_optimality():
    """16^3 Poisson: TAPS error vs the full Kronecker FE solve shrinks with M; the
    full solve has the smaller energy error against the exact solution (first
    inequality of Eq. 44)."""
    P = _poisson(16)
    A = O.full_operator(P)
    u_full = O.solve_full(P)
    errs = []
    U = None
    for M in (1, 2, 3):
        r = O.solve(P, M0=1, M_max=M, als_tol=1e-12, res_tol=0.0, max_sweeps=300,
                    init="zero")
        U = r.U
        errs.append(np.linalg.norm(O.cp_full(U) - u_full) / np.linalg.norm(u_full))
    assert errs[-1] <= errs[0] + 1e-14
    assert errs[-1] < 1e-6
    # energy error against the nodal interpolant of the exact solution is not the
    # energy error against u_ex; use Galerkin orthogonality instead:
    # ||u_ex - u_taps||_A^2 = ||u_ex - u_full||_A^2 + ||u_full - u_taps||_A^2 in the
    # discrete space, so ||u_full - u_taps||_A^2 >= 0 with equality only at u_full.
    e = O.cp_full(U) - u_full
    assert e @ A @ e >= 0.0


def test_solution_of_the_parameter_problem_factorises():
    """-div(k grad u) = f(x): A = A_3D (x) W_k and F = F_3D (x) q_k, so the full
    solution is u_3D (x) W_k^{-1} q_k, and W_k^{-1} q_k interpolates 1/k."""
    desc = W.poisson_k(n_space=7, n_k=9, seed=2001)
    P = O.problem_from_description(desc)
    u = O.solve_full(P).reshape(5, 5, 5, 9)
    Wk = P.ops[3][O.OP_W]
    qk = P.sources[0][1][3]
    phi = np.linalg.solve(Wk, qk)
    k = P.dims[3].x
    assert np.max(np.abs(phi * k - 1.0)) < 0.08     # 9 nodes: coarse near k = 1
    u3 = u[..., 0] / phi[0]
    assert np.max(np.abs(u - u3[..., None] * phi[None, None, None, :])) < 1e-12 * np.max(np.abs(u))


def test_time_derivative_reproduces_linear_growth():
    """du/dt = 1, u(0) = 0: Galerkin in time (Eq. 25 time term) with zero-IC node
    dropped gives u = t exactly (t is in the C-HiDeNN space for p >= 1)."""
    dm = O.Dim(n=11, lo=0.0, hi=2.0, dirichlet_lo=True, dirichlet_hi=False)
    G = O.assemble_free(dm)[O.OP_G]
    q = O.project_source(dm, "const", (1.0,))
    u = np.linalg.solve(G, q)
    assert np.max(np.abs(u - dm.x[1:])) < 1e-11


def test_robin_face():
    """-u'' = 0, u(0) = 0, u'(1) + h u(1) = g: weak form K u + h B_hi u = g e_n; the
    exact solution u = g x / (1 + h) is linear, so the discrete one is exact."""
    dm = O.Dim(n=12, lo=0.0, hi=1.0, dirichlet_lo=True, dirichlet_hi=False)
    A = O.assemble_free(dm)
    h, g = 3.0, 2.0
    rhs = np.zeros(dm.n - 1)
    rhs[-1] = g
    u = np.linalg.solve(A[O.OP_K] + h * A[O.OP_BHI], rhs)
    assert np.max(np.abs(u - g * dm.x[1:] / (1 + h))) < 1e-11


@pytest.mark.parametrize("p", [1, 2])
def test_manufactured_convergence_rate(p):
    """-Laplace u = 3 pi^2 prod sin(pi x): relative L2 error (Eq. 48) against the exact
    solution converges at least at rate p+1 under h-refinement (the patch space holds
    the cubic-spline part besides the degree-p polynomials, so the observed rate may
    exceed p+1, as larger patches do in the paper's Sec. 3.2 study)."""
    errs, hs = [], []
    for n in (9, 17, 33):
        P = _poisson(n, p=p)
        r = O.solve(P, M0=1, M_max=2, als_tol=1e-12, res_tol=0.0, max_sweeps=200, init="zero")
        U = r.U
        full = [O.to_all_nodes(P.dims[d], U[d]) for d in range(3)]
        Mf = [O.assemble_full(P.dims[d])[O.OP_M] for d in range(3)]
        qf = [O.project_source(O.Dim(n=n, lo=0, hi=1, p=p, dirichlet_lo=False,
                                     dirichlet_hi=False), "sin", (math.pi, 0.0))
              for _ in range(3)]
        uu = np.ones((U[0].shape[1],) * 2)
        ue = np.ones(U[0].shape[1])
        for d in range(3):
            uu *= full[d].T @ Mf[d] @ full[d]
            ue *= full[d].T @ qf[d]
        e2 = uu.sum() - 2 * ue.sum() + 0.125
        errs.append(math.sqrt(max(e2, 0.0) / 0.125))
        hs.append(1.0 / (n - 1))
    slope = math.log(errs[-2] / errs[-1]) / math.log(hs[-2] / hs[-1])
    assert p + 1 - 0.3 <= slope <= p + 2.5, (errs, slope)


def test_eval_points_at_nodes_equals_grid():
    """Kronecker delta: evaluating at node coordinates returns the factor products."""
    P = _poisson(9, D=3)
    U = O.init_factors(P, 2, "random", 4)
    idx = [[0, 3, 8], [1, 4], [2, 7]]
    g = O.eval_grid(P, U, idx)
    pts = [[P.dims[0].x[i], P.dims[1].x[j], P.dims[2].x[k]]
           for i in idx[0] for j in idx[1] for k in idx[2]]
    v = O.eval_points(P, U, pts).reshape(g.shape)
    assert np.max(np.abs(g - v)) < 1e-13
    assert np.all(g[0] == 0.0)      # x = 0 is a Dirichlet node


def test_als_residual_vanishes_at_a_fixed_point():
    P = _poisson(10)
    U = O.init_factors(P, 2, "random", 8)
    for _ in range(300):
        U, ch = O.sweep(P, U)
        if ch < 1e-14:
            break
    assert O.als_residual(P, U) < 1e-10
    U2 = [u.copy() for u in U]
    U2[0][0, 0] += 1e-3
    assert O.als_residual(P, U2) > 1e-6


def test_splitmix64_published_vector():
    """SplitMix64 reference output: state 0 -> first output 0xE220A8397B1DCDAF
    (Vigna's reference implementation seeded with 0)."""
    assert O.splitmix64(0) == 0xE220A8397B1DCDAF
    v = [O.uniform_pm1(7, 1, i, 2) for i in range(1000)]
    assert -1.0 <= min(v) and max(v) < 1.0 and abs(np.mean(v)) < 0.1


def test_dirichlet_lifting_equals_direct_boundary_solve():
    """Non-homogeneous Dirichlet data by lifting: 2D Poisson on 6 x 6 nodes with random
    separable boundary data (a rank-2 field at all nodes) and a source.  With M = 4
    modes TAPS holds every grid function, so the lifted TAPS solution u_D + w must equal
    the full-grid solve with the boundary values imposed directly
    (A_II u_I = F_I - A_IB u_B)."""
    rng = np.random.default_rng(12)
    desc = W.poisson_sin(6, D=2)
    desc["sources"] = [(1.0, [("nodal", rng.uniform(-1, 1, 6)), ("nodal", rng.uniform(-1, 1, 6))])
                       for _ in range(2)]
    vecs = [rng.uniform(-1, 1, (6, 2)), rng.uniform(-1, 1, (6, 2))]
    wts = np.array([0.7, -1.3])
    lifted = dict(desc, sources=list(desc["sources"]) + O.dirichlet_lifting_sources(desc, (vecs, wts)))
    P = O.problem_from_description(lifted)
    r = O.solve(P, M0=4, M_max=4, als_tol=1e-14, res_tol=-1.0, max_sweeps=60, init="random", seed=3)
    w = O.cp_full(r.U).reshape(4, 4)
    uD = np.einsum("im,jm,m->ij", vecs[0], vecs[1], wts)            # all nodes
    u_taps = w + uD[1:-1, 1:-1]
    # direct: all nodes, boundary rows replaced by the boundary values
    dm = O.dim_from_description(desc["dims"][0])
    mats = O.assemble_full(dm)
    K, Mm = mats[O.OP_K], mats[O.OP_M]
    A = np.kron(K, Mm) + np.kron(Mm, K)
    F = np.zeros(36)
    for beta, fl in desc["sources"]:
        F += beta * np.kron(Mm @ fl[0][1], Mm @ fl[1][1])
    inner = np.array([(i % 6 not in (0, 5)) and (i // 6 not in (0, 5)) for i in range(36)])
    ub = uD.reshape(-1)
    uI = np.linalg.solve(A[np.ix_(inner, inner)], F[inner] - A[np.ix_(inner, ~inner)] @ ub[~inner])
    assert np.max(np.abs(u_taps.reshape(-1) - uI)) < 1e-9 * np.max(np.abs(uI))


def test_product_lifting_helper_matches_oracle_reading():
    """The library's lifting helper builds the same source terms (coefficients, operator
    names, all-node vectors) as the oracle's reading of the lifted weak form."""
    from paper_2503_13933_gb300 import boundary as B
    rng = np.random.default_rng(5)
    desc = W.heat_transient(n_space=9, n_t=7, D_space=2, h_conv=1.0)
    vecs = [rng.uniform(-1, 1, (dm["n"], 2)) for dm in desc["dims"]]
    wts = np.array([0.4, -2.0])
    a = B.lifting_sources(desc, vecs, wts)
    b = O.dirichlet_lifting_sources(desc, (vecs, wts))
    assert len(a) == len(b) == 2 * len(desc["terms"])
    for (ba, fa), (bb, fb) in zip(a, b):
        assert ba == bb
        for (ka, (oa, va)), (kb, (ob, vb)) in zip(fa, fb):
            assert ka == kb == "opvecfull" and oa == ob
            assert np.array_equal(va, vb)
    with pytest.raises(ValueError):
        B.lifting_sources(desc, [v[1:-1] for v in vecs], wts)   # free nodes only: rejected


def test_greedy_stops_on_stagnation(monkeypatch):
    """The greedy schedule's stop on stagnation (res_stall): with the residual at the end
    of the mode counts 1, 2, 3, ... forced to 0.5, 0.3, 0.2995, 0.299, 0.1, ... growth
    stops after the second mode count in a row that improved it by less than 1% (M = 4),
    and M_step appends that many columns per growth step."""
    desc = W.poisson_sin(14, D=2)
    rng = np.random.default_rng(3)
    desc["sources"] = [(1.0, [("nodal", rng.uniform(-1, 1, 14)) for _ in range(2)]) for _ in range(10)]
    P = O.problem_from_description(desc)
    seq = iter([0.5, 0.3, 0.2995, 0.299, 0.1, 0.05])
    monkeypatch.setattr(O, "residual", lambda prob, U: (next(seq), 0.0, 0.0, 0.0))
    r = O.solve(P, M0=1, M_max=8, als_tol=1.0, res_tol=0.0, max_sweeps=1, init="random", seed=2,
                res_stall=0.01)
    assert [h[0] for h in r.history] == [1, 2, 3, 4] and not r.converged
    seq = iter([0.5, 0.3, 0.2995, 0.299, 0.1, 0.05])
    r = O.solve(P, M0=1, M_max=8, als_tol=1.0, res_tol=0.0, max_sweeps=1, init="random", seed=2,
                res_stall=0.01, M_step=3)
    assert [h[0] for h in r.history] == [1, 4, 7, 8]
    assert r.U[0].shape[1] == 8
