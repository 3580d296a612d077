"""Pins of the oracle's relative L2 error against an exact solution (Sec. 3) and of
the eight-dimensional space-parameter-time problem of Sec. 3.2 (exact solution
known in closed form)."""
import math

import numpy as np
import pytest

from oracle import taps_oracle as O
from paper_2503_13933_gb300 import workloads as W


def _interp_at(dim, V, xs):
    """C-HiDeNN interpolants of the columns of V (all nodes) at points xs, point by
    point through the shape functions (Eq. 13)."""
    x = dim.x
    out = np.zeros((len(xs), V.shape[1]))
    for i, xp in enumerate(xs):
        e = O.locate(x, xp)
        ids, N, _ = O.shape_functions(x, dim.s, dim.a, dim.p, e, xp)
        out[i] = np.asarray(N) @ V[np.array(ids)]
    return out


def _tensor_rule(dim):
    gp, gw = O.gauss_legendre(dim.n_quad)
    x = dim.x
    xs = np.concatenate([x[e] + gp * (x[e + 1] - x[e]) for e in range(dim.n - 1)])
    ws = np.concatenate([gw * (x[e + 1] - x[e]) for e in range(dim.n - 1)])
    return xs, ws


def test_relative_l2_error_matches_brute_force_tensor_sum():
    """3D, random CP field (M = 3, weights), exact solution sin(2 y + 0.3) times a
    coupled pair 1 - exp(-3 x z): the Gram expansion equals the direct sum of
    (u - u_ex)^2 over the tensor quadrature grid, the field evaluated point by point."""
    rng = np.random.default_rng(3)
    dims = [O.Dim(n=6, lo=0.0, hi=1.0, s=1, p=1, n_quad=4), O.Dim(n=7, lo=-1.0, hi=0.5, s=2, p=2, n_quad=4),
            O.Dim(n=5, lo=0.5, hi=2.0, s=1, p=1, n_quad=4)]
    V = [rng.uniform(-1, 1, (d.n, 3)) for d in dims]
    c = np.array([0.5, -1.2, 2.0])
    sep = [None, ("sin", (2.0, 0.3)), None]
    fn = lambda a, b: 1.0 - np.exp(-3.0 * a * b)
    got = O.relative_l2_error(dims, V, c, sep, (0, 2), fn)
    rules = [_tensor_rule(d) for d in dims]
    F = [_interp_at(d, v, r[0]) for d, v, r in zip(dims, V, rules)]
    u = np.einsum("am,bm,cm,m->abc", F[0], F[1], F[2], c)
    xa, xb, xc = (r[0] for r in rules)
    ex = np.sin(2.0 * xb + 0.3)[None, :, None] * fn(xa[:, None, None], xc[None, None, :])
    w = np.einsum("a,b,c->abc", *(r[1] for r in rules))
    ref = math.sqrt(np.sum(w * (u - ex) ** 2) / np.sum(w * ex ** 2))
    assert abs(got - ref) <= 1e-9 * ref


def test_relative_l2_error_zero_for_reproduced_polynomials():
    """C-HiDeNN reproduces polynomials up to order p: the nodal values of the exact
    solution 1 + 2x - x^2 times the pair a*b (p = 2 and p = 1 dims) give error ~ 0, to
    the sqrt(eps) floor of the expansion; half the field gives exactly 1/2."""
    dims = [O.Dim(n=9, lo=0.0, hi=1.0, s=2, p=2), O.Dim(n=8, lo=1.0, hi=2.0, s=2, p=2),
            O.Dim(n=7, lo=0.0, hi=0.3, s=1, p=1)]
    V = [(1.0 + 2.0 * dims[0].x - dims[0].x ** 2)[:, None], dims[1].x[:, None], dims[2].x[:, None]]
    err = O.relative_l2_error(dims, V, [1.0], [("poly", (1.0, 2.0, -1.0)), None, None], (1, 2),
                              lambda a, b: a * b)
    assert err < 1e-6
    err_half = O.relative_l2_error(dims, V, [0.5], [("poly", (1.0, 2.0, -1.0)), None, None], (1, 2),
                                   lambda a, b: a * b)
    assert abs(err_half - 0.5) < 1e-9


def test_spt_lifting_matches_exact_solution_on_the_boundary():
    """The lifting of the Sec. 3.2 problem equals u_ex's nodal values on every spatial
    boundary node and vanishes at the interior nodes (checked on a 5^8 grid)."""
    n = 5
    desc, (vecs, wts), ex = W.spt_manufactured(n)
    full = np.einsum("am,bm,cm,dm,em,fm,gm,hm,m->abcdefgh", *vecs, wts)
    X = [np.linspace(dm["lo"], dm["hi"], n) for dm in desc["dims"]]
    g = np.exp(-25.0 * X[0] ** 2)[:, None] * np.exp(-25.0 * X[1] ** 2)[None, :]
    E = W.spt_exact_pair(X[3][:, None], X[7][None, :])
    uex = np.einsum("ab,c,dh,e,f,g->abcdefgh", g, np.ones(n), E, X[4], X[5], X[6])
    bnd = np.zeros((n, n, n), dtype=bool)
    bnd[[0, -1], :, :] = bnd[:, [0, -1], :] = bnd[:, :, [0, -1]] = True
    scale = np.max(np.abs(uex))
    assert np.max(np.abs(full[bnd] - uex[bnd])) < 1e-10 * scale
    assert np.max(np.abs(full[~bnd])) < 1e-12 * scale


def test_spt_oracle_converges_to_the_exact_solution():
    """Sec. 3.2, s = p = 2, M = 12: the lifted TAPS solution's relative L2 error against
    u_ex falls with refinement at the rate of a p = 2 method (order >= 2.5 in h
    between 10 and 14 nodes per dim) and is below 1e-2 at 14 nodes."""
    errs = []
    for n in (10, 14):
        desc, lift, ex = W.spt_manufactured(n)
        P = O.problem_from_description(dict(desc, sources=list(desc["sources"])
                                            + O.dirichlet_lifting_sources(desc, lift)))
        r = O.solve(P, M0=12, M_max=12, als_tol=1e-8, res_tol=-1.0, max_sweeps=40, init="random", seed=3)
        V, c = O.lifted_field_factors(P.dims, r.U, lift)
        errs.append(O.relative_l2_error(P.dims, V, c, ex["sep"], ex["pair"], W.spt_exact_pair))
    rate = math.log(errs[0] / errs[1]) / math.log(13 / 9)
    assert errs[1] < 1e-2 and rate > 2.5, (errs, rate)


def test_st_source_is_the_exact_solutions_residual():
    """The Sec. 3.1 source as built (the reading f = du_ex/dt - Laplace u_ex): its
    nodal (x, t) SVD factors reproduce f at nodes, and f matches central differences of
    u_ex at interior points to the differences' own error."""
    desc, _, _ = W.st_manufactured(40)
    x, y, t = (np.linspace(dm["lo"], dm["hi"], dm["n"]) for dm in desc["dims"])
    rng = np.random.default_rng(2)
    h = 1e-4
    for _ in range(5):
        i, j, k = rng.integers(5, 35), rng.integers(5, 35), rng.integers(5, 35)
        f = 0.0
        for beta, fac in desc["sources"]:
            vy = fac[1][1][j] if fac[1][0] == "nodal" else math.exp(-y[j] ** 2)
            f += beta * fac[0][1][i] * vy * fac[2][1][k]
        u = lambda a, b, c: W.st_exact(np.array([[a, b, c]]))[0]
        ut = (u(x[i], y[j], t[k] + h) - u(x[i], y[j], t[k] - h)) / (2 * h)
        lap = ((u(x[i] + h, y[j], t[k]) - 2 * u(x[i], y[j], t[k]) + u(x[i] - h, y[j], t[k]))
               + (u(x[i], y[j] + h, t[k]) - 2 * u(x[i], y[j], t[k]) + u(x[i], y[j] - h, t[k]))) / h ** 2
        scale = abs(ut) + abs(lap) + 1e-3
        assert abs(f - (ut - lap)) < 1e-4 * scale, (f, ut - lap)


def test_st_oracle_converges_to_the_exact_solution():
    """Sec. 3.1 on a shortened window (x in [0, 10], y in [-4, 4], t in [0, 0.02]),
    s = p = 1, modes 1..8 greedily: the lifted solution's error against u_ex falls at
    order >= 1.6 in h from 24 to 48 nodes per dim (p + 1 = 2) and is below 5e-3."""
    rng_ = dict(x=(0.0, 10.0), y=(-4.0, 4.0), t=(0.0, 0.02))
    errs = []
    for n in (24, 48):
        desc, lift, ex = W.st_manufactured(n, s=1, p=1, ranges=rng_)
        P = O.problem_from_description(dict(desc, sources=list(desc["sources"])
                                            + O.dirichlet_lifting_sources(desc, lift)))
        r = O.solve(P, M0=1, M_max=8, als_tol=1e-3, res_tol=-1.0, max_sweeps=5, init="random", seed=3)
        V, c = O.lifted_field_factors(P.dims, r.U, lift)
        errs.append(O.relative_l2_error(P.dims, V, c, ex["sep"], ex["pair"], W.st_exact_pair))
    rate = math.log(errs[0] / errs[1]) / math.log(47 / 23)
    assert errs[1] < 5e-3 and rate > 1.6, (errs, rate)


def test_relative_l2_error_separable_exact_matches_brute_force():
    """No coupled pair: exact solution sin(3x) (x) poly, random CP field; the Gram
    expansion equals the direct tensor sum point by point."""
    rng = np.random.default_rng(11)
    dims = [O.Dim(n=8, lo=0.0, hi=1.0, s=2, p=2, n_quad=4), O.Dim(n=6, lo=-1.0, hi=1.0, s=1, p=1, n_quad=4)]
    V = [rng.uniform(-1, 1, (d.n, 2)) for d in dims]
    c = np.array([1.5, -0.4])
    sep = [("sin", (3.0, 0.0)), ("poly", (0.5, -1.0, 0.25))]
    got = O.relative_l2_error(dims, V, c, sep)
    rules = [_tensor_rule(d) for d in dims]
    F = [_interp_at(d, v, r[0]) for d, v, r in zip(dims, V, rules)]
    u = np.einsum("am,bm,m->ab", F[0], F[1], c)
    xa, xb = rules[0][0], rules[1][0]
    ex = np.sin(3.0 * xa)[:, None] * (0.5 - xb + 0.25 * xb ** 2)[None, :]
    w = np.outer(rules[0][1], rules[1][1])
    ref = math.sqrt(np.sum(w * (u - ex) ** 2) / np.sum(w * ex ** 2))
    assert abs(got - ref) <= 1e-9 * ref
