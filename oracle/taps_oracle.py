"""Plain, slow, FP64 CPU oracle of the TAPS hot path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.
The product path (the CUDA library and its Python binding) never calls it, and it
calls nothing of the product: it shares no code, table or constant generator with
the GPU kernels.  Inputs reach it as plain numbers built by
``paper_2503_13933_gb300.workloads`` (seeded generators holding none of the
method's arithmetic).

Every function states the passage of the paper (Guo et al., "Tensor-decomposition-
based A Priori Surrogate (TAPS) modeling for ultra large-scale simulations") that it
follows.  Where the paper is silent, the reading taken is stated beside the code:

* C-HiDeNN patch function (Eq. 1, Sec. 2.1): the formula is deferred to the
  C-HiDeNN literature.  Reading: radial point interpolation with polynomial
  reproduction on the nodal patch A_s^i = {j : |j-i| <= s} (truncated at the ends),
  cubic-spline kernel with support a*h, monomials centred at x_i and scaled by h.
* Quadrature (Table 1, "Gaussian integration"): 6-point Gauss-Legendre per element.
* Solver convergence (Sec. 2.6, "relative change of all solution matrices"):
  max_d ||U_d^new - U_d^old||_F / ||U_d^new||_F after column normalisation.
* Residual (not defined by the paper): rho = ||F - A u||_2 / ||F||_2 on the free
  nodal unknowns, evaluated with the Gram identity term by term.

Pins (tests/test_oracle_*.py): Kronecker delta, partition of unity, polynomial
reproduction, dilation independence, textbook special cases (linear hats,
quadratic Lagrange), closed-form matrix integrals, dense-vs-block-banded solve,
explicit full-grid residual, brute-force Kronecker FE solve, manufactured-solution
convergence rates, the rank-1-in-k property of the space-parameter problem.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Operator kinds of the 1D matrices (Sec. 2.5, Eqs. 31-34): the index of each kind
# is part of the problem description both implementations read.
OP_K, OP_M, OP_G, OP_W, OP_BLO, OP_BHI = 0, 1, 2, 3, 4, 5
OP_NAMES = {OP_K: "K", OP_M: "M", OP_G: "G", OP_W: "W", OP_BLO: "Blo", OP_BHI: "Bhi"}


# ---------------------------------------------------------------------------------
# Shape functions (Sec. 2.1, Eq. 1; Kronecker delta Eq. 3)
# ---------------------------------------------------------------------------------
def cubic_spline(z):
    """Cubic-spline window phi(z), z >= 0 (the kernel of the patch function)."""
    z = abs(z)
    if z <= 0.5:
        return 2.0 / 3.0 - 4.0 * z * z + 4.0 * z ** 3
    if z <= 1.0:
        return 4.0 / 3.0 - 4.0 * z + 4.0 * z * z - 4.0 / 3.0 * z ** 3
    return 0.0


def cubic_spline_dz(z):
    """d phi / dz for z >= 0."""
    z = abs(z)
    if z <= 0.5:
        return -8.0 * z + 12.0 * z * z
    if z <= 1.0:
        return -4.0 + 8.0 * z - 4.0 * z * z
    return 0.0


def patch(i, n, s):
    """Nodal patch A_s^i: nodes within s elements of node i, truncated at the ends."""
    return list(range(max(0, i - s), min(n - 1, i + s) + 1))


def patch_matrix(x, i, s, a, p, h):
    """Moment matrix G_i = [[R, P], [P^T, 0]] of node i's convolution patch (Eq. 1).

    R_jk = phi(|x_j - x_k| / (a h)), P_jq = ((x_j - x_i)/h)^q, q = 0..p.
    """
    nodes = patch(i, len(x), s)
    na = len(nodes)
    if na < p + 1:
        raise ValueError(f"patch of node {i} has {na} < p+1 = {p + 1} nodes")
    G = np.zeros((na + p + 1, na + p + 1))
    for r, j in enumerate(nodes):
        for c, k in enumerate(nodes):
            G[r, c] = cubic_spline(abs(x[j] - x[k]) / (a * h))
        for q in range(p + 1):
            G[r, na + q] = ((x[j] - x[i]) / h) ** q
            G[na + q, r] = G[r, na + q]
    return nodes, G


def patch_function(x, i, s, a, p, h, xe):
    """Patch function W^i_j(xe) and its derivative for every j in A_s^i (Eq. 1).

    W^i(xe) = [phi(xe)^T, P(xe)^T] G_i^{-1}, first |A_s^i| entries: the RBF +
    polynomial interpolant of unit nodal data, evaluated at xe.
    """
    nodes, G = patch_matrix(x, i, s, a, p, h)
    na = len(nodes)
    row = np.zeros(na + p + 1)
    drow = np.zeros(na + p + 1)
    for r, j in enumerate(nodes):
        d = xe - x[j]
        row[r] = cubic_spline(abs(d) / (a * h))
        drow[r] = cubic_spline_dz(abs(d) / (a * h)) * (math.copysign(1.0, d) if d != 0 else 0.0) / (a * h)
    for q in range(p + 1):
        t = (xe - x[i]) / h
        row[na + q] = t ** q
        drow[na + q] = q * t ** (q - 1) / h if q > 0 else 0.0
    # W solves G W = row (G symmetric) -> W = G^{-1} row.
    W = np.linalg.solve(G, row)[:na]
    dW = np.linalg.solve(G, drow)[:na]
    return nodes, W, dW


def shape_functions(x, s, a, p, e, xe):
    """C-HiDeNN shape functions on element e at xe (Eq. 1, Eq. 31/32).

    N~_k(xe) = N_e(xe) W^e_k(xe) + N_{e+1}(xe) W^{e+1}_k(xe), k in e-s .. e+1+s,
    with N_e, N_{e+1} the linear finite-element hats of the element's two nodes.
    Returns (global node ids, N~, dN~/dx).
    """
    n = len(x)
    h = x[e + 1] - x[e]
    lo = max(0, e - s)
    hi = min(n - 1, e + 1 + s)
    ids = list(range(lo, hi + 1))
    N = np.zeros(len(ids))
    B = np.zeros(len(ids))
    hat = [(x[e + 1] - xe) / h, (xe - x[e]) / h]
    dhat = [-1.0 / h, 1.0 / h]
    for c, i in enumerate((e, e + 1)):
        nodes, W, dW = patch_function(x, i, s, a, p, h, xe)
        for r, j in enumerate(nodes):
            k = j - lo
            N[k] += hat[c] * W[r]
            B[k] += dhat[c] * W[r] + hat[c] * dW[r]
    return ids, N, B


def locate(x, xe):
    """Element containing xe on the node grid x (last element for the right end)."""
    e = int(np.searchsorted(x, xe, side="right")) - 1
    return min(max(e, 0), len(x) - 2)


def gauss_legendre(nq):
    """Gauss-Legendre points/weights on [0, 1] (Table 1: Gaussian integration)."""
    t, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (t + 1.0), 0.5 * w


# ---------------------------------------------------------------------------------
# 1D matrices (Sec. 2.5, Eqs. 31-35: stiffness, mass, time derivative, weighted mass)
# ---------------------------------------------------------------------------------
@dataclass
class Dim:
    """One independent dimension: uniform nodes, C-HiDeNN hyperparameters, BCs."""
    n: int
    lo: float
    hi: float
    s: int = 2
    a: float = 20.0
    p: int = 2
    n_quad: int = 6
    dirichlet_lo: bool = True
    dirichlet_hi: bool = True
    weight_poly: tuple = (0.0, 0.0, 0.0, 0.0)

    @property
    def x(self):
        return np.linspace(self.lo, self.hi, self.n)

    @property
    def free(self):
        f = list(range(self.n))
        if self.dirichlet_hi:
            f = f[:-1]
        if self.dirichlet_lo:
            f = f[1:]
        return np.array(f, dtype=int)


def poly_eval(c, xv):
    return sum(cj * xv ** j for j, cj in enumerate(c))


def shape_tables(dim: Dim):
    """Per element, per Gauss point: node ids, N~, B~, weight*|J| (Eq. 1, Table 1)."""
    x = dim.x
    gp, gw = gauss_legendre(dim.n_quad)
    tab = []
    for e in range(dim.n - 1):
        h = x[e + 1] - x[e]
        pts = []
        for t, w in zip(gp, gw):
            xe = x[e] + t * h
            ids, N, B = shape_functions(x, dim.s, dim.a, dim.p, e, xe)
            pts.append((xe, w * h, ids, N, B))
        tab.append(pts)
    return tab


def assemble_full(dim: Dim, tab=None):
    """Dense 1D matrices over ALL nodes (Eqs. 33-35, Sec. 2.5).

    K_ij = int B~_i B~_j, M_ij = int N~_i N~_j, G_ij = int N~_i B~_j (test i, trial
    j: the time-derivative term of Eq. 25), W_ij = int N~_i w(x) N~_j (weighted mass,
    the k-weighted parametric term of Eq. 33), B_lo/B_hi = boundary point masses
    (convection on a face, Eq. 21 / Eq. 25 boundary integral, by the Kronecker delta).
    """
    if tab is None:
        tab = shape_tables(dim)
    n = dim.n
    mats = {k: np.zeros((n, n)) for k in (OP_K, OP_M, OP_G, OP_W)}
    for pts in tab:
        for xe, wj, ids, N, B in pts:
            ids = np.array(ids)
            wv = poly_eval(dim.weight_poly, xe)
            mats[OP_K][np.ix_(ids, ids)] += wj * np.outer(B, B)
            mats[OP_M][np.ix_(ids, ids)] += wj * np.outer(N, N)
            mats[OP_G][np.ix_(ids, ids)] += wj * np.outer(N, B)
            mats[OP_W][np.ix_(ids, ids)] += wj * wv * np.outer(N, N)
    mats[OP_BLO] = np.zeros((n, n))
    mats[OP_BLO][0, 0] = 1.0
    mats[OP_BHI] = np.zeros((n, n))
    mats[OP_BHI][n - 1, n - 1] = 1.0
    return mats


def assemble_free(dim: Dim, tab=None):
    """1D matrices restricted to the free nodes (Dirichlet / zero-IC nodes dropped,
    Eq. 5: the Kronecker delta makes the constrained nodal value the BC value)."""
    full = assemble_full(dim, tab)
    f = dim.free
    return {k: v[np.ix_(f, f)].copy() for k, v in full.items()}


# Source factors: g(x) on one dimension, given as plain data.
def source_factor_values(kind, par, xv):
    if kind == "const":
        return np.full_like(np.asarray(xv, dtype=float), par[0])
    if kind == "sin":          # sin(w x + phase)
        return np.sin(par[0] * xv + par[1])
    if kind == "gauss":        # exp(-(x-c)^2 / (2 sigma^2))
        return np.exp(-((xv - par[0]) ** 2) / (2.0 * par[1] ** 2))
    if kind == "poly":
        return poly_eval(par, xv)
    raise ValueError(kind)


def project_source(dim: Dim, kind, par, nodal=None, tab=None):
    """q_i = int N~_i g(x) dx on the free nodes (forcing term of Eq. 30).

    kind 'nodal': g is the C-HiDeNN interpolant of nodal values -> q = M_full g.
    """
    n = dim.n
    if kind == "nodal":
        full = assemble_full(dim, tab)[OP_M] @ np.asarray(nodal, dtype=float)
        return full[dim.free]
    if tab is None:
        tab = shape_tables(dim)
    q = np.zeros(n)
    for pts in tab:
        for xe, wj, ids, N, B in pts:
            q[np.array(ids)] += wj * source_factor_values(kind, par, xe) * N
    return q[dim.free]


# ---------------------------------------------------------------------------------
# Problem in separated form (Sec. 2.4-2.5, Eqs. 25, 33-36, 41-42)
# ---------------------------------------------------------------------------------
@dataclass
class Problem:
    """A = sum_t alpha_t (x)_d Op[t][d];  F = sum_r beta_r (x)_d q[r][d]."""
    dims: list
    ops: list              # ops[d] = dict kind -> (n_free x n_free) matrix
    terms: list            # list of (alpha, [op kind per dim])
    sources: list          # list of (beta, [q vector per dim])

    @property
    def D(self):
        return len(self.dims)

    @property
    def nfree(self):
        return [len(dm.free) for dm in self.dims]


OP_WEIGHTED = 16   # op code OP_WEIGHTED + j: weighted operator j of the dim


def assemble_weighted(dim: Dim, base, w, tab=None):
    """A weighted 1D operator over all nodes, the weight a C-HiDeNN field
    w(x) = sum_k N~_k(x) w_k of nodal values w (App. A: rho c_p(u) and k(u) kept in the
    separated form, so each of their modes weights the 1D integrals of Eqs. 33-35):
        'K': int w B~_i B~_j,   'M': int w N~_i N~_j,
        'G': int N~_i d/dt (w N~_j) = int N~_i (w' N~_j + w B~_j)   (the time derivative
             of the product rho c_p(u) u in the weak form of App. A).
    Element-by-element Gauss sums, as assemble_full."""
    if tab is None:
        tab = shape_tables(dim)
    w = np.asarray(w, dtype=float)
    A = np.zeros((dim.n, dim.n))
    for pts in tab:
        for xe, wj, ids, N, B in pts:
            ids = np.array(ids)
            N, B = np.asarray(N), np.asarray(B)
            wv, dwv = N @ w[ids], B @ w[ids]
            if base == "K":
                A[np.ix_(ids, ids)] += wj * wv * np.outer(B, B)
            elif base == "M":
                A[np.ix_(ids, ids)] += wj * wv * np.outer(N, N)
            elif base == "G":
                A[np.ix_(ids, ids)] += wj * (dwv * np.outer(N, N) + wv * np.outer(N, B))
            else:
                raise ValueError(base)
    return A


def build_problem(dims, terms, sources, weighted=None):
    """dims: list of Dim; terms: list of (alpha, [op per dim]); sources: list of
    (beta, [(kind, par) or ('nodal', values) per dim]); kinds 'opvec' (free-node vector)
    and 'opvecfull' (all-node vector) give par = (operator name, vector).
    weighted[d]: list of (base 'K'|'M'|'G', all-node weights), op OP_WEIGHTED + j."""
    tabs = [shape_tables(dm) for dm in dims]
    ops = [assemble_free(dm, tb) for dm, tb in zip(dims, tabs)]
    full_mass = {}     # all-node mass matrix of a dim, assembled once for its nodal sources
    for d, wl in enumerate(weighted or []):
        for j, (base, w) in enumerate(wl or []):
            f = dims[d].free
            ops[d][OP_WEIGHTED + j] = assemble_weighted(dims[d], base, w, tabs[d])[np.ix_(f, f)]
    src = []
    for beta, facs in sources:
        qs = []
        for d, (dm, tb, (kind, par)) in enumerate(zip(dims, tabs, facs)):
            if kind == "nodal":
                # q = M_full g restricted to the free nodes (project_source's 'nodal' case)
                if d not in full_mass:
                    full_mass[d] = assemble_full(dm, tb)[OP_M]
                qs.append((full_mass[d] @ np.asarray(par, dtype=float))[dm.free])
            elif kind == "opvec":
                # the projection of a field already in the C-HiDeNN space: q = Op v
                qs.append(ops[d][OP_BY_NAME[par[0]]] @ np.asarray(par[1], dtype=float))
            elif kind == "opvecfull":
                # a field given at all nodes, constrained ones included (the lifting of
                # non-homogeneous Dirichlet data): q = (Op_all v)[free nodes]
                full = assemble_full(dm, tb)[OP_BY_NAME[par[0]]] @ np.asarray(par[1], dtype=float)
                qs.append(full[dm.free])
            else:
                qs.append(project_source(dm, kind, par, tab=tb))
        src.append((float(beta), qs))
    return Problem(dims=list(dims), ops=ops, terms=[(float(a), list(o)) for a, o in terms],
                   sources=src)


# ---------------------------------------------------------------------------------
# Subspace iteration (Algorithm 1, Sec. 2.6; Eq. 43)
# ---------------------------------------------------------------------------------
def gram(U, Op):
    """Gamma = U^T Op U (M x M): the coefficient integrals of Eq. 34."""
    return U.T @ (Op @ U)


def coefficients(prob: Problem, U, d):
    """C_op for dim d (Eq. 34/35: Hadamard product over the other dimensions, summed
    over the operator terms that share dim d's matrix) and the RHS F_d (Eq. 41's Q)."""
    M = U[0].shape[1]
    C = {}
    for alpha, opk in prob.terms:
        prod = np.full((M, M), alpha)
        for e in range(prob.D):
            if e != d:
                prod = prod * gram(U[e], prob.ops[e][opk[e]])
        C[opk[d]] = C.get(opk[d], np.zeros((M, M))) + prod
    F = np.zeros((prob.nfree[d], M))
    for beta, qs in prob.sources:
        c = np.full(M, beta)
        for e in range(prob.D):
            if e != d:
                c = c * (U[e].T @ qs[e])
        F += np.outer(qs[d], c)
    return C, F


def reduced_matrix_dense(prob: Problem, d, C):
    """The reduced operator of Eq. 36-40 reshaped with I = (node, mode), node-major:
    A[(i,m),(j,n)] = sum_op Op[i,j] C_op[m,n] = sum_op kron(Op, C_op)."""
    A = None
    for op, Cop in C.items():
        term = np.kron(prob.ops[d][op], Cop)
        A = term if A is None else A + term
    return A


def solve_dense(A, F):
    """Dense LU with partial pivoting (library solve) of the reduced system."""
    n, M = F.shape
    return np.linalg.solve(A, F.reshape(-1)).reshape(n, M)


def band_halfwidth(prob: Problem, d):
    hb = 0
    for op in prob.ops[d].values():
        nz = np.nonzero(op)
        if len(nz[0]):
            hb = max(hb, int(np.max(np.abs(nz[0] - nz[1]))))
    return hb


def solve_block_banded(prob: Problem, d, C, F):
    """Block Gaussian elimination without pivoting of the node-major block-banded
    reduced system (Eq. 43): block (i,j) = sum_op Op[i,j] C_op, half-bandwidth hb.

    Forward: for each block row k, D_k = A_kk; W_kj = D_k^{-1} A_kj, z_k = D_k^{-1} F_k;
    A_ij -= A_ik W_kj, F_i -= A_ik z_k for i, j in k+1..k+hb.
    Backward: x_k = z_k - sum_j W_kj x_j.
    """
    n, M = F.shape
    hb = band_halfwidth(prob, d)
    blocks = {}
    for i in range(n):
        for j in range(max(0, i - hb), min(n, i + hb + 1)):
            B = np.zeros((M, M))
            for op, Cop in C.items():
                B += prob.ops[d][op][i, j] * Cop
            blocks[(i, j)] = B
    rhs = [F[i].copy() for i in range(n)]
    W = {}
    z = [None] * n
    for k in range(n):
        Dk = blocks[(k, k)]
        js = range(k + 1, min(n, k + hb + 1))
        for j in js:
            W[(k, j)] = np.linalg.solve(Dk, blocks[(k, j)])
        z[k] = np.linalg.solve(Dk, rhs[k])
        for i in js:
            Lik = blocks[(i, k)]
            for j in js:
                blocks[(i, j)] = blocks[(i, j)] - Lik @ W[(k, j)]
            rhs[i] = rhs[i] - Lik @ z[k]
    X = np.zeros((n, M))
    for k in range(n - 1, -1, -1):
        xk = z[k].copy()
        for j in range(k + 1, min(n, k + hb + 1)):
            xk -= W[(k, j)] @ X[j]
        X[k] = xk
    return X


def fast_diag_pencil(prob: Problem, d, C):
    """Operator pencil of dim d for fast diagonalisation (Sec. 2.6): returns (opA, opB)
    with opB mass-like (M or W) and both symmetric, opA None for a single operator;
    None if the dim's operators do not form such a pencil."""
    ops = list(C.keys())
    if any(o == OP_G for o in ops) or not 1 <= len(ops) <= 2:
        return None
    if len(ops) == 1:
        return None, ops[0]
    mass = [o for o in ops if o in (OP_M, OP_W)]
    if not mass:
        return None
    b = mass[0]
    return [o for o in ops if o != b][0], b


def solve_fast_diag(prob: Problem, d, C, F):
    """Fast diagonalisation of sum_op Op U C_op^T = F (Sec. 2.6): with the generalised
    eigenpairs A phi = mu B phi (Phi^T B Phi = I; library symmetric-definite eigensolver),
    U = Phi Y and (mu_i C_A + C_B) Y[i]^T = (Phi^T F)[i]^T for each i."""
    import scipy.linalg
    opA, opB = fast_diag_pencil(prob, d, C)
    B = prob.ops[d][opB]
    if opA is None:
        Phi = np.linalg.inv(np.linalg.cholesky(B)).T
        mu = np.zeros(B.shape[0])
    else:
        mu, Phi = scipy.linalg.eigh(prob.ops[d][opA], B)
    G = Phi.T @ F
    M = F.shape[1]
    Y = np.zeros_like(G)
    for i in range(G.shape[0]):
        T = C[opB] + (mu[i] * C[opA] if opA is not None else 0.0)
        Y[i] = np.linalg.solve(T, G[i])
    return Phi @ Y


def mode_diag_pair(prob: Problem, d, C):
    """Operator pair of dim d for diagonalisation on the mode side (Sec. 2.6: the
    Sylvester form of the reduced system, cost M^3 + M^2 n_d + the banded solves):
    returns (opX, opY), opX mass-like when the pair has one, if dim d has one or two
    operators (opY None for one) and every other dim's operators are symmetric (then
    every Gram of the other dims, and so every C_op of dim d, is symmetric); None
    otherwise."""
    ops = list(C.keys())
    if not 1 <= len(ops) <= 2:
        return None
    for alpha, opk in prob.terms:
        for e in range(prob.D):
            if e != d and opk[e] == OP_G:
                return None
    if len(ops) == 1:
        return ops[0], None
    mass = [o for o in ops if o in (OP_M, OP_W)]
    x = mass[0] if mass else ops[0]
    return x, [o for o in ops if o != x][0]


def solve_mode_diag(prob: Problem, d, C, F):
    """Diagonalisation on the mode side of Op_X U C_X + Op_Y U C_Y = F (C symmetric):
    with the generalised eigenpairs C_Y w = lam C_X w (W^T C_X W = I, W^T C_Y W =
    diag(lam); library symmetric-definite eigensolver), U = Z W^T where each column
    solves the banded n_d x n_d system (Op_X + lam_j Op_Y) z_j = (F W)_j (library
    dense solve)."""
    import scipy.linalg
    opX, opY = mode_diag_pair(prob, d, C)
    CX = 0.5 * (C[opX] + C[opX].T)
    if opY is None:    # Op_X U C_X = F: W = L^-T (C_X = L L^T), lam = 0
        Wm = np.linalg.inv(np.linalg.cholesky(CX)).T
        lam = np.zeros(CX.shape[0])
        OpY = np.zeros_like(prob.ops[d][opX])
    else:
        CY = 0.5 * (C[opY] + C[opY].T)
        lam, Wm = scipy.linalg.eigh(CY, CX)
        OpY = prob.ops[d][opY]
    G = F @ Wm
    Z = np.zeros_like(G)
    for j in range(G.shape[1]):
        Z[:, j] = np.linalg.solve(prob.ops[d][opX] + lam[j] * OpY, G[:, j])
    return Z @ Wm.T


def normalise_columns(Ud):
    """Unit 2-norm columns; sign makes the largest-magnitude entry positive.
    (Scale normalisation is not stated by the paper; the next dimension's solve
    absorbs it, so the represented field is unchanged after a full sweep.)"""
    Ud = Ud.copy()
    for m in range(Ud.shape[1]):
        col = Ud[:, m]
        nrm = math.sqrt(float(np.dot(col, col)))
        if nrm == 0.0:
            continue
        k = int(np.argmax(np.abs(col)))
        sgn = 1.0 if col[k] >= 0 else -1.0
        Ud[:, m] = col / (sgn * nrm)
    return Ud


def sweep(prob: Problem, U, solver="banded"):
    """One subspace-iteration sweep (Algorithm 1 inner loop, Eq. 43).

    For d = 1..D in order, with the other factors at their latest values
    (Gauss-Seidel), solve sum_op Op_d U_d C_op^T = F_d for U_d; normalise U_d for
    d < D.  Returns the new factors and max_d ||dU_d||_F / ||U_d||_F.

    solver: "banded" (block elimination), "dense", "fastdiag" (node-side pencil where
    the dim's operators allow, else mode-side for two operators with symmetric
    coefficients, else banded) or "modediag" (mode-side for one or two operators with
    symmetric coefficients, else node-side, else banded).
    """
    U = [u.copy() for u in U]
    change = 0.0
    for d in range(prob.D):
        C, F = coefficients(prob, U, d)
        if solver == "dense":
            Ud = solve_dense(reduced_matrix_dense(prob, d, C), F)
        elif solver == "modediag" and mode_diag_pair(prob, d, C) is not None:
            Ud = solve_mode_diag(prob, d, C, F)
        elif solver in ("fastdiag", "modediag") and fast_diag_pencil(prob, d, C) is not None:
            Ud = solve_fast_diag(prob, d, C, F)
        elif solver == "fastdiag" and len(C) == 2 and mode_diag_pair(prob, d, C) is not None:
            Ud = solve_mode_diag(prob, d, C, F)
        else:
            Ud = solve_block_banded(prob, d, C, F)
        if d < prob.D - 1:
            Ud = normalise_columns(Ud)
        nrm = np.linalg.norm(Ud)
        dif = np.linalg.norm(Ud - U[d])
        change = max(change, dif / nrm if nrm > 0 else math.inf)
        U[d] = Ud
    return U, change


# ---------------------------------------------------------------------------------
# Residual (Gram identity) and explicit full-grid forms for tiny grids
# ---------------------------------------------------------------------------------
def residual(prob: Problem, U):
    """rho = ||F - A u|| / ||F||, u = sum_m (x)_d U_d[:,m] (Eq. 7), expanded as
    ||F||^2 - 2 F^T A u + ||A u||^2, each a sum of products of 1D inner products."""
    D = prob.D
    M = U[0].shape[1]
    R = len(prob.terms)
    Rf = len(prob.sources)
    FF = np.ones((Rf, Rf))
    FA = np.ones((Rf, R, M))
    AA = np.ones((R, M, R, M))
    for d in range(D):
        Q = np.stack([qs[d] for _, qs in prob.sources], axis=1)        # n x Rf
        Y = np.stack([prob.ops[d][opk[d]] @ U[d] for _, opk in prob.terms], axis=0)  # R x n x M
        FF *= Q.T @ Q
        FA *= np.einsum("ir,tim->rtm", Q, Y)
        AA *= np.einsum("tim,sin->tmsn", Y, Y)
    a = np.array([t[0] for t in prob.terms])
    b = np.array([s[0] for s in prob.sources])
    nF2 = float(b @ FF @ b)
    fau = float(np.einsum("r,t,rtm->", b, a, FA))
    au2 = float(np.einsum("t,s,tmsn->", a, a, AA))
    r2 = nF2 - 2.0 * fau + au2
    return math.sqrt(max(r2, 0.0) / nF2), nF2, fau, au2


def kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def full_operator(prob: Problem):
    """Explicit A = sum_t alpha_t (x)_d Op_{t,d} on the free grid (tiny cases only)."""
    A = None
    for alpha, opk in prob.terms:
        T = alpha * kron_all([prob.ops[d][opk[d]] for d in range(prob.D)])
        A = T if A is None else A + T
    return A


def full_rhs(prob: Problem):
    F = None
    for beta, qs in prob.sources:
        T = beta * kron_all([q.reshape(-1, 1) for q in qs]).reshape(-1)
        F = T if F is None else F + T
    return F


def cp_full(U):
    """Full tensor of u = sum_m prod_d U_d[:, m] (Eq. 7), C order (last dim fastest)."""
    M = U[0].shape[1]
    out = 0.0
    for m in range(M):
        out = out + kron_all([u[:, m].reshape(-1, 1) for u in U]).reshape(-1)
    return out


def residual_explicit(prob: Problem, U):
    A = full_operator(prob)
    F = full_rhs(prob)
    u = cp_full(U)
    return float(np.linalg.norm(F - A @ u) / np.linalg.norm(F))


def solve_full(prob: Problem):
    """Brute force: the full (not decomposed) C-HiDeNN Galerkin solution on the
    tensor grid (the u^{C-HiDeNN} of Eq. 44)."""
    return np.linalg.solve(full_operator(prob), full_rhs(prob))


# ---------------------------------------------------------------------------------
# Initialisation: counter-based uniform draws (SplitMix64, Steele-Lea-Flood 2014)
# ---------------------------------------------------------------------------------
_MASK = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 output function applied to state x (published constants)."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def uniform_pm1(seed, d, i, m):
    """U(-1,1) draw keyed on (seed, dim, row, mode): the counter packs
    seed (24 bits) | dim (8) | mode (12) | row (20); top 53 bits of the output."""
    ctr = ((seed & 0xFFFFFF) << 40) | ((d & 0xFF) << 32) | ((m & 0xFFF) << 20) | (i & 0xFFFFF)
    z = splitmix64(ctr)
    return 2.0 * ((z >> 11) * (1.0 / 9007199254740992.0)) - 1.0


def init_column(prob: Problem, d, m, how, seed=0):
    """Initial column m of U_d (Algorithm 1 starts from random values).
    'random': U(-1,1) counter-based draws; 'zero': zero in the first dimension,
    ones elsewhere (the first solve of a sweep is dimension 1)."""
    n = prob.nfree[d]
    if how == "random":
        return np.array([uniform_pm1(seed, d, i, m) for i in range(n)])
    if how == "zero":
        return np.zeros(n) if d == 0 else np.ones(n)
    raise ValueError(how)


def init_factors(prob: Problem, M, how="random", seed=0):
    return [np.stack([init_column(prob, d, m, how, seed) for m in range(M)], axis=1)
            for d in range(prob.D)]


# ---------------------------------------------------------------------------------
# Greedy mode schedule + sweeps to tolerance (Algorithm 1 with growing M)
# ---------------------------------------------------------------------------------
@dataclass
class SolveResult:
    U: list
    history: list = field(default_factory=list)   # (M, sweep, change, rho)
    rho: float = math.inf
    converged: bool = False


def solve(prob: Problem, M0=1, M_max=8, als_tol=1e-10, res_tol=1e-6, max_sweeps=200,
          init="zero", seed=0, solver="banded", U0=None, res_stall=0.0, M_step=1):
    """Run Algorithm 1 for M = M0..M_max modes, adding M_step columns per step.
    At each M, sweep until the factor change <= als_tol or rho <= res_tol (or
    max_sweeps); stop growing M once rho <= res_tol, or (res_stall > 0) once rho at the
    end of a mode count has been above (1 - res_stall) times its value at the end of the
    previous mode count for two mode counts in a row (the greedy schedule's stop on
    stagnation, reading O6)."""
    if U0 is not None:
        U = [u.copy() for u in U0]
    else:
        U = init_factors(prob, M0, init, seed)
    res = SolveResult(U=U)
    M = U[0].shape[1]
    rho_prev, stalls = math.inf, 0
    while True:
        for it in range(max_sweeps):
            U, change = sweep(prob, U, solver)
            rho = residual(prob, U)[0]
            res.history.append((M, it, change, rho))
            if rho <= res_tol or change <= als_tol:
                break
        res.U, res.rho = U, rho
        if rho <= res_tol:
            res.converged = True
            return res
        if M >= M_max:
            return res
        if res_stall > 0.0:
            stalls = stalls + 1 if not rho <= (1.0 - res_stall) * rho_prev else 0
            rho_prev = rho
            if stalls >= 2:
                return res
        Mn = min(M_max, M + max(1, M_step))
        U = [np.concatenate([U[d]] + [init_column(prob, d, m, init, seed)[:, None] for m in range(M, Mn)], axis=1)
             for d in range(prob.D)]
        M = Mn


# ---------------------------------------------------------------------------------
# Evaluation (Eq. 13)
# ---------------------------------------------------------------------------------
def to_all_nodes(dim: Dim, Ud):
    """Scatter free-node factor rows into all nodes (constrained nodes carry 0)."""
    full = np.zeros((dim.n, Ud.shape[1]))
    full[dim.free] = Ud
    return full


def eval_grid(prob: Problem, U, idx):
    """u on the tensor grid of node indices idx[d] (all-node numbering), Eq. 7/13
    at nodes (Kronecker delta: nodal value = factor entry).  C order output."""
    rows = [to_all_nodes(prob.dims[d], U[d])[np.asarray(idx[d])] for d in range(prob.D)]
    out = 0.0
    for m in range(U[0].shape[1]):
        out = out + kron_all([r[:, m].reshape(-1, 1) for r in rows]).reshape(-1)
    return np.asarray(out).reshape([len(i) for i in idx])


def eval_points(prob: Problem, U, pts):
    """u^TD(x) = sum_m prod_d sum_I N~_I(x_d) U_d[I, m] at arbitrary points (Eq. 13)."""
    pts = np.atleast_2d(np.asarray(pts, dtype=float))
    out = np.zeros(len(pts))
    full = [to_all_nodes(prob.dims[d], U[d]) for d in range(prob.D)]
    for p_i, xp in enumerate(pts):
        prod = np.ones(U[0].shape[1])
        for d, dm in enumerate(prob.dims):
            x = dm.x
            e = locate(x, xp[d])
            ids, N, _ = shape_functions(x, dm.s, dm.a, dm.p, e, xp[d])
            prod = prod * (N @ full[d][ids])
        out[p_i] = prod.sum()
    return out


# ---------------------------------------------------------------------------------
# Problem descriptions (plain data from the seeded workload generators)
# ---------------------------------------------------------------------------------
OP_BY_NAME = {"K": OP_K, "M": OP_M, "G": OP_G, "W": OP_W, "Blo": OP_BLO, "Bhi": OP_BHI}


def dim_from_description(dm):
    return Dim(n=dm["n"], lo=dm["lo"], hi=dm["hi"], s=dm["s"], a=dm["a"], p=dm["p"],
               n_quad=dm["n_quad"], dirichlet_lo=dm["dirichlet_lo"],
               dirichlet_hi=dm["dirichlet_hi"], weight_poly=tuple(dm["weight_poly"]))


def op_code(name):
    """'K', 'M', ... or 'w<j>' (the dim's weighted operator j)."""
    return OP_WEIGHTED + int(name[1:]) if name.startswith("w") else OP_BY_NAME[name]


def problem_from_description(desc):
    dims = [dim_from_description(dm) for dm in desc["dims"]]
    terms = [(a, [op_code(o) for o in ops]) for a, ops in desc["terms"]]
    return build_problem(dims, terms, desc["sources"], desc.get("weighted"))


def als_residual(prob: Problem, U):
    """Relative residual of the coupled subspace system (Eq. 42): for every d,
    r_d = K^[d](U_{e!=d}) U_d - Q^[d](U_{e!=d}) = sum_op Op_d U_d C_op^T - F_d,
    evaluated with all factors at their current values; returns max_d ||r_d||/||F_d||."""
    worst = 0.0
    for d in range(prob.D):
        C, F = coefficients(prob, U, d)
        r = -F.copy()
        for op, Cop in C.items():
            r += prob.ops[d][op] @ U[d] @ Cop.T
        nf = np.linalg.norm(F)
        worst = max(worst, np.linalg.norm(r) / nf if nf > 0 else math.inf)
    return worst


# ---------------------------------------------------------------------------------
# Warm-start network (not in the paper: the learned initialisation that replaces the
# random start of Algorithm 1).  FP64, written from the chain rule.
# Layout of the flat parameter vector: per layer W [out][in] row-major, then b [out].
# ---------------------------------------------------------------------------------
def mlp_unpack(p, dims):
    out, off = [], 0
    for i, o in zip(dims[:-1], dims[1:]):
        W = p[off:off + i * o].reshape(o, i)
        off += i * o
        b = p[off:off + o]
        off += o
        out.append((W, b))
    return out


def mlp_forward(p, dims, X):
    """Activations A_0 = X, A_{l+1} = tanh(A_l W_l^T + b_l) (linear last layer)."""
    acts = [np.asarray(X, dtype=float)]
    layers = mlp_unpack(np.asarray(p, dtype=float), dims)
    for l, (W, b) in enumerate(layers):
        Z = acts[-1] @ W.T + b
        acts.append(np.tanh(Z) if l < len(layers) - 1 else Z)
    return acts


def mlp_loss_grad(p, dims, X, T):
    """Mean squared error over all outputs and its gradient (same flat layout)."""
    layers = mlp_unpack(np.asarray(p, dtype=float), dims)
    acts = mlp_forward(p, dims, X)
    Y = acts[-1]
    n = Y.size
    loss = float(np.sum((Y - T) ** 2) / n)
    G = 2.0 * (Y - T) / n
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        A = acts[l]
        grads[l] = (G.T @ A, G.sum(axis=0))
        if l > 0:
            G = (G @ W) * (1.0 - A ** 2)
    flat = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return loss, flat


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma & Ba 2015) with bias-corrected moments; returns new p, m, v."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------------
# Time slabs (Sec. 2.4, Eq. 16; App. B Eq. 56): initial condition by lifting.
# ---------------------------------------------------------------------------------
def slab_end_state(U, time_dim, prev=None):
    """(spatial/parametric factors, weights) of u(., t_max): the time factors' last rows
    weight the modes; the previous slab's lifting modes are kept in front."""
    facs = [None if d == time_dim else np.array(u) for d, u in enumerate(U)]
    wts = np.array(U[time_dim][-1, :])
    if prev is not None:
        pf, pw = prev
        facs = [None if d == time_dim else np.concatenate([pf[d], facs[d]], axis=1)
                for d in range(len(U))]
        wts = np.concatenate([pw, wts])
    return facs, wts


def slab_next_description(desc, state, time_dim, t_shift):
    """Next slab: time window shifted; force += -alpha_t w_m (x)_d (Op_{t,d} U_d[:,m]) (x) M_t 1
    for each term without time derivative (d/dt of the constant lifting is zero)."""
    facs, wts = state
    nd = dict(desc)
    nd["dims"] = [dict(dm) for dm in desc["dims"]]
    nd["dims"][time_dim]["lo"] += t_shift
    nd["dims"][time_dim]["hi"] += t_shift
    extra = []
    for alpha, ops in desc["terms"]:
        if ops[time_dim] == "G":
            continue
        for m in range(len(wts)):
            extra.append((-alpha * wts[m],
                          [("const", (1.0,)) if d == time_dim else ("opvec", (ops[d], facs[d][:, m]))
                           for d in range(len(ops))]))
    nd["sources"] = list(desc["sources"]) + extra
    return nd


def slab_compress(desc, state, time_dim, U0, sweeps):
    """Mode compression of a slab end state (App. B): the L2 projection of
    u_end = sum_m w_m (x)_d U_d[:, m] onto the modes of U0 (fewer), i.e. the weighted
    residual equation (x)_d M_d u_F = (x)_d M_d u_end over the dims other than time,
    solved by Algorithm 1 sweeps (block elimination) from the given factors.  Returns
    the compressed state (weights 1: the normalisation puts the scale in the last dim)."""
    facs, wts = state
    keep = [d for d in range(len(desc["dims"])) if d != time_dim]
    cdesc = dict(name="compress", dims=[desc["dims"][d] for d in keep],
                 terms=[(1.0, ["M"] * len(keep))],
                 sources=[(float(wts[m]), [("opvec", ("M", facs[d][:, m])) for d in keep])
                          for m in range(len(wts))])
    P = problem_from_description(cdesc)
    U = [u.copy() for u in U0]
    for _ in range(sweeps):
        U, _ = sweep(P, U, solver="banded")
    out = [None] * len(desc["dims"])
    for j, d in enumerate(keep):
        out[d] = U[j]
    return out, np.ones(U[0].shape[1])


def dirichlet_lifting_sources(desc, lift):
    """Non-homogeneous Dirichlet data by lifting (Sec. 2.5 weak form with u = u_D + w,
    w = 0 on the constrained nodes): for a lifting u_D = sum_m w_m (x)_d v_{d,m} given at
    all nodes (only its values at constrained nodes matter for the final field), the
    problem for w gains, per operator term t and lifting mode m, the separable source
    -alpha_t w_m (x)_d (Op_{t,d} v_{d,m})[free nodes]."""
    vecs, wts = lift
    out = []
    for alpha, ops in desc["terms"]:
        for m in range(len(wts)):
            out.append((-float(alpha) * float(wts[m]),
                        [("opvecfull", (ops[d], np.asarray(vecs[d][:, m], dtype=float)))
                         for d in range(len(ops))]))
    return out


# ---------------------------------------------------------------------------------
# Accuracy against an exact solution (the relative L2 error of Sec. 3)
# ---------------------------------------------------------------------------------
def _quadrature_values(dim: Dim, V, tab=None):
    """Gauss points, weights and the C-HiDeNN interpolants of the columns of V (all
    nodes) at those points, over the whole dim (every element's rule)."""
    if tab is None:
        tab = shape_tables(dim)
    xs, ws, F = [], [], []
    for pts in tab:
        for xe, wj, ids, N, B in pts:
            xs.append(xe)
            ws.append(wj)
            F.append(np.asarray(N) @ V[np.array(ids)])
    return np.array(xs), np.array(ws), np.array(F)


def relative_l2_error(dims, V, c, sep, pair=None, pair_fn=None):
    """Relative L2 error (Sec. 3) of u = sum_m c_m prod_d (sum_i N~_i(x_d) V[d][i, m])
    against u_ex = prod_{d not in pair} sep[d](x_d) * pair_fn(x_a, x_b), (a, b) = pair,
    over the tensor domain, each 1D integral by the dims' own Gauss rules.  Through
    |u - u_ex|^2 = |u|^2 - 2 (u, u_ex) + |u_ex|^2, the first a Hadamard product of
    per-dim Gram matrices, so the computed error has an absolute floor near
    sqrt(eps) * |u_ex| (the rounding limit of the paper's S-P-T study).
    sep[d] is a source factor (kind, params) of source_factor_values."""
    D = len(dims)
    c = np.asarray(c, dtype=float)
    q = [_quadrature_values(dims[d], np.asarray(V[d], dtype=float)) for d in range(D)]
    pd = set(pair) if pair is not None else set()
    G = np.ones((len(c), len(c)))
    cross = np.ones(len(c))
    ex2 = 1.0
    for d in range(D):
        xs, ws, F = q[d]
        G *= F.T @ (ws[:, None] * F)
        if d in pd:
            continue
        g = source_factor_values(sep[d][0], sep[d][1], xs)
        cross *= F.T @ (ws * g)
        ex2 *= float(np.sum(ws * g * g))
    if pair is not None:
        (xa, wa, Fa), (xb, wb, Fb) = q[pair[0]], q[pair[1]]
        E = pair_fn(xa[:, None], xb[None, :]) * np.outer(wa, wb)
        cross *= np.einsum("am,ab,bm->m", Fa, E, Fb)
        ex2 *= float(np.sum(pair_fn(xa[:, None], xb[None, :]) ** 2 * np.outer(wa, wb)))
    err2 = float(c @ G @ c - 2.0 * c @ cross + ex2)
    return math.sqrt(max(err2, 0.0) / ex2)


def lifted_field_factors(dims, U, lift):
    """The CP factors (all nodes) and weights of u = u_D + w: the solved w (free-node
    factors, zero at the constrained nodes) and the lifting's modes."""
    vecs, wts = lift
    M = U[0].shape[1]
    V = [np.concatenate([to_all_nodes(dims[d], U[d]), np.asarray(vecs[d], dtype=float)], axis=1)
         for d in range(len(dims))]
    return V, np.concatenate([np.ones(M), np.asarray(wts, dtype=float)])


# ---------------------------------------------------------------------------------
# Nonlinear problems: global-local iteration (App. A, Algorithm 2)
# ---------------------------------------------------------------------------------
def cp_factors_all_nodes(dims, U):
    """The factors of u over all nodes (constrained nodes 0)."""
    return [to_all_nodes(dm, u) for dm, u in zip(dims, U)]


def nonlinear_global_description(desc, law, V):
    """The linear global stage of Algorithm 2 for rho c_p(u) du/dt-type problems on
    space dims 0..D-2 and time dim D-1: with rho c_p = m_c u + n_c and k = m_k u + n_k
    linear in u (Sec. 3.3), both are separated fields with the modes of the current u
    (all-node factors V) plus a constant mode, and the weak form of App. A,
        int du d/dt[c u] + int grad du . k grad u = int du f,
    becomes, per mode j of c (coefficient m_c, or n_c for the constant), the term
    (x)_{d<D-1} M[V_d,j] (x) G[V_t,j], and per mode j of k and space direction e the
    term K[V_e,j] in dim e, M[V_d,j] in the other space dims and M[V_t,j] in time
    (X[v] the operator weighted by the interpolant of v; the constant mode uses the
    unweighted K, M, G).  desc: the problem's dims and sources (its terms are
    replaced); law = (m_c, n_c, m_k, n_k)."""
    m_c, n_c, m_k, n_k = law
    D = len(desc["dims"])
    Ds = D - 1
    M = V[0].shape[1] if V is not None else 0
    weighted = [[] for _ in range(D)]
    names = [dict() for _ in range(D)]

    def wop(d, base, j):
        key = (base, j)
        if key not in names[d]:
            names[d][key] = f"w{len(weighted[d])}"
            weighted[d].append((base, np.asarray(V[d][:, j], dtype=float)))
        return names[d][key]

    terms = [(n_c, ["M"] * Ds + ["G"])]
    terms += [(n_k, ["K" if d == e else "M" for d in range(Ds)] + ["M"]) for e in range(Ds)]
    for j in range(M):
        if m_c != 0.0:
            terms.append((m_c, [wop(d, "M", j) for d in range(Ds)] + [wop(Ds, "G", j)]))
        if m_k != 0.0:
            for e in range(Ds):
                terms.append((m_k, [wop(d, "K" if d == e else "M", j) for d in range(Ds)]
                              + [wop(Ds, "M", j)]))
    return dict(desc, terms=terms, weighted=weighted)


def cp_change(U_new, U_old):
    """|u_new - u_old| / |u_new| in the Euclidean norm of the nodal tensors (the
    convergence check of Algorithm 2, App. A), by Gram products of the factors.

    Expanding |a|^2 + |b|^2 - 2 <a, b> cancels to ~sqrt(eps) relative, far above the
    changes a converging iteration reaches.  So the difference itself is written as a
    CP tensor whose terms are all small, by telescoping each mode's product
    (the shorter factor set padded with zero columns):
        prod_d a_d - prod_d b_d = sum_k (prod_{d<k} b_d) (a_k - b_k) (prod_{d>k} a_d),
    and its squared norm is the sum over pairs of those D*M terms of the products of
    their 1D inner products."""
    D = len(U_new)
    Mx = max(U_new[0].shape[1], U_old[0].shape[1])

    def pad(u):
        return np.concatenate([u, np.zeros((u.shape[0], Mx - u.shape[1]))], axis=1)

    A = [pad(u) for u in U_new]
    B = [pad(u) for u in U_old]
    terms = []     # per telescoped term (k, m): its factor in every dim
    for k in range(D):
        for m in range(Mx):
            terms.append([B[d][:, m] if d < k else (A[d][:, m] - B[d][:, m] if d == k else A[d][:, m])
                          for d in range(D)])
    T = len(terms)
    G = np.ones((T, T))
    for d in range(D):
        F = np.stack([t[d] for t in terms], axis=1)
        G *= F.T @ F
    GA = np.ones((U_new[0].shape[1],) * 2)
    for a in U_new:
        GA *= a.T @ a
    nn = float(np.sum(GA))
    return math.sqrt(max(float(np.sum(G)), 0.0) / nn) if nn > 0 else 0.0


def nonlinear_solve(desc, law, M, sweeps, max_iters=50, tol=1e-10, seed=0, solver="banded", U0=None):
    """Algorithm 2: start from u = 0 (rho c_p = n_c, k = n_k), then repeat the global
    stage (the linear problem of nonlinear_global_description, Algorithm 1 with M modes
    and `sweeps` subspace iterations from the previous factors; U0 or random factors the
    first time) and the local update of rho c_p(u), k(u) (here exact: the fields are linear in
    u, so the update is the new factors), until the relative change of u <= tol.
    Returns (factors, history of changes)."""
    dims = [dim_from_description(dm) for dm in desc["dims"]]
    U = [np.array(u, dtype=float) for u in U0] if U0 is not None else None
    V, hist = None, []
    for it in range(max_iters):
        P = problem_from_description(nonlinear_global_description(desc, law, V))
        if U is None:
            U = init_factors(P, M, "random", seed)
        U_old = [u.copy() for u in U]
        for _ in range(sweeps):
            U, _ = sweep(P, U, solver)
        ch = cp_change(U, U_old) if it > 0 else float("inf")
        hist.append(ch)
        V = cp_factors_all_nodes(dims, U)
        if ch <= tol:
            break
    return U, hist
