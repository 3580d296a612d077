"""Seeded synthetic workloads: problem descriptions as plain data.

This module holds no arithmetic of the method.  It only draws the numbers that
describe a problem (grid sizes, C-HiDeNN hyperparameters, operator terms, source
parameters), so that the CUDA path and the independent CPU oracle can be fed the
same input.  A description is a dict:

    dims    : list of {kind, n, lo, hi, s, a, p, n_quad, dirichlet_lo, dirichlet_hi,
                       weight_poly}
    terms   : list of (alpha, [operator name per dim])      A = sum_t alpha_t (x)_d Op
    sources : list of (beta, [(factor kind, params) per dim]) F = sum_r beta_r (x)_d q

Operator names: 'K' stiffness, 'M' mass, 'G' time derivative, 'W' weighted mass
(weight polynomial of the dim), 'Blo'/'Bhi' boundary point mass at the low/high end.
Source factor kinds: ('const', (c,)), ('sin', (w, phase)) = sin(w x + phase),
('gauss', (c, sigma)) = exp(-(x-c)^2/(2 sigma^2)), ('poly', (c0, c1, ...)),
('nodal', values over all nodes).
"""
from __future__ import annotations

import math

import numpy as np

SPACE, PARAM, TIME = 0, 1, 2


def dim(n, lo=0.0, hi=1.0, *, kind=SPACE, s=2, a=20.0, p=2, n_quad=6,
        dirichlet_lo=True, dirichlet_hi=True, weight_poly=(0.0, 0.0, 0.0, 0.0)):
    w = tuple(float(c) for c in weight_poly) + (0.0,) * (4 - len(weight_poly))
    return dict(kind=kind, n=int(n), lo=float(lo), hi=float(hi), s=int(s), a=float(a),
                p=int(p), n_quad=int(n_quad), dirichlet_lo=bool(dirichlet_lo),
                dirichlet_hi=bool(dirichlet_hi), weight_poly=w[:4])


def poisson_sin(n=64, D=3, s=2, a=20.0, p=2, n_quad=6):
    """-Laplace u = D pi^2 prod sin(pi x_d) on [0,1]^D, homogeneous Dirichlet.
    Exact solution prod sin(pi x_d).  (3D, 64 nodes/dim, s,a,p = 2,20,2 is the plain
    FP64 configuration; 16 nodes/dim is its brute-force case.)"""
    dims = [dim(n, 0.0, 1.0, s=s, a=a, p=p, n_quad=n_quad) for _ in range(D)]
    terms = [(1.0, ["K" if d == t else "M" for d in range(D)]) for t in range(D)]
    sources = [(D * math.pi ** 2, [("sin", (math.pi, 0.0))] * D)]
    return dict(name=f"poisson_sin_{D}d_n{n}", dims=dims, terms=terms, sources=sources)


def gaussian_sources(rng, n_gauss, n_space):
    """Seeded separable Gaussian bumps: amplitude U[0.5,2], width U[0.05,0.2],
    centre U[0.2,0.8] per spatial dim."""
    out = []
    for _ in range(n_gauss):
        A = rng.uniform(0.5, 2.0)
        sig = rng.uniform(0.05, 0.2)
        c = rng.uniform(0.2, 0.8, size=n_space)
        out.append((float(A), float(sig), [float(ci) for ci in c]))
    return out


def poisson_k(n_space=256, n_k=32, seed=2000, s=2, a=20.0, p=2, n_gauss=4, k_lo=1.0,
              k_hi=10.0):
    """Space-parameter problem: -div(k grad u) = f on [0,1]^3 with the conductivity k in
    [k_lo, k_hi] as a 4th independent dimension.  f = sum of n_gauss seeded separable
    Gaussians (independent of k)."""
    rng = np.random.default_rng(seed)
    g = gaussian_sources(rng, n_gauss, 3)
    dims = [dim(n_space, 0.0, 1.0, s=s, a=a, p=p) for _ in range(3)]
    dims.append(dim(n_k, k_lo, k_hi, kind=PARAM, s=s, a=a, p=p, dirichlet_lo=False,
                    dirichlet_hi=False, weight_poly=(0.0, 1.0)))
    terms = [(1.0, ["K" if d == t else "M" for d in range(3)] + ["W"]) for t in range(3)]
    sources = [(A, [("gauss", (c[d], sig)) for d in range(3)] + [("const", (1.0,))])
               for A, sig, c in g]
    return dict(name=f"poisson_k_{n_space}^3x{n_k}_seed{seed}", dims=dims, terms=terms,
                sources=sources, params=g)


def heat_transient(n_space=32, n_t=16, D_space=3, T=1.0, rho_cp=1.0, k=1.0, seed=3000,
                   n_gauss=2, s=2, a=20.0, p=2, h_conv=0.0):
    """rho c_p du/dt - k Laplace u = f on [0,1]^D_space x (0,T], zero initial condition,
    homogeneous Dirichlet on the low/high faces of every spatial dim; with h_conv > 0
    the high face of the last spatial dim is a convection (Robin) face instead.
    f = seeded separable Gaussians in space times a linear ramp in time."""
    rng = np.random.default_rng(seed)
    g = gaussian_sources(rng, n_gauss, D_space)
    dims = []
    for d in range(D_space):
        robin_hi = h_conv > 0 and d == D_space - 1
        dims.append(dim(n_space, 0.0, 1.0, s=s, a=a, p=p, dirichlet_hi=not robin_hi))
    dims.append(dim(n_t, 0.0, T, kind=TIME, s=s, a=a, p=p, dirichlet_lo=True,
                    dirichlet_hi=False))
    D = D_space + 1
    terms = [(rho_cp, ["M"] * D_space + ["G"])]
    for e in range(D_space):
        terms.append((k, ["K" if d == e else "M" for d in range(D_space)] + ["M"]))
    if h_conv > 0:
        terms.append((h_conv, ["M"] * (D_space - 1) + ["Bhi", "M"]))
    sources = [(A, [("gauss", (c[d], sig)) for d in range(D_space)] +
                [("poly", (0.0, 1.0 / T))]) for A, sig, c in g]
    return dict(name=f"heat_{D_space}d_n{n_space}_t{n_t}_seed{seed}", dims=dims,
                terms=terms, sources=sources, params=g)


def large_space_time_parameter(n_space=1536, n_t=256, n_p=16, n_r=16, seed=5000):
    """The large configuration's separated operator on a 3D space (n_space nodes per
    dim, widths 15.35 x 15.35 x 7.675 mm), one time slab (n_t nodes) and two parameter
    dims (n_p laser powers in [100, 400] W, n_r radii in [30, 80] um): diffusion and
    time-derivative terms, a Gaussian source in space, linear in P, constant in r and
    a ramp in time.  Used for the full-size reconstruction of a space slice at fixed
    (t, P, r)."""
    rng = np.random.default_rng(seed)
    Lx, Lz = 15.35e-3, 7.675e-3
    dims = [dim(n_space, 0.0, Lx), dim(n_space, 0.0, Lx), dim(n_space, 0.0, Lz),
            dim(n_t, 0.0, 2e-3, kind=TIME, dirichlet_lo=True, dirichlet_hi=False),
            dim(n_p, 100.0, 400.0, kind=PARAM, dirichlet_lo=False, dirichlet_hi=False),
            dim(n_r, 30e-6, 80e-6, kind=PARAM, dirichlet_lo=False, dirichlet_hi=False)]
    terms = [(1.0, ["M", "M", "M", "G", "M", "M"])]
    for e in range(3):
        terms.append((1.0, ["K" if d == e else "M" for d in range(3)] + ["M", "M", "M"]))
    c = rng.uniform(0.3, 0.7, size=3)
    sources = [(1.0, [("gauss", (c[0] * Lx, 0.05 * Lx)), ("gauss", (c[1] * Lx, 0.05 * Lx)),
                      ("gauss", (c[2] * Lz, 0.05 * Lz)), ("poly", (0.0, 1.0)),
                      ("poly", (0.0, 1.0)), ("const", (1.0,))])]
    return dict(name=f"large_{n_space}^3_t{n_t}_P{n_p}_r{n_r}", dims=dims, terms=terms, sources=sources)


def lpbf_slab(n_xy=512, n_z=128, n_t=128, n_par=16, slab=0, n_slabs=8, svd_tol=1e-10, s=2, a=20.0, p=2):
    """Single-track laser powder-bed fusion in space-parameter-time (Sec. 3.4 setting):
    rho c_p du/dt - div(k grad u) = f on x, y in [0, 2.555 mm] (n_xy nodes), z in
    [0, 0.635 mm] (n_z), one time slab of n_t nodes, and three parameter dims of n_par
    nodes: laser power P in [100, 400] W, spot radius r in [30, 80] um, conductivity k in
    [10, 30] W/m/K.  Ti-6Al-4V: rho = 4270 kg/m^3, c_p = 745 J/kg/K; absorptivity 0.25,
    penetration depth d_v = 50 um, scan speed 0.5 m/s; the track runs along x at
    y0 = W/2 from x = 0.3 mm to 2.25 mm over n_slabs slabs.  u = T - T0: zero initial
    condition, Dirichlet at the bottom face, free convection h = 14.73 W/m^2/K on the
    other five faces.

    The moving source (2 eta P / (pi r^2 d_v)) exp(-2((x - x0(t))^2 + (y - y0)^2) / r^2)
    1(z >= H - d_v) is separable in P, y (at fixed r) and z; in (x, t) it is not.  Its CP
    form is built as input data, the same for every solver: one group of terms per
    r node r_j (the C-HiDeNN shape functions are Kronecker deltas at the nodes), whose
    (x, t) part is the SVD of the nodal matrix exp(-2 (x_a - x0(t_b))^2 / r_j^2)
    truncated at svd_tol relative to its largest singular value."""
    Lxy, H = 2.555e-3, 0.635e-3
    rho_cp, h_conv, eta, d_v, V = 4270.0 * 745.0, 14.73, 0.25, 50e-6, 0.5
    x_start, x_end = 0.3e-3, 2.25e-3
    T_slab = (x_end - x_start) / V / n_slabs
    t0, t1 = slab * T_slab, (slab + 1) * T_slab
    free = dict(dirichlet_lo=False, dirichlet_hi=False)
    dims = [dim(n_xy, 0.0, Lxy, s=s, a=a, p=p, **free), dim(n_xy, 0.0, Lxy, s=s, a=a, p=p, **free),
            dim(n_z, 0.0, H, s=s, a=a, p=p, dirichlet_lo=True, dirichlet_hi=False),
            dim(n_t, t0, t1, kind=TIME, s=s, a=a, p=p, dirichlet_lo=True, dirichlet_hi=False),
            dim(n_par, 100.0, 400.0, kind=PARAM, s=s, a=a, p=p, **free),
            dim(n_par, 30e-6, 80e-6, kind=PARAM, s=s, a=a, p=p, **free),
            dim(n_par, 10.0, 30.0, kind=PARAM, s=s, a=a, p=p, weight_poly=(0.0, 1.0), **free)]
    terms = [(rho_cp, ["M", "M", "M", "G", "M", "M", "M"])]
    for e in range(3):
        terms.append((1.0, ["K" if d == e else "M" for d in range(3)] + ["M", "M", "M", "W"]))
    for face in (["Blo", "M", "M"], ["Bhi", "M", "M"], ["M", "Blo", "M"], ["M", "Bhi", "M"],
                 ["M", "M", "Bhi"]):
        terms.append((h_conv, face + ["M", "M", "M", "M"]))
    x = np.linspace(0.0, Lxy, n_xy)
    z = np.linspace(0.0, H, n_z)
    t = np.linspace(t0, t1, n_t)
    x0 = x_start + V * t
    y0 = 0.5 * Lxy
    z_ind = (z >= H - d_v).astype(float)
    r_nodes = np.linspace(30e-6, 80e-6, n_par)
    sources = []
    for j, rj in enumerate(r_nodes):
        E = np.exp(-2.0 * (x[:, None] - x0[None, :]) ** 2 / rj ** 2)
        Uu, sv, Vt = np.linalg.svd(E, full_matrices=False)
        rank = max(1, int(np.sum(sv > svd_tol * sv[0])))
        yj = np.exp(-2.0 * (x - y0) ** 2 / rj ** 2)
        ej = np.zeros(n_par)
        ej[j] = 2.0 * eta / (np.pi * rj ** 2 * d_v)
        for q in range(rank):
            sources.append((1.0, [("nodal", sv[q] * Uu[:, q]), ("nodal", yj), ("nodal", z_ind),
                                  ("nodal", Vt[q]), ("poly", (0.0, 1.0)), ("nodal", ej),
                                  ("const", (1.0,))]))
    return dict(name=f"lpbf_{n_xy}x{n_xy}x{n_z}_t{n_t}_par{n_par}_slab{slab}", dims=dims, terms=terms,
                sources=sources)


def lpbf_large(n_xy=1536, n_z=1536, n_t=256, n_par=16, h_xy=10e-6, h_z=5e-6, T_slab=0.2e-3, k=22.0,
               svd_tol=1e-8, x_start=None, y0=None, s=2, a=20.0, p=2):
    """The large space-parameter-time configuration: a moving Gaussian laser source over
    a 3D block of n_xy x n_xy x n_z nodes at h = (10, 10, 5) um (15.35 x 15.35 x 7.675 mm
    at full size, 3.6e9 spatial nodes), one time slab of n_t nodes over T_slab, and the
    laser power P in [100, 400] W and spot radius r in [30, 80] um as parameter dims of
    n_par nodes each; conductivity k fixed (22 W/m/K), Ti-6Al-4V rho c_p, absorptivity
    0.25, penetration depth d_v = 50 um, scan speed 0.5 m/s along x, the slab's path
    (V T_slab long: 0.1 mm at the default 0.2 ms) centred in the block, y0 = W/2.

    u = T - T0 with a zero initial condition and u = 0 on the bottom and the four side
    faces (the block is ~15 x the heat-affected zone wide: the far field stays at T0);
    the top face is insulated (convection at h = 14.73 W/m^2/K carries ~1e-6 of the
    laser's flux density and is left out).  The source, as in lpbf_slab, is one group
    of CP terms per r node (Kronecker delta in r): the SVD of the nodal (x, t) matrix
    exp(-2 (x - x0(t))^2 / r_j^2) truncated at svd_tol, times the y Gaussian, the
    top-layer indicator, P and 2 eta / (pi r_j^2 d_v).  With the defaults R_f = 239
    (1301 for a 2 ms slab, whose 1 mm path the modes of one slab cannot follow)."""
    Lxy, H = (n_xy - 1) * h_xy, (n_z - 1) * h_z
    rho_cp, eta, d_v, V = 4270.0 * 745.0, 0.25, 50e-6, 0.5
    x_start = 0.5 * Lxy - 0.5 * V * T_slab if x_start is None else x_start
    y0 = 0.5 * Lxy if y0 is None else y0
    free = dict(dirichlet_lo=False, dirichlet_hi=False)
    dims = [dim(n_xy, 0.0, Lxy, s=s, a=a, p=p), dim(n_xy, 0.0, Lxy, s=s, a=a, p=p),
            dim(n_z, 0.0, H, s=s, a=a, p=p, dirichlet_lo=True, dirichlet_hi=False),
            dim(n_t, 0.0, T_slab, kind=TIME, s=s, a=a, p=p, dirichlet_lo=True, dirichlet_hi=False),
            dim(n_par, 100.0, 400.0, kind=PARAM, s=s, a=a, p=p, **free),
            dim(n_par, 30e-6, 80e-6, kind=PARAM, s=s, a=a, p=p, **free)]
    terms = [(rho_cp, ["M", "M", "M", "G", "M", "M"])]
    for e in range(3):
        terms.append((k, ["K" if d == e else "M" for d in range(3)] + ["M", "M", "M"]))
    x = np.linspace(0.0, Lxy, n_xy)
    z = np.linspace(0.0, H, n_z)
    t = np.linspace(0.0, T_slab, n_t)
    x0 = x_start + V * t
    z_ind = (z >= H - d_v - 1e-12).astype(float)
    r_nodes = np.linspace(30e-6, 80e-6, n_par)
    sources = []
    for j, rj in enumerate(r_nodes):
        E = np.exp(-2.0 * (x[:, None] - x0[None, :]) ** 2 / rj ** 2)
        yj = np.exp(-2.0 * (x - y0) ** 2 / rj ** 2)
        ej = np.zeros(n_par)
        ej[j] = 2.0 * eta / (np.pi * rj ** 2 * d_v)
        for sv, ux, vt in _svd_modes(E, svd_tol):
            sources.append((1.0, [("nodal", sv * ux), ("nodal", yj), ("nodal", z_ind), ("nodal", vt),
                                  ("poly", (0.0, 1.0)), ("nodal", ej)]))
    return dict(name=f"lpbf_large_{n_xy}x{n_xy}x{n_z}_t{n_t}_P{n_par}_r{n_par}", dims=dims, terms=terms,
                sources=sources, params=dict(k=k, x_start=x_start, y0=y0, V=V, T_slab=T_slab))


def with_conductivity(desc, k):
    """A copy of a lpbf_large description with conductivity k (the coefficient of its
    three diffusion terms; the source and the dims are shared)."""
    terms = [desc["terms"][0]] + [(float(k), ops) for _, ops in desc["terms"][1:]]
    return dict(desc, terms=terms, params=dict(desc["params"], k=float(k)),
                name=desc["name"] + f"_k{k:g}")


def batch_instances(count=256, seed=4000, n_lo=32, n_hi=1024, M_lo=4, M_hi=32):
    """Independent instances: D in {3..6}, n_d uniform in [n_lo, n_hi], a mode count
    in [M_lo, M_hi], Poisson or transient (last dim time) 50/50, 1..4 separable
    Gaussian sources.  Returns (descriptions, mode counts)."""
    out, Ms = [], []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        D = int(rng.integers(3, 7))
        transient = bool(rng.integers(0, 2))
        ns = [int(v) for v in rng.integers(n_lo, n_hi + 1, size=D)]
        M = int(rng.integers(M_lo, M_hi + 1))
        Rf = int(rng.integers(1, 5))
        Ds = D - 1 if transient else D
        g = gaussian_sources(rng, Rf, Ds)
        dims = [dim(ns[d], 0.0, 1.0) for d in range(Ds)]
        if transient:
            dims.append(dim(ns[-1], 0.0, 1.0, kind=TIME, dirichlet_lo=True,
                            dirichlet_hi=False))
            terms = [(1.0, ["M"] * Ds + ["G"])]
            terms += [(1.0, ["K" if d == e else "M" for d in range(Ds)] + ["M"])
                      for e in range(Ds)]
            sources = [(A, [("gauss", (c[d], sig)) for d in range(Ds)] +
                        [("const", (1.0,))]) for A, sig, c in g]
        else:
            terms = [(1.0, ["K" if d == e else "M" for d in range(D)]) for e in range(D)]
            sources = [(A, [("gauss", (c[d], sig)) for d in range(D)]) for A, sig, c in g]
        out.append(dict(name=f"batch_{seed + i}", dims=dims, terms=terms, sources=sources))
        Ms.append(M)
    return out, Ms


def random_factors(desc, M, seed):
    """Seeded U(-1,1) initial factors (one array per dim, free nodes x M), drawn with
    numpy's generator; passed to both implementations as input."""
    rng = np.random.default_rng(seed)
    out = []
    for dm in desc["dims"]:
        nf = dm["n"] - int(dm["dirichlet_lo"]) - int(dm["dirichlet_hi"])
        out.append(rng.uniform(-1.0, 1.0, size=(nf, M)))
    return out


def n_free(dm):
    return dm["n"] - int(dm["dirichlet_lo"]) - int(dm["dirichlet_hi"])


SPT_RANGES = dict(x=(-0.5, 0.5), y=(-0.5, 0.5), z=(-0.5, 0.5), k=(1.0, 2.0), P=(1.0, 2.0),
                  rho=(1.0, 2.0), cp=(1.0, 2.0), t=(0.0, 0.2))


def _svd_modes(E, tol):
    Uu, sv, Vt = np.linalg.svd(E, full_matrices=False)
    rank = max(1, int(np.sum(sv > tol * sv[0])))
    return [(float(sv[q]), Uu[:, q].copy(), Vt[q].copy()) for q in range(rank)]


def spt_manufactured(n=16, s=2, a=20.0, p=2, n_quad=6, svd_tol=1e-12, ranges=None):
    """The eight-dimensional space-parameter-time heat problem of Sec. 3.2 (Eq. 1 with the
    source of that section): rho c_p du/dt - k Laplace u = f in x, y, z, the parameters
    k, P, rho, c_p, and t, n nodes per dim, with the non-separable exact solution
        u_ex = rho c_p P (1 - exp(-15 k t)) exp(-25 x^2 - 25 y^2),
    zero initial condition and u = u_ex on every spatial face.

    Domain (not stated in the paper; this reading): x, y, z in [-0.5, 0.5], k, P, rho,
    c_p in [1, 2], t in [0, 0.2].  Dims in the order x, y, z, k, P, rho, c_p, t.

    Input construction: exp(-25 x^2) enters as the Gaussian source kind (sigma^2 = 1/50);
    (1 - 50 x^2) exp(-25 x^2) and the (k, t)-coupled factors k exp(-15 k t) and
    k (1 - exp(-15 k t)) enter through their C-HiDeNN nodal interpolants, the coupled
    ones as the SVD of their nodal matrices truncated at svd_tol relative to the largest
    singular value.  The boundary data is a lifting (all-node factors) equal to u_ex's
    nodal values on the spatial boundary nodes and zero at interior nodes:
        u_D = u_ex * (1 - prod_{d in x,y,z} (1 - chi_d)),  chi_d = end-node indicator,
    expanded into its 7 separable sign terms times the SVD of 1 - exp(-15 k t).

    Returns (desc, lift, exact): lift = (vecs, weights) over all nodes; exact =
    (separable factors per dim as (kind, params) or None for the coupled pair,
    the coupled pair's dims, its function name)."""
    R = dict(SPT_RANGES, **(ranges or {}))
    names = ["x", "y", "z", "k", "P", "rho", "cp", "t"]
    kinds = [SPACE] * 3 + [PARAM] * 4 + [TIME]
    dims = []
    for nm, kd in zip(names, kinds):
        lo, hi = R[nm]
        if kd == SPACE:
            dims.append(dim(n, lo, hi, s=s, a=a, p=p, n_quad=n_quad))
        elif kd == PARAM:
            dims.append(dim(n, lo, hi, kind=PARAM, s=s, a=a, p=p, n_quad=n_quad, dirichlet_lo=False,
                            dirichlet_hi=False, weight_poly=(0.0, 1.0)))
        else:
            dims.append(dim(n, lo, hi, kind=TIME, s=s, a=a, p=p, n_quad=n_quad, dirichlet_lo=True,
                            dirichlet_hi=False))
    X = {nm: np.linspace(*R[nm], n) for nm in names}
    # rho c_p du/dt: W (weight = the coordinate) on rho and c_p, G in time
    terms = [(1.0, ["M"] * 5 + ["W", "W", "G"])]
    # -k Laplace u: K in one spatial dim, W on k
    for e in range(3):
        terms.append((1.0, ["K" if d == e else "M" for d in range(3)] + ["W", "M", "M", "M", "M"]))
    sig = math.sqrt(1.0 / 50.0)
    g = ("gauss", (0.0, sig))
    hx = (1.0 - 50.0 * X["x"] ** 2) * np.exp(-25.0 * X["x"] ** 2)
    hy = (1.0 - 50.0 * X["y"] ** 2) * np.exp(-25.0 * X["y"] ** 2)
    kk, tt = np.meshgrid(X["k"], X["t"], indexing="ij")
    one = ("const", (1.0,))
    lin = ("poly", (0.0, 1.0))
    sq = ("poly", (0.0, 0.0, 1.0))
    sources = []
    # 15 rho^2 c_p^2 k P exp(-15 k t) G(x) G(y)
    for sv, uk, vt in _svd_modes(kk * np.exp(-15.0 * kk * tt), svd_tol):
        sources.append((15.0 * sv, [g, g, one, ("nodal", uk), lin, sq, sq, ("nodal", vt)]))
    # 50 rho c_p k P (1 - exp(-15 k t)) G(x) G(y) [(1 - 50 x^2) + (1 - 50 y^2)]
    for sv, uk, vt in _svd_modes(kk * (1.0 - np.exp(-15.0 * kk * tt)), svd_tol):
        sources.append((50.0 * sv, [("nodal", hx), g, one, ("nodal", uk), lin, lin, lin, ("nodal", vt)]))
        sources.append((50.0 * sv, [g, ("nodal", hy), one, ("nodal", uk), lin, lin, lin, ("nodal", vt)]))
    # lifting of the boundary data
    gx, gy, onez = np.exp(-25.0 * X["x"] ** 2), np.exp(-25.0 * X["y"] ** 2), np.ones(n)
    chi = np.zeros(n)
    chi[[0, -1]] = 1.0
    modes_E = _svd_modes(1.0 - np.exp(-15.0 * kk * tt), svd_tol)
    cols = [[] for _ in range(8)]
    wts = []
    for mask in range(1, 8):
        sign = -1.0 if bin(mask).count("1") % 2 == 0 else 1.0
        base = [gx, gy, onez]
        sp = [base[d] * chi if mask >> d & 1 else base[d] for d in range(3)]
        for sv, uk, vt in modes_E:
            for d in range(3):
                cols[d].append(sp[d])
            cols[3].append(uk)
            cols[4].append(X["P"])
            cols[5].append(X["rho"])
            cols[6].append(X["cp"])
            cols[7].append(vt)
            wts.append(sign * sv)
    vecs = [np.stack(c, axis=1) for c in cols]
    exact = dict(sep=[g, g, one, None, lin, lin, lin, None], pair=(3, 7), pair_fn="1-exp(-15kt)")
    desc = dict(name=f"spt_manufactured_n{n}_s{s}p{p}", dims=dims, terms=terms, sources=sources)
    return desc, (vecs, np.array(wts)), exact


def spt_exact_pair(k, t):
    """The (k, t)-coupled factor of the Sec. 3.2 exact solution."""
    return 1.0 - np.exp(-15.0 * k * t)


def spt_exact(X):
    """The Sec. 3.2 exact solution at points X [n, 8] (x, y, z, k, P, rho, c_p, t)."""
    x, y, _, k, Pw, rho, cp, t = np.asarray(X, dtype=float).T
    return rho * cp * Pw * spt_exact_pair(k, t) * np.exp(-25.0 * x ** 2 - 25.0 * y ** 2)


ST_RANGES = dict(x=(0.0, 20.0), y=(-5.0, 5.0), t=(0.0, 0.1))


def st_exact_pair(x, t):
    """The (x, t)-coupled factor of the Sec. 3.1 exact solution (the moving Gaussian)."""
    return (1.0 - np.exp(-15.0 * t)) * np.exp(-(x - 100.0 * t - 5.0) ** 2)


def st_exact(X):
    """The Sec. 3.1 exact solution at points X [n, 3] (x, y, t)."""
    x, y, t = np.asarray(X, dtype=float).T
    return st_exact_pair(x, t) * np.exp(-y ** 2)


def st_manufactured(n=100, n_t=None, s=1, a=20.0, p=1, n_quad=6, svd_tol=1e-12, ranges=None):
    """The space-time moving-source problem of Sec. 3.1: du/dt - Laplace u = f in x, y, t
    with the non-separable exact solution
        u_ex = (1 - exp(-15 t)) exp(-y^2 - (x - 100 t - 5)^2),
    zero initial condition and u = u_ex on the spatial boundary; n nodes per spatial dim,
    n_t (default n) in time.

    Readings (the paper states neither the domain nor a source consistent with u_ex: its
    source has the Gaussian centred at x = 100 t - 5 and the opposite sign on the
    15 exp(-15 t) term): x in [0, 20], y in [-5, 5], t in [0, 0.1], rho c_p = k = 1, and
    f = du_ex/dt - Laplace u_ex from u_ex as printed:
        f = [15 e^{-15t} H + 200 xi E H + (2 - 4 xi^2) E H] e^{-y^2} + E H (2 - 4 y^2) e^{-y^2},
    E = 1 - e^{-15 t}, xi = x - 100 t - 5, H = e^{-xi^2}.  The (x, t) parts enter through
    the SVD of their nodal matrices (truncated at svd_tol), y parts as the Gaussian kind
    and the nodal interpolant of (2 - 4 y^2) e^{-y^2}.  The lifting (boundary nodes
    only) is u_ex's nodal values times 1 - (1 - chi_x)(1 - chi_y), 3 sign terms.

    Returns (desc, lift, exact) as spt_manufactured."""
    R = dict(ST_RANGES, **(ranges or {}))
    n_t = n if n_t is None else n_t
    dims = [dim(n, *R["x"], s=s, a=a, p=p, n_quad=n_quad), dim(n, *R["y"], s=s, a=a, p=p, n_quad=n_quad),
            dim(n_t, *R["t"], kind=TIME, s=s, a=a, p=p, n_quad=n_quad, dirichlet_lo=True, dirichlet_hi=False)]
    terms = [(1.0, ["M", "M", "G"]), (1.0, ["K", "M", "M"]), (1.0, ["M", "K", "M"])]
    x, y, t = (np.linspace(*R[k], m) for k, m in (("x", n), ("y", n), ("t", n_t)))
    xx, tt = np.meshgrid(x, t, indexing="ij")
    E = 1.0 - np.exp(-15.0 * tt)
    xi = xx - 100.0 * tt - 5.0
    H = np.exp(-xi ** 2)
    f2 = 15.0 * np.exp(-15.0 * tt) * H + 200.0 * xi * E * H + (2.0 - 4.0 * xi ** 2) * E * H
    gy = ("gauss", (0.0, math.sqrt(0.5)))
    hy = (2.0 - 4.0 * y ** 2) * np.exp(-y ** 2)
    sources = [(sv, [("nodal", ux), gy, ("nodal", vt)]) for sv, ux, vt in _svd_modes(f2, svd_tol)]
    sources += [(sv, [("nodal", ux), ("nodal", hy), ("nodal", vt)]) for sv, ux, vt in _svd_modes(E * H, svd_tol)]
    chi = np.zeros(n)
    chi[[0, -1]] = 1.0
    ey = np.exp(-y ** 2)
    cols = [[], [], []]
    wts = []
    for sv, ux, vt in _svd_modes(E * H, svd_tol):
        for xf, yf, sign in ((ux * chi, ey, 1.0), (ux, ey * chi, 1.0), (ux * chi, ey * chi, -1.0)):
            cols[0].append(xf)
            cols[1].append(yf)
            cols[2].append(vt)
            wts.append(sign * sv)
    vecs = [np.stack(c, axis=1) for c in cols]
    exact = dict(sep=[None, gy, None], pair=(0, 2))
    desc = dict(name=f"st_manufactured_n{n}_t{n_t}_s{s}p{p}", dims=dims, terms=terms, sources=sources)
    return desc, (vecs, np.array(wts)), exact


NONLINEAR_LAW = (0.5, 1.0, 0.3, 1.0)   # (m_c, n_c, m_k, n_k) of the manufactured case
NONLINEAR_MODES = ((1.0, 1.0, 1), (0.5, 2.0, 2), (0.25, 3.0, 3))   # (amplitude, omega, k)


def _harm_mul(a, b):
    """Product of two harmonics ('s'|'c', k) as a list of (coef, harmonic):
    sin a sin b = (cos(a-b) - cos(a+b))/2, cos a cos b = (cos(a-b) + cos(a+b))/2,
    sin a cos b = (sin(a+b) + sin(a-b))/2, with sin(-k) = -sin k, cos(-k) = cos k."""
    (ta, ka), (tb, kb) = a, b
    def s_(k):
        return [(1.0 if k > 0 else -1.0, ("s", abs(k)))] if k != 0 else []
    def c_(k):
        return [(1.0, ("c", abs(k)))]
    if ta == "s" and tb == "s":
        return [(0.5 * c, h) for c, h in c_(ka - kb)] + [(-0.5 * c, h) for c, h in c_(ka + kb)]
    if ta == "c" and tb == "c":
        return [(0.5 * c, h) for c, h in c_(ka - kb)] + [(0.5 * c, h) for c, h in c_(ka + kb)]
    if ta == "c":
        (ta, ka), (tb, kb) = b, a
    return [(0.5 * c, h) for c, h in s_(ka + kb)] + [(0.5 * c, h) for c, h in s_(ka - kb)]


def nonlinear_manufactured(n=32, n_t=None, s=2, a=20.0, p=2, law=NONLINEAR_LAW, modes=NONLINEAR_MODES):
    """A manufactured nonlinear space-time problem for the global-local solver of
    App. A: d/dt[c(u) u] - d/dx (k(u) du/dx) = f on x in [0, 1], t in [0, 1], with the
    linear laws c = m_c u + n_c, k = m_k u + n_k (as in Sec. 3.3), u = 0 at x = 0, 1
    and at t = 0, and the exact solution of CP rank 3
        u = sum_a A_a sin(omega_a t) sin(k_a pi x).
    f = (2 m_c u + n_c) du/dt - m_k (du/dx)^2 - (m_k u + n_k) d2u/dx2, expanded into
    separable harmonics by the product-to-sum identities: every factor is a sine or a
    cosine (the sine kind with phase pi/2; cos 0 = 1 the constant kind).
    Returns the description (dims, sources; the terms are the solver's)."""
    m_c, n_c, m_k, n_k = law
    n_t = n if n_t is None else n_t
    dims = [dim(n, 0.0, 1.0, s=s, a=a, p=p),
            dim(n_t, 0.0, 1.0, kind=TIME, s=s, a=a, p=p, dirichlet_lo=True, dirichlet_hi=False)]
    pi = math.pi
    # u, du/dt, du/dx, d2u/dx2 as lists of (coef, x-harmonic in units of pi, t-harmonic)
    U = [(A, ("s", k), ("s", w)) for A, w, k in modes]
    Ut = [(A * w, ("s", k), ("c", w)) for A, w, k in modes]
    Ux = [(A * k * pi, ("c", k), ("s", w)) for A, w, k in modes]
    Uxx = [(-A * (k * pi) ** 2, ("s", k), ("s", w)) for A, w, k in modes]
    acc = {}

    def add(coef, hx, ht):
        key = (hx, ht)
        acc[key] = acc.get(key, 0.0) + coef

    def prod(coef, P, Q):
        for ca, xa, ta in P:
            for cb, xb, tb in Q:
                for cx, hx in _harm_mul(xa, xb):
                    for ct, ht in _harm_mul(ta, tb):
                        add(coef * ca * cb * cx * ct, hx, ht)

    prod(2.0 * m_c, U, Ut)
    for c, hx, ht in Ut:
        add(n_c * c, hx, ht)
    prod(-m_k, Ux, Ux)
    prod(-m_k, U, Uxx)
    for c, hx, ht in Uxx:
        add(-n_k * c, hx, ht)

    def factor(h, scale):
        t, k = h
        if t == "c" and k == 0:
            return ("const", (1.0,))
        return ("sin", (k * scale, 0.0 if t == "s" else 0.5 * pi))

    sources = [(c, [factor(hx, pi), factor(ht, 1.0)]) for (hx, ht), c in sorted(acc.items())
               if abs(c) > 1e-14 and not (hx[0] == "s" and hx[1] == 0) and not (ht[0] == "s" and ht[1] == 0)]
    return dict(name=f"nonlinear_manufactured_n{n}_t{n_t}", dims=dims, terms=[], sources=sources)


def nonlinear_exact(X, modes=NONLINEAR_MODES):
    """The manufactured solution at points X [n, 2] (x, t)."""
    x, t = np.asarray(X, dtype=float).T
    return sum(A * np.sin(w * t) * np.sin(k * math.pi * x) for A, w, k in modes)


def nonlinear_exact_factors(modes=NONLINEAR_MODES):
    """Its separable form: per mode (amplitude, x-function, t-function)."""
    return [(A, (lambda x, k=k: np.sin(k * math.pi * x)), (lambda t, w=w: np.sin(w * t))) for A, w, k in modes]


# Sec. 3.3 (Inconel 718): rho c_p = m_cp u + n_cp, k = m_k u + n_k in mm, s, W, K
INCONEL_LAW = (6.11e-7, 3.25e-3, 1.52e-5, 5.29e-3)   # (m_c, n_c, m_k, n_k)


def nonlinear_track(n_xy=101, n_z=11, n_t=113, P=200.0, eta=0.25, d_v=0.1, r=0.5, V=500.0,
                    svd_tol=1e-10, s=2, a=20.0, p=2):
    """The moving-source problem with temperature-dependent coefficients of Sec. 3.3:
    a 10 mm x 10 mm x 1 mm plate (n_xy x n_xy x n_z nodes; 10 elements across the
    source diameter at the default 101 nodes), homogeneous Dirichlet on the left and
    right faces (x = 0, 10 mm), insulated elsewhere, zero initial temperature rise, time
    step 1.6e-4 s (n_t = 113: the source crosses x = 0.5 .. 9.5 mm at V = 500 mm/s), and
    the linear laws INCONEL_LAW for rho c_p(u) and k(u).

    Readings (the paper gives no power, absorptivity or penetration depth for this
    case): the moving source of Sec. 2.4, 2 eta P / (pi r^2 d_v) exp(-2((x - x0(t))^2 +
    (y - y0)^2) / r^2) on the top layer z >= H - d_v, with P = 200 W, eta = 0.25,
    d_v = 0.1 mm, r = 0.5 mm, y0 = 5 mm, x0(t) = 0.5 mm + V t.  The (x, t) part enters as
    the SVD of its nodal matrix truncated at svd_tol; y as the Gaussian kind
    (sigma = r / 2); z as the nodal top-layer indicator.  Returns the description
    (dims with time last, sources; the terms are the solver's)."""
    Lx, H = 10.0, 1.0
    T_end = 1.6e-4 * (n_t - 1)
    dims = [dim(n_xy, 0.0, Lx, s=s, a=a, p=p),
            dim(n_xy, 0.0, Lx, s=s, a=a, p=p, dirichlet_lo=False, dirichlet_hi=False),
            dim(n_z, 0.0, H, s=s, a=a, p=p, dirichlet_lo=False, dirichlet_hi=False),
            dim(n_t, 0.0, T_end, kind=TIME, s=s, a=a, p=p, dirichlet_lo=True, dirichlet_hi=False)]
    x = np.linspace(0.0, Lx, n_xy)
    z = np.linspace(0.0, H, n_z)
    t = np.linspace(0.0, T_end, n_t)
    E = np.exp(-2.0 * (x[:, None] - (0.5 + V * t[None, :])) ** 2 / r ** 2)
    amp = 2.0 * eta * P / (math.pi * r ** 2 * d_v)
    top = (z >= H - d_v - 1e-12).astype(float)
    sources = [(amp * sv, [("nodal", ux), ("gauss", (5.0, 0.5 * r)), ("nodal", top), ("nodal", vt)])
               for sv, ux, vt in _svd_modes(E, svd_tol)]
    return dict(name=f"nonlinear_track_{n_xy}x{n_xy}x{n_z}_t{n_t}", dims=dims, terms=[], sources=sources)
