"""The separated (CP) form of the moving laser source built as input data for the
powder-bed-fusion slabs: pinned against the source formula of Sec. 2.4 evaluated
directly at grid nodes."""
import numpy as np

from paper_2503_13933_gb300 import workloads as W


def _factor_values(kind, par, xs):
    if kind == "nodal":
        return np.asarray(par, dtype=float)
    if kind == "poly":
        return sum(c * xs ** k for k, c in enumerate(par))
    if kind == "const":
        return np.full_like(xs, par[0])
    raise ValueError(kind)


def test_moving_source_cp_reproduces_the_formula():
    """(2 eta P / (pi r^2 d_v)) exp(-2((x - x0(t))^2 + (y - y0)^2) / r^2) 1(z >= H - d_v)
    at 600 random (x, y, z, t, P, r, k) node tuples of slab 3 equals the sum of the CP
    terms to the SVD truncation level."""
    n_xy, n_z, n_t, n_par, n_slabs, slab = 40, 12, 16, 5, 8, 3
    desc = W.lpbf_slab(n_xy=n_xy, n_z=n_z, n_t=n_t, n_par=n_par, slab=slab, n_slabs=n_slabs)
    grids = [np.linspace(dm["lo"], dm["hi"], dm["n"]) for dm in desc["dims"]]
    vals = [[_factor_values(k, p, grids[d]) for d, (k, p) in enumerate(facs)]
            for _, facs in desc["sources"]]
    rng = np.random.default_rng(11)
    idx = np.stack([rng.integers(0, dm["n"], 600) for dm in desc["dims"]], axis=1)
    cp = np.zeros(600)
    for (beta, _), v in zip(desc["sources"], vals):
        term = np.full(600, beta)
        for d in range(7):
            term *= v[d][idx[:, d]]
        cp += term
    x, y, z, t, P, r = (grids[d][idx[:, d]] for d in range(6))
    eta, d_v, V, H, Lxy = 0.25, 50e-6, 0.5, 0.635e-3, 2.555e-3
    x0 = 0.3e-3 + V * t
    f = (2 * eta * P / (np.pi * r ** 2 * d_v) * np.exp(-2 * ((x - x0) ** 2 + (y - Lxy / 2) ** 2) / r ** 2)
         * (z >= H - d_v))
    scale = 2 * eta * 400.0 / (np.pi * (30e-6) ** 2 * d_v)
    assert np.max(np.abs(cp - f)) <= 1e-8 * scale
    # the time window of slab 3
    T_slab = (2.25e-3 - 0.3e-3) / V / n_slabs
    assert abs(desc["dims"][3]["lo"] - 3 * T_slab) < 1e-15 and abs(desc["dims"][3]["hi"] - 4 * T_slab) < 1e-15


def test_lpbf_operator_terms():
    """Nine operator terms: rho c_p (time derivative), diffusion in x, y, z weighted by
    the conductivity dim (W), convection on the five non-bottom faces."""
    desc = W.lpbf_slab(n_xy=10, n_z=8, n_t=6, n_par=3)
    terms = desc["terms"]
    assert len(terms) == 9
    assert terms[0] == (4270.0 * 745.0, ["M", "M", "M", "G", "M", "M", "M"])
    assert [t[1][6] for t in terms[1:4]] == ["W", "W", "W"]
    faces = sorted(tuple(t[1][:3]) for t in terms[4:])
    assert faces == sorted([("Blo", "M", "M"), ("Bhi", "M", "M"), ("M", "Blo", "M"), ("M", "Bhi", "M"),
                            ("M", "M", "Bhi")])
    assert desc["dims"][2]["dirichlet_lo"] and not desc["dims"][2]["dirichlet_hi"]
    assert not desc["dims"][0]["dirichlet_lo"] and not desc["dims"][0]["dirichlet_hi"]
