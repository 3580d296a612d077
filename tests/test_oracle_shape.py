"""Pins of the oracle's C-HiDeNN shape functions (Eq. 1, Eq. 3, Sec. 2.1) against
properties the paper states and textbook special cases -- never against itself."""
import os

import numpy as np
import pytest

from oracle import taps_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _grid(n, lo=0.0, hi=1.0):
    return np.linspace(lo, hi, n)


@pytest.mark.parametrize("s,p", [(1, 1), (2, 2), (2, 1), (3, 3), (4, 3)])
def test_kronecker_delta_at_nodes(s, p):
    """Eq. 3: N~_k(x_l) = delta_kl, on every element including the truncated ends."""
    x = _grid(14)
    for e in range(len(x) - 1):
        for side in (0, 1):
            ids, N, _ = O.shape_functions(x, s, 20.0, p, e, x[e + side])
            expect = np.array([1.0 if k == e + side else 0.0 for k in ids])
            assert np.max(np.abs(N - expect)) < 1e-12


@pytest.mark.parametrize("s,p", [(1, 1), (2, 2), (2, 1), (3, 3), (4, 3)])
def test_partition_of_unity_and_reproduction(s, p):
    """Partition of unity (Sec. 2.1) and reproduction of polynomials up to order p
    (the reproducing order p of Eq. 1), for values and derivatives."""
    rng = np.random.default_rng(1)
    x = _grid(13, -0.3, 2.1)
    for _ in range(60):
        xe = rng.uniform(x[0], x[-1])
        e = O.locate(x, xe)
        ids, N, B = O.shape_functions(x, s, 20.0, p, e, xe)
        xs = x[ids]
        for q in range(p + 1):
            assert abs(N @ xs ** q - xe ** q) < 1e-11 * max(1.0, abs(xe) ** q)
            dq = q * xe ** (q - 1) if q > 0 else 0.0
            assert abs(B @ xs ** q - dq) < 1e-9 * max(1.0, abs(xe) ** q)


def test_reproduction_fails_beyond_p():
    """Negative control: p=1 does NOT reproduce x^2 (a check that the reproduction
    test can fail)."""
    x = _grid(13)
    e = 5
    xe = x[e] + 0.3 * (x[1] - x[0])
    ids, N, _ = O.shape_functions(x, 2, 20.0, 1, e, xe)
    assert abs(N @ x[ids] ** 2 - xe ** 2) > 1e-6


@pytest.mark.parametrize("p", [1, 2, 3])
def test_dilation_independence(p):
    """For p >= 1 and a >= 2(s+1) every kernel argument stays below 1/2, where the
    constant and quadratic kernel terms are annihilated by the polynomial
    constraints: the patch interpolant is the cubic polyharmonic spline + degree-p
    polynomial, whatever a is.  a = 20 and a = 40 must give the same tables."""
    x = _grid(11)
    for e in (0, 4, 9):
        xe = x[e] + 0.41 * (x[1] - x[0])
        s_ = max(2, p)
        _, N1, B1 = O.shape_functions(x, s_, 20.0, p, e, xe)
        _, N2, B2 = O.shape_functions(x, s_, 40.0, p, e, xe)
        assert np.max(np.abs(N1 - N2)) < 1e-11
        assert np.max(np.abs(B1 - B2)) < 1e-9


def test_quadratic_lagrange_special_case():
    """s=1, p=2, interior patch: W^i is the quadratic Lagrange basis (golden file)."""
    rows = np.loadtxt(os.path.join(GOLD, "quadratic_lagrange_s1p2.txt"))
    x = np.arange(7, dtype=float)          # h = 1
    i = 3
    for t, l0, l1, l2, d0, d1, d2 in rows:
        nodes, W, dW = O.patch_function(x, i, 1, 20.0, 2, 1.0, x[i] + t)
        assert nodes == [2, 3, 4]
        assert np.max(np.abs(W - [l0, l1, l2])) < 1e-13
        assert np.max(np.abs(dW - [d0, d1, d2])) < 1e-12


def test_linear_hats_special_case():
    """s=0, p=0 reduces to linear finite elements: K, M, G interior stencils and end
    entries equal the textbook values (golden file)."""
    gold = {}
    for line in open(os.path.join(GOLD, "linear_hat_matrices.txt")):
        if line.strip() and not line.startswith("#"):
            k, a, b, c = line.split()
            gold[k] = np.array([float(a), float(b), float(c)])
    n, L = 9, 2.0
    h = L / (n - 1)
    dm = O.Dim(n=n, lo=0.0, hi=L, s=0, a=20.0, p=0, dirichlet_lo=False, dirichlet_hi=False)
    mats = O.assemble_full(dm)
    scale = {"K": 1.0 / h, "M": h / 6.0, "G": 1.0}
    for name, op in (("K", O.OP_K), ("M", O.OP_M), ("G", O.OP_G)):
        A = mats[op]
        for i in range(1, n - 1):
            assert np.allclose(A[i, i - 1:i + 2], scale[name] * gold[name], atol=1e-13)
        if name != "G":                     # G has a zero interior diagonal
            assert np.count_nonzero(np.abs(A) > 1e-14) == 3 * n - 2
    assert abs(mats[O.OP_K][0, 0] - 1.0 / h) < 1e-13
    assert abs(mats[O.OP_M][0, 0] - h / 3.0) < 1e-13
    assert abs(mats[O.OP_G][0, 0] + 0.5) < 1e-13


def test_truncated_patch_too_small_is_an_error():
    """A truncated end patch with fewer than p+1 nodes cannot reproduce order p."""
    x = _grid(8)
    with pytest.raises(ValueError):
        O.patch_matrix(x, 0, 1, 20.0, 2, x[1] - x[0])
