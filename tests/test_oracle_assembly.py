"""Pins of the oracle's 1D matrices (Eqs. 31-35) by closed-form integrals, symmetry
and definiteness, and quadrature exactness."""
import numpy as np
import pytest

from oracle import taps_oracle as O


def _all(n, lo, hi, s=2, p=2, nq=6, w=(0.0, 1.0)):
    return O.Dim(n=n, lo=lo, hi=hi, s=s, a=20.0, p=p, n_quad=nq, dirichlet_lo=False,
                 dirichlet_hi=False, weight_poly=w)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_closed_form_integrals(p):
    lo, hi = 0.5, 2.0
    dm = _all(17, lo, hi, s=max(2, p), p=p)   # truncated end patches need s+1 >= p+1
    A = O.assemble_full(dm)
    x = dm.x
    one = np.ones_like(x)
    K, M, G, W = A[O.OP_K], A[O.OP_M], A[O.OP_G], A[O.OP_W]
    L = hi - lo
    assert abs(one @ M @ one - L) < 1e-13                      # int 1
    assert abs(one @ M @ x - (hi ** 2 - lo ** 2) / 2) < 1e-13  # int x
    assert abs(x @ M @ x - (hi ** 3 - lo ** 3) / 3) < 1e-12    # int x^2 (p>=1)
    assert np.max(np.abs(K @ one)) < 1e-11                     # K 1 = 0
    assert abs(x @ K @ x - L) < 1e-11                          # int (x')^2
    assert np.max(np.abs(G @ one)) < 1e-12                     # G 1 = 0
    assert abs(one @ G @ x - L) < 1e-12                        # int 1 * (x)'
    assert abs(one @ W @ one - (hi ** 2 - lo ** 2) / 2) < 1e-12  # int w, w(x)=x
    if p >= 2:
        x2 = x ** 2
        assert abs(x2 @ K @ x2 - 4.0 * (hi ** 3 - lo ** 3) / 3) < 1e-10
    # G + G^T = e_n e_n^T - e_0 e_0^T (integration by parts + Kronecker delta, Eq. 3)
    E = np.zeros_like(G)
    E[-1, -1], E[0, 0] = 1.0, -1.0
    assert np.max(np.abs(G + G.T - E)) < 1e-12


def test_symmetry_and_definiteness():
    dm = _all(20, 0.0, 1.0)
    A = O.assemble_full(dm)
    K, M = A[O.OP_K], A[O.OP_M]
    assert np.max(np.abs(K - K.T)) < 1e-12
    assert np.max(np.abs(M - M.T)) < 1e-15
    ev = np.linalg.eigvalsh(M)
    assert ev.min() > 0
    evk = np.linalg.eigvalsh(K)
    assert abs(evk[0]) < 1e-10 and evk[1] > 1e-3              # null space = span{1}
    dmf = O.Dim(n=20, lo=0.0, hi=1.0)                           # Dirichlet both ends
    Kf = O.assemble_free(dmf)[O.OP_K]
    np.linalg.cholesky(Kf)                                      # SPD after Dirichlet


def test_band_structure():
    """Every 1D matrix is banded with half-bandwidth 2s+1 (shape functions of nodes
    more than 2s+1 apart share no element)."""
    for s in (1, 2, 3):
        dm = _all(24, 0.0, 1.0, s=s, p=1)
        K = O.assemble_full(dm)[O.OP_K]
        i, j = np.nonzero(np.abs(K) > 1e-15)
        assert np.max(np.abs(i - j)) == 2 * s + 1


def test_quadrature_exact():
    """Shape functions are degree-4 polynomials per element for p <= 3, so 6 and 10
    Gauss points agree to rounding for every matrix."""
    a = O.assemble_full(_all(12, 0.0, 1.0, nq=6))
    b = O.assemble_full(_all(12, 0.0, 1.0, nq=10))
    for k in (O.OP_K, O.OP_M, O.OP_G, O.OP_W):
        assert np.max(np.abs(a[k] - b[k])) < 1e-12 * max(1.0, np.max(np.abs(b[k])))
    c = O.assemble_full(_all(12, 0.0, 1.0, nq=3))            # under-integrated: differs
    assert np.max(np.abs(c[O.OP_M] - b[O.OP_M])) > 1e-8 * np.max(np.abs(b[O.OP_M]))


def test_source_projection():
    dm = _all(33, 0.0, 1.0)
    one = np.ones(dm.n)
    q = O.project_source(dm, "sin", (np.pi, 0.0))
    assert abs(q @ one - 2.0 / np.pi) < 1e-12                   # int sin(pi x)
    q2 = O.project_source(dm, "poly", (1.0, 2.0, 3.0))
    assert abs(q2 @ one - (1.0 + 1.0 + 1.0)) < 1e-13            # int 1+2x+3x^2
    assert abs(q2 @ dm.x - (0.5 + 2.0 / 3.0 + 0.75)) < 1e-13    # int x(1+2x+3x^2)
    qg = O.project_source(dm, "gauss", (0.4, 0.1))
    from math import erf, sqrt, pi
    exact = 0.1 * sqrt(pi / 2) * (erf(0.6 / (0.1 * sqrt(2))) + erf(0.4 / (0.1 * sqrt(2))))
    assert abs(qg @ one - exact) < 1e-9
    nod = np.sin(dm.x)
    qn = O.project_source(dm, "nodal", None, nodal=nod)
    assert np.allclose(qn, O.assemble_full(dm)[O.OP_M] @ nod)
