"""The mode-side eigen-solve (Sec. 2.6: the M x M symmetric-definite pencil of the
coefficient matrices) on its own, through taps_util_md_pencil: FP32 rotations, FP64
first-order corrections of the basis, FP64 rotations when a correction is rejected.
Checked against the dense symmetric-definite eigensolver the oracle uses: the basis
must be C_X-orthonormal and diagonalise C_Y as well as the library routine's does, and
the eigenvalues must agree."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

scipy_linalg = pytest.importorskip("scipy.linalg")


@pytest.fixture(scope="module")
def T():
    from paper_2503_13933_gb300 import taps
    taps.lib()
    return taps


def _pencil(kind, M, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, M))
    CX = A @ A.T / M + 0.5 * np.eye(M)
    if kind == "graded":   # C_X and C_Y over six orders of magnitude
        D = np.diag(np.logspace(-1.5, 1.5, M))
        CX = D @ CX @ D
    if kind == "clustered":   # eigenvalues in exact groups of three (degenerate pencil)
        L = np.linalg.cholesky(CX)
        V, _ = np.linalg.qr(rng.standard_normal((M, M)))
        lam = np.repeat(np.linspace(1.0, 3.0, (M + 2) // 3), 3)[:M]
        CY = L @ V @ np.diag(lam) @ V.T @ L.T
    elif kind == "single":
        CY = None
    else:
        B = rng.standard_normal((M, M))
        CY = B @ B.T / M
        if kind == "graded":
            CY = D @ CY @ D
    # the device sees the coefficients as the sweep forms them: symmetric up to rounding
    CX = CX + 1e-15 * np.abs(CX).max() * rng.standard_normal((M, M))
    return CX, CY


def _metrics(CX, CY, W, lam):
    Sx, Sy = 0.5 * (CX + CX.T), (0.5 * (CY + CY.T) if CY is not None else None)
    ex = np.abs(W.T @ Sx @ W - np.eye(len(W))).max()
    if Sy is None:
        return ex, 0.0
    G = W.T @ Sy @ W
    ey = np.abs(G - np.diag(np.diag(G))).max() / max(np.abs(lam).max(), 1e-300)
    return ex, ey


@pytest.mark.parametrize("kind,M", [("random", 33), ("random", 64), ("random", 100), ("random", 116),
                                    ("graded", 64), ("graded", 100), ("clustered", 48), ("clustered", 99),
                                    ("single", 64)])
def test_mode_side_eigensolve_matches_dense_solver(T, kind, M):
    CX, CY = _pencil(kind, M, seed=7000 + M)
    dev = "cuda"
    cx = torch.tensor(CX, device=dev)
    cy = torch.tensor(CY, device=dev) if CY is not None else None
    W = torch.empty((M, M), dtype=torch.float64, device=dev)
    lam = torch.empty(M, dtype=torch.float64, device=dev)
    refined = T.md_pencil(cx, cy, W, lam)
    Wg, lg = W.cpu().numpy(), lam.cpu().numpy()
    Sx = 0.5 * (CX + CX.T)
    if CY is None:
        ref_lam = np.zeros(M)
        ref_W = np.linalg.inv(np.linalg.cholesky(Sx)).T
    else:
        ref_lam, ref_W = scipy_linalg.eigh(0.5 * (CY + CY.T), Sx)
    ex, ey = _metrics(CX, CY, Wg, lg)
    rx, ry = _metrics(CX, CY, ref_W, ref_lam if CY is not None else np.zeros(M))
    print(f"{kind} M={M} refined={refined}: |W'CxW-I| {ex:.2e} (library {rx:.2e}), "
          f"offdiag(W'CyW)/max|lam| {ey:.2e} (library {ry:.2e})")
    assert ex <= max(10 * rx, 1e-12), (ex, rx)
    assert ey <= max(10 * ry, 1e-12), (ey, ry)
    scale = max(np.abs(ref_lam).max(), 1e-300)
    kappa = np.linalg.cond(Sx)
    assert np.abs(np.sort(lg) - np.sort(ref_lam)).max() <= 1e-12 * max(1.0, kappa) * scale
    if kind == "random":
        # well-separated eigenvalues: the FP32 basis is in the corrections' quadratic regime
        assert refined == 1
    if kind == "single":
        assert np.all(lg == 0.0)


def test_mode_side_eigensolve_rejects_bad_arguments(T):
    x = torch.zeros((20, 20), dtype=torch.float64, device="cuda")
    lam = torch.zeros(20, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TapsError):
        T.md_pencil(x, x, x, lam)   # M = 20: the one-CTA eigen-solve's range
