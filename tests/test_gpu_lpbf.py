"""The powder-bed-fusion space-parameter-time slab (3 space dims with convection faces,
time, laser power, spot radius and conductivity: 7 dims, a moving source of rank ~R_f
in CP form) on the GPU against the oracle: sweeps from the same factors, and two
chained slabs."""
import numpy as np
import pytest

from oracle import taps_oracle as O
from paper_2503_13933_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_13933_gb300 import build, taps
    import os
    if not os.path.exists(taps.LIB_PATH):
        build.build()
    taps.lib()
    return taps


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_lpbf_slab_sweeps_match_oracle(T):
    """Two sweeps, M = 6: space dims by the node-side pencil with convection-face
    corrections (four or three operators), time on the mode side, the parameter dims by
    the node-side pencil; no block elimination."""
    desc = W.lpbf_slab(n_xy=24, n_z=12, n_t=10, n_par=5)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    M = 6
    U0 = W.random_factors(desc, M, seed=3)
    U = P.factors(M)
    U.set(U0)
    P.profile_reset()
    P.sweep(U, 2, solver=T.SOLVER_FASTDIAG)
    Uo = [u.copy() for u in U0]
    for _ in range(2):
        Uo, _ = O.sweep(Po, Uo, solver="fastdiag")
    got = U.get()
    for d in range(7):
        assert rel(got[d], Uo[d]) < 1e-10, (d, rel(got[d], Uo[d]))
    prof = P.profile()
    assert prof["block_lu"]["launches"] == 0
    assert prof["modediag"]["launches"] == 2 * 4
    assert prof["fastdiag"]["launches"] == 2 * (3 * 1 + 3 * 5)   # parameter dims; space dims
    # the Eq. 42 residual of the GPU's factors, recomputed by the oracle
    r_gpu = P.residual(U, T.RES_ALS)
    r_o = O.als_residual(Po, got)
    assert abs(r_gpu - r_o) <= 1e-8 * max(r_o, 1e-300)


def test_lpbf_two_slabs_match_oracle(T):
    """Slab 0 swept, its end state lifted into slab 1 (moving source of slab 1 plus the
    lifting terms), slab 1 swept: the same fields as the oracle's own chaining.  The
    parameter dims have more nodes than modes, so every factor keeps full column rank
    (with M above a dim's node count the reduced systems lose conditioning and the
    ~5e-13 agreement of the two sides' bands grows past 1e-10 within three sweeps)."""
    from paper_2503_13933_gb300 import slabs as S
    M, tdim = 5, 3
    kw = dict(n_xy=20, n_z=10, n_t=8, n_par=6, n_slabs=8)
    d0 = W.lpbf_slab(slab=0, **kw)
    P0, P0o = T.Problem(d0), O.problem_from_description(d0)
    U0 = W.random_factors(d0, M, seed=4)
    U = P0.factors(M)
    U.set(U0)
    P0.sweep(U, 3, solver=T.SOLVER_FASTDIAG)
    Uo = [u.copy() for u in U0]
    for _ in range(3):
        Uo, _ = O.sweep(P0o, Uo, solver="fastdiag")
    g0 = U.get()
    assert rel(O.cp_full(g0), O.cp_full(Uo)) < 1e-10
    d1 = W.lpbf_slab(slab=1, **kw)
    d1g = S.next_slab(d1, S.end_state(g0, tdim), 0.0)
    d1o = O.slab_next_description(d1, O.slab_end_state(Uo, tdim), tdim, 0.0)
    assert len(d1g["sources"]) == len(d1o["sources"]) == len(d1["sources"]) + 8 * M   # 8 terms without d/dt
    P1, P1o = T.Problem(d1g), O.problem_from_description(d1o)
    V0 = W.random_factors(d1g, M, seed=5)
    V = P1.factors(M)
    V.set(V0)
    P1.sweep(V, 3, solver=T.SOLVER_FASTDIAG)
    Vo = [v.copy() for v in V0]
    for _ in range(3):
        Vo, _ = O.sweep(P1o, Vo, solver="fastdiag")
    assert rel(O.cp_full(V.get()), O.cp_full(Vo)) < 1e-9


def test_lpbf_slab_block_elimination_matches_oracle(T):
    """The same sweeps with block elimination everywhere (the plain path)."""
    desc = W.lpbf_slab(n_xy=16, n_z=10, n_t=8, n_par=6)
    P = T.Problem(desc)
    Po = O.problem_from_description(desc)
    M = 4
    U0 = W.random_factors(desc, M, seed=13)
    U = P.factors(M)
    U.set(U0)
    P.sweep(U, 2, solver=T.SOLVER_BLOCK_LU)
    Uo = [u.copy() for u in U0]
    for _ in range(2):
        Uo, _ = O.sweep(Po, Uo, solver="banded")
    got = U.get()
    for d in range(7):
        assert rel(got[d], Uo[d]) < 1e-10, (d, rel(got[d], Uo[d]))
