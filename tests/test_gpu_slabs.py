"""Slab chaining on the GPU (Eq. 16 by lifting) against the oracle's own chaining."""
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


def test_two_slabs_match_the_oracle(T):
    """2D heat with a convection face, two slabs of 6 modes, the same seeded factors on
    both sides for 4 sweeps each: the lifting sources and slab-2 factors agree."""
    from paper_2503_13933_gb300 import slabs as S
    desc = W.heat_transient(n_space=12, n_t=8, D_space=2, T=0.5, h_conv=2.0, seed=3040)
    M, tdim = 6, 2
    # slab 1
    P1, P1o = T.Problem(desc), O.problem_from_description(desc)
    U0 = W.random_factors(desc, M, seed=1)
    U1 = P1.factors(M)
    U1.set(U0)
    P1.sweep(U1, 4)
    U1o = [u.copy() for u in U0]
    for _ in range(4):
        U1o, _ = O.sweep(P1o, U1o)
    g1 = U1.get()
    # slab 2 descriptions from each side's own chaining code
    d2 = S.next_slab(desc, S.end_state(g1, tdim), 0.5)
    d2o = O.slab_next_description(desc, O.slab_end_state(U1o, tdim), tdim, 0.5)
    assert len(d2["sources"]) == len(d2o["sources"]) == len(desc["sources"]) + 3 * M
    P2, P2o = T.Problem(d2), O.problem_from_description(d2o)
    for r in range(len(d2["sources"])):
        for d in range(3):
            q, qo = P2.source(r, d), P2o.sources[r][1][d]
            assert np.max(np.abs(q - qo)) <= 1e-9 * max(1.0, np.max(np.abs(qo)))
    V0 = W.random_factors(d2, M, seed=2)
    U2 = P2.factors(M)
    U2.set(V0)
    P2.sweep(U2, 4)
    U2o = [u.copy() for u in V0]
    for _ in range(4):
        U2o, _ = O.sweep(P2o, U2o)
    a, b = O.cp_full(U2.get()), O.cp_full(U2o)
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)


def test_mode_compression_matches_oracle(T):
    """App. B: an end state of 10 modes on a 3-space-dim slab compressed to 4 modes on
    the GPU and in the oracle, from the same initial factors and for the same number
    of sweeps: the same compressed field."""
    from paper_2503_13933_gb300 import slabs as S
    desc = W.heat_transient(n_space=11, n_t=6, D_space=3, seed=3050)
    rng = np.random.default_rng(3)
    nf = [W.n_free(dm) for dm in desc["dims"]]
    facs = [rng.uniform(-1, 1, (nf[d], 10)) if d < 3 else None for d in range(4)]
    wts = rng.uniform(0.5, 1.5, 10)
    sg = S.EndState(facs, wts, 3)
    U0 = W.random_factors(dict(dims=desc["dims"][:3]), 4, seed=8)
    cg = S.compress(desc, sg, U0, sweeps=6)
    co = O.slab_compress(desc, (facs, wts), 3, U0, sweeps=6)
    fg = np.einsum("im,jm,km,m->ijk", cg.U[0], cg.U[1], cg.U[2], cg.weight)
    fo = np.einsum("im,jm,km,m->ijk", co[0][0], co[0][1], co[0][2], co[1])
    assert np.linalg.norm(fg - fo) <= 1e-10 * np.linalg.norm(fo)
    # a 4-mode approximation of a rank-10 field: closer to it than the zero field
    fe = np.einsum("im,jm,km,m->ijk", facs[0], facs[1], facs[2], wts)
    assert np.linalg.norm(fg - fe) < np.linalg.norm(fe)
