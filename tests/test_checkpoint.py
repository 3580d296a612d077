"""Checkpoint round trip of a problem description with every source kind (CPU), and a
resumed solve on the GPU that continues exactly where the interrupted one stopped."""
import json

import numpy as np
import pytest

from paper_2503_13933_gb300 import checkpoint as C
from paper_2503_13933_gb300 import workloads as W


class _FakeFactors:
    def __init__(self, facs):
        self.facs = facs

    def get(self):
        return [f.copy() for f in self.facs]


def test_checkpoint_round_trip(tmp_path):
    desc = W.lpbf_slab(n_xy=10, n_z=8, n_t=6, n_par=3)
    from paper_2503_13933_gb300 import slabs as S
    st = S.EndState([np.ones((W.n_free(dm), 2)) if d != 3 else None for d, dm in enumerate(desc["dims"])],
                    [0.5, 1.5], 3)
    desc = S.next_slab(desc, st, 0.0)      # adds opvec sources
    facs = W.random_factors(desc, 3, seed=1)
    p = tmp_path / "ck.npz"
    C.save(p, desc, _FakeFactors(facs), history=[(3, 0.5, 0.1)], sweeps_done=4)
    d2, f2, done, hist = C.load(p)
    assert done == 4 and hist == [(3, 0.5, 0.1)]
    assert all(np.array_equal(a, b) for a, b in zip(facs, f2))
    assert d2["dims"] == [dict(dm, weight_poly=tuple(dm["weight_poly"])) for dm in desc["dims"]]
    assert [list(t[1]) for t in d2["terms"]] == [list(t[1]) for t in desc["terms"]]
    assert len(d2["sources"]) == len(desc["sources"])
    for (b1, f1), (b2, g2) in zip(desc["sources"], d2["sources"]):
        assert b1 == b2
        for (k1, p1), (k2, p2) in zip(f1, g2):
            assert k1 == k2
            if k1 == "nodal":
                assert np.array_equal(np.asarray(p1), p2)
            elif k1 == "opvec":
                assert p1[0] == p2[0] and np.array_equal(np.asarray(p1[1]), p2[1])
            else:
                assert tuple(float(v) for v in p1) == tuple(p2)


def test_history_jsonl(tmp_path):
    p = tmp_path / "h.jsonl"
    C.write_history_jsonl(p, dict(history=[(2, 0.3, 1e-2), (2, 0.1, 1e-3)]))
    lines = [json.loads(s) for s in open(p)]
    assert lines[1] == dict(sweep=2, M=2, change=0.1, rho=1e-3)


@pytest.mark.gpu
def test_resumed_solve_continues_exactly(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_13933_gb300 import build, taps
    import os
    if not os.path.exists(taps.LIB_PATH):
        build.build()
    desc = W.poisson_k(n_space=14, n_k=8, seed=2030)
    U0 = W.random_factors(desc, 4, seed=3)
    P = taps.Problem(desc)
    U = P.factors(4)
    U.set(U0)
    P.sweep(U, 5, solver=taps.SOLVER_FASTDIAG)
    straight = U.get()
    P2 = taps.Problem(desc)
    U2 = P2.factors(4)
    U2.set(U0)
    P2.sweep(U2, 2, solver=taps.SOLVER_FASTDIAG)
    C.save(tmp_path / "ck.npz", desc, U2, sweeps_done=2)
    P3, U3, done, _ = C.resume(tmp_path / "ck.npz")
    P3.sweep(U3, 5 - done, solver=taps.SOLVER_FASTDIAG)
    for a, b in zip(straight, U3.get()):
        assert np.array_equal(a, b)
