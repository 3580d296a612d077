"""The bench's multi-rank path (one process per GPU, launched by torch.distributed.run)
exercised on the CPU with the gloo backend and two ranks: the rendezvous, the barrier,
the max over ranks of the timed values, the per-rank workload seeds (independent
instances, weak scaling, no data-path collective) and the reference arm's rank-0-only
output."""
import contextlib
import io
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2503_13933_gb300 import workloads as W
    r, w, local = bench.dist_init()
    assert (r, w, local) == (rank, world, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    # every rank reports the max over ranks of its own timing
    got = bench.allmax(1.5 + rank, w)
    # per-rank workloads: the single-instance seed and the batched instances differ by rank
    seed = bench.WORKLOAD["seed"] + rank
    desc = W.poisson_k(8, 4, seed=seed)
    descs, Ms = W.batch_instances(count=3, seed=4000 + 1000 * rank, n_lo=8, n_hi=12, M_lo=2, M_hi=3)
    # the reference arm: ranks other than 0 return at once without output
    buf = io.StringIO()
    if rank != 0:
        with contextlib.redirect_stdout(buf):
            bench.run_reference(None, rank, w)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(repr(dict(max=got, seed=seed, src=desc["sources"][0][0],
                          batch=[len(d["dims"]) for d in descs] + Ms, ref_out=buf.getvalue())))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [eval(open(tmp_path / f"rank{r}.txt").read()) for r in range(2)]
    assert res[0]["max"] == res[1]["max"] == 2.5
    assert res[0]["seed"] != res[1]["seed"]
    assert res[0]["src"] != res[1]["src"] or res[0]["batch"] != res[1]["batch"]
    assert res[1]["ref_out"] == ""
