"""The bench's multi-rank path (one process per GPU, launched by torch.distributed.run)
exercised on the CPU with the gloo backend and two ranks: the rendezvous, the barrier,
the max over ranks of the timed values, the per-rank workload seeds (independent
instances, weak scaling, no data-path collective), the partition of a fixed set of batched
instances over the ranks with the host gather of their reports, and the reference arm's
rank-0-only output."""
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
    # per-rank workloads: the single-instance seed differs by rank (replicas)
    seed = bench.WORKLOAD["seed"] + rank
    desc = W.poisson_k(8, 4, seed=seed)
    # a fixed set of batched instances partitioned over the ranks; per-instance reports
    # (index, status, change) gathered on the host
    count = 11
    mine = bench.partition(count, rank, w)
    gathered = bench.gather_reports([(i, -2 if i == 7 else 0, 0.1 * i) for i in mine], w)
    # the reference arm: ranks other than 0 return at once without output
    buf = io.StringIO()
    if rank != 0:
        with contextlib.redirect_stdout(buf):
            bench.run_reference(None, rank, w)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(repr(dict(max=got, seed=seed, src=desc["sources"][0][0],
                          ref_out=buf.getvalue(),
                          mine=mine, gathered=gathered)))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [eval(open(tmp_path / f"rank{r}.txt").read()) for r in range(2)]
    assert res[0]["max"] == res[1]["max"] == 2.5
    assert res[0]["seed"] != res[1]["seed"]
    assert res[0]["src"] != res[1]["src"]
    assert res[1]["ref_out"] == ""
    # the partition covers the fixed set exactly once; every rank holds the complete,
    # ordered gather of all ranks' reports
    assert sorted(res[0]["mine"] + res[1]["mine"]) == list(range(11))
    assert not set(res[0]["mine"]) & set(res[1]["mine"])
    for r in res:
        assert [g[0] for g in r["gathered"]] == list(range(11))
        assert [g[1] for g in r["gathered"]] == [-2 if i == 7 else 0 for i in range(11)]
        assert r["gathered"] == res[0]["gathered"]
