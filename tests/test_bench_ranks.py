"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

bench.py --gpus N runs N independent replicas (the workload has no exchange
step between lattices); what the ranks share is host logic: the process
group, barriers, the maximum time over ranks, the whole-job throughput, and
the reference arm printed by rank 0 alone.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup(world)
    try:
        assert (w, r) == (world, rank) and dist.get_backend() == "gloo"
        bench.barrier(w)
        t = bench.max_over_ranks(w, 1.5 + rank)   # rank 1 is the slow one
        rate = bench.job_value(1e6, w, t)
        # the sharded ensemble's host logic: summed updates, gathered rows
        total = bench.sum_over_ranks(w, 10.0 * (rank + 1))
        rows = bench.gather_lists(w, [(rank, k) for k in range(rank + 1)])
        # the reference arm: rank 0 alone runs and prints
        buf = io.StringIO()

        class A:
            steps, warmup = 1, 0
        bench.W = dict(bench.W, nx=16, ny=16, nz=16)
        bench.CELLS = 16 ** 3
        with redirect_stdout(buf):
            bench.run_reference(A, w, r)
        out.put((r, t, rate, buf.getvalue(), total, rows))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, o0, s0, g0), (r1, t1, v1, o1, s1, g1) = res
    assert s0 == s1 == 30.0                        # sum over ranks
    assert g0 == g1 == [(0, 0), (1, 0), (1, 1)]    # every rank's rows, rank order
    assert t0 == t1 == 2.5                         # max over ranks
    assert v0 == v1 == pytest.approx(2e6 / 2.5 / 1e6)  # both replicas' units / slowest time
    assert '"impl": "reference"' in o0 and o1 == ""   # rank 0 prints, rank 1 does no work


def test_ensemble_shards_cover_the_domains_once():
    """The ensemble's domains over N ranks: disjoint shards that together
    are all domains, each with a like share of the cells."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1708_01608_gb300.workloads import ENSEMBLE_256, ensemble_domains
    doms = ensemble_domains(ENSEMBLE_256)
    total = sum(d["nx"] * d["ny"] for d in doms)
    for world in (1, 2, 4, 8):
        shards = [bench.ensemble_shard(doms, world, r) for r in range(world)]
        seen = sorted(id(d) for sh in shards for d in sh)
        assert seen == sorted(id(d) for d in doms)
        cells = [sum(d["nx"] * d["ny"] for d in sh) for sh in shards]
        assert sum(cells) == total
        assert max(cells) - min(cells) <= max(d["nx"] * d["ny"] for d in doms)
