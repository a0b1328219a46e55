"""The benchmark's multi-rank logic on CPU: two gloo ranks (one process
each, rendezvous on 127.0.0.1) join the process group the way bench.py
does under torchrun, meet at the barrier, and agree on the job's time (the
slowest rank's) and on the whole-job rate of independent replicas."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_setup()
    import torch.distributed as dist
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    # rank k took (k + 1) * 100 ms for its 10 steps: the job took 200 ms
    rate, total_ms = bench.job_rate(100.0 * (r + 1), 10, w)
    # the reference arm: only rank 0 does work; the others return at once
    other = bench.run_reference(None, r, w) if r != 0 else None
    out.put((r, w, local, total_ms, rate, other))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_job_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    for r in res:
        assert r[3] == pytest.approx(200.0)
        assert r[4] == pytest.approx(2 * 10 / 0.2)   # both replicas' steps over the slowest rank's time
    assert res[1][5] is None
