"""The multi-rank host logic of bench.py (one process per GPU, replicas) on CPU:
two gloo ranks rendezvous on 127.0.0.1, take the maximum of their step times
and report the whole-job rate.  No GPU and no compute kernels."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(WORLD_SIZE=str(ws), RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench

    got_ws, got_rank, _ = bench.dist_setup()
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    slowest = bench.allreduce_max(got_ws, ms)
    bench.barrier(got_ws)
    out.put((got_rank, got_ws, slowest, bench.job_rate(got_ws, slowest)))
    import torch.distributed as dist

    dist.destroy_process_group()


@pytest.mark.skipif(torch.cuda.is_available(), reason="exercises the gloo fallback of the host logic")
def test_two_gloo_ranks_take_the_slowest_step_and_report_the_whole_job():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for _, ws, slowest, rate in res:
        assert ws == 2 and slowest == 15.0
        assert rate == pytest.approx(2 * 1e3 / 15.0)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.allreduce_max(1, 3.5) == 3.5
    assert bench.job_rate(1, 50.0) == pytest.approx(20.0)
