"""The multi-rank host logic of bench.py (one process per GPU, one shard of the
seeded batch per rank) on CPU: two gloo ranks rendezvous on 127.0.0.1, take
disjoint contiguous instance shards of one seeded sequence, take the maximum of
their step times, sum their statistics and report the whole-job rate.  No GPU
and no compute kernels."""
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
    shard = bench.shard_instances(got_ws, got_rank, n=8)
    its = bench.allreduce_sum(got_ws, float(3 + rank))  # per-rank statistics gathered after timing
    out.put((got_rank, got_ws, slowest, bench.job_rate(got_ws, slowest, len(shard)), shard, its))
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
    for _, ws, slowest, rate, shard, its in res:
        assert ws == 2 and slowest == 15.0 and its == 7.0
        assert rate == pytest.approx(2 * 8 * 1e3 / 15.0)
    # the shards are disjoint and together the seeded sequence of 16 instances;
    # rank 0's shard is the one-GPU batch
    from paper_2303_03848_b300 import synth

    whole = synth.batched_instances(0, 16, **__import__("bench").BATCH)
    assert res[0][4] + res[1][4] == whole
    assert res[0][4] == synth.batched_instances(0, 8, **__import__("bench").BATCH)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.allreduce_max(1, 3.5) == 3.5
    assert bench.allreduce_sum(1, 3.5) == 3.5
    assert bench.job_rate(1, 50.0) == pytest.approx(20.0)
    assert bench.job_rate(1, 500.0, 4096) == pytest.approx(8192.0)


def test_executed_point_steps_count_the_live_slices():
    # iteration k (0-based) propagates slices k..P-1: K iterations of an instance
    # execute sum_{k<K} (P - k) slice propagations of (Nx - 2) x steps point-steps
    import bench

    insts = [dict(Nx=10, P=4, fine_steps=3), dict(Nx=6, P=2, fine_steps=5)]
    assert bench.executed_pt_steps(insts, [2, 1]) == 8 * 3 * (4 + 3) + 4 * 5 * 2
