"""The N > 1 path of bench.py on CPU: two gloo ranks, max-over-ranks timing
and the whole-job (weak-scaling) rate.  The denoiser itself shards by image
(replicas, no data-path collective), so only the aggregation is exchanged."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 * (rank + 1), world)
    rate = bench.whole_job_rate(1_000_000, 4, world, ms)
    dist.barrier()
    q.put((rank, ms, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_and_weak_scaling_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [20.0, 20.0]
    # 2 ranks x 4 steps x 1 Mpix in 20 ms -> 400 Mpix/s
    assert got[0][2] == pytest.approx(400.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(2_000_000, 5, 1, 10.0) == pytest.approx(1000.0)


def test_cpu_baseline_block_reports_threads_and_single_thread_leg():
    """The bench's cpu_baseline: the oracle on all its threads (cores = the
    OpenMP thread count it used) plus a one-thread leg; thread count restored."""
    import bench
    import oracle as O
    before = O.max_threads()
    blk = bench.cpu_baseline_block(1, 0)
    assert blk["kind"] == "oracle" and blk["unit"] == "Mpix/s" and blk["value"] > 0
    assert blk["cores"] == before and blk["single_thread"]["cores"] == 1
    assert blk["single_thread"]["value"] > 0
    assert O.max_threads() == before
