"""The N > 1 path of bench.py on CPU: two gloo ranks (world size 2, 127.0.0.1).

The filter does not shard (one problem per GPU; the paper's multi-node decomposition has
nothing to split on one GPU), so N GPUs run N independent replicas: a barrier around the
timed region, the slowest rank's time, and the whole-job rate = units of all ranks / that
time.  The reference arm runs on rank 0 only.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, got_local = bench._dist()
        bench._barrier(ws)
        slowest = bench._max_over_ranks(10.0 + 5.0 * rank, ws)     # rank 1 is the slow one
        rate = bench.whole_job_rate(1e9, ws, slowest)
        ref = bench.run_reference(type("A", (), {"workload": "tiny", "warmup": 0, "steps": 1})(), ws, rank) \
            if rank == 1 else "skipped"
        q.put((rank, got_ws, got_rank, got_local, slowest, rate, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, local, slowest, rate, ref in out:
        assert (ws, r, local) == (2, rank, rank)
        assert slowest == 15.0                      # max over ranks, on both ranks
        assert rate == pytest.approx(2 * 1e9 / 15e-3 / 1e9)
    assert out[1][6] is None                        # the reference arm does no work on rank 1


def test_single_rank_helpers():
    import bench
    assert bench._max_over_ranks(3.5, 1) == 3.5
    bench._barrier(1)
    assert bench.whole_job_rate(2e9, 1, 1000.0) == pytest.approx(2.0)
