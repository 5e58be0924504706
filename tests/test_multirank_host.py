"""The N > 1 path on the CPU (gloo, world size 2, 127.0.0.1).

The SPDHG+ path does not shard: `bench.py --gpus N` runs N independent replicas (weak scaling),
with no collective on the data path.  What the ranks share is host logic, tested here: the
timing of the job is the maximum over ranks, the whole-job rate is N x (units per rank) / that
time, and the reference arm runs on rank 0 alone (the other ranks return 0 without work).
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = 100.0 + 50.0 * rank                        # rank 1 is the slow one
    t = bench.max_over_ranks(ms)
    env = bench.dist_env()

    class Args:
        steps, warmup = 3, 3
    ref = bench.run_reference(Args()) if rank != 0 else None   # rank 0 would run the oracle
    out.put((rank, t, bench.aggregate_rate(5, ws, t / 1e3), env, ref))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_and_skip_the_reference_off_rank_0():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate, env, ref in res:
        assert t == 150.0                              # max over ranks
        assert rate == pytest.approx(2 * 5 / 0.150)    # whole-job units per second
        assert env == (ws, rank, rank)
    assert res[1][4] == 0                              # rank 1: reference arm returns 0, no work
