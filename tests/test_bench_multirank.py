"""The multi-rank host logic of bench.py on CPU: two gloo ranks (no GPU).
Replicas register distinct pairs, the timing is the maximum over ranks and
the job value aggregates every rank's registrations; the reference arm runs
on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = bench.rank_seeds(rank, (1, 2, 3))
    mine = 10.0 + 5.0 * rank            # rank 1 is the slower one
    slowest = bench.max_over_ranks(mine, world)
    ms_reg, ms_step, rate = bench.aggregate(slowest, 4, 3, world, 1000, 10, 10)
    out.put((rank, seeds, slowest, ms_reg, ms_step, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, reg0, st0, rate0), (r1, s1, m1, reg1, st1, rate1) = res
    assert not set(s0) & set(s1)                 # distinct pairs per rank
    assert m0 == m1 == 15.0                       # max over ranks, seen by all
    assert reg0 == pytest.approx(15.0 / (4 * 3 * 2))
    assert st0 == pytest.approx(15.0 / 4)
    assert rate0 == pytest.approx(1000 * 100 * 24 / 0.015)


def test_reference_arm_other_ranks_do_nothing(capsys):
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(A(), rank=1) is None
    assert capsys.readouterr().out == ""
