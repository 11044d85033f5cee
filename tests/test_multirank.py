"""The multi-rank plumbing of bench.py on CPU with two gloo ranks: the slowest
rank's time is what every rank reports, whole-job time per frame counts every
replica's frames, and the reference arm does no work on ranks other than 0."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.rank_env()
        t = bench.max_over_ranks(10.0 + 5.0 * rank, w)     # rank 1 is the slower replica
        v = bench.replica_ms_per_frame(t, 20, w)
        dist.barrier()
        out[rank] = (w, r, lr, t, v)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_replica():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][:3] == (2, 0, 0) and res[1][:3] == (2, 1, 1)
    assert res[0][3] == res[1][3] == 15.0
    assert res[0][4] == res[1][4] == pytest.approx(15.0 / 40)


def test_reference_arm_is_rank_zero_only(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload, warmup, steps, gpus = "tiny", 1, 1, 2

    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""


def test_single_rank_is_a_no_op():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_ms_per_frame(30.0, 10, 1) == 3.0
