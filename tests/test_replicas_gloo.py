"""The multi-rank bookkeeping of bench.py, run as two gloo ranks on the CPU: barrier, max over
ranks of the timed region, and the whole-job grind time over the job's units (replicas: every
rank's problem; direction sharding: the one shared problem)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench

    w, r, local = bench._dist()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        bench._barrier(w)
        ms = 10.0 * (r + 1)  # rank 1 is the slower one
        mx = bench._max_over_ranks(w, ms)
        out[r] = (w, r, local, mx, bench.whole_job_grind(mx, bench.job_units(1000, w, False)),
                  bench.whole_job_grind(mx, bench.job_units(1000, w, True)))
        bench._barrier(w)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_and_whole_job_value():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        w, rr, local, mx, value, value_sharded = out[r]
        assert (w, rr, local) == (world, r, r)
        assert mx == 20.0  # max over ranks
        assert abs(value - 20.0 * 1e6 / 2000) < 1e-9  # replicas: both ranks' units over the slowest time
        assert abs(value_sharded - 20.0 * 1e6 / 1000) < 1e-9  # directions shared: the one problem's units


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse

    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(config="small_box", n=0, groups=0, polar=0, azimuthal=0, order=1, warmup=3, steps=1,
                              gpus=2)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
