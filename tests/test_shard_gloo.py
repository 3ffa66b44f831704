"""Direction sharding, on the CPU with two gloo ranks: the partition of a direction set and the
partner sum of the partial scalar flux (paper_2510_11513_gb300.shard).  Each rank sweeps its
share of the directions with the oracle; the sum over ranks of the partial fluxes (Eq. (2) over
each share) must be the oracle's flux over the whole set, and the rank shares must cover the set
exactly once."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cfg():
    import workloads as W
    return W.two_material_box(n=4, G=4, n_polar=4, n_az=8, precision="f64")


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import oracle
    from paper_2510_11513_gb300 import shard

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg = _cfg()
        om, w = oracle.product_quadrature(cfg["n_polar"], cfg["n_azimuthal"])
        o_r, w_r = shard.shard_quadrature(om, w, rank, world)
        P = oracle.Problem(cfg, omega=o_r, w=w_r)
        phi_in = np.random.default_rng(3).uniform(0.0, 1.0, (P.C, P.G, 4))  # the same on every rank
        part = np.ascontiguousarray(P.transport_step(phi_in, threads=1))
        hook = shard.TorchAllreduce(device="cpu")
        assert hook(part.ctypes.data, part.size, 0) == 0 and hook.calls == 1
        out[rank] = (shard.direction_shard(len(w), rank, world).tolist(), float(w_r.sum()), part)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_partial_fluxes_sum_to_the_whole_set(world):
    import oracle

    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    cfg = _cfg()
    om, w = oracle.product_quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    idx = sorted(i for r in range(world) for i in out[r][0])
    assert idx == list(range(len(w)))  # every direction exactly once
    assert abs(sum(out[r][1] for r in range(world)) - 4.0 * np.pi) < 1e-12
    P = oracle.Problem(cfg)
    phi_in = np.random.default_rng(3).uniform(0.0, 1.0, (P.C, P.G, 4))
    ref = P.transport_step(phi_in, threads=1)
    for r in range(world):
        got = out[r][2]
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-13  # every rank holds the full flux


def test_direction_shard_arguments():
    from paper_2510_11513_gb300 import shard
    assert shard.direction_shard(5, 0, 2).tolist() == [0, 2, 4]
    assert shard.direction_shard(5, 1, 2).tolist() == [1, 3]
    for bad in ((5, 2, 2), (5, -1, 2), (1, 0, 2)):
        with pytest.raises(ValueError):
            shard.direction_shard(*bad)
