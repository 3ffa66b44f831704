"""Direction sharding across processes, one GPU each.

Each process sweeps a share of the direction set: a problem built on a quadrature that holds
only those directions (explicit omega and w, tf_quadrature_create).  Its scalar flux is then a
partial quadrature sum (Eq. (2) over its own directions), and the library hands that partial
flux, and the step's boundary leakage, to a reduce function after every transport step
(tf_problem_set_reduce); `TorchAllreduce` is such a function: one in-place sum over the process
group on the library's stream (NCCL on GPUs).  Every process then continues from the same full
flux and takes the same stopping decision.

This module partitions and marshals; the sum itself is torch.distributed's collective.
"""
from __future__ import annotations

import numpy as np


def direction_shard(n_dirs: int, rank: int, world: int) -> np.ndarray:
    """Indices of the directions rank `rank` of `world` sweeps: every world-th direction from
    `rank` on, so each share mixes all octants and the shares differ in size by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    if n_dirs < world:
        raise ValueError("fewer directions than ranks")
    return np.arange(rank, n_dirs, world)


def shard_quadrature(omega: np.ndarray, w: np.ndarray, rank: int, world: int):
    """(omega, w) of rank `rank`'s share of a direction set."""
    idx = direction_shard(len(w), rank, world)
    return np.ascontiguousarray(omega[idx]), np.ascontiguousarray(w[idx])


class _DeviceBuffer:
    """A device array of `count` doubles at `ptr`, seen by torch without a copy."""

    def __init__(self, ptr: int, count: int):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None, "stream": None}


class TorchAllreduce:
    """A tf_reduce_fn: sums the partial buffer at `ptr` over the processes of `group` (default:
    the world) with torch.distributed.all_reduce.  device "cuda": a device buffer, the sum
    enqueued on the library's stream (NCCL); "cpu": a host buffer (gloo), summed before
    returning."""

    def __init__(self, group=None, device: str = "cuda"):
        self.group = group
        self.device = device
        self.calls = 0

    def __call__(self, ptr: int, count: int, stream: int) -> int:
        import ctypes

        import torch
        import torch.distributed as dist
        try:
            if self.device == "cpu":
                t = torch.from_numpy(np.ctypeslib.as_array((ctypes.c_double * int(count)).from_address(int(ptr))))
                dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
            else:
                t = torch.as_tensor(_DeviceBuffer(ptr, count), device="cuda")
                s = torch.cuda.ExternalStream(int(stream)) if stream else torch.cuda.default_stream()
                with torch.cuda.stream(s):
                    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
            self.calls += 1
            return 0
        except Exception:  # the library turns a nonzero return into TF_ERR_CUDA
            return 1
