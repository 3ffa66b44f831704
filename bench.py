"""Benchmark: sweep grind time of the unstructured S_N transport sweep on GB300.

One "step" is one source iteration: source update, the persistent sweep of
every direction, the phi reduction, and the FP64 stopping test.  The default
workload is the corner-source box: 48^3 jittered hexes Kuhn-split into
663,552 tetrahedra, 192 directions (12 polar x 16 azimuthal), 64 groups, FP32
local solves with FP64 phi/residual.  The metric is grind time: nanoseconds
per (cell, direction, group) unit; lower is better.

Prints one JSON line (rank 0).  With torchrun, N ranks run N independent
replicas (the path does not shard across GPUs) and the slowest rank's time
is reported; `value` counts all ranks' units.

--impl reference times the CPU oracle (the plain FP64 program) on a bounded
sample of the same workload, on this machine's host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "sweep grind time ns/(cell·dir·group) and time-to-1e-6 vs plain FP64 GPU"
UNIT = "ns/(cell·dir·group)"
L2_BYTES = 129 * 1024 * 1024


def kernel_source_sha1(sources):
    """SHA-1 over a kernel variant's device sources (files of csrc/, concatenated in order)."""
    import hashlib
    h = hashlib.sha1()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2510_11513_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic(workload, precision, kernel_label, units):
    """DRAM bytes (read + write) of one sweep-kernel launch of `units` units on `workload`, from
    the committed one-pass ncu record of that kernel variant (profiles/traffic_*.json) whose
    source files still hash to the recorded SHA-1: the record's bytes per unit, captured on the
    workload itself or on a smaller case of it that the record names (scaled by the units of one
    launch); None when no current record applies."""
    import glob
    for f in glob.glob(os.path.join(ROOT, "profiles", "traffic_*.json")):
        try:
            rec = json.load(open(f))
            sha = kernel_source_sha1(rec["kernel_sources"])
        except (OSError, ValueError, KeyError):
            continue
        if (workload in rec.get("applies_to", []) and rec.get("precision") == precision
                and rec.get("kernel_source_sha1") == sha and rec.get("kernel") == kernel_label):
            per_unit = (rec["dram_bytes_read"] + rec["dram_bytes_write"]) / rec["units_per_launch"]
            return per_unit * units
    return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for k, n in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_units(units_per_rank, world, sharded):
    """Units the whole job processes per step: with direction sharding the ranks share one
    problem (each sweeps its directions), so the job's units are the sum of the ranks' shares;
    replicas each solve the whole problem, world times the units."""
    return units_per_rank * world if not sharded else units_per_rank


def whole_job_grind(ms_per_step, units_job):
    """Grind time of the whole job (ns per unit) from the slowest rank's time per step."""
    return ms_per_step * 1e6 / units_job


def cpu_oracle_sample(cfg, n_dirs=None, threads=None, groups=16):
    """Oracle (plain FP64 CPU) grind time on a bounded sample: `n_dirs` directions of the
    workload's quadrature and its first `groups` energy groups (all cells), one source
    update + sweep.  Each oracle thread sweeps whole directions, so the wall time of a
    sample is about one direction's sweep of the sampled groups."""
    import oracle
    threads = threads or os.cpu_count() or 1
    n_dirs = n_dirs or threads
    G = int(cfg["n_groups"])
    if groups and groups < G:
        cfg = dict(cfg, n_groups=groups, sigma_t=np.ascontiguousarray(cfg["sigma_t"][:, :groups]),
                   sigma_s=np.ascontiguousarray(cfg["sigma_s"][:, :groups, :groups]),
                   Q=np.ascontiguousarray(cfg["Q"][:, :groups]))
    om, w = oracle.product_quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    D = om.shape[0]
    idx = np.linspace(0, D - 1, n_dirs).round().astype(int)
    order = cfg.get("order", 1)
    if order == 2:
        from oracle import p2 as o2
        P = o2.Problem2(cfg, omega=om[idx], w=w[idx])
    elif order == 3:
        from oracle import p3 as o3
        P = o3.Problem3(cfg, omega=om[idx], w=w[idx])
    else:
        P = oracle.Problem(cfg, omega=om[idx], w=w[idx])
    nodes = {2: 10, 3: 20}.get(order, 4)
    phi = np.random.default_rng(0).uniform(0.0, 1.0, (P.C, P.G, nodes))
    t0 = time.perf_counter()
    q = P.source(phi)
    _, _, used = P.sweep(q, threads=threads)
    dt = time.perf_counter() - t0
    units = P.C * P.G * n_dirs
    return {"value": dt / units * 1e9, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{n_dirs} of {D} directions x {P.C} cells x {P.G} of {G} groups, one source update + sweep, "
                      f"{dt:.1f} s wall on {used} threads"}


def cpu_baseline(cfg, repeats=3):
    """The oracle's grind time on this machine's cores: the median of `repeats` all-core samples
    (their spread alongside) and one single-thread sample (one direction, the first 16 groups)."""
    runs = [cpu_oracle_sample(cfg) for _ in range(repeats)]
    vals = sorted(r["value"] for r in runs)
    out = dict(runs[0])
    out["value"] = statistics.median(vals)
    out["spread"] = {"min": vals[0], "max": vals[-1], "samples": len(vals)}
    one = cpu_oracle_sample(cfg, n_dirs=1, threads=1)
    out["single_thread"] = {"value": one["value"], "unit": one["unit"], "cores": one["cores"], "sample": one["sample"]}
    return out


def make_config(args):
    """The named workload, optionally resized (--n, --groups, --polar, --azimuthal) for profiling runs."""
    kw = {}
    if args.n:
        kw["n"] = args.n
    if args.groups:
        kw["G"] = args.groups
    if args.polar:
        kw["n_polar"] = args.polar
    if args.azimuthal:
        kw["n_az"] = args.azimuthal
    return W.CONFIGS[args.config](**kw)


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    cfg = make_config(args)
    if args.order >= 2:
        cfg = (W.order2 if args.order == 2 else W.order3)(cfg)
    threads = os.cpu_count() or 1
    # warm-up steps (untimed), then timed steps; each step is a bounded sample
    for _ in range(args.warmup):
        cpu_oracle_sample(cfg, n_dirs=threads, threads=threads, groups=2)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_oracle_sample(cfg, n_dirs=threads, threads=threads)
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / max(args.steps, 1) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "cells": len(cfg["tets"]),
                       "directions": cfg["n_polar"] * cfg["n_azimuthal"], "groups": cfg["n_groups"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"],
                             "spread": {"min": float(min(vals)), "max": float(max(vals)), "samples": len(vals)}},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SCHEDULES = {"amt": 0, "bsp": 1, "bsp_launch": 2}


def _schedule_leg(tf, cfg, prec, local, stream, steps, schedule, torch):
    """One schedule on one workload: warm-up sweep, then `steps` source iterations
    timed with CUDA events; returns ms per step, sweep-kernel ms and warp-time split."""
    dev = torch.device("cuda", local)
    pr = tf.Problem.from_config(cfg, precision=prec, device=local, schedule=SCHEDULES[schedule],
                                order=cfg.get("order", 1))
    ph = torch.zeros((pr.n_cells, pr.n_groups, pr.n_nodes), dtype=torch.float64, device=dev)
    pr.source_iterate(ph, 0.0, 1, stream=stream)
    st0 = pr.stats()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = pr.source_iterate(ph, 0.0, steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    st = pr.stats()
    ms = e0.elapsed_time(e1) / steps
    sweep_ms = (st["cum_sweep_event_seconds"] - st0["cum_sweep_event_seconds"]) / steps * 1e3
    out = {"ms_per_step": ms, "sweep_ms": sweep_ms, "grind": ms * 1e6 / pr.n_units,
           "warp_wait_frac": st["wait_seconds"] / max(st["wait_seconds"] + st["busy_seconds"], 1e-30),
           "n_buckets": st["n_buckets"], "launches_per_step": st["launches_per_step"],
           "grid_ctas": st["grid_ctas"], "cells_per_task": st["cells_per_task"], "iterations": r["iterations"]}
    pr.close()
    del pr, ph
    torch.cuda.synchronize(dev)
    return out


def schedule_ablation(tf, cfg, prec, local, stream, steps, torch, amt=None):
    """Many-task (AMT) against bulk-synchronous (BSP: grid barrier after every
    (octant, t-level) bucket; BSP_LAUNCH: one launch per bucket) on one workload.
    `amt` reuses a measurement of the AMT schedule made elsewhere."""
    res = {"workload": cfg["name"], "steps": steps}
    for name in ("amt", "bsp", "bsp_launch"):
        if name == "amt" and amt is not None:
            res[name] = amt
            continue
        res[name] = _schedule_leg(tf, cfg, prec, local, stream, steps, name, torch)
    for name in ("bsp", "bsp_launch"):
        res[f"amt_speedup_over_{name}"] = res[name]["ms_per_step"] / res["amt"]["ms_per_step"]
    return res


# FP32 peak of the CUDA cores: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz (maximum SM clock).
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _inflow_faces(prob, tf, nf):
    """Mean interior and boundary inflow faces per (cell, direction), from the sweep graph."""
    inflow, _ = tf.tf_graph_levels(prob.mesh.h, prob.quad.h, prob.n_cells, prob.n_dirs)
    nbr = prob.mesh.geometry()["nbr"]
    interior = (nbr >= 0).astype(np.uint8)  # [C][nf]
    n_in = sum(float((((inflow >> f) & 1) * interior[None, :, f]).mean()) for f in range(nf))
    n_bd = sum(float((((inflow >> f) & 1) * (1 - interior[None, :, f])).mean()) for f in range(nf))
    return n_in, n_bd


def p2_flops_per_unit(prob, tf, order=2):
    """Algorithmic (minimum) flops of one higher-order unit, an FMA counting 2.  Work that depends
    only on the cell and the direction (the streaming matrix V sum_k (Omega . grad lambda_k) C_k
    and the inflow face matrices |Omega . N_f| F_f: the group-independent part W of the matrix)
    is needed once per (cell, direction) and is divided by the group count G.  Per unit:
    A_g = W + sigma_t,g (V M) (one FMA per entry), b = (V M) q (one FMA per entry plus the
    scaling), the elimination without pivoting and the back substitution of an n x n system
    (sum_{m<n} m (2 m + 3) + n^2 flops), and per interior inflow face the face term F_f psi_up.
    Second order (n = 10): 200 + 210 + 815 per unit, 78 per face; 160 + 78 per face per
    (cell, direction).  Third order (n = 20): 800 + 820 + 5,910 per unit, 220 per face;
    3,624 + 200 per face per (cell, direction)."""
    n_in, _ = _inflow_faces(prob, tf, 4)
    G = prob.n_groups
    if order == 3:
        return 7530.0 + 220.0 * n_in + (3624.0 + 200.0 * n_in) / G, n_in
    return 1225.0 + 78.0 * n_in + (160.0 + 78.0 * n_in) / G, n_in


def hex_flops_per_unit(prob, tf):
    """Algorithmic (minimum) flops of one trilinear-hexahedron unit, an FMA counting 2.  Per unit:
    A_g = W + sigma_t,g M 128, b = M q 128, the 8 x 8 elimination 364 and back substitution 72,
    per interior inflow face the face term into b 32.  Per (cell, direction), divided by the group
    count G: the streaming matrix W = sum_d Omega_d G_d 384 and, per inflow face (interior or
    boundary), the 4 x 4 face matrix -Omega . F_f (80) added into W (16)."""
    n_in, n_bd = _inflow_faces(prob, tf, 6)
    G = prob.n_groups
    return 692.0 + 32.0 * n_in + (384.0 + 96.0 * (n_in + n_bd)) / G, n_in


def second_order_leg(tf, cfg, prec, local, stream, steps, torch, order=2):
    """A higher-order element (order 2: ten nodes, 3: twenty) on one workload: grind time
    of a source iteration and the sweep kernel's ALU roofline (bound by FP32 arithmetic:
    about 1,800 / 12,000 flops against 80-320 bytes per unit)."""
    dev = torch.device("cuda", local)
    pr = tf.Problem.from_config(cfg, precision=prec, device=local, order=1 if order == "hex" else order)
    ph = torch.zeros((pr.n_cells, pr.n_groups, pr.n_nodes), dtype=torch.float64, device=dev)
    pr.source_iterate(ph, 0.0, 1, stream=stream)
    st0 = pr.stats()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = pr.source_iterate(ph, 0.0, steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    st = pr.stats()
    ms = e0.elapsed_time(e1) / steps
    sweep_s = (st["cum_sweep_event_seconds"] - st0["cum_sweep_event_seconds"]) / steps
    flops, n_in = hex_flops_per_unit(pr, tf) if order == "hex" else p2_flops_per_unit(pr, tf, order)
    achieved = flops * pr.n_units / sweep_s / 1e12
    klabel = f"sweep_kernel<float, {st['kernel_mode']}>"
    out = {"workload": cfg["name"], "units_per_step": pr.n_units, "ms_per_step": ms,
           "grind": ms * 1e6 / pr.n_units, "unit": UNIT, "sweep_ms": sweep_s * 1e3,
           "phi_ms": (st["cum_phi_event_seconds"] - st0["cum_phi_event_seconds"]) / steps * 1e3,
           "cells_per_task": st["cells_per_task"], "balance": r["balance"],
           "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": achieved / FP32_ALU_PEAK_TFLOPS, "flops_per_unit": flops,
                        "mean_interior_inflow_faces": n_in, "kernel": klabel,
                        "traffic": _traffic(cfg["name"], "fp32", klabel, pr.n_units),
                        "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}}
    pr.close()
    del pr, ph
    torch.cuda.synchronize(dev)
    return out


def run_ours(args):
    import torch

    import paper_2510_11513_gb300 as tf

    world, rank, local = _dist()
    torch.cuda.set_device(local)  # before the process group: NCCL binds each rank to its current device
    if world > 1:
        import datetime

        import torch.distributed as dist
        # a rank that fails ends the others' next collective with an error instead of a long wait
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo",
                                timeout=datetime.timedelta(minutes=5))
    dev = torch.device("cuda", local)
    cfg = make_config(args)
    if args.order >= 2:
        cfg = (W.order2 if args.order == 2 else W.order3)(cfg)
    prec = tf.TF_FP64 if args.precision == "fp64" else tf.TF_FP32
    t_setup = time.perf_counter()
    # N > 1: each rank sweeps a share of the directions and the partial scalar fluxes are summed
    # over the ranks after every transport step (strong scaling), or (--shard replicas) each rank
    # solves the whole problem on its own (weak scaling)
    sharded = world > 1 and args.shard == "directions"
    qopts = {}
    if sharded:
        from paper_2510_11513_gb300 import shard
        om_all, w_all = tf.tf_quadrature_get(tf.Quadrature(cfg["n_polar"], cfg["n_azimuthal"]).h)
        qopts["omega"], qopts["w"] = shard.shard_quadrature(om_all, w_all, rank, world)
    prob = tf.Problem.from_config(cfg, precision=prec, device=local, cells_per_task=args.cells_per_task,
                                  warps_per_cta=args.warps_per_cta, octant_window=args.octant_window,
                                  keep_ready=args.keep_ready,
                                  staging=args.staging, pairing=args.pairing, schedule=SCHEDULES[args.schedule],
                                  order=args.order, task_shape=args.task_shape, patch_extent=args.patch_extent,
                                  **qopts)
    if sharded:
        prob.set_reduce(shard.TorchAllreduce())
    t_setup = time.perf_counter() - t_setup
    C, G, D = prob.n_cells, prob.n_groups, prob.n_dirs
    units = prob.n_units  # this rank's units per step
    D_job = cfg["n_polar"] * cfg["n_azimuthal"]
    # the whole job's units per step: all directions of the one problem (sharded), or every replica's
    units_job = job_units(C * D_job * G if sharded else units, world, sharded)
    stream = torch.cuda.current_stream(dev)
    nodes = prob.n_nodes
    phi = torch.zeros((C, G, nodes), dtype=torch.float64, device=dev)
    # warm-up: W source iterations from zero
    prob.source_iterate(phi, 0.0, args.warmup, stream=stream)
    st0 = prob.stats()
    clocks = ClockSampler(local)
    clocks.start()
    _barrier(world)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = prob.source_iterate(phi, 0.0, args.steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    _barrier(world)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms = _max_over_ranks(world, ms)
    st1 = prob.stats()
    assert res["iterations"] == args.steps
    ms_per_step = ms / args.steps
    grind = ms_per_step * 1e6 / units  # ns per unit (per GPU)
    value = whole_job_grind(ms_per_step, units_job)  # all ranks' units over the slowest rank's time
    sweep_s = (st1["cum_sweep_event_seconds"] - st0["cum_sweep_event_seconds"]) / args.steps
    phi_s = (st1["cum_phi_event_seconds"] - st0["cum_phi_event_seconds"]) / args.steps
    src_s = (st1["cum_source_event_seconds"] - st0["cum_source_event_seconds"]) / args.steps
    s = 4 if prec == tf.TF_FP32 else 8
    mode = st1["kernel_mode"]
    # algorithmic bytes of the sweep kernel per unit: q (4 s), psi store (4 s), and the
    # cell record + cell-list entry once per (cell, direction), amortised over G
    geo = 128 if prec == tf.TF_FP32 else 256
    b_unit = 8 * s + (geo + 4) / G
    if args.order >= 2:  # source and psi rows of NB nodes, the cell record + list entry per (cell, direction)
        b_unit = 2 * nodes * s + ((144 if args.order == 2 else 160) + 4) / G
    peak, peak_kind = _peaks()
    achieved = b_unit * units / sweep_s / 1e9
    klabel = ("sweep_kernel" if args.schedule == "amt" else "bsp_sweep_kernel") + \
        f"<{'float' if s == 4 else 'double'}, {mode}>"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None, "dtype": "f32" if prec == tf.TF_FP32 else "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "cells": C, "directions": D_job, "groups": G,
                       "units_per_step": units_job, "precision": args.precision, "phi_accumulate": "fp32-pair->fp64",
                       "l2": "inputs larger than L2 (psi store %.1f GB)" % (units * nodes * s / 1e9),
                       "element_order": args.order,
                       "parallelism": (f"directions{world}" if sharded else f"replicas{world}"),
                       "setup_s": round(t_setup, 2), "schedule": args.schedule,
                       "task_shape": "patches" if st1["task_shape"] == tf.TF_TASK_PATCHES else "t-level blocks"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": _traffic(cfg["name"], args.precision, klabel, units),
                         "kernel": klabel,
                         "bytes_per_unit": b_unit, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": b_unit * units},
            "breakdown_ms": {"source": src_s * 1e3, "sweep": sweep_s * 1e3, "phi": phi_s * 1e3,
                             "other": ms_per_step - (src_s + sweep_s + phi_s) * 1e3},
            "scheduling": {"n_tasks": st1["n_tasks"], "cells_per_task": st1["cells_per_task"],
                           "max_level": st1["max_level"], "grid_ctas": st1["grid_ctas"],
                           "warps_per_cta": st1["warps_per_cta"], "mean_ready": st1["mean_ready"],
                           "wait_frac": st1["wait_seconds"] / max(st1["wait_seconds"] + st1["busy_seconds"], 1e-30),
                           "data_wait_frac": st1["data_wait_seconds"] / max(st1["busy_seconds"], 1e-30),
                           "n_chunks": st1["n_chunks"], "octant_window": args.octant_window or 8,
                           "keep_ready": args.keep_ready or 1,
                           # mean task time of the last sweep and the critical-path bound
                           # (longest chain of t-levels x that time)
                           "mean_task_us": st1["busy_seconds"] * 1e6 / max(1, st1["tasks_executed"]),
                           "critical_path_ms": (st1["max_level"] + 1) * st1["busy_seconds"] * 1e3 /
                           max(1, st1["tasks_executed"])},
            "gpu_launches": int((st1["launches_per_step"] + 2) * args.steps),
            "clocks": clk}
    if args.order >= 2 and prec == tf.TF_FP32:
        # the higher-order kernels are bound by FP32 arithmetic, not by HBM
        flops, n_in = p2_flops_per_unit(prob, tf, args.order)
        ach = flops * units / sweep_s / 1e12
        line["roofline"] = {"bound": "alu", "achieved": ach, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": ach / FP32_ALU_PEAK_TFLOPS,
                            "traffic": _traffic(cfg["name"], args.precision, klabel, units), "kernel": klabel,
                            "flops_per_unit": flops, "mean_interior_inflow_faces": n_in,
                            "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                            "bytes_per_unit": b_unit, "hbm_achieved_gbs": achieved}
    # end to end: tf_sweep with pinned host buffers (H2D of phi_in, D2H of phi_out inside)
    if not args.no_e2e:
        hin = torch.zeros((C, G, nodes), dtype=torch.float64).pin_memory()
        hin.copy_(phi.cpu())
        hout = torch.zeros_like(hin).pin_memory()
        prob.sweep(hin, hout, stream=stream)
        torch.cuda.synchronize(dev)
        _barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            prob.sweep(hin, hout, stream=stream)
            hin, hout = hout, hin
        torch.cuda.synchronize(dev)
        _barrier(world)
        e2e_ms = _max_over_ranks(world, (time.perf_counter() - t0) * 1e3) / args.steps
        nbytes = C * G * nodes * 8
        line["e2e"] = {"value": whole_job_grind(e2e_ms, units_job), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                       "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_ms,
                       "call": "tf_sweep(host pinned phi_in, host pinned phi_out)"}
    amt_main = None
    if args.schedule == "amt":
        amt_main = {"ms_per_step": ms_per_step, "sweep_ms": sweep_s * 1e3, "grind": grind,
                    "warp_wait_frac": line["scheduling"]["wait_frac"], "n_buckets": 0,
                    "launches_per_step": st1["launches_per_step"], "grid_ctas": st1["grid_ctas"],
                    "cells_per_task": st1["cells_per_task"], "iterations": args.steps}
    prob.close()
    del prob
    torch.cuda.synchronize(dev)
    if not args.no_bsp_compare and world == 1 and args.order == 1:
        # the paper's comparison (Sec. 3.6): many-task against level-synchronous buckets,
        # on this workload and on the 16^3-hex one nearest the paper's own
        abl = [schedule_ablation(tf, cfg, prec, local, stream, args.bsp_steps, torch, amt_main)]
        abl.append(schedule_ablation(tf, W.paper_context_box(), prec, local, stream, 5, torch))
        # and with the second-order element, where each task carries about 20 x more arithmetic
        abl.append(schedule_ablation(tf, W.order2(W.paper_context_box()), prec, local, stream, 5, torch))
        line["schedule_ablation"] = abl
    if not args.no_second_order and world == 1 and prec == tf.TF_FP32 and args.order == 1:
        # the paper's second-order element, on the two-material box (805 M units per step)
        line["second_order"] = second_order_leg(tf, W.order2(W.two_material_box()), prec, local, stream, 3, torch)
        # and the third-order element on the 16^3-hex workload (50 M units per step)
        line["third_order"] = second_order_leg(tf, W.order3(W.paper_context_box()), prec, local, stream, 2, torch,
                                               order=3)
        # trilinear hexahedra: the paper's own 16^3 workload (256 directions, 10 groups) and the
        # two-material box as a twisted hex grid (134 M units per step); a failure of this leg is
        # reported in the line instead of ending the run
        hexl = []
        for hcfg in (W.paper_hex_box, lambda: W.hex_problem(W.two_material_box())):
            try:
                hexl.append(second_order_leg(tf, hcfg(), prec, local, stream, 3, torch, order="hex"))
            except Exception as e:  # noqa: BLE001
                hexl.append({"error": f"{type(e).__name__}: {e}"})
        line["hexahedra"] = hexl
    if not args.no_fp64_compare and prec == tf.TF_FP32:
        p64 = tf.Problem.from_config(cfg, precision=tf.TF_FP64, device=local, order=args.order)
        phi64 = torch.zeros((C, G, nodes), dtype=torch.float64, device=dev)
        p64.source_iterate(phi64, 0.0, 1, stream=stream)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        p64.source_iterate(phi64, 0.0, args.fp64_steps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        line["fp64_plain_gpu"] = {"ms_per_step": ms64, "grind": ms64 * 1e6 / units, "unit": UNIT,
                                  "fp32_speedup": ms64 / ms_per_step, "n_chunks": p64.stats()["n_chunks"]}
        del p64
    if not args.no_time_to_tol:
        # time to the stopping test 1e-6 on the two-material box (196,608 tets, 128 directions,
        # 32 groups): FP32 sweep with FP64 phi/residual against the plain FP64 GPU sweep
        tcfg = W.two_material_box()
        out = {"workload": tcfg["name"], "tol": tcfg["tol"]}
        for name, pr in (("fp32", tf.TF_FP32), ("fp64", tf.TF_FP64)):
            pt = tf.Problem.from_config(tcfg, precision=pr, device=local)
            ph = torch.zeros((pt.n_cells, pt.n_groups, 4), dtype=torch.float64, device=dev)
            pt.source_iterate(ph, 0.0, 1, stream=stream)  # warm-up sweep
            ph.zero_()
            torch.cuda.synchronize(dev)
            e0.record(stream)
            r = pt.source_iterate(ph, tcfg["tol"], 2000, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            out[name] = {"seconds": e0.elapsed_time(e1) / 1e3, "iterations": r["iterations"],
                         "converged": r["converged"], "residual": r["residual"], "balance": r["balance"]}
            del pt, ph
        out["fp64_over_fp32"] = out["fp64"]["seconds"] / out["fp32"]["seconds"]
        line["time_to_tol"] = out
    if not args.no_batch and world == 1 and args.order == 1:
        # batched problems (16 of the batch workload's uneven problems) at the default and the
        # autotuned task grain, each to the 1e-6 stopping test
        line["batch"] = {"default": batch_leg(tf, torch, 16, False, 1e-6),
                         "autotuned": batch_leg(tf, torch, 16, True, 1e-6)}
    if not args.no_learned and world == 1 and args.order == 1:
        # the learned start: 32 training layouts, 4 held-out layouts from zero and from the network
        lk = dict(n=24, G=16, n_polar=8, n_az=8)
        line["learned"] = learned_leg(tf, torch, lk, 32, 4, 1, 20, 1024, 1e-3, 0, 1e-6)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def batch_leg(tf, torch, count, autotune, tol, seed=None):
    """`count` independent problems of the batch workload (uneven meshes, direction sets and
    group counts) iterated to the stopping test together in shared persistent launches, with the
    autotuned task grain (busy-time criterion) or the default one.  Returns the aggregate grind
    time over the units actually swept, the setup time and each problem's time to tol."""
    dev = torch.device("cuda", torch.cuda.current_device())
    kw = {} if seed is None else {"seed": seed}
    cfgs = W.batch_of_problems(count=count, **kw)
    psi = [len(c["tets"]) * c["n_polar"] * c["n_azimuthal"] * c["n_groups"] * 16 for c in cfgs]
    free = torch.cuda.mem_get_info()[0]
    budget = 0.6 * free
    t0 = time.perf_counter()
    probs = []
    for c, pb in zip(cfgs, psi):
        share = budget * pb / sum(psi) if sum(psi) > budget else 0.0
        probs.append(tf.Problem.from_config(c, precision=tf.TF_FP32, psi_budget_gb=share / 1e9,
                                            cells_per_task=-2 if autotune else 0))
    setup = time.perf_counter() - t0
    phis = [torch.zeros((p.n_cells, p.n_groups, 4), dtype=torch.float64, device=dev) for p in probs]
    tf.source_iterate_batch(probs, phis, 0.0, 1)  # warm-up iteration
    for ph in phis:
        ph.zero_()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st, infos = tf.source_iterate_batch(probs, phis, tol, 2000)
    e1.record()
    torch.cuda.synchronize(dev)
    sec = e0.elapsed_time(e1) / 1e3
    swept = sum(p.n_units * i["iterations"] for p, i in zip(probs, infos))
    out = {"workload": f"batch_{len(cfgs)}_problems", "problems": len(cfgs), "autotune": bool(autotune),
           "tol": tol, "seconds": sec, "grind": sec * 1e9 / swept, "unit": UNIT,
           "units_per_sweep": sum(p.n_units for p in probs), "units_swept": swept, "setup_s": round(setup, 2),
           "all_converged": st == tf.TF_OK,
           "per_problem": [{"cells": p.n_cells, "directions": p.n_dirs, "groups": p.n_groups,
                            "cells_per_task": p.stats()["cells_per_task"], "kernel_mode": p.stats()["kernel_mode"],
                            "octant_window": p.stats()["tuned_window"] or 8,
                            "iterations": i["iterations"], "seconds_to_tol": round(i["seconds"], 4),
                            "converged": i["converged"], "balance": i["balance"]} for p, i in zip(probs, infos)]}
    for p in probs:
        p.close()
    del probs, phis
    torch.cuda.synchronize(dev)
    return out


def run_batch(args):
    """The batch workload on its own (--config batch): one JSON line."""
    import torch

    import paper_2510_11513_gb300 as tf

    torch.cuda.set_device(0)
    b = batch_leg(tf, torch, args.batch_count, args.autotune, args.batch_tol)
    line = {"metric": METRIC, "value": b["grind"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": b["seconds"] * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": b["workload"], "problems": b["problems"], "units_per_sweep": b["units_per_sweep"],
                       "tol": b["tol"], "setup_s": b["setup_s"], "autotune": b["autotune"]},
            "all_converged": b["all_converged"], "per_problem": b["per_problem"]}
    print(json.dumps(line), flush=True)


def learned_leg(tf, torch, kw, train_layouts, eval_layouts, eval_fp64, epochs, batch, lr, seed, tol,
                weight_floor=None, overshoot_weight=1.0, shrink=1.0, context=None, sample_cells=0, gen_batch=1):
    """Learned initial flux on the learned-start layouts: converged fluxes of `train_layouts`
    layouts from the plain FP32 solver, the network trained by the library's kernels, then
    `eval_layouts` held-out layouts solved from zero and from the learned start to the same
    stopping test (the first `eval_fp64` also against a tightly converged FP64 solve)."""
    from paper_2510_11513_gb300 import learned as L

    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    train = (W.random_layout(layout=k, **kw) for k in range(train_layouts))  # built as consumed
    context = L.CONTEXT_STEPS if context is None else tuple(context)
    X, T, Wt, gen = L.generate(train, tol=tol, max_iters=5000, device=dev, weight_floor=weight_floor,
                               context=context, sample_cells=sample_cells, seed=seed, batch=gen_batch,
                               precision=tf.TF_FP32)
    t_gen = time.perf_counter() - t0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ls = L.LearnedStart(kw["G"], hidden=64, seed=seed, overshoot_weight=overshoot_weight, shrink=shrink,
                        context=context)
    hist = ls.fit(X, T, Wt, epochs=epochs, batch=batch, lr=lr, seed=seed)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    samples = X.shape[0]
    del X, T, Wt
    rows = []
    for k in range(eval_layouts):
        cfg = W.random_layout(layout=10000 + k, **kw)
        prob = tf.Problem.from_config(cfg, precision=tf.TF_FP32)
        Xh = L.cell_features(prob.mesh, cfg, dev, context=ls.context)
        phi0 = torch.zeros((prob.n_cells, prob.n_groups, 4), dtype=torch.float64, device=dev)
        torch.cuda.synchronize(dev)
        start = ls.initial_flux(Xh)
        a = time.perf_counter()
        r0 = prob.source_iterate(phi0, tol, 5000)
        torch.cuda.synchronize(dev)
        s0 = time.perf_counter() - a
        start_err = float((start - phi0).norm() / phi0.norm())  # the zero start's is 1
        del start
        a = time.perf_counter()
        phi1, r1 = ls.solve(prob, Xh, tol, 5000)
        torch.cuda.synchronize(dev)
        s1 = time.perf_counter() - a
        row = {"layout": 10000 + k, "iters_zero": r0["iterations"], "iters_learned": r1["iterations"],
               "s_zero": round(s0, 4), "s_learned": round(s1, 4), "predict_s": round(r1["predict_seconds"], 5),
               "converged": bool(r0["converged"] and r1["converged"]), "start_rel_l2_err": round(start_err, 4)}
        if k < eval_fp64:
            p64 = tf.Problem.from_config(cfg, precision=tf.TF_FP64)
            ref = torch.zeros_like(phi0)
            r64 = p64.source_iterate(ref, 1e-10, 8000)
            scale = ref.abs().amax(dim=(0, 2), keepdim=True)
            row["err_zero"] = float(((phi0 - ref).abs() / scale).max())
            row["err_learned"] = float(((phi1 - ref).abs() / scale).max())
            row["fp64_iters"] = r64["iterations"]
            p64.close()
        rows.append(row)
        prob.close()
    iz = sum(r["iters_zero"] for r in rows)
    il = sum(r["iters_learned"] for r in rows)
    return {"workload": f"learned_start_layouts_{kw['n']}^3_D{kw['n_polar'] * kw['n_az']}_G{kw['G']}",
            "train_layouts": train_layouts, "eval_layouts": eval_layouts, "samples": samples, "epochs": epochs,
            "context_steps": list(context), "sample_cells": sample_cells,
            "batch": batch, "lr": lr, "tol": tol, "weight_floor": weight_floor,
            "overshoot_weight": overshoot_weight, "shrink": shrink,
            "s_learned": sum(r["s_learned"] for r in rows) / len(rows),
            "s_zero": sum(r["s_zero"] for r in rows) / len(rows),
            "iterations_zero": iz, "iterations_learned": il, "iteration_ratio": il / max(iz, 1),
            "start_rel_l2_err_mean": sum(r["start_rel_l2_err"] for r in rows) / len(rows),
            "generate_s": round(t_gen, 1), "generate_solve_s": round(sum(g["solve_seconds"] for g in gen), 2),
            "generate_iterations": ([g["iterations"] for g in gen] if len(gen) <= 64 else
                                    {"mean": sum(g["iterations"] for g in gen) / len(gen),
                                     "min": min(g["iterations"] for g in gen), "max": max(g["iterations"] for g in gen)}),
            "train_s": round(t_train, 2),
            "loss_history": [round(float(h), 5) for h in hist], "per_layout": rows}


def run_learned(args):
    """Learned initial flux (--config layout) on its own: one JSON line."""
    import torch

    import paper_2510_11513_gb300 as tf

    torch.cuda.set_device(0)
    kw = dict(n=args.n or 24, G=args.groups or 16, n_polar=args.polar or 8, n_az=args.azimuthal or 8)
    floor = args.weight_floor if args.weight_floor >= 0 else None
    ctx = () if args.context == "none" else (None if args.context == "default" else
                                             tuple(int(x) for x in args.context.split(",")))
    r = learned_leg(tf, torch, kw, args.train_layouts, args.eval_layouts, args.eval_fp64, args.epochs,
                    args.train_batch, args.lr, args.seed, args.batch_tol, floor, args.overshoot_weight, args.shrink,
                    context=ctx, sample_cells=args.sample_cells, gen_batch=args.gen_batch)
    line = {"metric": "time to 1e-6 per layout, learned start (zero-start alongside)", "value": r["s_learned"],
            "unit": "s", "n_gpus": 1, "steps": r["eval_layouts"], "warmup": 0, "ms_per_step": 1e3 * r["s_learned"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
            "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "train_layouts", "eval_layouts", "samples", "epochs", "batch",
                                         "lr", "tol", "weight_floor", "overshoot_weight", "shrink", "context_steps",
                                         "sample_cells")},
            **{k: r[k] for k in ("iterations_zero", "iterations_learned", "iteration_ratio", "generate_s",
                                 "generate_solve_s", "generate_iterations", "train_s", "loss_history",
                                 "start_rel_l2_err_mean", "per_layout")},
            "zero_start_s": r["s_zero"]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="corner_source", choices=sorted(W.CONFIGS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--cells-per-task", type=int, default=0)
    ap.add_argument("--warps-per-cta", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true", help="skip the plain FP64 GPU sweep comparison")
    ap.add_argument("--no-time-to-tol", action="store_true", help="skip the time-to-1e-6 comparison")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--schedule", default="amt", choices=sorted(SCHEDULES),
                    help="task schedule of the timed sweep: many-task (amt) or bulk-synchronous")
    ap.add_argument("--no-bsp-compare", action="store_true", help="skip the many-task vs bulk-synchronous legs")
    ap.add_argument("--no-second-order", action="store_true", help="skip the second-order element leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-problems leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-start leg")
    ap.add_argument("--order", type=int, default=1, choices=[1, 2, 3],
                    help="finite-element order of the timed sweep (2: ten nodes, 3: twenty nodes)")
    ap.add_argument("--bsp-steps", type=int, default=2, help="timed steps of each schedule in the comparison")
    ap.add_argument("--octant-window", type=int, default=0, help="octants active at once (0 = library default)")
    ap.add_argument("--keep-ready", type=int, default=0, help="ready tasks a warp keeps and runs next (0 = library default)")
    ap.add_argument("--staging", type=int, default=0, help="0 auto, 1 no shared-memory staging, 2 two stages, 3 three stages")
    ap.add_argument("--pairing", type=int, default=0, help="0 auto, 1 off, 2 packed group pairs when G is even")
    ap.add_argument("--task-shape", type=int, default=0, help="0 auto, 1 t-level blocks, 2 spatial patches")
    ap.add_argument("--shard", default="directions", choices=["directions", "replicas"],
                    help="N > 1: split the directions over the ranks (partial flux summed every step) or run replicas")
    ap.add_argument("--patch-extent", type=float, default=0.0, help="spatial patches: region edge in cell sizes (0 = default)")
    ap.add_argument("--batch-count", type=int, default=64, help="--config batch: number of problems")
    ap.add_argument("--batch-tol", type=float, default=1e-6)
    ap.add_argument("--autotune", type=int, default=1, help="--config batch: autotuned task grain (1) or default (0)")
    ap.add_argument("--n", type=int, default=0, help="hexes per box edge (default: the workload's)")
    ap.add_argument("--groups", type=int, default=0)
    ap.add_argument("--polar", type=int, default=0)
    ap.add_argument("--azimuthal", type=int, default=0)
    ap.add_argument("--train-layouts", type=int, default=64, help="--config layout: training layouts")
    ap.add_argument("--eval-layouts", type=int, default=8, help="--config layout: held-out layouts")
    ap.add_argument("--eval-fp64", type=int, default=2, help="--config layout: held-out layouts checked against FP64")
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--train-batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--weight-floor", type=float, default=-1.0,
                    help="--config layout: loss weights (phi/max)^2 + floor; negative = unweighted")
    ap.add_argument("--shrink", type=float, default=1.0, help="--config layout: factor on the predicted flux")
    ap.add_argument("--context", default="default",
                    help="--config layout: context steps of the inputs ('default', 'none' = one ring, or e.g. 4,16,64)")
    ap.add_argument("--sample-cells", type=int, default=0, help="--config layout: training cells kept per layout (0 = all)")
    ap.add_argument("--gen-batch", type=int, default=1,
                    help="--config layout: training layouts solved together in shared launches")
    ap.add_argument("--overshoot-weight", type=float, default=1.0,
                    help="--config layout: loss weight of overshooting outputs (1 = plain squared error)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batch":
        run_batch(args)
    elif args.config == "layout":
        run_learned(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
