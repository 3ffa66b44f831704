"""Parity at the full workload sizes, in the launch configuration the bench times.

corner-source box (663,552 tets, 192 directions, 64 groups, FP32): one sweep
from a seeded phi; the oracle solves sampled directions one by one (all
cells, all groups) from the same source, phi of sampled cells is checked
against the FP64 quadrature sum of the device's own psi, and phi of every cell
in groups 0..7 against the oracle's transport step over all 192 directions.
two-material box (196,608 tets, 128 directions, 32 groups, FP32): one full
transport step compared with the oracle's, element by element.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
import paper_2510_11513_gb300 as tf  # noqa: E402

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_corner_source_full_size_sampled():
    cfg = W.corner_source_box()
    prob = tf.Problem.from_config(cfg, precision=tf.TF_FP32)  # the bench's launch configuration
    C, G, D = prob.n_cells, prob.n_groups, prob.n_dirs
    rng = np.random.default_rng(42)
    phi_in = rng.uniform(0.0, 1.0, (C, G, 4))
    out = torch.zeros((C, G, 4), dtype=torch.float64, device="cuda")
    prob.sweep(torch.from_numpy(phi_in).cuda(), out)
    st = prob.stats()
    assert st["tasks_executed"] == st["n_tasks"] and st["n_chunks"] == 1
    # oracle on sampled directions, all cells and groups, same source
    sample = [0, 101, 191]
    om, w = oracle.product_quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    P = oracle.Problem(cfg, omega=om[sample], w=w[sample])
    q = P.source(phi_in)
    buf = torch.empty((C, G, 4), dtype=torch.float32, device="cuda")
    for k, a in enumerate(sample):
        ref = P.sweep_direction(k, q)
        got = prob.psi(a, buf).double().cpu().numpy()
        assert _rel(got, ref) < 2e-5, a
    # phi of sampled cells = FP64 sum over all directions of w_a psi_a (device psi)
    cells = torch.from_numpy(np.sort(rng.choice(C, 4096, replace=False))).cuda()
    acc = torch.zeros((len(cells), G, 4), dtype=torch.float64, device="cuda")
    for a in range(D):
        acc += w[a] * prob.psi(a, buf)[cells].double()
    got_phi = out[cells]
    assert _rel(got_phi.cpu().numpy(), acc.cpu().numpy()) < 1e-12


def test_corner_source_full_size_phi_of_eight_groups_against_oracle():
    """phi of the bench workload (all 663,552 cells, all 192 directions) after one transport step,
    element by element against the oracle, for groups 0..7.  The workload scatters downward only,
    so the source of groups 0..7 depends on phi of groups 0..7 alone: the oracle solves the problem
    cut to its first eight groups (sigma_t, sigma_s and Q sliced), which is the full problem's first
    eight groups exactly."""
    import os

    cfg = W.corner_source_box()
    S = cfg["sigma_s"]
    assert np.all(np.tril(S, -1) == 0.0)  # sigma_s[m][g_from][g_to] = 0 for g_to < g_from: no upscatter
    prob = tf.Problem.from_config(cfg, precision=tf.TF_FP32)  # the bench's launch configuration
    C, G = prob.n_cells, prob.n_groups
    phi_in = np.random.default_rng(43).uniform(0.0, 1.0, (C, G, 4))
    out = torch.zeros((C, G, 4), dtype=torch.float64, device="cuda")
    prob.sweep(torch.from_numpy(phi_in).cuda(), out)
    got = out[:, :8].cpu().numpy()
    prob.close()
    g8 = dict(cfg, n_groups=8, sigma_t=np.ascontiguousarray(cfg["sigma_t"][:, :8]),
              sigma_s=np.ascontiguousarray(S[:, :8, :8]), Q=np.ascontiguousarray(cfg["Q"][:, :8]))
    ref = oracle.Problem(g8).transport_step(np.ascontiguousarray(phi_in[:, :8]), threads=os.cpu_count() or 1)
    assert _rel(got, ref) < 2e-5


def test_two_material_full_size_one_step():
    cfg = W.two_material_box()
    prob = tf.Problem.from_config(cfg, precision=tf.TF_FP32)
    C, G = prob.n_cells, prob.n_groups
    phi_in = np.random.default_rng(7).uniform(0.0, 1.0, (C, G, 4))
    out = torch.zeros((C, G, 4), dtype=torch.float64, device="cuda")
    prob.sweep(torch.from_numpy(phi_in).cuda(), out)
    P = oracle.Problem(cfg)
    import os
    ref = P.transport_step(phi_in, threads=os.cpu_count() or 1)
    assert _rel(out.cpu().numpy(), ref) < 2e-5
