"""Parity of the third-order (twenty-node) CUDA sweep with the third-order oracle.

Tolerances as for the lower orders (relative to the oracle's max-norm): FP64 1e-11,
FP32 2e-5.  Several tasks, ragged group counts and cell blocks, direction chunks.
"""
import numpy as np
import pytest

import workloads as W
from oracle import p3 as o3

torch = pytest.importorskip("torch")
import paper_2510_11513_gb300 as tf  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {tf.TF_FP64: 1e-11, tf.TF_FP32: 2e-5}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _box(n, G, seed=5, two_material=False):
    if two_material:
        return W.order3(W.two_material_box(n=n, G=G, n_polar=2, n_az=8, seed=seed))
    return W.order3(W.small_box(n=n, G=G, n_polar=2, n_az=8, seed=seed))


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
@pytest.mark.parametrize("G,opts", [(1, {}), (3, dict(cells_per_task=5)), (32, {}), (7, dict(dir_chunk=5)), (16, {}),
                                    (9, dict(cells_per_task=3))])
def test_one_sweep_matches_oracle(precision, G, opts):
    cfg = _box(n=3, G=G)
    P = o3.Problem3(cfg)
    phi_in = np.random.default_rng(11).uniform(0.0, 1.0, (P.C, G, 20))
    ref = P.transport_step(phi_in, threads=8)
    prob = tf.Problem.from_config(cfg, precision=precision, order=3, **opts)
    out = torch.zeros_like(_dev(phi_in))
    prob.sweep(_dev(phi_in), out)
    assert _rel(out.cpu().numpy(), ref) < TOL[precision]
    st = prob.stats()
    assert st["tasks_executed"] == st["n_tasks"] and st["kernel_mode"] == 7


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
def test_psi_of_directions_matches_oracle(precision):
    cfg = _box(n=3, G=4)
    P = o3.Problem3(cfg)
    phi_in = np.random.default_rng(2).uniform(0.0, 1.0, (P.C, 4, 20))
    q = P.source(phi_in)
    prob = tf.Problem.from_config(cfg, precision=precision, order=3)
    prob.sweep(_dev(phi_in), torch.zeros_like(_dev(phi_in)))
    dt = torch.float64 if precision == tf.TF_FP64 else torch.float32
    for a in (0, 9, P.D - 1):
        buf = torch.empty((P.C, 4, 20), dtype=dt, device="cuda")
        assert _rel(prob.psi(a, buf).double().cpu().numpy(), P.sweep_direction(a, q)) < TOL[precision], a


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
def test_converged_source_iteration_matches_oracle(precision):
    cfg = _box(n=3, G=3, two_material=True)
    P = o3.Problem3(cfg)
    ref, it_ref, _ = P.source_iterate(1e-8, 500, threads=8)
    prob = tf.Problem.from_config(cfg, precision=precision, order=3)
    phi = torch.zeros((P.C, 3, 20), dtype=torch.float64, device="cuda")
    res = prob.source_iterate(phi, 1e-8 if precision == tf.TF_FP64 else 1e-6, 500)
    assert res["converged"]
    if precision == tf.TF_FP64:
        assert abs(res["iterations"] - it_ref) <= 1
    assert _rel(phi.cpu().numpy(), ref) < (1e-7 if precision == tf.TF_FP64 else 2e-5)
    ig, _ = P.integrated_flux(phi.cpu().numpy())
    assert np.allclose(res["integrated_flux"], ig, rtol=1e-12, atol=0)
    assert res["balance"] < (1e-12 if precision == tf.TF_FP64 else 1e-5), res["balance"]


@pytest.mark.parametrize("schedule", [tf.TF_SCHED_BSP, tf.TF_SCHED_BSP_LAUNCH])
def test_bulk_synchronous_schedules_same_result(schedule):
    cfg = _box(n=3, G=4)
    phi_in = _dev(np.random.default_rng(8).uniform(0.0, 1.0, (len(cfg["tets"]), 4, 20)))
    a = tf.Problem.from_config(cfg, order=3)
    b = tf.Problem.from_config(cfg, order=3, schedule=schedule)
    out_a, out_b = torch.zeros_like(phi_in), torch.zeros_like(phi_in)
    a.sweep(phi_in, out_a)
    b.sweep(phi_in, out_b)
    assert torch.equal(out_a, out_b)
