"""Regression values written by tests/golden/make_golden.py from the oracle alone:
the oracle must keep reproducing them (CPU), and the library must match them (GPU)."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import p2 as o2
from oracle import p3 as o3
from oracle import q1hex as oh

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_regression.json")))


def _step_case(order):
    mod, maker, cls, nb = {2: (o2, W.order2, o2.Problem2, 10), 3: (o3, W.order3, o3.Problem3, 20)}[order]
    cfg = maker(W.small_box(n=2, G=3, n_polar=2, n_az=8))
    phi0 = np.random.default_rng(GOLD[f"order{order}_step"]["seed"]).uniform(0.0, 1.0, (len(cfg["tets"]), 3, nb))
    return cfg, cls, phi0


def test_oracle_reproduces_small_box():
    g = GOLD["small_box"]
    P = oracle.Problem(W.small_box())
    phi, it, r = P.source_iterate(g["tol"], 1000, threads=4)
    ig, tot, plain, _ = P.integrated_flux(phi)
    assert it == g["iterations"]
    assert np.allclose(ig, g["integrated_flux"], rtol=1e-12, atol=0)
    assert np.allclose(plain, g["nodal_sum"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("order", [2, 3])
def test_oracle_reproduces_higher_order_step(order):
    cfg, cls, phi0 = _step_case(order)
    Q = cls(cfg)
    step = Q.transport_step(phi0, threads=4)
    ig, _ = Q.integrated_flux(step)
    g = GOLD[f"order{order}_step"]
    assert np.allclose(ig, g["integrated_flux"], rtol=1e-12, atol=0)
    cs = float(np.sum(step * np.arange(1, step.size + 1).reshape(step.shape) / step.size))
    assert abs(cs - g["checksum"]) <= 1e-12 * abs(g["checksum"])


def test_oracle_reproduces_hex_small_box():
    g = GOLD["hex_small_box"]
    P = oh.ProblemHex(W.hex_problem(W.small_box(), twist=g["twist"]))
    phi, it, r = P.source_iterate(g["tol"], 1000, threads=4)
    ig, _ = P.integrated_flux(phi)
    assert it == g["iterations"]
    assert np.allclose(ig, g["integrated_flux"], rtol=1e-12, atol=0)


@pytest.mark.gpu
def test_library_matches_golden_small_box():
    torch = pytest.importorskip("torch")
    import paper_2510_11513_gb300 as tf

    g = GOLD["small_box"]
    prob = tf.Problem.from_config(W.small_box(), precision=tf.TF_FP64)
    phi = torch.zeros((prob.n_cells, 4, 4), dtype=torch.float64, device="cuda")
    res = prob.source_iterate(phi, g["tol"], 1000)
    assert abs(res["iterations"] - g["iterations"]) <= 1
    assert np.allclose(res["integrated_flux"], g["integrated_flux"], rtol=1e-10, atol=0)


@pytest.mark.gpu
@pytest.mark.parametrize("order", [2, 3])
def test_library_matches_golden_higher_order_step(order):
    torch = pytest.importorskip("torch")
    import paper_2510_11513_gb300 as tf

    cfg, _, phi0 = _step_case(order)
    prob = tf.Problem.from_config(cfg, precision=tf.TF_FP64, order=order)
    phi_in = torch.from_numpy(phi0).cuda()
    out = torch.zeros_like(phi_in)
    prob.sweep(phi_in, out)
    # the integrated flux (Eq. 3) of the device's step, integrated with the oracle's weights
    Q = (o2.Problem2 if order == 2 else o3.Problem3)(cfg)
    ig_dev, _ = Q.integrated_flux(out.cpu().numpy())
    assert np.allclose(ig_dev, GOLD[f"order{order}_step"]["integrated_flux"], rtol=1e-11, atol=0)
