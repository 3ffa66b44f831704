"""Edge cases of the CUDA sweep against the oracle: a single tetrahedron (every
face on the boundary), a single direction, directions exactly parallel to
faces (unjittered boundary faces and Kuhn diagonals: s_f = 0, classified as
outflow by both codes), and the private ready-task stack of the many-task
kernel at depths 2 and 4 (same results, only the order of tasks changes)."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import p2 as o2

torch = pytest.importorskip("torch")
import paper_2510_11513_gb300 as tf  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {tf.TF_FP64: 1e-11, tf.TF_FP32: 2e-5}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _single_tet(G):
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 1.0, 0.1], [0.1, 0.2, 1.0]])
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    st = np.linspace(0.5, 2.0, G)[None, :]
    ss = np.zeros((1, G, G))
    for g in range(G):
        ss[0, g, g:] = 0.4 * st[0, g] / (G - g)
    return {"xyz": xyz, "tets": tets, "n_groups": G, "n_materials": 1, "cell_material": np.zeros(1, np.int32),
            "sigma_t": st, "sigma_s": ss, "Q": np.ones((1, G, 4)), "n_polar": 4, "n_azimuthal": 8,
            "name": "single_tet"}


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
@pytest.mark.parametrize("G", [1, 3, 32])
def test_single_tetrahedron(precision, G):
    cfg = _single_tet(G)
    P = oracle.Problem(cfg)
    phi_in = np.random.default_rng(1).uniform(0.0, 1.0, (1, G, 4))
    ref = P.transport_step(phi_in)
    prob = tf.Problem.from_config(cfg, precision=precision)
    out = torch.zeros_like(_dev(phi_in))
    prob.sweep(_dev(phi_in), out)
    assert _rel(out.cpu().numpy(), ref) < TOL[precision]
    # the same cell with the second-order element
    cfg2 = W.order2(cfg)
    P2 = o2.Problem2(cfg2)
    phi2 = np.random.default_rng(2).uniform(0.0, 1.0, (1, G, 10))
    ref2 = P2.transport_step(phi2)
    prob2 = tf.Problem.from_config(cfg2, precision=precision, order=2)
    out2 = torch.zeros_like(_dev(phi2))
    prob2.sweep(_dev(phi2), out2)
    assert _rel(out2.cpu().numpy(), ref2) < TOL[precision]


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
def test_single_direction(precision):
    cfg = W.small_box(n=5, G=4)
    om = np.array([[0.3, -0.5, np.sqrt(1.0 - 0.34)]])
    w = np.array([4.0 * np.pi])
    P = oracle.Problem(cfg, omega=om, w=w)
    phi_in = np.random.default_rng(3).uniform(0.0, 1.0, (P.C, 4, 4))
    ref = P.transport_step(phi_in)
    prob = tf.Problem.from_config(cfg, precision=precision, omega=om, w=w)
    out = torch.zeros_like(_dev(phi_in))
    prob.sweep(_dev(phi_in), out)
    assert _rel(out.cpu().numpy(), ref) < TOL[precision]
    assert prob.stats()["n_dirs"] == 1


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
def test_directions_parallel_to_faces(precision):
    """The six axis directions and the four (+-1, +-1, 0)/sqrt 2 diagonals: on the box's
    boundary faces and on unjittered Kuhn diagonals Omega.N_f is exactly zero."""
    cfg = W.small_box(n=4, G=3)
    ax = np.vstack([np.eye(3), -np.eye(3)])
    dg = np.array([[1, 1, 0], [1, -1, 0], [-1, 1, 0], [-1, -1, 0]]) / np.sqrt(2.0)
    om = np.vstack([ax, dg])
    w = np.full(len(om), 4.0 * np.pi / len(om))
    P = oracle.Problem(cfg, omega=om, w=w)
    phi_in = np.random.default_rng(4).uniform(0.0, 1.0, (P.C, 3, 4))
    ref = P.transport_step(phi_in)
    prob = tf.Problem.from_config(cfg, precision=precision, omega=om, w=w)
    mesh_masks, _ = tf.tf_graph_levels(prob.mesh.h, prob.quad.h, P.C, len(om))
    assert np.array_equal(mesh_masks, P.inflow)
    out = torch.zeros_like(_dev(phi_in))
    prob.sweep(_dev(phi_in), out)
    assert _rel(out.cpu().numpy(), ref) < TOL[precision]


@pytest.mark.parametrize("keep", [2, 4])
@pytest.mark.parametrize("G,opts", [(64, {}), (6, {}), (4, dict(pairing=1))])
def test_private_ready_stack_same_result(keep, G, opts):
    cfg = W.small_box(n=6, G=G, n_polar=2, n_az=8)
    phi_in = _dev(np.random.default_rng(5).uniform(0.0, 1.0, (len(cfg["tets"]), G, 4)))
    a = tf.Problem.from_config(cfg, **opts)
    b = tf.Problem.from_config(cfg, keep_ready=keep, **opts)
    out_a, out_b = torch.zeros_like(phi_in), torch.zeros_like(phi_in)
    a.sweep(phi_in, out_a)
    b.sweep(phi_in, out_b)
    assert torch.equal(out_a, out_b)
    st = b.stats()
    assert st["tasks_executed"] == st["n_tasks"]
