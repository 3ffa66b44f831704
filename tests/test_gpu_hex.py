"""Parity of the trilinear-hexahedron CUDA sweep (sweep mode 8) with the hexahedral oracle.

Tolerances as for the tetrahedra (relative to the oracle's max-norm): FP64 1e-11, FP32
2e-5.  Twisted grids (0.25 rad over the height, no jitter: acyclic sweep graphs), sizes
spanning several tasks, ragged group counts and cell blocks, several direction chunks.
"""
import numpy as np
import pytest

import workloads as W
from oracle import q1hex as oh

torch = pytest.importorskip("torch")
import paper_2510_11513_gb300 as tf  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {tf.TF_FP64: 1e-11, tf.TF_FP32: 2e-5}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _box(n, G, seed=5, two_material=False, twist=0.25):
    maker = W.two_material_box if two_material else W.small_box
    return W.hex_problem(maker(n=n, G=G, n_polar=2, n_az=8, seed=seed), twist=twist)


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
@pytest.mark.parametrize("G,opts", [(1, {}), (4, {}), (5, dict(cells_per_task=3)), (8, {}), (9, dict(cells_per_task=3)),
                                    (32, {}), (32, dict(staging=1)), (37, dict(cells_per_task=2, dir_chunk=5)),
                                    (12, dict(dir_chunk=7)), (64, dict(cells_per_task=5, dir_chunk=9))])
def test_one_sweep_matches_oracle(precision, G, opts):
    cfg = _box(n=4 if G >= 32 else 5, G=G)
    P = oh.ProblemHex(cfg)
    phi_in = np.random.default_rng(11).uniform(0.0, 1.0, (P.C, G, 8))
    ref = P.transport_step(phi_in, threads=8)
    prob = tf.Problem.from_config(cfg, precision=precision, **opts)
    assert prob.n_nodes == 8
    out = torch.zeros_like(_dev(phi_in))
    prob.sweep(_dev(phi_in), out)
    assert _rel(out.cpu().numpy(), ref) < TOL[precision]
    st = prob.stats()
    assert st["tasks_executed"] == st["n_tasks"]
    assert st["kernel_mode"] == (9 if G >= 8 and opts.get("staging", 0) != 1 else 8)


@pytest.mark.parametrize("precision,G", [(tf.TF_FP64, 6), (tf.TF_FP32, 6), (tf.TF_FP32, 32)])
def test_psi_of_directions_matches_oracle(precision, G):
    cfg = _box(n=4, G=G, twist=0.6)
    P = oh.ProblemHex(cfg)
    phi_in = np.random.default_rng(2).uniform(0.0, 1.0, (P.C, G, 8))
    q = P.source(phi_in)
    prob = tf.Problem.from_config(cfg, precision=precision)
    prob.sweep(_dev(phi_in), torch.zeros_like(_dev(phi_in)))
    dt = torch.float64 if precision == tf.TF_FP64 else torch.float32
    for a in (0, 5, P.D - 1):
        buf = torch.empty((P.C, G, 8), dtype=dt, device="cuda")
        got = prob.psi(a, buf).double().cpu().numpy()
        assert _rel(got, P.sweep_direction(a, q)) < TOL[precision], a


@pytest.mark.parametrize("precision,G", [(tf.TF_FP64, 4), (tf.TF_FP32, 4), (tf.TF_FP32, 32)])
def test_converged_source_iteration_matches_oracle(precision, G):
    """Two materials, up- and downscatter: the device iteration stops at the same test, with
    phi, the integrated flux (Eq. 3 with the trilinear field) and the particle balance of the
    device against the oracle."""
    cfg = _box(n=4, G=G, two_material=True)
    P = oh.ProblemHex(cfg)
    ref, it_ref, r_ref = P.source_iterate(1e-8, 500, threads=8)
    prob = tf.Problem.from_config(cfg, precision=precision)
    phi = torch.zeros((P.C, G, 8), dtype=torch.float64, device="cuda")
    tol = 1e-8 if precision == tf.TF_FP64 else 1e-6
    res = prob.source_iterate(phi, tol, 500)
    assert res["converged"]
    if precision == tf.TF_FP64:
        assert abs(res["iterations"] - it_ref) <= 1
    assert _rel(phi.cpu().numpy(), ref) < (1e-7 if precision == tf.TF_FP64 else 2e-5)
    ig, tot = P.integrated_flux(phi.cpu().numpy())
    assert np.allclose(res["integrated_flux"], ig, rtol=1e-12, atol=0)
    assert res["balance"] < (1e-12 if precision == tf.TF_FP64 else 1e-5), res["balance"]


def test_golden_hex_small_box():
    """The 8^3 box as twisted hexahedra converged in FP64 against the oracle's stored values."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_regression.json")))["hex_small_box"]
    cfg = W.hex_problem(W.small_box(), twist=g["twist"])
    prob = tf.Problem.from_config(cfg, precision=tf.TF_FP64)
    phi = torch.zeros((prob.n_cells, 4, 8), dtype=torch.float64, device="cuda")
    res = prob.source_iterate(phi, g["tol"], 1000)
    assert abs(res["iterations"] - g["iterations"]) <= 1
    assert np.allclose(res["integrated_flux"], g["integrated_flux"], rtol=1e-10, atol=0)


def test_host_buffers_and_aliasing():
    cfg = _box(n=3, G=3)
    P = oh.ProblemHex(cfg)
    phi_in = np.random.default_rng(4).uniform(0.0, 1.0, (P.C, 3, 8))
    ref = P.transport_step(phi_in)
    prob = tf.Problem.from_config(cfg, precision=tf.TF_FP64)
    hin = torch.from_numpy(phi_in.copy()).pin_memory()
    hout = torch.zeros_like(hin).pin_memory()
    prob.sweep(hin, hout)
    assert _rel(hout.numpy(), ref) < 1e-11
    buf = _dev(phi_in)
    prob.sweep(buf, buf)
    assert _rel(buf.cpu().numpy(), ref) < 1e-11


@pytest.mark.parametrize("schedule", [tf.TF_SCHED_BSP, tf.TF_SCHED_BSP_LAUNCH])
@pytest.mark.parametrize("precision,G", [(tf.TF_FP64, 5), (tf.TF_FP32, 5), (tf.TF_FP32, 32)])
def test_bulk_synchronous_schedules_same_result(schedule, precision, G):
    cfg = _box(n=4, G=G)
    P = oh.ProblemHex(cfg)
    phi_in = np.random.default_rng(8).uniform(0.0, 1.0, (P.C, G, 8))
    ref = P.transport_step(phi_in, threads=8)
    a = tf.Problem.from_config(cfg, precision=precision)
    b = tf.Problem.from_config(cfg, precision=precision, schedule=schedule)
    out_a, out_b = torch.zeros_like(_dev(phi_in)), torch.zeros_like(_dev(phi_in))
    a.sweep(_dev(phi_in), out_a)
    b.sweep(_dev(phi_in), out_b)
    assert torch.equal(out_a, out_b)
    assert _rel(out_b.cpu().numpy(), ref) < TOL[precision]
    st = b.stats()
    assert st["tasks_executed"] == st["n_tasks"] and st["n_buckets"] > 0
    assert st["kernel_mode"] == a.stats()["kernel_mode"] == (9 if G >= 8 else 8)


def test_hexahedral_rejections():
    """Hexahedra take only the trilinear (order 1) element, and the cell-average source layout
    of order 1; S1, prescribed inflow and batching are accepted (tested below)."""
    cfg = _box(n=2, G=2)
    C = len(cfg["hexes"])
    with pytest.raises(tf.TfError) as e:
        tf.Problem.from_config(cfg, order=2)
    assert e.value.status == tf.TF_ERR_ARG
    with pytest.raises(ValueError):
        tf.Problem.from_config(dict(cfg, Q=np.zeros((C, 2, 4))))


# ------------------------------------------------- prescribed inflow and the S1 source
def _linear_field(rng, G):
    return rng.uniform(1.0, 2.0, G), rng.uniform(-0.5, 0.5, (G, 3))


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
@pytest.mark.parametrize("G,opts", [(3, {}), (8, {}), (8, dict(staging=1)), (32, dict(dir_chunk=5))])
def test_inflow_and_s1_one_sweep_match_oracle(precision, G, opts):
    """Random S1 and prescribed inflow: one transport step against the hexahedral oracle, on
    both device variants (per-unit registers and the shared group-independent matrices)."""
    cfg = _box(n=4, G=G, twist=0.6)
    C, nv = len(cfg["hexes"]), len(cfg["xyz"])
    rng = np.random.default_rng(17)
    S1 = rng.uniform(-1.0, 1.0, (C, G, 3))
    psi_in = rng.uniform(0.0, 1.0, (nv, G))
    P = oh.ProblemHex(cfg, S1=S1, psi_in=psi_in)
    phi_in = rng.uniform(0.0, 1.0, (C, G, 8))
    ref = P.transport_step(phi_in, threads=8)
    prob = tf.Problem.from_config(cfg, S1=S1, psi_inflow=psi_in, precision=precision, **opts)
    out = torch.zeros((C, G, 8), dtype=torch.float64, device="cuda")
    prob.sweep(_dev(phi_in), out)
    assert _rel(out.cpu().numpy(), ref) < TOL[precision]


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
def test_manufactured_linear_field_on_the_device(precision):
    """psi = alpha + beta.x lies in the trilinear space: with S1 = beta, inflow psi on the boundary
    and Q = 4 pi (sigma_t psi - sum_g' sigma_s[g'->g] psi_g'), source iteration on the device
    converges to phi = 4 pi psi at every node of the twisted grid."""
    cfg = W.hex_problem(W.two_material_box(n=4, G=3, n_polar=2, n_az=8), twist=0.4)
    rng = np.random.default_rng(3)
    alpha, beta = _linear_field(rng, 3)
    xyz, hexes = cfg["xyz"], cfg["hexes"]
    C = len(hexes)
    exact_v = alpha[None, :] + xyz @ beta.T
    exact = exact_v[hexes].transpose(0, 2, 1)
    mat = cfg["cell_material"]
    Q = np.empty_like(exact)
    for c in range(C):
        m = mat[c]
        Q[c] = 4.0 * np.pi * (cfg["sigma_t"][m][:, None] * exact[c] - cfg["sigma_s"][m].T @ exact[c])
    cfg = dict(cfg, Q=Q)
    prob = tf.Problem.from_config(cfg, S1=np.broadcast_to(beta, (C, 3, 3)).copy(), psi_inflow=exact_v,
                                  precision=precision)
    phi = torch.zeros((C, 3, 8), dtype=torch.float64, device="cuda")
    r = prob.source_iterate(phi, 1e-12 if precision == tf.TF_FP64 else 1e-6, 2000)
    assert r["converged"]
    err = np.max(np.abs(phi.cpu().numpy() - 4.0 * np.pi * exact)) / (4.0 * np.pi * np.max(exact))
    assert err < (1e-10 if precision == tf.TF_FP64 else 2e-5), err
    # the device's particle balance, with the prescribed inflow in the boundary leakage
    assert r["balance"] < (1e-12 if precision == tf.TF_FP64 else 1e-5), r["balance"]


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
def test_batched_hexahedra_with_tetrahedra(precision):
    """Hexahedral problems (both device variants) batched with a tetrahedral one in shared
    persistent launches: each problem's step equals its own single-problem step bit for bit, and
    the hexahedral ones match the oracle."""
    cfgs = [_box(n=4, G=8, twist=0.5), _box(n=3, G=3, seed=9, two_material=True, twist=0.3),
            W.two_material_box(n=4, G=32, n_polar=2, n_az=8)]
    probs = [tf.Problem.from_config(c, precision=precision) for c in cfgs]
    nb = [8, 8, 4]
    rng = np.random.default_rng(23)
    ins = [rng.uniform(0.0, 1.0, (p.n_cells, p.n_groups, k)) for p, k in zip(probs, nb)]
    outs = [torch.zeros((p.n_cells, p.n_groups, k), dtype=torch.float64, device="cuda") for p, k in zip(probs, nb)]
    tf.sweep_batch(probs, [_dev(x) for x in ins], outs)
    for p, x, o in zip(probs, ins, outs):
        single = torch.zeros_like(o)
        p.sweep(_dev(x), single)
        assert torch.equal(single, o)
    for c, x, o in zip(cfgs[:2], ins[:2], outs[:2]):
        ref = oh.ProblemHex(c).transport_step(x, threads=8)
        assert _rel(o.cpu().numpy(), ref) < TOL[precision]


# ------------------------------------------------- lagged back edges (grids with cyclic sweep graphs)
def _cyclic(G, n=4, seed=5):
    cfg = W.hex_problem(W.small_box(n=n, G=G, n_polar=8, n_az=16, seed=seed), twist=0.6)
    cfg["Q"] = np.random.default_rng(seed).uniform(0.0, 1.0, cfg["Q"].shape)
    return cfg


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
@pytest.mark.parametrize("G,opts", [(3, {}), (8, {}), (8, dict(staging=1)), (32, dict(dir_chunk=37))])
def test_lagged_steps_match_oracle(precision, G, opts):
    """Two consecutive transport steps with lag_cycles: the first reads zero on the lagged faces,
    the second the first step's psi (gathered after each direction chunk's sweep); both against
    the oracle's steps, in both hexahedral modes and over several direction chunks."""
    cfg = _cyclic(G)
    P = oh.ProblemHex(cfg, lag=True)
    prob = tf.Problem.from_config(cfg, precision=precision, lag_cycles=1, **opts)
    assert prob.stats()["lagged_faces"] == int(np.unpackbits(P.lag).sum()) > 0
    phi = np.random.default_rng(13).uniform(0.0, 1.0, (P.C, G, 8))
    for _ in range(2):
        ref = P.transport_step(phi, threads=8)
        out = torch.zeros_like(_dev(phi))
        prob.sweep(_dev(phi), out)
        assert _rel(out.cpu().numpy(), ref) < TOL[precision]
        phi = ref
    st = prob.stats()
    assert st["tasks_executed"] == st["n_tasks"]
    assert st["kernel_mode"] == (9 if G >= 8 and opts.get("staging", 0) != 1 else 8)


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
def test_lagged_source_iteration_matches_oracle(precision):
    """Converged source iteration with lagged faces against the oracle's (whose fixed point is
    pinned to the lag-free dense solves)."""
    cfg = _cyclic(4)
    P = oh.ProblemHex(cfg, lag=True)
    ref, it_ref, _ = P.source_iterate(1e-10, 2000, threads=8)
    prob = tf.Problem.from_config(cfg, precision=precision, lag_cycles=1)
    phi = torch.zeros((P.C, 4, 8), dtype=torch.float64, device="cuda")
    res = prob.source_iterate(phi, 1e-10 if precision == tf.TF_FP64 else 1e-6, 2000)
    assert res["converged"]
    if precision == tf.TF_FP64:
        assert abs(res["iterations"] - it_ref) <= 1
    assert _rel(phi.cpu().numpy(), ref) < (1e-8 if precision == tf.TF_FP64 else 2e-5)
    assert res["balance"] < (1e-8 if precision == tf.TF_FP64 else 1e-5), res["balance"]


@pytest.mark.parametrize("schedule", [tf.TF_SCHED_BSP, tf.TF_SCHED_BSP_LAUNCH])
def test_lagged_bulk_synchronous_schedules_same_result(schedule):
    cfg = _cyclic(8)
    a = tf.Problem.from_config(cfg, lag_cycles=1)
    b = tf.Problem.from_config(cfg, lag_cycles=1, schedule=schedule)
    phi = _dev(np.random.default_rng(2).uniform(0.0, 1.0, (len(cfg["hexes"]), 8, 8)))
    for _ in range(2):
        out_a, out_b = torch.zeros_like(phi), torch.zeros_like(phi)
        a.sweep(phi, out_a)
        b.sweep(phi, out_b)
        assert torch.equal(out_a, out_b)
        phi = out_a


def test_lagged_problem_is_not_batched():
    cfg = _cyclic(3)
    a = tf.Problem.from_config(cfg, lag_cycles=1)
    b = tf.Problem.from_config(_box(n=3, G=3))
    phis = [torch.zeros((p.n_cells, 3, 8), dtype=torch.float64, device="cuda") for p in (a, b)]
    with pytest.raises(tf.TfError) as e:
        tf.sweep_batch([a, b], phis, phis)
    assert e.value.status == tf.TF_ERR_ARG


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
def test_lagged_steps_with_inflow_and_s1_match_oracle(precision):
    """Lagged back edges together with prescribed boundary inflow and the S1 source: two
    consecutive transport steps against the oracle."""
    cfg = _cyclic(8)
    C, nv = len(cfg["hexes"]), len(cfg["xyz"])
    rng = np.random.default_rng(29)
    S1 = rng.uniform(-1.0, 1.0, (C, 8, 3))
    psi_in = rng.uniform(0.0, 1.0, (nv, 8))
    P = oh.ProblemHex(cfg, S1=S1, psi_in=psi_in, lag=True)
    prob = tf.Problem.from_config(cfg, S1=S1, psi_inflow=psi_in, precision=precision, lag_cycles=1)
    phi = rng.uniform(0.0, 1.0, (C, 8, 8))
    for _ in range(2):
        ref = P.transport_step(phi, threads=8)
        out = torch.zeros_like(_dev(phi))
        prob.sweep(_dev(phi), out)
        assert _rel(out.cpu().numpy(), ref) < TOL[precision]
        phi = ref
