"""Spatial-patch tasks (tf_options.task_shape = TF_TASK_PATCHES) on the GPU.  A patch lists cells
that depend on each other; the kernel variants that take them (lanes over one cell's groups:
registers, two- and three-stage shared-memory staging) hand a cell's solution to the later
cells of the same task through shared memory, or copy it back from L2.  The local solves are
the same arithmetic on the same upwind values, so psi and phi must be bit-identical to the
t-level-block tasks, and within tolerance of the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
import paper_2510_11513_gb300 as tf  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {tf.TF_FP64: 1e-11, tf.TF_FP32: 2e-5}


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision,G,opts", [
    (tf.TF_FP32, 64, {}),                                   # two stages (the bench's variant)
    (tf.TF_FP32, 32, {}),
    (tf.TF_FP32, 128, dict(cells_per_task=20)),
    (tf.TF_FP32, 64, dict(staging=3, patch_extent=3.0)),    # three stages
    (tf.TF_FP32, 64, dict(staging=1)),                      # registers only
    (tf.TF_FP64, 32, {}),                                   # FP64: three stages
    (tf.TF_FP64, 64, dict(staging=1, dir_chunk=7)),         # registers, several direction chunks
    (tf.TF_FP32, 32, dict(cells_per_task=5, dir_chunk=9)),  # small pieces, chunks
])
def test_patches_bit_equal_to_level_blocks_and_match_oracle(precision, G, opts):
    cfg = W.two_material_box(n=7, G=G, n_polar=4, n_az=8)
    C = len(cfg["tets"])
    phi_in = torch.from_numpy(np.random.default_rng(21).uniform(0.0, 1.0, (C, G, 4))).cuda()
    lv = tf.Problem.from_config(cfg, precision=precision, task_shape=tf.TF_TASK_LEVELS,
                                **{k: v for k, v in opts.items() if k not in ("patch_extent",)})
    pa = tf.Problem.from_config(cfg, precision=precision, task_shape=tf.TF_TASK_PATCHES, **opts)
    assert pa.stats()["task_shape"] == tf.TF_TASK_PATCHES and lv.stats()["task_shape"] == tf.TF_TASK_LEVELS
    out_l, out_p = torch.zeros_like(phi_in), torch.zeros_like(phi_in)
    lv.sweep(phi_in, out_l)
    pa.sweep(phi_in, out_p)
    st = pa.stats()
    assert st["tasks_executed"] == st["n_tasks"]
    assert torch.equal(out_l, out_p)
    # psi of the last direction (the rows the in-task handoffs produced), bit for bit
    D = pa.n_dirs
    dt = torch.float64 if precision == tf.TF_FP64 else torch.float32
    a = torch.empty((C, G, 4), dtype=dt, device="cuda")
    b = torch.empty_like(a)
    lv.psi(D - 1, a)
    pa.psi(D - 1, b)
    assert torch.equal(a, b)
    ref = oracle.Problem(cfg).transport_step(phi_in.cpu().numpy(), threads=8)
    assert _rel(out_p.cpu().numpy(), ref) < TOL[precision]


def test_patches_source_iteration_and_balance():
    cfg = W.two_material_box(n=8, G=32, n_polar=4, n_az=8)
    res = []
    for shape in (tf.TF_TASK_LEVELS, tf.TF_TASK_PATCHES):
        p = tf.Problem.from_config(cfg, precision=tf.TF_FP32, task_shape=shape)
        phi = torch.zeros((p.n_cells, 32, 4), dtype=torch.float64, device="cuda")
        r = p.source_iterate(phi, 1e-6, 300, history=True)
        assert r["converged"] and r["balance"] < 1e-5
        res.append((phi.cpu().numpy(), r))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1]["residual_history"], res[1][1]["residual_history"])


def test_patches_in_a_batch_and_on_the_bench_mesh_size():
    """Patch problems in a batched launch beside t-level problems, each bit-equal to its own run."""
    cfgs = [W.two_material_box(n=6, G=64, n_polar=4, n_az=8, seed=91), W.two_material_box(n=9, G=32, n_polar=2, n_az=8)]
    shapes = [tf.TF_TASK_PATCHES, tf.TF_TASK_LEVELS]
    probs = [tf.Problem.from_config(c, precision=tf.TF_FP32, task_shape=s) for c, s in zip(cfgs, shapes)]
    ins = [torch.from_numpy(np.random.default_rng(4).uniform(0, 1, (p.n_cells, p.n_groups, 4))).cuda() for p in probs]
    outs = [torch.zeros_like(x) for x in ins]
    tf.sweep_batch(probs, ins, outs)
    for p, x, o in zip(probs, ins, outs):
        single = torch.zeros_like(x)
        p.sweep(x, single)
        assert torch.equal(single, o)
