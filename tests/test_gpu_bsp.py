"""The bulk-synchronous sweep schedules (level by level, a barrier after every
(octant, t-level) bucket; Sec. 2.1) against the oracle and against the
many-task schedule.

Both schedules run the same local solves (with their own task grain) and every
solve reads only finished upwind rows, so psi, phi and the whole source
iteration are bit-identical between them; the oracle bounds both (1e-11 FP64,
2e-5 FP32).
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
import paper_2510_11513_gb300 as tf  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {tf.TF_FP64: 1e-11, tf.TF_FP32: 2e-5}
SCHEDULES = [tf.TF_SCHED_BSP, tf.TF_SCHED_BSP_LAUNCH]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _expected_buckets(P, dir_chunk):
    """Buckets per sweep from the oracle's t-levels: per direction chunk, per octant
    present in it, the largest level count over the octant's directions."""
    D = P.D
    Dc = dir_chunk if dir_chunk > 0 else D
    octant = ((P.omega[:, 0] < 0) * 1 + (P.omega[:, 1] < 0) * 2 + (P.omega[:, 2] < 0) * 4).astype(int)
    levels = P.level.max(axis=1) + 1
    n = 0
    for a0 in range(0, D, Dc):
        a1 = min(D, a0 + Dc)
        for o in set(octant[a0:a1].tolist()):
            n += int(max(levels[a] for a in range(a0, a1) if octant[a] == o))
    return n


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("precision,G,opts", [
    (tf.TF_FP64, 4, {}), (tf.TF_FP32, 4, {}),                            # any-G path
    (tf.TF_FP32, 6, dict(cells_per_task=5)),                             # packed group pairs
    (tf.TF_FP32, 32, dict(pairing=1)),                                   # staged, two stages
    (tf.TF_FP64, 32, dict(cells_per_task=7, dir_chunk=11)),              # staged, three stages, chunks
    (tf.TF_FP32, 64, dict(pairing=1, staging=1, cells_per_task=9)),      # registers, G = 64
    (tf.TF_FP32, 37, dict(cells_per_task=3, dir_chunk=5)),               # ragged G, many chunks
])
def test_bsp_sweep_matches_oracle_and_amt_bitwise(schedule, precision, G, opts):
    cfg = W.small_box(n=4 if G >= 32 else 6, G=G, n_polar=4, n_az=8)
    P = oracle.Problem(cfg)
    phi_in = np.random.default_rng(5).uniform(0.0, 1.0, (P.C, G, 4))
    ref = P.transport_step(phi_in, threads=8)
    amt = tf.Problem.from_config(cfg, precision=precision, **opts)
    bsp = tf.Problem.from_config(cfg, precision=precision, schedule=schedule, **opts)
    out_a = torch.zeros_like(_dev(phi_in))
    out_b = torch.zeros_like(out_a)
    amt.sweep(_dev(phi_in), out_a)
    bsp.sweep(_dev(phi_in), out_b)
    b = out_b.cpu().numpy()
    assert _rel(b, ref) < TOL[precision]
    assert np.array_equal(b, out_a.cpu().numpy())
    st = bsp.stats()
    assert st["tasks_executed"] == st["n_tasks"]
    if "cells_per_task" not in opts:
        # the bulk-synchronous default grain: a quarter of the t-level blocks', at least 2; on the
        # packed-pairs path a quarter of 256 / G cells (at most 16), the grain it was measured at
        pairing = opts.get("pairing", 0)
        paired = precision == tf.TF_FP32 and G % 2 == 0 and (pairing == 2 or (pairing == 0 and G % 32 != 0))
        if paired:
            assert st["cells_per_task"] == max(2, max(4, min(16, 256 // G)) // 4)
        else:
            lv = tf.Problem.from_config(cfg, precision=precision, task_shape=tf.TF_TASK_LEVELS, **opts)
            assert st["cells_per_task"] == max(2, lv.stats()["cells_per_task"] // 4)
            lv.close()
    assert st["n_buckets"] == _expected_buckets(P, opts.get("dir_chunk", 0))
    assert amt.stats()["n_buckets"] == 0
    # psi of one direction too (the rows the downwind tasks consumed; the last chunk's)
    d = P.D - 1
    pa = torch.empty((P.C, G, 4), dtype=torch.float64 if precision == tf.TF_FP64 else torch.float32, device="cuda")
    pb = torch.empty_like(pa)
    amt.psi(d, pa)
    bsp.psi(d, pb)
    assert torch.equal(pa, pb)


@pytest.mark.parametrize("precision", [tf.TF_FP64, tf.TF_FP32])
def test_bsp_source_iteration_identical_to_amt(precision):
    """Source iteration to 1e-6 on the two-material box: the same iterations, the
    same residual history bit for bit, the same phi, and the device balance holds."""
    cfg = W.two_material_box(n=6, G=12, n_polar=2, n_az=8)
    res, phis = [], []
    for schedule in (tf.TF_SCHED_AMT, tf.TF_SCHED_BSP, tf.TF_SCHED_BSP_LAUNCH):
        prob = tf.Problem.from_config(cfg, precision=precision, schedule=schedule)
        phi = torch.zeros((prob.n_cells, prob.n_groups, 4), dtype=torch.float64, device="cuda")
        res.append(prob.source_iterate(phi, 1e-6, 200, history=True))
        phis.append(phi.cpu().numpy())
    for r, p in zip(res[1:], phis[1:]):
        assert r["converged"] and r["iterations"] == res[0]["iterations"]
        assert np.array_equal(r["residual_history"], res[0]["residual_history"])
        assert np.array_equal(p, phis[0])
        assert r["balance"] < (1e-12 if precision == tf.TF_FP64 else 1e-5)


def test_bsp_barrier_wait_limit_returns_timeout():
    """Fault injection on the host side: every grid barrier waits for one CTA more
    than the grid holds, so each CTA's bounded wait runs out; the kernel returns
    TF_ERR_TIMEOUT and the device stays usable."""
    cfg = W.small_box(n=3, G=2, n_polar=2, n_az=8)
    C = 6 * 27
    bad = tf.Problem.from_config(cfg, precision=tf.TF_FP64, schedule=tf.TF_SCHED_BSP, inject_stall=1,
                                 wait_limit_s=0.25)
    phi_in = _dev(np.random.default_rng(3).uniform(0.0, 1.0, (C, 2, 4)))
    out = torch.zeros_like(phi_in)
    with pytest.raises(tf.TfError) as e:
        bad.sweep(phi_in, out)
    assert e.value.status == tf.TF_ERR_TIMEOUT
    good = tf.Problem.from_config(cfg, precision=tf.TF_FP64, schedule=tf.TF_SCHED_BSP)
    good.sweep(phi_in, out)
    ref = oracle.Problem(cfg).transport_step(phi_in.cpu().numpy())
    assert _rel(out.cpu().numpy(), ref) < 1e-11


def test_bsp_rejected_where_undefined():
    cfg = W.small_box(n=3, G=2, n_polar=2, n_az=8)
    with pytest.raises(tf.TfError) as e:
        tf.Problem.from_config(cfg, schedule=3)
    assert e.value.status == tf.TF_ERR_ARG
    with pytest.raises(tf.TfError) as e:
        tf.Problem.from_config(cfg, schedule=tf.TF_SCHED_BSP_LAUNCH, inject_stall=1)
    assert e.value.status == tf.TF_ERR_ARG
    a = tf.Problem.from_config(cfg)
    b = tf.Problem.from_config(cfg, schedule=tf.TF_SCHED_BSP)
    phis = [torch.zeros((6 * 27, 2, 4), dtype=torch.float64, device="cuda") for _ in range(2)]
    with pytest.raises(tf.TfError) as e:
        tf.sweep_batch([a, b], phis, phis)
    assert e.value.status == tf.TF_ERR_ARG
