"""Batched problems in shared persistent launches (tf_sweep / tf_source_iterate
with several handles): each problem's result must equal its oracle result and
its result when run alone, whatever mix of sizes, direction sets, group counts
(kernel variants) and direction chunks share the launch."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
import paper_2510_11513_gb300 as tf  # noqa: E402

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


MIX = [  # (n, G, n_polar, n_az, extra options)
    (5, 8, 2, 8, {}), (4, 16, 4, 8, {}), (6, 32, 2, 8, {}), (3, 64, 4, 8, dict(dir_chunk=11)), (4, 5, 2, 8, {}),
    (3, 64, 2, 8, dict(pairing=2)),
]


def _problems(precision, mix=MIX):
    cfgs, probs = [], []
    for j, (n, G, npol, naz, opts) in enumerate(mix):
        seed = W.BASE_SEED + 100 + j
        cfg = W.two_material_box(n=n, G=G, n_polar=npol, n_az=naz, seed=seed)
        while cfg["Q"].sum() == 0.0:  # small boxes can draw only the source-free material
            seed += 1000
            cfg = W.two_material_box(n=n, G=G, n_polar=npol, n_az=naz, seed=seed)
        cfgs.append(cfg)
        probs.append(tf.Problem.from_config(cfg, precision=precision, **opts))
    return cfgs, probs


@pytest.mark.parametrize("precision,tol", [(tf.TF_FP32, 2e-5), (tf.TF_FP64, 1e-11)])
def test_batched_sweep_matches_oracle_and_single(precision, tol):
    mix = MIX if precision == tf.TF_FP32 else [m for m in MIX if "pairing" not in m[4]]
    cfgs, probs = _problems(precision, mix)
    rng = np.random.default_rng(5)
    ins = [rng.uniform(0, 1, (p.n_cells, p.n_groups, 4)) for p in probs]
    dins = [torch.from_numpy(x).cuda() for x in ins]
    outs = [torch.zeros_like(x) for x in dins]
    tf.sweep_batch(probs, dins, outs)
    for cfg, p, x, o in zip(cfgs, probs, ins, outs):
        ref = oracle.Problem(cfg).transport_step(x, threads=8)
        assert _rel(o.cpu().numpy(), ref) < tol
        alone = torch.zeros_like(o)
        p.sweep(torch.from_numpy(x).cuda(), alone)
        assert _rel(o.cpu().numpy(), alone.cpu().numpy()) < (1e-6 if precision == tf.TF_FP32 else 1e-13)


def test_batched_source_iteration_matches_single_runs():
    cfgs, probs = _problems(tf.TF_FP32, MIX[:4])
    phis = [torch.zeros((p.n_cells, p.n_groups, 4), dtype=torch.float64, device="cuda") for p in probs]
    st, infos = tf.source_iterate_batch(probs, phis, 1e-6, 500, history=True)
    assert st == tf.TF_OK
    for cfg, p, ph, info in zip(cfgs, probs, phis, infos):
        assert info["converged"] and info["seconds"] > 0
        alone = torch.zeros_like(ph)
        r = p.source_iterate(alone, 1e-6, 500)
        assert abs(r["iterations"] - info["iterations"]) <= 1
        assert _rel(ph.cpu().numpy(), alone.cpu().numpy()) < 1e-5
        ref, _, _ = oracle.Problem(cfg).source_iterate(1e-12, 1000, threads=8)
        assert _rel(ph.cpu().numpy(), ref) < 2e-5
        assert abs(info["integrated_total"] - r["integrated_total"]) / r["integrated_total"] < 1e-5
    # problems that converge earlier leave the launch; their time is recorded when they converge
    order = np.argsort([i["iterations"] for i in infos])
    secs = [infos[k]["seconds"] for k in order]
    assert all(a <= b + 1e-9 for a, b in zip(secs, secs[1:]))


def test_autotuned_task_grain():
    cfg = W.two_material_box(n=6, G=16, n_polar=4, n_az=8, seed=W.BASE_SEED + 77)
    p = tf.Problem.from_config(cfg, precision=tf.TF_FP32, cells_per_task=-1)
    st = p.stats()
    assert st["tuned_n"] >= 2 and not st["tuned_cached"]
    assert st["cells_per_task"] in st["tuned_candidates"]
    # the default grain is the first candidate (the incumbent); another grain replaces it only
    # when its trial is at least 5 % faster than the best so far
    n = st["tuned_n"]
    cand, secs = list(st["tuned_candidates"][:n]), list(st["tuned_seconds"][:n])
    best, best_t = cand[0], secs[0]
    for b, t in zip(cand[1:], secs[1:]):
        if 0.0 <= t < 0.95 * best_t:
            best, best_t = b, t
    assert st["cells_per_task"] == best
    # phase 2 (kernel variant, octant window) leaves valid knobs, and the problem runs with them
    assert st["tuned_pairing"] in (0, 1, 2) and st["tuned_staging"] in (0, 1) and st["tuned_window"] in (0, 2)
    if st["tuned_pairing"] == 1:
        assert st["kernel_mode"] != 3
    if st["tuned_pairing"] == 0:
        assert st["kernel_mode"] == 3  # 16 groups: packed pairs unless turned off
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (p.n_cells, 16, 4))
    out = torch.zeros((p.n_cells, 16, 4), dtype=torch.float64, device="cuda")
    p.sweep(torch.from_numpy(x).cuda(), out)
    assert _rel(out.cpu().numpy(), oracle.Problem(cfg).transport_step(x, threads=8)) < 2e-5
    # same class (precision, groups, directions, size): the cached choice is reused
    q = tf.Problem.from_config(W.two_material_box(n=6, G=16, n_polar=4, n_az=8, seed=W.BASE_SEED + 78),
                               precision=tf.TF_FP32, cells_per_task=-1)
    assert q.stats()["tuned_cached"] == 1 and q.stats()["cells_per_task"] == st["cells_per_task"]
