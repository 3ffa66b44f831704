"""Task graphs of the sweep (tf_graph_tasks), checked on the CPU against the oracle's own cell
dependency graph (its neighbours and inflow masks, which are bit-equal to the library's).

Both task shapes must cover every (direction, cell) once, list a task's cells so that an
upwind cell in the same task comes first, give each task the in-degree of its distinct other
upwind tasks (the dependency counter's start, Sec. 3.5), and form an acyclic task graph per
direction (Sec. 2.1: the sweep is a DAG per angle).  t-level blocks hold cells of one t-level;
spatial patches hold at most 64 cells and keep most upwind faces inside the task."""
import numpy as np
import pytest

import oracle
import paper_2510_11513_gb300 as tf
import workloads as W


def _cell_edges(og, inflow):
    """Upwind cell of every (direction, cell, face): -1 unless the face is an interior inflow face."""
    nbr = og["nbr"]
    fin = ((inflow[:, :, None] >> np.arange(4)) & 1).astype(bool)
    return np.where(fin & (nbr[None] >= 0), nbr[None], -1)


def _check(task_of, position, indeg, up, level, shape):
    D, C = task_of.shape
    T = len(indeg)
    dir_of = np.full(T, -1)
    for a in range(D):
        ts = np.unique(task_of[a])
        assert np.all(dir_of[ts] == -1), "a task spans two directions"
        dir_of[ts] = a
    assert np.all(dir_of >= 0) and task_of.min() >= 0 and task_of.max() == T - 1
    # positions: 0 .. n-1 inside every task
    flat_t = task_of.ravel()
    sizes = np.bincount(flat_t, minlength=T)
    key = flat_t.astype(np.int64) * 4096 + position.ravel()
    assert len(np.unique(key)) == D * C
    assert np.all(position.ravel() < sizes[flat_t])
    if shape == tf.TF_TASK_PATCHES:
        assert sizes.max() <= 64
    valid = up >= 0
    uu = np.where(valid, up, 0)
    t_up = np.take_along_axis(task_of, uu.reshape(D, -1), 1).reshape(D, C, 4)
    p_up = np.take_along_axis(position, uu.reshape(D, -1), 1).reshape(D, C, 4)
    same = valid & (t_up == task_of[:, :, None])
    assert np.all(p_up[same] < np.broadcast_to(position[:, :, None], same.shape)[same]), "upwind listed after downwind"
    # in-degrees and acyclicity of the task graph
    src = t_up[valid & ~same]
    dst = np.broadcast_to(task_of[:, :, None], same.shape)[valid & ~same]
    edges = np.unique(np.stack([src, dst], 1), axis=0)
    assert np.array_equal(np.bincount(edges[:, 1], minlength=T), indeg)
    deg = indeg.copy()
    order = np.argsort(edges[:, 0], kind="stable")
    edges = edges[order]
    starts = np.searchsorted(edges[:, 0], np.arange(T + 1))
    ready = list(np.flatnonzero(deg == 0))
    seen = 0
    while ready:
        t = ready.pop()
        seen += 1
        for d in edges[starts[t]:starts[t + 1], 1]:
            deg[d] -= 1
            if deg[d] == 0:
                ready.append(d)
    assert seen == T, "the task graph has a cycle"
    if shape == tf.TF_TASK_LEVELS:
        assert not same.any()
        for a in range(D):
            lv = np.zeros(T, np.int64) - 1
            np.maximum.at(lv, task_of[a], level[a])
            assert np.array_equal(lv[task_of[a]], level[a]), "a t-level block mixes levels"
    return same.sum() / max(valid.sum(), 1)


@pytest.mark.parametrize("G,opts", [
    (64, dict()),                                     # the default for G = 64: patches
    (64, dict(task_shape=tf.TF_TASK_LEVELS)),
    (32, dict(task_shape=tf.TF_TASK_PATCHES, patch_extent=3.0, cells_per_task=24)),
    (32, dict(precision=tf.TF_FP64, task_shape=tf.TF_TASK_PATCHES)),  # three stages
    (8, dict()),                                      # packed group pairs: t-level blocks
])
def test_task_graph_against_oracle(G, opts):
    cfg = W.two_material_box(n=7, G=G, n_polar=4, n_az=8)
    m = tf.Mesh(cfg["xyz"], cfg["tets"])
    q = tf.Quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    og = oracle.geometry(cfg["xyz"], cfg["tets"])
    om, _ = oracle.product_quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    inflow, level = oracle.graph(og, om)
    o = tf.options(**opts)
    task_of, position, indeg = tf.tf_graph_tasks(m.h, q.h, m.n_cells, q.n_dirs, G, o)
    patches = o.task_shape == tf.TF_TASK_PATCHES or (o.task_shape == tf.TF_TASK_AUTO and G % 32 == 0)
    frac = _check(task_of, position, indeg, _cell_edges(og, inflow), level,
                  tf.TF_TASK_PATCHES if patches else tf.TF_TASK_LEVELS)
    if patches:
        assert frac > 0.5  # most upwind faces stay inside their task


def test_patches_keep_most_faces_inside_on_the_bench_mesh_sample():
    """The 48^3 bench mesh (663,552 tetrahedra) with a sample of its 192 directions: the patch
    graph is valid and more than half of the upwind faces are inside their task."""
    cfg = W.corner_source_box()
    og = oracle.geometry(cfg["xyz"], cfg["tets"])
    om, w = oracle.product_quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    sample = [0, 47, 95, 131, 191]
    inflow, level = oracle.graph(og, om[sample])
    m = tf.Mesh(cfg["xyz"], cfg["tets"])
    q = tf.Quadrature(omega=om[sample], w=w[sample])
    task_of, position, indeg = tf.tf_graph_tasks(m.h, q.h, m.n_cells, len(sample), 64)
    frac = _check(task_of, position, indeg, _cell_edges(og, inflow), level, tf.TF_TASK_PATCHES)
    assert 0.5 < frac < 0.8


def test_task_shape_arguments():
    cfg = W.small_box(n=3, G=4)
    m = tf.Mesh(cfg["xyz"], cfg["tets"])
    q = tf.Quadrature(2, 4)
    for bad in (dict(task_shape=tf.TF_TASK_PATCHES),                         # G = 4: packed pairs
                dict(task_shape=7), dict(patch_extent=-1.0)):
        with pytest.raises(tf.TfError) as e:
            tf.tf_graph_tasks(m.h, q.h, m.n_cells, q.n_dirs, 4, tf.options(**bad))
        assert e.value.status == tf.TF_ERR_ARG
    with pytest.raises(tf.TfError) as e:  # patches: at most 64 cells
        tf.tf_graph_tasks(m.h, q.h, m.n_cells, q.n_dirs, 32, tf.options(task_shape=tf.TF_TASK_PATCHES,
                                                                        cells_per_task=65))
    assert e.value.status == tf.TF_ERR_ARG
    with pytest.raises(tf.TfError) as e:  # patches and a bulk-synchronous schedule
        tf.tf_graph_tasks(m.h, q.h, m.n_cells, q.n_dirs, 32, tf.options(task_shape=tf.TF_TASK_PATCHES,
                                                                        schedule=tf.TF_SCHED_BSP))
    assert e.value.status == tf.TF_ERR_ARG
