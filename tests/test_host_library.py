"""Host-side tests of the native library (no GPU): it loads, exports every
symbol the C header declares, and its host precompute (geometry, quadrature,
face classification, t-levels) is bit-identical to the oracle's."""
import re

import numpy as np
import pytest

import oracle
import paper_2510_11513_gb300 as tf
import workloads as W
from paper_2510_11513_gb300 import build as tfbuild


def test_library_exports_every_declared_symbol():
    import ctypes
    import os
    inc = os.path.join(os.path.dirname(tfbuild.HERE), "include")
    headers = sorted(f for f in os.listdir(inc) if f.endswith(".h"))
    assert {"tfsweep.h", "tflearn.h"} <= set(headers)
    declared = set()
    for h in headers:
        text = open(os.path.join(inc, h)).read()
        declared |= set(re.findall(r"^\s*(?:tf_status|void|const char \*)\s*(tf_\w+)\s*\(", text, re.M))
    assert {"tf_mesh_create", "tf_quadrature_create", "tf_problem_create", "tf_sweep", "tf_source_iterate",
            "tf_destroy", "tf_mlp_create", "tf_mlp_train", "tf_mlp_predict_phi"} <= declared
    lib = ctypes.CDLL(tf.load().__dict__["_name"])
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(tf.tfsweep.SYMBOLS) >= declared


@pytest.mark.parametrize("maker,kw", [
    (W.small_box, dict()),
    (W.two_material_box, dict(n=8)),
    (W.corner_source_box, dict(n=6, G=8)),
])
def test_mesh_quadrature_graph_bit_exact(maker, kw):
    cfg = maker(**kw)
    m = tf.Mesh(cfg["xyz"], cfg["tets"])
    q = tf.Quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    g = m.geometry()
    og = oracle.geometry(cfg["xyz"], cfg["tets"])
    for k in ("vol", "normal", "nbr", "nbr_node"):
        assert np.array_equal(g[k], og[k]), k
    om, w = oracle.product_quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    assert np.array_equal(q.omega, om) and np.array_equal(q.w, w)
    inflow, level = tf.tf_graph_levels(m.h, q.h, m.n_cells, q.n_dirs)
    oi, ol = oracle.graph(og, om)
    assert np.array_equal(inflow, oi)
    assert np.array_equal(level, ol)


def test_graph_bit_exact_full_size_two_material_sample():
    """Full 32^3 mesh with the 128-direction set: levels of a direction sample."""
    cfg = W.two_material_box()
    m = tf.Mesh(cfg["xyz"], cfg["tets"])
    q = tf.Quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    og = oracle.geometry(cfg["xyz"], cfg["tets"])
    g = m.geometry()
    assert np.array_equal(g["normal"], og["normal"])
    om, w = oracle.product_quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    sample = [0, 37, 64, 127]
    q2 = tf.Quadrature(omega=om[sample], w=w[sample])
    inflow, level = tf.tf_graph_levels(m.h, q2.h, m.n_cells, len(sample))
    oi, ol = oracle.graph(og, om[sample])
    assert np.array_equal(inflow, oi) and np.array_equal(level, ol)


def test_mesh_errors():
    xyz, tets = W.jittered_kuhn_mesh(2, 5)
    bad = tets.copy()
    bad[3, [2, 3]] = bad[3, [3, 2]]
    with pytest.raises(tf.TfError) as e:
        tf.Mesh(xyz, bad)
    assert e.value.status == tf.TF_ERR_MESH
    with pytest.raises(tf.TfError) as e:
        tf.Mesh(xyz, np.concatenate([tets, tets[:1]]))
    assert e.value.status == tf.TF_ERR_MESH
    oob = tets.copy()
    oob[0, 0] = len(xyz)
    with pytest.raises(tf.TfError) as e:
        tf.Mesh(xyz, oob)
    assert e.value.status == tf.TF_ERR_MESH


def test_argument_errors():
    with pytest.raises(tf.TfError) as e:
        tf.Quadrature(0, 8)
    assert e.value.status == tf.TF_ERR_ARG
    with pytest.raises(tf.TfError) as e:
        tf.Quadrature(omega=np.array([[1.0, 1.0, 0.0]]), w=np.array([1.0]))
    assert e.value.status == tf.TF_ERR_ARG
    cfg = W.small_box(n=2)
    m = tf.Mesh(cfg["xyz"], cfg["tets"])
    q = tf.Quadrature(2, 8)
    bad_mat = cfg["cell_material"].copy()
    bad_mat[0] = 5
    with pytest.raises(tf.TfError) as e:
        tf.Problem(m, q, cfg["n_groups"], 1, bad_mat, cfg["sigma_t"], cfg["sigma_s"], cfg["Q"])
    assert e.value.status == tf.TF_ERR_ARG
    with pytest.raises(tf.TfError) as e:
        tf.Problem(m, q, 0, 1, cfg["cell_material"], cfg["sigma_t"], cfg["sigma_s"], cfg["Q"])
    assert e.value.status == tf.TF_ERR_ARG


def test_status_strings():
    lib = tf.load()
    for s in range(9):
        assert lib.tf_status_string(s)
