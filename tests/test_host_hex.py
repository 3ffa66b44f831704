"""The library's host path for trilinear hexahedra (tf_mesh_create_hex, tf_mesh_hex_integrals,
tf_mesh_geometry, tf_graph_levels) against the hexahedral oracle, on the CPU: element
integrals within rounding (the library integrates polynomials exactly, the oracle by
Gauss quadrature), integrated face area vectors, neighbours, face classification and
t-levels bit for bit."""
import numpy as np
import pytest

import workloads as W
from oracle import product_quadrature
from oracle import q1hex as H

tf = pytest.importorskip("paper_2510_11513_gb300")


@pytest.mark.parametrize("n,twist,seed", [(3, 0.0, 1), (4, 0.6, 2), (6, 1.0, 3)])
def test_integrals_and_geometry_match_oracle(n, twist, seed):
    xyz, hexes = W.twisted_hex_mesh(n, seed, twist=twist)
    ref = H.geometry(xyz, hexes)
    m = tf.HexMesh(xyz, hexes)
    g = m.geometry()
    it = m.integrals()
    scale = np.max(ref["vol"])
    assert np.max(np.abs(g["vol"] - ref["vol"])) < 1e-14 * scale
    assert np.max(np.abs(it["mass"] - ref["mass"])) < 1e-17
    assert np.max(np.abs(it["grad"] - ref["grad"])) < 1e-15
    assert np.max(np.abs(it["face"] - ref["face"])) < 1e-15
    # the integrated face area vectors follow one canonical formula: bit for bit
    assert np.array_equal(g["normal"], ref["nbar"])
    assert np.array_equal(g["nbr"], ref["nbr"])
    assert np.array_equal(g["nbr_node"], ref["nbr_node"])


@pytest.mark.parametrize("twist,jitter,n_polar,n_az", [(0.0, 0.15, 2, 8), (0.25, 0.0, 8, 32), (0.5, 0.05, 4, 8),
                                                        (0.25, 0.05, 8, 16)])
def test_graph_bit_exact(twist, jitter, n_polar, n_az):
    cfg = W.hex_problem(W.small_box(n=6, G=1, n_polar=n_polar, n_az=n_az), twist=twist, jitter=jitter)
    geom = H.geometry(cfg["xyz"], cfg["hexes"])
    om, _ = product_quadrature(n_polar, n_az)
    inflow_ref, level_ref = H.graph(geom, om)
    m = tf.HexMesh(cfg["xyz"], cfg["hexes"])
    q = tf.Quadrature(n_polar, n_az)
    assert np.array_equal(q.omega, om)
    inflow, level = tf.tf_graph_levels(m.h, q.h, m.n_cells, q.n_dirs)
    assert np.array_equal(inflow, inflow_ref)
    assert np.array_equal(level, level_ref)


def test_errors():
    xyz, hexes = W.twisted_hex_mesh(2, 1)
    bad = hexes.copy()
    bad[0, [0, 1]] = bad[0, [1, 0]]  # mirrored cell
    with pytest.raises(tf.TfError) as e:
        tf.HexMesh(xyz, bad)
    assert e.value.status == tf.TF_ERR_MESH
    bad = hexes.copy()
    bad[1, 3] = len(xyz)
    with pytest.raises(tf.TfError) as e:
        tf.HexMesh(xyz, bad)
    assert e.value.status == tf.TF_ERR_MESH
    with pytest.raises(tf.TfError) as e:
        tf.HexMesh(xyz, np.concatenate([hexes, hexes[:1]]))
    assert e.value.status == tf.TF_ERR_MESH
    with pytest.raises(tf.TfError) as e:
        tf.HexMesh(xyz[:0], hexes[:0])
    assert e.value.status == tf.TF_ERR_ARG
    tet = tf.Mesh(*W.jittered_kuhn_mesh(2, 1))
    with pytest.raises(tf.TfError) as e:
        tf.tf_mesh_hex_integrals(tet.h, 48)
    assert e.value.status == tf.TF_ERR_ARG
    m = tf.HexMesh(xyz, hexes)
    q = tf.Quadrature(2, 4)
    C = len(hexes)
    with pytest.raises(tf.TfError) as e:  # hexahedra: trilinear only (checked before any device work)
        tf.tf_problem_create(m.h, q.h, 1, 1, np.zeros(C, np.int32), np.ones((1, 1)), np.zeros((1, 1, 1)),
                             np.zeros((C, 1, 8)), S1=np.zeros((C, 1, 3)), opt=tf.options(order=2))
    assert e.value.status == tf.TF_ERR_ARG


def test_cycle_reported_like_the_oracle():
    """A strongly twisted, jittered grid whose sweep graph has a cycle for some of 64
    directions: the library reports TF_ERR_CYCLE where the oracle reports its cycle."""
    from oracle import OracleError
    cfg = W.hex_problem(W.small_box(n=5, G=1, n_polar=4, n_az=16), twist=1.3, jitter=0.15)
    geom = H.geometry(cfg["xyz"], cfg["hexes"])
    om, _ = product_quadrature(4, 16)
    with pytest.raises(OracleError):
        H.graph(geom, om)
    m = tf.HexMesh(cfg["xyz"], cfg["hexes"])
    q = tf.Quadrature(4, 16)
    with pytest.raises(tf.TfError) as e:
        tf.tf_graph_levels(m.h, q.h, m.n_cells, q.n_dirs)
    assert e.value.status == tf.TF_ERR_CYCLE


def test_graph_bit_exact_paper_sized_workload():
    """The paper's runtime-table size (16^3 twisted hexahedra, 256 directions): inflow masks and
    t-levels of the library equal the oracle's."""
    cfg = W.paper_hex_box()
    geom = H.geometry(cfg["xyz"], cfg["hexes"])
    om, _ = product_quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    inflow_ref, level_ref = H.graph(geom, om)
    m = tf.HexMesh(cfg["xyz"], cfg["hexes"])
    q = tf.Quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    inflow, level = tf.tf_graph_levels(m.h, q.h, m.n_cells, q.n_dirs)
    assert np.array_equal(inflow, inflow_ref) and np.array_equal(level, level_ref)
    assert level.max() + 1 == 61
