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


# ------------------------------------------------------------- lagged back edges
@pytest.mark.parametrize("n,twist,jitter,npol,naz", [(4, 0.6, 0.0, 8, 16), (8, 0.5, 0.0, 8, 16),
                                                      (5, 1.3, 0.15, 4, 16), (8, 0.25, 0.0, 8, 16)])
def test_lag_sets_match_the_oracle(n, twist, jitter, npol, naz):
    """tf_graph_lag picks the same lagged faces as the oracle (the same cycle walk), with the
    same inflow masks and levels; an acyclic grid gets none."""
    cfg = W.hex_problem(W.small_box(n=n, G=1, n_polar=npol, n_az=naz), twist=twist, jitter=jitter)
    geom = H.geometry(cfg["xyz"], cfg["hexes"])
    om, _ = product_quadrature(npol, naz)
    inflow, level, lag = H.graph(geom, om, lag=True)
    m = tf.HexMesh(cfg["xyz"], cfg["hexes"])
    q = tf.Quadrature(npol, naz)
    i2, l2, g2 = tf.tf_graph_lag(m.h, q.h, m.n_cells, q.n_dirs)
    assert np.array_equal(inflow, i2) and np.array_equal(level, l2) and np.array_equal(lag, g2)
    assert lag.any() == (twist > 0.3)


def test_lagged_task_graph_is_acyclic_with_the_non_lagged_in_degrees():
    """Tasks of a problem with lag_cycles on a grid with cycles: every (direction, cell) once,
    in-degrees = distinct upwind tasks across non-lagged faces, and an acyclic task graph."""
    cfg = W.hex_problem(W.small_box(n=6, G=4, n_polar=8, n_az=16), twist=0.5)
    geom = H.geometry(cfg["xyz"], cfg["hexes"])
    om, _ = product_quadrature(8, 16)
    inflow, _, lag = H.graph(geom, om, lag=True)
    assert lag.any()
    m = tf.HexMesh(cfg["xyz"], cfg["hexes"])
    q = tf.Quadrature(8, 16)
    with pytest.raises(tf.TfError) as e:
        tf.tf_graph_tasks(m.h, q.h, m.n_cells, q.n_dirs, 4)
    assert e.value.status == tf.TF_ERR_CYCLE
    task_of, position, indeg = tf.tf_graph_tasks(m.h, q.h, m.n_cells, q.n_dirs, 4, tf.options(lag_cycles=1))
    D, C = task_of.shape
    T = len(indeg)
    nbr = geom["nbr"]
    edges = set()
    for a in range(D):
        for c in range(C):
            for f in range(6):
                u = nbr[c, f]
                if (inflow[a, c] >> f & 1) and u >= 0 and not (lag[a, c] >> f & 1):
                    assert task_of[a, u] != task_of[a, c]  # t-level blocks hold independent cells
                    edges.add((int(task_of[a, u]), int(task_of[a, c])))
    assert sorted(np.unique(task_of)) == list(range(T))
    deg = np.zeros(T, np.int64)
    for _, t in edges:
        deg[t] += 1
    assert np.array_equal(deg, indeg)
    out = {}
    for s_, t in edges:
        out.setdefault(s_, []).append(t)
    ready = list(np.flatnonzero(deg == 0))
    seen = 0
    while ready:
        s_ = ready.pop()
        seen += 1
        for t in out.get(s_, []):
            deg[t] -= 1
            if deg[t] == 0:
                ready.append(t)
    assert seen == T


def test_lag_option_rejections():
    """lag_cycles takes 0 or 1, hexahedral meshes and t-level tasks (checked before any device work)."""
    cfg = W.hex_problem(W.small_box(n=2, G=1, n_polar=2, n_az=4), twist=0.25)
    m = tf.HexMesh(cfg["xyz"], cfg["hexes"])
    q = tf.Quadrature(2, 4)
    C = m.n_cells
    args = (m.h, q.h, 1, 1, np.zeros(C, np.int32), np.ones((1, 1)), np.zeros((1, 1, 1)), np.zeros((C, 1, 8)))
    for o in (tf.options(lag_cycles=2), tf.options(lag_cycles=1, task_shape=tf.TF_TASK_PATCHES)):
        with pytest.raises(tf.TfError) as e:
            tf.tf_problem_create(*args, opt=o)
        assert e.value.status == tf.TF_ERR_ARG
    tet = tf.Mesh(*W.jittered_kuhn_mesh(2, 1))
    with pytest.raises(tf.TfError) as e:
        tf.tf_problem_create(tet.h, q.h, 1, 1, np.zeros(tet.n_cells, np.int32), np.ones((1, 1)), np.zeros((1, 1, 1)),
                             np.zeros((tet.n_cells, 1, 4)), opt=tf.options(lag_cycles=1))
    assert e.value.status == tf.TF_ERR_ARG
