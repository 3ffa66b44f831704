"""Host-side tests of the native library (no GPU): it loads, exports every
symbol the C header declares, and its host precompute (geometry, quadrature,
face classification, t-levels) is bit-identical to the oracle's."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2510_11513_gb300 as tf
import workloads as W
from paper_2510_11513_gb300 import build as tfbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def test_empty_inputs_rejected():
    xyz, tets = W.jittered_kuhn_mesh(1, 5)
    with pytest.raises(tf.TfError) as e:
        tf.Mesh(xyz, np.zeros((0, 4), dtype=np.int32))
    assert e.value.status == tf.TF_ERR_ARG
    with pytest.raises(tf.TfError) as e:
        tf.Quadrature(omega=np.zeros((0, 3)), w=np.zeros(0))
    assert e.value.status == tf.TF_ERR_ARG
    with pytest.raises(tf.TfError) as e:
        tf.Mesh(xyz[:3], tets[:1])  # fewer than four vertices
    assert e.value.status == tf.TF_ERR_ARG


def test_status_strings():
    lib = tf.load()
    for s in range(9):
        assert lib.tf_status_string(s)


def test_second_order_element_tables_exact(tmp_path):
    """The exact rationals the second-order kernels use (csrc/p2_tables.h, compiled
    here as host C++) against exact monomial integration of the basis polynomials."""
    import subprocess

    from fractions import Fraction

    from p2_checks import _mul, basis_polys, face_nodes, integrate_cell, tables

    src = tmp_path / "t.cpp"
    src.write_text(
        '#include <cstdio>\n#include "p2_tables.h"\nint main() {\n'
        '  for (int i = 0; i < 10; ++i) std::printf("%.17g\\n", p2_p(i));\n'
        '  for (int i = 0; i < 10; ++i) for (int m = 0; m < 4; ++m) std::printf("%.17g\\n", p2_P(i, m));\n'
        '  for (int i = 0; i < 10; ++i) for (int j = 0; j < 10; ++j) std::printf("%.17g\\n", p2_M(i, j));\n'
        '  for (int b = 0; b < 6; ++b) for (int c = 0; c < 6; ++c) std::printf("%.17g\\n", p2_F(b, c));\n'
        '  for (int f = 0; f < 4; ++f) for (int b = 0; b < 6; ++b) std::printf("%d\\n", p2_face_node(f, b));\n'
        '  return 0; }\n')
    exe = tmp_path / "t"
    inc = os.path.join(ROOT, "paper_2510_11513_gb300", "csrc")
    subprocess.check_call(["g++", "-std=c++17", f"-I{inc}", str(src), "-o", str(exe)])
    vals = [float(x) for x in subprocess.check_output([str(exe)]).split()]
    p, M, Dk, F = tables()
    got_p, got_P = np.array(vals[:10]), np.array(vals[10:50]).reshape(10, 4)
    got_M, got_F = np.array(vals[50:150]).reshape(10, 10), np.array(vals[150:186]).reshape(6, 6)
    got_fn = np.array(vals[186:210], dtype=int).reshape(4, 6)
    assert np.allclose(got_p, p, rtol=0, atol=1e-16)
    assert np.allclose(got_M, M, rtol=0, atol=1e-16)
    B = basis_polys()
    lam = [{tuple(int(j == k) for j in range(4)): Fraction(1)} for k in range(4)]
    P = np.array([[float(integrate_cell(_mul(B[i], lam[m]))) for m in range(4)] for i in range(10)])
    assert np.allclose(got_P, P, rtol=0, atol=1e-16)
    # the streaming matrix the kernel forms from P and p equals int phi_i d phi_j / d lambda_k exactly
    E = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
    for k in range(4):
        for i in range(10):
            for j in range(10):
                if j < 4:
                    v = (4 * got_P[i, j] - got_p[i]) if j == k else 0.0
                else:
                    a, b = E[j - 4]
                    v = 4 * got_P[i, b] if k == a else (4 * got_P[i, a] if k == b else 0.0)
                assert abs(v - Dk[k][i][j]) < 1e-15, (k, i, j)
    for f in range(4):
        assert list(got_fn[f]) == face_nodes(f)
        sub = F[f][np.ix_(face_nodes(f), face_nodes(f))]
        assert np.allclose(got_F, sub, rtol=0, atol=1e-16)


def test_python_structs_match_the_c_header(tmp_path):
    """The ctypes mirrors of tf_options, tf_iter_info and tf_stats have the size and the
    field offsets the C compiler gives the header's structs (the C ABI the binding uses)."""
    import ctypes
    import subprocess

    from paper_2510_11513_gb300 import tfsweep as T

    structs = [("tf_options", T.tf_options), ("tf_iter_info", T.tf_iter_info), ("tf_stats", T.tf_stats)]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "tfsweep.h"', "int main(void) {"]
    for cname, py in structs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.check_call(["gcc", "-std=c11", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)]).decode().splitlines():
        a, b, c = line.split()
        got[(a, b)] = int(c)
    for cname, py in structs:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_third_order_element_tables_exact(tmp_path):
    """The host-built tables of the third-order kernels (csrc/p3_tables.cpp) against exact
    monomial integration in rational arithmetic: integrals, mass, streaming and face tables."""
    import subprocess

    from p2_checks import face_nodes, tables

    src = tmp_path / "t.cpp"
    src.write_text(
        '#include <cstdio>\n#include "tf_internal.h"\nint main() {\n'
        '  tf::P3Tables t; tf::p3_element_tables(t);\n'
        '  for (int i = 0; i < 20; ++i) std::printf("%.17g\\n", t.p[i]);\n'
        '  for (int i = 0; i < 400; ++i) std::printf("%.17g\\n", t.M[i]);\n'
        '  for (int k = 0; k < 4; ++k) for (int i = 0; i < 400; ++i) std::printf("%.17g\\n", t.C[k][i]);\n'
        '  for (int f = 0; f < 4; ++f) for (int r = 0; r < 10; ++r) std::printf("%d\\n", t.fn[f][r]);\n'
        '  for (int f = 0; f < 4; ++f) for (int r = 0; r < 100; ++r) std::printf("%.17g\\n", t.F[f][r]);\n'
        '  return 0; }\n')
    exe = tmp_path / "t"
    csrc = os.path.join(ROOT, "paper_2510_11513_gb300", "csrc")
    subprocess.check_call(["g++", "-std=c++17", f"-I{csrc}", f"-I{os.path.join(ROOT, 'include')}", "-I/usr/local/cuda/include",
                           str(src), os.path.join(csrc, "p3_tables.cpp"), "-o", str(exe)])
    v = np.array([float(x) for x in subprocess.check_output([str(exe)]).split()])
    p, M, Dk, F = tables(3)
    assert np.allclose(v[:20], p, rtol=0, atol=1e-15)
    assert np.allclose(v[20:420].reshape(20, 20), M, rtol=0, atol=1e-15)
    assert np.allclose(v[420:2020].reshape(4, 20, 20), Dk, rtol=0, atol=1e-14)
    fn = v[2020:2060].astype(int).reshape(4, 10)
    Fg = v[2060:2460].reshape(4, 10, 10)
    for f in range(4):
        assert list(fn[f]) == face_nodes(f, 3)
        assert np.allclose(Fg[f], F[f][np.ix_(face_nodes(f, 3), face_nodes(f, 3))], rtol=0, atol=1e-15)
