"""Pins of the second-order (ten-node) oracle to the mathematics.

* element integrals against exact monomial integration (rational arithmetic);
* a quadratic manufactured solution is reproduced exactly by one sweep in every
  direction, and source iteration converges to it (the space contains it);
* a single-direction sweep equals the dense solve of the global upwind-DG system
  assembled independently (exact tables, dict-based upwind coupling) -- this pins
  the inflow-face terms, which a continuous manufactured solution cannot see;
* per-cell particle balance with face averages in closed form;
* planted mistakes in copies of the oracle fail at least one of these.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import p2 as o2
from p2_checks import FOUR_PI, dense_direction_solve, face_nodes, mms_inputs, tables

HERE = os.path.dirname(os.path.abspath(__file__))


def _box(n=2, G=2, n_polar=2, n_az=8, seed=7):
    return W.order2(W.small_box(n=n, G=G, n_polar=n_polar, n_az=n_az, seed=seed))


def test_basis_integrals_closed_form():
    p = o2.basis_integrals()
    assert np.allclose(p, [-1 / 20] * 4 + [1 / 5] * 6, rtol=0, atol=1e-15)
    assert abs(p.sum() - 1.0) < 1e-15


def test_mass_matrix_exact():
    ref = tables()[1]
    got = o2.mass_matrix()
    assert np.max(np.abs(got - ref)) < 1e-15
    # vertex-vertex diagonal 1/70, vertex-vertex off-diagonal 1/420 (the textbook values)
    assert abs(ref[0, 0] - 1 / 70) < 1e-16 and abs(ref[0, 1] - 1 / 420) < 1e-16


def _mms(n=2, G=2, seed=3):
    cfg = _box(n=n, G=G)
    nodes = o2.node_coordinates(cfg["xyz"], cfg["tets"])
    Q, S1, psi_bc, psi = mms_inputs(cfg, nodes, np.random.default_rng(seed))
    cfg = dict(cfg)
    cfg["Q"] = Q
    return cfg, S1, psi_bc, psi


def test_quadratic_manufactured_solution_one_sweep_exact():
    cfg, S1, psi_bc, psi = _mms()
    P = o2.Problem2(cfg, S1=S1, psi_bc=psi_bc)
    q = P.source(FOUR_PI * psi)
    phi, psi_all, _ = P.sweep(q, keep_psi=True, threads=4)
    scale = np.abs(psi).max()
    for a in range(P.D):
        assert np.abs(psi_all[a] - psi).max() < 1e-11 * scale, a
    assert np.abs(phi - FOUR_PI * psi).max() < 1e-11 * FOUR_PI * scale


def test_quadratic_manufactured_solution_source_iteration():
    cfg, S1, psi_bc, psi = _mms(G=2)
    P = o2.Problem2(cfg, S1=S1, psi_bc=psi_bc)
    phi, it, r = P.source_iterate(1e-13, 400, threads=4)
    assert r < 1e-13
    assert np.abs(phi - FOUR_PI * psi).max() < 1e-10 * FOUR_PI * np.abs(psi).max()


@pytest.mark.parametrize("n,a", [(1, 0), (1, 5), (2, 3), (2, 12)])
def test_sweep_equals_dense_global_solve(n, a):
    cfg = _box(n=n, G=1)
    P = o2.Problem2(cfg)
    q = np.random.default_rng(n * 31 + a).uniform(0.2, 1.0, (P.C, 1, 10))
    psi = P.sweep_direction(a, q)[:, 0, :]
    ref = dense_direction_solve(P.geom, P.omega[a], P.sigma_t[P.material, 0], q[:, 0, :], P.inflow[a])
    assert np.abs(psi - ref).max() < 1e-12 * np.abs(ref).max()


def _face_average(vals, f):
    """Mean over the face opposite vertex f of the quadratic field with nodal values vals[10]:
    int_F phi_vertex = 0 and int_F phi_edge = A / 3, so it is the mean of the three edge nodes."""
    return np.mean([vals[i] for i in face_nodes(f)[3:]])


def test_per_cell_particle_balance():
    cfg = _box(n=2, G=2)
    P = o2.Problem2(cfg)
    rng = np.random.default_rng(4)
    q = rng.uniform(0.1, 1.0, (P.C, P.G, 10))
    keys = {}
    for c, t in enumerate(P.geom["tets"]):
        keys[c] = t
    pint = np.array([-1 / 20] * 4 + [1 / 5] * 6)
    for a in (0, 7):
        psi = P.sweep_direction(a, q)
        O = P.omega[a]
        worst = 0.0
        for c in range(P.C):
            V = P.geom["vol"][c]
            for g in range(P.G):
                sig = P.sigma_t[P.material[c], g]
                bal = sig * V * pint @ psi[c, g] - V * pint @ q[c, g]
                for f in range(4):
                    s = float(P.geom["normal"][c, f] @ O)
                    if (P.inflow[a, c] >> f) & 1:
                        n = P.geom["nbr"][c, f]
                        if n < 0:
                            continue  # vacuum: no inflow
                        # the neighbour's face across which c is downwind: the face whose vertex set matches
                        fv = set(int(v) for i, v in enumerate(P.geom["tets"][c]) if i != f)
                        (fn,) = [h for h in range(4)
                                 if set(int(v) for i, v in enumerate(P.geom["tets"][n]) if i != h) == fv]
                        bal -= abs(s) * _face_average(psi[n, g], fn)
                    else:
                        bal += s * _face_average(psi[c, g], f)
                worst = max(worst, abs(bal) / (V * np.abs(q[c, g]).max()))
        assert worst < 1e-12, (a, worst)


# ------------------------------------------------------------ planted mistakes
MUTANTS = {
    "drop_face_matrix": ("A[i][j] = Kc[i][j] + sig * Mc[i][j] + Fc[i][j];", "A[i][j] = Kc[i][j] + sig * Mc[i][j];"),
    "streaming_sign": ("Kc[i][j] += W * phi[i] * sj;", "Kc[i][j] -= W * phi[i] * sj;"),
    "streaming_transposed": ("Kc[i][j] += W * phi[i] * sj;", "Kc[j][i] += W * phi[i] * sj;"),
    "edge_basis_factor": ("phi[4 + e] = 4.0 * l[EDGE[e][0]] * l[EDGE[e][1]];",
                          "phi[4 + e] = 2.0 * l[EDGE[e][0]] * l[EDGE[e][1]];"),
    "vertex_basis": ("phi[v] = l[v] * (2.0 * l[v] - 1.0);", "phi[v] = l[v] * (2.0 * l[v] + 1.0);"),
    "face_signed": ("fw[f][k] = fabs(s) * we[k];", "fw[f][k] = s * we[k];"),
    "upwind_own_field": ("const double *pn = psi + ((size_t)n * G + g) * NB;",
                         "const double *pn = psi + ((size_t)c * G + g) * NB;"),
    "wrong_edge_list": ("{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}", "{0, 1}, {0, 2}, {0, 3}, {1, 2}, {2, 3}, {1, 3}"),
    "mass_dropped_sigma": ("+ sig * Mc[i][j] + Fc[i][j];", "+ Mc[i][j] + Fc[i][j];"),
    "quadrature_jacobian": ("(1.0 - u) * (1.0 - u) * (1.0 - v);", "(1.0 - u) * (1.0 - v);"),
}


def _pins_fail(src):
    """True if at least one pin fails (or the oracle errors) with the modified source."""
    try:
        cfg, S1, psi_bc, psi = _mms()
        P = o2.Problem2(cfg, S1=S1, psi_bc=psi_bc, src=src)
        q = P.source(FOUR_PI * psi)
        _, psi_all, _ = P.sweep(q, keep_psi=True)
        if np.abs(psi_all - psi[None]).max() > 1e-9 * np.abs(psi).max():
            return True
        cfg1 = _box(n=1, G=1)
        P1 = o2.Problem2(cfg1, src=src)
        q1 = np.random.default_rng(9).uniform(0.2, 1.0, (P1.C, 1, 10))
        for a in (0, 5):
            got = P1.sweep_direction(a, q1)[:, 0, :]
            ref = dense_direction_solve(P1.geom, P1.omega[a], P1.sigma_t[P1.material, 0], q1[:, 0, :], P1.inflow[a])
            if np.abs(got - ref).max() > 1e-9 * np.abs(ref).max():
                return True
        return False
    except oracle.OracleError:
        return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(o2.SRC).read()
    assert src.count(old) >= 1, name
    bad = tmp_path / f"tf_oracle_p2_{name}.c"
    bad.write_text(src.replace(old, new, 1))
    assert _pins_fail(str(bad)), name


def test_unmodified_oracle_passes_the_same_checks():
    assert not _pins_fail(o2.SRC)
