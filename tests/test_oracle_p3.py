"""Pins of the third-order (twenty-node) oracle to the mathematics, as for the
second-order one: exact monomial integrals, a cubic manufactured solution (in the
space, so reproduced exactly), dense global solves assembled independently, per-cell
particle balance with exact face averages, and planted mistakes."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import p3 as o3
from p2_checks import (FOUR_PI, _mul, basis_polys, cubic_field, dense_direction_solve, face_nodes,
                       integrate_face, mms_inputs, tables)


def _box(n=2, G=2, seed=7):
    return W.order3(W.small_box(n=n, G=G, n_polar=2, n_az=8, seed=seed))


def test_basis_integrals_exact():
    p = o3.basis_integrals()
    assert np.allclose(p, tables(3)[0], rtol=0, atol=1e-15)
    assert np.allclose(p[:4], 1 / 40) and np.allclose(p[4:16], 0, atol=1e-15) and np.allclose(p[16:], 9 / 40)


def test_mass_matrix_exact():
    assert np.max(np.abs(o3.mass_matrix() - tables(3)[1])) < 1e-15


def _mms(n=2, G=2, seed=3):
    cfg = _box(n=n, G=G)
    nodes = o3.node_coordinates(cfg["xyz"], cfg["tets"])
    Q, S1, psi_bc, psi = mms_inputs(cfg, nodes, np.random.default_rng(seed), field=cubic_field)
    cfg = dict(cfg)
    cfg["Q"] = Q
    return cfg, S1, psi_bc, psi


def test_cubic_manufactured_solution_one_sweep_exact():
    cfg, S1, psi_bc, psi = _mms()
    P = o3.Problem3(cfg, S1=S1, psi_bc=psi_bc)
    q = P.source(FOUR_PI * psi)
    phi, psi_all, _ = P.sweep(q, keep_psi=True, threads=4)
    scale = np.abs(psi).max()
    for a in range(P.D):
        assert np.abs(psi_all[a] - psi).max() < 1e-11 * scale, a


def test_cubic_manufactured_solution_source_iteration():
    cfg, S1, psi_bc, psi = _mms(G=2)
    P = o3.Problem3(cfg, S1=S1, psi_bc=psi_bc)
    phi, it, r = P.source_iterate(1e-13, 400, threads=4)
    assert r < 1e-13
    assert np.abs(phi - FOUR_PI * psi).max() < 1e-10 * FOUR_PI * np.abs(psi).max()


@pytest.mark.parametrize("n,a", [(1, 0), (1, 5), (2, 3)])
def test_sweep_equals_dense_global_solve(n, a):
    cfg = _box(n=n, G=1)
    P = o3.Problem3(cfg)
    q = np.random.default_rng(n * 31 + a).uniform(0.2, 1.0, (P.C, 1, 20))
    psi = P.sweep_direction(a, q)[:, 0, :]
    ref = dense_direction_solve(P.geom, P.omega[a], P.sigma_t[P.material, 0], q[:, 0, :], P.inflow[a], order=3)
    assert np.abs(psi - ref).max() < 1e-12 * np.abs(ref).max()


def test_per_cell_particle_balance():
    """Outflow s_f <psi>_f - inflow |s_f| <psi_up>_f + sigma_t int psi - int q = 0 per cell,
    with the face averages from exact face integrals of the basis."""
    cfg = _box(n=2, G=2)
    P = o3.Problem3(cfg)
    B = basis_polys(3)
    one = {(0, 0, 0, 0): 1}
    fav = np.array([[float(integrate_face(_mul(b, one), f)) for b in B] for f in range(4)])  # [f][i]
    pint = tables(3)[0]
    q = np.random.default_rng(4).uniform(0.1, 1.0, (P.C, P.G, 20))
    for a in (0, 7):
        psi = P.sweep_direction(a, q)
        O = P.omega[a]
        worst = 0.0
        for c in range(P.C):
            V = P.geom["vol"][c]
            for g in range(P.G):
                bal = P.sigma_t[P.material[c], g] * V * pint @ psi[c, g] - V * pint @ q[c, g]
                for f in range(4):
                    s = float(P.geom["normal"][c, f] @ O)
                    if (P.inflow[a, c] >> f) & 1:
                        n = P.geom["nbr"][c, f]
                        if n < 0:
                            continue
                        fv = set(int(v) for i, v in enumerate(P.geom["tets"][c]) if i != f)
                        (fn,) = [h for h in range(4)
                                 if set(int(v) for i, v in enumerate(P.geom["tets"][n]) if i != h) == fv]
                        bal -= abs(s) * fav[fn] @ psi[n, g]
                    else:
                        bal += s * fav[f] @ psi[c, g]
                worst = max(worst, abs(bal) / (V * np.abs(q[c, g]).max()))
        assert worst < 1e-12, (a, worst)


def test_face_nodes_have_zero_lambda():
    """The face node lists used above: ten nodes per face, vertex f excluded, its centre included."""
    for f in range(4):
        fn = face_nodes(f, 3)
        assert len(fn) == 10 and f not in fn and 16 + f in fn


MUTANTS = {
    "drop_face_matrix": ("A[i][j] = Kc[i][j] + sig * Mc[i][j] + Fc[i][j];", "A[i][j] = Kc[i][j] + sig * Mc[i][j];"),
    "streaming_sign": ("Kc[i][j] += W * phi[i] * sj;", "Kc[i][j] -= W * phi[i] * sj;"),
    "lattice_step": ("const double t = (3.0 * x - m) / (m + 1.0), dt = 3.0 / (m + 1.0);",
                     "const double t = (3.0 * x - m) / (m + 2.0), dt = 3.0 / (m + 2.0);"),
    "edge_node_swap": ("al[EDGE[e][0]] = second ? 1 : 2;", "al[EDGE[e][0]] = second ? 2 : 1;"),
    "derivative_rule": ("d = d * t + p * dt;", "d = d * t + dt;"),
    "face_signed": ("fw[f][k] = fabs(s) * we[k];", "fw[f][k] = s * we[k];"),
    "quadrature_jacobian": ("(1.0 - u) * (1.0 - u) * (1.0 - v);", "(1.0 - u) * (1.0 - v);"),
}


def _pins_fail(src):
    try:
        cfg, S1, psi_bc, psi = _mms()
        P = o3.Problem3(cfg, S1=S1, psi_bc=psi_bc, src=src)
        _, psi_all, _ = P.sweep(P.source(FOUR_PI * psi), keep_psi=True)
        if np.abs(psi_all - psi[None]).max() > 1e-9 * np.abs(psi).max():
            return True
        P1 = o3.Problem3(_box(n=1, G=1), src=src)
        q1 = np.random.default_rng(9).uniform(0.2, 1.0, (P1.C, 1, 20))
        for a in (0, 5):
            got = P1.sweep_direction(a, q1)[:, 0, :]
            ref = dense_direction_solve(P1.geom, P1.omega[a], P1.sigma_t[P1.material, 0], q1[:, 0, :], P1.inflow[a],
                                        order=3)
            if np.abs(got - ref).max() > 1e-9 * np.abs(ref).max():
                return True
        return False
    except oracle.OracleError:
        return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(o3.SRC).read()
    assert src.count(old) >= 1, name
    bad = tmp_path / f"tf_oracle_p3_{name}.c"
    bad.write_text(src.replace(old, new, 1))
    assert _pins_fail(str(bad)), name


def test_unmodified_oracle_passes_the_same_checks():
    assert not _pins_fail(o3.SRC)
