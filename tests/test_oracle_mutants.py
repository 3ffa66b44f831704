"""Planted mistakes: each one, written into a copy of the oracle's C source on
the CPU, must make at least one pin fail.  This shows the pins are sensitive
to the plausible errors (a dropped term, a wrong sign or index, a transposed
operand), not only that the oracle passes them."""
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle_checks import FOUR_PI, cell_balance, global_direction_system, mms_problem

MUTANTS = {
    "face_matrix_dropped": ("A[i][j] += mf;", "A[i][j] += 0.0 * mf;"),
    "face_rhs_dropped": ("b[i] += mf * up[j];", "b[i] += 0.0 * mf * up[j];"),
    "streaming_sign": ("stream[j] = (V / 4.0) *", "stream[j] = -(V / 4.0) *"),
    "mass_diagonal": ("(i == j ? 2.0 : 1.0) * qc[j]", "(i == j ? 1.0 : 1.0) * qc[j]"),
    "upwind_node_index": ("up[i] = psi[((size_t)n * G + g) * 4 + k];",
                          "up[i] = psi[((size_t)n * G + g) * 4 + (k + 1) % 4];"),
    "gradient_transposed": ("O[0] * gr[3 * j] + O[1] * gr[3 * j + 1]", "O[0] * gr[3 * j + 1] + O[1] * gr[3 * j]"),
    "normal_inward": ("if (side > 0.0)", "if (side < 0.0)"),
    "weight_half": ("w[a] = wm[i] * (2.0 * M_PI / n_az);", "w[a] = wm[i] * (M_PI / n_az);"),
    "level_not_incremented": ("if (lev[n] < lev[c] + 1) lev[n] = lev[c] + 1;", "if (lev[n] < lev[c]) lev[n] = lev[c];"),
    "classification_reversed": ("if (s < -eps) m", "if (s > eps) m"),
    "sigma_mass_scale": ("sig * (V / 20.0)", "sig * (V / 24.0)"),
    "s1_dropped": ("b[i] += (V / 4.0) * os;", "b[i] += 0.0 * os;"),
}


def _battery(lib):
    """Run a fast subset of the pins with a given oracle build; return the names that fail."""
    failed = []
    om, w = oracle.product_quadrature(4, 8, lib)
    if abs(w.sum() - FOUR_PI) > 1e-12 or np.max(np.abs(w @ om)) > 1e-12:
        failed.append("quadrature")
    rng = np.random.default_rng(0)
    # dense global solve on 2^3 hexes with inflow
    xyz, tets = W.jittered_kuhn_mesh(2, 99)
    C = len(tets)
    G = 1
    cfg = dict(xyz=xyz, tets=tets, n_groups=G, cell_material=np.zeros(C, np.int32),
               sigma_t=np.array([[1.3]]), sigma_s=np.zeros((1, 1, 1)), Q=np.zeros((C, 1, 4)),
               n_polar=2, n_azimuthal=8)
    psi_in = rng.uniform(0, 1, (len(xyz), G))
    try:
        om2, w2 = oracle.product_quadrature(2, 8)  # reference quadrature from the unmodified build
        P = oracle.Problem(cfg, omega=om2, w=w2, psi_in=psi_in, lib=lib)
        q = rng.uniform(0, 1, (C, G, 4))
        for a in (0, 5, 11):
            psi = P.sweep_direction(a, q)
            ref, _ = global_direction_system(xyz, tets, om2[a], np.full(C, 1.3), q[:, 0], None, psi_in[:, 0])
            if np.max(np.abs(psi[:, 0] - ref)) > 1e-10 * np.max(np.abs(ref)):
                failed.append("dense_lu")
                break
    except oracle.OracleError:
        failed.append("dense_lu(error)")
    # manufactured solution
    try:
        rng2 = np.random.default_rng(4)
        xyz, tets = W.jittered_kuhn_mesh(2, 1234)
        C = len(tets)
        base = dict(xyz=xyz, tets=tets, n_groups=2, cell_material=np.zeros(C, np.int32),
                    sigma_t=rng2.uniform(0.5, 2, (1, 2)), sigma_s=rng2.uniform(0, 0.2, (1, 2, 2)),
                    Q=np.zeros((C, 2, 4)), n_polar=2, n_azimuthal=8)
        mcfg, S1, psi_v, exact = mms_problem(base)
        om2, w2 = oracle.product_quadrature(2, 8)
        P = oracle.Problem(mcfg, omega=om2, w=w2, S1=S1, psi_in=psi_v, lib=lib)
        phi, psi, _ = P.sweep(P.source(FOUR_PI * exact), keep_psi=True)
        if np.max(np.abs(psi - exact[None])) > 1e-10 * np.max(np.abs(exact)):
            failed.append("mms")
        # balance on one direction
        if cell_balance(P, psi[0], P.source(FOUR_PI * exact), 0, S1=S1, psi_in=psi_v) > 1e-10:
            failed.append("balance")
    except oracle.OracleError:
        failed.append("mms(error)")
    return failed


def test_unmodified_oracle_passes_battery():
    assert _battery(oracle.load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    with open(oracle.SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = os.path.join(tmp_path, f"mut_{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = oracle.load(src=path)
    assert _battery(lib) != [], f"planted mistake {name} passed every pin"


def test_transposed_scattering_matrix_is_caught(monkeypatch):
    """The source update with sigma_s[g->g'] read as [to][from] fails the MMS pin."""
    rng = np.random.default_rng(4)
    xyz, tets = W.jittered_kuhn_mesh(2, 1234)
    C = len(tets)
    base = dict(xyz=xyz, tets=tets, n_groups=3, cell_material=np.zeros(C, np.int32),
                sigma_t=rng.uniform(0.5, 2, (1, 3)), sigma_s=rng.uniform(0, 0.2, (1, 3, 3)),
                Q=np.zeros((C, 3, 4)), n_polar=2, n_azimuthal=8)
    mcfg, S1, psi_v, exact = mms_problem(base)
    P = oracle.Problem(mcfg, S1=S1, psi_in=psi_v)
    good = P.sweep(P.source(FOUR_PI * exact))[0]
    assert np.max(np.abs(good - FOUR_PI * exact)) < 1e-12 * np.max(FOUR_PI * exact)
    P.sigma_s = np.ascontiguousarray(np.transpose(P.sigma_s, (0, 2, 1)))
    bad = P.sweep(P.source(FOUR_PI * exact))[0]
    assert np.max(np.abs(bad - FOUR_PI * exact)) > 1e-6 * np.max(FOUR_PI * exact)
