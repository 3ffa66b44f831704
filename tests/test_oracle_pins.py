"""Pins of the CPU oracle against the mathematics (no GPU).

Each test compares the oracle with something other than itself: a library
routine (numpy's Gauss-Legendre, determinant, inverse, dense LU), a closed
form (quadrature moments, a manufactured linear solution), a conservation
identity, or brute force on tiny meshes.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle_checks import (FOUR_PI, cell_balance, face_geometry, global_direction_system, match_faces,
                           mms_problem, tet_volume)


# ------------------------------------------------------------------ quadrature
@pytest.mark.parametrize("n", [1, 2, 3, 4, 8, 12, 16])
def test_gauss_legendre_matches_numpy(n):
    x, w = oracle.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) < 4e-16
    assert np.max(np.abs(w - wr)) < 4e-15


@pytest.mark.parametrize("npol,naz", [(2, 4), (4, 8), (8, 16), (12, 16), (8, 8)])
def test_product_quadrature_moments(npol, naz):
    om, w = oracle.product_quadrature(npol, naz)
    assert np.allclose(np.linalg.norm(om, axis=1), 1.0, rtol=0, atol=1e-15)
    assert abs(w.sum() - FOUR_PI) < 1e-13
    assert np.max(np.abs(w @ om)) < 1e-14
    second = np.einsum("a,ai,aj->ij", w, om, om)
    assert np.max(np.abs(second - FOUR_PI / 3.0 * np.eye(3))) < 1e-13
    # half-offset azimuths: no component is zero; with n_az/4 even also |Ox| != |Oy|
    assert np.min(np.abs(om[:, :2])) > 1e-3
    if (naz // 4) % 2 == 0:
        assert np.min(np.abs(np.abs(om[:, 0]) - np.abs(om[:, 1]))) > 1e-6


# ------------------------------------------------------------------- geometry
@pytest.mark.parametrize("n", [1, 2, 5])
def test_geometry_identities(n):
    xyz, tets = W.jittered_kuhn_mesh(n, W.BASE_SEED + n)
    g = oracle.geometry(xyz, tets)
    C = len(tets)
    ref_vol = np.array([tet_volume(xyz[t]) for t in tets])
    assert np.max(np.abs(g["vol"] - ref_vol)) < 1e-15 * 6 / n ** 3 * 10
    assert abs(g["vol"].sum() - 1.0) < 1e-13
    assert np.max(np.abs(g["normal"].sum(axis=1))) < 1e-15
    assert np.max(np.abs(g["grad"].sum(axis=1))) < 1e-10
    # basis gradients: b_j(x_k) = delta_jk
    for c in range(C):
        x = xyz[tets[c]]
        vals = g["grad"][c] @ (x - x[0]).T  # [j][k] = grad b_j . (x_k - x_0)
        expect = np.eye(4) - np.eye(4)[:, [0]]
        assert np.max(np.abs(vals - expect)) < 1e-12
        for f in range(4):
            nodes, area, nrm = face_geometry(x, f)
            assert np.max(np.abs(g["normal"][c, f] - area * nrm)) < 1e-15
    # neighbours and upwind-node map against a dict-based matcher
    nbr = match_faces(tets)
    assert np.array_equal(g["nbr"], nbr)
    assert (g["nbr"] < 0).sum() == 12 * n * n
    for c in range(C):
        for f in range(4):
            nb = g["nbr"][c, f]
            if nb < 0:
                continue
            # exactly opposite normals on the shared face
            fb = int(np.nonzero(g["nbr"][nb] == c)[0][0])
            assert np.array_equal(g["normal"][c, f], -g["normal"][nb, fb])
            for i in range(4):
                k = g["nbr_node"][c, f, i]
                if i == f:
                    assert k == -1
                else:
                    assert tets[nb][k] == tets[c][i]


def test_inverted_and_nonconforming_meshes_rejected():
    xyz, tets = W.jittered_kuhn_mesh(2, 5)
    bad = tets.copy()
    bad[3, [2, 3]] = bad[3, [3, 2]]
    with pytest.raises(oracle.OracleError) as e:
        oracle.geometry(xyz, bad)
    assert e.value.code == oracle.ORA_ERR_MESH
    dup = np.concatenate([tets, tets[:1]])
    with pytest.raises(oracle.OracleError) as e:
        oracle.geometry(xyz, dup)
    assert e.value.code == oracle.ORA_ERR_MESH


# ---------------------------------------------------------------------- graph
@pytest.mark.parametrize("n", [2, 4])
def test_levels_brute_force(n):
    xyz, tets = W.jittered_kuhn_mesh(n, 11)
    g = oracle.geometry(xyz, tets)
    om, w = oracle.product_quadrature(4, 8)
    inflow, level = oracle.graph(g, om)
    C = len(tets)
    for a in range(len(om)):
        # brute force: classification by sign, then levels by repeated relaxation
        s = np.einsum("d,cfd->cf", om[a], g["normal"])
        eps = 1e-12 * np.linalg.norm(g["normal"], axis=2)
        mask = (s < -eps)
        assert np.array_equal(mask, (inflow[a][:, None] >> np.arange(4)) & 1 == 1)
        lev = np.zeros(C, dtype=np.int64)
        for _ in range(C + 1):
            new = lev.copy()
            for c in range(C):
                ups = [g["nbr"][c, f] for f in range(4) if mask[c, f] and g["nbr"][c, f] >= 0]
                new[c] = 0 if not ups else 1 + max(lev[u] for u in ups)
            if np.array_equal(new, lev):
                break
            lev = new
        assert np.array_equal(lev, level[a])
        # the two sides of an interior face never both call it inflow
        for c in range(C):
            for f in range(4):
                nb = g["nbr"][c, f]
                if nb >= 0 and mask[c, f]:
                    fb = int(np.nonzero(g["nbr"][nb] == c)[0][0])
                    assert not mask[nb, fb]


def test_cycle_detected():
    # three cells in a ring: each has one interior inflow face from the previous cell
    Om = np.array([[0.0, 0.0, 1.0]])
    nbr = -np.ones((3, 4), dtype=np.int32)
    normal = np.zeros((3, 4, 3))
    for c in range(3):
        nbr[c, 0] = (c + 2) % 3
        normal[c, 0] = [0.0, 0.0, -1.0]  # inflow
        nbr[c, 1] = (c + 1) % 3
        normal[c, 1] = [0.0, 0.0, 1.0]  # outflow
        normal[c, 2] = [1.0, 0.0, 0.0]
        normal[c, 3] = [-1.0, 0.0, 0.0]
    geom = dict(vol=np.ones(3), nbr=nbr, normal=normal)
    with pytest.raises(oracle.OracleError) as e:
        oracle.graph(geom, Om)
    assert e.value.code == oracle.ORA_ERR_CYCLE


# ------------------------------------------------------------- local / global
def test_single_cell_against_dense_solve():
    """One tetrahedron: all four faces are boundary faces; random inflow values."""
    rng = np.random.default_rng(3)
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.1], [0.1, 0.2, 1.1]])
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    om, w = oracle.product_quadrature(2, 8)
    G = 3
    cfg = dict(xyz=xyz, tets=tets, n_groups=G, cell_material=np.zeros(1, np.int32),
               sigma_t=rng.uniform(0.2, 3.0, (1, G)), sigma_s=np.zeros((1, G, G)), Q=np.zeros((1, G, 4)),
               n_polar=2, n_azimuthal=8)
    S1 = rng.uniform(-1, 1, (1, G, 3))
    psi_in = rng.uniform(0, 2, (4, G))
    P = oracle.Problem(cfg, omega=om, w=w, S1=S1, psi_in=psi_in)
    q = rng.uniform(0, 1, (1, G, 4))
    for a in range(len(om)):
        psi = P.sweep_direction(a, q)
        for g in range(G):
            ref, smin = global_direction_system(xyz, tets, om[a], cfg["sigma_t"][0, [g]], q[:, g],
                                                S1[:, g], psi_in[:, g])
            assert smin > 1e-8
            assert np.max(np.abs(psi[:, g] - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("n,inflow", [(1, False), (2, False), (2, True)])
def test_sweep_equals_dense_global_solve(n, inflow):
    """The sweep in t-level order solves the global block-triangular system."""
    rng = np.random.default_rng(n)
    xyz, tets = W.jittered_kuhn_mesh(n, 99)
    C = len(tets)
    G = 2
    cfg = dict(xyz=xyz, tets=tets, n_groups=G, cell_material=rng.integers(0, 2, C).astype(np.int32),
               sigma_t=rng.uniform(0.3, 4.0, (2, G)), sigma_s=np.zeros((2, G, G)), Q=np.zeros((C, G, 4)),
               n_polar=2, n_azimuthal=8)
    psi_in = rng.uniform(0, 1, (len(xyz), G)) if inflow else None
    om, w = oracle.product_quadrature(2, 8)
    P = oracle.Problem(cfg, omega=om, w=w, psi_in=psi_in)
    q = rng.uniform(0, 1, (C, G, 4))
    for a in range(len(om)):
        psi = P.sweep_direction(a, q)
        for g in range(G):
            st = cfg["sigma_t"][cfg["cell_material"], g]
            ref, smin = global_direction_system(xyz, tets, om[a], st, q[:, g], None,
                                                None if psi_in is None else psi_in[:, g])
            assert smin > 1e-8
            assert np.max(np.abs(psi[:, g] - ref)) < 1e-12 * np.max(np.abs(ref))


# ------------------------------------------------------------------------ MMS
def _mms_cfg(n=3, G=3, seed=17):
    rng = np.random.default_rng(seed)
    xyz, tets = W.jittered_kuhn_mesh(n, 1234)
    C = len(tets)
    M = 2
    sig_t = rng.uniform(0.5, 2.0, (M, G))
    S = rng.uniform(0.0, 0.15, (M, G, G))  # non-symmetric, up- and down-scatter
    return dict(xyz=xyz, tets=tets, n_groups=G, cell_material=rng.integers(0, M, C).astype(np.int32),
                sigma_t=sig_t, sigma_s=S, Q=np.zeros((C, G, 4)), n_polar=4, n_azimuthal=8)


def test_mms_single_sweep_exact():
    cfg, S1, psi_v, exact = mms_problem(_mms_cfg())
    P = oracle.Problem(cfg, S1=S1, psi_in=psi_v)
    phi_exact = FOUR_PI * exact
    q = P.source(phi_exact)
    phi, psi, _ = P.sweep(q, keep_psi=True)
    assert np.max(np.abs(psi - exact[None])) < 1e-13 * np.max(np.abs(exact))
    assert np.max(np.abs(phi - phi_exact)) < 1e-13 * np.max(np.abs(phi_exact))


def test_mms_source_iteration_converges_to_exact():
    cfg, S1, psi_v, exact = mms_problem(_mms_cfg(n=2, G=2, seed=5))
    P = oracle.Problem(cfg, S1=S1, psi_in=psi_v)
    phi, it, r = P.source_iterate(1e-13, 400)
    assert r < 1e-13
    assert np.max(np.abs(phi - FOUR_PI * exact)) < 1e-11 * np.max(np.abs(FOUR_PI * exact))
    # Eq. (3) integrated flux of phi = 4 pi (alpha + beta . x) equals 4 pi (alpha + beta . centre)
    ig, tot, _, _ = P.integrated_flux(phi)
    rng_alpha = exact  # nodal values; integral of a linear field = volume-weighted nodal mean
    ref = FOUR_PI * np.einsum("c,cgi->g", P.geom["vol"] / 4.0, rng_alpha)
    assert np.max(np.abs(ig - ref)) < 1e-11 * np.max(np.abs(ref))


# -------------------------------------------------------------------- balance
def test_cell_balance_each_direction():
    cfg = W.small_box(n=3, G=3, n_polar=2, n_az=8)
    rng = np.random.default_rng(9)
    psi_in = rng.uniform(0, 1, (len(cfg["xyz"]), 3))
    S1 = rng.uniform(-0.3, 0.3, (len(cfg["tets"]), 3, 3))
    P = oracle.Problem(cfg, S1=S1, psi_in=psi_in)
    phi0 = rng.uniform(0, 1, (P.C, P.G, 4))
    q = P.source(phi0)
    for a in range(P.D):
        psi = P.sweep_direction(a, q)
        assert cell_balance(P, psi, q, a, S1=S1, psi_in=psi_in) < 1e-12


def test_global_balance_after_iteration():
    """Summed over cells and directions: leakage + absorption = source (to roundoff)."""
    cfg = W.small_box(n=4, G=2, n_polar=2, n_az=8)
    P = oracle.Problem(cfg)
    rng = np.random.default_rng(1)
    phi_old = rng.uniform(0, 1, (P.C, P.G, 4))
    q = P.source(phi_old)
    phi, psi, _ = P.sweep(q, keep_psi=True)
    # boundary leakage per group from psi, absorption from phi, source from q
    xyz, tets = cfg["xyz"], cfg["tets"]
    nbr = P.geom["nbr"]
    leak = np.zeros(P.G)
    for a in range(P.D):
        for c in range(P.C):
            for f in range(4):
                if nbr[c, f] >= 0:
                    continue
                nodes, area, nrm = face_geometry(xyz[tets[c]], f)
                s = np.dot(P.omega[a], nrm) * area
                if s > 0:
                    leak += P.w[a] * s * psi[a, c][:, nodes].mean(axis=1)
    st = P.sigma_t[P.material]
    vol = P.geom["vol"]
    absorb = np.einsum("c,cg,cgi->g", vol / 4.0, st, phi)
    source = FOUR_PI * np.einsum("c,cgi->g", vol / 4.0, q)
    assert np.max(np.abs(leak + absorb - source) / source) < 1e-12


def test_thick_medium_interior_matches_infinite_medium():
    """Deep inside an optically thick box with a uniform source, phi -> Q / sigma_a."""
    n, G = 4, 1
    xyz, tets = W.jittered_kuhn_mesh(n, 3)
    C = len(tets)
    xyz = xyz * 8.0  # 8 units wide, sigma_t = 5 => 40 mean free paths
    cfg = dict(xyz=xyz, tets=tets, n_groups=G, cell_material=np.zeros(C, np.int32),
               sigma_t=np.array([[5.0]]), sigma_s=np.array([[[2.5]]]), Q=np.ones((C, G, 4)),
               n_polar=4, n_azimuthal=8)
    P = oracle.Problem(cfg)
    phi, it, r = P.source_iterate(1e-12, 200)
    centre = np.linalg.norm(xyz[tets].mean(axis=1) - 4.0, axis=1) < 1.5
    assert np.max(np.abs(phi[centre] - 1.0 / 2.5)) < 2e-3


def test_residual_definition_special_cases():
    a = np.zeros((2, 2, 4))
    assert oracle.Problem.residual(a, a) == 0.0
    b = a.copy()
    b[0, 0, 0] = 2.0
    c = b.copy()
    c[0, 0, 0] = 1.0
    assert oracle.Problem.residual(b, c) == pytest.approx(0.5)
    # pointwise with a floor: a tiny value next to a large one in the same group
    b[1, 0, 1] = 1e-30
    c[1, 0, 1] = 0.0
    c[0, 0, 0] = 2.0
    assert oracle.Problem.residual(b, c, floor=1e-10) == pytest.approx(1e-30 / (1e-10 * 2.0))
    # default (max-norm per group): the same change measured against the group's max
    assert oracle.Problem.residual(b, c) == pytest.approx(1e-30 / 2.0)
    # groups are normalised separately
    d, e = np.zeros((1, 2, 4)), np.zeros((1, 2, 4))
    d[0, 0, 0], d[0, 1, 0] = 1.0, 1e-20
    e[0, 0, 0], e[0, 1, 0] = 1.0, 0.5e-20
    assert oracle.Problem.residual(d, e) == pytest.approx(0.5)
