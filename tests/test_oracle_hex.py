"""Pins of the trilinear-hexahedron oracle (`oracle/q1hex.py`, `oracle/tf_oracle_hex.c`)
against what the mathematics fixes: exact rational element integrals, closed forms on
boxes, the divergence theorem, closed surfaces, whole-mesh dense solves without a
sweep order, manufactured linear fields (which upwind DG reproduces exactly),
particle balance and mirror symmetry."""
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from hex_checks import (CORNERS, cube_tables, dense_direction_solve, exact_tables, face_vertices,
                        match_faces, numeric_tables)
from oracle import FOUR_PI, OracleError, product_quadrature
from oracle import q1hex as H


def _single(X):
    return H.geometry(np.asarray(X, dtype=np.float64), np.arange(8, dtype=np.int32)[None])


def _distorted_hex(seed):
    rng = np.random.default_rng(seed)
    return [[Fraction(a) + Fraction(int(rng.integers(-4, 5)), 24) for a in c] for c in CORNERS]


def test_face_node_order():
    for f in range(6):
        assert H.face_nodes(f) == face_vertices(f)


def test_tables_exact_on_a_distorted_hex():
    """Every integral of a hexahedron with rational corners (non-planar faces) against
    exact rational integration of the symbolic map."""
    pytest.importorskip("sympy")
    X = _distorted_hex(3)
    E = exact_tables(X)
    g = _single([[float(x) for x in r] for r in X])
    f = lambda a: np.array(a, dtype=object).astype(np.float64)  # noqa: E731
    assert abs(float(E["vol"]) - g["vol"][0]) < 1e-15
    assert np.max(np.abs(f(E["M"]) - g["mass"][0])) < 1e-16
    assert np.max(np.abs(f(E["G"]) - g["grad"][0])) < 1e-15
    assert np.max(np.abs(f(E["F"]) - g["face"][0])) < 1e-15
    assert np.max(np.abs(f(E["Nbar"]) - g["nbar"][0])) < 1e-15


@pytest.mark.parametrize("h,origin", [((1.0, 1.0, 1.0), (0, 0, 0)), ((0.5, 0.7, 1.1), (0.3, -2.0, 5.0)),
                                      ((0.01, 0.02, 0.005), (1, 1, 1))])
def test_tables_closed_form_on_boxes(h, origin):
    X = np.array([[origin[d] + h[d] * c[d] for d in range(3)] for c in CORNERS])
    g = _single(X)
    ref = cube_tables(h)
    # edge vectors are differences of coordinates of size |origin|: relative rounding ~ |origin| / h
    rel = 1e-14 * (1.0 + np.max(np.abs(origin)) / min(h))
    assert abs(g["vol"][0] - ref["vol"]) < rel * ref["vol"]
    for key, name in (("mass", "M"), ("grad", "G"), ("face", "F"), ("nbar", "Nbar")):
        scale = np.max(np.abs(ref[name]))
        assert np.max(np.abs(g[key][0] - ref[name])) < rel * scale, key


def test_tables_numeric_on_a_twisted_mesh():
    """Every cell of a jittered, twisted 3^3 mesh against a 4-point Gauss rule that uses the
    inverse Jacobian at each point and its own face orientation."""
    xyz, hexes = W.twisted_hex_mesh(3, 11, twist=0.6)
    g = H.geometry(xyz, hexes)
    for c in range(len(hexes)):
        ref = numeric_tables(xyz[hexes[c]])
        sc = ref["vol"]
        assert abs(g["vol"][c] - ref["vol"]) < 1e-14
        assert np.max(np.abs(g["mass"][c] - ref["M"])) < 1e-14 * sc
        assert np.max(np.abs(g["grad"][c] - ref["G"])) < 1e-13 * sc ** (2 / 3)
        assert np.max(np.abs(g["face"][c] - ref["F"])) < 1e-13 * sc ** (2 / 3)
        assert np.max(np.abs(g["nbar"][c] - ref["Nbar"])) < 1e-13 * sc ** (2 / 3)


def test_integral_identities():
    """Divergence theorem per basis function, gradient of a constant, partition of unity,
    closed surfaces, face integral of the normal, symmetry and definiteness."""
    xyz, hexes = W.twisted_hex_mesh(3, 4, twist=0.8)
    g = H.geometry(xyz, hexes)
    G, F, M = g["grad"], g["face"], g["mass"]
    # int_K d_d b_j = oint N_d b_j
    lhs = G.sum(axis=2)
    rhs = np.zeros_like(lhs)
    for f in range(6):
        rhs[:, :, face_vertices(f)] += F[:, f].sum(axis=2)
    assert np.max(np.abs(lhs - rhs)) < 1e-15
    assert np.max(np.abs(G.sum(axis=3))) < 1e-15  # gradient of sum_j b_j = 1
    assert np.max(np.abs(M.sum(axis=(1, 2)) - g["vol"])) < 1e-16
    assert np.max(np.abs(g["nbar"].sum(axis=1))) < 1e-16
    assert np.max(np.abs(F.sum(axis=(3, 4)) - g["nbar"])) < 1e-16
    assert np.max(np.abs(M - M.transpose(0, 2, 1))) < 1e-18
    assert np.max(np.abs(F - F.transpose(0, 1, 2, 4, 3))) < 1e-17
    assert np.min(np.linalg.eigvalsh(M)) > 0
    # G_d + G_d^T = oint N_d b_i b_j (integration by parts of int b_i d_d b_j)
    Sface = np.zeros_like(G)
    for f in range(6):
        fv = face_vertices(f)
        Sface[:, :, np.ix_(fv, fv)[0], np.ix_(fv, fv)[1]] += F[:, f]
    assert np.max(np.abs(G + G.transpose(0, 1, 3, 2) - Sface)) < 1e-15


def test_mesh_volume_neighbours_and_opposite_normals():
    xyz, hexes = W.twisted_hex_mesh(4, 9, twist=0.0)
    g = H.geometry(xyz, hexes)
    assert abs(g["vol"].sum() - 1.0) < 1e-14  # jitter moves interior vertices only
    xyz, hexes = W.twisted_hex_mesh(4, 9, twist=0.7)
    g = H.geometry(xyz, hexes)
    nbr, nn = g["nbr"], g["nbr_node"]
    assert (nbr < 0).sum() == 6 * 16
    ref = match_faces(hexes)
    for c in range(len(hexes)):
        for f in range(6):
            n = nbr[c, f]
            if n < 0:
                assert (c, f) not in ref
                continue
            assert ref[(c, f)][0] == n
            fb = list(nbr[n]).index(c)
            assert np.array_equal(g["nbar"][n, fb], -g["nbar"][c, f])  # bitwise opposite
            for k, v in enumerate(face_vertices(f)):
                assert hexes[n][nn[c, f, k]] == hexes[c][v]
    # the twist turns the top by 0.7 rad about the vertical axis: the total volume equals the
    # untwisted one minus what the bilinear side faces cut off, so it is below 1
    assert 0.99 < g["vol"].sum() < 1.0


def test_rejects_inverted_and_bad_meshes():
    X = np.array([[c[0], c[1], c[2]] for c in CORNERS], dtype=np.float64)
    X[[0, 1]] = X[[1, 0]]  # mirror: negative Jacobian
    with pytest.raises(OracleError):
        _single(X)
    xyz, hexes = W.twisted_hex_mesh(2, 1)
    bad = hexes.copy()
    bad[0, 0] = len(xyz)
    with pytest.raises(OracleError):
        H.geometry(xyz, bad)
    tri = np.concatenate([hexes, hexes[:1]])  # one face shared by three cells
    with pytest.raises(OracleError):
        H.geometry(xyz, tri)


def test_levels_are_longest_upwind_paths():
    cfg = W.hex_problem(W.small_box(n=4, G=1, n_polar=2, n_az=8), twist=0.5)
    P = H.ProblemHex(cfg)
    nbr, nbar = P.geom["nbr"], P.geom["nbar"]
    for a in range(P.D):
        O = P.omega[a]
        lev = P.level[a]
        for c in range(P.C):
            ups = []
            for f in range(6):
                s = O @ nbar[c, f]
                inflow = bool(P.inflow[a, c] >> f & 1)
                assert inflow == (s < -1e-12 * np.linalg.norm(nbar[c, f]))
                if inflow and nbr[c, f] >= 0:
                    ups.append(lev[nbr[c, f]])
            assert lev[c] == (1 + max(ups) if ups else 0)


@pytest.mark.parametrize("twist,seed", [(0.0, 1), (0.5, 2), (1.2, 3)])
def test_dense_whole_mesh_solve(twist, seed):
    """The sweep of one direction equals the whole-mesh dense solve (no order, no levels),
    with boundary inflow and an anisotropic source."""
    xyz, hexes = W.twisted_hex_mesh(2, seed, twist=twist)
    C = len(hexes)
    rng = np.random.default_rng(seed)
    G = 2
    sig = np.array([[0.7, 2.5]])
    cfg = dict(xyz=xyz, hexes=hexes, n_groups=G, cell_material=np.zeros(C, np.int32), sigma_t=sig,
               sigma_s=np.zeros((1, G, G)), Q=np.zeros((C, G, 8)), n_polar=2, n_azimuthal=8)
    S1 = rng.uniform(-1, 1, (C, G, 3))
    psi_in = rng.uniform(0, 1, (len(xyz), G))
    P = H.ProblemHex(cfg, S1=S1, psi_in=psi_in)
    q = rng.uniform(0, 1, (C, G, 8))
    for a in (0, 3, 9, 14):
        psi = P.sweep_direction(a, q)
        for g in range(G):
            ref = dense_direction_solve(xyz, hexes, P.omega[a], np.full(C, sig[0, g]), q[:, g], S1[:, g],
                                        psi_in[:, g])
            assert np.max(np.abs(psi[:, g] - ref)) < 1e-12 * np.max(np.abs(ref)), (a, g)


def _linear_field(rng, G):
    alpha = rng.uniform(1.0, 2.0, G)
    beta = rng.uniform(-0.5, 0.5, (G, 3))
    return alpha, beta


@pytest.mark.parametrize("twist", [0.0, 0.9])
def test_manufactured_linear_field_one_sweep(twist):
    """psi = alpha + beta.x solves Omega.grad psi + sigma psi = sigma psi + Omega.beta; a linear
    field of x lies in the trilinear space, so the sweep reproduces it at every node."""
    cfg = W.hex_problem(W.small_box(n=3, G=3, n_polar=2, n_az=8), twist=twist)
    rng = np.random.default_rng(7)
    alpha, beta = _linear_field(rng, 3)
    xyz, hexes = cfg["xyz"], cfg["hexes"]
    C = len(hexes)
    exact_v = alpha[None, :] + xyz @ beta.T  # [nv][G]
    exact = exact_v[hexes].transpose(0, 2, 1)  # [C][G][8]
    P = H.ProblemHex(cfg, S1=np.broadcast_to(beta, (C, 3, 3)).copy(), psi_in=exact_v)
    sig = P.sigma_t[0]
    q = sig[None, :, None] * exact
    for a in range(P.D):
        psi = P.sweep_direction(a, q)
        assert np.max(np.abs(psi - exact)) < 1e-12, a


def test_manufactured_source_iteration_with_scattering():
    """A scattering problem whose fixed point is the linear field: Q = 4 pi (sigma_t psi -
    sum_g' sigma_s[g'->g] psi_g'); the source iteration converges to psi at every node and
    phi = 4 pi psi."""
    cfg = W.hex_problem(W.two_material_box(n=3, G=3, n_polar=2, n_az=8), twist=0.4)
    rng = np.random.default_rng(3)
    alpha, beta = _linear_field(rng, 3)
    xyz, hexes = cfg["xyz"], cfg["hexes"]
    C = len(hexes)
    exact_v = alpha[None, :] + xyz @ beta.T
    exact = exact_v[hexes].transpose(0, 2, 1)
    mat = cfg["cell_material"]
    Q = np.empty_like(exact)
    for c in range(C):
        m = mat[c]
        Q[c] = FOUR_PI * (cfg["sigma_t"][m][:, None] * exact[c] - cfg["sigma_s"][m].T @ exact[c])
    cfg = dict(cfg, Q=Q)
    P = H.ProblemHex(cfg, S1=np.broadcast_to(beta, (C, 3, 3)).copy(), psi_in=exact_v)
    phi, it, r = P.source_iterate(1e-13, 400, threads=4)
    assert r < 1e-13
    assert np.max(np.abs(phi - FOUR_PI * exact)) < 1e-10 * FOUR_PI * np.max(exact)


def test_particle_balance_per_direction():
    """Vacuum boundaries: for every direction and group, absorption plus boundary outflow
    leakage equals the volumetric source (interior face terms cancel in pairs), with the
    leakage and integrals from the independent 4-point tables."""
    cfg = W.hex_problem(W.small_box(n=3, G=2, n_polar=2, n_az=8), twist=0.7)
    P = H.ProblemHex(cfg)
    rng = np.random.default_rng(5)
    q = rng.uniform(0, 1, (P.C, P.G, 8))
    tabs = [numeric_tables(cfg["xyz"][cfg["hexes"][c]]) for c in range(P.C)]
    nbr = P.geom["nbr"]
    for a in (0, 6, 13):
        O = P.omega[a]
        psi = P.sweep_direction(a, q)
        for g in range(P.G):
            src = absn = leak = 0.0
            for c, t in enumerate(tabs):
                rows = t["M"].sum(axis=1)
                src += rows @ q[c, g]
                absn += P.sigma_t[0, g] * rows @ psi[c, g]
                for f in range(6):
                    if nbr[c, f] >= 0:
                        continue
                    s = O @ t["Nbar"][f]
                    if s < -1e-12 * np.linalg.norm(t["Nbar"][f]):
                        continue  # vacuum inflow
                    fv = face_vertices(f)
                    leak += np.einsum("d,dkl->kl", O, t["F"][f]).sum(axis=0) @ psi[c, g, fv]
            assert abs(src - absn - leak) < 1e-13 * src, (a, g)


def test_mirror_symmetry():
    """Untwisted, unjittered box, one material, a source box symmetric about x = 1/2 and a
    quadrature symmetric under Omega_x -> -Omega_x: phi is symmetric under x -> 1 - x."""
    n = 4
    base = W.small_box(n=n, G=2, n_polar=2, n_az=8)
    xyz, hexes = W.twisted_hex_mesh(n, 1, jitter=0.0, twist=0.0)
    cfg = W.hex_problem(base, twist=0.0)
    Q = np.zeros((n ** 3, 2, 8))
    for c in range(n ** 3):
        i, j, k = c % n, (c // n) % n, c // (n * n)
        if i in (1, 2) and j == 1 and k >= 2:  # symmetric about x = 1/2 only
            Q[c, 0], Q[c, 1] = 1.0, 0.5
    cfg.update(xyz=xyz, hexes=hexes, Q=Q)
    P = H.ProblemHex(cfg)
    phi, _, _ = P.source_iterate(1e-12, 100, threads=4)
    for c in range(P.C):
        i, j, k = c % n, (c // n) % n, c // (n * n)
        m = (n - 1 - i) + n * (j + n * k)
        for v in range(8):
            assert np.allclose(phi[c, :, v], phi[m, :, v ^ 1], rtol=1e-12, atol=0), (c, v)


def test_integrated_flux_and_degenerate_inputs():
    cfg = W.hex_problem(W.small_box(n=2, G=2, n_polar=2, n_az=4), twist=0.3)
    P = H.ProblemHex(cfg)
    phi = np.ones((P.C, 2, 8))
    ig, tot = P.integrated_flux(phi)
    assert np.allclose(ig, P.geom["vol"].sum(), rtol=1e-14) and abs(tot - 2 * P.geom["vol"].sum()) < 1e-14
    zero = P.sweep(np.zeros((P.C, 2, 8)))[0]
    assert not zero.any()
    # zero groups and zero directions
    cfg0 = dict(cfg, n_groups=0, sigma_t=np.zeros((1, 0)), sigma_s=np.zeros((1, 0, 0)), Q=np.zeros((P.C, 0, 8)))
    P0 = H.ProblemHex(cfg0)
    assert P0.sweep(np.zeros((P.C, 0, 8)))[0].shape == (P.C, 0, 8)
    om, w = product_quadrature(2, 4)
    P1 = H.ProblemHex(cfg, omega=om[:0], w=w[:0])
    assert not P1.sweep(np.ones((P.C, 2, 8)))[0].any()


# ----------------------------------------------------------------- planted mistakes
MUTANTS = {
    "face_orientation": ("if (!s) { N[0] = -N[0];", "if (s) { N[0] = -N[0];"),
    "cofactor_transposed": ("cof[0][d] * db[j][0] + cof[1][d] * db[j][1] + cof[2][d] * db[j][2]",
                            "cof[d][0] * db[j][0] + cof[d][1] * db[j][1] + cof[d][2] * db[j][2]"),
    "mass_without_det": ("Mc[8 * i + j] += wt * det * b[i] * b[j];", "Mc[8 * i + j] += wt * b[i] * b[j];"),
    "face_term_sign": ("Fin[f][k][l] = -((O[0]", "Fin[f][k][l] = ((O[0]"),
    "face_rhs_dropped": ("b[i] += Fin[f][k][l] * up[l];", "b[i] += 0.0 * up[l];"),
    "upwind_node": ("psi[((size_t)n * G + g) * 8 + P->nbr_node[24 * c + 4 * f + k]]",
                    "psi[((size_t)n * G + g) * 8 + P->nbr_node[24 * c + 4 * f + (k ^ 1)]]"),
    "s1_dropped": ("b[i] += os * rowm[i];", "b[i] += 0.0 * os;"),
    "streaming_transposed": ("S[i][j] = (O[0] * Gc[8 * i + j] + O[1] * Gc[64 + 8 * i + j]) + O[2] * Gc[128 + 8 * i + j];",
                             "S[i][j] = (O[0] * Gc[8 * j + i] + O[1] * Gc[64 + 8 * j + i]) + O[2] * Gc[128 + 8 * j + i];"),
    "gauss_node": ("x[0] = 0.5 - h; x[1] = 0.5;", "x[0] = 0.5 - h; x[1] = 0.51;"),
    "classification_reversed": ("if (s < -eps) m", "if (s > eps) m"),
    "level_not_incremented": ("if (lev[n] < lev[c] + 1) lev[n] = lev[c] + 1;",
                              "if (lev[n] < lev[c]) lev[n] = lev[c];"),
}


def _battery(src):
    """Fast subset of the pins above against a modified oracle; returns the failing names."""
    failed = []
    lib = H.load(src)
    xyz, hexes = W.twisted_hex_mesh(2, 5, twist=0.8)
    C = len(hexes)
    try:
        g = H.geometry(xyz, hexes, lib)
        for c in range(C):
            ref = numeric_tables(xyz[hexes[c]])
            if (np.max(np.abs(g["mass"][c] - ref["M"])) > 1e-13 or np.max(np.abs(g["grad"][c] - ref["G"])) > 1e-13
                    or np.max(np.abs(g["face"][c] - ref["F"])) > 1e-13):
                failed.append("tables")
                break
    except OracleError:
        failed.append("tables(error)")
    rng = np.random.default_rng(2)
    cfg = dict(xyz=xyz, hexes=hexes, n_groups=1, cell_material=np.zeros(C, np.int32), sigma_t=np.array([[1.4]]),
               sigma_s=np.zeros((1, 1, 1)), Q=np.zeros((C, 1, 8)), n_polar=2, n_azimuthal=8)
    S1 = rng.uniform(-1, 1, (C, 1, 3))
    psi_in = rng.uniform(0, 1, (len(xyz), 1))
    try:
        P = H.ProblemHex(cfg, S1=S1, psi_in=psi_in, src=src)
        q = rng.uniform(0, 1, (C, 1, 8))
        for a in (0, 5, 11):
            psi = P.sweep_direction(a, q)
            ref = dense_direction_solve(xyz, hexes, P.omega[a], np.full(C, 1.4), q[:, 0], S1[:, 0], psi_in[:, 0])
            if np.max(np.abs(psi[:, 0] - ref)) > 1e-11 * np.max(np.abs(ref)):
                failed.append("dense")
                break
    except OracleError:
        failed.append("dense(error)")
    return failed


def test_unmodified_oracle_passes_the_battery():
    assert _battery(None) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    with open(H.SRC) as f:
        text = f.read()
    assert text.count(old) == 1, name
    src = tmp_path / f"mut_{name}.c"
    src.write_text(text.replace(old, new))
    assert _battery(str(src)), name
    os.remove(src)


def test_thick_medium_interior_matches_infinite_medium():
    """Deep inside an optically thick twisted box with a uniform source, phi -> Q / sigma_a (the
    central cells are three cells and 15 mean free paths from the boundary; upwind DG damps the
    boundary's influence cell by cell: 1.9e-4 here, 2.3e-3 with two cells to the boundary)."""
    n, G = 8, 1
    xyz, hexes = W.twisted_hex_mesh(n, 3, jitter=0.0, twist=0.25)
    C = len(hexes)
    xyz = xyz * 8.0  # 8 units wide, sigma_t = 5 => 40 mean free paths
    cfg = dict(xyz=xyz, hexes=hexes, n_groups=G, cell_material=np.zeros(C, np.int32), sigma_t=np.array([[5.0]]),
               sigma_s=np.array([[[2.5]]]), Q=np.ones((C, G, 8)), n_polar=4, n_azimuthal=8)
    P = H.ProblemHex(cfg)
    phi, it, r = P.source_iterate(1e-12, 200, threads=4)
    centre = np.linalg.norm(xyz[hexes].mean(axis=1) - 4.0, axis=1) < 1.5
    assert centre.sum() == 8
    assert np.max(np.abs(phi[centre] - 1.0 / 2.5)) < 1e-3


# ------------------------------------------------------------- lagged back edges
# The paper assumes an acyclic sweep graph per direction; twisted hexahedral grids with many
# directions have cycles.  Lagging one face per cycle (it reads the previous transport step's
# upwind values) keeps the sweep defined; at convergence the lag must not matter.
def _cyclic_cfg(G=2, n=4, twist=0.6):
    return W.hex_problem(W.small_box(n=n, G=G, n_polar=8, n_az=16), twist=twist)


def _dependency_graph_without_lags(P, a):
    """Kahn's algorithm over the non-lagged inflow faces, written out here: returns the
    longest-upwind-path levels, or None if a cycle remains."""
    nbr, C = P.geom["nbr"], P.C
    ups = [[nbr[c, f] for f in range(6) if (P.inflow[a, c] >> f & 1) and nbr[c, f] >= 0
            and not (P.lag[a, c] >> f & 1)] for c in range(C)]
    downs = [[] for _ in range(C)]
    for c in range(C):
        for u in ups[c]:
            downs[u].append(c)
    deg = [len(u) for u in ups]
    lev = [0] * C
    ready = [c for c in range(C) if deg[c] == 0]
    seen = 0
    while ready:
        u = ready.pop()
        seen += 1
        for c in downs[u]:
            lev[c] = max(lev[c], lev[u] + 1)
            deg[c] -= 1
            if deg[c] == 0:
                ready.append(c)
    return lev if seen == C else None


def test_lag_changes_nothing_on_an_acyclic_grid():
    cfg = W.hex_problem(W.small_box(n=4, G=2, n_polar=4, n_az=8), twist=0.25)
    P0, P1 = H.ProblemHex(cfg), H.ProblemHex(cfg, lag=True)
    assert not P1.lag.any()
    assert np.array_equal(P0.inflow, P1.inflow) and np.array_equal(P0.level, P1.level)
    phi = np.random.default_rng(3).uniform(0, 1, (P0.C, 2, 8))
    assert np.array_equal(P0.transport_step(phi), P1.transport_step(phi))


def test_lagged_faces_break_every_cycle():
    """The grid has cycles (the plain graph is an error); every lagged face is an interior
    inflow face, the graph without them is acyclic, and the levels are its longest upwind paths."""
    cfg = _cyclic_cfg()
    with pytest.raises(OracleError):
        H.ProblemHex(cfg)
    P = H.ProblemHex(cfg, lag=True)
    lagged_dirs = [a for a in range(P.D) if P.lag[a].any()]
    assert len(lagged_dirs) >= 8
    for a in range(P.D):
        for c in range(P.C):
            for f in range(6):
                if P.lag[a, c] >> f & 1:
                    assert P.inflow[a, c] >> f & 1 and P.geom["nbr"][c, f] >= 0
        lev = _dependency_graph_without_lags(P, a)
        assert lev is not None, a
        assert np.array_equal(np.array(lev), P.level[a]), a
    # one face per cycle: far fewer lagged faces than inflow faces
    assert int(np.unpackbits(P.lag).sum()) < 0.02 * int(np.unpackbits(P.inflow).sum())


def test_lagged_sweep_iterates_to_the_dense_solve():
    """For a fixed source, repeating the lagged sweep of one direction (each repetition reads
    the previous one's upwind values on the lagged faces) converges to the whole-mesh dense
    solve, which has no sweep order and no lag; with boundary inflow and S1."""
    cfg = _cyclic_cfg(G=2)
    xyz, hexes = cfg["xyz"], cfg["hexes"]
    C = len(hexes)
    rng = np.random.default_rng(5)
    S1 = rng.uniform(-1, 1, (C, 2, 3))
    psi_in = rng.uniform(0, 1, (len(xyz), 2))
    P = H.ProblemHex(cfg, S1=S1, psi_in=psi_in, lag=True)
    q = rng.uniform(0, 1, (C, 2, 8))
    sig = np.asarray(cfg["sigma_t"])[np.asarray(cfg["cell_material"])]
    for a in [a for a in range(P.D) if P.lag[a].any()][:3]:
        P.psi_prev = np.zeros((P.D, C, 2, 8))
        first = None
        for _ in range(400):
            psi = P.sweep_direction(a, q)
            if first is None:
                first = psi.copy()
            change = np.max(np.abs(psi - P.psi_prev[a]))
            P.psi_prev[a] = psi
            if change < 1e-15 * np.max(np.abs(psi)):
                break
        for g in range(2):
            ref = dense_direction_solve(xyz, hexes, P.omega[a], sig[:, g], q[:, g], S1[:, g], psi_in[:, g])
            assert np.max(np.abs(psi[:, g] - ref)) < 1e-11 * np.max(np.abs(ref)), (a, g)
            # the first lagged sweep (zero on the lagged faces) is not yet the answer
            assert np.max(np.abs(first[:, g] - ref)) > 1e-6 * np.max(np.abs(ref)), (a, g)


def test_lagged_source_iteration_converges_to_the_lag_free_answer():
    """Source iteration with lagged faces converges; at its fixed point every direction's psi is
    the dense (lag-free) solve of that direction with the converged source."""
    cfg = _cyclic_cfg(G=2)
    cfg["Q"] = np.random.default_rng(7).uniform(0.0, 1.0, cfg["Q"].shape)
    P = H.ProblemHex(cfg, lag=True)
    phi, it, r = P.source_iterate(1e-12, 2000, threads=8)
    assert r < 1e-12 and it > 2
    q = P.source(phi)
    sig = np.asarray(cfg["sigma_t"])[np.asarray(cfg["cell_material"])]
    for a in [a for a in range(P.D) if P.lag[a].any()][:3]:
        for g in range(2):
            ref = dense_direction_solve(cfg["xyz"], cfg["hexes"], P.omega[a], sig[:, g], q[:, g])
            assert np.max(np.abs(P.psi_prev[a][:, g] - ref)) < 1e-9 * np.max(np.abs(ref)), (a, g)


LAG_MUTANTS = {
    "lag_reads_current_psi": ("if (n >= 0 && lagged)", "if (n >= 0 && lagged && 0)"),
    "lag_wrong_face": ("lg[cur] |= (uint8_t)(1u << fo);", "lg[cur] |= (uint8_t)(1u << ((fo + 1) % 6));"),
    "lag_previous_psi_ignored": ("up[k] = P->psi_prev ? P->psi_prev[", "up[k] = 0 ? P->psi_prev["),
}


def _lag_battery(src):
    """The dense-solve limit of repeated lagged sweeps on one cyclic direction, against a
    modified oracle; returns whether it still holds."""
    cfg = _cyclic_cfg(G=1)
    C = len(cfg["hexes"])
    try:
        P = H.ProblemHex(cfg, lag=True, src=src)
        a = next(a for a in range(P.D) if P.lag[a].any())
        q = np.random.default_rng(1).uniform(0, 1, (C, 1, 8))
        P.psi_prev = np.zeros((P.D, C, 1, 8))
        for _ in range(300):
            P.psi_prev[a] = P.sweep_direction(a, q)
        sig = np.asarray(cfg["sigma_t"])[np.asarray(cfg["cell_material"])]
        ref = dense_direction_solve(cfg["xyz"], cfg["hexes"], P.omega[a], sig[:, 0], q[:, 0])
        return bool(np.max(np.abs(P.psi_prev[a][:, 0] - ref)) < 1e-11 * np.max(np.abs(ref)))
    except (OracleError, StopIteration):
        return False


def test_unmodified_oracle_passes_the_lag_battery():
    assert _lag_battery(None)


@pytest.mark.parametrize("name", sorted(LAG_MUTANTS))
def test_planted_lag_mistake_is_caught(name, tmp_path):
    old, new = LAG_MUTANTS[name]
    with open(H.SRC) as f:
        text = f.read()
    assert text.count(old) == 1, name
    src = tmp_path / f"mut_{name}.c"
    src.write_text(text.replace(old, new))
    assert not _lag_battery(str(src)), name
    os.remove(src)
