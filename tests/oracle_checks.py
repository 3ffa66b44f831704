"""Independent checks that pin the oracle to the mathematics, not to itself.

Everything here is re-derived from the definitions with different machinery
than the oracle uses: element integrals by exact quadrature rules (Keast's
degree-2 rule on tetrahedra, the edge-midpoint rule on triangles) instead of
closed forms; geometry with numpy's inverse/cross/determinant; face matching
with a Python dict; the global single-direction upwind-DG system solved with
dense LU (numpy.linalg.solve) instead of a sweep.

Each check returns an error measure so that both the pins (error small) and
the planted-mistake tests (error large) can use it.
"""
from __future__ import annotations

import numpy as np

KEAST_A = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
KEAST_B = (5.0 - np.sqrt(5.0)) / 20.0
FOUR_PI = 4.0 * np.pi


def keast_points(x):
    """4-point degree-2 rule on the tetrahedron with vertices x[4][3]; weights V/4."""
    lam = np.full((4, 4), KEAST_B)
    np.fill_diagonal(lam, KEAST_A)
    return lam  # barycentric coordinates of the 4 points (rows)


def tet_volume(x):
    return np.linalg.det(np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]], axis=1)) / 6.0


def basis_gradients(x):
    J = np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]], axis=1)  # columns are edges
    Ji = np.linalg.inv(J)
    g = np.zeros((4, 3))
    g[1:] = Ji
    g[0] = -Ji.sum(axis=0)
    return g


def face_geometry(x, f):
    """Nodes, area, outward unit normal of the face opposite local vertex f."""
    nodes = [i for i in range(4) if i != f]
    p = x[nodes]
    cr = np.cross(p[1] - p[0], p[2] - p[0])
    area = 0.5 * np.linalg.norm(cr)
    n = cr / np.linalg.norm(cr)
    if np.dot(n, x[f] - p.mean(axis=0)) > 0:
        n = -n
    return nodes, area, n


def element_integrals(x):
    """stream[d][i][j] = int b_i d_d b_j, mass[i][j] = int b_i b_j, by Keast quadrature."""
    V = tet_volume(x)
    lam = keast_points(x)
    g = basis_gradients(x)
    mass = np.einsum("q,qi,qj->ij", np.full(4, V / 4.0), lam, lam)
    bint = np.einsum("q,qi->i", np.full(4, V / 4.0), lam)
    stream = np.einsum("i,jd->dij", bint, g)
    return V, stream, mass


def face_mass(area):
    """int_f b_i b_j on a triangle by the edge-midpoint rule (exact for quadratics),
    for the three face nodes in order."""
    mids = np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]])
    return np.einsum("q,qi,qj->ij", np.full(3, area / 3.0), mids, mids)


def match_faces(tets):
    """nbr[c][f] (or -1) with a dict over sorted vertex triples."""
    owner = {}
    nbr = -np.ones((len(tets), 4), dtype=np.int64)
    for c, t in enumerate(tets):
        for f in range(4):
            key = tuple(sorted(int(t[i]) for i in range(4) if i != f))
            owner.setdefault(key, []).append((c, f))
    for lst in owner.values():
        assert len(lst) <= 2
        if len(lst) == 2:
            (c0, f0), (c1, f1) = lst
            nbr[c0, f0] = c1
            nbr[c1, f1] = c0
    return nbr


def global_direction_system(xyz, tets, omega, sig_t, q, S1=None, psi_in=None):
    """Assemble and solve, by dense LU, the upwind-DG system of ONE direction and
    ONE group on the whole mesh (unknowns psi[c][i], 4 per cell).

    q: [C][4] angular source per steradian (nodal); S1: [C][3] or None;
    psi_in: [nv] boundary inflow per vertex or None (vacuum).  sig_t: [C].
    Returns psi [C][4] and the smallest |Omega.n| A over faces (to confirm no
    face sits on the inflow threshold)."""
    Cn = len(tets)
    nbr = match_faces(tets)
    A = np.zeros((4 * Cn, 4 * Cn))
    b = np.zeros(4 * Cn)
    smin = np.inf
    for c, t in enumerate(tets):
        x = xyz[t]
        V, stream, mass = element_integrals(x)
        r = slice(4 * c, 4 * c + 4)
        A[r, r] += np.einsum("d,dij->ij", omega, stream) + sig_t[c] * mass
        b[r] += mass @ q[c]
        if S1 is not None:
            b[r] += (V / 4.0) * np.dot(omega, S1[c])
        for f in range(4):
            nodes, area, n = face_geometry(x, f)
            s = np.dot(omega, n) * area
            smin = min(smin, abs(s))
            if s >= 0:
                continue
            Mf = -np.dot(omega, n) * face_mass(area)
            for a_, i in enumerate(nodes):
                for b_, j in enumerate(nodes):
                    A[4 * c + i, 4 * c + j] += Mf[a_, b_]
                    nb = nbr[c, f]
                    if nb >= 0:
                        k = int(np.nonzero(tets[nb] == t[j])[0][0])
                        A[4 * c + i, 4 * nb + k] -= Mf[a_, b_]
                    elif psi_in is not None:
                        b[4 * c + i] += Mf[a_, b_] * psi_in[t[j]]
    psi = np.linalg.solve(A, b).reshape(Cn, 4)
    return psi, smin


def mms_problem(cfg, seed=7):
    """Manufactured solution psi_g(x) = alpha_g + beta_g . x (direction independent).

    Q_g = 4 pi (sigma_t,g psi_g - sum_g' sigma_s[g'->g] psi_g') at the nodes (the
    total isotropic source that balances Eq. (1) for a linear psi), S1_g = beta_g
    (the angular term Omega . grad psi), inflow = psi on boundary vertices.
    Returns (cfg with Q replaced, S1 [C][G][3], psi_in [nv][G], exact psi [C][G][4])."""
    rng = np.random.default_rng(seed)
    G = cfg["n_groups"]
    alpha = rng.uniform(1.0, 2.0, G)
    beta = rng.uniform(-0.5, 0.5, (G, 3))
    xyz, tets = cfg["xyz"], cfg["tets"]
    psi_v = alpha[None, :] + xyz @ beta.T  # [nv][G]
    psi_nodes = psi_v[tets]  # [C][4][G]
    psi_exact = np.transpose(psi_nodes, (0, 2, 1)).copy()  # [C][G][4]
    mat = cfg["cell_material"]
    st = cfg["sigma_t"][mat]  # [C][G]
    Ss = cfg["sigma_s"][mat]  # [C][G][G] from->to
    scat = np.einsum("cgi,cgh->chi", psi_exact, Ss)
    Q = FOUR_PI * (st[:, :, None] * psi_exact - scat)
    S1 = np.repeat(beta[None], len(tets), axis=0)
    out = dict(cfg)
    out["Q"] = Q
    return out, S1, psi_v, psi_exact


def cell_balance(P, psi, q, a, S1=None, psi_in=None):
    """Per (cell, group) particle balance of one direction's solution psi [C][G][4]
    computed from numpy geometry: net leakage + absorption - source, divided by
    the sum of the magnitudes of those terms.  Returns the max relative error."""
    xyz, tets = P.cfg["xyz"], P.cfg["tets"]
    O = P.omega[a]
    nbr = match_faces(tets)
    st = P.sigma_t[P.material]  # [C][G]
    Cn, G = psi.shape[0], psi.shape[1]
    worst = 0.0
    for c in range(Cn):
        x = xyz[tets[c]]
        V = tet_volume(x)
        leak = np.zeros(G)
        mag = np.zeros(G)
        for f in range(4):
            nodes, area, n = face_geometry(x, f)
            s = np.dot(O, n) * area
            if s >= 0:
                tr = psi[c][:, nodes].mean(axis=1)
            else:
                nb = nbr[c, f]
                if nb >= 0:
                    ks = [int(np.nonzero(tets[nb] == tets[c][i])[0][0]) for i in nodes]
                    tr = psi[nb][:, ks].mean(axis=1)
                elif psi_in is not None:
                    tr = psi_in[tets[c][nodes]].mean(axis=0)
                else:
                    tr = np.zeros(G)
            leak += s * tr
            mag += np.abs(s * tr)
        absn = st[c] * (V / 4.0) * psi[c].sum(axis=1)
        src = (V / 4.0) * q[c].sum(axis=1)
        if S1 is not None:
            src = src + V * (S1[c] @ O)
        err = leak + absn - src
        worst = max(worst, float(np.max(np.abs(err) / (mag + np.abs(absn) + np.abs(src) + 1e-300))))
    return worst
