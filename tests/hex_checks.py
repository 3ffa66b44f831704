"""Independent checks for the trilinear-hexahedron oracle (`oracle/q1hex.py`).

Nothing here calls the oracle: these helpers recompute what the oracle must
produce by other routes, so that a test can pin it.

  * `exact_tables`: the element integrals of one hexahedron with rational
    vertex coordinates, in exact rational arithmetic with sympy (symbolic
    map, Jacobian adjugate, polynomial integration over the unit cube; the
    outward face orientation from the face-to-centroid side test).
  * `numeric_tables`: the same integrals in floating point by a 4-point
    Gauss rule with the inverse Jacobian at every point (not the cofactor
    columns), faces oriented by the centroid side test.
  * `cube_tables`: the closed forms on an axis-aligned box (tensor products
    of the 1D linear-element matrices).
  * `dense_direction_solve`: the whole-mesh upwind-DG system of one
    direction, assembled from `numeric_tables` with its own face matching,
    solved as one dense system (no sweep order, no t-levels).
"""
from __future__ import annotations

from fractions import Fraction
from itertools import product

import numpy as np

CORNERS = [(v & 1, (v >> 1) & 1, (v >> 2) & 1) for v in range(8)]


def face_vertices(f):
    """Local vertices on reference face xi_d = s (f = 2d + s), increasing."""
    d, s = divmod(f, 2)
    return [v for v in range(8) if CORNERS[v][d] == s]


# ----------------------------------------------------------------- exact (sympy)
def exact_tables(X):
    """X: [8][3] of Fractions.  Returns dict of Fraction arrays (as nested lists):
    vol, M[8][8], G[3][8][8] (int b_i d_x_d b_j), F[6][3][4][4] (int_f N_d b_k b_l,
    N outward), Nbar[6][3]."""
    import sympy as sp

    xi = sp.symbols("x0 x1 x2")
    b = []
    for a in CORNERS:
        e = sp.Integer(1)
        for d in range(3):
            e *= xi[d] if a[d] else (1 - xi[d])
        b.append(sp.expand(e))
    xs = [sp.expand(sum(sp.Rational(X[v][r].numerator, X[v][r].denominator) * b[v] for v in range(8)))
          for r in range(3)]
    J = sp.Matrix(xs).jacobian(list(xi))
    det = sp.expand(J.det())
    adjT = J.adjugate().T  # det(J) J^{-T}

    def cube_int(e):
        p = sp.Poly(sp.expand(e), *xi)
        tot = sp.Integer(0)
        for mon, co in p.terms():
            tot += co / ((mon[0] + 1) * (mon[1] + 1) * (mon[2] + 1))
        return Fraction(int(sp.fraction(tot)[0]), int(sp.fraction(tot)[1]))

    vol = cube_int(det)
    M = [[cube_int(b[i] * b[j] * det) for j in range(8)] for i in range(8)]
    dref = [[sp.diff(b[j], xi[k]) for k in range(3)] for j in range(8)]
    phys = [[sp.expand(sum(adjT[d, k] * dref[j][k] for k in range(3))) for j in range(8)] for d in range(3)]
    G = [[[cube_int(b[i] * phys[d][j]) for j in range(8)] for i in range(8)] for d in range(3)]
    centroid = [sum(X[v][r] for v in range(8)) / 8 for r in range(3)]
    F, Nbar = [], []
    for f in range(6):
        d, s = divmod(f, 2)
        others = [k for k in range(3) if k != d]
        sub = {xi[d]: s}
        t1 = [sp.diff(xs[r], xi[others[0]]).subs(sub) for r in range(3)]
        t2 = [sp.diff(xs[r], xi[others[1]]).subs(sub) for r in range(3)]
        N = [sp.expand(t1[1] * t2[2] - t1[2] * t2[1]), sp.expand(t1[2] * t2[0] - t1[0] * t2[2]),
             sp.expand(t1[0] * t2[1] - t1[1] * t2[0])]

        def face_int(e):
            p = sp.Poly(sp.expand(e.subs(sub)), xi[others[0]], xi[others[1]])
            tot = sp.Integer(0)
            for mon, co in p.terms():
                tot += co / ((mon[0] + 1) * (mon[1] + 1))
            return Fraction(int(sp.fraction(tot)[0]), int(sp.fraction(tot)[1]))

        nb = [face_int(N[r]) for r in range(3)]
        fv = face_vertices(f)
        fc = [sum(X[v][r] for v in fv) / 4 for r in range(3)]
        side = sum(nb[r] * (fc[r] - centroid[r]) for r in range(3))
        sign = 1 if side > 0 else -1
        nb = [sign * x for x in nb]
        Nbar.append(nb)
        F.append([[[sign * face_int(N[r] * b[k] * b[l]) for l in fv] for k in fv] for r in range(3)])
    return dict(vol=vol, M=M, G=G, F=F, Nbar=Nbar)


# ----------------------------------------------------------------- numeric
def _basis(x):
    """Values [8] and reference gradients [8][3] of the trilinear basis at x (3,)."""
    b = np.empty(8)
    db = np.empty((8, 3))
    for v, a in enumerate(CORNERS):
        l = [x[d] if a[d] else 1.0 - x[d] for d in range(3)]
        dl = [1.0 if a[d] else -1.0 for d in range(3)]
        b[v] = l[0] * l[1] * l[2]
        db[v] = (dl[0] * l[1] * l[2], l[0] * dl[1] * l[2], l[0] * l[1] * dl[2])
    return b, db


def numeric_tables(X, npts=4):
    """Float tables of one hexahedron (X [8][3]) by an npts-point Gauss rule per axis."""
    X = np.asarray(X, dtype=np.float64)
    gx, gw = np.polynomial.legendre.leggauss(npts)
    gx, gw = 0.5 * (gx + 1.0), 0.5 * gw
    M = np.zeros((8, 8))
    G = np.zeros((3, 8, 8))
    vol = 0.0
    for (p, q, r) in product(range(npts), repeat=3):
        b, db = _basis((gx[p], gx[q], gx[r]))
        J = X.T @ db  # J[r][k] = d x_r / d xi_k
        dJ = np.linalg.det(J)
        wt = gw[p] * gw[q] * gw[r] * dJ
        gphys = db @ np.linalg.inv(J)  # [8][3]: grad_x b_j = J^{-T} grad_xi b_j
        vol += wt
        M += wt * np.outer(b, b)
        for d in range(3):
            G[d] += wt * np.outer(b, gphys[:, d])
    centroid = X.mean(axis=0)
    F = np.zeros((6, 3, 4, 4))
    Nbar = np.zeros((6, 3))
    for f in range(6):
        d, s = divmod(f, 2)
        o = [k for k in range(3) if k != d]
        fv = face_vertices(f)
        acc = np.zeros((3, 4, 4))
        nb = np.zeros(3)
        for p, q in product(range(npts), repeat=2):
            x = [0.0] * 3
            x[d], x[o[0]], x[o[1]] = float(s), gx[p], gx[q]
            b, db = _basis(x)
            J = X.T @ db
            N = np.cross(J[:, o[0]], J[:, o[1]])
            wt = gw[p] * gw[q]
            nb += wt * N
            acc += wt * N[:, None, None] * np.outer(b[fv], b[fv])[None]
        sign = 1.0 if nb @ (X[fv].mean(axis=0) - centroid) > 0 else -1.0
        F[f] = sign * acc
        Nbar[f] = sign * nb
    return dict(vol=vol, M=M, G=G, F=F, Nbar=Nbar)


def cube_tables(h):
    """Closed forms on the box [0,h0]x[0,h1]x[0,h2] (h a 3-vector): tensor products of
    the 1D linear-element mass m = [[1/3, 1/6], [1/6, 1/3]] * length and the 1D
    convection g[a][b] = int l_a l_b' = (+1/2 if b else -1/2)."""
    h = np.asarray(h, dtype=np.float64)
    m = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    g = np.array([[-0.5, 0.5], [-0.5, 0.5]])
    M = np.zeros((8, 8))
    G = np.zeros((3, 8, 8))
    for i, a in enumerate(CORNERS):
        for j, c in enumerate(CORNERS):
            M[i, j] = np.prod([m[a[d], c[d]] * h[d] for d in range(3)])
            for d in range(3):
                G[d, i, j] = np.prod([(g[a[e], c[e]] if e == d else m[a[e], c[e]] * h[e]) for e in range(3)])
    F = np.zeros((6, 3, 4, 4))
    Nbar = np.zeros((6, 3))
    for f in range(6):
        d, s = divmod(f, 2)
        o = [k for k in range(3) if k != d]
        area = h[o[0]] * h[o[1]]
        fv = face_vertices(f)
        sgn = 1.0 if s else -1.0
        Nbar[f, d] = sgn * area
        for k, vk in enumerate(fv):
            for l, vl in enumerate(fv):
                F[f, d, k, l] = sgn * np.prod([m[CORNERS[vk][e], CORNERS[vl][e]] * h[e] for e in o])
    return dict(vol=float(np.prod(h)), M=M, G=G, F=F, Nbar=Nbar)


# ----------------------------------------------------------------- dense solve
def match_faces(hexes):
    """{(cell, face): (neighbour, {local vertex of cell: local vertex of neighbour})}."""
    owners = {}
    for c, hx in enumerate(hexes):
        for f in range(6):
            key = tuple(sorted(int(hx[v]) for v in face_vertices(f)))
            owners.setdefault(key, []).append((c, f))
    out = {}
    for key, lst in owners.items():
        assert len(lst) <= 2
        if len(lst) == 2:
            for (c, f), (n, _) in (lst, lst[::-1]):
                out[(c, f)] = (n, {v: list(hexes[n]).index(hexes[c][v]) for v in face_vertices(f)})
    return out


def dense_direction_solve(xyz, hexes, omega, sigma_t_c, q, S1=None, psi_in=None, eps=1e-12):
    """psi [C][8] of one direction and one group for the whole mesh as a single dense
    system.  Face f of cell c is inflow iff Omega.Nbar < -eps |Nbar| with Nbar from the
    face quadrature; the inflow face term is -int_f (Omega.N) b_k (psi_k - psi_up,k)."""
    C = len(hexes)
    tabs = [numeric_tables(xyz[hexes[c]]) for c in range(C)]
    nb = match_faces(hexes)
    A = np.zeros((8 * C, 8 * C))
    rhs = np.zeros(8 * C)
    for c, t in enumerate(tabs):
        r0 = 8 * c
        A[r0:r0 + 8, r0:r0 + 8] += np.einsum("d,dij->ij", omega, t["G"]) + sigma_t_c[c] * t["M"]
        rhs[r0:r0 + 8] += t["M"] @ q[c]
        if S1 is not None:
            rhs[r0:r0 + 8] += (omega @ S1[c]) * t["M"].sum(axis=1)
        for f in range(6):
            s = omega @ t["Nbar"][f]
            if not s < -eps * np.linalg.norm(t["Nbar"][f]):
                continue
            fv = face_vertices(f)
            W = -np.einsum("d,dkl->kl", omega, t["F"][f])
            for k, vk in enumerate(fv):
                for l, vl in enumerate(fv):
                    A[r0 + vk, r0 + vl] += W[k, l]
                    if (c, f) in nb:
                        n, mp = nb[(c, f)]
                        A[r0 + vk, 8 * n + mp[vl]] -= W[k, l]
                    elif psi_in is not None:
                        rhs[r0 + vk] += W[k, l] * psi_in[hexes[c][vl]]
    return np.linalg.solve(A, rhs).reshape(C, 8)
