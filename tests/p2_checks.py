"""Independent checks for the second-order (ten-node) element.

Element integrals here are exact: the ten basis functions are written as
polynomials in the barycentric coordinates (dicts of exponent tuples with
rational coefficients) and integrated monomial by monomial with
  int_K lambda^a dV = 6 V a! / (|a| + 3)!,   int_F lambda^a dA = 2 A a! / (|a| + 2)!
(a! = product of the factorials of the exponents), instead of the oracle's
collapsed Gauss-Legendre quadrature.  Upwind coupling is found by matching
global vertices and vertex pairs with a dict instead of the oracle's
evaluation of the neighbour's field at physical points.
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial, prod

import numpy as np

EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
FOUR_PI = 4.0 * np.pi


# ------------------------------------------------------------ polynomials in lambda
def _mono(k, n=4):
    e = [0] * n
    e[k] = 1
    return tuple(e)


def _mul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(a + b for a, b in zip(ea, eb))
            out[e] = out.get(e, 0) + ca * cb
    return {e: c for e, c in out.items() if c != 0}


def _add(p, q, s=1):
    out = dict(p)
    for e, c in q.items():
        out[e] = out.get(e, 0) + s * c
    return {e: c for e, c in out.items() if c != 0}


def node_alphas(order):
    """Lattice multi-indices of the nodes, in the element's node order: vertices; per edge
    (a,b) its interior nodes from a towards b; (third order) the face centres, face f opposite vertex f."""
    out = []
    for v in range(4):
        out.append(tuple(order if k == v else 0 for k in range(4)))
    for a, b in EDGES:
        for t in range(order - 1, 0, -1):  # lambda_a = t / order
            out.append(tuple(t if k == a else (order - t if k == b else 0) for k in range(4)))
    if order == 3:
        for f in range(4):
            out.append(tuple(0 if k == f else 1 for k in range(4)))
    return out


def basis_polys(order=2):
    """The Lagrange basis on the equispaced lattice as polynomials in (lambda_0..lambda_3):
    phi_alpha = prod_k prod_{m < alpha_k} (order lambda_k - m) / (m + 1)."""
    out = []
    for al in node_alphas(order):
        p = {(0, 0, 0, 0): Fraction(1)}
        for k in range(4):
            for m in range(al[k]):
                fac = {_mono(k): Fraction(order, m + 1), (0, 0, 0, 0): Fraction(-m, m + 1)}
                p = _mul(p, {e: c for e, c in fac.items() if c != 0})
        out.append(p)
    return out


def dpoly(p, k):
    """d p / d lambda_k."""
    out = {}
    for e, c in p.items():
        if e[k] > 0:
            f = list(e)
            f[k] -= 1
            out[tuple(f)] = out.get(tuple(f), 0) + c * e[k]
    return out


def integrate_cell(p):
    """int_K p dV / V."""
    s = Fraction(0)
    for e, c in p.items():
        s += c * 6 * Fraction(prod(factorial(x) for x in e), factorial(sum(e) + 3))
    return s


def integrate_face(p, f):
    """int_F p dA / A over the face opposite vertex f (lambda_f = 0 there)."""
    s = Fraction(0)
    for e, c in p.items():
        if e[f] != 0:
            continue
        s += c * 2 * Fraction(prod(factorial(x) for x in e), factorial(sum(e) + 2))
    return s


def reference_tables(order=2):
    """Exact per-unit-volume / per-unit-area tables: p[i] = int phi_i / V, M[i][j] = int phi_i phi_j / V,
    Dk[k][i][j] = int phi_i d phi_j / d lambda_k / V, F[f][i][j] = int_F phi_i phi_j / A (float arrays)."""
    B = basis_polys(order)
    p = np.array([float(integrate_cell(b)) for b in B])
    M = np.array([[float(integrate_cell(_mul(bi, bj))) for bj in B] for bi in B])
    Dk = np.array([[[float(integrate_cell(_mul(bi, dpoly(bj, k)))) for bj in B] for bi in B] for k in range(4)])
    F = np.array([[[float(integrate_face(_mul(bi, bj), f)) for bj in B] for bi in B] for f in range(4)])
    return p, M, Dk, F


_TABLES = {}


def tables(order=2):
    if order not in _TABLES:
        _TABLES[order] = reference_tables(order)
    return _TABLES[order]


def face_nodes(f, order=2):
    """Local node indices on the face opposite vertex f (the nodes whose lambda_f is zero)."""
    return [i for i, al in enumerate(node_alphas(order)) if al[f] == 0]


def global_node_keys(tets, order=2):
    """Per cell, the global identity of each node: the multiset of global vertices its
    lattice multi-index weights (vertex -> ((v, order),); edge node -> ((va, ta), (vb, tb)); ...)."""
    keys = []
    als = node_alphas(order)
    for t in np.asarray(tets):
        keys.append([tuple(sorted((int(t[k]), al[k]) for k in range(4) if al[k])) for al in als])
    return keys


# ------------------------------------------------------------ dense global system
def dense_direction_solve(geom, omega_a, sigma_t_c, q, inflow_mask, order=2):
    """Single direction, single group: assemble the global (NB C) x (NB C) upwind-DG
    system with the exact tables and dict-based coupling, solve it densely.
    sigma_t_c [C], q [C][NB] (per steradian), inflow_mask [C]; vacuum boundary."""
    p, M, Dk, F = tables(order)
    nb = M.shape[0]
    tets = geom["tets"]
    Cn = tets.shape[0]
    keys = global_node_keys(tets, order)
    where = {}
    for c in range(Cn):
        for i, k in enumerate(keys[c]):
            where.setdefault(k, []).append((c, i))
    A = np.zeros((nb * Cn, nb * Cn))
    b = np.zeros(nb * Cn)
    for c in range(Cn):
        V = geom["vol"][c]
        og = geom["grad"][c] @ omega_a
        K = V * np.einsum("k,kij->ij", og, Dk)
        rc = slice(nb * c, nb * c + nb)
        A[rc, rc] += K + sigma_t_c[c] * V * M
        b[rc] += V * M @ q[c]
        for f in range(4):
            if not (inflow_mask[c] >> f) & 1:
                continue
            s = abs(float(geom["normal"][c, f] @ omega_a))
            Ff = s * F[f]
            A[rc, rc] += Ff
            n = int(geom["nbr"][c, f])
            if n < 0:
                continue
            for j in face_nodes(f, order):
                (nj,) = [i for (cc, i) in where[keys[c][j]] if cc == n]
                A[rc, nb * n + nj] -= Ff[:, j]
    return np.linalg.solve(A, b).reshape(Cn, nb)


# ------------------------------------------------------------ manufactured solution
def cubic_field(rng, G):
    """psi_g(x) = quadratic part + sum_d c_gd x_d^3 + e_g x y z per group; (value, gradient) callables."""
    val2, grad2 = quadratic_field(rng, G)
    c3 = rng.uniform(-0.3, 0.3, (G, 3))
    e3 = rng.uniform(-0.3, 0.3, G)

    def value(x):
        return val2(x) + np.einsum("...d,gd->...g", x ** 3, c3) + e3 * (x[..., 0] * x[..., 1] * x[..., 2])[..., None]

    def gradient(x):
        g = grad2(x) + 3.0 * np.einsum("...d,gd->...gd", x ** 2, c3)
        xyz = np.stack([x[..., 1] * x[..., 2], x[..., 0] * x[..., 2], x[..., 0] * x[..., 1]], axis=-1)
        return g + e3[:, None] * xyz[..., None, :]

    return value, gradient


def quadratic_field(rng, G):
    """psi_g(x) = a_g + b_g . x + x^T S_g x per group (S symmetric); returns (value, gradient) callables."""
    a = rng.uniform(0.5, 1.5, G)
    bb = rng.uniform(-0.5, 0.5, (G, 3))
    S = rng.uniform(-0.3, 0.3, (G, 3, 3))
    S = 0.5 * (S + S.transpose(0, 2, 1))

    def value(x):  # x [..., 3] -> [..., G]
        return a + np.einsum("...d,gd->...g", x, bb) + np.einsum("...d,gde,...e->...g", x, S, x)

    def gradient(x):  # -> [..., G, 3]
        return bb + 2.0 * np.einsum("gde,...e->...gd", S, x)

    return value, gradient


def mms_inputs(cfg, node_xyz, rng, field=None):
    """Q, S1, psi_bc and the exact nodal psi [C][G][nodes] of a manufactured solution (quadratic
    unless `field` is given; direction independent, so phi = 4 pi psi):
    Q = 4 pi (sigma_t psi - sum_g' sigma_s[g'->g] psi_g'), S1 = grad psi (the streaming term
    Omega . grad psi enters as the source Omega . S1)."""
    G = int(cfg["n_groups"])
    value, gradient = (field or quadratic_field)(rng, G)
    psi = value(node_xyz).transpose(0, 2, 1)  # [C][G][10]
    S1 = gradient(node_xyz).transpose(0, 2, 1, 3)  # [C][G][10][3]
    mat = np.asarray(cfg["cell_material"])
    st = np.asarray(cfg["sigma_t"])[mat]  # [C][G]
    ss = np.asarray(cfg["sigma_s"])[mat]  # [C][G'][G]
    Q = FOUR_PI * (st[:, :, None] * psi - np.einsum("chg,chi->cgi", ss, psi))
    return Q, S1, psi.copy(), psi
