"""Plain FP64 CPU oracle for the upwind-DG sweep on trilinear (eight-node) hexahedra.

TEST INFRASTRUCTURE ONLY (same rules as the rest of `oracle/`).  The C part
(`tf_oracle_hex.c`) computes the element integrals by quadrature, the face
neighbours, the face classification and t-levels, and sweeps; this module adds
the source update, stopping test, integrated flux and source iteration in numpy.

Node order per cell: the eight vertices of hexes[c], local vertex a + 2b + 4c at
the reference corner (a, b, c).  Arrays: Q, q, phi [C][G][8]; psi [C][G][8] per
direction.  Face f = 2d + s is the reference face xi_d = s.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import FOUR_PI, ORA_OK, OracleError, _p, build, product_quadrature

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tf_oracle_hex.c")
NB = 8

_libs: dict = {}


class _ProblemHex(C.Structure):
    _fields_ = [
        ("nc", C.c_int64), ("nv", C.c_int64), ("G", C.c_int32), ("D", C.c_int32),
        ("xyz", C.c_void_p), ("hexes", C.c_void_p), ("mass", C.c_void_p), ("grad", C.c_void_p),
        ("face", C.c_void_p), ("nbar", C.c_void_p), ("nbr", C.c_void_p), ("nbr_node", C.c_void_p),
        ("omega", C.c_void_p), ("w", C.c_void_p), ("inflow", C.c_void_p), ("level", C.c_void_p),
        ("material", C.c_void_p), ("sigma_t", C.c_void_p), ("S1", C.c_void_p), ("psi_in", C.c_void_p),
        ("lag", C.c_void_p), ("psi_prev", C.c_void_p),
    ]


def load(src=None):
    """The hexahedral oracle library (`src`: a modified copy for planted-mistake tests)."""
    key = src or SRC
    if key not in _libs:
        lib = C.CDLL(build(src=key))
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
        lib.orah_face_node.argtypes = [i32, i32]
        lib.orah_geometry.argtypes = [i64, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.orah_graph.argtypes = [i64, vp, vp, i32, vp, vp, vp]
        lib.orah_graph_lag.argtypes = [i64, vp, vp, i32, vp, vp, vp, vp]
        lib.orah_sweep_direction.argtypes = [C.POINTER(_ProblemHex), i32, vp, vp]
        lib.orah_sweep.argtypes = [C.POINTER(_ProblemHex), vp, i32, vp, vp, vp, i32, C.POINTER(C.c_int)]
        _libs[key] = lib
    return _libs[key]


def _check(code, what):
    if code != ORA_OK:
        raise OracleError(code, what)


def face_nodes(f, lib=None):
    """Local vertices of face f in face-local order."""
    lib = lib or load()
    return [lib.orah_face_node(f, k) for k in range(4)]


def geometry(xyz, hexes, lib=None):
    """Element integrals and neighbours: vol [C], mass [C][8][8], grad [C][3][8][8]
    (int b_i d_d b_j), face [C][6][3][4][4] (int_f N_d b_k b_l), nbar [C][6][3],
    nbr [C][6], nbr_node [C][6][4]."""
    lib = lib or load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    hexes = np.ascontiguousarray(hexes, dtype=np.int32)
    nc = hexes.shape[0]
    g = dict(vol=np.zeros(nc), mass=np.zeros((nc, 8, 8)), grad=np.zeros((nc, 3, 8, 8)),
             face=np.zeros((nc, 6, 3, 4, 4)), nbar=np.zeros((nc, 6, 3)),
             nbr=np.zeros((nc, 6), dtype=np.int32), nbr_node=np.zeros((nc, 6, 4), dtype=np.int32))
    _check(lib.orah_geometry(xyz.shape[0], _p(xyz), nc, _p(hexes), _p(g["vol"]), _p(g["mass"]), _p(g["grad"]),
                             _p(g["face"]), _p(g["nbar"]), _p(g["nbr"]), _p(g["nbr_node"])), "geometry")
    g["xyz"], g["hexes"] = xyz, hexes
    return g


def graph(geom, omega, lib=None, lag=False):
    """Inflow-face bitmask [D][C] (uint8, six bits) and t-level [D][C] (int32); with lag, also the
    lagged back edges [D][C] (bit f: inflow face f reads the previous step's upwind psi), chosen
    whenever no cell is ready as the open inflow faces of the lowest-numbered waiting cell."""
    lib = lib or load()
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    D, nc = omega.shape[0], geom["vol"].shape[0]
    inflow = np.zeros((D, nc), dtype=np.uint8)
    level = np.zeros((D, nc), dtype=np.int32)
    if not lag:
        _check(lib.orah_graph(nc, _p(geom["nbr"]), _p(geom["nbar"]), D, _p(omega), _p(inflow), _p(level)), "graph")
        return inflow, level
    lagged = np.zeros((D, nc), dtype=np.uint8)
    _check(lib.orah_graph_lag(nc, _p(geom["nbr"]), _p(geom["nbar"]), D, _p(omega), _p(inflow), _p(level),
                              _p(lagged)), "graph_lag")
    return inflow, level, lagged


class ProblemHex:
    """One transport problem on trilinear hexahedra on the oracle."""

    NB = NB

    def __init__(self, cfg, omega=None, w=None, S1=None, psi_in=None, src=None, lag=False):
        """lag: break cycles of the sweep graphs by lagged back edges (graph()); transport steps
        then read the previous step's psi on those faces (zero before the first step)."""
        self.lib = load(src)
        self.cfg = cfg
        self.geom = geometry(cfg["xyz"], cfg["hexes"], self.lib)
        if omega is None:
            omega, w = product_quadrature(cfg["n_polar"], cfg["n_azimuthal"])
        self.omega = np.ascontiguousarray(omega, dtype=np.float64)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        if lag:
            self.inflow, self.level, self.lag = graph(self.geom, self.omega, self.lib, lag=True)
        else:
            self.inflow, self.level = graph(self.geom, self.omega, self.lib)
            self.lag = None
        self.G = int(cfg["n_groups"])
        self.C = self.geom["vol"].shape[0]
        self.D = self.omega.shape[0]
        self.material = np.ascontiguousarray(cfg["cell_material"], dtype=np.int32)
        self.sigma_t = np.ascontiguousarray(cfg["sigma_t"], dtype=np.float64)
        self.sigma_s = np.ascontiguousarray(cfg["sigma_s"], dtype=np.float64)
        self.Q = np.ascontiguousarray(cfg["Q"], dtype=np.float64)
        if self.Q.shape != (self.C, self.G, NB):
            raise ValueError(f"Q must be [C][G][{NB}]")
        self.S1 = None if S1 is None else np.ascontiguousarray(S1, dtype=np.float64)
        self.psi_in = None if psi_in is None else np.ascontiguousarray(psi_in, dtype=np.float64)
        g = self.geom
        self._s = _ProblemHex(self.C, g["xyz"].shape[0], self.G, self.D, _p(g["xyz"]), _p(g["hexes"]),
                              _p(g["mass"]), _p(g["grad"]), _p(g["face"]), _p(g["nbar"]), _p(g["nbr"]),
                              _p(g["nbr_node"]), _p(self.omega), _p(self.w), _p(self.inflow), _p(self.level),
                              _p(self.material), _p(self.sigma_t), _p(self.S1), _p(self.psi_in), _p(self.lag), None)
        self.psi_prev = None  # lagged faces: psi [D][C][G][8] of the previous transport step
        # int_K b_i dV per cell and node: the row sums of the mass matrix (partition of unity)
        self.p_int = g["mass"].sum(axis=2)

    def source(self, phi):
        """q = (Q + sum_g' sigma_s[g'->g] phi_g') / (4 pi) at the eight nodes."""
        q = self.Q.copy()
        for m in range(self.sigma_s.shape[0]):
            idx = np.nonzero(self.material == m)[0]
            if idx.size:
                q[idx] += np.einsum("cgi,gh->chi", phi[idx], self.sigma_s[m])
        return q / FOUR_PI

    def sweep_direction(self, a, q):
        self._set_prev()
        psi = np.zeros((self.C, self.G, NB))
        q = np.ascontiguousarray(q, dtype=np.float64)
        _check(self.lib.orah_sweep_direction(C.byref(self._s), int(a), _p(q), _p(psi)), "sweep_direction")
        return psi

    def _set_prev(self):
        self._s.psi_prev = _p(self.psi_prev) if (self.lag is not None and self.psi_prev is not None) else None

    def sweep(self, q, dirs=None, threads=1, keep_psi=False):
        """phi of the listed directions (all by default); lagged faces read self.psi_prev."""
        self._set_prev()
        q = np.ascontiguousarray(q, dtype=np.float64)
        dirs = np.arange(self.D, dtype=np.int32) if dirs is None else np.ascontiguousarray(dirs, dtype=np.int32)
        phi = np.zeros((self.C, self.G, NB))
        psi = np.zeros((len(dirs), self.C, self.G, NB)) if keep_psi else None
        used = C.c_int(0)
        _check(self.lib.orah_sweep(C.byref(self._s), _p(q), len(dirs), _p(dirs), _p(phi), _p(psi), int(threads),
                                   C.byref(used)), "sweep")
        return phi, psi, used.value

    def transport_step(self, phi, threads=1):
        """One source update and sweep.  With lagged back edges the step reads, and then replaces,
        self.psi_prev (so consecutive calls are consecutive steps of source iteration)."""
        if self.lag is None:
            return self.sweep(self.source(phi), threads=threads)[0]
        phi_new, psi, _ = self.sweep(self.source(phi), threads=threads, keep_psi=True)
        self.psi_prev = psi
        return phi_new

    @staticmethod
    def residual(phi_new, phi_old, floor=1.0):
        """Largest per-group max-norm relative change (floor = 1), as for the tetrahedra."""
        gmax = np.abs(phi_new).max(axis=(0, 2))
        den = np.maximum(np.abs(phi_new), floor * gmax[None, :, None])
        diff = np.abs(phi_new - phi_old)
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.where(diff == 0.0, 0.0, diff / den)
        return float(r.max()) if r.size else 0.0

    def integrated_flux(self, phi):
        """Eq. (3) with the trilinear field: per-group int phi = sum_c sum_i (int_K b_i) phi[c][g][i];
        and the total over groups."""
        ig = np.einsum("ci,cgi->g", self.p_int, phi)
        return ig, float(ig.sum())

    def source_iterate(self, tol, max_iters, phi0=None, threads=1):
        phi = np.zeros((self.C, self.G, NB)) if phi0 is None else np.array(phi0, dtype=np.float64)
        self.psi_prev = None
        r = np.inf
        it = 0
        for it in range(1, max_iters + 1):
            new = self.transport_step(phi, threads)
            r = self.residual(new, phi)
            phi = new
            if r < tol:
                break
        return phi, it, r
