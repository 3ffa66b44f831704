"""Plain FP64 CPU oracle for the second-order (quadratic, ten-node) upwind-DG
sweep on tetrahedra.

TEST INFRASTRUCTURE ONLY (same rules as the rest of `oracle/`).  The C part
(`tf_oracle_p2.c`) assembles every local system by quadrature and sweeps; this
module reuses the first-order oracle's geometry, face classification and
t-levels (they do not depend on the element order), and adds the source
update, stopping test, integrated flux and source iteration in numpy.

Node order per cell: the four vertices of tets[c] in their local order, then
the midpoints of the local edges (0,1) (0,2) (0,3) (1,2) (1,3) (2,3).
Arrays: Q, q, phi [C][G][10]; psi [C][G][10] per direction.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import FOUR_PI, ORA_OK, OracleError, _p, build, geometry, graph, product_quadrature
from . import load as load1

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tf_oracle_p2.c")
NB = 10
EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))

_libs: dict = {}


class _Problem2(C.Structure):
    _fields_ = [
        ("nc", C.c_int64), ("G", C.c_int32), ("D", C.c_int32),
        ("xyz", C.c_void_p), ("tets", C.c_void_p), ("vol", C.c_void_p), ("grad", C.c_void_p),
        ("normal", C.c_void_p), ("nbr", C.c_void_p), ("omega", C.c_void_p), ("w", C.c_void_p),
        ("inflow", C.c_void_p), ("level", C.c_void_p), ("material", C.c_void_p), ("sigma_t", C.c_void_p),
        ("S1", C.c_void_p), ("psi_bc", C.c_void_p),
    ]


def load(src=None):
    """The second-order oracle library (`src`: a modified copy for planted-mistake tests)."""
    key = src or SRC
    if key not in _libs:
        lib = C.CDLL(build(src=key))
        vp, i32 = C.c_void_p, C.c_int
        lib.ora2_basis_integrals.argtypes = [vp]
        lib.ora2_mass.argtypes = [vp]
        lib.ora2_sweep_direction.argtypes = [C.POINTER(_Problem2), i32, vp, vp]
        lib.ora2_sweep.argtypes = [C.POINTER(_Problem2), vp, i32, vp, vp, vp, i32, C.POINTER(C.c_int)]
        _libs[key] = lib
    return _libs[key]


def _check(code, what):
    if code != ORA_OK:
        raise OracleError(code, what)


def basis_integrals(lib=None):
    """int_K phi_i / V for the ten basis functions (quadrature)."""
    out = np.zeros(NB)
    _check((lib or load()).ora2_basis_integrals(_p(out)), "basis_integrals")
    return out


def mass_matrix(lib=None):
    """int_K phi_i phi_j / V (quadrature)."""
    out = np.zeros((NB, NB))
    _check((lib or load()).ora2_mass(_p(out)), "mass")
    return out


def node_coordinates(xyz, tets):
    """Physical coordinates of the ten nodes of every cell, [C][10][3]."""
    v = np.asarray(xyz, dtype=np.float64)[np.asarray(tets)]
    mid = np.stack([0.5 * (v[:, a] + v[:, b]) for a, b in EDGES], axis=1)
    return np.concatenate([v, mid], axis=1)


class Problem2:
    """One second-order transport problem on the oracle."""

    NB = NB

    @staticmethod
    def _load(src):
        return load(src)

    def _fn(self, name):
        return getattr(self.lib, "ora2_" + name)

    def __init__(self, cfg, omega=None, w=None, S1=None, psi_bc=None, src=None):
        NB = self.NB
        self.lib1 = load1()
        self.lib = self._load(src)
        self.cfg = cfg
        self.geom = geometry(cfg["xyz"], cfg["tets"], self.lib1)
        if omega is None:
            omega, w = product_quadrature(cfg["n_polar"], cfg["n_azimuthal"], self.lib1)
        self.omega = np.ascontiguousarray(omega, dtype=np.float64)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.inflow, self.level = graph(self.geom, self.omega, self.lib1)
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
        self.psi_bc = None if psi_bc is None else np.ascontiguousarray(psi_bc, dtype=np.float64)
        g = self.geom
        self._s = _Problem2(self.C, self.G, self.D, _p(g["xyz"]), _p(g["tets"]), _p(g["vol"]), _p(g["grad"]),
                            _p(g["normal"]), _p(g["nbr"]), _p(self.omega), _p(self.w), _p(self.inflow),
                            _p(self.level), _p(self.material), _p(self.sigma_t), _p(self.S1), _p(self.psi_bc))
        self.p_int = np.zeros(NB)
        _check(self._fn("basis_integrals")(_p(self.p_int)), "basis_integrals")

    def source(self, phi):
        """q = (Q + sum_g' sigma_s[g'->g] phi_g') / (4 pi) at the ten nodes."""
        q = self.Q.copy()
        for m in range(self.sigma_s.shape[0]):
            idx = np.nonzero(self.material == m)[0]
            if idx.size:
                q[idx] += np.einsum("cgi,gh->chi", phi[idx], self.sigma_s[m])
        return q / FOUR_PI

    def sweep_direction(self, a, q):
        psi = np.zeros((self.C, self.G, self.NB))
        q = np.ascontiguousarray(q, dtype=np.float64)
        _check(self._fn("sweep_direction")(C.byref(self._s), int(a), _p(q), _p(psi)), "sweep_direction")
        return psi

    def sweep(self, q, dirs=None, threads=1, keep_psi=False):
        q = np.ascontiguousarray(q, dtype=np.float64)
        dirs = np.arange(self.D, dtype=np.int32) if dirs is None else np.ascontiguousarray(dirs, dtype=np.int32)
        phi = np.zeros((self.C, self.G, self.NB))
        psi = np.zeros((len(dirs), self.C, self.G, self.NB)) if keep_psi else None
        used = C.c_int(0)
        _check(self._fn("sweep")(C.byref(self._s), _p(q), len(dirs), _p(dirs), _p(phi), _p(psi), int(threads),
                                 C.byref(used)), "sweep")
        return phi, psi, used.value

    def transport_step(self, phi, threads=1):
        return self.sweep(self.source(phi), threads=threads)[0]

    @staticmethod
    def residual(phi_new, phi_old, floor=1.0):
        """Largest per-group max-norm relative change (floor = 1), as for the linear element."""
        gmax = np.abs(phi_new).max(axis=(0, 2))
        den = np.maximum(np.abs(phi_new), floor * gmax[None, :, None])
        diff = np.abs(phi_new - phi_old)
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.where(diff == 0.0, 0.0, diff / den)
        return float(r.max()) if r.size else 0.0

    def integrated_flux(self, phi):
        """Eq. (3) with the quadratic field: per-group int phi = sum_c V_c sum_i p_i phi[c][g][i],
        p_i = int_K phi_i / V; and the total over groups."""
        ig = np.einsum("c,i,cgi->g", self.geom["vol"], self.p_int, phi)
        return ig, float(ig.sum())

    def source_iterate(self, tol, max_iters, phi0=None, threads=1):
        phi = np.zeros((self.C, self.G, self.NB)) if phi0 is None else np.array(phi0, dtype=np.float64)
        r = np.inf
        it = 0
        for it in range(1, max_iters + 1):
            new = self.transport_step(phi, threads)
            r = self.residual(new, phi)
            phi = new
            if r < tol:
                break
        return phi, it, r
