"""Plain FP64 CPU oracle for the unstructured S_N transport sweep.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
bench's CPU-baseline / reference leg may import this package.  It shares no
code with the CUDA library (`paper_2510_11513_gb300`) and never imports it.

The C part (`tf_oracle.c`) holds quadrature, geometry, face classification,
t-levels and the per-direction sweep; this module adds, in plain numpy, the
scattering-source update (right-hand side of Eq. (1) with isotropic
scattering), the stopping test, the integrated flux of Eq. (3) and the
source-iteration loop.

Source convention: Q[c][g][i] is the total isotropic volumetric source at node
i, so the angular source per steradian is (Q + sum_g' sigma_s[g'->g] phi_g')/(4 pi).
"""
from __future__ import annotations

import ctypes as C
import hashlib
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tf_oracle.c")
BUILD = os.path.join(HERE, "_build")

ORA_OK, ORA_ERR_ARG, ORA_ERR_MESH, ORA_ERR_CYCLE = 0, 1, 2, 3
FOUR_PI = 4.0 * np.pi

_lock = threading.Lock()
_libs: dict = {}


def build(defines=(), openmp=True, src=None) -> str:
    """Compile tf_oracle.c (or `src`, a modified copy that a planted-mistake test
    writes) with gcc -O2 -ffp-contract=off; returns the .so path."""
    src = src or SRC
    os.makedirs(BUILD, exist_ok=True)
    flags = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
             "-D_GNU_SOURCE"]
    if openmp:
        flags.append("-fopenmp")
    flags += [f"-D{d}" for d in defines]
    with open(src, "rb") as f:
        key = hashlib.sha1(f.read() + " ".join(flags).encode()).hexdigest()[:12]
    out = os.path.join(BUILD, f"libtforacle_{key}.so")
    if not os.path.exists(out):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *flags, src, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


class _Problem(C.Structure):
    _fields_ = [
        ("nc", C.c_int64), ("nv", C.c_int64), ("G", C.c_int32), ("D", C.c_int32),
        ("xyz", C.c_void_p), ("tets", C.c_void_p), ("vol", C.c_void_p), ("grad", C.c_void_p),
        ("normal", C.c_void_p), ("nbr", C.c_void_p), ("nbr_node", C.c_void_p),
        ("omega", C.c_void_p), ("w", C.c_void_p), ("inflow", C.c_void_p), ("level", C.c_void_p),
        ("material", C.c_void_p), ("sigma_t", C.c_void_p), ("S1", C.c_void_p), ("psi_in", C.c_void_p),
    ]


def load(defines=(), src=None):
    key = (tuple(defines), src)
    with _lock:
        if key not in _libs:
            lib = C.CDLL(build(defines, src=src))
            vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
            lib.ora_gauss_legendre.argtypes = [i32, vp, vp]
            lib.ora_product_quadrature.argtypes = [i32, i32, vp, vp]
            lib.ora_geometry.argtypes = [i64, vp, i64, vp, vp, vp, vp, vp, vp]
            lib.ora_graph.argtypes = [i64, vp, vp, i32, vp, vp, vp]
            lib.ora_sweep_direction.argtypes = [C.POINTER(_Problem), i32, vp, vp]
            lib.ora_sweep.argtypes = [C.POINTER(_Problem), vp, i32, vp, vp, vp, i32, C.POINTER(C.c_int)]
            _libs[key] = lib
        return _libs[key]


def _p(a):
    return None if a is None else a.ctypes.data


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what}: status {code}")
        self.code = code


def _check(code, what):
    if code != ORA_OK:
        raise OracleError(code, what)


# ----------------------------------------------------------------- quadrature
def gauss_legendre(n, lib=None):
    lib = lib or load()
    x = np.zeros(n)
    w = np.zeros(n)
    _check(lib.ora_gauss_legendre(n, _p(x), _p(w)), "gauss_legendre")
    return x, w


def product_quadrature(n_polar, n_az, lib=None):
    """Omega [D][3] and w [D] of the product rule (sum w = 4 pi)."""
    lib = lib or load()
    D = n_polar * n_az
    om = np.zeros((D, 3))
    w = np.zeros(D)
    _check(lib.ora_product_quadrature(n_polar, n_az, _p(om), _p(w)), "product_quadrature")
    return om, w


# ------------------------------------------------------------------- geometry
def geometry(xyz, tets, lib=None):
    lib = lib or load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    nc, nv = tets.shape[0], xyz.shape[0]
    g = dict(vol=np.zeros(nc), grad=np.zeros((nc, 4, 3)), normal=np.zeros((nc, 4, 3)),
             nbr=np.zeros((nc, 4), dtype=np.int32), nbr_node=np.zeros((nc, 4, 4), dtype=np.int32))
    _check(lib.ora_geometry(nv, _p(xyz), nc, _p(tets), _p(g["vol"]), _p(g["grad"]), _p(g["normal"]),
                            _p(g["nbr"]), _p(g["nbr_node"])), "geometry")
    g["xyz"], g["tets"] = xyz, tets
    return g


def graph(geom, omega, lib=None):
    """Inflow-face bitmask [D][C] (uint8) and t-level [D][C] (int32)."""
    lib = lib or load()
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    D, nc = omega.shape[0], geom["vol"].shape[0]
    inflow = np.zeros((D, nc), dtype=np.uint8)
    level = np.zeros((D, nc), dtype=np.int32)
    _check(lib.ora_graph(nc, _p(geom["nbr"]), _p(geom["normal"]), D, _p(omega), _p(inflow), _p(level)),
           "graph")
    return inflow, level


# -------------------------------------------------------------------- problem
class Problem:
    """One transport problem on the oracle: geometry, graph, cross sections."""

    def __init__(self, cfg, omega=None, w=None, S1=None, psi_in=None, defines=(), lib=None):
        self.lib = lib or load(defines)
        self.cfg = cfg
        self.geom = geometry(cfg["xyz"], cfg["tets"], self.lib)
        if omega is None:
            omega, w = product_quadrature(cfg["n_polar"], cfg["n_azimuthal"], self.lib)
        self.omega = np.ascontiguousarray(omega, dtype=np.float64)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.inflow, self.level = graph(self.geom, self.omega, self.lib)
        self.G = int(cfg["n_groups"])
        self.C = self.geom["vol"].shape[0]
        self.D = self.omega.shape[0]
        self.material = np.ascontiguousarray(cfg["cell_material"], dtype=np.int32)
        self.sigma_t = np.ascontiguousarray(cfg["sigma_t"], dtype=np.float64)
        self.sigma_s = np.ascontiguousarray(cfg["sigma_s"], dtype=np.float64)
        self.Q = np.ascontiguousarray(cfg["Q"], dtype=np.float64)
        self.S1 = None if S1 is None else np.ascontiguousarray(S1, dtype=np.float64)
        self.psi_in = None if psi_in is None else np.ascontiguousarray(psi_in, dtype=np.float64)
        g = self.geom
        self._s = _Problem(self.C, g["xyz"].shape[0], self.G, self.D, _p(g["xyz"]), _p(g["tets"]),
                           _p(g["vol"]), _p(g["grad"]), _p(g["normal"]), _p(g["nbr"]), _p(g["nbr_node"]),
                           _p(self.omega), _p(self.w), _p(self.inflow), _p(self.level), _p(self.material),
                           _p(self.sigma_t), _p(self.S1), _p(self.psi_in))

    # ------------------------------------------------------------ pieces
    def source(self, phi):
        """Angular source per steradian q = (Q + sum_g' sigma_s[g'->g] phi_g') / (4 pi), [C][G][4]."""
        q = self.Q.copy()
        for m in range(self.sigma_s.shape[0]):
            idx = np.nonzero(self.material == m)[0]
            if idx.size:
                q[idx] += np.einsum("cgi,gh->chi", phi[idx], self.sigma_s[m])
        return q / FOUR_PI

    def sweep_direction(self, a, q):
        psi = np.zeros((self.C, self.G, 4))
        q = np.ascontiguousarray(q, dtype=np.float64)
        _check(self.lib.ora_sweep_direction(C.byref(self._s), int(a), _p(q), _p(psi)), "sweep_direction")
        return psi

    def sweep(self, q, dirs=None, threads=1, keep_psi=False):
        """phi = sum_a w_a psi_a over `dirs` (default all); returns (phi, psi or None, threads used)."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        dirs = np.arange(self.D, dtype=np.int32) if dirs is None else np.ascontiguousarray(dirs, dtype=np.int32)
        phi = np.zeros((self.C, self.G, 4))
        psi = np.zeros((len(dirs), self.C, self.G, 4)) if keep_psi else None
        used = C.c_int(0)
        _check(self.lib.ora_sweep(C.byref(self._s), _p(q), len(dirs), _p(dirs), _p(phi), _p(psi),
                                  int(threads), C.byref(used)), "sweep")
        return phi, psi, used.value

    def transport_step(self, phi, threads=1):
        """One source update followed by one sweep of every direction."""
        return self.sweep(self.source(phi), threads=threads)[0]

    @staticmethod
    def residual(phi_new, phi_old, floor=1.0):
        """Stopping test: max over (cell, group, node) of |phi_new - phi_old| /
        max(|phi_new|, floor * max over (cell, node) of |phi_new| in that group).
        floor = 1 (default) is the largest per-group max-norm relative change;
        a small floor (1e-10) gives the pointwise relative change."""
        gmax = np.abs(phi_new).max(axis=(0, 2))  # per group
        den = np.maximum(np.abs(phi_new), floor * gmax[None, :, None])
        diff = np.abs(phi_new - phi_old)
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.where(diff == 0.0, 0.0, diff / den)
        return float(r.max()) if r.size else 0.0

    def integrated_flux(self, phi):
        """Eq. (3): per-group spatial integral sum_c (V_c/4) sum_i phi[c][g][i], and the plain
        nodal sum sum_c sum_i phi[c][g][i] as the equation writes it; totals over groups."""
        vol = self.geom["vol"]
        ig = np.einsum("c,cgi->g", vol / 4.0, phi)
        plain = phi.sum(axis=(0, 2))
        return ig, float(ig.sum()), plain, float(plain.sum())

    def source_iterate(self, tol, max_iters, phi0=None, threads=1, callback=None, floor=1.0):
        """Group-Jacobi source iteration from phi0 (zeros by default) until the
        stopping test is below tol or max_iters sweeps were done."""
        phi = np.zeros((self.C, self.G, 4)) if phi0 is None else np.array(phi0, dtype=np.float64)
        r = np.inf
        it = 0
        for it in range(1, max_iters + 1):
            new = self.transport_step(phi, threads)
            r = self.residual(new, phi, floor)
            phi = new
            if callback:
                callback(it, r, phi)
            if r < tol:
                break
        return phi, it, r
