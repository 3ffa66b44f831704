"""Plain FP64 CPU oracle for the third-order (cubic, twenty-node) upwind-DG sweep
on tetrahedra.

TEST INFRASTRUCTURE ONLY (same rules as the rest of `oracle/`).  The C part
(`tf_oracle_p3.c`) assembles every local system by quadrature and sweeps; the
problem class is the second-order one with twenty nodes (same geometry, graph,
source update, stopping test and integrated flux).

Node order per cell: the four vertices of tets[c]; two nodes per local edge
(a,b) in the order (0,1) (0,2) (0,3) (1,2) (1,3) (2,3), first the one at
(lambda_a, lambda_b) = (2/3, 1/3), then (1/3, 2/3); the centres of the faces
opposite vertices 0..3.
Arrays: Q, q, phi [C][G][20].
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _p, build
from .p2 import EDGES, Problem2, _check, _Problem2

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tf_oracle_p3.c")
NB = 20

_libs: dict = {}


def load(src=None):
    """The third-order oracle library (`src`: a modified copy for planted-mistake tests)."""
    key = src or SRC
    if key not in _libs:
        lib = C.CDLL(build(src=key))
        vp, i32 = C.c_void_p, C.c_int
        lib.ora3_basis_integrals.argtypes = [vp]
        lib.ora3_mass.argtypes = [vp]
        lib.ora3_sweep_direction.argtypes = [C.POINTER(_Problem2), i32, vp, vp]
        lib.ora3_sweep.argtypes = [C.POINTER(_Problem2), vp, i32, vp, vp, vp, i32, C.POINTER(C.c_int)]
        _libs[key] = lib
    return _libs[key]


def basis_integrals(lib=None):
    """int_K phi_i / V for the twenty basis functions (quadrature)."""
    out = np.zeros(NB)
    _check((lib or load()).ora3_basis_integrals(_p(out)), "basis_integrals")
    return out


def mass_matrix(lib=None):
    """int_K phi_i phi_j / V (quadrature)."""
    out = np.zeros((NB, NB))
    _check((lib or load()).ora3_mass(_p(out)), "mass")
    return out


def node_coordinates(xyz, tets):
    """Physical coordinates of the twenty nodes of every cell, [C][20][3]."""
    v = np.asarray(xyz, dtype=np.float64)[np.asarray(tets)]
    edge = []
    for a, b in EDGES:
        edge.append((2.0 * v[:, a] + v[:, b]) / 3.0)
        edge.append((v[:, a] + 2.0 * v[:, b]) / 3.0)
    faces = [(v.sum(axis=1) - v[:, f]) / 3.0 for f in range(4)]
    return np.concatenate([v, np.stack(edge, axis=1), np.stack(faces, axis=1)], axis=1)


class Problem3(Problem2):
    """One third-order transport problem on the oracle."""

    NB = NB

    @staticmethod
    def _load(src):
        return load(src)

    def _fn(self, name):
        return getattr(self.lib, "ora3_" + name)
