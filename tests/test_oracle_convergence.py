"""Convergence under mesh refinement: the oracles' discretisations are consistent and reach
the accuracy order of upwind DG with degree-p elements (error O(h^(p+1)) on these meshes,
at least O(h^(p+1/2)) in general) for a smooth solution that none of the element spaces
contains, so that a dropped or wrong face, mass or streaming term, or a wrong upwind
trace, shows up as a lost order.

One direction, one group, no scattering: psi(x) = exp(k.x) + sin(m.x) / 2 solves
Omega.grad psi + sigma psi = q with q = Omega.grad psi + sigma psi, given at the element
nodes (its interpolant), and the inflow psi on the boundary."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import p2 as o2
from oracle import p3 as o3
from oracle import q1hex as oh

K = np.array([0.7, -0.4, 0.5])
MV = np.array([3.0, 2.0, -1.0])
SIGMA = 1.5


def psi_exact(x):
    return np.exp(x @ K) + 0.5 * np.sin(x @ MV)


def source(x, omega):
    grad = np.exp(x @ K)[..., None] * K + 0.5 * np.cos(x @ MV)[..., None] * MV
    return grad @ omega + SIGMA * psi_exact(x)


def _cfg(n, order):
    base = W.small_box(n=n, G=1, n_polar=2, n_az=4)
    base = dict(base, sigma_t=np.array([[SIGMA]]), sigma_s=np.zeros((1, 1, 1)))
    if order == "hex":
        return W.hex_problem(base, twist=0.25)
    return {1: lambda c: c, 2: W.order2, 3: W.order3}[order](base)


def _error(n, order, a=1):
    cfg = _cfg(n, order)
    if order == "hex":
        xyz = cfg["xyz"]
        nodes = xyz[cfg["hexes"]]  # [C][8][3]
        P = oh.ProblemHex(cfg, psi_in=psi_exact(xyz)[:, None].copy())
        vol = P.geom["vol"]
    elif order == 1:
        xyz = cfg["xyz"]
        nodes = xyz[cfg["tets"]]
        P = oracle.Problem(cfg, psi_in=psi_exact(xyz)[:, None].copy())
        vol = P.geom["vol"]
    else:
        mod = o2 if order == 2 else o3
        nodes = mod.node_coordinates(cfg["xyz"], cfg["tets"])
        cls = o2.Problem2 if order == 2 else o3.Problem3
        P = cls(cfg, psi_bc=psi_exact(nodes)[:, None, :].copy())
        vol = P.geom["vol"]
    om = P.omega[a]
    q = source(nodes, om)[:, None, :]
    psi = P.sweep_direction(a, q)[:, 0]
    err = psi - psi_exact(nodes)
    return float(np.sqrt(np.sum(vol[:, None] * err ** 2) / nodes.shape[1]))


@pytest.mark.parametrize("order,sizes,rate_min", [(1, (4, 8, 16), 1.8), (2, (2, 4, 8), 2.6), (3, (2, 4, 8), 3.5),
                                                  ("hex", (4, 8, 16), 1.8)])
def test_refinement_order(order, sizes, rate_min):
    errs = [_error(n, order) for n in sizes]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert errs[0] > errs[1] > errs[2], errs
    assert rates[-1] > rate_min, (errs, rates)
