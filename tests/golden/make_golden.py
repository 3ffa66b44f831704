"""Writes tests/golden/oracle_regression.json from the CPU oracle alone (no library
code): reference values that later changes to the oracle or the library must keep.

  * the 8^3-hex box (3,072 tets, 32 directions, 4 groups, one material, downscatter,
    source in the central hexes): source iteration to the max-norm test 1e-10, the
    iteration count and the integrated flux of Eq. (3) per group;
  * one transport step from a seeded flux for the second- and third-order elements on
    a 2^3-hex box: the integrated flux per group and a nodal checksum;
  * the same 8^3 box as trilinear hexahedra (orthogonal grid twisted by 0.25 rad):
    source iteration to 1e-10, the iteration count and the integrated flux per group.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from oracle import p2 as o2  # noqa: E402
from oracle import p3 as o3  # noqa: E402
from oracle import q1hex as oh  # noqa: E402


def main():
    out = {"written_by": "tests/golden/make_golden.py (oracle only)"}
    cfg = W.small_box()
    P = oracle.Problem(cfg)
    phi, it, r = P.source_iterate(1e-10, 1000, threads=8)
    ig, tot, plain, ptot = P.integrated_flux(phi)
    out["small_box"] = {"workload": cfg["name"], "tol": 1e-10, "iterations": it, "residual": r,
                        "integrated_flux": ig.tolist(), "integrated_total": tot, "nodal_sum": plain.tolist()}
    for order, mod, maker, cls, nb in ((2, o2, W.order2, o2.Problem2, 10), (3, o3, W.order3, o3.Problem3, 20)):
        c = maker(W.small_box(n=2, G=3, n_polar=2, n_az=8))
        Q = cls(c)
        phi0 = np.random.default_rng(2510115130 + order).uniform(0.0, 1.0, (Q.C, 3, nb))
        step = Q.transport_step(phi0, threads=4)
        ig, tot = Q.integrated_flux(step)
        out[f"order{order}_step"] = {"seed": 2510115130 + order, "integrated_flux": ig.tolist(),
                                     "checksum": float(np.sum(step * np.arange(1, step.size + 1).reshape(step.shape)
                                                              / step.size))}
    hcfg = W.hex_problem(W.small_box(), twist=0.25)
    Ph = oh.ProblemHex(hcfg)
    phi, it, r = Ph.source_iterate(1e-10, 1000, threads=8)
    ig, tot = Ph.integrated_flux(phi)
    out["hex_small_box"] = {"workload": hcfg["name"], "twist": 0.25, "tol": 1e-10, "iterations": it, "residual": r,
                            "integrated_flux": ig.tolist(), "integrated_total": tot}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
