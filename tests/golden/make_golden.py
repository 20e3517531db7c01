"""Writes the stored expected values under tests/golden/ from the FP64 oracle only.

Run from the repository root:  python tests/golden/make_golden.py
The fixture is the 1-D workload (N = M = 256, eps = 1e-2, rho1 = rho2 = 1,
masses 1.0 / 1.5) after 1000 iterations of plain Sinkhorn and of TI-Sinkhorn
(H-Sinkhorn, Sec. 3) from f_0 = 0, and the dual value F_eps at each.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import uot as O                      # noqa: E402
from paper_2201_00730_gb300 import workloads as W  # noqa: E402


def build():
    p = W.config1()
    C = O.cost_matrix(p.x, p.y)
    out = {"workload": p.name, "iters": 1000}
    for name, fn in (("plain", O.sinkhorn), ("ti", O.ti_sinkhorn)):
        r = fn(C, p.a, p.b, p.eps, p.rho1, p.rho2, 1000)
        out[name] = {
            "f": [float(v) for v in r.f],
            "g": [float(v) for v in r.g],
            "value": float(O.dual_value(C, p.a, p.b, r.f, r.g, p.eps, p.rho1, p.rho2)),
            "residual": float(O.fixed_point_residual(C, p.a, p.b, r.f, r.g, p.eps, p.rho1, p.rho2)),
            "lambda": r.lam,
        }
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "config1_1000iters.json"), "w") as fh:
        json.dump(build(), fh, indent=0)
