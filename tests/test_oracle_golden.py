"""The stored 1-D fixture is reproduced by the oracle (guards the oracle against drift)."""
import json
import os

import torch

from oracle import uot as O
from paper_2201_00730_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "config1_1000iters.json")


def test_golden_config1_reproduced():
    d = json.load(open(GOLDEN))
    p = W.config1()
    C = O.cost_matrix(p.x, p.y)
    for name, fn in (("plain", O.sinkhorn), ("ti", O.ti_sinkhorn)):
        r = fn(C, p.a, p.b, p.eps, p.rho1, p.rho2, d["iters"])
        assert (r.f - torch.tensor(d[name]["f"], dtype=torch.float64)).abs().max() < 1e-13
        assert (r.g - torch.tensor(d[name]["g"], dtype=torch.float64)).abs().max() < 1e-13
    # both algorithms reach the same fixed point (T3) on this workload; plain Sinkhorn's
    # residual 8.8e-12 at rate ~0.98 per iteration leaves an error of ~residual / 0.02
    assert d["plain"]["residual"] < 1e-11 and d["ti"]["residual"] < 1e-15
    assert max(abs(u - v) for u, v in zip(d["plain"]["f"], d["ti"]["f"])) < 1e-9
    assert abs(d["plain"]["value"] - d["ti"]["value"]) < 1e-12
