"""Every allowed value of every tuning knob gives the oracle's iterates (the shapes
only move work between CTAs), the workspace size does not depend on the table,
and the autotuner produces a cache that loads and keeps the results."""
import json

import numpy as np
import pytest
import torch

from oracle import uot as O
from paper_2201_00730_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    from paper_2201_00730_gb300 import build, uot
    build.build()
    return uot


@pytest.fixture(autouse=True)
def clean_table(U):
    U.tune_clear()
    yield
    U.tune_clear()


def dev_t(v):
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda:0")


def close(got, ref, eps):
    got, ref = got.double().cpu(), ref.double().cpu()
    err = (got - ref).abs()
    return bool((err <= 1e-4 * eps + 2 * 2.0 ** -23 * ref.abs()).all()), err.max().item()


# (path, knob, problem, ordering or "dense")
CASES = [
    ("tiled", "tile.rows", (611, 437, 2), 1),
    ("tiled", "tile.cta_cost", (5000, 3000, 3), 1),
    ("tiled", "tile.waves", (5000, 3000, 3), 1),
    ("direct", "points.rows", (2100, 1300, 3), 2),
    ("direct", "points.resident", (2100, 1300, 2), 2),
    ("dense", "dense.row_chunk", (700, 5000, 2), "dense"),
    ("dense", "dense.col_ctas", (900, 1100, 2), "dense"),
]


@pytest.mark.parametrize("path,knob,shape,ordering", CASES, ids=[c[1] for c in CASES])
def test_every_allowed_value_matches_oracle(U, path, knob, shape, ordering):
    from paper_2201_00730_gb300 import autotune as A
    n, m, d = shape
    pr = W.random_problem(n, m, d, seed=61, eps=0.05, rho1=0.3, rho2=2.0, mass_a=1.3, mass_b=0.6, zero_frac=0.1)
    if ordering == "dense":
        Cf = W.dense_cost_f32(pr.x, pr.y)
        spec = U.Spec(dev_t(pr.a), dev_t(pr.b), pr.eps, pr.rho1, pr.rho2, C=dev_t(Cf))
        C = O._t(Cf)
    else:
        spec = U.Spec(dev_t(pr.a), dev_t(pr.b), pr.eps, pr.rho1, pr.rho2, x=dev_t(pr.x), y=dev_t(pr.y),
                      ordering=ordering)
        C = O.cost_matrix(pr.x, pr.y)
    T = 7
    ref = O.ti_sinkhorn(C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, T)
    ws_bytes = U.workspace_size(spec)
    for v in A.KNOBS[knob]:
        U.tune_set(knob, v)
        assert U.workspace_size(spec) == ws_bytes  # sized for every allowed shape
        r = U.solve(spec, "ti", max_iter=T)
        for got, want, name in ((r.f, ref.f, "f"), (r.g, ref.g, "g")):
            ok, err = close(got, want, pr.eps)
            assert ok, f"{knob}={v}: {name} max err {err:.3e}"
        assert abs(r.lam - ref.lam) < 1e-4 * pr.eps


def test_batched_grid_values_match_default(U):
    from paper_2201_00730_gb300 import autotune as A
    probs = W.config4(count=24, lo=64, hi=600, seed=71)
    ref = U.solve_batched(probs, "ti", max_iter=30, tol=0.0)
    for v in A.KNOBS["batch.ctas_per_sm"]:
        U.tune_set("batch.ctas_per_sm", v)
        out = U.solve_batched(probs, "ti", max_iter=30, tol=0.0)
        for k, p in enumerate(probs):
            assert close(out.f[k], ref.f[k], p.eps)[0] and close(out.g[k], ref.g[k], p.eps)[0], (v, k)
    # and the default against the oracle on a few problems
    for k in (0, 7, 23):
        p = probs[k]
        o = O.ti_sinkhorn(O.cost_matrix(p.x, p.y), p.a, p.b, p.eps, p.rho1, p.rho2, 30)
        assert close(ref.f[k], o.f, p.eps)[0] and close(ref.g[k], o.g, p.eps)[0], k


def test_autotuner_cache_round_trip(U, tmp_path):
    from paper_2201_00730_gb300 import autotune as A
    pr = W.config2(1.0, n=4096)
    entries = A.tune_problem(pr, "tiled", iters=5, reps=2, log=lambda *a: None)
    path = tmp_path / "cache.json"
    key = A._device_key(torch.device("cuda:0"))
    path.write_text(json.dumps(dict(key, entries=entries)))
    U.tune_clear()
    assert A.load(str(path))
    for e in entries:
        assert U.tune_get(e["knob"], e["dim"], 4096 * 4096) == e["value"]
    # the tuned solve keeps the built-in result
    spec = A._spec(pr, torch.device("cuda:0"), "tiled")
    r1 = U.solve(spec, "ti", max_iter=20)
    U.tune_clear()
    r0 = U.solve(spec, "ti", max_iter=20)
    assert close(r1.f, r0.f, pr.eps)[0] and close(r1.g, r0.g, pr.eps)[0]
