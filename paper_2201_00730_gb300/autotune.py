"""Autotuner for the launch shapes of the sweeps.

For each tuning workload it times a short solve with every allowed value of the
knobs that govern that workload's sweeps (one knob at a time, keeping the best
value of the knobs before it), keeps a value only if its potentials agree with
those of the built-in shape (max |diff| <= 1e-4 eps + 4 ulp, the potentials'
tolerance against the FP64 oracle) and it is at least 2 % faster, and records the
winners keyed by (knob, dimension, size bucket floor(log2(N M))).  The result is
a JSON cache that `load` (or the library itself, through UOT_TUNE_FILE at plan
creation) applies; the shapes only change speed, never results beyond rounding.

    python -m paper_2201_00730_gb300.autotune [--out FILE] [--quick]

The library's own table of knobs and allowed values is the authority; KNOBS
mirrors it so that the tuner knows what to try.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import uot as U
from . import workloads as W

KNOBS = {
    "tile.rows": (2, 4),
    "tile.cta_cost": (5, 10, 15, 25, 40),
    "tile.waves": (1, 2, 3, 4),
    "points.rows": (1, 2, 4),
    "points.resident": (2, 3, 4, 6),
    "dense.row_chunk": (2048, 4096, 8192),
    "dense.col_ctas": (2, 4, 8),
    "batch.ctas_per_sm": (1, 2, 3, 4),
}

# knobs of each path, in the order they are tuned
PATH_KNOBS = {
    "tiled": ("tile.rows", "tile.waves", "tile.cta_cost"),
    "direct": ("points.rows", "points.resident"),
    "dense": ("dense.row_chunk", "dense.col_ctas"),
}

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")


def _device_key(dev) -> dict:
    p = torch.cuda.get_device_properties(dev)
    return {"device": p.name, "sm_count": int(p.multi_processor_count)}


def _spec(pr, dev, path):
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    if path == "dense":
        Cm = W.dense_cost_f32_device(pr.x, pr.y, dev)
        return U.Spec(t(pr.a), t(pr.b), pr.eps, pr.rho1, pr.rho2, C=Cm)
    return U.Spec(t(pr.a), t(pr.b), pr.eps, pr.rho1, pr.rho2, x=t(pr.x), y=t(pr.y),
                  ordering=1 if path == "tiled" else 2)


def _timed_solve(spec, iters, reps):
    """Median seconds of a `iters`-iteration TI solve (fresh workspace: it is sized
    for the current table), and the potentials of the last run."""
    ws = spec.workspace()
    r = U.solve(spec, "ti", max_iter=iters, ws=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        e0.record()
        r = U.solve(spec, "ti", max_iter=iters, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    return float(np.median(ts)), r


def _close(a, b, eps) -> bool:
    a, b = a.double(), b.double()
    return bool(((a - b).abs() <= 1e-4 * eps + 4 * 2.0 ** -23 * b.abs()).all())


def _agree(r, ref, eps) -> bool:
    return _close(r.f, ref.f, eps) and _close(r.g, ref.g, eps)


def tune_problem(pr, path: str, dev="cuda:0", iters: int = 20, reps: int = 3, log=print) -> list[dict]:
    """Tunes the knobs of `path` ('tiled', 'direct' or 'dense') on problem pr; returns the
    entries (knob, dim, bucket, value) that beat the built-in shape."""
    dev = torch.device(dev)
    spec = _spec(pr, dev, path)
    dim = -1 if path == "dense" else int(pr.x.shape[1])
    bucket = U.tune_bucket(int(pr.n) * int(pr.m))
    knobs = PATH_KNOBS[path]
    for k in knobs:
        U.tune_set(k, 0, dim, bucket)
    t_ref, ref = _timed_solve(spec, iters, reps)
    best_t = t_ref
    out = []
    for k in knobs:
        chosen = 0
        for v in KNOBS[k]:
            U.tune_set(k, v, dim, bucket)
            t, r = _timed_solve(spec, iters, reps)
            ok = _agree(r, ref, pr.eps)
            log(f"  {path} n={pr.n} m={pr.m} dim={dim} bucket={bucket} {k}={v}: {t * 1e3:.3f} ms"
                f"{'' if ok else ' (results differ: rejected)'}")
            if ok and t < 0.98 * best_t:
                best_t, chosen = t, v
        U.tune_set(k, chosen, dim, bucket)
        if chosen:
            out.append({"knob": k, "dim": dim, "bucket": bucket, "value": int(chosen)})
    log(f"  {path} n={pr.n}: built-in {t_ref * 1e3:.3f} ms, tuned {best_t * 1e3:.3f} ms")
    return out


def tune_batched(problems, dev="cuda:0", iters: int = 50, reps: int = 3, log=print) -> list[dict]:
    """Tunes the persistent grid of the batched solver."""
    U.tune_set("batch.ctas_per_sm", 0)

    def run():
        ts = []
        out = None
        for _ in range(reps + 1):
            out = U.solve_batched(problems, "ti", max_iter=iters, tol=0.0, device=dev, timing=True)
            ts.append(out.device_s)
        return float(np.median(ts[1:])), out

    t_ref, ref = run()
    best_t, chosen = t_ref, 0
    for v in KNOBS["batch.ctas_per_sm"]:
        U.tune_set("batch.ctas_per_sm", v)
        t, r = run()
        ok = all(_close(a, b, p.eps) and _close(c, d, p.eps)
                 for a, b, c, d, p in zip(r.f, ref.f, r.g, ref.g, problems))
        log(f"  batched count={len(problems)} batch.ctas_per_sm={v}: {t * 1e3:.3f} ms"
            f"{'' if ok else ' (results differ: rejected)'}")
        if ok and t < 0.98 * best_t:
            best_t, chosen = t, v
    U.tune_set("batch.ctas_per_sm", chosen)
    return [{"knob": "batch.ctas_per_sm", "dim": -1, "bucket": -1, "value": int(chosen)}] if chosen else []


def default_workloads(quick: bool = False):
    """The workloads tuned by default: the 3-D clouds of the headline problem at a
    few sizes on the tiled and direct paths, a dense cost, a ragged batch."""
    sizes = (4096, 20000) if quick else (4096, 20000, 65536)
    items = []
    for n in sizes:
        items.append(("tiled", W.config2(1.0, n=n)))
    items.append(("direct", W.random_problem(8192, 8192, 3, seed=41, eps=1e-2)))
    items.append(("dense", W.random_problem(4096, 6144, 2, seed=42, eps=5e-2)))
    if not quick:
        items.append(("dense", W.config2(1.0)))  # the 1.6 GB cost of the headline problem
    return items


def run(path: str = CACHE, dev="cuda:0", quick: bool = False, log=print) -> dict:
    """Tunes the default workloads and writes the cache; returns its content."""
    dev = torch.device(dev)
    U.tune_clear()
    entries = []
    for kind, pr in default_workloads(quick):
        entries += tune_problem(pr, kind, dev, log=log)
    probs = W.config4(count=256 if quick else 1024)
    entries += tune_batched(probs, dev, log=log)
    cache = dict(_device_key(dev), created=time.strftime("%Y-%m-%dT%H:%M:%S"), entries=entries)
    with open(path, "w") as fh:
        json.dump(cache, fh, indent=1)
    return cache


def load(path: str = CACHE, dev="cuda:0", check_device: bool = True) -> bool:
    """Applies a cache written by `run` (only on the device it was measured on,
    unless check_device is False); returns whether it was applied."""
    if not os.path.exists(path):
        return False
    with open(path) as fh:
        cache = json.load(fh)
    if check_device:
        if not torch.cuda.is_available():
            return False
        key = _device_key(torch.device(dev))
        if cache.get("device") != key["device"] or cache.get("sm_count") != key["sm_count"]:
            return False
    U.tune_load(path)
    return True


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default=CACHE)
    ap.add_argument("--quick", action="store_true")
    args = ap.parse_args()
    cache = run(args.out, quick=args.quick)
    print(json.dumps(cache, indent=1))


if __name__ == "__main__":
    main()
