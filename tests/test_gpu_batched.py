"""Batched ragged solver (uot_sinkhorn_batched) against the FP64 oracle and the single-problem path."""
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


def ragged(count, seed, lo=1, hi=300, eps=(0.02, 0.2), rho=(0.2, 5.0)):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n, m = int(rng.integers(lo, hi)), int(rng.integers(lo, hi))
        d = int(rng.integers(1, 4))
        p = W.random_problem(n, m, d, seed=seed * 1000 + k, eps=float(np.exp(rng.uniform(*np.log(eps)))),
                             rho1=float(np.exp(rng.uniform(*np.log(rho)))),
                             rho2=float(np.exp(rng.uniform(*np.log(rho)))),
                             mass_a=float(rng.uniform(0.5, 2)), mass_b=float(rng.uniform(0.5, 2)),
                             zero_frac=0.1 if k % 5 == 0 else 0.0)
        out.append(p)
    return out


def close(got, ref, eps):
    ref = torch.as_tensor(ref, dtype=torch.float64)
    err = (got.double().cpu() - ref).abs()
    return bool((err <= 1e-4 * eps + 2 * 2.0 ** -23 * ref.abs()).all()), err.max().item()


@pytest.mark.parametrize("method", ["ti", "plain"])
def test_batched_iterates_match_oracle(U, method):
    probs = ragged(24, seed=3)
    T = 40
    r = U.solve_batched(probs, method, max_iter=T, tol=0.0, check_every=10)
    fn = O.ti_sinkhorn if method == "ti" else O.sinkhorn
    for k, p in enumerate(probs):
        C = O.cost_matrix(p.x, p.y)
        ref = fn(C, p.a, p.b, p.eps, p.rho1, p.rho2, T)
        assert r.iters[k] == T
        ok, e = close(r.f[k], ref.f, p.eps)
        assert ok, (k, "f", e, p.name)
        ok, e = close(r.g[k], ref.g, p.eps)
        assert ok, (k, "g", e, p.name)
        res_ref = O.fixed_point_residual(C, p.a, p.b, ref.f, ref.g, p.eps, p.rho1, p.rho2).item()
        assert abs(r.residual[k] - res_ref) <= 1e-4 * p.eps + 1e-3 * res_ref
        if method == "ti":
            assert abs(r.lam[k] - ref.lam) < 1e-4 * p.eps


def test_batched_matches_single_solves_with_tolerance(U):
    probs = ragged(16, seed=5, lo=20, hi=700)
    r = U.solve_batched(probs, "ti", max_iter=5000, tol=1e-5, check_every=5)
    for k, p in enumerate(probs):
        dev = torch.device("cuda:0")
        t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
        spec = U.Spec(t(p.a), t(p.b), p.eps, p.rho1, p.rho2, x=t(p.x), y=t(p.y), ordering=2)
        s = U.solve(spec, "ti", max_iter=5000, tol=1e-5, check_every=5)
        assert r.converged[k] and s.converged
        assert abs(r.iters[k] - s.iters) <= 5, (k, r.iters[k], s.iters)
        assert (r.f[k] - s.f).abs().max().item() < 1e-4 * p.eps + 1e-5


def test_batched_config4_sample(U):
    probs = W.config4(count=48, lo=64, hi=1024)
    r = U.solve_batched(probs, "ti", max_iter=20000, tol=1e-6, check_every=10)
    assert all(r.converged), [k for k, c in enumerate(r.converged) if not c]
    # spot-check the fixed point of a few problems against the FP64 oracle's fixed-point equations
    for k in (0, 7, 23, 47):
        p = probs[k]
        C = O.cost_matrix(p.x, p.y)
        f, g = r.f[k].double().cpu(), r.g[k].double().cpu()
        rr = O.fixed_point_residual(C, p.a, p.b, f, g, p.eps, p.rho1, p.rho2).item()
        assert rr < 1e-6 + 1e-4 * p.eps + 4e-7, (k, rr)


def test_batched_reports_bad_weights(U):
    probs = ragged(4, seed=9)
    probs[2].a = probs[2].a.copy()
    probs[2].a[0] = -1.0
    with pytest.raises(U.UOTError) as ei:
        U.solve_batched(probs, "ti", max_iter=5)
    assert ei.value.status == 4


def test_batched_graph_replay_matches_plain_launches(U):
    """The CUDA-graph path (a non-default stream: each chunk of check_every iterations captured once
    and replayed) against the plain-launch path (legacy default stream), on the same batch: same
    iteration counts, same potentials within the potentials' tolerance; also under a caller's
    torch.cuda.Stream."""
    probs = W.config4(count=40, lo=64, hi=2048, seed=77)
    rg = U.solve_batched(probs, "ti", max_iter=20000, tol=1e-6, check_every=10, graph=True)
    rp = U.solve_batched(probs, "ti", max_iter=20000, tol=1e-6, check_every=10, graph=False)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        rs = U.solve_batched(probs, "ti", max_iter=20000, tol=1e-6, check_every=10)
    torch.cuda.synchronize()
    assert all(rg.converged) and all(rp.converged) and all(rs.converged)
    for k, p in enumerate(probs):
        assert rg.iters[k] == rp.iters[k] == rs.iters[k], (k, rg.iters[k], rp.iters[k], rs.iters[k])
        for other in (rp, rs):
            ok, e = close(rg.f[k], other.f[k].double().cpu(), p.eps)
            assert ok, (k, "f", e)
            ok, e = close(rg.g[k], other.g[k].double().cpu(), p.eps)
            assert ok, (k, "g", e)
