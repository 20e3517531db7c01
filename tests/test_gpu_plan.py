"""Plans (uot_plan_create / uot_plan_solve): the whole solve enqueued with no host
synchronisation, its loop a conditional while node of a CUDA graph, the stopping
rule evaluated on the device.  Against the host-driven entry points (same kernels)
and the FP64 oracle; captured into a caller's CUDA graph and replayed."""
import ctypes as C

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


def spec_of(U, p, ordering=0, dense=False):
    dev = torch.device("cuda:0")
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    if dense:
        return U.Spec(t(p.a), t(p.b), p.eps, p.rho1, p.rho2, C=t(W.dense_cost_f32(p.x, p.y)))
    return U.Spec(t(p.a), t(p.b), p.eps, p.rho1, p.rho2, x=t(p.x), y=t(p.y), ordering=ordering)


def pot_tol(eps, ref):
    return 1e-4 * eps + 2.0 * 2.0 ** -23 * ref.abs()


def same(got, ref, eps):
    got, ref = got.double().cpu(), ref.double().cpu()
    return bool(((got - ref).abs() <= pot_tol(eps, ref)).all()), (got - ref).abs().max().item()


CASES = {
    "tiled_3d": (lambda: W.random_problem(3000, 2600, 3, seed=5, eps=2e-2, rho1=0.7, rho2=2.0, mass_b=0.8), 1, False),
    "tiled_2d": (lambda: W.random_problem(3000, 2600, 2, seed=6, eps=2e-2, rho1=0.7, rho2=2.0, mass_b=0.8), 1, False),
    "direct": (lambda: W.random_problem(1200, 900, 3, seed=7, eps=5e-2, rho1=0.5, rho2=1.5), 2, False),
    "small": (lambda: W.random_problem(300, 257, 1, seed=8, eps=1e-2, rho1=1.0, rho2=0.3), 0, False),
    "dense": (lambda: W.random_problem(700, 1029, 2, seed=9, eps=5e-2, rho1=2.0, rho2=0.4), 0, True),
}


@pytest.mark.parametrize("method", ["ti", "plain", "g"])
@pytest.mark.parametrize("kind", list(CASES))
def test_plan_matches_host_driven_solve(U, kind, method):
    """Same iterate count, residual, lambda and potentials as the host-driven solve, both when the
    tolerance stops the loop and when max_iter does (status UOT_NOT_CONVERGED in the device result)."""
    mk, ordering, dense = CASES[kind]
    p = mk()
    spec = spec_of(U, p, ordering, dense)
    for max_iter, tol in ((3000, 1e-6), (37, 1e-9)):
        ref = U.solve(spec, method, max_iter=max_iter, tol=tol, check_every=5)
        plan = U.Plan(spec, method, max_iter=max_iter, tol=tol, check_every=5)
        plan.solve()
        r = plan.result()
        assert r.iters == ref.iters and bool(r.converged) == ref.converged, (r.iters, ref.iters)
        assert r.status == ref.status, (r.status, ref.status)
        assert abs(r.residual - ref.residual) <= 1e-12 + 1e-6 * ref.residual
        assert abs(r.lambda_ - ref.lam) <= 1e-12 + 1e-9 * abs(ref.lam)
        for got, want in ((plan.f, ref.f), (plan.g, ref.g)):
            ok, e = same(got, want, p.eps)
            assert ok, (kind, method, max_iter, e)
        plan.close()


def test_plan_solve_against_oracle_with_history(U):
    """TI through a plan on the tensor-core tiled path: T iterations (tol = 0) against the oracle,
    and the residual history written on the device equals the host-driven one."""
    p = W.random_problem(2100, 1700, 3, seed=12, eps=2e-2, rho1=0.6, rho2=1.8, mass_b=1.4)
    spec = spec_of(U, p, ordering=1)
    T = 40
    plan = U.Plan(spec, "ti", max_iter=T, tol=0.0, history=True)
    plan.solve()
    r = plan.result()
    assert r.iters == T
    ref = O.ti_sinkhorn(O.cost_matrix(p.x, p.y), p.a, p.b, p.eps, p.rho1, p.rho2, T)
    for got, want in ((plan.f, ref.f), (plan.g, ref.g)):
        ok, e = same(got, want, p.eps)
        assert ok, e
    host = U.solve(spec, "ti", max_iter=T, tol=0.0, history=True)
    hp, hh = plan.history[1:T + 1].double().cpu(), host.history[1:T + 1].double().cpu()
    assert bool(((hp - hh).abs() <= 1e-6 * hh.abs() + 1e-12).all())
    plan.close()


def test_plan_captured_in_a_cuda_graph_and_replayed(U):
    """A solve enqueued while the caller captures a CUDA graph becomes part of that graph: replaying
    it solves again (no host involvement), and after the weights change in place a replay gives the
    host-driven solution of the new problem."""
    p = W.random_problem(2500, 2300, 3, seed=13, eps=2e-2, rho1=1.0, rho2=1.0, mass_b=1.3)
    spec = spec_of(U, p, ordering=1)
    plan = U.Plan(spec, "ti", max_iter=5000, tol=1e-6, check_every=10)
    plan.solve()  # warm-up outside the capture (library-side graph)
    torch.cuda.synchronize()
    G = torch.cuda.CUDAGraph()
    with torch.cuda.graph(G):
        plan.solve()
    plan.f.zero_()
    plan.g.zero_()
    G.replay()
    r = plan.result()
    ref = U.solve(spec, "ti", max_iter=5000, tol=1e-6, check_every=10)
    assert r.iters == ref.iters and r.converged
    for got, want in ((plan.f, ref.f), (plan.g, ref.g)):
        ok, e = same(got, want, p.eps)
        assert ok, e
    # new weights in the same buffers: the replayed graph solves the new problem
    rng = np.random.default_rng(2)
    spec.a.copy_(torch.from_numpy((rng.exponential(1.0, p.n) / p.n).astype(np.float32)))
    spec.b.copy_(torch.from_numpy((rng.exponential(1.0, p.m) * 1.5 / p.m).astype(np.float32)))
    G.replay()
    r2 = plan.result()
    ref2 = U.solve(spec, "ti", max_iter=5000, tol=1e-6, check_every=10)
    assert r2.iters == ref2.iters and r2.converged
    for got, want in ((plan.f, ref2.f), (plan.g, ref2.g)):
        ok, e = same(got, want, p.eps)
        assert ok, e
    del G
    plan.close()
