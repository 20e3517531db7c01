"""Anderson extrapolation of F-, H- and G-Sinkhorn on the GPU against the FP64 oracle
(appendix, "Combining Sinkhorn with Anderson acceleration"; oracle `anderson_sinkhorn`)."""
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


def spec_of(U, p, dense=False, ordering=0):
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    if dense:
        return U.Spec(t(p.a), t(p.b), p.eps, p.rho1, p.rho2, C=t(W.dense_cost_f32(p.x, p.y)), p=p.p)
    return U.Spec(t(p.a), t(p.b), p.eps, p.rho1, p.rho2, x=t(p.x), y=t(p.y), p=p.p, ordering=ordering)


def assert_pot_close(got, ref, eps, what):
    got = got.detach().double().cpu()
    ref = torch.as_tensor(ref, dtype=torch.float64)
    err = (got - ref).abs()
    tol = 1e-4 * eps + 2 * torch.finfo(torch.float32).eps * ref.abs()
    assert bool((err <= tol).all()), f"{what}: max err {err.max().item():.3e}"


@pytest.mark.parametrize("method", ["plain", "ti", "g"])
@pytest.mark.parametrize("kind", ["tiled", "direct", "dense"])
def test_anderson_iterates_match_oracle(U, method, kind):
    """Ragged problem, K = 4: extrapolations after iterations 4, 8 and 12 (T = 14),
    after 4 only (T = 5), none (T = 4: the last iteration is never extrapolated)."""
    pr = W.random_problem(611, 437, 2, seed=21, eps=0.05, rho1=0.3, rho2=2.0, mass_a=1.3, mass_b=0.6,
                          zero_frac=0.1)
    dense = kind == "dense"
    spec = spec_of(U, pr, dense=dense, ordering={"tiled": 1, "direct": 2, "dense": 0}[kind])
    C = O._t(W.dense_cost_f32(pr.x, pr.y)) if dense else O.cost_matrix(pr.x, pr.y)
    for T in (4, 5, 14):
        r = U.solve(spec, method, max_iter=T, anderson_k=4, anderson_reg=1e-7)
        ref = O.anderson_sinkhorn(C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, T, method=method, K=4, r=1e-7)
        assert r.iters == T
        assert_pot_close(r.f, ref.f, pr.eps, f"{method} f after {T}")
        assert_pot_close(r.g, ref.g, pr.eps, f"{method} g after {T}")
        if method != "plain":
            assert abs(r.lam - ref.lam) < 1e-4 * pr.eps


@pytest.mark.parametrize("method", ["plain", "ti", "g"])
def test_anderson_converges_faster_to_the_same_fixed_point(U, method):
    """The appendix's claim on the 1-D problem (eps = 1e-2 << rho = 1), K = 4, r = 1e-7:
    fewer iterations to residual 1e-6 than the same solver without extrapolation, same
    fixed point, and the stopping test sees a plain iterate (checks every 10 iterations
    never coincide with an extrapolation)."""
    pr = W.config1()
    spec = spec_of(U, pr, ordering=2)
    base = U.solve(spec, method, max_iter=20000, tol=1e-6, check_every=10)
    acc = U.solve(spec, method, max_iter=20000, tol=1e-6, check_every=10, anderson_k=4, anderson_reg=1e-7)
    assert base.converged and acc.converged and acc.residual <= 1e-6
    assert acc.iters < base.iters
    assert (acc.f - base.f).abs().max().item() < 1e-4
    C = O.cost_matrix(pr.x, pr.y)
    res = O.fixed_point_residual(C, pr.a, pr.b, acc.f.double().cpu(), acc.g.double().cpu(), pr.eps, pr.rho1,
                                 pr.rho2).item()
    assert res < 2e-6


def test_anderson_with_residual_history_and_warm_start(U):
    """Residual history and a warm start coexist with the extrapolation; the history's
    checked entries are the returned pair's residuals."""
    pr = W.random_problem(300, 200, 1, seed=5, eps=0.05, rho1=1.0, rho2=0.5)
    spec = spec_of(U, pr, ordering=2)
    f0 = torch.linspace(-0.1, 0.1, 300, device="cuda")
    r = U.solve(spec, "ti", max_iter=400, tol=1e-7, check_every=5, history=True, f0=f0, anderson_k=3)
    assert r.converged
    h = r.history.cpu()
    assert abs(h[r.iters].item() - r.residual) <= 1e-12 + 1e-6 * r.residual
    C = O.cost_matrix(pr.x, pr.y)
    res = O.fixed_point_residual(C, pr.a, pr.b, r.f.double().cpu(), r.g.double().cpu(), pr.eps, pr.rho1,
                                 pr.rho2).item()
    assert abs(res - r.residual) <= 1e-4 * pr.eps + 1e-3 * res
