"""Unrolled gradient of the truncated TI solve (uot_grad_unrolled) against FP64 autograd of the oracle."""
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


def rel_l2(got, ref):
    got = got.detach().double().cpu()
    ref = torch.as_tensor(ref, dtype=torch.float64)
    return ((got - ref).norm() / ref.norm()).item()


@pytest.mark.parametrize("n,m,d,T,K,eps,r1,r2", [
    (40, 31, 1, 5, 2, 0.1, 0.5, 1.3),
    (120, 97, 3, 30, 4, 0.05, 0.3, 2.0),
    (64, 80, 5, 12, 5, 0.2, 1.0, 0.7),
    (200, 150, 2, 60, 20, 0.02, 1.0, 1.0),
])
def test_unrolled_matches_autograd(U, n, m, d, T, K, eps, r1, r2):
    p = W.random_problem(n, m, d, seed=n + T, eps=eps, rho1=r1, rho2=r2, mass_a=1.2, mass_b=0.8, zero_frac=0.05)
    dev = torch.device("cuda:0")
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    spec = U.Spec(t(p.a), t(p.b), p.eps, p.rho1, p.rho2, x=t(p.x), y=t(p.y))
    val, g = U.grad_unrolled(spec, T=T, ckpt_every=K)
    rv, ga, gb, gx, gy = O.unrolled_grads(p.x, p.y, p.a, p.b, p.eps, p.rho1, p.rho2, T)
    assert abs(val.item() - rv.item()) < 1e-6 * abs(rv.item())
    for k, ref in (("a", ga), ("b", gb), ("x", gx), ("y", gy)):
        assert rel_l2(g[k], ref) < 1e-4, (k, rel_l2(g[k], ref))


def test_unrolled_equals_envelope_when_converged(U):
    """Once the truncated solve has converged, unrolled and envelope gradients coincide."""
    p = W.random_problem(150, 130, 2, seed=77, eps=0.2, rho1=0.5, rho2=0.5, mass_a=1.0, mass_b=2.0)
    dev = torch.device("cuda:0")
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    spec = U.Spec(t(p.a), t(p.b), p.eps, p.rho1, p.rho2, x=t(p.x), y=t(p.y))
    val, g = U.grad_unrolled(spec, T=200, ckpt_every=20)
    r = U.solve(spec, "ti", max_iter=200)
    e = U.grad(spec, r.f, r.g)
    for k in ("a", "b", "x", "y"):
        assert rel_l2(g[k], e[k].double().cpu()) < 1e-4, k
