"""Pins of the general-phi^* oracle (F- and G-Sinkhorn with the Berg entropy, Sec. 3)."""
import math

import numpy as np
import pytest
import torch

from oracle import general_phi as GP
from oracle import uot as O

scipy_opt = pytest.importorskip("scipy.optimize")
scipy_special = pytest.importorskip("scipy.special")


def problem(n, m, seed, mb=1.5):
    rng = np.random.default_rng(seed)
    x = rng.random((n, 1))
    y = rng.random((m, 1)) * 0.8 + 0.2
    a = rng.exponential(1.0, n)
    b = rng.exponential(1.0, m)
    a, b = a / a.sum(), mb * b / b.sum()
    C = O.cost_matrix(x, y)
    return C, torch.tensor(a), torch.tensor(b)


@pytest.mark.parametrize("rho,eps", [(1.0, 0.1), (0.05, 0.5), (10.0, 0.01)])
def test_aprox_kl_is_the_linear_closed_form(rho, eps):
    x = torch.linspace(-3, 3, 13, dtype=torch.float64)
    got = GP.aprox(GP.KL(rho), x, eps)
    assert torch.allclose(got, O.aprox_kl(x, eps, rho), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("rho,eps", [(1.0, 0.1), (0.3, 0.5), (5.0, 0.05)])
def test_aprox_berg_is_the_lambert_w_form(rho, eps):
    """Berg: e^{(x - y)/eps} = rho/(rho - y) gives y = rho - eps W((rho/eps) e^{(rho - x)/eps}) (x up to
    rho + 15 eps, where rho - y is still far above the rounding of rho)."""
    xs = np.concatenate([np.linspace(-1.5, 1.0, 11) * rho, rho + eps * np.array([-3.0, 0.0, 5.0, 15.0])])
    got = GP.aprox(GP.Berg(rho), torch.tensor(xs), eps).numpy()
    ref = rho - eps * np.real(scipy_special.lambertw((rho / eps) * np.exp((rho - xs) / eps)))
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-12 * rho)
    assert (got < rho).all()


def test_lambda_star_kl_is_prop2():
    C, a, b = problem(9, 7, seed=1)
    rng = np.random.default_rng(2)
    fb, gb = torch.tensor(rng.normal(0, 0.3, 9)), torch.tensor(rng.normal(0, 0.3, 7))
    for r1, r2 in [(1.0, 1.0), (0.2, 3.0)]:
        got = GP.lambda_star(a, b, fb, gb, GP.KL(r1), GP.KL(r2)).item()
        assert abs(got - O.lambda_star(a, b, fb, gb, r1, r2).item()) < 1e-12


@pytest.mark.parametrize("r1,r2", [(1.0, 1.0), (0.3, 2.0)])
def test_lambda_star_berg_equal_masses(r1, r2):
    """Berg: lambda* is the root of <a, phi_1^*'(-fb - l)> - <b, phi_2^*'(-gb + l)> (Prop. 1's equal masses),
    found here independently by brentq on the domain."""
    C, a, b = problem(8, 10, seed=3)
    rng = np.random.default_rng(4)
    fb, gb = torch.tensor(rng.normal(0, 0.2, 8)), torch.tensor(rng.normal(0, 0.2, 10))
    d1, d2 = GP.Berg(r1), GP.Berg(r2)
    lam = GP.lambda_star(a, b, fb, gb, d1, d2).item()
    gfun = lambda l: (a * d1.dphi_star(-fb - l)).sum().item() - (b * d2.dphi_star(-gb + l)).sum().item()
    lo = -r1 - fb.min().item() + 1e-12
    hi = r2 + gb.min().item() - 1e-12
    ref = scipy_opt.brentq(gfun, lo, hi, xtol=1e-15)
    assert abs(lam - ref) < 1e-10
    assert abs(gfun(lam)) < 1e-10


@pytest.mark.parametrize("T", [1, 5, 30])
def test_general_sinkhorns_with_kl_are_the_kl_oracle(T):
    """The generic loops with the KL divergence reproduce oracle.uot's F- and G-Sinkhorn iterates."""
    C, a, b = problem(6, 5, seed=5)
    eps, r1, r2 = 0.1, 0.7, 1.3
    f, g = GP.f_sinkhorn(C, a, b, eps, GP.KL(r1), GP.KL(r2), T)
    ref = O.sinkhorn(C, a, b, eps, r1, r2, T)
    assert torch.allclose(f, ref.f, atol=1e-12) and torch.allclose(g, ref.g, atol=1e-12)
    f, g, lam = GP.g_sinkhorn(C, a, b, eps, GP.KL(r1), GP.KL(r2), T)
    ref = O.g_sinkhorn(C, a, b, eps, r1, r2, T)
    assert torch.allclose(f, ref.f, atol=1e-12) and torch.allclose(g, ref.g, atol=1e-12)
    assert abs(lam.item() - ref.lam) < 1e-12


def maximise_dual(C, a, b, eps, d1, d2):
    """Independent solver: L-BFGS-B on -F_eps over (f, g) inside the Berg domain (f > -rho1, g > -rho2)."""
    Cn, an, bn = C.numpy(), a.numpy(), b.numpy()
    N, M = Cn.shape

    def fun(v):
        f, g = v[:N], v[N:]
        E = np.exp((f[:, None] + g[None, :] - Cn) / eps)
        val = (an * d1.rho * np.log1p(f / d1.rho)).sum() + (bn * d2.rho * np.log1p(g / d2.rho)).sum() \
            - eps * (an[:, None] * bn[None, :] * (E - 1.0)).sum()
        gf = an * d1.rho / (d1.rho + f) - an * (E * bn[None, :]).sum(1)
        gg = bn * d2.rho / (d2.rho + g) - bn * (E * an[:, None]).sum(0)
        return -val, -np.concatenate([gf, gg])

    bounds = [(-d1.rho + 1e-9, None)] * N + [(-d2.rho + 1e-9, None)] * M
    res = scipy_opt.minimize(fun, np.zeros(N + M), jac=True, method="L-BFGS-B", bounds=bounds,
                             options={"maxiter": 20000, "ftol": 1e-15, "gtol": 1e-13, "maxcor": 30})
    return -res.fun, res.x[:N], res.x[N:]


@pytest.mark.parametrize("eps,rho", [(0.1, 1.0), (0.5, 0.2)])
def test_berg_sinkhorns_reach_the_dual_maximiser(eps, rho):
    """Berg entropy: F- and G-Sinkhorn converge to the maximiser of F_eps found by an independent solver,
    where the first-order conditions hold."""
    C, a, b = problem(6, 5, seed=7)
    d1, d2 = GP.Berg(rho), GP.Berg(1.5 * rho)
    v_star, f_star, g_star = maximise_dual(C, a, b, eps, d1, d2)
    f1, g1 = GP.f_sinkhorn(C, a, b, eps, d1, d2, 400)
    f2, g2, _ = GP.g_sinkhorn(C, a, b, eps, d1, d2, 400)
    for f, g in ((f1, g1), (f2, g2)):
        v = GP.dual_value(C, a, b, f, g, eps, d1, d2).item()
        assert abs(v - v_star) < 1e-9 * max(1.0, abs(v_star))
        assert np.allclose(f.numpy(), f_star, atol=2e-5) and np.allclose(g.numpy(), g_star, atol=2e-5)
        E = torch.exp((f[:, None] + g[None, :] - C) / eps)
        gf = a * d1.dphi_star(-f) - a * (E * b[None, :]).sum(1)
        gg = b * d2.dphi_star(-g) - b * (E * a[:, None]).sum(0)
        assert gf.abs().max().item() < 1e-9 and gg.abs().max().item() < 1e-9
