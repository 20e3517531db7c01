"""Full-size workloads on the GPU, checked on sampled rows and columns by the oracle.

At N = M = 20000 (3-D mixtures, eps = 1e-3, the timed workload) and
N = M = 262144 (3-D uniform) the oracle cannot run whole solves, but it can
evaluate one half-step of one row exactly from the GPU's other potential.  The
returned pair (f, g) of both solvers satisfies f = aprox(Smin_b(C - g)) up to
rounding (the last half-step is an f-step, and the translation of Prop. 1
preserves the relation), and |g - aprox(Smin_a(C - f))| is bounded by the
reported fixed-point residual.
"""
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


def spec_of(U, p):
    dev = torch.device("cuda:0")
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    return U.Spec(t(p.a), t(p.b), p.eps, p.rho1, p.rho2, x=t(p.x), y=t(p.y), p=p.p)


def sampled_certificate(pr, f, g, residual, k=160, seed=0):
    """Max violation of the f- and g-equations on k sampled rows and columns, in
    units of the tolerance 1e-4 eps + 2 ulp (+ the residual on the g side)."""
    rng = np.random.default_rng(seed)
    f = f.double().cpu()
    g = g.double().cpu()
    rows = rng.choice(pr.x.shape[0], size=k, replace=False)
    cols = rng.choice(pr.y.shape[0], size=k, replace=False)
    Cr = O.cost_matrix(pr.x[rows], pr.y)
    fr = O.aprox_kl(O.smin_rows(Cr, pr.b, g, pr.eps), pr.eps, pr.rho1)
    Cc = O.cost_matrix(pr.x, pr.y[cols])
    gc = O.aprox_kl(O.smin_cols(Cc, pr.a, f, pr.eps), pr.eps, pr.rho2)
    tol_f = 1e-4 * pr.eps + 2.0 * 2.0 ** -23 * fr.abs()
    tol_g = 1e-4 * pr.eps + 2.0 * 2.0 ** -23 * gc.abs() + residual
    vf = ((f[rows] - fr).abs() / tol_f).max().item()
    vg = ((g[cols] - gc).abs() / tol_g).max().item()
    return vf, vg


@pytest.mark.parametrize("policy", ["auto", "off"])
def test_config2_full_size_solve_sampled(U, policy):
    pr = W.config2(1.0)
    spec = spec_of(U, pr)
    r = U.solve(spec, "ti", max_iter=20000, tol=1e-6, check_every=10, lse_reference=policy)
    assert r.converged and r.residual <= 1e-6
    vf, vg = sampled_certificate(pr, r.f, r.g, r.residual)
    assert vf <= 1.0 and vg <= 1.0, (vf, vg)
    # Prop. 1: equal masses after the translation
    f, g = r.f.double().cpu(), r.g.double().cpu()
    A = (O._t(pr.a) * torch.exp(-f / pr.rho1)).sum().item()
    B = (O._t(pr.b) * torch.exp(-g / pr.rho2)).sum().item()
    assert abs(A - B) < 1e-5 * A


def test_config2_full_size_dual_value(U):
    """Dual value of the GPU's potentials against the oracle's FP64 sum over all
    4e8 entries (row blocks of the cost, same formula)."""
    pr = W.config2(1.0)
    spec = spec_of(U, pr)
    r = U.solve(spec, "ti", max_iter=200, tol=0.0)
    val = U.dual_value(spec, r.f, r.g)[0].item()
    f, g = r.f.double().cpu(), r.g.double().cpu()
    a, b = O._t(pr.a), O._t(pr.b)
    eps = pr.eps
    lin = -pr.rho1 * (a * torch.expm1(-f / pr.rho1)).sum() - pr.rho2 * (b * torch.expm1(-g / pr.rho2)).sum()
    cross = torch.zeros((), dtype=torch.float64)
    for i0 in range(0, pr.x.shape[0], 1000):
        C = O.cost_matrix(pr.x[i0:i0 + 1000], pr.y)
        E = torch.exp((f[i0:i0 + 1000, None] + g[None, :] - C) / eps)
        cross += (a[i0:i0 + 1000, None] * b[None, :] * E).sum()
    ref = (lin - eps * (cross - a.sum() * b.sum())).item()
    # same definition as the oracle's dual_value (Sec. 2 dual with phi* of rho KL)
    small = W.random_problem(50, 40, 3, seed=1, eps=eps, rho1=pr.rho1, rho2=pr.rho2)
    fs, gs = torch.linspace(-0.1, 0.1, 50, dtype=torch.float64), torch.linspace(0.05, -0.05, 40, dtype=torch.float64)
    Cs = O.cost_matrix(small.x, small.y)
    As, Bs = O._t(small.a), O._t(small.b)
    mine = (-pr.rho1 * (As * torch.expm1(-fs / pr.rho1)).sum() - pr.rho2 * (Bs * torch.expm1(-gs / pr.rho2)).sum()
            - eps * ((As[:, None] * Bs[None, :] * torch.exp((fs[:, None] + gs[None, :] - Cs) / eps)).sum()
                     - As.sum() * Bs.sum()))
    assert abs(mine.item() - O.dual_value(Cs, As, Bs, fs, gs, eps, pr.rho1, pr.rho2).item()) < 1e-12
    assert abs(val - ref) < 1e-6 * abs(ref), (val, ref)


@pytest.mark.parametrize("method", ["plain", "ti"])
def test_config5_full_size_iterations_sampled(U, method):
    """N = M = 262144 (6.9e10 cost entries per sweep): a few iterations, sampled rows."""
    pr = W.config5()
    spec = spec_of(U, pr)
    r = U.solve(spec, method, max_iter=12, tol=0.0)
    assert r.iters == 12
    vf, vg = sampled_certificate(pr, r.f, r.g, r.residual, k=96, seed=1)
    assert vf <= 1.0 and vg <= 1.0, (vf, vg)
