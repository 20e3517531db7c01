"""Tensor-core sweeps (dim >= 32: split-FP16 cross term on tcgen05 for the solver and softmin
sweeps, 3xTF32 mma.sync fragments for the moment and adjoint sweeps) against the FP64 oracle."""
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


def gauss_problem(n, m, d, seed, eps, rho, ma=1.0, mb=2.0, shift=0.0):
    rx, ry = np.random.default_rng(seed), np.random.default_rng(seed + 1)
    sd = np.sqrt(1.0 / (2 * d))
    p = W.random_problem(n, m, d, seed=seed, eps=eps, rho1=rho, rho2=rho, mass_a=ma, mass_b=mb)
    p.x = (sd * rx.standard_normal((n, d)) + shift).astype(np.float32)
    p.y = (sd * ry.standard_normal((m, d)) + shift).astype(np.float32)
    return p


def spec_of(U, p):
    dev = torch.device("cuda:0")
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    return U.Spec(t(p.a), t(p.b), p.eps, p.rho1, p.rho2, x=t(p.x), y=t(p.y))


def assert_close(got, ref, eps, what):
    ref = torch.as_tensor(ref, dtype=torch.float64)
    err = (got.double().cpu() - ref).abs()
    tol = 1e-4 * eps + 2 * 2.0 ** -23 * ref.abs()
    assert bool((err <= tol).all()), (what, err.max().item(), 1e-4 * eps)


@pytest.mark.parametrize("n,m,d,eps,shift", [
    (300, 517, 32, 0.05, 0.0), (1000, 700, 64, 0.05, 0.0), (129, 257, 48, 0.1, 0.0), (400, 300, 40, 0.05, 3.0),
])
def test_softmin_mma(U, n, m, d, eps, shift):
    p = gauss_problem(n, m, d, seed=d + n, eps=eps, rho=0.5, shift=shift)
    spec = spec_of(U, p)
    rng = np.random.default_rng(3)
    g = (0.2 * rng.standard_normal(m)).astype(np.float32)
    f = (0.2 * rng.standard_normal(n)).astype(np.float32)
    C = O.cost_matrix(p.x, p.y)
    assert_close(U.softmin(spec, torch.from_numpy(g).cuda(), 0), O.smin_rows(C, p.b, g, eps), eps, "rows")
    assert_close(U.softmin(spec, torch.from_numpy(f).cuda(), 1), O.smin_cols(C, p.a, f, eps), eps, "cols")


@pytest.mark.parametrize("n,m,d", [(1, 1, 33), (5, 3, 56), (127, 20000, 32), (3000, 129, 64), (1300, 4100, 64),
                                   (2900, 2100, 32)])
def test_softmin_tcgen05_edges(U, n, m, d):
    """One row block against 157 key tiles (one or two units a CTA, a short last tile), a
    single point, dim not a multiple of 8, fewer keys than one 128-key tile, CTAs whose unit
    ranges cross a row-block boundary (11 x 33 and 23 x 17 units over the SMs), zero weights."""
    p = gauss_problem(n, m, d, seed=7 * d + n, eps=0.05, rho=0.5)
    if n > 4:
        p.a[::10] = 0.0
    if m > 4:
        p.b[::7] = 0.0
    spec = spec_of(U, p)
    rng = np.random.default_rng(5)
    g = (0.3 * rng.standard_normal(m)).astype(np.float32)
    f = (0.3 * rng.standard_normal(n)).astype(np.float32)
    C = O.cost_matrix(p.x, p.y)
    assert_close(U.softmin(spec, torch.from_numpy(g).cuda(), 0), O.smin_rows(C, p.b, g, p.eps), p.eps, "rows")
    assert_close(U.softmin(spec, torch.from_numpy(f).cuda(), 1), O.smin_cols(C, p.a, f, p.eps), p.eps, "cols")


@pytest.mark.parametrize("scale,shift", [(1e-3, 0.0), (1e3, 5e3), (1.0, 40.0)])
def test_softmin_tcgen05_coordinate_scales(U, scale, shift):
    """The power-of-two scaling of the FP16 split: clouds far below and far above unit size,
    and clouds far from the origin (the common centre comes off first); eps scales with the
    squared size so that the softmins stay comparable."""
    n, m, d = 700, 900, 48
    eps = 0.05 * scale * scale
    p = gauss_problem(n, m, d, seed=97, eps=eps, rho=0.5 * scale * scale)
    p.x = (p.x * scale + shift).astype(np.float32)
    p.y = (p.y * scale + shift).astype(np.float32)
    spec = spec_of(U, p)
    rng = np.random.default_rng(11)
    g = (0.3 * eps * rng.standard_normal(m)).astype(np.float32)
    f = (0.3 * eps * rng.standard_normal(n)).astype(np.float32)
    C = O.cost_matrix(p.x, p.y)
    assert_close(U.softmin(spec, torch.from_numpy(g).cuda(), 0), O.smin_rows(C, p.b, g, p.eps), p.eps, "rows")
    assert_close(U.softmin(spec, torch.from_numpy(f).cuda(), 1), O.smin_cols(C, p.a, f, p.eps), p.eps, "cols")


@pytest.mark.parametrize("method", ["plain", "ti", "g"])
def test_tcgen05_iterates_match_oracle(U, method):
    """Ragged D = 40 problem with zero weights and rho1 != rho2: iterate-by-iterate parity of
    the solvers on the tcgen05 sweeps."""
    p = gauss_problem(611, 437, 40, seed=21, eps=0.05, rho=0.3)
    p.rho2 = 2.0
    p.a[::10] = 0.0
    spec = spec_of(U, p)
    C = O.cost_matrix(p.x, p.y)
    solver = {"plain": O.sinkhorn, "ti": O.ti_sinkhorn, "g": O.g_sinkhorn}[method]
    for T in (1, 7):
        r = U.solve(spec, method, max_iter=T)
        ref = solver(C, p.a, p.b, p.eps, p.rho1, p.rho2, T)
        assert_close(r.f, ref.f, p.eps, f"{method} f after {T}")
        assert_close(r.g, ref.g, p.eps, f"{method} g after {T}")
        if method != "plain":
            assert abs(r.lam - ref.lam) < 1e-4 * p.eps


def test_d64_solve_and_grads_match_oracle(U):
    """Config-3 shape at reduced size: N = M = 1024, D = 64, eps = 5e-2, rho = 0.5, masses 1 / 2."""
    p = gauss_problem(1024, 1024, 64, seed=1003, eps=5e-2, rho=0.5)
    spec = spec_of(U, p)
    r = U.solve(spec, "ti", max_iter=5000, tol=1e-7, check_every=5)
    assert r.converged
    C = O.cost_matrix(p.x, p.y)
    ref = O.ti_sinkhorn(C, p.a, p.b, p.eps, p.rho1, p.rho2, 20000, tol=1e-12, check_every=10)
    # converged to r <= 1e-7: distance to the fixed point is bounded by r / (1 - rate)
    assert (r.f.double().cpu() - ref.f).abs().max().item() < 2e-5
    val = U.dual_value(spec, r.f, r.g)[0].item()
    ref_val = O.dual_value(C, p.a, p.b, ref.f, ref.g, p.eps, p.rho1, p.rho2).item()
    assert abs(val - ref_val) < 1e-6 * abs(ref_val)
    gr = U.grad(spec, r.f, r.g)
    ea, eb, ex, ey = O.envelope_grads(p.x, p.y, p.a, p.b, r.f.double().cpu(), r.g.double().cpu(),
                                      p.eps, p.rho1, p.rho2)
    for k, e in (("a", ea), ("b", eb), ("x", ex), ("y", ey)):
        rel = ((gr[k].double().cpu() - e).norm() / e.norm()).item()
        assert rel < 1e-4, (k, rel)


@pytest.mark.parametrize("n,m,d,T,K", [(96, 80, 48, 12, 5), (130, 110, 64, 20, 20)])
def test_unrolled_high_dim_matches_autograd(U, n, m, d, T, K):
    """Unrolled backward with the tensor-core moment and adjoint sweeps (dim >= 32) against FP64
    autograd of the oracle's truncated TI solve."""
    p = gauss_problem(n, m, d, seed=d + T, eps=0.1, rho=0.5)
    spec = spec_of(U, p)
    val, g = U.grad_unrolled(spec, T=T, ckpt_every=K)
    rv, ga, gb, gx, gy = O.unrolled_grads(p.x, p.y, p.a, p.b, p.eps, p.rho1, p.rho2, T)
    assert abs(val.item() - rv.item()) < 1e-6 * abs(rv.item())
    for k, ref in (("a", ga), ("b", gb), ("x", gx), ("y", gy)):
        ref = torch.as_tensor(ref, dtype=torch.float64)
        rel = ((g[k].double().cpu() - ref).norm() / ref.norm()).item()
        assert rel < 1e-4, (k, rel)
