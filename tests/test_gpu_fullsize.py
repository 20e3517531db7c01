"""Every workload at its full size on the GPU, checked by the FP64 oracle.

At these sizes the oracle cannot run whole solves, but it can evaluate exactly,
in FP64, anything that involves a few rows or columns of the cost: one
half-step of a row from the GPU's other potential, a softmin, an envelope
gradient.  The returned pair (f, g) of a solve satisfies f = aprox(Smin_b(C - g))
up to rounding (the last half-step is an f-step, and the translation of Prop. 1
preserves the relation), and |g - aprox(Smin_a(C - f))| is bounded by the
reported fixed-point residual: that is the sampled certificate.  Where the
oracle can reach every entry (the 20000-point clouds: 4e8 entries; the
16384-point sub-sample of the 262144-point clouds) it does, in row blocks.

Tolerances: potentials and softmins 1e-4 eps + 2 ulp_f32 (the rounding of a
float32 output), values relative 1e-6, gradients relative l2 1e-4 per tensor.
"""
import math

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


def dev_t(v):
    return torch.from_numpy(np.ascontiguousarray(v)).to(torch.device("cuda:0"))


def spec_of(U, p, C=None):
    if C is not None:
        return U.Spec(dev_t(p.a), dev_t(p.b), p.eps, p.rho1, p.rho2, C=C)
    return U.Spec(dev_t(p.a), dev_t(p.b), p.eps, p.rho1, p.rho2, x=dev_t(p.x), y=dev_t(p.y), p=p.p)


def pot_tol(eps, ref):
    return 1e-4 * eps + 2.0 * 2.0 ** -23 * ref.abs()


def rel_l2(got, ref):
    ref = torch.as_tensor(ref, dtype=torch.float64)
    return ((got.double().cpu() - ref).norm() / ref.norm()).item()


def sampled_certificate(pr, f, g, residual, k=160, seed=0, C=None):
    """Max violation of the f- and g-equations on k sampled rows and columns, in
    units of the tolerance 1e-4 eps + 2 ulp (+ the residual on the g side).  With C
    (a device float32 matrix) the rows and columns come from the stored cost."""
    rng = np.random.default_rng(seed)
    f = f.double().cpu()
    g = g.double().cpu()
    n, m = pr.a.shape[0], pr.b.shape[0]
    rows = rng.choice(n, size=min(k, n), replace=False)
    cols = rng.choice(m, size=min(k, m), replace=False)
    if C is None:
        Cr = O.cost_matrix(pr.x[rows], pr.y)
        Cc = O.cost_matrix(pr.x, pr.y[cols])
    else:
        Cr = C[torch.as_tensor(rows, device=C.device)].cpu()
        Cc = C[:, torch.as_tensor(cols, device=C.device)].cpu()
    fr = O.aprox_kl(O.smin_rows(Cr, pr.b, g, pr.eps), pr.eps, pr.rho1)
    gc = O.aprox_kl(O.smin_cols(Cc, pr.a, f, pr.eps), pr.eps, pr.rho2)
    vf = ((f[rows] - fr).abs() / pot_tol(pr.eps, fr)).max().item()
    vg = ((g[cols] - gc).abs() / (pot_tol(pr.eps, gc) + residual)).max().item()
    return vf, vg


def mass_gap(pr, f, g):
    """Prop. 1: <a, e^{-f/rho1}> = <b, e^{-g/rho2}> for the translated pair; relative gap."""
    f, g = f.double().cpu(), g.double().cpu()
    A = (O._t(pr.a) * torch.exp(-f / pr.rho1)).sum().item()
    B = (O._t(pr.b) * torch.exp(-g / pr.rho2)).sum().item()
    return abs(A - B) / A


def gap_bound(pr, f, g, residual, mass):
    """Duality gap of a pair whose f- and g-equations hold within df and dg (cost units).

    With pi1 = a e^{-f/rho1 + u_f}, pi2 = b e^{-g/rho2 + u_g}, u = d (1/eps + 1/rho), the gap
    P - D reduces to rho1 <pi1, u_f - 1 + e^{-u_f}> + rho2 <pi2, u_g - 1 + e^{-u_g}> >= 0, at
    most m(pi) (rho1 u_f^2 + rho2 u_g^2) for |u| <= 1.  Here df is the softmin tolerance and dg
    adds the fixed-point residual."""
    df = 1e-4 * pr.eps + 2.0 ** -22 * f.abs().max().item()
    dg = residual + 1e-4 * pr.eps + 2.0 ** -22 * g.abs().max().item()
    uf = df * (1.0 / pr.eps + 1.0 / pr.rho1)
    ug = dg * (1.0 / pr.eps + 1.0 / pr.rho2)
    return mass * (pr.rho1 * uf * uf + pr.rho2 * ug * ug)


def exact_softmins_blocked(x, y, a, b, f, g, eps, block=1000):
    """S_i = Smin_b^eps(C_i. - g) and S'_j = Smin_a^eps(C_.j - f) over every entry, in FP64,
    by row blocks of the oracle's cost (the column log-sum-exps of the blocks are combined at
    the end)."""
    a, b, f, g = map(O._t, (a, b, f, g))
    S = torch.empty(x.shape[0], dtype=torch.float64)
    col_parts = []
    for i0 in range(0, x.shape[0], block):
        Cb = O.cost_matrix(x[i0:i0 + block], y)
        S[i0:i0 + block] = O.smin_rows(Cb, b, g, eps)
        col_parts.append(O.log_dot_exp(a[i0:i0 + block], ((f[i0:i0 + block, None] - Cb) / eps).T))
    Sp = -eps * torch.logsumexp(torch.stack(col_parts), dim=0)
    return S, Sp


# ------------------------------------------------------------------ 3-D mixtures, N = M = 20000

@pytest.mark.parametrize("rho", [0.1, 1.0, 10.0])
@pytest.mark.parametrize("policy", ["auto", "off"])
def test_config2_full_size_solve_sampled(U, rho, policy):
    """TI-Sinkhorn to residual 1e-6 in the timed launch configuration, every rho of the workload."""
    pr = W.config2(rho)
    spec = spec_of(U, pr)
    r = U.solve(spec, "ti", max_iter=20000, tol=1e-6, check_every=10, lse_reference=policy)
    assert r.converged and r.residual <= 1e-6
    vf, vg = sampled_certificate(pr, r.f, r.g, r.residual)
    assert vf <= 1.0 and vg <= 1.0, (vf, vg)
    assert mass_gap(pr, r.f, r.g) < 1e-5


@pytest.mark.parametrize("rho", [0.1, 1.0, 10.0])
def test_config2_full_size_values_all_entries(U, rho):
    """Dual value, primal value, plan mass and duality gap of the GPU's converged pair against the
    oracle's FP64 sums over all 4e8 entries (exact row and column softmins by row blocks, then the
    O(N + M) forms of the dual and primal objectives)."""
    pr = W.config2(rho)
    spec = spec_of(U, pr)
    r = U.solve(spec, "ti", max_iter=20000, tol=1e-6, check_every=10)
    assert r.converged
    out = U.dual_value(spec, r.f, r.g, primal=True).cpu()
    val, prim, mpi = out[0].item(), out[1].item(), out[2].item()
    f, g = r.f.double().cpu(), r.g.double().cpu()
    S, Sp = exact_softmins_blocked(pr.x, pr.y, pr.a, pr.b, f, g, pr.eps)
    D = O.dual_from_softmin(pr.a, pr.b, f, g, S, pr.eps, pr.rho1, pr.rho2).item()
    P = O.primal_from_softmins(pr.a, pr.b, f, g, S, Sp, pr.eps, pr.rho1, pr.rho2).item()
    m_ref = (O._t(pr.a) * torch.exp((f - S) / pr.eps)).sum().item()
    assert abs(val - D) < 1e-6 * abs(D), (val, D)
    assert abs(prim - P) < 1e-6 * abs(P), (prim, P)
    # m(pi) = sum_i a_i e^{(f_i - S_i)/eps}: a softmin error dS (<= 1e-4 eps) moves each term by dS/eps
    assert abs(mpi - m_ref) < 1e-4 * m_ref, (mpi, m_ref)
    assert 0.0 <= P - D + 1e-9 * abs(D) <= gap_bound(pr, f, g, r.residual, m_ref) + 1e-9 * abs(D), (P - D,)


def test_config2_dense_full_size(U):
    """The same clouds as a stored 20000 x 20000 FP32 cost (1.6 GB, larger than L2): softmins on
    sampled rows and columns against the oracle on the stored values, then a TI solve to 1e-6
    certified on sampled rows and columns of the stored cost."""
    pr = W.config2(1.0)
    C = W.dense_cost_f32_device(pr.x, pr.y, torch.device("cuda:0"))
    spec = spec_of(U, pr, C=C)
    rng = np.random.default_rng(21)
    g0 = (0.05 * rng.standard_normal(pr.m)).astype(np.float32)
    f0 = (0.05 * rng.standard_normal(pr.n)).astype(np.float32)
    S = U.softmin(spec, dev_t(g0), 0).double().cpu()
    Sp = U.softmin(spec, dev_t(f0), 1).double().cpu()
    rows = torch.as_tensor(rng.choice(pr.n, 160, replace=False))
    cols = torch.as_tensor(rng.choice(pr.m, 160, replace=False))
    ref_r = O.smin_rows(C[rows.cuda()].cpu(), pr.b, g0, pr.eps)
    ref_c = O.smin_cols(C[:, cols.cuda()].cpu(), pr.a, f0, pr.eps)
    assert bool(((S[rows] - ref_r).abs() <= pot_tol(pr.eps, ref_r)).all()), (S[rows] - ref_r).abs().max().item()
    assert bool(((Sp[cols] - ref_c).abs() <= pot_tol(pr.eps, ref_c)).all()), (Sp[cols] - ref_c).abs().max().item()
    r = U.solve(spec, "ti", max_iter=20000, tol=1e-6, check_every=10)
    assert r.converged
    vf, vg = sampled_certificate(pr, r.f, r.g, r.residual, C=C)
    assert vf <= 1.0 and vg <= 1.0, (vf, vg)
    assert mass_gap(pr, r.f, r.g) < 1e-5
    del C, spec
    torch.cuda.empty_cache()


# ------------------------------------------------------------------ D = 64 Gaussians, N = M = 8192

@pytest.fixture(scope="module")
def cfg3(U):
    pr = W.config3()
    spec = spec_of(U, pr)
    r = U.solve(spec, "ti", max_iter=5000, tol=1e-6, check_every=5)
    assert r.converged
    return pr, spec, r


def test_config3_full_size_solve_sampled(U, cfg3):
    """TI-Sinkhorn to residual 1e-6 on the tensor-core sweeps, certified on sampled rows and
    columns at 1e-4 eps + 2 ulp (plus the residual on the g side)."""
    pr, spec, r = cfg3
    vf, vg = sampled_certificate(pr, r.f, r.g, r.residual, k=128, seed=3)
    assert vf <= 1.0 and vg <= 1.0, (vf, vg)
    assert mass_gap(pr, r.f, r.g) < 1e-5


def test_config3_envelope_grads_sampled(U, cfg3):
    """Envelope gradients with respect to a, x (sampled rows) and b, y (sampled columns) against
    the oracle's envelope formula evaluated in FP64 over every key of those rows and columns."""
    pr, spec, r = cfg3
    gr = U.grad(spec, r.f, r.g)
    f, g = r.f.double().cpu(), r.g.double().cpu()
    rng = np.random.default_rng(5)
    rows = rng.choice(pr.n, 96, replace=False)
    cols = rng.choice(pr.m, 96, replace=False)
    ga, _, gx, _ = O.envelope_grads(pr.x[rows], pr.y, pr.a[rows], pr.b, f[rows], g, pr.eps, pr.rho1, pr.rho2)
    _, gb, _, gy = O.envelope_grads(pr.x, pr.y[cols], pr.a, pr.b[cols], f, g[cols], pr.eps, pr.rho1, pr.rho2)
    # (the row quantities use every column and the full m(b), the column ones every row and m(a))
    for name, got, ref in (("a", gr["a"].cpu()[rows], ga), ("x", gr["x"].cpu()[rows], gx),
                           ("b", gr["b"].cpu()[cols], gb), ("y", gr["y"].cpu()[cols], gy)):
        assert rel_l2(got, ref) < 1e-4, (name, rel_l2(got, ref))


def test_config3_unrolled_matches_envelope_when_converged(U, cfg3):
    """Unrolled backward through T = 200 TI iterations (checkpoints every 20): the iterate has
    converged long before T = 200, so the derivative of F_eps(f_T, g_T) equals the envelope
    gradient at the fixed point (the terms through the potentials vanish with the residual)."""
    pr, spec, r = cfg3
    val, gu = U.grad_unrolled(spec, T=200, ckpt_every=20)
    ref_val = U.dual_value(spec, r.f, r.g)[0].item()
    assert abs(val.item() - ref_val) < 1e-6 * abs(ref_val), (val.item(), ref_val)
    ge = U.grad(spec, r.f, r.g)
    for k in ("a", "b", "x", "y"):
        assert rel_l2(gu[k], ge[k].double().cpu()) < 1e-4, (k, rel_l2(gu[k], ge[k].double().cpu()))


def test_config3_finite_differences_of_the_value(U, cfg3):
    """Central differences of UOT with h = 1e-3 along 8 random unit directions in R^{N x D} (the
    value from a TI solve warm-started at the optimum and solved to 1e-7, then the FP64 dual value)
    against <grad_x, d> from the envelope gradient.  Values computed from FP32 potentials carry
    noise of ~1e-8; each direction is therefore drawn half along the gradient and half isotropic,
    so that the directional derivative stands well above that noise (a purely isotropic direction
    in 524288 dimensions sees only 1/724 of the gradient's norm)."""
    pr, spec, r = cfg3
    gx = U.grad(spec, r.f, r.g, wrt=("x",))["x"].double()
    ghat = gx / gx.norm()
    rng = np.random.default_rng(11)
    h = 1e-3
    x0 = dev_t(pr.x)
    errs = []
    for _ in range(8):
        d = torch.from_numpy(rng.standard_normal(pr.x.shape)).cuda()
        d = ghat + d / d.norm()
        d /= d.norm()
        vals = []
        for sgn in (1.0, -1.0):
            xs = (x0.double() + sgn * h * d).float().contiguous()
            sp = U.Spec(spec.a, spec.b, pr.eps, pr.rho1, pr.rho2, x=xs, y=spec.y)
            rr = U.solve(sp, "ti", max_iter=5000, tol=1e-7, check_every=5, f0=r.f)
            assert rr.converged
            vals.append(U.dual_value(sp, rr.f, rr.g)[0].item())
        # the perturbed points are rounded to FP32: the realised step is (xs+ - xs-) / 2
        dd = ((x0.double() + h * d).float().double() - (x0.double() - h * d).float().double()) / 2
        fd = (vals[0] - vals[1]) / 2
        ana = (gx * dd).sum().item()
        errs.append(abs(fd - ana) / abs(ana))
    assert max(errs) < 2e-3, errs


# ------------------------------------------------------------------ 4096 ragged problems

def _config4_selection(probs, k_rand=64, seed=7):
    """The 16 largest and 16 smallest problems by N*M, plus k_rand others drawn at random."""
    size = np.array([p.n * p.m for p in probs])
    order = np.argsort(size)
    chosen = list(order[-16:]) + list(order[:16])
    rest = np.setdiff1d(np.arange(len(probs)), chosen)
    chosen += list(np.random.default_rng(seed).choice(rest, k_rand, replace=False))
    return [int(k) for k in chosen]


def test_config4_across_the_full_size_range(U):
    """96 problems of the 4096-problem workload (N, M log-uniform in [64, 4096], the largest and
    smallest included), solved in one batched call to residual 1e-6: the FP64 oracle evaluates both
    fixed-point equations of every problem at the GPU's pair, checks Prop. 1's mass equality, and
    for problems small enough runs the same number of TI iterations from zero and compares the
    translated pairs element by element."""
    probs = W.config4()
    sel = _config4_selection(probs)
    batch = [probs[k] for k in sel]
    assert max(p.n * p.m for p in batch) > 0.9 * 4096 * 4096 * 0.5
    r = U.solve_batched(batch, "ti", max_iter=20000, tol=1e-6, check_every=10)
    assert all(r.converged), [k for k, c in enumerate(r.converged) if not c]
    compared = 0
    for k, p in enumerate(batch):
        C = O.cost_matrix(p.x, p.y)
        f, g = r.f[k].double().cpu(), r.g[k].double().cpu()
        fr = O.aprox_kl(O.smin_rows(C, p.b, g, p.eps), p.eps, p.rho1)
        gc = O.aprox_kl(O.smin_cols(C, p.a, f, p.eps), p.eps, p.rho2)
        assert bool(((f - fr).abs() <= pot_tol(p.eps, fr)).all()), (k, "f", (f - fr).abs().max().item())
        assert bool(((g - gc).abs() <= pot_tol(p.eps, gc) + r.residual[k]).all()), (k, "g")
        # the reported residual is the g-equation's violation (R7), to the sweep's accuracy
        assert abs((g - gc).abs().max().item() - r.residual[k]) <= 1e-4 * p.eps + 2.0 ** -22 * gc.abs().max().item()
        assert mass_gap(p, r.f[k], r.g[k]) < 1e-5, k
        if r.iters[k] * p.n * p.m <= 3e8:
            ref = O.ti_sinkhorn(C, p.a, p.b, p.eps, p.rho1, p.rho2, r.iters[k])
            assert bool(((f - ref.f).abs() <= pot_tol(p.eps, ref.f)).all()), (k, (f - ref.f).abs().max().item())
            assert bool(((g - ref.g).abs() <= pot_tol(p.eps, ref.g)).all()), (k, (g - ref.g).abs().max().item())
            compared += 1
    assert compared >= 16


def test_config4_whole_workload(U):
    """All 4096 problems in one batched call: every one converges to 1e-6; the oracle evaluates the
    fixed-point equations of 32 of them (random) at the GPU's pairs."""
    probs = W.config4()
    r = U.solve_batched(probs, "ti", max_iter=20000, tol=1e-6, check_every=10)
    assert all(r.converged), [k for k, c in enumerate(r.converged) if not c][:10]
    for k in np.random.default_rng(9).choice(len(probs), 32, replace=False):
        p = probs[k]
        C = O.cost_matrix(p.x, p.y)
        f, g = r.f[k].double().cpu(), r.g[k].double().cpu()
        rr = O.fixed_point_residual(C, p.a, p.b, f, g, p.eps, p.rho1, p.rho2).item()
        assert rr <= r.residual[k] + 1e-4 * p.eps + 2.0 ** -22 * max(f.abs().max().item(), g.abs().max().item())


# ------------------------------------------------------------------ 3-D uniform, N = M = 262144

@pytest.fixture(scope="module")
def cfg5(U):
    pr = W.config5()
    spec = spec_of(U, pr)
    r = U.solve(spec, "ti", max_iter=20000, tol=1e-6, check_every=10)
    assert r.converged
    return pr, spec, r


def test_config5_converged_certificate(U, cfg5):
    """N = M = 262144 (6.9e10 entries per sweep) solved to residual 1e-6.  Certificate: the f- and
    g-equations on 96 sampled rows and columns; Prop. 1's mass equality, and lambda* of the returned
    pair is 0 to within the FP32 rounding of the potentials; the GPU's full row and column softmins
    at the pair, checked on the same samples, give the oracle's O(N + M) dual and primal values,
    which the GPU's own FP64 dual value, primal value and plan mass must match; the gap is within
    what the residual allows."""
    pr, spec, r = cfg5
    vf, vg = sampled_certificate(pr, r.f, r.g, r.residual, k=96, seed=1)
    assert vf <= 1.0 and vg <= 1.0, (vf, vg)
    f, g = r.f.double().cpu(), r.g.double().cpu()
    assert mass_gap(pr, r.f, r.g) < 1e-5
    lam = O.lambda_star(pr.a, pr.b, f, g, pr.rho1, pr.rho2).item()
    assert abs(lam) <= 2.0 ** -23 * max(f.abs().max().item(), g.abs().max().item()), lam
    S = U.softmin(spec, r.g, 0).double().cpu()
    Sp = U.softmin(spec, r.f, 1).double().cpu()
    rng = np.random.default_rng(2)
    rows = rng.choice(pr.n, 96, replace=False)
    cols = rng.choice(pr.m, 96, replace=False)
    ref_r = O.smin_rows(O.cost_matrix(pr.x[rows], pr.y), pr.b, g, pr.eps)
    ref_c = O.smin_cols(O.cost_matrix(pr.x, pr.y[cols]), pr.a, f, pr.eps)
    assert bool(((S[rows] - ref_r).abs() <= pot_tol(pr.eps, ref_r)).all())
    assert bool(((Sp[cols] - ref_c).abs() <= pot_tol(pr.eps, ref_c)).all())
    D = O.dual_from_softmin(pr.a, pr.b, f, g, S, pr.eps, pr.rho1, pr.rho2).item()
    P = O.primal_from_softmins(pr.a, pr.b, f, g, S, Sp, pr.eps, pr.rho1, pr.rho2).item()
    m_pi = (O._t(pr.a) * torch.exp((f - S) / pr.eps)).sum().item()
    out = U.dual_value(spec, r.f, r.g, primal=True).cpu()
    assert abs(out[0].item() - D) < 1e-6 * abs(D), (out[0].item(), D)
    assert abs(out[1].item() - P) < 1e-6 * abs(P), (out[1].item(), P)
    assert abs(out[2].item() - m_pi) < 1e-4 * m_pi
    assert 0.0 <= P - D + 1e-9 * abs(D) <= gap_bound(pr, f, g, r.residual, m_pi) + 1e-9 * abs(D), (P - D,)


def test_config5_grad_x_sampled(U, cfg5):
    """Envelope gradient with respect to x (and a) on 64 sampled rows against the oracle's formula
    over all 262144 keys of each row."""
    pr, spec, r = cfg5
    gr = U.grad(spec, r.f, r.g, wrt=("a", "x"))
    f, g = r.f.double().cpu(), r.g.double().cpu()
    rows = np.random.default_rng(4).choice(pr.n, 64, replace=False)
    ga, _, gx, _ = O.envelope_grads(pr.x[rows], pr.y, pr.a[rows], pr.b, f[rows], g, pr.eps, pr.rho1, pr.rho2)
    assert rel_l2(gr["x"].cpu()[rows], gx) < 1e-4, rel_l2(gr["x"].cpu()[rows], gx)
    assert rel_l2(gr["a"].cpu()[rows], ga) < 1e-4, rel_l2(gr["a"].cpu()[rows], ga)


def test_config5_subsample_16384_full_oracle(U):
    """The first 16384 points of each cloud (masses kept): 6 TI iterations from zero on the GPU
    and in the full FP64 oracle, compared element by element; then the GPU solve to 1e-6 with its
    exact FP64 residual over all 2.7e8 entries."""
    full = W.config5()
    n = 16384
    pr = W.Problem(full.x[:n].copy(), full.y[:n].copy(),
                   (full.a[:n] / full.a[:n].sum() * 1.0).astype(np.float32),
                   (full.b[:n] / full.b[:n].sum() * 1.3).astype(np.float32),
                   full.eps, full.rho1, full.rho2, 2.0, name="3-D uniform sub-sample N=M=16384")
    spec = spec_of(U, pr)
    C = O.cost_matrix(pr.x, pr.y)
    T = 6
    r = U.solve(spec, "ti", max_iter=T, tol=0.0)
    ref = O.ti_sinkhorn(C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, T)
    assert bool(((r.f.double().cpu() - ref.f).abs() <= pot_tol(pr.eps, ref.f)).all())
    assert bool(((r.g.double().cpu() - ref.g).abs() <= pot_tol(pr.eps, ref.g)).all())
    assert abs(r.lam - ref.lam) < 1e-4 * pr.eps
    rc = U.solve(spec, "ti", max_iter=20000, tol=1e-6, check_every=10)
    assert rc.converged
    rr = O.fixed_point_residual(C, pr.a, pr.b, rc.f.double().cpu(), rc.g.double().cpu(), pr.eps, pr.rho1,
                                pr.rho2).item()
    assert rr <= rc.residual + 1e-4 * pr.eps + 2.0 ** -22 * rc.g.abs().max().item(), (rr, rc.residual)
