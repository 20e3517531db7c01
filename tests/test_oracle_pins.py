"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than itself: a
closed form, an invariant the paper proves, an independent solver, or brute
force on tiny inputs.  Problems use N != M, rho1 != rho2 and unequal masses so
that a swapped operand or a transposed index fails.
"""
import math

import numpy as np
import pytest
import torch

from oracle import uot as O
from paper_2201_00730_gb300 import workloads as W

F64 = torch.float64


def tiny(n=5, m=4, d=2, seed=3, eps=0.3, rho1=0.7, rho2=1.9, ma=1.3, mb=0.6):
    p = W.random_problem(n, m, d, seed=seed, eps=eps, rho1=rho1, rho2=rho2, mass_a=ma, mass_b=mb)
    C = O.cost_matrix(p.x, p.y)
    return p, C, O._t(p.a), O._t(p.b)


# ---------------------------------------------------------------- elementary

def test_cost_matrix_brute_force():
    p = W.random_problem(4, 3, 3, seed=1)
    C = O.cost_matrix(p.x, p.y)
    for i in range(4):
        for j in range(3):
            s = sum((float(p.x[i, k]) - float(p.y[j, k])) ** 2 for k in range(3))
            assert abs(C[i, j].item() - s) < 1e-15
    C3 = O.cost_matrix(p.x, p.y, p=3.0)
    for i in range(4):
        for j in range(3):
            s = sum((float(p.x[i, k]) - float(p.y[j, k])) ** 2 for k in range(3)) ** 1.5
            assert abs(C3[i, j].item() - s) < 1e-14


def test_softmin_brute_force_and_shift():
    rng = np.random.default_rng(0)
    w = rng.random(7)
    w[2] = 0.0                      # a zero weight drops out of the sum
    h = rng.standard_normal(7)
    for eps in (0.05, 0.5, 3.0):
        ref = -eps * math.log(sum(wi * math.exp(-hi / eps) for wi, hi in zip(w, h)))
        got = O.softmin(w, h, eps).item()
        assert abs(got - ref) < 1e-13 * max(1.0, abs(ref))
        # Smin(h + tau) = Smin(h) + tau (App. B, proof of Prop. 4)
        assert abs(O.softmin(w, h + 0.37, eps).item() - (got + 0.37)) < 1e-13


def test_softmin_single_column_exact():
    # M = 1: S_i = C_i1 - g_1 - eps log b_1 exactly
    p = W.random_problem(6, 1, 2, seed=4)
    C = O.cost_matrix(p.x, p.y)
    g = torch.tensor([0.31], dtype=F64)
    eps = 0.07
    S = O.smin_rows(C, p.b, g, eps)
    ref = C[:, 0] - g[0] - eps * math.log(float(p.b[0]))
    assert torch.allclose(S, ref, rtol=0, atol=1e-14)


def test_smin_rows_cols_are_transposes():
    p, C, a, b = tiny()
    f = torch.linspace(-0.2, 0.3, 5, dtype=F64)
    # column softmin of C is the row softmin of C^T
    assert torch.allclose(O.smin_cols(C, a, f, 0.3), O.smin_rows(C.T, a, f, 0.3), atol=1e-15)
    # brute-force one entry of each
    j = 2
    ref = -0.3 * math.log(sum(float(a[i]) * math.exp((float(f[i]) - float(C[i, j])) / 0.3) for i in range(5)))
    assert abs(O.smin_cols(C, a, f, 0.3)[j].item() - ref) < 1e-14


def test_kl_and_primal_brute_force():
    mu = np.array([0.2, 0.0, 0.5])
    nu = np.array([0.1, 0.3, 0.4])
    ref = sum(m * math.log(m / n) for m, n in zip(mu, nu) if m > 0) - mu.sum() + nu.sum()
    assert abs(O.kl_div(mu, nu).item() - ref) < 1e-15
    assert O.kl_div([0.1], [0.0]).item() == math.inf


def test_dual_and_primal_from_softmins_brute_force():
    """The O(N + M) forms of the dual (Eq. eq-dual-uot-kl) and of the primal (Eq. eq-primal-uot-kl)
    at an arbitrary pair (f, g), not an optimum, against the double sums written out term by term."""
    p, C, a, b = tiny(n=5, m=4, eps=0.3, rho1=0.7, rho2=1.9)
    f = [0.11, -0.32, 0.05, 0.4, -0.07]
    g = [-0.2, 0.15, 0.33, -0.01]
    eps, r1, r2 = p.eps, p.rho1, p.rho2
    A, B = [float(v) for v in a], [float(v) for v in b]
    Cl = [[float(C[i, j]) for j in range(4)] for i in range(5)]
    # dual: sum_i a_i phi-part + sum_j b_j phi-part - eps sum_ij a_i b_j (e^{(f_i + g_j - C_ij)/eps} - 1)
    ref = (sum(A[i] * r1 * (1 - math.exp(-f[i] / r1)) for i in range(5))
           + sum(B[j] * r2 * (1 - math.exp(-g[j] / r2)) for j in range(4))
           - eps * sum(A[i] * B[j] * (math.exp((f[i] + g[j] - Cl[i][j]) / eps) - 1)
                       for i in range(5) for j in range(4)))
    S = O.smin_rows(C, b, g, eps)
    Sp = O.smin_cols(C, a, f, eps)
    assert abs(O.dual_from_softmin(a, b, f, g, S, eps, r1, r2).item() - ref) < 1e-13
    # primal at the plan pi_ij = a_i b_j e^{(f_i + g_j - C_ij)/eps}: <pi, C> + eps KL(pi|ab) + rho KLs
    pi = [[A[i] * B[j] * math.exp((f[i] + g[j] - Cl[i][j]) / eps) for j in range(4)] for i in range(5)]

    def kl(mu, nu):
        return sum(m * math.log(m / n) for m, n in zip(mu, nu) if m > 0) - sum(mu) + sum(nu)

    flat = [pi[i][j] for i in range(5) for j in range(4)]
    ab = [A[i] * B[j] for i in range(5) for j in range(4)]
    row = [sum(pi[i]) for i in range(5)]
    col = [sum(pi[i][j] for i in range(5)) for j in range(4)]
    pref = (sum(pi[i][j] * Cl[i][j] for i in range(5) for j in range(4)) + eps * kl(flat, ab)
            + r1 * kl(row, A) + r2 * kl(col, B))
    got = O.primal_from_softmins(a, b, f, g, S, Sp, eps, r1, r2).item()
    assert abs(got - pref) < 1e-12 * max(1.0, abs(pref))


def test_dual_and_primal_from_softmins_zero_gap_at_newton_optimum():
    """At the maximiser of F_eps found by the independent damped-Newton solver both O(N + M) forms
    give the same value (zero duality gap, T4)."""
    p, C, a, b = tiny(6, 5, 2, 7, 0.2, 0.6, 1.4)
    fN, gN = newton_dual(C, a, b, p.eps, p.rho1, p.rho2)
    S = O.smin_rows(C, b, gN, p.eps)
    Sp = O.smin_cols(C, a, fN, p.eps)
    D = O.dual_from_softmin(a, b, fN, gN, S, p.eps, p.rho1, p.rho2).item()
    P = O.primal_from_softmins(a, b, fN, gN, S, Sp, p.eps, p.rho1, p.rho2).item()
    assert abs(D - P) < 1e-11 * max(1.0, abs(D))


# ------------------------------------------------------------ N = M = 1 (T1)

def n1_closed_form(a, b, c, eps, rho1, rho2):
    """Minimiser of pi c + eps KL(pi|ab) + rho1 KL(pi|a) + rho2 KL(pi|b) over pi >= 0."""
    logpi = (eps * math.log(a * b) + rho1 * math.log(a) + rho2 * math.log(b) - c) / (eps + rho1 + rho2)
    pi = math.exp(logpi)
    val = eps * a * b + rho1 * a + rho2 * b - (eps + rho1 + rho2) * pi
    f = -rho1 * math.log(pi / a)
    g = -rho2 * math.log(pi / b)
    return pi, val, f, g


@pytest.mark.parametrize("a,b,c,eps,rho1,rho2", [
    (1.0, 1.5, 0.3, 0.01, 1.0, 1.0),
    (0.4, 2.2, 1.7, 0.2, 0.3, 5.0),
    (3.0, 0.1, 0.0, 1.0, 2.0, 0.5),
])
def test_n1_closed_form(a, b, c, eps, rho1, rho2):
    pi, val, f, g = n1_closed_form(a, b, c, eps, rho1, rho2)
    C = torch.tensor([[c]], dtype=F64)
    A, B = torch.tensor([a], dtype=F64), torch.tensor([b], dtype=F64)
    ti = O.ti_sinkhorn(C, A, B, eps, rho1, rho2, 50)
    assert abs(ti.f.item() - f) < 1e-12 and abs(ti.g.item() - g) < 1e-12
    fs = O.sinkhorn(C, A, B, eps, rho1, rho2, 200000, tol=1e-14, check_every=50)
    assert abs(fs.f.item() - f) < 1e-10 and abs(fs.g.item() - g) < 1e-10
    assert abs(O.dual_value(C, A, B, ti.f, ti.g, eps, rho1, rho2).item() - val) < 1e-12
    P = O.transport_plan(C, A, B, ti.f, ti.g, eps)
    assert abs(P.item() - pi) < 1e-12
    assert abs(O.primal_value(C, A, B, P, eps, rho1, rho2).item() - val) < 1e-12
    # envelope derivatives: dUOT/da = eps b + rho1 - (rho1 + eps) pi / a
    ga, gb, gx, gy = O.envelope_grads([[0.0]], [[math.sqrt(c)]], A, B, ti.f, ti.g, eps, rho1, rho2)
    assert abs(ga.item() - (eps * b + rho1 - (rho1 + eps) * pi / a)) < 1e-11
    assert abs(gb.item() - (eps * a + rho2 - (rho2 + eps) * pi / b)) < 1e-11
    # dUOT/dc = +pi (primal <pi, C>), and dc/dx = 2 (x - y) = -2 sqrt(c) for x = 0, y = sqrt(c)
    assert abs(gx.item() - pi * (-2 * math.sqrt(c))) < 1e-11
    assert abs(gy.item() - pi * (2 * math.sqrt(c))) < 1e-11


# --------------------------------------------------------------- invariants

def test_lambda_star_mass_equality_T5():
    """Phi(fb, gb) equalises the re-weighted masses (Prop. 1 / Prop. 2)."""
    p, C, a, b = tiny(rho1=0.4, rho2=2.5)
    g = torch.Generator().manual_seed(0)
    for _ in range(5):
        fb = torch.randn(5, generator=g, dtype=F64)
        gb = torch.randn(4, generator=g, dtype=F64) * 2
        f, gg, lam = O.phi_map(a, b, fb, gb, p.rho1, p.rho2)
        ma = (a * torch.exp(-f / p.rho1)).sum()
        mb = (b * torch.exp(-gg / p.rho2)).sum()
        assert abs(ma - mb) < 1e-13 * ma
        # lambda* maximises G(fb, gb, .) = F(fb + lam, gb - lam)
        G = lambda l: O.dual_value(C, a, b, fb + l, gb - l, p.eps, p.rho1, p.rho2).item()
        L = lam.item()
        assert G(L) >= G(L + 1e-4) and G(L) >= G(L - 1e-4)


def test_lambda_star_smin_form_and_shift_T7():
    p, C, a, b = tiny(rho1=0.4, rho2=2.5)
    fb = torch.tensor([0.1, -0.3, 0.2, 0.5, 0.0], dtype=F64)
    gb = torch.tensor([0.7, -0.1, 0.4, 0.2], dtype=F64)
    r1, r2 = p.rho1, p.rho2
    t1, t2 = r1 / (r1 + r2), r2 / (r1 + r2)
    lam = O.lambda_star(a, b, fb, gb, r1, r2).item()
    alt = t1 * O.softmin(b, gb, r2).item() - t2 * O.softmin(a, fb, r1).item()
    assert abs(lam - alt) < 1e-14
    # lambda*(fb + tau, gb) = lambda*(fb, gb + tau) - tau (App. B)
    tau = 0.83
    assert abs(O.lambda_star(a, b, fb + tau, gb, r1, r2).item()
               - (O.lambda_star(a, b, fb, gb + tau, r1, r2).item() - tau)) < 1e-13


def test_h_invariance_and_prop3_T6():
    p, C, a, b = tiny(rho1=0.4, rho2=2.5)
    fb = torch.tensor([0.1, -0.3, 0.2, 0.5, 0.0], dtype=F64)
    gb = torch.tensor([0.7, -0.1, 0.4, 0.2], dtype=F64)
    f, g, _ = O.phi_map(a, b, fb, gb, p.rho1, p.rho2)
    H = O.h_value(C, a, b, fb, gb, p.eps, p.rho1, p.rho2).item()
    assert abs(H - O.dual_value(C, a, b, f, g, p.eps, p.rho1, p.rho2).item()) < 1e-13
    H2 = O.h_value(C, a, b, fb + 0.6, gb - 0.6, p.eps, p.rho1, p.rho2).item()
    assert abs(H - H2) < 1e-13


def _half_step_optimality(C, a, b, fb, gb, eps, rho1, rho2):
    """Residual of the optimality equation of fb given gb (Sec. 3, eq-optim-h-sink):
    e^{fb/eps} <b, e^{(gb - C)/eps}> = e^{-(fb + lambda*(fb, gb))/rho1}, in log form."""
    lam = O.lambda_star(a, b, fb, gb, rho1, rho2)
    lhs = fb / eps + torch.logsumexp(O.log_weights(b)[None, :] + (gb[None, :] - C) / eps, dim=1)
    rhs = -(fb + lam) / rho1
    return (lhs - rhs).abs().max().item()


@pytest.mark.parametrize("rho1,rho2", [(0.7, 0.7), (0.4, 2.5), (3.0, 0.2)])
def test_h_half_steps_solve_their_equations_T8(rho1, rho2):
    p, C, a, b = tiny(rho1=rho1, rho2=rho2, eps=0.15)
    gen = torch.Generator().manual_seed(1)
    fb0 = torch.randn(5, generator=gen, dtype=F64) * 0.3
    gb = O.psi_g(C, a, b, fb0, p.eps, rho1, rho2)
    # g half-step: the same equation with the roles of (a, fb, rho1), (b, gb, rho2) swapped
    assert _half_step_optimality(C.T, b, a, gb, fb0, p.eps, rho2, rho1) < 1e-12
    fb = O.psi_f(C, a, b, gb, p.eps, rho1, rho2)
    assert _half_step_optimality(C, a, b, fb, gb, p.eps, rho1, rho2) < 1e-12


def test_prop4_equal_rho_form():
    """For rho1 = rho2 the general update reduces to Prop. 4 with xi = eps/(eps + 2 rho)."""
    p, C, a, b = tiny(rho1=0.8, rho2=0.8, eps=0.2)
    rho, eps = 0.8, 0.2
    gb = torch.tensor([0.3, -0.2, 0.1, 0.6], dtype=F64)
    f_hat = rho / (rho + eps) * O.smin_rows(C, b, gb, eps) - 0.5 * eps / (rho + eps) * O.softmin(b, gb, rho)
    xi = eps / (eps + 2 * rho)
    ref = f_hat + xi * O.softmin(a, f_hat, rho)
    assert torch.allclose(O.psi_f(C, a, b, gb, eps, rho, rho), ref, atol=1e-14, rtol=0)


def test_psi_translation_and_nonexpansive_T9():
    p, C, a, b = tiny(rho1=0.4, rho2=2.5, eps=0.2)
    gen = torch.Generator().manual_seed(2)
    for _ in range(10):
        u = torch.randn(5, generator=gen, dtype=F64)
        v = torch.randn(5, generator=gen, dtype=F64)
        gu = O.psi_g(C, a, b, u, p.eps, p.rho1, p.rho2)
        gv = O.psi_g(C, a, b, v, p.eps, p.rho1, p.rho2)
        assert (gu - gv).abs().max() <= (u - v).abs().max() + 1e-14
        # Psi(fb + tau) = Psi(fb) - tau (Prop. in App. B)
        assert torch.allclose(O.psi_g(C, a, b, u + 0.45, p.eps, p.rho1, p.rho2), gu - 0.45, atol=1e-13, rtol=0)


# ---------------------------------------------------- fixed point and solvers

def newton_dual(C, a, b, eps, rho1, rho2, iters=200):
    """Damped Newton ascent on the concave dual F_eps (independent of Sinkhorn)."""
    n, m = C.shape
    z = torch.zeros(n + m, dtype=F64)
    def F(z):
        return O.dual_value(C, a, b, z[:n], z[n:], eps, rho1, rho2)
    for _ in range(iters):
        f, g = z[:n], z[n:]
        P = a[:, None] * b[None, :] * torch.exp((f[:, None] + g[None, :] - C) / eps)
        ea = a * torch.exp(-f / rho1)
        eb = b * torch.exp(-g / rho2)
        grad = torch.cat([ea - P.sum(1), eb - P.sum(0)])
        if grad.abs().max() < 1e-15:
            break
        Hm = torch.zeros(n + m, n + m, dtype=F64)
        Hm[:n, :n] = torch.diag(-ea / rho1 - P.sum(1) / eps)
        Hm[n:, n:] = torch.diag(-eb / rho2 - P.sum(0) / eps)
        Hm[:n, n:] = -P / eps
        Hm[n:, :n] = -P.T / eps
        step = -torch.linalg.solve(Hm, grad)
        t, F0 = 1.0, F(z)
        while F(z + t * step) < F0 + 0.25 * t * (grad @ step) and t > 1e-12:
            t *= 0.5
        z = z + t * step
    return z[:n], z[n:]


@pytest.mark.parametrize("seed,n,m,eps,rho1,rho2", [
    (0, 5, 4, 0.3, 0.7, 1.9),
    (1, 6, 6, 0.1, 2.0, 0.5),
    (2, 3, 6, 1.0, 0.2, 0.2),
    (3, 6, 2, 0.05, 5.0, 3.0),
])
def test_fixed_point_matches_newton_T12(seed, n, m, eps, rho1, rho2):
    p, C, a, b = tiny(n, m, 2, seed, eps, rho1, rho2)
    fN, gN = newton_dual(C, a, b, eps, rho1, rho2)
    ti = O.ti_sinkhorn(C, a, b, eps, rho1, rho2, 20000, tol=1e-14, check_every=5)
    fs = O.sinkhorn(C, a, b, eps, rho1, rho2, 200000, tol=1e-14, check_every=20)
    gs = O.g_sinkhorn(C, a, b, eps, rho1, rho2, 200000, tol=1e-14, check_every=20)
    for r in (ti, fs, gs):
        assert (r.f - fN).abs().max() < 1e-11
        assert (r.g - gN).abs().max() < 1e-11
    # value = primal = dual at the optimum, gap -> 0 (T4)
    D = O.dual_value(C, a, b, ti.f, ti.g, eps, rho1, rho2).item()
    P = O.primal_value(C, a, b, O.transport_plan(C, a, b, ti.f, ti.g, eps), eps, rho1, rho2).item()
    assert abs(D - P) < 1e-12 * max(1, abs(D))
    # optimal marginals pi1 = a e^{-f/rho1}, pi2 = b e^{-g/rho2}
    pi = O.transport_plan(C, a, b, ti.f, ti.g, eps)
    assert torch.allclose(pi.sum(1), a * torch.exp(-ti.f / rho1), atol=1e-12, rtol=0)
    assert torch.allclose(pi.sum(0), b * torch.exp(-ti.g / rho2), atol=1e-12, rtol=0)


def test_gap_decreases_along_iterations_T4():
    p = W.config1()
    C = O.cost_matrix(p.x, p.y)
    a, b = O._t(p.a), O._t(p.b)
    gaps = []
    for T in (5, 50, 400):
        r = O.ti_sinkhorn(C, a, b, p.eps, p.rho1, p.rho2, T)
        D = O.dual_value(C, a, b, r.f, r.g, p.eps, p.rho1, p.rho2).item()
        P = O.primal_value(C, a, b, O.transport_plan(C, a, b, r.f, r.g, p.eps), p.eps, p.rho1, p.rho2).item()
        assert P >= D - 1e-12           # weak duality
        gaps.append(P - D)
    assert gaps[0] > gaps[1] > gaps[2] and gaps[2] < 1e-9


def test_translation_decay_T2():
    """F-Sinkhorn from f* + tau decays as (rho1 rho2 / ((rho1+eps)(rho2+eps)))^t tau;
    H-Sinkhorn from fb_0 = f* + tau returns Phi = (f*, g*) after one iteration."""
    p, C, a, b = tiny(6, 5, 2, 7, 0.2, 0.9, 1.6)
    eps, r1, r2 = p.eps, p.rho1, p.rho2
    ref = O.ti_sinkhorn(C, a, b, eps, r1, r2, 5000, tol=1e-15, check_every=1)
    tau = 0.5
    f = ref.f + tau
    k = r1 * r2 / ((r1 + eps) * (r2 + eps))
    for t in range(1, 6):
        f, g = O.f_sinkhorn_iteration(C, a, b, f, eps, r1, r2)
        assert torch.allclose(f - ref.f, torch.full_like(f, k ** t * tau), atol=1e-12, rtol=0)
    fb, gb = O.h_sinkhorn_iteration(C, a, b, ref.f + tau, eps, r1, r2)
    f1, g1, _ = O.phi_map(a, b, fb, gb, r1, r2)
    assert (f1 - ref.f).abs().max() < 1e-12 and (g1 - ref.g).abs().max() < 1e-12


def test_rates_T10():
    """F-Sinkhorn rate -> (rho/(rho+eps))^2 per iteration; H-Sinkhorn is faster (Thm. 1)."""
    p = W.config1()
    C = O.cost_matrix(p.x, p.y)
    a, b = O._t(p.a), O._t(p.b)
    ref = O.ti_sinkhorn(C, a, b, p.eps, p.rho1, p.rho2, 3000, tol=1e-14, check_every=10)
    fr = O.sinkhorn(C, a, b, p.eps, p.rho1, p.rho2, 300, keep_iterates=True)
    hr = O.ti_sinkhorn(C, a, b, p.eps, p.rho1, p.rho2, 60, keep_iterates=True)
    ef = [(f - ref.f).abs().max().item() for _, f, _ in fr.history]
    eh = [(f - ref.f).abs().max().item() for _, f, _ in hr.history if (f - ref.f).abs().max() > 1e-12]
    kf = O.contraction_rate(ef[100:])
    kh = O.contraction_rate(eh)
    assert abs(kf - (p.rho1 / (p.rho1 + p.eps)) ** 2) < 2e-3
    assert kh < kf - 0.05


def test_contraction_rate_estimator():
    e = [3.0 * 0.9 ** t for t in range(30)]
    assert abs(O.contraction_rate(e) - 0.9) < 1e-12


def test_balanced_limit_T11():
    """Equal masses and rho -> infinity: potentials approach balanced Sinkhorn's (mod a constant)."""
    p = W.random_problem(7, 6, 1, seed=9, eps=0.1, mass_a=1.0, mass_b=1.0)
    C = O.cost_matrix(p.x, p.y)
    a, b = O._t(p.a), O._t(p.b)
    # balanced log-domain Sinkhorn written out here: f = Smin_b(C - g), g = Smin_a(C - f)
    f = torch.zeros(7, dtype=F64)
    for _ in range(5000):
        g = O.softmin(a, (C - f[:, None]).T, 0.1)
        f = O.softmin(b, C - g[None, :], 0.1)
    errs = []
    for rho in (1e2, 1e3, 1e4):
        r = O.ti_sinkhorn(C, a, b, 0.1, rho, rho, 20000, tol=1e-13, check_every=10)
        d = r.f - f
        errs.append((d - d.mean()).abs().max().item())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-4
    # ratio of successive errors ~ 1/10 (first order in 1/rho)
    assert 0.03 < errs[1] / errs[0] < 0.3


# ------------------------------------------------------------- gradients T13

def _solve_value(x, y, a, b, eps, r1, r2):
    C = O.cost_matrix(x, y)
    r = O.ti_sinkhorn(C, a, b, eps, r1, r2, 20000, tol=1e-14, check_every=5)
    return O.dual_value(C, a, b, r.f, r.g, eps, r1, r2).item(), r


def test_envelope_grads_vs_central_differences():
    p = W.random_problem(6, 5, 2, seed=11, eps=0.2, rho1=0.6, rho2=1.7, mass_a=1.2, mass_b=0.7)
    x, y, a, b = (O._t(v) for v in (p.x, p.y, p.a, p.b))
    val, r = _solve_value(x, y, a, b, p.eps, p.rho1, p.rho2)
    ga, gb, gx, gy = O.envelope_grads(x, y, a, b, r.f, r.g, p.eps, p.rho1, p.rho2)
    gen = torch.Generator().manual_seed(5)
    h = 1e-4
    for (var, grad) in (("a", ga), ("b", gb), ("x", gx), ("y", gy)):
        for _ in range(3):
            base = {"a": a, "b": b, "x": x, "y": y}
            v = base[var]
            u = torch.randn(v.shape, generator=gen, dtype=F64)
            if var in ("a", "b"):
                u = u * v           # relative step in the weights
            u = u / u.norm()
            vals = []
            for s in (+1, -1):
                args = dict(base)
                args[var] = v + s * h * u
                vals.append(_solve_value(args["x"], args["y"], args["a"], args["b"], p.eps, p.rho1, p.rho2)[0])
            fd = (vals[0] - vals[1]) / (2 * h)
            an = (grad * u).sum().item()
            assert abs(fd - an) < 1e-7 * max(1.0, abs(an)), (var, fd, an)


def test_unrolled_grads_vs_central_differences():
    p = W.random_problem(5, 4, 2, seed=12, eps=0.3, rho1=0.5, rho2=1.1, mass_a=1.0, mass_b=1.4)
    x, y, a, b = (O._t(v) for v in (p.x, p.y, p.a, p.b))
    T = 4
    val, ga, gb, gx, gy = O.unrolled_grads(x, y, a, b, p.eps, p.rho1, p.rho2, T)
    gen = torch.Generator().manual_seed(6)
    h = 1e-5
    for var, grad in (("a", ga), ("b", gb), ("x", gx), ("y", gy)):
        base = {"a": a, "b": b, "x": x, "y": y}
        v = base[var]
        u = torch.randn(v.shape, generator=gen, dtype=F64)
        u = u / u.norm()
        vals = []
        for s in (+1, -1):
            args = dict(base)
            args[var] = v + s * h * u
            vals.append(O.truncated_ti_value(args["x"], args["y"], args["a"], args["b"],
                                             p.eps, p.rho1, p.rho2, T).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        an = (grad * u).sum().item()
        assert abs(fd - an) < 1e-8 * max(1.0, abs(an)), (var, fd, an)


def test_unrolled_matches_envelope_when_converged():
    p = W.random_problem(5, 4, 1, seed=13, eps=0.5, rho1=0.5, rho2=0.5, mass_a=1.0, mass_b=2.0)
    x, y, a, b = (O._t(v) for v in (p.x, p.y, p.a, p.b))
    val, ga, gb, gx, gy = O.unrolled_grads(x, y, a, b, p.eps, p.rho1, p.rho2, 200)
    v2, r = _solve_value(x, y, a, b, p.eps, p.rho1, p.rho2)
    ea, eb, ex, ey = O.envelope_grads(x, y, a, b, r.f, r.g, p.eps, p.rho1, p.rho2)
    assert abs(val.item() - v2) < 1e-12
    for u, e in ((ga, ea), (gb, eb), (gx, ex), (gy, ey)):
        assert (u - e).abs().max() < 1e-9


def test_unrolled_grads_with_zero_weights_vs_one_sided_differences():
    """A zero weight keeps its derivative (the softmin is smooth in w_j at w_j = 0, Sec. 3 definition):
    autograd of the oracle agrees with a forward difference there."""
    p = W.random_problem(6, 5, 1, seed=14, eps=0.3, rho1=0.6, rho2=1.2, mass_a=1.0, mass_b=1.1, zero_frac=0.34)
    x, y, a, b = (O._t(v) for v in (p.x, p.y, p.a, p.b))
    T = 3
    val, ga, gb, gx, gy = O.unrolled_grads(x, y, a, b, p.eps, p.rho1, p.rho2, T)
    for w, g, name in ((a, ga, "a"), (b, gb, "b")):
        zeros = (w == 0).nonzero().flatten()
        assert zeros.numel() > 0
        for k in zeros.tolist():
            h = 1e-7
            w2 = w.clone()
            w2[k] = h
            args = {"a": a, "b": b, name: w2}
            fd = (O.truncated_ti_value(x, y, args["a"], args["b"], p.eps, p.rho1, p.rho2, T).item() - val.item()) / h
            assert abs(fd - g[k].item()) < 1e-5 * max(1.0, abs(fd)), (name, k, fd, g[k].item())


# ---- Anderson extrapolation (appendix, "Combining Sinkhorn with Anderson acceleration")

def test_anderson_weights_exact_on_a_linear_contraction():
    """For x_{k+1} = A x_k + b in R^3 and K = 4 residuals, the constrained minimiser has
    U c = 0, so sum_k c_k x_k is the fixed point (I - A)^{-1} b up to the regularisation."""
    rng = np.random.default_rng(0)
    for _ in range(5):
        d = 3
        A = rng.standard_normal((d, d))
        A = 0.7 * A / np.linalg.norm(A, 2)
        b = rng.standard_normal(d)
        xs = [rng.standard_normal(d)]
        for _k in range(4):
            xs.append(A @ xs[-1] + b)
        U = np.stack([xs[k + 1] - xs[k] for k in range(4)], axis=1)
        c = O.anderson_weights(torch.tensor(U), 1e-14).numpy()
        assert abs(c.sum() - 1.0) < 1e-12
        xe = sum(c[k] * xs[k] for k in range(4))
        assert np.abs(xe - np.linalg.solve(np.eye(d) - A, b)).max() < 1e-8


def test_anderson_weights_symmetric_and_regularised_limits():
    """Orthogonal residuals of equal norm: every weight is 1/K (symmetry).  A huge r makes
    G + r I ~ r I, so the weights tend to 1/K whatever U is; two identical
    residual directions of different lengths (a rank-deficient G) and a tiny r puts the
    weight on a combination with U c ~ 0."""
    U = np.eye(4) * 3.0
    assert np.allclose(O.anderson_weights(torch.tensor(U), 1e-7).numpy(), 0.25, atol=1e-12)
    rng = np.random.default_rng(1)
    U = rng.standard_normal((10, 4))
    assert np.allclose(O.anderson_weights(torch.tensor(U), 1e9).numpy(), 0.25, atol=1e-8)
    v = rng.standard_normal(6)
    U = np.stack([v, 2 * v, rng.standard_normal(6), rng.standard_normal(6)], axis=1)
    c = O.anderson_weights(torch.tensor(U), 1e-14).numpy()
    assert np.abs(U @ c).max() < 1e-5 * np.abs(U).max() and abs(c.sum() - 1) < 1e-12


@pytest.mark.parametrize("method", ["plain", "ti", "g"])
def test_anderson_without_extrapolation_is_the_base_solver(method):
    """K > n_iter: no block ever completes, and the iterates are those of the base solver."""
    pr = W.random_problem(40, 30, 1, seed=3, eps=0.05, rho1=0.7, rho2=1.3)
    C = O.cost_matrix(pr.x, pr.y)
    base = {"plain": O.sinkhorn, "ti": O.ti_sinkhorn, "g": O.g_sinkhorn}[method](
        C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, 12)
    acc = O.anderson_sinkhorn(C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, 12, method=method, K=50)
    assert torch.equal(acc.f, base.f) and torch.equal(acc.g, base.g)


@pytest.mark.parametrize("method", ["plain", "ti", "g"])
def test_anderson_same_fixed_point_in_fewer_iterations(method):
    """The appendix's claim on the 1-D problem (eps = 1e-2 << rho = 1): with K = 4,
    r = 1e-7 every variant reaches the same fixed point, to residual 1e-9, in fewer
    iterations than without extrapolation."""
    pr = W.config1()
    C = O.cost_matrix(pr.x, pr.y)
    base = {"plain": O.sinkhorn, "ti": O.ti_sinkhorn, "g": O.g_sinkhorn}[method](
        C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, 5000, tol=1e-9, check_every=10)
    acc = O.anderson_sinkhorn(C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, 5000, method=method, K=4, r=1e-7,
                              tol=1e-9, check_every=10)
    assert acc.residual <= 1e-9 and base.residual <= 1e-9
    assert acc.iters < base.iters
    assert (acc.f - base.f).abs().max().item() < 1e-6 and (acc.g - base.g).abs().max().item() < 1e-6
