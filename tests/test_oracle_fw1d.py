"""Pins of the 1-D Frank-Wolfe oracle (Sec. 4, Algs. 1-2) against things other than itself."""
import math

import numpy as np
import pytest
import torch

from oracle import fw1d as W
from oracle import uot as O

scipy_opt = pytest.importorskip("scipy.optimize")


def sorted_problem(n, m, seed, zeros=False, equal=True):
    rng = np.random.default_rng(seed)
    x = np.sort(rng.normal(0.0, 1.0, n))
    y = np.sort(rng.normal(0.3, 0.8, m))
    a = rng.exponential(1.0, n)
    b = rng.exponential(1.0, m)
    if zeros and n > 2:
        a[1] = 0.0
    if zeros and m > 3:
        b[-2] = 0.0
    if equal:
        b *= a.sum() / b.sum()
    return x, a, y, b


def lp_ot(C, a, b):
    """Balanced OT by scipy's HiGHS LP solver: min <pi, C> s.t. pi 1 = a, pi^T 1 = b, pi >= 0."""
    N, M = C.shape
    A_eq = np.zeros((N + M, N * M))
    for i in range(N):
        A_eq[i, i * M:(i + 1) * M] = 1.0
    for j in range(M):
        A_eq[N + j, j::M] = 1.0
    res = scipy_opt.linprog(C.ravel(), A_eq=A_eq, b_eq=np.concatenate([a, b]), bounds=(0, None), method="highs")
    assert res.status == 0
    return res.fun


@pytest.mark.parametrize("n,m", [(1, 1), (1, 4), (5, 1), (6, 5), (9, 13), (20, 7)])
@pytest.mark.parametrize("p", [1.0, 1.5, 2.0])
def test_solve_ot_1d_is_an_optimal_primal_dual_pair(n, m, p):
    x, a, y, b = sorted_problem(n, m, seed=10 * n + m, zeros=True)
    C = np.abs(x[:, None] - y[None, :]) ** p
    plan, f, g = W.solve_ot_1d(x, a, y, b, p)
    P = plan.numpy()
    # a coupling of a and b
    assert (P >= -1e-15).all()
    assert np.allclose(P.sum(1), a, atol=1e-12) and np.allclose(P.sum(0), b, atol=1e-12)
    cost = (P * C).sum()
    # optimal: equal to the LP optimum
    assert abs(cost - lp_ot(C, a, b)) <= 1e-9 * max(1.0, abs(cost))
    # dual feasible, complementary slack, and strong duality
    S = f.numpy()[:, None] + g.numpy()[None, :]
    assert (S <= C + 1e-12 * (1 + np.abs(C))).all()
    assert np.allclose(S[P > 1e-13], C[P > 1e-13], atol=1e-11)
    assert abs((f.numpy() * a).sum() + (g.numpy() * b).sum() - cost) <= 1e-10 * max(1.0, abs(cost))


@pytest.mark.parametrize("p", [1.0, 2.0, 3.0])
def test_solve_ot_1d_equal_counts_match_in_order(p):
    """Equal counts and uniform weights: the monotone (identity) matching, cost mean |x_i - y_i|^p."""
    rng = np.random.default_rng(4)
    x = np.sort(rng.uniform(-1, 1, 12))
    y = np.sort(rng.uniform(0, 2, 12))
    w = np.full(12, 1.0 / 12)
    plan, f, g = W.solve_ot_1d(x, w, y, w, p)
    assert torch.allclose(plan, torch.eye(12, dtype=torch.float64) / 12, atol=1e-15)
    cost = (plan.numpy() * np.abs(x[:, None] - y[None, :]) ** p).sum()
    assert abs(cost - np.mean(np.abs(x - y) ** p)) < 1e-14


def test_reweighted_histograms_have_equal_masses():
    """Prop. 1: at lambda*, <a~> = <b~>, so the LMO is a balanced problem."""
    x, a, y, b = sorted_problem(15, 11, seed=3, equal=False)
    rng = np.random.default_rng(9)
    fb, gb = rng.normal(0, 0.5, 15), rng.normal(0, 0.5, 11)
    for rho1, rho2 in [(0.1, 0.1), (1.0, 3.0), (10.0, 0.5)]:
        at, bt, _ = W.reweighted_histograms(a, b, fb, gb, rho1, rho2)
        assert abs(at.sum().item() - bt.sum().item()) < 1e-12 * at.sum().item()


@pytest.mark.parametrize("rho1,rho2", [(1.0, 1.0), (0.1, 2.0), (5.0, 0.3)])
def test_fw_one_point_closed_form(rho1, rho2):
    """N = M = 1: pi* = (a^rho1 b^rho2 e^{-c})^{1/(rho1+rho2)}, f* = -rho1 log(pi*/a), g* = c - f*."""
    x, y, a, b = [0.2], [1.1], [0.7], [1.9]
    c = (1.1 - 0.2) ** 2
    log_pi = (rho1 * math.log(0.7) + rho2 * math.log(1.9) - c) / (rho1 + rho2)
    f_star = -rho1 * (log_pi - math.log(0.7))
    res = W.fw_uot_1d(x, a, y, b, rho1, rho2, n_iter=3)
    assert abs(res.f.item() - f_star) < 1e-13
    assert abs(res.g.item() - (c - f_star)) < 1e-13


def primal_uot0(C, a, b, rho1, rho2):
    """Independent solver of the eps = 0 primal: L-BFGS-B over the plan's entries (kept >= 1e-14)."""
    N, M = C.shape

    def fun(v):
        P = v.reshape(N, M)
        p1, p2 = P.sum(1), P.sum(0)
        val = (P * C).sum() + rho1 * (p1 * np.log(p1 / a) - p1 + a).sum() + rho2 * (p2 * np.log(p2 / b) - p2 + b).sum()
        grad = C + rho1 * np.log(p1 / a)[:, None] + rho2 * np.log(p2 / b)[None, :]
        return val, grad.ravel()

    v0 = np.outer(a, b).ravel() / max(a.sum(), b.sum())
    res = scipy_opt.minimize(fun, v0, jac=True, method="L-BFGS-B", bounds=[(1e-14, None)] * (N * M),
                             options={"maxiter": 20000, "ftol": 1e-15, "gtol": 1e-12, "maxcor": 30})
    return res.fun


@pytest.mark.parametrize("rho", [0.5, 2.0])
def test_fw_reaches_the_primal_optimum(rho):
    """Strong duality at eps = 0: F_0 of the FW potentials rises to the primal optimum found by an
    independent solver, and never exceeds it (weak duality)."""
    x, a, y, b = sorted_problem(6, 5, seed=int(10 * rho), equal=False)
    C = np.abs(x[:, None] - y[None, :]) ** 2
    p_star = primal_uot0(C, a, b, rho, rho)
    res = W.fw_uot_1d(x, a, y, b, rho, rho, n_iter=400, step="linesearch", keep_history=True)
    d = W.f0_value(a, b, res.f, res.g, rho, rho).item()
    assert all(h <= p_star + 1e-9 for h in res.h_history)
    assert abs(d - p_star) < 1e-7 * max(1.0, abs(p_star))
    # the fixed step converges to the same value, more slowly
    res2 = W.fw_uot_1d(x, a, y, b, rho, rho, n_iter=2000)
    d2 = W.f0_value(a, b, res2.f, res2.g, rho, rho).item()
    assert d2 <= p_star + 1e-9 and abs(d2 - p_star) < 1e-4 * max(1.0, abs(p_star))


def test_linesearch_is_not_worse_than_the_fixed_step():
    """From the same iterate, the line-search step's H_0 is >= the 2/(2+t) step's."""
    x, a, y, b = sorted_problem(10, 8, seed=12, equal=False)
    rng = np.random.default_rng(2)
    for t in range(5):
        fb, gb = torch.tensor(rng.normal(0, 0.3, 10)), torch.tensor(rng.normal(0, 0.3, 8))
        at, bt, _ = W.reweighted_histograms(a, b, fb, gb, 1.0, 1.0)
        _, r, s = W.solve_ot_1d(x, at, y, bt, 2.0)
        gm = 2.0 / (2.0 + t)
        h_fixed = W.h0_value(a, b, (1 - gm) * fb + gm * r, (1 - gm) * gb + gm * s, 1.0, 1.0).item()
        gl = W._line_search(a, b, fb, gb, r, s, 1.0, 1.0)
        h_ls = W.h0_value(a, b, (1 - gl) * fb + gl * r, (1 - gl) * gb + gl * s, 1.0, 1.0).item()
        assert h_ls >= h_fixed - 1e-12


def test_h0_is_f0_at_the_optimal_translation():
    """H_0(fb, gb) = max over lambda of F_0(fb + lambda, gb - lambda), the maximiser being Prop. 2's."""
    x, a, y, b = sorted_problem(7, 9, seed=5, equal=False)
    rng = np.random.default_rng(1)
    fb, gb = rng.normal(0, 0.4, 7), rng.normal(0, 0.4, 9)
    h = W.h0_value(a, b, fb, gb, 0.7, 1.3).item()
    lams = np.linspace(-3, 3, 6001)
    vals = [W.f0_value(a, b, fb + l, gb - l, 0.7, 1.3).item() for l in lams[::20]]
    assert h >= max(vals) - 1e-12
    lam = O.lambda_star(a, b, fb, gb, 0.7, 1.3).item()
    for dl in (-1e-3, 1e-3):
        assert W.f0_value(a, b, fb + lam + dl, gb - lam - dl, 0.7, 1.3).item() <= h + 1e-15
