"""Pins of the 1-D multi-marginal / barycenter oracle (Sec. 5, Alg. 3) against things other than itself."""
import itertools

import numpy as np
import pytest
import torch

from oracle import fw1d as FW
from oracle import mmot1d as MM
from oracle import uot as O

scipy_opt = pytest.importorskip("scipy.optimize")


def measures(sizes, seed, equal=True):
    rng = np.random.default_rng(seed)
    xs, als = [], []
    for k, n in enumerate(sizes):
        xs.append(np.sort(rng.normal(0.3 * k, 1.0, n)))
        a = rng.exponential(1.0, n)
        als.append(a / a.sum() if equal else a)
    return xs, als


def dense_cost(xs, w):
    shape = [len(x) for x in xs]
    C = np.zeros(shape)
    for tup in itertools.product(*[range(n) for n in shape]):
        C[tup] = MM.mm_cost([xs[k][i] for k, i in enumerate(tup)], w)
    return C


def lp_mot(C, als):
    """Balanced multi-marginal OT by scipy's HiGHS LP solver on the full tensor."""
    shape = C.shape
    nv = C.size
    rows, rhs = [], []
    for k, n in enumerate(shape):
        for i in range(n):
            sel = np.zeros(shape)
            idx = [slice(None)] * len(shape)
            idx[k] = i
            sel[tuple(idx)] = 1.0
            rows.append(sel.ravel())
            rhs.append(als[k][i])
    res = scipy_opt.linprog(C.ravel(), A_eq=np.array(rows), b_eq=np.array(rhs), bounds=(0, None), method="highs")
    assert res.status == 0
    return res.fun


@pytest.mark.parametrize("sizes,w", [((3, 4, 2), (0.2, 0.5, 0.3)), ((1, 5, 3), (1 / 3, 1 / 3, 1 / 3)),
                                     ((4, 4, 4, 2), (0.1, 0.2, 0.3, 0.4)), ((6, 1), (0.5, 0.5))])
def test_solve_mot_is_an_optimal_primal_dual_pair(sizes, w):
    xs, als = measures(sizes, seed=sum(sizes))
    plan, fs = MM.solve_mot_1d(xs, als, w)
    margs = MM.plan_marginals(plan, list(sizes))
    for g, a in zip(margs, als):
        assert np.allclose(g.numpy(), a, atol=1e-12)
    assert all(m >= -1e-15 for _, m in plan)
    C = dense_cost(xs, w)
    cost = sum(m * C[tup] for tup, m in plan)
    assert abs(cost - lp_mot(C, als)) <= 1e-9 * max(1.0, abs(cost))
    S = np.zeros(C.shape)
    for k, f in enumerate(fs):
        shape = [1] * len(sizes)
        shape[k] = sizes[k]
        S = S + f.numpy().reshape(shape)
    assert (S <= C + 1e-12 * (1 + np.abs(C))).all()
    for tup, m in plan:
        if m > 1e-13:
            assert abs(S[tup] - C[tup]) < 1e-11
    assert abs(sum((f.numpy() * a).sum() for f, a in zip(fs, als)) - cost) <= 1e-10 * max(1.0, abs(cost))


def test_solve_mot_two_marginals_is_solve_ot_1d():
    """K = 2: C = omega_1 omega_2 |x - y|^2, and Alg. 3 is Alg. 1 with its duals translated."""
    xs, als = measures((7, 5), seed=3)
    w = (0.3, 0.7)
    c0 = w[0] * w[1]
    plan, (F1, F2) = MM.solve_mot_1d(xs, als, w)
    P2, f, g = FW.solve_ot_1d(xs[0], als[0], xs[1], als[1], 2.0)
    dense = torch.zeros(7, 5, dtype=torch.float64)
    for (i, j), m in plan:
        dense[i, j] += m
    assert torch.allclose(dense, P2, atol=1e-15)
    t = F1[0].item()
    assert torch.allclose(F1 - t, c0 * (f - f[0]), atol=1e-13)
    assert torch.allclose(F2 + t, c0 * g, atol=1e-13)


def quantile_average(xs, als, w):
    """The 1-D W2 barycenter in closed form: quantile function sum_k omega_k Q_k (Agueh-Carlier in 1-D),
    returned as atoms (points, masses) over the merged breakpoints of the K cumulative distributions."""
    cums = [np.cumsum(a) for a in als]
    br = np.unique(np.concatenate([[0.0]] + [c[:-1] for c in cums] + [[1.0]]))
    pts, ms = [], []
    for lo, hi in zip(br[:-1], br[1:]):
        if hi - lo <= 1e-15:
            continue
        u = 0.5 * (lo + hi)
        q = [x[min(np.searchsorted(c, u), len(x) - 1)] for x, c in zip(xs, cums)]
        pts.append(sum(wk * qk for wk, qk in zip(w, q)))
        ms.append(hi - lo)
    return np.array(pts), np.array(ms)


def test_balanced_barycenter_is_the_quantile_average():
    """Balanced case: the barycenter of Prop. prop:barycentermulti from Alg. 3's plan equals the closed-form
    1-D W2 barycenter, and the plan's cost equals sum_k omega_k W2^2(alpha_k, barycenter)."""
    xs, als = measures((9, 6, 11), seed=8)
    w = (0.25, 0.45, 0.3)
    plan, _ = MM.solve_mot_1d(xs, als, w)
    pts, wts = MM.barycenter_from_plan(xs, plan, w)
    qp, qm = quantile_average(xs, als, w)
    # compare as distributions: CDFs at every atom of either
    grid = np.union1d(pts.numpy(), qp)
    cdf = lambda p, m: np.array([m[p <= g + 1e-13].sum() for g in grid])
    assert np.allclose(cdf(pts.numpy(), wts.numpy()), cdf(qp, qm), atol=1e-12)
    cost = sum(m * MM.mm_cost([xs[k][i] for k, i in enumerate(tup)], w) for tup, m in plan)

    def w2sq(x, a, p, m):
        # 1-D W2^2 by the quantile integral over merged breakpoints
        ca, cm = np.cumsum(a), np.cumsum(m)
        br = np.unique(np.concatenate([[0.0], ca, cm]))
        tot = 0.0
        for lo, hi in zip(br[:-1], br[1:]):
            u = 0.5 * (lo + hi)
            qa = x[min(np.searchsorted(ca, u), len(x) - 1)]
            qb = p[min(np.searchsorted(cm, u), len(p) - 1)]
            tot += (hi - lo) * (qa - qb) ** 2
        return tot

    order = np.argsort(qp)
    obj = sum(wk * w2sq(x, a, qp[order], qm[order]) for wk, x, a in zip(w, xs, als))
    assert abs(cost - obj) < 1e-12


def test_lambda_star_two_marginals_is_prop2():
    """K = 2 with rho KL: lambda = (l, -l), l = Prop. 2's lambda* with rho_k = omega_k rho."""
    xs, als = measures((8, 6), seed=5, equal=False)
    rng = np.random.default_rng(4)
    fs = [rng.normal(0, 0.5, 8), rng.normal(0, 0.5, 6)]
    for w, rho in [((0.5, 0.5), 1.0), ((0.2, 0.8), 3.0)]:
        lam = MM.lambda_star_mm(als, fs, w, rho)
        ref = O.lambda_star(als[0], als[1], fs[0], fs[1], w[0] * rho, w[1] * rho).item()
        assert abs(lam[0].item() - ref) < 1e-12 and abs(lam[1].item() + ref) < 1e-12


def test_lambda_star_multi_equal_masses_and_maximality():
    """K = 4: the re-weighted measures have equal masses (Prop. prop-optim-trans-multimarg), the translation
    sums to zero, and no zero-sum perturbation increases the dual."""
    xs, als = measures((5, 7, 3, 6), seed=9, equal=False)
    rng = np.random.default_rng(6)
    fs = [torch.tensor(rng.normal(0, 0.4, len(x))) for x in xs]
    w, rho = (0.1, 0.4, 0.2, 0.3), 0.7
    at, lam = MM.reweighted(als, fs, w, rho)
    masses = [a.sum().item() for a in at]
    assert max(masses) - min(masses) < 1e-12 * max(masses)
    assert abs(lam.sum().item()) < 1e-12
    best = MM.dual_value_mm(als, [f + lam[k] for k, f in enumerate(fs)], w, rho).item()
    for _ in range(20):
        d = torch.tensor(rng.normal(0, 0.05, 4))
        d -= d.mean()
        v = MM.dual_value_mm(als, [f + lam[k] + d[k] for k, f in enumerate(fs)], w, rho).item()
        assert v <= best + 1e-13


def test_fw_two_marginals_is_the_two_measure_fw():
    """K = 2: FW on H for the multi-marginal problem is Alg. 2 with rho_k = omega_k rho and the cost
    omega_1 omega_2 |x - y|^2 (points scaled by sqrt(omega_1 omega_2))."""
    xs, als = measures((12, 9), seed=13, equal=False)
    w, rho = (0.35, 0.65), 0.8
    res = MM.fw_barycenter_1d(xs, als, w, rho, n_iter=40)
    s = np.sqrt(w[0] * w[1])
    ref = FW.fw_uot_1d(s * xs[0], als[0], s * xs[1], als[1], w[0] * rho, w[1] * rho, 40, 2.0)
    assert torch.allclose(res.fs[0], ref.f, atol=1e-11)
    assert torch.allclose(res.fs[1], ref.g, atol=1e-11)


def primal_mm(xs, als, w, rho):
    """Independent solver of the unbalanced multi-marginal primal: L-BFGS-B over the dense tensor."""
    C = dense_cost(xs, w)
    shape = C.shape
    K = len(shape)

    def fun(v):
        G = v.reshape(shape)
        val = (G * C).sum()
        grad = C.copy()
        for k in range(K):
            axes = tuple(a for a in range(K) if a != k)
            gk = G.sum(axis=axes)
            val += w[k] * rho * (gk * np.log(gk / als[k]) - gk + als[k]).sum()
            sh = [1] * K
            sh[k] = shape[k]
            grad = grad + (w[k] * rho * np.log(gk / als[k])).reshape(sh)
        return val, grad.ravel()

    v0 = np.full(C.size, 1.0 / C.size)
    res = scipy_opt.minimize(fun, v0, jac=True, method="L-BFGS-B", bounds=[(1e-14, None)] * C.size,
                             options={"maxiter": 50000, "ftol": 1e-15, "gtol": 1e-12, "maxcor": 30})
    return res.fun


def test_fw_barycenter_reaches_the_primal_optimum():
    """K = 3: the dual value of the FW potentials rises to the primal optimum of Eq. (eq-multimarg) found by an
    independent solver, never above it."""
    xs, als = measures((4, 3, 3), seed=21, equal=False)
    w, rho = (0.3, 0.3, 0.4), 0.6
    p_star = primal_mm(xs, als, w, rho)
    vals = []
    fbs = [torch.zeros(len(x), dtype=torch.float64) for x in xs]
    for t in range(3000):
        at, _ = MM.reweighted(als, fbs, w, rho)
        _, r = MM.solve_mot_1d(xs, at, w)
        tau = 2.0 / (2.0 + t)
        fbs = [(1 - tau) * fb + tau * rk for fb, rk in zip(fbs, r)]
        if t % 300 == 299:
            lam = MM.lambda_star_mm(als, fbs, w, rho)
            vals.append(MM.dual_value_mm(als, [fb + lam[k] for k, fb in enumerate(fbs)], w, rho).item())
    assert all(v <= p_star + 1e-9 for v in vals)
    assert abs(vals[-1] - p_star) < 1e-4 * max(1.0, abs(p_star))
    res = MM.fw_barycenter_1d(xs, als, w, rho, n_iter=3000)
    assert abs(MM.dual_value_mm(als, res.fs, w, rho).item() - vals[-1]) < 1e-12
    # the barycenter's mass is the common mass of the re-weighted measures
    at, _ = MM.reweighted(als, res.fbs, w, rho)
    assert abs(res.bary_weights.sum().item() - at[0].sum().item()) < 1e-12
