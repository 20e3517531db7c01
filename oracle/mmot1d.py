"""FP64 CPU oracle for 1-D unbalanced multi-marginal OT and UOT barycenters (Sec. 5).

TEST INFRASTRUCTURE ONLY.  Like oracle.uot and oracle.fw1d, this is the slow,
plain reference for the CUDA path; only the test suite, the smoke check and
the CPU-baseline leg of the benchmark may import it, and it shares no code
with the kernels or their bindings.

What it computes (Sejourne, Vialard, Peyre, AISTATS 2022, Sec. 5), for K
measures (x_k, alpha_k) on the line with sorted points, weights omega_k >= 0
summing to one, and the squared-distance ground cost c(x, y) = |x - y|^2:

  * multi-marginal cost C(z_1..z_K) = min_b sum_k omega_k c(z_k, b)
    = sum_k omega_k (z_k - B(z))^2 with the barycentric map B(z) = sum_k omega_k z_k
    (Eq. EqCostMultiMarginal);
  * SolveMOT (Alg. 3): balanced multi-marginal OT between sorted measures of
    equal mass by one pass: the measure whose current point has the least
    remaining mass moves to its next point, every measure's remaining mass
    drops by that amount, and the new point's potential is the cost of the
    current index tuple minus the other measures' current potentials;
  * the optimal translation of the K-marginal dual for rho KL (Prop. "KL
    setting" after Prop. prop-optim-trans-multimarg):
    q_k = log <alpha_k, e^{-f_k / (omega_k rho)}>,
    lambda_k = omega_k rho q_k - omega_k / (sum_l omega_l) sum_l omega_l rho q_l;
  * Frank-Wolfe on the translation-invariant functional H: fb <- (1 - tau_t) fb + tau_t r,
    r = SolveMOT between the re-weighted measures
    alpha~_k = alpha_k e^{-(fb_k + lambda_k) / (omega_k rho)}, tau_t = 2 / (2 + t);
  * the barycenter of Prop. prop:barycentermulti: points B(x_(1,i_1), .., x_(K,i_K))
    over the support of the plan, with the plan's masses as weights.

Readings (also in the design notes): Alg. 3 moves the measure p with the
smallest remaining mass among those not at their last point and leaves the
last index tuple with the mass that is left; the paper's "tilde alpha_k =
grad phi_k^*(-fb_k - lambda_k)" is read with the weight alpha_k and the 1/omega_k
scaling that the dual Eq. (eq-dual-multimarg) puts on the potentials.

Parity status: SolveMOT is pinned against scipy's LP solver on the full
K-tensor and LP duality, against the two-marginal walk at K = 2, and against
the closed-form 1-D W2 barycenter (quantile averaging) in the balanced case;
lambda* against Prop. 2 at K = 2, the equal-mass property and a direct
maximisation; Frank-Wolfe against the two-marginal FW oracle at K = 2 and an
independent primal solver at K = 3.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

F64 = torch.float64


def _t(v) -> torch.Tensor:
    if isinstance(v, torch.Tensor):
        return v.to(device="cpu", dtype=F64)
    return torch.as_tensor(v, dtype=F64)


def mm_cost(zs, w) -> float:
    """C(z_1..z_K) = sum_k omega_k (z_k - B(z))^2, B(z) = sum_k omega_k z_k (squared distance)."""
    b = sum(wk * zk for wk, zk in zip(w, zs))
    return sum(wk * (zk - b) ** 2 for wk, zk in zip(w, zs))


def barycentric_map(zs, w) -> float:
    """B(z) = argmin_b sum_k omega_k |z_k - b|^2 = sum_k omega_k z_k."""
    return sum(wk * zk for wk, zk in zip(w, zs))


def solve_mot_1d(xs, alphas, w):
    """Alg. 3: returns (plan, fs) with plan a list of (index tuple, mass) and fs the K dual potentials."""
    xs = [_t(x).tolist() for x in xs]
    al = [_t(a).tolist() for a in alphas]
    K = len(xs)
    N = [len(x) for x in xs]
    f = [[0.0] * n for n in N]
    idx = [0] * K
    rem = [al[k][0] for k in range(K)]
    f[0][0] = mm_cost([xs[k][0] for k in range(K)], w)
    plan = []
    while any(idx[k] < N[k] - 1 for k in range(K)):
        movable = [k for k in range(K) if idx[k] < N[k] - 1]
        p = min(movable, key=lambda k: (rem[k], k))
        mass = rem[p]
        plan.append((tuple(idx), mass))
        rem = [rem[k] - mass for k in range(K)]
        idx[p] += 1
        c = mm_cost([xs[k][idx[k]] for k in range(K)], w)
        f[p][idx[p]] = c - sum(f[k][idx[k]] for k in range(K) if k != p)
        rem[p] = al[p][idx[p]]
    plan.append((tuple(idx), rem[0]))  # the last tuple takes what is left
    return plan, [torch.tensor(fk, dtype=F64) for fk in f]


def plan_marginals(plan, N):
    """The K marginals of a sparse plan."""
    out = [torch.zeros(n, dtype=F64) for n in N]
    for tup, m in plan:
        for k, i in enumerate(tup):
            out[k][i] += m
    return out


def lambda_star_mm(alphas, fs, w, rho: float) -> torch.Tensor:
    """Optimal translation of the K-marginal rho KL dual (sum_k lambda_k = 0)."""
    q = []
    for a, f, wk in zip(alphas, fs, w):
        a, f = _t(a), _t(f)
        live = a > 0
        z = -f[live] / (wk * rho)
        m = z.max()
        q.append((m + torch.log((a[live] * torch.exp(z - m)).sum())).item())
    q = torch.tensor(q, dtype=F64)
    wt = _t(w)
    return wt * rho * q - wt / wt.sum() * (wt * rho * q).sum()


def dual_value_mm(alphas, fs, w, rho: float) -> torch.Tensor:
    """F(f) = sum_k <alpha_k, omega_k rho (1 - e^{-f_k / (omega_k rho)})> (Eq. eq-dual-multimarg, rho KL)."""
    return sum((_t(a) * wk * rho * (1.0 - torch.exp(-_t(f) / (wk * rho)))).sum() for a, f, wk in zip(alphas, fs, w))


def primal_value_mm(xs, alphas, w, rho: float, plan) -> torch.Tensor:
    """<gamma, C> + sum_k omega_k rho KL(gamma_k | alpha_k) (Eq. eq-multimarg) for a sparse plan."""
    from oracle.uot import kl_div

    xs = [_t(x).tolist() for x in xs]
    cost = sum(m * mm_cost([xs[k][i] for k, i in enumerate(tup)], w) for tup, m in plan)
    margs = plan_marginals(plan, [len(x) for x in xs])
    return torch.tensor(cost, dtype=F64) + sum(wk * rho * kl_div(g, _t(a)) for g, a, wk in zip(margs, alphas, w))


def reweighted(alphas, fbs, w, rho: float):
    lam = lambda_star_mm(alphas, fbs, w, rho)
    at = [_t(a) * torch.exp(-(_t(f) + lam[k]) / (w[k] * rho)) for k, (a, f) in enumerate(zip(alphas, fbs))]
    return at, lam


@dataclass
class MMResult:
    fs: list          # translated potentials fb_k + lambda_k
    fbs: list         # Frank-Wolfe iterate
    lam: torch.Tensor
    plan: list        # the last LMO's plan (between the re-weighted measures)
    bary_points: torch.Tensor
    bary_weights: torch.Tensor


def barycenter_from_plan(xs, plan, w):
    xs = [_t(x).tolist() for x in xs]
    pts = [barycentric_map([xs[k][i] for k, i in enumerate(tup)], w) for tup, m in plan if m > 0]
    wts = [m for tup, m in plan if m > 0]
    return torch.tensor(pts, dtype=F64), torch.tensor(wts, dtype=F64)


def fw_barycenter_1d(xs, alphas, w, rho: float, n_iter: int) -> MMResult:
    """Frank-Wolfe on H for the unbalanced multi-marginal problem (Sec. 5), tau_t = 2 / (2 + t)."""
    fbs = [torch.zeros(len(_t(x)), dtype=F64) for x in xs]
    plan = None
    for t in range(n_iter):
        at, _ = reweighted(alphas, fbs, w, rho)
        plan, r = solve_mot_1d(xs, at, w)
        tau = 2.0 / (2.0 + t)
        fbs = [(1.0 - tau) * fb + tau * rk for fb, rk in zip(fbs, r)]
    lam = lambda_star_mm(alphas, fbs, w, rho)
    fs = [fb + lam[k] for k, fb in enumerate(fbs)]
    # the barycenter from the LMO plan at the final iterate (its marginals are the optimal ones at convergence)
    at, _ = reweighted(alphas, fbs, w, rho)
    plan, _ = solve_mot_1d(xs, at, w)
    pts, wts = barycenter_from_plan(xs, plan, w)
    return MMResult(fs, fbs, lam, plan, pts, wts)
