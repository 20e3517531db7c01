"""FP64 CPU oracle for 1-D unregularised UOT (eps = 0) by Frank-Wolfe on H_0.

TEST INFRASTRUCTURE ONLY.  Like oracle.uot, this module is the slow, plain
reference that the CUDA path is checked against; only the test suite, the
smoke check and the CPU-baseline leg of the benchmark may import it.  It shares
no code with the CUDA kernels or their bindings.

What it computes (Sejourne, Vialard, Peyre, AISTATS 2022, Sec. 4):

  * SolveOT1D (Alg. 1): exact balanced 1-D OT between sorted point sets with
    equal total masses, C_ij = |x_i - y_j|^p (p >= 1), by one pass over the
    two sorted lists (the north-west corner rule).  The dual potentials are
    set along the pass: f at the first point is 0, and each newly reached
    point's potential is the cost of the current pair minus the potential of
    the other side's current point.
  * Frank-Wolfe on H_0 (Alg. 2): (fb, gb) <- (1 - gamma_t)(fb, gb) + gamma_t (r_t, s_t),
    where (r_t, s_t) is SolveOT1D between the re-weighted histograms of
    Eq. (fw-updated-histo): for KL, grad phi_i^*(x) = e^{x / rho_i}, so
    a~ = a e^{-(fb + lambda*) / rho1} and b~ = b e^{-(gb - lambda*) / rho2},
    lambda* = lambda*(fb, gb) of Prop. 2 (which makes both masses equal,
    Prop. 1).  gamma_t = 2 / (2 + t), or a line search on H_0 along the step.
    The returned pair is Phi(fb, gb) = (fb + lambda*, gb - lambda*).

Reading of a garbled line (also in the design notes): Alg. 1's first branch
is printed with the test a >= b, but its body sends the remaining mass a of
point i to (i, j) and leaves b - a at point j, which needs a <= b.  The walk
advances i when a <= b (and always once j is the last point), j otherwise.

Parity status: SolveOT1D is pinned against scipy's LP solver, the identity
matching of equal-count uniform samples, and LP duality; Frank-Wolfe is pinned
against the closed form of the one-point problem and against an independent
primal solver of the eps = 0 problem (scipy L-BFGS-B on the plan); the line
search is pinned by never doing worse than the fixed step on H_0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

from oracle.uot import lambda_star

F64 = torch.float64


def _t(v) -> torch.Tensor:
    if isinstance(v, torch.Tensor):
        return v.to(device="cpu", dtype=F64)
    return torch.as_tensor(v, dtype=F64)


def cost_1d(xi: float, yj: float, p: float) -> float:
    """C_ij = |x_i - y_j|^p for scalars (Sec. 4, the 1-D costs of Alg. 1)."""
    d = abs(xi - yj)
    if p == 2.0:
        return d * d
    if p == 1.0:
        return d
    return d ** p


def solve_ot_1d(x, a, y, b, p: float = 2.0):
    """Alg. 1: balanced 1-D OT between sorted (x, a) and (y, b), sum a = sum b.

    Returns (plan, f, g): plan is the dense N x M coupling (for checking), f and
    g the dual potentials built along the pass.  Plain Python loop, O(N + M).
    """
    x, a, y, b = _t(x), _t(a), _t(y), _t(b)
    N, M = x.numel(), y.numel()
    xs, ys, av, bv = x.tolist(), y.tolist(), a.tolist(), b.tolist()
    plan = torch.zeros(N, M, dtype=F64)
    f = [0.0] * N
    g = [0.0] * M
    i, j = 0, 0
    f[0] = 0.0
    g[0] = cost_1d(xs[0], ys[0], p) - f[0]
    ma, mb = av[0], bv[0]  # mass of point i / point j not yet transported
    while i < N - 1 or j < M - 1:
        if (ma <= mb and i < N - 1) or j == M - 1:
            # point i is exhausted first: its remaining mass goes to (i, j)
            plan[i, j] += ma
            mb -= ma
            i += 1
            f[i] = cost_1d(xs[i], ys[j], p) - g[j]
            ma = av[i]
        else:
            plan[i, j] += mb
            ma -= mb
            j += 1
            g[j] = cost_1d(xs[i], ys[j], p) - f[i]
            mb = bv[j]
    plan[N - 1, M - 1] += ma  # the last pair takes what is left (equal to mb up to rounding)
    return plan, torch.tensor(f, dtype=F64), torch.tensor(g, dtype=F64)


def reweighted_histograms(a, b, fb, gb, rho1: float, rho2: float):
    """Eq. (fw-updated-histo) for KL: a~ = a e^{-(fb + lambda*)/rho1}, b~ = b e^{-(gb - lambda*)/rho2}."""
    a, b, fb, gb = _t(a), _t(b), _t(fb), _t(gb)
    lam = lambda_star(a, b, fb, gb, rho1, rho2)
    at = a * torch.exp(-(fb + lam) / rho1)
    bt = b * torch.exp(-(gb - lam) / rho2)
    return at, bt, lam


def f0_value(a, b, f, g, rho1: float, rho2: float) -> torch.Tensor:
    """Dual objective at eps = 0 (Sec. 1, F_0): <a, rho1 (1 - e^{-f/rho1})> + <b, rho2 (1 - e^{-g/rho2})>."""
    a, b, f, g = _t(a), _t(b), _t(f), _t(g)
    return (a * rho1 * (1.0 - torch.exp(-f / rho1))).sum() + (b * rho2 * (1.0 - torch.exp(-g / rho2))).sum()


def h0_value(a, b, fb, gb, rho1: float, rho2: float) -> torch.Tensor:
    """H_0(fb, gb) = F_0(fb + lambda*, gb - lambda*) (Sec. 2, definition of H)."""
    lam = lambda_star(a, b, fb, gb, rho1, rho2)
    return f0_value(a, b, _t(fb) + lam, _t(gb) - lam, rho1, rho2)


def primal_value_0(C, a, b, plan, rho1: float, rho2: float) -> torch.Tensor:
    """Primal UOT objective at eps = 0: <pi, C> + rho1 KL(pi_1 | a) + rho2 KL(pi_2 | b) (Sec. 1)."""
    from oracle.uot import kl_div

    C, a, b, plan = _t(C), _t(a), _t(b), _t(plan)
    return (plan * C).sum() + rho1 * kl_div(plan.sum(1), a) + rho2 * kl_div(plan.sum(0), b)


def _line_search(a, b, fb, gb, r, s, rho1, rho2, iters: int = 80) -> float:
    """gamma in [0, 1] maximising the concave gamma -> H_0 on the segment, by golden-section search."""
    def h(gm):
        return h0_value(a, b, (1 - gm) * fb + gm * r, (1 - gm) * gb + gm * s, rho1, rho2).item()

    lo, hi = 0.0, 1.0
    q = (math.sqrt(5.0) - 1.0) / 2.0
    c, d = hi - q * (hi - lo), lo + q * (hi - lo)
    hc, hd = h(c), h(d)
    for _ in range(iters):
        if hc >= hd:
            hi, d, hd = d, c, hc
            c = hi - q * (hi - lo)
            hc = h(c)
        else:
            lo, c, hc = c, d, hd
            d = lo + q * (hi - lo)
            hd = h(d)
    best = max((h(0.0), 0.0), (h(1.0), 1.0), (h(0.5 * (lo + hi)), 0.5 * (lo + hi)))
    return best[1]


@dataclass
class FWResult:
    f: torch.Tensor            # Phi(fb, gb), first component
    g: torch.Tensor
    fb: torch.Tensor           # the Frank-Wolfe iterate itself
    gb: torch.Tensor
    lam: float
    h_history: list = field(default_factory=list)   # H_0 of the iterate after each step
    last_plan: torch.Tensor | None = None             # the last LMO's coupling


def fw_uot_1d(x, a, y, b, rho1: float, rho2: float, n_iter: int, p: float = 2.0, step: str = "fixed",
              fb0=None, gb0=None, keep_history: bool = False) -> FWResult:
    """Alg. 2 on sorted 1-D inputs; step "fixed" (gamma_t = 2/(2+t)) or "linesearch"."""
    x, a, y, b = _t(x), _t(a), _t(y), _t(b)
    fb = torch.zeros_like(a) if fb0 is None else _t(fb0).clone()
    gb = torch.zeros_like(b) if gb0 is None else _t(gb0).clone()
    hist = []
    plan = None
    for t in range(n_iter):
        at, bt, _ = reweighted_histograms(a, b, fb, gb, rho1, rho2)
        plan, r, s = solve_ot_1d(x, at, y, bt, p)
        if step == "fixed":
            gm = 2.0 / (2.0 + t)
        elif step == "linesearch":
            gm = _line_search(a, b, fb, gb, r, s, rho1, rho2)
        else:
            raise ValueError(step)
        fb = (1.0 - gm) * fb + gm * r
        gb = (1.0 - gm) * gb + gm * s
        if keep_history:
            hist.append(h0_value(a, b, fb, gb, rho1, rho2).item())
    lam = lambda_star(a, b, fb, gb, rho1, rho2)
    return FWResult(fb + lam, gb - lam, fb, gb, float(lam), hist, plan)
