"""FP64 CPU oracle for F- and G-Sinkhorn with a general smooth phi^* (Sec. 3).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the slow, plain reference
for the CUDA path, imported only by the test suite, the smoke check and the
CPU-baseline leg of the benchmark; it shares no code with the kernels.

G-Sinkhorn applies to any divergence whose conjugate phi^* is smooth
(Sec. 3); the paper demonstrates it with the Berg entropy
phi(x) = rho (x - 1 - log x), phi^*(q) = -rho log(1 - q/rho) (q < rho), next to
rho KL, phi^*(q) = rho (e^{q/rho} - 1).  For these the oracle computes:

  * the anisotropic prox aprox_{phi^*}(x) = argmin_y eps e^{(x - y)/eps} + phi^*(y)
    (Sec. 3), as the root of (x - y)/eps = log phi^*'(y) (strictly decreasing in
    y), found by scipy's brentq inside a bracket grown until it changes sign;
  * lambda*(fb, gb) = argmax_lambda <a, -phi_1^*(-fb - lambda)> + <b, -phi_2^*(-gb + lambda)>
    (Prop. 1; the entropic term does not depend on lambda) by Newton's method
    on the concave 1-D function, whose gradient and Hessian cost O(N + M) (Sec. 3),
    damped to stay in the domain and to increase the objective;
  * F-Sinkhorn: g <- -aprox_2(-Smin_a^eps(C - f)), f <- -aprox_1(-Smin_b^eps(C - g));
  * G-Sinkhorn: gb <- -aprox_2(-Smin_a^eps(C - fb - lambda)) + lambda,
    fb <- -aprox_1(-Smin_b^eps(C - gb + lambda)) - lambda, lambda <- lambda*(fb, gb),
    returning (fb + lambda, gb - lambda);
  * the dual F_eps(f, g) = <a, -phi_1^*(-f)> + <b, -phi_2^*(-g)> - eps <a (x) b, e^{(f (+) g - C)/eps} - 1>.

The pairing is the rest of the oracle's: f with (a, rho1), g with (b, rho2).

Parity status: the prox is pinned against rho/(rho + eps) x for KL and against
the Lambert-W closed form for Berg; lambda* against Prop. 2 for KL and against
an independent root of its derivative (equal masses) for Berg; F- and
G-Sinkhorn for KL against oracle.uot's iterates; for Berg, both reach the
maximiser of F_eps found by an independent solver, where the first-order
conditions hold.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from oracle.uot import smin_cols, smin_rows

F64 = torch.float64


def _t(v) -> torch.Tensor:
    if isinstance(v, torch.Tensor):
        return v.to(device="cpu", dtype=F64)
    return torch.as_tensor(v, dtype=F64)


@dataclass
class KL:
    """rho KL: phi^*(q) = rho (e^{q/rho} - 1) on all of R."""
    rho: float
    upper: float = math.inf

    def phi_star(self, q):
        return self.rho * (torch.exp(_t(q) / self.rho) - 1.0)

    def log_dphi_star(self, q: float) -> float:
        return q / self.rho

    def dphi_star(self, q):
        return torch.exp(_t(q) / self.rho)

    def d2phi_star(self, q):
        return torch.exp(_t(q) / self.rho) / self.rho


@dataclass
class Berg:
    """Berg entropy: phi^*(q) = -rho log(1 - q/rho) for q < rho."""
    rho: float

    @property
    def upper(self) -> float:
        return self.rho

    def phi_star(self, q):
        return -self.rho * torch.log1p(-_t(q) / self.rho)

    def log_dphi_star(self, q: float) -> float:
        return math.log(self.rho) - math.log(self.rho - q)

    def dphi_star(self, q):
        return self.rho / (self.rho - _t(q))

    def d2phi_star(self, q):
        return self.rho / (self.rho - _t(q)) ** 2


def aprox(div, x, eps: float) -> torch.Tensor:
    """aprox_{phi^*}(x) elementwise: the root y of (x - y)/eps - log phi^*'(y) (decreasing in y)."""
    from scipy.optimize import brentq

    out = []
    for xi in _t(x).reshape(-1).tolist():
        h = lambda y: (xi - y) / eps - div.log_dphi_star(y)
        lo, step = min(xi, 0.0) - 1.0, 1.0
        if div.upper < math.inf:
            lo = min(lo, div.upper - 1.0)
        while h(lo) <= 0.0:
            step *= 2.0
            lo -= step
        if div.upper < math.inf:
            d = min(1.0, (div.upper - lo) / 2.0)
            hi = div.upper - d
            while hi < div.upper and h(hi) >= 0.0:
                d /= 2.0
                hi = div.upper - d
            if hi >= div.upper:
                # the root lies above the largest double below the bound: that double is the rounded root
                out.append(math.nextafter(div.upper, -math.inf))
                continue
        else:
            hi, step = max(xi, 0.0) + 1.0, 1.0
            while h(hi) >= 0.0:
                step *= 2.0
                hi += step
        out.append(brentq(h, lo, hi, xtol=1e-300, rtol=4 * 2.0 ** -52, maxiter=500))
    return torch.tensor(out, dtype=F64).reshape(_t(x).shape)


def neg_conj(div, f) -> torch.Tensor:
    """-phi^*(-f), the marginal term of the dual."""
    return -div.phi_star(-_t(f))


def lambda_star(a, b, fb, gb, div1, div2, iters: int = 100) -> torch.Tensor:
    """argmax over lambda of <a, -phi_1^*(-fb - lambda)> + <b, -phi_2^*(-gb + lambda)> by damped Newton."""
    a, b, fb, gb = _t(a), _t(b), _t(fb), _t(gb)
    la, lb = a > 0, b > 0
    fa, gbb, aa, bb = fb[la], gb[lb], a[la], b[lb]
    # domain: -fb - lambda < upper_1 and -gb + lambda < upper_2 on the live entries
    lo = -math.inf if div1.upper == math.inf else (-div1.upper - fa.min()).item()
    hi = math.inf if div2.upper == math.inf else (div2.upper + gbb.min()).item()

    def obj(l):
        return (aa * neg_conj(div1, fa + l)).sum().item() + (bb * neg_conj(div2, gbb - l)).sum().item()

    def grad(l):
        return (aa * div1.dphi_star(-fa - l)).sum().item() - (bb * div2.dphi_star(-gbb + l)).sum().item()

    def hess(l):
        return -(aa * div1.d2phi_star(-fa - l)).sum().item() - (bb * div2.d2phi_star(-gbb + l)).sum().item()

    lam = 0.0
    if not (lo < lam < hi):
        lam = 0.5 * (lo + hi) if (lo > -math.inf and hi < math.inf) else (lo + 1.0 if hi == math.inf else hi - 1.0)
    for _ in range(iters):
        g, h = grad(lam), hess(lam)
        step = -g / h
        nxt = lam + step
        t = 1.0
        while not (lo < nxt < hi) or obj(nxt) < obj(lam) - 1e-15 * abs(obj(lam)):
            t *= 0.5
            nxt = lam + t * step
            if t < 1e-30:
                nxt = lam
                break
        if nxt == lam:
            break
        lam = nxt
    return torch.tensor(lam, dtype=F64)


def dual_value(C, a, b, f, g, eps: float, div1, div2) -> torch.Tensor:
    """F_eps(f, g) for general phi^* (Sec. 1)."""
    C, a, b, f, g = _t(C), _t(a), _t(b), _t(f), _t(g)
    ent = (a[:, None] * b[None, :] * (torch.exp((f[:, None] + g[None, :] - C) / eps) - 1.0)).sum()
    return (a * neg_conj(div1, f)).sum() + (b * neg_conj(div2, g)).sum() - eps * ent


def f_sinkhorn(C, a, b, eps: float, div1, div2, n_iter: int, f0=None):
    """F-Sinkhorn (Sec. 3) for general phi^*, from f_0 (default 0); returns (f, g)."""
    C = _t(C)
    f = torch.zeros(C.shape[0], dtype=F64) if f0 is None else _t(f0).clone()
    g = torch.zeros(C.shape[1], dtype=F64)
    for _ in range(n_iter):
        g = -aprox(div2, -smin_cols(C, a, f, eps), eps)
        f = -aprox(div1, -smin_rows(C, b, g, eps), eps)
    return f, g


def g_sinkhorn(C, a, b, eps: float, div1, div2, n_iter: int):
    """G-Sinkhorn (Sec. 3) for general phi^* from (fb, lambda) = (0, 0); returns (f, g, lambda)."""
    C = _t(C)
    fb = torch.zeros(C.shape[0], dtype=F64)
    gb = torch.zeros(C.shape[1], dtype=F64)
    lam = torch.tensor(0.0, dtype=F64)
    for _ in range(n_iter):
        gb = -aprox(div2, -smin_cols(C, a, fb + lam, eps), eps) + lam
        fb = -aprox(div1, -smin_rows(C, b, gb - lam, eps), eps) - lam
        lam = lambda_star(a, b, fb, gb, div1, div2)
    return fb + lam, gb - lam, lam
