"""FP64 CPU oracle for entropic unbalanced OT with rho*KL marginal penalties.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the library never does, and
it shares no code with the CUDA kernels or their bindings.

Everything is plain PyTorch CPU arithmetic in float64 on dense N x M arrays,
written in the paper's order and notation (Sejourne, Vialard, Peyre,
"Faster Unbalanced Optimal Transport: Translation invariant Sinkhorn and 1-D
Frank-Wolfe", AISTATS 2022):

  * primal problem           -- Sec. 1, Eq. (eq-primal-uot-kl)
  * dual functional F_eps    -- Sec. 1, Eq. (eq-dual-uot-kl)
  * softmin, aprox           -- Sec. 3, "F-Sinkhorn"
  * optimal translation      -- Sec. 2, Prop. 2 (eq-opt-trans-kl), and the
                                Smin form of lambda* in the proof of the
                                Lipschitz property of Phi (App. B)
  * explicit H_eps           -- Sec. 2, Prop. 3
  * F-Sinkhorn               -- Sec. 3
  * H-Sinkhorn (TI-Sinkhorn) -- Sec. 3, Prop. 4 and its proof in App. B,
                                general rho1 != rho2 (Eq. eq-general-iter-h-sink)
  * G-Sinkhorn               -- Sec. 3, with the +-lambda_t terms made explicit
  * Anderson extrapolation   -- appendix "Combining Sinkhorn with Anderson
                                acceleration" (restarted blocks of K iterations)

Conventions fixed where the paper is ambiguous (each is also listed in the
design notes):
  * phi_i^*(x) = rho_i (exp(x/rho_i) - 1), so -phi^*(-f) = rho (1 - e^{-f/rho});
    this is the form used in the proofs of Props. 2, 3 and 4 (the display in
    Sec. 2 drops the sign of the exponent).
  * f is paired with (a, x, rho1, index i), g with (b, y, rho2, index j).
  * One iteration is the g half-step followed by the f half-step; f_0 = 0.
  * Zero weights are allowed and drop out of every sum (log 0 = -inf).

Parity status: every function here is pinned by a test in tests/ against a
closed form, an invariant or an independent solver (see test_oracle_*.py);
none is "parity unpinned".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

F64 = torch.float64


def _t(v) -> torch.Tensor:
    """Promote an array-like to a float64 CPU tensor (values are not changed)."""
    if isinstance(v, torch.Tensor):
        return v.to(device="cpu", dtype=F64)
    return torch.as_tensor(v, dtype=F64)


# --------------------------------------------------------------------------
# Cost and elementary operators
# --------------------------------------------------------------------------

def cost_matrix(x, y, p: float = 2.0) -> torch.Tensor:
    """C_ij = |x_i - y_j|_2^p for point clouds x (N x D) and y (M x D).

    Sec. 1 writes the cost as C_ij = d(x_i, x_j)^p; the 1-D experiments
    (Sec. 4) use |x - y|^p.  The direct-difference form is used (no
    |x|^2 + |y|^2 - 2 x.y expansion).
    """
    x, y = _t(x), _t(y)
    if x.dim() == 1:
        x = x[:, None]
    if y.dim() == 1:
        y = y[:, None]
    d = x[:, None, :] - y[None, :, :]
    sq = (d * d).sum(-1)
    if p == 2.0:
        return sq
    return sq.sqrt() ** p


def log_weights(w) -> torch.Tensor:
    """log w with log 0 = -inf (zero weights drop out of every sum)."""
    w = _t(w)
    out = torch.full_like(w, -math.inf)
    pos = w > 0
    out[pos] = torch.log(w[pos])
    return out


def log_dot_exp(w, z) -> torch.Tensor:
    """log <w, exp(z)> = log sum_i w_i e^{z_i} over the last axis, with the weights kept outside the
    exponential (so a zero weight has the derivative e^{z_i} / <w, e^z>, like any other) and the largest
    exponent of a positive weight taken out first for range (it cancels exactly)."""
    w = _t(w)
    live = w > 0
    zm = torch.where(live, z, torch.full_like(z, -math.inf))
    m = zm.max(dim=-1, keepdim=True).values.detach()
    return m.squeeze(-1) + torch.log((w * torch.exp(z - m)).sum(-1))


def softmin(w, h, eps: float) -> torch.Tensor:
    """Smin_w^eps(h) = -eps log <w, exp(-h/eps)>, reduced over the last axis.

    Definition of the softmin in Sec. 3 ("F-Sinkhorn"), written with the weights
    outside the exponential as in the definition.
    """
    w, h = _t(w), _t(h)
    return -eps * log_dot_exp(w, -h / eps)


def smin_rows(C, b, g, eps: float) -> torch.Tensor:
    """S_i = Smin_b^eps(C(x_i, .) - g), the softmin over j of every row i.

    This is the argument of -aprox in the f-update of F-Sinkhorn (Sec. 3).
    """
    C, g = _t(C), _t(g)
    return softmin(b, C - g[None, :], eps)


def smin_cols(C, a, f, eps: float) -> torch.Tensor:
    """S'_j = Smin_a^eps(C(., y_j) - f), the softmin over i of every column j.

    This is the argument of -aprox in the g-update of F-Sinkhorn (Sec. 3).
    """
    C, f = _t(C), _t(f)
    return softmin(a, (C - f[:, None]).T, eps)


def aprox_kl(x, eps: float, rho: float):
    """Anisotropic prox of phi^* for rho*KL: aprox(x) = rho/(eps+rho) x (Sec. 3)."""
    return rho / (eps + rho) * x


def lambda_star(a, b, fb, gb, rho1: float, rho2: float) -> torch.Tensor:
    """Optimal translation of Prop. 2 (eq-opt-trans-kl).

    lambda* = rho1 rho2/(rho1+rho2) * log( <a, e^{-fb/rho1}> / <b, e^{-gb/rho2}> ),
    with both logs taken as stabilised log-sum-exps (Prop. 2, remark after it).
    """
    la = log_dot_exp(a, -_t(fb) / rho1)
    lb = log_dot_exp(b, -_t(gb) / rho2)
    return rho1 * rho2 / (rho1 + rho2) * (la - lb)


def phi_map(a, b, fb, gb, rho1: float, rho2: float):
    """Phi(fb, gb) = (fb + lambda*, gb - lambda*): the dual iterates of H (Sec. 1)."""
    lam = lambda_star(a, b, fb, gb, rho1, rho2)
    return _t(fb) + lam, _t(gb) - lam, lam


# --------------------------------------------------------------------------
# Objectives
# --------------------------------------------------------------------------

def dual_value(C, a, b, f, g, eps: float, rho1: float, rho2: float) -> torch.Tensor:
    """F_eps(f, g) of Eq. (eq-dual-uot-kl) with phi_i^* of rho_i*KL:

    <a, rho1 (1 - e^{-f/rho1})> + <b, rho2 (1 - e^{-g/rho2})>
        - eps <a (x) b, exp((f (+) g - C)/eps) - 1>.
    """
    C, a, b, f, g = map(_t, (C, a, b, f, g))
    t1 = (a * rho1 * (1.0 - torch.exp(-f / rho1))).sum()
    t2 = (b * rho2 * (1.0 - torch.exp(-g / rho2))).sum()
    e = torch.exp((f[:, None] + g[None, :] - C) / eps) - 1.0
    t3 = eps * (a[:, None] * b[None, :] * e).sum()
    return t1 + t2 - t3


def h_value(C, a, b, fb, gb, eps: float, rho1: float, rho2: float) -> torch.Tensor:
    """Explicit H_eps of Prop. 3 (eq-dual-form-hell)."""
    C, a, b, fb, gb = map(_t, (C, a, b, fb, gb))
    tau1, tau2 = rho1 / (rho1 + rho2), rho2 / (rho1 + rho2)
    A = (a * torch.exp(-fb / rho1)).sum()
    B = (b * torch.exp(-gb / rho2)).sum()
    e = torch.exp((fb[:, None] + gb[None, :] - C) / eps) - 1.0
    return (rho1 * a.sum() + rho2 * b.sum() - eps * (a[:, None] * b[None, :] * e).sum()
            - (rho1 + rho2) * A ** tau1 * B ** tau2)


def transport_plan(C, a, b, f, g, eps: float) -> torch.Tensor:
    """pi_ij = a_i b_j exp((f_i + g_j - C_ij)/eps): the primal plan of dual potentials."""
    C, a, b, f, g = map(_t, (C, a, b, f, g))
    return a[:, None] * b[None, :] * torch.exp((f[:, None] + g[None, :] - C) / eps)


def kl_div(mu, nu) -> torch.Tensor:
    """KL(mu|nu) = sum mu log(mu/nu) - m(mu) + m(nu) (Sec. 1), 0 log 0 = 0."""
    mu, nu = _t(mu), _t(nu)
    pos = mu > 0
    if bool((nu[pos] <= 0).any()):
        return torch.tensor(math.inf, dtype=F64)
    return (mu[pos] * torch.log(mu[pos] / nu[pos])).sum() - mu.sum() + nu.sum()


def primal_value(C, a, b, pi, eps: float, rho1: float, rho2: float) -> torch.Tensor:
    """Objective of Eq. (eq-primal-uot-kl) at a plan pi:

    <pi, C> + eps KL(pi | a(x)b) + rho1 KL(pi 1 | a) + rho2 KL(pi^T 1 | b).
    """
    C, a, b, pi = map(_t, (C, a, b, pi))
    ab = a[:, None] * b[None, :]
    return ((pi * C).sum() + eps * kl_div(pi.flatten(), ab.flatten())
            + rho1 * kl_div(pi.sum(1), a) + rho2 * kl_div(pi.sum(0), b))


def dual_from_softmin(a, b, f, g, S, eps: float, rho1: float, rho2: float) -> torch.Tensor:
    """F_eps(f, g) of Eq. (eq-dual-uot-kl) from the row softmins S_i = Smin_b^eps(C(x_i, .) - g).

    The double sum of the dual collapses over j by the definition of Smin (Sec. 3):
    sum_j b_j e^{(g_j - C_ij)/eps} = e^{-S_i/eps}, so
        F = <a, rho1 (1 - e^{-f/rho1})> + <b, rho2 (1 - e^{-g/rho2})>
            - eps sum_i a_i e^{(f_i - S_i)/eps} + eps m(a) m(b).
    Only O(N + M) work once S is known, for problems whose N x M cost cannot be formed.
    """
    a, b, f, g, S = map(_t, (a, b, f, g, S))
    t1 = (a * rho1 * (1.0 - torch.exp(-f / rho1))).sum()
    t2 = (b * rho2 * (1.0 - torch.exp(-g / rho2))).sum()
    t3 = eps * ((a * torch.exp((f - S) / eps)).sum() - a.sum() * b.sum())
    return t1 + t2 - t3


def primal_from_softmins(a, b, f, g, S, Sp, eps: float, rho1: float, rho2: float) -> torch.Tensor:
    """Objective of Eq. (eq-primal-uot-kl) at the plan pi_ij = a_i b_j e^{(f_i + g_j - C_ij)/eps}
    from the row and column softmins S_i = Smin_b^eps(C(x_i, .) - g), S'_j = Smin_a^eps(C(., y_j) - f).

    Its marginals are pi1_i = a_i e^{(f_i - S_i)/eps} and pi2_j = b_j e^{(g_j - S'_j)/eps}
    (definition of Smin), and log(pi_ij / (a_i b_j)) = (f_i + g_j - C_ij)/eps turns
    <pi, C> + eps KL(pi | a(x)b) into <pi1, f> + <pi2, g> - eps m(pi) + eps m(a) m(b), so
        P = <pi1, f> + <pi2, g> - eps m(pi) + eps m(a) m(b) + rho1 KL(pi1 | a) + rho2 KL(pi2 | b).
    """
    a, b, f, g, S, Sp = map(_t, (a, b, f, g, S, Sp))
    pi1 = a * torch.exp((f - S) / eps)
    pi2 = b * torch.exp((g - Sp) / eps)
    mpi = pi1.sum()
    return ((pi1 * f).sum() + (pi2 * g).sum() - eps * mpi + eps * a.sum() * b.sum()
            + rho1 * kl_div(pi1, a) + rho2 * kl_div(pi2, b))


def fixed_point_residual(C, a, b, f, g, eps: float, rho1: float, rho2: float) -> torch.Tensor:
    """Sup-norm violation of the F-Sinkhorn fixed-point equations by (f, g):

    max( |f - rho1/(rho1+eps) Smin_b^eps(C - g)|_inf,
         |g - rho2/(rho2+eps) Smin_a^eps(C - f)|_inf ).

    These are the equations that characterise the optimum (App. B, last part of
    the convergence theorem for H-Sinkhorn).  The paper itself reports
    |f_t - f*|_inf with a precomputed f*; this residual is the stopping rule the
    library uses, in cost units.
    """
    rf = (_t(f) - aprox_kl(smin_rows(C, b, g, eps), eps, rho1)).abs().max()
    rg = (_t(g) - aprox_kl(smin_cols(C, a, f, eps), eps, rho2)).abs().max()
    return torch.maximum(rf, rg)


# --------------------------------------------------------------------------
# Sinkhorn iterations
# --------------------------------------------------------------------------

def f_sinkhorn_iteration(C, a, b, f, eps: float, rho1: float, rho2: float):
    """One F-Sinkhorn iteration (Sec. 3): g <- -aprox(-Smin_a(C - f)); f <- -aprox(-Smin_b(C - g)).

    With aprox linear for KL, -aprox(-s) = aprox(s).
    """
    g = aprox_kl(smin_cols(C, a, f, eps), eps, rho2)
    f = aprox_kl(smin_rows(C, b, g, eps), eps, rho1)
    return f, g


def psi_g(C, a, b, fb, eps: float, rho1: float, rho2: float) -> torch.Tensor:
    """H-Sinkhorn g half-step gb = argmax_gb H(fb, gb), general rho1 != rho2.

    App. B, proof of Prop. 4, with the roles of (a, fb, rho1) and (b, gb, rho2)
    swapped as stated there:
      g_hat = rho2/(rho2+eps) Smin_a^eps(C - fb) - eps/(eps+rho2) * rho2/(rho1+rho2) * Smin_a^rho1(fb)
      k     = eps/(eps+rho2) * rho1/(rho1+rho2)
      gb    = g_hat + k/(1-k) Smin_b^rho2(g_hat)
    """
    fb = _t(fb)
    g_hat = (rho2 / (rho2 + eps) * smin_cols(C, a, fb, eps)
             - eps / (eps + rho2) * rho2 / (rho1 + rho2) * softmin(a, fb, rho1))
    k = eps / (eps + rho2) * rho1 / (rho1 + rho2)
    return g_hat + k / (1.0 - k) * softmin(b, g_hat, rho2)


def psi_f(C, a, b, gb, eps: float, rho1: float, rho2: float) -> torch.Tensor:
    """H-Sinkhorn f half-step fb = argmax_fb H(fb, gb), general rho1 != rho2.

    App. B, proof of Prop. 4 (Eq. eq-general-iter-h-sink):
      f_hat = rho1/(rho1+eps) Smin_b^eps(C - gb) - eps/(eps+rho1) * rho1/(rho1+rho2) * Smin_b^rho2(gb)
      k     = eps/(eps+rho1) * rho2/(rho1+rho2)
      fb    = f_hat + k/(1-k) Smin_a^rho1(f_hat)
    """
    gb = _t(gb)
    f_hat = (rho1 / (rho1 + eps) * smin_rows(C, b, gb, eps)
             - eps / (eps + rho1) * rho1 / (rho1 + rho2) * softmin(b, gb, rho2))
    k = eps / (eps + rho1) * rho2 / (rho1 + rho2)
    return f_hat + k / (1.0 - k) * softmin(a, f_hat, rho1)


def h_sinkhorn_iteration(C, a, b, fb, eps: float, rho1: float, rho2: float):
    """One H-Sinkhorn iteration (Sec. 3): gb_{t+1} = Psi(fb_t), fb_{t+1} = Psi(gb_{t+1})."""
    gb = psi_g(C, a, b, fb, eps, rho1, rho2)
    fb = psi_f(C, a, b, gb, eps, rho1, rho2)
    return fb, gb


def g_sinkhorn_iteration(C, a, b, fb, lam, eps: float, rho1: float, rho2: float):
    """One G-Sinkhorn iteration (Sec. 3), alternate maximisation of G(fb, gb, lambda).

    The paper's display omits the +-lambda_t on the left-hand sides; maximising
    G over gb at fixed (fb, lambda) gives gb - lambda = aprox(Smin_a(C - fb - lambda)),
    and likewise for fb, so:
      gb_{t+1} = aprox_2(Smin_a^eps(C - fb_t - lambda_t)) + lambda_t
      fb_{t+1} = aprox_1(Smin_b^eps(C - gb_{t+1} + lambda_t)) - lambda_t
      lambda_{t+1} = lambda*(fb_{t+1}, gb_{t+1}).
    """
    fb = _t(fb)
    gb = aprox_kl(smin_cols(C, a, fb + lam, eps), eps, rho2) + lam
    fb = aprox_kl(smin_rows(C, b, gb - lam, eps), eps, rho1) - lam
    lam = lambda_star(a, b, fb, gb, rho1, rho2)
    return fb, gb, lam


@dataclass
class SolveResult:
    f: torch.Tensor                 # dual potential f (translated, for TI)
    g: torch.Tensor                 # dual potential g
    iters: int                      # full iterations run
    residual: float                 # fixed_point_residual at exit (nan if not computed)
    lam: float = 0.0                # lambda* at exit (TI / G), 0 for plain
    fb: torch.Tensor | None = None  # H / G state
    gb: torch.Tensor | None = None
    history: list = field(default_factory=list)  # (iteration, residual) pairs


def sinkhorn(C, a, b, eps, rho1, rho2, n_iter, tol=0.0, check_every=1, f0=None,
             keep_iterates=False) -> SolveResult:
    """Plain F-Sinkhorn from f_0 (default 0), up to n_iter iterations.

    Stops early once fixed_point_residual <= tol, checked every check_every
    iterations.  With keep_iterates, history holds (t, f_t, g_t).
    """
    C = _t(C)
    f = torch.zeros(C.shape[0], dtype=F64) if f0 is None else _t(f0).clone()
    g = torch.zeros(C.shape[1], dtype=F64)
    hist, res, t = [], math.nan, 0
    for t in range(1, n_iter + 1):
        f, g = f_sinkhorn_iteration(C, a, b, f, eps, rho1, rho2)
        if keep_iterates:
            hist.append((t, f.clone(), g.clone()))
        if tol > 0 and t % check_every == 0:
            res = float(fixed_point_residual(C, a, b, f, g, eps, rho1, rho2))
            if not keep_iterates:
                hist.append((t, res))
            if res <= tol:
                break
    return SolveResult(f, g, t, res, 0.0, None, None, hist)


def ti_sinkhorn(C, a, b, eps, rho1, rho2, n_iter, tol=0.0, check_every=1, fb0=None,
                keep_iterates=False) -> SolveResult:
    """H-Sinkhorn (translation invariant Sinkhorn) from fb_0 (default 0).

    Output is the translated pair (f, g) = Phi(fb, gb) (Sec. 1).  With
    keep_iterates, history holds (t, f_t, g_t) of the translated iterates.
    """
    C = _t(C)
    fb = torch.zeros(C.shape[0], dtype=F64) if fb0 is None else _t(fb0).clone()
    gb = torch.zeros(C.shape[1], dtype=F64)
    hist, res, t = [], math.nan, 0
    for t in range(1, n_iter + 1):
        fb, gb = h_sinkhorn_iteration(C, a, b, fb, eps, rho1, rho2)
        if keep_iterates or (tol > 0 and t % check_every == 0):
            f, g, _ = phi_map(a, b, fb, gb, rho1, rho2)
            if keep_iterates:
                hist.append((t, f.clone(), g.clone()))
            if tol > 0 and t % check_every == 0:
                res = float(fixed_point_residual(C, a, b, f, g, eps, rho1, rho2))
                if not keep_iterates:
                    hist.append((t, res))
                if res <= tol:
                    break
    f, g, lam = phi_map(a, b, fb, gb, rho1, rho2)
    return SolveResult(f, g, t, res, float(lam), fb, gb, hist)


def g_sinkhorn(C, a, b, eps, rho1, rho2, n_iter, tol=0.0, check_every=1) -> SolveResult:
    """G-Sinkhorn (Sec. 3) from (fb_0, lambda_0) = (0, 0); output (fb + lambda, gb - lambda)."""
    C = _t(C)
    fb = torch.zeros(C.shape[0], dtype=F64)
    gb = torch.zeros(C.shape[1], dtype=F64)
    lam = torch.tensor(0.0, dtype=F64)
    hist, res, t = [], math.nan, 0
    for t in range(1, n_iter + 1):
        fb, gb, lam = g_sinkhorn_iteration(C, a, b, fb, lam, eps, rho1, rho2)
        if tol > 0 and t % check_every == 0:
            res = float(fixed_point_residual(C, a, b, fb + lam, gb - lam, eps, rho1, rho2))
            hist.append((t, res))
            if res <= tol:
                break
    return SolveResult(fb + lam, gb - lam, t, res, float(lam), fb, gb, hist)


def anderson_weights(U, r: float) -> torch.Tensor:
    """Anderson extrapolation weights (appendix, "Combining Sinkhorn with Anderson
    acceleration"): c = (G + r I)^{-1} 1 / 1^T (G + r I)^{-1} 1 with G = U^T U, the
    minimiser of c^T (G + r I) c under 1^T c = 1, for the K residuals as the columns
    of U.  The regularisation is relative: G is divided by its trace first (the
    paper's r = 1e-7 is scale-free only in that reading)."""
    U = _t(U)
    G = U.T @ U
    tr = torch.trace(G)
    if tr > 0:
        G = G / tr
    z = torch.linalg.solve(G + r * torch.eye(G.shape[0], dtype=F64), torch.ones(G.shape[0], dtype=F64))
    return z / z.sum()


def anderson_sinkhorn(C, a, b, eps, rho1, rho2, n_iter, method="ti", K=4, r=1e-7, tol=0.0,
                      check_every=1) -> SolveResult:
    """F- ('plain'), H- ('ti') or G-Sinkhorn ('g') with Anderson extrapolation (appendix).

    The iterate x is f (F), fb (H) or fb with lambda carried alongside (G).  From a
    block start x_0, base iterations x_{k+1} = T(x_k) give residuals u_k = x_{k+1} - x_k;
    after every K-th iteration t (t % K == 0), unless t is the last one or a residual
    check, the last K + 1 iterates x_{t-K}, ..., x_t are replaced by the extrapolation
    sum_{k<K} c_k x_{t-K+k}, c = anderson_weights([u_0 ... u_{K-1}], r), which starts the
    next block (lambda of G takes the same combination).  The returned pair is always
    the last base iterate's, as for the plain solvers.
    """
    C = _t(C)
    x = torch.zeros(C.shape[0], dtype=F64)
    lam = torch.tensor(0.0, dtype=F64)
    hist, lams = [x.clone()], [lam.clone()]
    res, t = math.nan, 0
    out = None
    for t in range(1, n_iter + 1):
        if method == "plain":
            x, g = f_sinkhorn_iteration(C, a, b, x, eps, rho1, rho2)
            out = (x, g, 0.0)
        elif method == "ti":
            x, gb = h_sinkhorn_iteration(C, a, b, x, eps, rho1, rho2)
            f, g, lo = phi_map(a, b, x, gb, rho1, rho2)
            out = (f, g, float(lo))
        else:
            x, gb, lam = g_sinkhorn_iteration(C, a, b, x, lam, eps, rho1, rho2)
            out = (x + lam, gb - lam, float(lam))
        check = tol > 0 and t % check_every == 0
        if check:
            res = float(fixed_point_residual(C, a, b, out[0], out[1], eps, rho1, rho2))
            if res <= tol:
                break
        hist.append(x.clone())
        lams.append(lam.clone())
        if t % K == 0 and t < n_iter and not check:
            xs, ls = hist[-(K + 1):], lams[-(K + 1):]
            U = torch.stack([xs[k + 1] - xs[k] for k in range(K)], dim=1)
            c = anderson_weights(U, r)
            x = sum(c[k] * xs[k] for k in range(K))
            lam = sum(c[k] * ls[k] for k in range(K))
            hist, lams = [x.clone()], [lam.clone()]
    f, g, lo = out
    return SolveResult(f, g, t, res, lo, None, None, [])


def contraction_rate(errors) -> float:
    """Rate estimate of Sec. 3 ("Empirical convergence study"): kappa = e^c with c the
    median over t of log e_{t+1} - log e_t, for errors e_t = |f_t - f*|_inf."""
    e = torch.as_tensor([float(v) for v in errors], dtype=F64)
    keep = e > 0
    le = torch.log(e[keep])
    if le.numel() < 2:
        return math.nan
    return float(torch.exp(torch.median(le[1:] - le[:-1])))


# --------------------------------------------------------------------------
# Gradients of UOT (envelope theorem) and of a truncated solve (autograd)
# --------------------------------------------------------------------------

def envelope_grads(x, y, a, b, f, g, eps, rho1, rho2, p: float = 2.0):
    """Gradients of UOT = F_eps(f*, g*) with respect to a, b, x, y at the optimal pair.

    By the envelope (Danskin) theorem, which the paper applies to lambda in the
    proof of Prop. 1, the derivative of sup_{f,g} F_eps in a parameter is the
    partial derivative of F_eps at the maximiser.  With S_i = Smin_b^eps(C_i. - g):

      dF/da_i = rho1 (1 - e^{-f_i/rho1}) - eps (e^{(f_i - S_i)/eps} - m(b))
      dF/db_j = rho2 (1 - e^{-g_j/rho2}) - eps (e^{(g_j - S'_j)/eps} - m(a))
      dF/dx_i = sum_j pi_ij dC_ij/dx_i,  dC/dx = p |x-y|^{p-2} (x - y)
      dF/dy_j = sum_i pi_ij dC_ij/dy_j

    (dF/dC_ij = +pi_ij, from the last term of F_eps.)

    All terms are evaluated in FP64 on the dense plan pi.
    """
    x, y, a, b, f, g = map(_t, (x, y, a, b, f, g))
    if x.dim() == 1:
        x = x[:, None]
    if y.dim() == 1:
        y = y[:, None]
    C = cost_matrix(x, y, p)
    S = smin_rows(C, b, g, eps)
    Sp = smin_cols(C, a, f, eps)
    ga = rho1 * (1 - torch.exp(-f / rho1)) - eps * (torch.exp((f - S) / eps) - b.sum())
    gbv = rho2 * (1 - torch.exp(-g / rho2)) - eps * (torch.exp((g - Sp) / eps) - a.sum())
    pi = transport_plan(C, a, b, f, g, eps)
    d = x[:, None, :] - y[None, :, :]
    if p == 2.0:
        w = 2.0 * pi
    else:
        r = torch.sqrt((d * d).sum(-1))
        w = torch.where(r > 0, p * r ** (p - 2.0), torch.zeros_like(r)) * pi
    gx = (w[:, :, None] * d).sum(1)
    gy = -(w[:, :, None] * d).sum(0)
    return ga, gbv, gx, gy


def truncated_ti_value(x, y, a, b, eps, rho1, rho2, T: int, p: float = 2.0):
    """F_eps(f_T, g_T) after T H-Sinkhorn iterations from fb_0 = 0 (differentiable).

    Plain autograd through this function gives the unrolled gradient of the
    truncated solve with respect to whichever of x, y, a, b require grad.
    """
    C = cost_matrix(x, y, p)
    fb = torch.zeros(C.shape[0], dtype=F64)
    for _ in range(T):
        fb, gb = h_sinkhorn_iteration(C, a, b, fb, eps, rho1, rho2)
    f, g, _ = phi_map(a, b, fb, gb, rho1, rho2)
    return dual_value(C, a, b, f, g, eps, rho1, rho2)


def unrolled_grads(x, y, a, b, eps, rho1, rho2, T: int, p: float = 2.0):
    """d/d(a, b, x, y) of truncated_ti_value by reverse-mode autograd in FP64."""
    xs, ys, as_, bs = (_t(v).clone().requires_grad_(True) for v in (x, y, a, b))
    val = truncated_ti_value(xs, ys, as_, bs, eps, rho1, rho2, T, p)
    ga, gb, gx, gy = torch.autograd.grad(val, (as_, bs, xs, ys))
    return val.detach(), ga, gb, gx, gy
