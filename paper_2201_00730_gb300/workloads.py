"""Seeded synthetic workloads for unbalanced OT (inputs only, no solver arithmetic).

Both the CUDA path and the FP64 oracle take their inputs from here.  Values
are drawn in float64 with numpy's default_rng and rounded once to float32;
the oracle promotes the same float32 values back to float64, so both sides
see bit-identical data.

The five workloads stand in for the paper's experiments (Sec. 3 and Sec. 4:
1-D mixtures with N = M = 200 and 5000, measures with unequal mass, eps up
to 1e-3, rho in {0.1, 1, 10}); no dataset item is reproduced.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One unbalanced OT problem: points (or a dense cost), weights and parameters."""
    x: np.ndarray            # (n, d) float32
    y: np.ndarray            # (m, d) float32
    a: np.ndarray            # (n,) float32, a_i >= 0
    b: np.ndarray            # (m,) float32, b_j >= 0
    eps: float
    rho1: float
    rho2: float
    p: float = 2.0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.x.shape[0]

    @property
    def m(self) -> int:
        return self.y.shape[0]

    @property
    def dim(self) -> int:
        return self.x.shape[1]


def _weights(rng, n, mass, zero_frac=0.0):
    """Exp(1) weights rescaled to total `mass`; a fraction may be set to exactly 0."""
    w = rng.exponential(1.0, size=n)
    if zero_frac > 0:
        k = int(round(zero_frac * n))
        if k >= n:
            k = n - 1
        if k > 0:
            w[rng.choice(n, size=k, replace=False)] = 0.0
    w = w / w.sum() * mass
    return w.astype(np.float32)


def random_problem(n, m, d=1, seed=0, eps=1e-2, rho1=1.0, rho2=1.0, mass_a=1.0, mass_b=1.5,
                   zero_frac=0.0, p=2.0, scale=1.0) -> Problem:
    """Uniform points in [0, scale]^d with Exp(1) weights of the given masses."""
    rng = np.random.default_rng(seed)
    x = (rng.random((n, d)) * scale).astype(np.float32)
    y = (rng.random((m, d)) * scale).astype(np.float32)
    a = _weights(rng, n, mass_a, zero_frac)
    b = _weights(rng, m, mass_b, zero_frac)
    return Problem(x, y, a, b, float(eps), float(rho1), float(rho2), float(p),
                   name=f"random n={n} m={m} d={d} seed={seed}")


def config1() -> Problem:
    """1-D, N = M = 256, x, y ~ U[0,1], masses 1.0 / 1.5, eps = 1e-2, rho1 = rho2 = 1."""
    rng = np.random.default_rng(1001)
    x = rng.random((256, 1)).astype(np.float32)
    y = rng.random((256, 1)).astype(np.float32)
    a = _weights(rng, 256, 1.0)
    b = _weights(rng, 256, 1.5)
    return Problem(x, y, a, b, 1e-2, 1.0, 1.0, 2.0, name="1-D N=M=256 eps=1e-2 rho=1")


def _mixture(rng, n, k, shift):
    """n points from an equal-weight mixture of k isotropic 3-D Gaussians (sigma 0.05)
    whose means are U[0.2, 0.8]^3 + shift."""
    means = rng.uniform(0.2, 0.8, size=(k, 3)) + shift
    comp = rng.integers(0, k, size=n)
    return (means[comp] + 0.05 * rng.standard_normal((n, 3))).astype(np.float32)


def config2(rho: float = 1.0, n: int = 20000) -> Problem:
    """3-D mixtures, N = M = 20000: x from 4 components, y from 6 shifted components,
    masses 1.0 / 0.7, eps = 1e-3, rho1 = rho2 = rho (0.1, 1 or 10)."""
    rng = np.random.default_rng(1002)
    x = _mixture(rng, n, 4, 0.0)
    y = _mixture(rng, n, 6, 0.1)
    a = _weights(rng, n, 1.0)
    b = _weights(rng, n, 0.7)
    return Problem(x, y, a, b, 1e-3, float(rho), float(rho), 2.0,
                   name=f"3-D mixtures N=M={n} eps=1e-3 rho={rho:g}")


def config3(n: int = 8192, d: int = 64) -> Problem:
    """D = 64 Gaussian clouds, N = M = 8192, x, y ~ N(0, I/(2D)) with independent seeds,
    masses 1.0 / 2.0, eps = 5e-2, rho1 = rho2 = 0.5."""
    rx = np.random.default_rng(1003)
    ry = np.random.default_rng(2003)
    sd = np.sqrt(1.0 / (2 * d))
    x = (sd * rx.standard_normal((n, d))).astype(np.float32)
    y = (sd * ry.standard_normal((n, d))).astype(np.float32)
    a = _weights(rx, n, 1.0)
    b = _weights(ry, n, 2.0)
    return Problem(x, y, a, b, 5e-2, 0.5, 0.5, 2.0, name=f"D={d} Gaussians N=M={n}")


def config4(count: int = 4096, lo: int = 64, hi: int = 4096, seed: int = 1004):
    """`count` independent problems: N_k, M_k = round(exp(U[ln lo, ln hi])), D_k in {1, 2},
    points U[0,1]^D, eps_k log-uniform [1e-3, 1e-1], rho_k log-uniform [0.1, 10] (rho1 = rho2),
    masses independently U[0.5, 2]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        m = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        d = int(rng.integers(1, 3))
        eps = float(np.exp(rng.uniform(np.log(1e-3), np.log(1e-1))))
        rho = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
        ma, mb = rng.uniform(0.5, 2.0, size=2)
        x = rng.random((n, d)).astype(np.float32)
        y = rng.random((m, d)).astype(np.float32)
        a = _weights(rng, n, ma)
        b = _weights(rng, m, mb)
        out.append(Problem(x, y, a, b, eps, rho, rho, 2.0, name=f"batch[{k}]"))
    return out


def config_fw1d(count: int = 1024, n: int = 200, seed: int = 1006, rho: float = 1.0):
    """`count` independent 1-D problems of the size of the paper's FW-vs-Sinkhorn comparison
    (Sec. 4: N = M = 200 histograms, rho = 1): sorted points, x from a two-component Gaussian
    mixture, y from a shifted one, Exp(1) weights rescaled to masses 1 and 1.5.  Each entry has
    x, a, y, b (float32, x and y ascending) and rho1 = rho2 = rho."""
    from types import SimpleNamespace
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        cx = rng.choice([-0.5, 0.5], size=n) + 0.2 * rng.standard_normal(n)
        cy = rng.choice([-0.2, 0.8], size=n) + 0.25 * rng.standard_normal(n)
        a = rng.exponential(1.0, n)
        b = rng.exponential(1.0, n)
        out.append(SimpleNamespace(x=np.sort(cx).astype(np.float32), a=(a / a.sum()).astype(np.float32),
                                   y=np.sort(cy).astype(np.float32), b=(1.5 * b / b.sum()).astype(np.float32),
                                   rho1=rho, rho2=rho))
    return out


def config5(n: int = 262144) -> Problem:
    """3-D uniform points in the unit cube, N = M = 262144, masses 1.0 / 1.3, eps = 1e-3,
    rho1 = rho2 = 1."""
    rng = np.random.default_rng(1005)
    x = rng.random((n, 3)).astype(np.float32)
    y = rng.random((n, 3)).astype(np.float32)
    a = _weights(rng, n, 1.0)
    b = _weights(rng, n, 1.3)
    return Problem(x, y, a, b, 1e-3, 1.0, 1.0, 2.0, name=f"3-D uniform N=M={n}")


def dense_cost_f32(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Materialise |x_i - y_j|^2 as a float32 matrix for the dense-cost path.

    This is an input format conversion (the same squared-distance definition the
    fused path evaluates on the fly), computed in float64 and rounded once.
    """
    out = np.empty((x.shape[0], y.shape[0]), dtype=np.float32)
    yy = y.astype(np.float64)
    step = max(1, (1 << 24) // max(1, y.shape[0]))
    for i0 in range(0, x.shape[0], step):
        xi = x[i0:i0 + step].astype(np.float64)
        d = xi[:, None, :] - yy[None, :, :]
        out[i0:i0 + step] = (d * d).sum(-1)
    return out


def dense_cost_f32_device(x: np.ndarray, y: np.ndarray, device, rows_per_block: int = 2048):
    """dense_cost_f32 built on `device` (a torch device) for matrices too large to build on the
    host quickly: the same squared distances, each coordinate difference and square in float64,
    summed over the coordinates in order, rounded once to float32."""
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(device=device, dtype=torch.float64)
    yd = torch.from_numpy(np.ascontiguousarray(y)).to(device=device, dtype=torch.float64)
    out = torch.empty((x.shape[0], y.shape[0]), dtype=torch.float32, device=device)
    for i0 in range(0, x.shape[0], rows_per_block):
        xi = xd[i0:i0 + rows_per_block]
        acc = torch.zeros((xi.shape[0], yd.shape[0]), dtype=torch.float64, device=device)
        for k in range(x.shape[1]):
            d = xi[:, k:k + 1] - yd[None, :, k]
            acc += d * d
        out[i0:i0 + rows_per_block] = acc.to(torch.float32)
    return out


def config_mmot1d(count: int = 64, K: int = 8, n: int = 200, seed: int = 1007, rho: float = 1.0, ragged: bool = False):
    """`count` independent 1-D multi-marginal problems of K measures, the shape of the paper's
    barycenter experiment (Sec. 5: K = 8 one-dimensional Gaussian mixtures): measure k has n points
    (with ragged, between n/2 and n) sorted from a two-component Gaussian mixture whose centres move
    with k, Exp(1) weights rescaled to a mass in [0.5, 2], uniform barycentric weights 1/K, rho."""
    from types import SimpleNamespace
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        xs, als = [], []
        for k in range(K):
            nk = int(rng.integers(max(1, n // 2), n + 1)) if ragged else n
            c = rng.choice([-1.0 + 0.25 * k, 0.5 + 0.1 * k], size=nk)
            xs.append(np.sort(c + 0.15 * rng.standard_normal(nk)).astype(np.float32))
            w = rng.exponential(1.0, nk)
            als.append((w / w.sum() * rng.uniform(0.5, 2.0)).astype(np.float32))
        out.append(SimpleNamespace(xs=xs, alphas=als, omega=[1.0 / K] * K, rho=float(rho)))
    return out
