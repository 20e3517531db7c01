"""Batched 1-D Frank-Wolfe on H_0 (Sec. 4, Algs. 1-2) through the C ABI against the FP64 oracle."""
import math
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from oracle import fw1d as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    from paper_2201_00730_gb300 import build, uot
    build.build()
    return uot


def make(n, m, seed, rho1, rho2, zeros=True):
    rng = np.random.default_rng(seed)
    x = np.sort(rng.normal(0.0, 1.0, n)).astype(np.float32)
    y = np.sort(rng.normal(0.3, 0.8, m)).astype(np.float32)
    a = rng.exponential(1.0 / n, n).astype(np.float32)
    b = rng.exponential(1.5 / m, m).astype(np.float32)
    if zeros and n > 3:
        a[n // 3] = 0.0
    if zeros and m > 3:
        b[m // 2] = 0.0
    return SimpleNamespace(x=x, a=a, y=y, b=b, rho1=rho1, rho2=rho2)


def oracle(q, T, p):
    f64 = lambda v: np.asarray(v, dtype=np.float64)
    return W.fw_uot_1d(f64(q.x), f64(q.a), f64(q.y), f64(q.b), q.rho1, q.rho2, T, p)


def scale(q, p):
    return 1.0 + float(np.abs(q.x.astype(np.float64)[:, None] - q.y.astype(np.float64)[None, :]).max() ** p)


BATCH = [(1, 1, 1.0, 1.0), (1, 7, 0.5, 2.0), (9, 1, 1.0, 0.3), (40, 33, 0.1, 1.0), (200, 200, 1.0, 1.0),
         (5, 300, 3.0, 0.7), (257, 31, 10.0, 10.0), (1000, 700, 1.0, 2.0)]


@pytest.mark.parametrize("p", [2.0, 1.0, 1.5])
@pytest.mark.parametrize("T", [1, 3, 25])
def test_fw1d_iterates_match_oracle(U, p, T):
    """A ragged batch (single points, one-sided singletons, zero weights, rho1 != rho2, one problem too
    large for the on-chip histograms) after T steps."""
    probs = [make(n, m, seed=100 * k + int(10 * p), rho1=r1, rho2=r2) for k, (n, m, r1, r2) in enumerate(BATCH)]
    out = U.fw1d_batched(probs, T, p)
    assert out.status == [0] * len(probs)
    for k, q in enumerate(probs):
        ref = oracle(q, T, p)
        tol = 1e-9 * scale(q, p)
        ef = (out.f[k].cpu() - ref.f).abs().max().item()
        eg = (out.g[k].cpu() - ref.g).abs().max().item()
        assert ef <= tol and eg <= tol, (k, ef, eg, tol)


def test_fw1d_long_run_value_matches_oracle(U):
    """2000 steps on N = M = 60 (rho = 0.5): the dual value F_0 of the GPU pair equals the oracle's."""
    q = make(60, 60, seed=7, rho1=0.5, rho2=0.5)
    out = U.fw1d_batched([q], 2000, 2.0)
    ref = oracle(q, 2000, 2.0)
    v_gpu = W.f0_value(q.a.astype(np.float64), q.b.astype(np.float64), out.f[0].cpu(), out.g[0].cpu(), 0.5, 0.5)
    v_ref = W.f0_value(q.a.astype(np.float64), q.b.astype(np.float64), ref.f, ref.g, 0.5, 0.5)
    assert abs(v_gpu.item() - v_ref.item()) <= 1e-10 * max(1.0, abs(v_ref.item()))
    assert (out.f[0].cpu() - ref.f).abs().max().item() <= 1e-7 * scale(q, 2.0)


@pytest.mark.parametrize("rho1,rho2", [(1.0, 1.0), (0.1, 2.0)])
def test_fw1d_one_point_closed_form(U, rho1, rho2):
    """N = M = 1: f* = rho1 rho2/(rho1+rho2) (log a - log b + c/rho2), g* = c - f*."""
    q = SimpleNamespace(x=np.array([0.25], np.float32), a=np.array([0.75], np.float32),
                        y=np.array([1.5], np.float32), b=np.array([2.0], np.float32), rho1=rho1, rho2=rho2)
    out = U.fw1d_batched([q], 4, 2.0)
    c = (1.5 - 0.25) ** 2
    f_star = rho1 * rho2 / (rho1 + rho2) * (math.log(0.75) - math.log(2.0) + c / rho2)
    assert abs(out.f[0].item() - f_star) < 1e-12 and abs(out.g[0].item() - (c - f_star)) < 1e-12


def test_fw1d_invalid_problems_are_reported_alone(U):
    """Unsorted points -> UOT_ERR_INVALID_ARG, a negative weight -> UOT_ERR_NONFINITE, each only for its own
    problem (NaN outputs there); the valid problems in the same batch still match the oracle."""
    good = make(20, 15, seed=1, rho1=1.0, rho2=1.0)
    unsorted = make(10, 10, seed=2, rho1=1.0, rho2=1.0)
    unsorted.x = unsorted.x[::-1].copy()
    negative = make(10, 10, seed=3, rho1=1.0, rho2=1.0)
    negative.b[4] = -0.5
    zero_mass = make(6, 6, seed=4, rho1=1.0, rho2=1.0)
    zero_mass.a[:] = 0.0
    out = U.fw1d_batched([good, unsorted, negative, zero_mass], 10, 2.0, check=False)
    assert out.status == [0, 1, 4, 4] and out.code == 1
    assert torch.isnan(out.f[1]).all() and torch.isnan(out.g[2]).all()
    ref = oracle(good, 10, 2.0)
    assert (out.f[0].cpu() - ref.f).abs().max().item() <= 1e-9 * scale(good, 2.0)
    with pytest.raises(U.UOTError):
        U.fw1d_batched([unsorted], 3, 2.0)


def test_fw1d_many_problems(U):
    """1000 problems of the paper's Fig. 5 size class (N, M around 200) in one call; spot checks."""
    rng = np.random.default_rng(11)
    probs = [make(int(rng.integers(150, 250)), int(rng.integers(150, 250)), seed=1000 + k, rho1=1.0, rho2=1.0)
             for k in range(1000)]
    out = U.fw1d_batched(probs, 20, 2.0)
    assert out.status == [0] * 1000
    for k in (0, 417, 999):
        ref = oracle(probs[k], 20, 2.0)
        assert (out.f[k].cpu() - ref.f).abs().max().item() <= 1e-9 * scale(probs[k], 2.0)
