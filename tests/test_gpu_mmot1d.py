"""Batched 1-D multi-marginal Frank-Wolfe and barycenters (Sec. 5, Alg. 3) on the GPU against
the FP64 oracle: translated potentials of every measure and the barycenter of the final plan
(points and masses), at 1e-9 (1 + largest cost), after 1, 3 and 25 steps on ragged batches."""
import numpy as np
import pytest
import torch

from oracle import mmot1d as MM
from paper_2201_00730_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    from paper_2201_00730_gb300 import build, uot
    build.build()
    return uot


def f64(v):
    return np.asarray(v, dtype=np.float64)


def check(got, q, T):
    ref = MM.fw_barycenter_1d([f64(x) for x in q.xs], [f64(a) for a in q.alphas], q.omega, q.rho, T)
    span = max(float(np.max(x)) for x in q.xs) - min(float(np.min(x)) for x in q.xs)
    tol = 1e-9 * (1.0 + span * span)
    for k in range(len(q.xs)):
        err = (got.f[k].cpu() - ref.fs[k]).abs().max().item()
        assert err <= tol, ("f", k, err, tol)
    assert got.bary_x.numel() == ref.bary_points.numel(), (got.bary_x.numel(), ref.bary_points.numel())
    assert (got.bary_x.cpu() - ref.bary_points).abs().max().item() <= tol
    assert (got.bary_w.cpu() - ref.bary_weights).abs().max().item() <= tol


@pytest.mark.parametrize("K", [2, 3, 5, 8])
@pytest.mark.parametrize("T", [1, 3, 25])
def test_mmot1d_matches_oracle(U, K, T):
    probs = W.config_mmot1d(count=6, K=K, n=40, seed=100 + K, ragged=True, rho=[0.5, 1.0, 3.0][K % 3])
    probs[0].alphas[0] = probs[0].alphas[0].copy()
    probs[0].alphas[0][::7] = 0.0  # zero weights
    probs[1].xs[1] = probs[1].xs[1][:1].copy()  # a one-point measure
    probs[1].alphas[1] = probs[1].alphas[1][:1].copy()
    out = U.mmot1d_batched(probs, T)
    for p in range(len(probs)):
        got = type("G", (), {})()
        got.f, got.bary_x, got.bary_w = out.f[p], out.bary_x[p], out.bary_w[p]
        check(got, probs[p], T)


def test_mmot1d_paper_size(U):
    """K = 8 measures of 200 points (the barycenter experiment's shape), 50 steps, 4 problems."""
    probs = W.config_mmot1d(count=4, K=8, n=200, seed=7)
    out = U.mmot1d_batched(probs, 50)
    for p in range(len(probs)):
        got = type("G", (), {})()
        got.f, got.bary_x, got.bary_w = out.f[p], out.bary_x[p], out.bary_w[p]
        check(got, probs[p], 50)
        # the barycenter's mass is the plan's, equal to each re-weighted marginal's
        assert out.bary_w[p].sum().item() > 0


def test_mmot1d_invalid_problem_reported_alone(U):
    probs = W.config_mmot1d(count=3, K=3, n=20, seed=9)
    probs[1].xs[0] = probs[1].xs[0][::-1].copy()  # not ascending
    out = U.mmot1d_batched(probs, 5, check=False)
    assert out.status == [0, 1, 0] and out.code == 1
    assert bool(torch.isnan(out.f[1][0]).all())
    got = type("G", (), {})()
    got.f, got.bary_x, got.bary_w = out.f[2], out.bary_x[2], out.bary_w[2]
    check(got, probs[2], 5)
