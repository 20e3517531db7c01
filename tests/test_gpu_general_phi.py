"""F- and G-Sinkhorn with a general phi^* (Sec. 3) on the GPU against the FP64
oracle: Berg and KL penalties on either side, every sweep path, iterate by
iterate; lambda* against the oracle's; KL/KL against uot_sinkhorn / uot_g_sinkhorn."""
import numpy as np
import pytest
import torch

from oracle import general_phi as GP
from oracle import uot as O
from paper_2201_00730_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    from paper_2201_00730_gb300 import build, uot
    build.build()
    return uot


def dev_t(v):
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda:0")


def assert_close(got, ref, eps, what):
    got, ref = got.double().cpu(), GP._t(ref)
    err = (got - ref).abs()
    tol = 1e-4 * eps + 4 * 2.0 ** -23 * ref.abs()
    assert bool((err <= tol).all()), f"{what}: max err {err.max().item():.3e} (eps {eps})"


def make(U, kind, seed):
    n, m = (611, 437) if kind != "small" else (300, 257)
    pr = W.random_problem(n, m, 2, seed=seed, eps=0.05, rho1=0.7, rho2=1.6, mass_a=1.3, mass_b=0.6, zero_frac=0.1)
    if kind == "dense":
        Cf = W.dense_cost_f32(pr.x, pr.y)
        return pr, U.Spec(dev_t(pr.a), dev_t(pr.b), pr.eps, pr.rho1, pr.rho2, C=dev_t(Cf)), GP._t(Cf)
    spec = U.Spec(dev_t(pr.a), dev_t(pr.b), pr.eps, pr.rho1, pr.rho2, x=dev_t(pr.x), y=dev_t(pr.y),
                  ordering={"tiled": 1, "direct": 2, "small": 0}[kind])
    return pr, spec, O.cost_matrix(pr.x, pr.y)


DIVS = {"kl": GP.KL, "berg": GP.Berg}
PAIRS = [("berg", "berg"), ("kl", "berg"), ("berg", "kl")]


@pytest.mark.parametrize("kind", ["tiled", "direct", "dense", "small"])
@pytest.mark.parametrize("phis", PAIRS, ids=["-".join(p) for p in PAIRS])
def test_f_sinkhorn_iterates(U, kind, phis):
    pr, spec, C = make(U, kind, 81)
    d1, d2 = DIVS[phis[0]](pr.rho1), DIVS[phis[1]](pr.rho2)
    for T in (1, 6):
        r = U.solve_phi(spec, "f", phis[0], phis[1], max_iter=T)
        f, g = GP.f_sinkhorn(C, pr.a, pr.b, pr.eps, d1, d2, T)
        assert_close(r.f, f, pr.eps, f"f after {T}")
        assert_close(r.g, g, pr.eps, f"g after {T}")
        assert r.lam == 0.0 and r.iters == T


@pytest.mark.parametrize("kind", ["tiled", "direct", "dense"])
@pytest.mark.parametrize("phis", PAIRS, ids=["-".join(p) for p in PAIRS])
def test_g_sinkhorn_iterates_and_lambda(U, kind, phis):
    pr, spec, C = make(U, kind, 82)
    d1, d2 = DIVS[phis[0]](pr.rho1), DIVS[phis[1]](pr.rho2)
    for T in (1, 5):
        r = U.solve_phi(spec, "g", phis[0], phis[1], max_iter=T)
        f, g, lam = GP.g_sinkhorn(C, pr.a, pr.b, pr.eps, d1, d2, T)
        assert abs(r.lam - float(lam)) <= 1e-4 * pr.eps + 1e-12 * abs(float(lam)), (T, r.lam, float(lam))
        assert_close(r.f, f, pr.eps, f"f after {T}")
        assert_close(r.g, g, pr.eps, f"g after {T}")


def test_lambda_is_the_maximiser_at_convergence(U):
    # at a G-Sinkhorn fixed point lambda* is 0 in the returned pair's frame: the derivative
    # <a, phi_1^*'(-f)> - <b, phi_2^*'(-g)> of the dual in a common shift vanishes (Prop. 1)
    pr, spec, C = make(U, "direct", 83)
    r = U.solve_phi(spec, "g", "berg", "berg", max_iter=400, tol=1e-6, check_every=10)
    assert r.converged
    f, g = r.f.double().cpu(), r.g.double().cpu()
    a, b = GP._t(pr.a), GP._t(pr.b)
    d1, d2 = GP.Berg(pr.rho1), GP.Berg(pr.rho2)
    grad = (a * d1.dphi_star(-f)).sum() - (b * d2.dphi_star(-g)).sum()
    scale = (a * d1.dphi_star(-f)).sum()
    assert abs(grad.item()) <= 1e-5 * scale.item()


@pytest.mark.parametrize("kind", ["tiled", "direct"])
def test_kl_kl_matches_the_kl_solvers(U, kind):
    pr, spec, C = make(U, kind, 84)
    T = 7
    rf = U.solve_phi(spec, "f", "kl", "kl", max_iter=T)
    ref = O.sinkhorn(C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, T)
    assert_close(rf.f, ref.f, pr.eps, "F-Sinkhorn f")
    rg = U.solve_phi(spec, "g", "kl", "kl", max_iter=T)
    refg = O.g_sinkhorn(C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, T)
    assert_close(rg.f, refg.f, pr.eps, "G-Sinkhorn f")
    assert_close(rg.g, refg.g, pr.eps, "G-Sinkhorn g")
