"""Fixed-reference sweeps of the tiled path (options.lse_reference) against the oracle.

Each row's log-sum-exp from the previous iteration can serve as the exponent
reference of the next sweep; rows that leave the window around it are
recomputed exactly.  Every setting must therefore give the oracle's iterates
within the usual tolerance, including runs where the reference misses.
"""
import numpy as np
import pytest
import torch

from oracle import uot as O
from paper_2201_00730_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    from paper_2201_00730_gb300 import build, uot
    build.build()
    return uot


def spec_of(U, p, ordering=1):
    dev = torch.device("cuda:0")
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    return U.Spec(t(p.a), t(p.b), p.eps, p.rho1, p.rho2, x=t(p.x), y=t(p.y), p=p.p, ordering=ordering)


# Morton tiles with the solver's half-steps on the tensor cores (1) and on CUDA cores only (3)
TILED = pytest.mark.parametrize("ordering", [1], ids=["tiled"])


def assert_pot_close(got, ref, eps, what=""):
    got = got.detach().double().cpu()
    ref = torch.as_tensor(ref, dtype=torch.float64)
    err = (got - ref).abs()
    tol = 1e-4 * eps + 2.0 * 2.0 ** -23 * ref.abs()
    assert not bool((err > tol).any()), f"{what}: max err {err.max().item():.3e} (eps={eps})"


@TILED
@pytest.mark.parametrize("policy", ["off", "auto", "eager"])
@pytest.mark.parametrize("method", ["plain", "ti"])
def test_iterates_match_oracle_every_policy(U, method, policy, ordering):
    pr = W.random_problem(1611, 1437, 3, seed=33, eps=0.02, rho1=0.3, rho2=2.0, mass_a=1.3, mass_b=0.6,
                          zero_frac=0.1)
    spec = spec_of(U, pr, ordering)
    C = O.cost_matrix(pr.x, pr.y)
    for T in (1, 2, 9, 80):
        r = U.solve(spec, method, max_iter=T, lse_reference=policy)
        ref = (O.ti_sinkhorn if method == "ti" else O.sinkhorn)(C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, T)
        assert_pot_close(r.f, ref.f, pr.eps, f"{policy} f after {T}")
        assert_pot_close(r.g, ref.g, pr.eps, f"{policy} g after {T}")
        if policy == "off":
            assert r.lse_misses == 0
        if method == "ti":
            assert abs(r.lam - ref.lam) < 1e-4 * pr.eps


@TILED
def test_eager_reference_misses_are_recomputed(U, ordering):
    """Strong damping (rho = eps = 0.01: aprox halves every half-step) and a warm
    start with one spike (+5 on one point) make the potentials fall by several
    units per iteration, i.e. hundreds of log2 units in every row's log-sum-exp,
    far beyond the window: the eager setting must recompute rows, and still
    match the oracle."""
    pr = W.random_problem(900, 1100, 2, seed=8, eps=1e-2, rho1=1e-2, rho2=1e-2, mass_a=1.0, mass_b=1.7)
    spec = spec_of(U, pr, ordering)
    C = O.cost_matrix(pr.x, pr.y)
    f0 = np.zeros(900, dtype=np.float32)
    f0[0] = 5.0
    misses = {}
    for method in ("plain", "ti"):
        r = U.solve(spec, method, max_iter=6, f0=torch.from_numpy(f0).cuda(), lse_reference="eager")
        misses[method] = r.lse_misses
        if method == "ti":
            ref = O.ti_sinkhorn(C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, 6, fb0=f0)
        else:
            ref = O.sinkhorn(C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, 6, f0=f0)
        assert_pot_close(r.f, ref.f, pr.eps, f"{method} f")
        assert_pot_close(r.g, ref.g, pr.eps, f"{method} g")
    assert misses["plain"] > 0, misses


@TILED
def test_policies_converge_to_the_same_fixed_point(U, ordering):
    pr = W.random_problem(3000, 2500, 3, seed=4, eps=5e-3, rho1=1.0, rho2=1.0, mass_a=1.0, mass_b=0.7)
    spec = spec_of(U, pr, ordering)
    out = {p: U.solve(spec, "ti", max_iter=5000, tol=1e-6, lse_reference=p) for p in ("off", "auto", "eager")}
    for p, r in out.items():
        assert r.converged, p
    assert abs(out["auto"].iters - out["off"].iters) <= 10
    for p in ("auto", "eager"):
        assert (out[p].f - out["off"].f).abs().max().item() < 1e-4 * pr.eps + 2e-5
        assert (out[p].g - out["off"].g).abs().max().item() < 1e-4 * pr.eps + 2e-5


def test_resident_solver_reference_misses(U):
    """The resident cluster solver (auto ordering, N M <= 2^20) takes each row's
    previous log-sum-exp as a fixed reference; with the strong damping and the
    spiked warm start above the references miss, the rows are redone exactly
    (counted in lse_misses) and the iterates still match the oracle."""
    pr = W.random_problem(900, 1100, 2, seed=8, eps=1e-2, rho1=1e-2, rho2=1e-2, mass_a=1.0, mass_b=1.7)
    spec = spec_of(U, pr, 0)
    C = O.cost_matrix(pr.x, pr.y)
    f0 = np.zeros(900, dtype=np.float32)
    f0[0] = 5.0
    for method in ("plain", "ti"):
        r = U.solve(spec, method, max_iter=6, f0=torch.from_numpy(f0).cuda())
        if method == "ti":
            ref = O.ti_sinkhorn(C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, 6, fb0=f0)
        else:
            ref = O.sinkhorn(C, pr.a, pr.b, pr.eps, pr.rho1, pr.rho2, 6, f0=f0)
        assert_pot_close(r.f, ref.f, pr.eps, f"{method} f")
        assert_pot_close(r.g, ref.g, pr.eps, f"{method} g")
        if method == "plain":
            assert r.lse_misses > 0
