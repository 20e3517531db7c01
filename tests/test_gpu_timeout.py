"""Failure detection on the GPU without a fault: every mbarrier wait of the tensor-core
sweep (dim >= 32) is bounded, and a wait that gives up must come back as UOT_ERR_TIMEOUT with the
CUDA context still usable.  The test hook uot_test_set_wait_limit(-1) lets the main-loop
waits poll no time at all, so that the first of them gives up; the waits that drain
copies and MMAs in flight keep their full limit."""
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


def spec_of(U, p, ordering=0):
    dev = torch.device("cuda:0")
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    return U.Spec(t(p.a), t(p.b), p.eps, p.rho1, p.rho2, x=t(p.x), y=t(p.y), ordering=ordering)


CASES = {
    # clouds on the tcgen05 cross-term sweep: one K block short of full, and two full ones
    "d48": lambda: W.random_problem(900, 700, 48, seed=32, eps=5e-2, rho1=0.5, rho2=0.5),
    "d64": lambda: W.random_problem(1000, 777, 64, seed=33, eps=5e-2, rho1=0.5, rho2=0.5),
}


@pytest.mark.parametrize("kind", list(CASES))
def test_wait_that_gives_up_reports_timeout_and_context_survives(U, kind):
    p = CASES[kind]()
    # unit expected squared distance, as the D = 64 workloads
    sd = np.sqrt(1.0 / (2.0 * p.x.shape[1]))
    rng = np.random.default_rng(5)
    p.x = (sd * rng.standard_normal(p.x.shape)).astype(np.float32)
    p.y = (sd * rng.standard_normal(p.y.shape)).astype(np.float32)
    spec = spec_of(U, p)
    L = U.lib()
    L.uot_test_set_wait_limit(-1)
    try:
        with pytest.raises(U.UOTError) as ei:
            U.solve(spec, "ti", max_iter=4, tol=1e-12, check_every=1)
        assert ei.value.status == 5, ei.value  # UOT_ERR_TIMEOUT
    finally:
        L.uot_test_set_wait_limit(0)
    torch.cuda.synchronize()  # the context is intact: nothing faulted
    # the same problem solves normally afterwards and matches the oracle
    T = 6
    r = U.solve(spec, "ti", max_iter=T, tol=0.0)
    ref = O.ti_sinkhorn(O.cost_matrix(p.x, p.y), p.a, p.b, p.eps, p.rho1, p.rho2, T)
    err = (r.f.double().cpu() - ref.f).abs()
    assert bool((err <= 1e-4 * p.eps + 2 * 2.0 ** -23 * ref.f.abs()).all()), err.max().item()


def test_gradient_wait_that_gives_up_leaves_nan_and_context_survives(U):
    """uot_grad is asynchronous: when a bounded wait of the tensor-core moment sweep
    (dim >= 32) gives up, the spatial gradients come back NaN rather than wrong but finite,
    and the next call on the same context gives the envelope gradients of the oracle."""
    p = CASES["d64"]()
    sd = np.sqrt(1.0 / (2.0 * p.x.shape[1]))
    rng = np.random.default_rng(7)
    p.x = (sd * rng.standard_normal(p.x.shape)).astype(np.float32)
    p.y = (sd * rng.standard_normal(p.y.shape)).astype(np.float32)
    spec = spec_of(U, p)
    r = U.solve(spec, "ti", max_iter=30, tol=0.0)
    L = U.lib()
    L.uot_test_set_wait_limit(-1)
    try:
        bad = U.grad(spec, r.f, r.g, wrt=("x", "y"))
        torch.cuda.synchronize()
    finally:
        L.uot_test_set_wait_limit(0)
    assert bool(torch.isnan(bad["x"]).any()) and bool(torch.isnan(bad["y"]).any())
    torch.cuda.synchronize()  # nothing faulted
    gr = U.grad(spec, r.f, r.g)
    ea, eb, ex, ey = O.envelope_grads(p.x, p.y, p.a, p.b, r.f.double().cpu(), r.g.double().cpu(),
                                      p.eps, p.rho1, p.rho2)
    for k, e in (("a", ea), ("b", eb), ("x", ex), ("y", ey)):
        assert bool(torch.isfinite(gr[k]).all()), k
        rel = ((gr[k].double().cpu() - e).norm() / e.norm()).item()
        assert rel < 1e-4, (k, rel)
