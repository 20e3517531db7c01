"""uot_softmin_noalloc against uot_softmin, through the C ABI.

uot_softmin_noalloc serves callers that cannot allocate device memory (a host
program without an allocator, a plug-in whose host forbids allocation, a
real-time loop): it runs the softmin sweep on a 32 MiB scratch array built into
the library.  This file is collected last so that a failure here leaves every
other test already run.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2201_00730_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _tol(eps, ref):
    return 1e-4 * eps + 2.0 * 2.0 ** -23 * ref.abs()


def _spec(U, p):
    dev = torch.device("cuda:0")
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    return U.Spec(t(p.a), t(p.b), p.eps, p.rho1, p.rho2, x=t(p.x), y=t(p.y))


def test_noalloc_matches_workspace_entry_point_two_calls_in_a_row():
    from paper_2201_00730_gb300 import build, uot as U
    build.build()
    rng = np.random.default_rng(3)
    cases = [(W.random_problem(20000, 13001, 3, seed=1, eps=1e-2, zero_frac=0.05), 0),
             (W.random_problem(5003, 7000, 2, seed=2, eps=5e-2), 1)]
    for p, axis in cases:
        spec = _spec(U, p)
        nk = p.m if axis == 0 else p.n
        pot = torch.from_numpy((0.2 * rng.standard_normal(nk)).astype(np.float32)).cuda()
        ref = U.softmin(spec, pot, axis).double()
        got = U.softmin_noalloc(spec, pot, axis).double()
        torch.cuda.synchronize()
        assert bool(((got - ref).abs() <= _tol(p.eps, ref)).all()), (got - ref).abs().max().item()
    # a repeat of the first problem after the second call left its data in the shared scratch
    p, axis = cases[0]
    spec = _spec(U, p)
    pot = torch.zeros(p.m, device="cuda")
    ref = U.softmin(spec, pot, 0).double()
    got = U.softmin_noalloc(spec, pot, 0).double()
    assert bool(((got - ref).abs() <= _tol(p.eps, ref)).all())


def test_noalloc_rejects_problems_beyond_the_scratch():
    from paper_2201_00730_gb300 import build, uot as U
    build.build()
    L = U.lib()
    big = U.Problem(400000, 400000, 3, 0, 2.0, 0, 1e-3, 1.0, 1.0, 256, 256, None, 256, 256)
    st = L.uot_softmin_noalloc(C.byref(big), 0, C.c_void_p(256), C.c_void_p(256), None)
    assert st == 7 and b"built-in scratch" in L.uot_last_error()
