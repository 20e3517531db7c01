"""The C-ABI library builds, loads and exports every entry point of include/uot.h;
struct layouts agree between the header and the Python binding; argument errors
come back before any device work (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "uot.h")


@pytest.fixture(scope="module")
def L():
    from paper_2201_00730_gb300 import build, uot
    build.build()
    return uot.lib()


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"UOT_API\s+[\w\s\*]+?\b(uot_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert "uot_ti_sinkhorn" in names and len(names) >= 8
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", L._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (uot_\w+)", out))
    assert set(names) <= exported


def test_struct_layout_matches_header():
    from paper_2201_00730_gb300 import uot
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "uot.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(uot_problem), offsetof(uot_problem, eps), offsetof(uot_problem, b),
         sizeof(uot_options), offsetof(uot_options, residual_history), sizeof(uot_result));
  printf("%zu\n", offsetof(uot_result, lambda));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    P, O, R = uot.Problem, uot.Options, uot.Result
    assert vals == [C.sizeof(P), P.eps.offset, P.b.offset, C.sizeof(O), O.residual_history.offset, C.sizeof(R),
                    R.lambda_.offset]


def test_argument_errors_without_device_work(L):
    from paper_2201_00730_gb300 import uot
    assert L.uot_workspace_size(None) == 0
    assert b"NULL" in L.uot_last_error()
    bad = uot.Problem(0, 5, 1, 0, 2.0, 0, 0.1, 1.0, 1.0, 8, 8, None, 8, 8)
    assert L.uot_workspace_size(C.byref(bad)) == 0
    assert b"n and m" in L.uot_last_error()
    neg = uot.Problem(4, 5, 1, 0, 2.0, 0, -0.1, 1.0, 1.0, 8, 8, None, 8, 8)
    st = L.uot_ti_sinkhorn(C.byref(neg), None, None, None, None, None, 0, None)
    assert st == 1 and b"eps" in L.uot_last_error()
    ok = uot.Problem(4, 5, 1, 0, 2.0, 0, 0.1, 1.0, 1.0, 256, 256, None, 256, 256)
    st = L.uot_sinkhorn(C.byref(ok), None, None, None, None, None, 0, None)
    assert st == 1 and b"options" in L.uot_last_error()
    opt = uot.Options(10, 1, 0.0, 0, 0, None)
    st = L.uot_sinkhorn(C.byref(ok), C.byref(opt), None, None, None, None, 0, None)
    assert st == 2  # no workspace
    bad_ref = uot.Options(10, 1, 0.0, 0, 3, None)
    st = L.uot_ti_sinkhorn(C.byref(ok), C.byref(bad_ref), 256, 256, None, 1 << 30, 1 << 40, None)
    assert st == 1 and b"lse_reference" in L.uot_last_error()
    bad_k = uot.Options(10, 1, 0.0, 0, 0, None, 7, 1e-7, None)
    st = L.uot_ti_sinkhorn(C.byref(ok), C.byref(bad_k), 256, 256, None, 1 << 30, 1 << 40, None)
    assert st == 1 and b"anderson_k" in L.uot_last_error()
    bad_reg = uot.Options(10, 1, 0.0, 0, 0, None, 4, -1.0, 1 << 30)
    st = L.uot_g_sinkhorn(C.byref(ok), C.byref(bad_reg), 256, 256, None, 1 << 30, 1 << 40, None)
    assert st == 1 and b"anderson_reg" in L.uot_last_error()
    no_buf = uot.Options(10, 1, 0.0, 0, 0, None, 4, 1e-7, None)
    st = L.uot_sinkhorn(C.byref(ok), C.byref(no_buf), 256, 256, None, 1 << 30, 1 << 40, None)
    assert st == 1 and b"anderson_buf" in L.uot_last_error()
    assert L.uot_anderson_workspace(100, 4) >= 5 * 100 * 4 and L.uot_anderson_workspace(100, 7) == 0
    assert L.uot_anderson_workspace(0, 4) == 0
    bad_order = uot.Problem(4, 5, 1, 0, 2.0, 4, 0.1, 1.0, 1.0, 256, 256, None, 256, 256)
    assert L.uot_workspace_size(C.byref(bad_order)) == 0 and b"ordering" in L.uot_last_error()
    st = L.uot_softmin(C.byref(ok), 3, 256, 256, 256, 1 << 30, None)
    assert st == 1 and b"axis" in L.uot_last_error()
    dense_unaligned = uot.Problem(4, 5, 0, 1, 2.0, 0, 0.1, 1.0, 1.0, None, None, 260, 256, 256)
    assert L.uot_workspace_size(C.byref(dense_unaligned)) == 0
    assert b"16-byte" in L.uot_last_error()
    assert L.uot_version().startswith(b"uot")


def test_fw1d_layout_and_argument_errors(L):
    """uot_fw1d_batch agrees between header and binding; bad batches fail on the host."""
    import numpy as np
    from paper_2201_00730_gb300 import uot
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "uot.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(uot_fw1d_batch), offsetof(uot_fw1d_batch, p), offsetof(uot_fw1d_batch, rho2),
         offsetof(uot_fw1d_batch, b));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    B = uot.FW1DBatch
    assert vals == [C.sizeof(B), B.p.offset, B.rho2.offset, B.b.offset]

    n = np.array([3, 4], dtype=np.int32)
    m = np.array([2, 5], dtype=np.int32)
    xo = np.array([0, 3], dtype=np.int64)
    yo = np.array([0, 2], dtype=np.int64)
    r1 = np.array([1.0, 0.5])
    r2 = np.array([1.0, 2.0])
    host = [n, m, xo, yo, r1, r2]
    ok = B(2, 10, 2.0, *[h.ctypes.data for h in host], 256, 256, 256, 256)
    nbytes = L.uot_fw1d_workspace_size(C.byref(ok))
    assert nbytes >= 6 * 8 * 7  # six FP64 working vectors over 7 points a side
    assert L.uot_fw1d_workspace_size(None) == 0
    for field, val, msg in [("count", 0, b"count"), ("n_iter", 0, b"n_iter"), ("p", 0.5, b"p must")]:
        bad = B(2, 10, 2.0, *[h.ctypes.data for h in host], 256, 256, 256, 256)
        setattr(bad, field, val)
        assert L.uot_fw1d_workspace_size(C.byref(bad)) == 0 and msg in L.uot_last_error()
    r_bad = np.array([1.0, -1.0])
    bad = B(2, 10, 2.0, n.ctypes.data, m.ctypes.data, xo.ctypes.data, yo.ctypes.data, r1.ctypes.data,
            r_bad.ctypes.data, 256, 256, 256, 256)
    assert L.uot_fw1d_workspace_size(C.byref(bad)) == 0 and b"rho" in L.uot_last_error()
    st = L.uot_fw1d_batched(C.byref(ok), None, 256, None, 256, 1 << 30, None)
    assert st == 1 and b"f and g" in L.uot_last_error()
    st = L.uot_fw1d_batched(C.byref(ok), 256, 256, None, None, 1 << 30, None)
    assert st == 2
    st = L.uot_fw1d_batched(C.byref(ok), 256, 256, None, 256, nbytes - 1, None)
    assert st == 2 and b"too small" in L.uot_last_error()


def test_plan_rejects_anderson_and_bad_variant(L):
    """Plans run the stopping rule on the device; Anderson extrapolation stays host-driven and is
    rejected before any CUDA call, as is an unknown variant."""
    from paper_2201_00730_gb300 import uot
    pr = uot.Problem(10, 12, 2, 0, 2.0, 0, 0.1, 1.0, 1.0, 256, 256, None, 256, 256)
    h = C.c_void_p()
    opt = uot.Options(10, 5, 0.0, 0, 0, None, 4, 1e-7, 256)
    assert L.uot_plan_create(C.byref(pr), C.byref(opt), 1, C.byref(h)) == 7
    assert b"Anderson" in L.uot_last_error() and not h.value
    opt = uot.Options(10, 5, 0.0, 0, 0, None, 0, 0.0, None)
    assert L.uot_plan_create(C.byref(pr), C.byref(opt), 5, C.byref(h)) == 1
    assert L.uot_plan_workspace_size(None) == 0


def test_sinkhorn_phi_rejects_bad_variant_and_divergence(L):
    """uot_sinkhorn_phi checks its variant and divergences before any CUDA call."""
    from paper_2201_00730_gb300 import uot
    pr = uot.Problem(10, 12, 2, 0, 2.0, 0, 0.1, 1.0, 1.0, 256, 256, None, 256, 256)
    opt = uot.Options(10, 5, 0.0, 0, 0, None, 0, 0.0, None)
    res = uot.Result()
    p = C.c_void_p(256)
    assert L.uot_sinkhorn_phi(C.byref(pr), C.byref(opt), 1, 0, 1, p, p, C.byref(res), p, 1 << 30, None) == 1
    assert b"variant" in L.uot_last_error()
    assert L.uot_sinkhorn_phi(C.byref(pr), C.byref(opt), 2, 0, 2, p, p, C.byref(res), p, 1 << 30, None) == 1
    assert b"UOT_PHI" in L.uot_last_error()
    assert L.uot_sinkhorn_phi(C.byref(pr), None, 0, 0, 0, p, p, C.byref(res), p, 1 << 30, None) == 1
