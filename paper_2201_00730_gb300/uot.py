"""Python binding of libuot (ctypes over the C ABI of include/uot.h).

Argument marshalling only: every step of every solve runs in the CUDA kernels
of libuot.so.  PyTorch provides device memory and the current stream.  There
is no CPU fallback: if the library is missing or no GPU is present, calls
raise.

Paper: Sejourne, Vialard, Peyre, "Faster Unbalanced Optimal Transport:
Translation invariant Sinkhorn and 1-D Frank-Wolfe" (AISTATS 2022).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libuot.so")

UOT_OK = 0
UOT_NOT_CONVERGED = 6
STATUS_NAMES = {0: "UOT_OK", 1: "UOT_ERR_INVALID_ARG", 2: "UOT_ERR_WORKSPACE", 3: "UOT_ERR_CUDA",
                4: "UOT_ERR_NONFINITE", 5: "UOT_ERR_TIMEOUT", 6: "UOT_NOT_CONVERGED", 7: "UOT_ERR_UNSUPPORTED"}
COST_POINTS, COST_DENSE = 0, 1


class UOTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Problem(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("dim", C.c_int32), ("cost_kind", C.c_int32),
                ("p", C.c_float), ("ordering", C.c_int32),
                ("eps", C.c_double), ("rho1", C.c_double), ("rho2", C.c_double),
                ("x", C.c_void_p), ("y", C.c_void_p), ("C", C.c_void_p), ("a", C.c_void_p), ("b", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("check_every", C.c_int32), ("tol", C.c_double),
                ("warm_start", C.c_int32), ("lse_reference", C.c_int32), ("residual_history", C.c_void_p),
                ("anderson_k", C.c_int32), ("anderson_reg", C.c_double), ("anderson_buf", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("status", C.c_int32), ("lse_misses", C.c_int32),
                ("residual", C.c_double), ("lambda_", C.c_double)]


class Batch(C.Structure):
    _fields_ = [("count", C.c_int32), ("reserved", C.c_int32),
                ("n", C.c_void_p), ("m", C.c_void_p), ("dim", C.c_void_p),
                ("eps", C.c_void_p), ("rho1", C.c_void_p), ("rho2", C.c_void_p),
                ("x_off", C.c_void_p), ("y_off", C.c_void_p), ("a_off", C.c_void_p), ("b_off", C.c_void_p),
                ("x", C.c_void_p), ("y", C.c_void_p), ("a", C.c_void_p), ("b", C.c_void_p)]


class FW1DBatch(C.Structure):
    _fields_ = [("count", C.c_int32), ("n_iter", C.c_int32), ("p", C.c_double),
                ("n", C.c_void_p), ("m", C.c_void_p), ("x_off", C.c_void_p), ("y_off", C.c_void_p),
                ("rho1", C.c_void_p), ("rho2", C.c_void_p),
                ("x", C.c_void_p), ("a", C.c_void_p), ("y", C.c_void_p), ("b", C.c_void_p)]


class MMOT1DBatch(C.Structure):
    _fields_ = [("count", C.c_int32), ("n_iter", C.c_int32), ("K", C.c_int32), ("reserved", C.c_int32),
                ("n", C.c_void_p), ("off", C.c_void_p), ("rho", C.c_void_p), ("omega", C.c_void_p),
                ("x", C.c_void_p), ("alpha", C.c_void_p)]


_lib = None


def lib() -> C.CDLL:
    """Load libuot.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libuot.so not found at {LIB_PATH}: build it with "
                               f"`python -m paper_2201_00730_gb300.build` (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        P, V, S = C.POINTER(Problem), C.c_void_p, C.c_size_t
        L.uot_workspace_size.argtypes = [P]
        L.uot_workspace_size.restype = S
        L.uot_softmin.argtypes = [P, C.c_int32, V, V, V, S, V]
        L.uot_softmin.restype = C.c_int
        L.uot_softmin_noalloc.argtypes = [P, C.c_int32, V, V, V]
        L.uot_softmin_noalloc.restype = C.c_int
        for fn in (L.uot_sinkhorn, L.uot_ti_sinkhorn, L.uot_g_sinkhorn):
            fn.argtypes = [P, C.POINTER(Options), V, V, C.POINTER(Result), V, S, V]
            fn.restype = C.c_int
        L.uot_dual_value.argtypes = [P, V, V, V, C.c_int32, V, S, V]
        L.uot_dual_value.restype = C.c_int
        L.uot_grad.argtypes = [P, V, V, V, V, V, V, V, S, V]
        L.uot_grad.restype = C.c_int
        L.uot_anderson_workspace.argtypes = [C.c_int32, C.c_int32]
        L.uot_anderson_workspace.restype = S
        L.uot_unrolled_workspace_size.argtypes = [P, C.c_int32, C.c_int32]
        L.uot_unrolled_workspace_size.restype = S
        L.uot_grad_unrolled.argtypes = [P, C.c_int32, C.c_int32, V, V, V, V, V, V, S, V]
        L.uot_grad_unrolled.restype = C.c_int
        L.uot_batch_workspace_size.argtypes = [C.POINTER(Batch)]
        L.uot_batch_workspace_size.restype = S
        L.uot_sinkhorn_batched.argtypes = [C.POINTER(Batch), C.POINTER(Options), C.c_int32, V, V,
                                           C.POINTER(Result), V, S, V]
        L.uot_sinkhorn_batched.restype = C.c_int
        L.uot_fw1d_workspace_size.argtypes = [C.POINTER(FW1DBatch)]
        L.uot_fw1d_workspace_size.restype = S
        L.uot_fw1d_batched.argtypes = [C.POINTER(FW1DBatch), V, V, C.POINTER(C.c_int32), V, S, V]
        L.uot_fw1d_batched.restype = C.c_int
        L.uot_plan_create.argtypes = [P, C.POINTER(Options), C.c_int32, C.POINTER(C.c_void_p)]
        L.uot_plan_create.restype = C.c_int
        L.uot_plan_destroy.argtypes = [V]
        L.uot_plan_destroy.restype = None
        L.uot_plan_workspace_size.argtypes = [V]
        L.uot_plan_workspace_size.restype = S
        L.uot_plan_solve.argtypes = [V, V, V, V, V, S, V]
        L.uot_plan_solve.restype = C.c_int
        L.uot_test_set_wait_limit.argtypes = [C.c_int64]
        L.uot_test_set_wait_limit.restype = None
        L.uot_mmot1d_workspace_size.argtypes = [C.POINTER(MMOT1DBatch)]
        L.uot_mmot1d_workspace_size.restype = S
        L.uot_mmot1d_barycenter_size.argtypes = [C.POINTER(MMOT1DBatch)]
        L.uot_mmot1d_barycenter_size.restype = S
        L.uot_mmot1d_batched.argtypes = [C.POINTER(MMOT1DBatch), V, V, V, C.POINTER(C.c_int32),
                                         C.POINTER(C.c_int32), V, S, V]
        L.uot_mmot1d_batched.restype = C.c_int
        L.uot_kernel_launches.argtypes = []
        L.uot_kernel_launches.restype = C.c_uint64
        L.uot_profile_begin.argtypes = []
        L.uot_profile_begin.restype = C.c_int
        L.uot_profile_end.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.uot_profile_end.restype = C.c_int
        L.uot_sinkhorn_phi_workspace_size.argtypes = [P]
        L.uot_sinkhorn_phi_workspace_size.restype = S
        L.uot_sinkhorn_phi.argtypes = [P, C.POINTER(Options), C.c_int32, C.c_int32, C.c_int32, V, V,
                                       C.POINTER(Result), V, S, V]
        L.uot_sinkhorn_phi.restype = C.c_int
        L.uot_tune_set.argtypes = [C.c_char_p, C.c_int32, C.c_int32, C.c_int64]
        L.uot_tune_set.restype = C.c_int
        L.uot_tune_get.argtypes = [C.c_char_p, C.c_int32, C.c_int64, C.POINTER(C.c_int64)]
        L.uot_tune_get.restype = C.c_int
        L.uot_tune_bucket.argtypes = [C.c_int64]
        L.uot_tune_bucket.restype = C.c_int32
        L.uot_tune_clear.argtypes = []
        L.uot_tune_clear.restype = C.c_int
        L.uot_tune_load.argtypes = [C.c_char_p]
        L.uot_tune_load.restype = C.c_int
        L.uot_last_error.argtypes = []
        L.uot_last_error.restype = C.c_char_p
        L.uot_version.argtypes = []
        L.uot_version.restype = C.c_char_p
        _lib = L
        _apply_packaged_tuning()
    return _lib


def _apply_packaged_tuning():
    """Loads the launch-shape cache shipped with the package when it was measured on
    this device (see autotune.py); the built-in shapes stay in force otherwise."""
    if os.environ.get("UOT_NO_TUNE_CACHE") or not torch.cuda.is_available():
        return
    from . import autotune
    try:
        autotune.load()
    except (OSError, ValueError, UOTError) as e:
        import warnings
        warnings.warn(f"tuning cache not applied: {e}")


def _check(status: int, allow=(UOT_OK,)) -> int:
    if status not in allow:
        raise UOTError(status, lib().uot_last_error().decode())
    return status


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev_f32(t, name, shape=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass
class Spec:
    """Device-resident problem: points (x, y) or a dense cost C, weights a, b, parameters."""
    a: torch.Tensor
    b: torch.Tensor
    eps: float
    rho1: float
    rho2: float
    x: torch.Tensor | None = None
    y: torch.Tensor | None = None
    C: torch.Tensor | None = None
    p: float = 2.0
    ordering: int = 0   # 0 automatic, 1 Morton tiles (dim <= 3, p = 2), 2 never

    def __post_init__(self):
        if self.C is None and (self.x is None or self.y is None):
            raise ValueError("give points x and y, or a dense cost C")
        if self.x is not None and self.x.dim() == 1:
            self.x = self.x[:, None].contiguous()
        if self.y is not None and self.y.dim() == 1:
            self.y = self.y[:, None].contiguous()
        n, m = self.a.shape[0], self.b.shape[0]
        _dev_f32(self.a, "a", (n,))
        _dev_f32(self.b, "b", (m,))
        if self.C is not None:
            _dev_f32(self.C, "C", (n, m))
        else:
            _dev_f32(self.x, "x", (n, self.x.shape[1]))
            _dev_f32(self.y, "y", (m, self.x.shape[1]))

    @property
    def n(self):
        return self.a.shape[0]

    @property
    def m(self):
        return self.b.shape[0]

    def struct(self) -> Problem:
        dense = self.C is not None
        return Problem(self.n, self.m, 0 if dense else self.x.shape[1], COST_DENSE if dense else COST_POINTS,
                       float(self.p), int(self.ordering), float(self.eps), float(self.rho1), float(self.rho2),
                       None if dense else self.x.data_ptr(), None if dense else self.y.data_ptr(),
                       self.C.data_ptr() if dense else None, self.a.data_ptr(), self.b.data_ptr())

    def workspace(self) -> torch.Tensor:
        pr = self.struct()
        nbytes = lib().uot_workspace_size(C.byref(pr))
        if nbytes == 0:
            raise UOTError(1, lib().uot_last_error().decode())
        return torch.empty(nbytes, dtype=torch.uint8, device=self.a.device)


def workspace_size(spec: Spec) -> int:
    pr = spec.struct()
    return int(lib().uot_workspace_size(C.byref(pr)))


def softmin(spec: Spec, pot: torch.Tensor, axis: int, ws: torch.Tensor | None = None) -> torch.Tensor:
    """axis 0: Smin_b^eps(C(x_i,.) - pot) for every i; axis 1: Smin_a^eps(C(.,y_j) - pot) for every j."""
    pr = spec.struct()
    nq, nk = (spec.n, spec.m) if axis == 0 else (spec.m, spec.n)
    _dev_f32(pot, "pot", (nk,))
    out = torch.empty(nq, dtype=torch.float32, device=spec.a.device)
    ws = spec.workspace() if ws is None else ws
    _check(lib().uot_softmin(C.byref(pr), axis, _ptr(pot), _ptr(out), _ptr(ws), ws.numel(), _stream()))
    return out


def softmin_noalloc(spec: Spec, pot: torch.Tensor, axis: int) -> torch.Tensor:
    """uot_softmin without a workspace: the library's built-in 32 MiB scratch is used.

    For callers that cannot allocate device memory; see include/uot.h.
    """
    pr = spec.struct()
    nq, nk = (spec.n, spec.m) if axis == 0 else (spec.m, spec.n)
    _dev_f32(pot, "pot", (nk,))
    out = torch.empty(nq, dtype=torch.float32, device=spec.a.device)
    _check(lib().uot_softmin_noalloc(C.byref(pr), axis, _ptr(pot), _ptr(out), _stream()))
    return out


@dataclass
class SolveOut:
    f: torch.Tensor
    g: torch.Tensor
    iters: int
    converged: bool
    status: int
    residual: float
    lam: float
    history: torch.Tensor | None = None
    lse_misses: int = 0


LSE_REFERENCE = {"auto": 0, "off": 1, "eager": 2}


def solve(spec: Spec, method: str = "ti", max_iter: int = 1000, tol: float = 0.0, check_every: int = 10,
          f0: torch.Tensor | None = None, history: bool = False, ws: torch.Tensor | None = None,
          f: torch.Tensor | None = None, g: torch.Tensor | None = None, lse_reference: str = "auto",
          anderson_k: int = 0, anderson_reg: float = 1e-7) -> SolveOut:
    """Plain ('plain'), translation-invariant ('ti', H-Sinkhorn) or G-Sinkhorn ('g') on the device.

    Returns the translated potentials (f, g), the iteration count and the
    fixed-point residual of the returned pair.  `lse_reference` ('auto', 'off',
    'eager') controls the fixed-reference sweeps of the tiled path (same result
    within rounding, different speed).  anderson_k in 2..6 turns on Anderson
    extrapolation every anderson_k iterations (regularisation anderson_reg,
    relative to the trace of the residuals' Gram matrix).
    """
    pr = spec.struct()
    dev = spec.a.device
    f = torch.empty(spec.n, dtype=torch.float32, device=dev) if f is None else _dev_f32(f, "f", (spec.n,))
    g = torch.empty(spec.m, dtype=torch.float32, device=dev) if g is None else _dev_f32(g, "g", (spec.m,))
    if f0 is not None:
        f.copy_(f0)
    hist = torch.full((max_iter + 1,), float("nan"), dtype=torch.float32, device=dev) if history else None
    if lse_reference not in LSE_REFERENCE:
        raise ValueError("lse_reference must be 'auto', 'off' or 'eager'")
    abuf = None
    if anderson_k:
        nbytes = int(lib().uot_anderson_workspace(spec.n, int(anderson_k)))
        if nbytes == 0:
            raise ValueError("anderson_k must be 0 or 2..6")
        abuf = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    opt = Options(int(max_iter), int(check_every), float(tol), 1 if f0 is not None else 0,
                  LSE_REFERENCE[lse_reference], None if hist is None else hist.data_ptr(),
                  int(anderson_k), float(anderson_reg), None if abuf is None else abuf.data_ptr())
    res = Result()
    ws = spec.workspace() if ws is None else ws
    if method not in ("ti", "plain", "g"):
        raise ValueError("method must be 'ti', 'plain' or 'g'")
    fn = {"ti": lib().uot_ti_sinkhorn, "plain": lib().uot_sinkhorn, "g": lib().uot_g_sinkhorn}[method]
    st = fn(C.byref(pr), C.byref(opt), _ptr(f), _ptr(g), C.byref(res), _ptr(ws), ws.numel(), _stream())
    _check(st, allow=(UOT_OK, UOT_NOT_CONVERGED))
    return SolveOut(f, g, res.iters, bool(res.converged), st, res.residual, res.lambda_, hist, res.lse_misses)


VARIANTS = {"plain": 0, "ti": 1, "g": 2}
PHI = {"kl": 0, "berg": 1}


def solve_phi(spec: Spec, method: str = "g", phi1: str = "berg", phi2: str = "berg", max_iter: int = 1000,
              tol: float = 0.0, check_every: int = 10, f0: torch.Tensor | None = None) -> SolveOut:
    """F-Sinkhorn ('f') or G-Sinkhorn ('g') with the divergences phi1 (on a) and phi2 (on b),
    each 'kl' or 'berg' (uot_sinkhorn_phi).  Returns (f, g), lambda (G) and the residual
    max |g_t - g_(t-1)| of the last iteration."""
    if method not in ("f", "g") or phi1 not in PHI or phi2 not in PHI:
        raise ValueError("method 'f' or 'g'; phi1, phi2 'kl' or 'berg'")
    pr = spec.struct()
    dev = spec.a.device
    f = torch.empty(spec.n, dtype=torch.float32, device=dev)
    g = torch.empty(spec.m, dtype=torch.float32, device=dev)
    if f0 is not None:
        f.copy_(f0)
    nbytes = int(lib().uot_sinkhorn_phi_workspace_size(C.byref(pr)))
    if nbytes == 0:
        raise UOTError(1, lib().uot_last_error().decode())
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    opt = Options(int(max_iter), int(check_every), float(tol), 1 if f0 is not None else 0, 0, None, 0, 0.0, None)
    res = Result()
    st = lib().uot_sinkhorn_phi(C.byref(pr), C.byref(opt), 0 if method == "f" else 2, PHI[phi1], PHI[phi2],
                                _ptr(f), _ptr(g), C.byref(res), _ptr(ws), ws.numel(), _stream())
    _check(st, allow=(UOT_OK, UOT_NOT_CONVERGED))
    return SolveOut(f, g, res.iters, bool(res.converged), st, res.residual, res.lambda_, None, 0)


class Plan:
    """A solve prepared once and run without host synchronisation (uot_plan_create / uot_plan_solve).

    solve() enqueues the whole solve on the current stream and returns at once; inside a
    torch.cuda.graph capture it becomes part of the captured graph.  The outcome is written to a
    device-side uot_result (result() reads it, synchronising).  Inputs are the Spec's tensors,
    which must stay alive; f, g and the workspace belong to the plan object.
    """

    def __init__(self, spec: Spec, method: str = "ti", max_iter: int = 1000, tol: float = 0.0,
                 check_every: int = 10, lse_reference: str = "auto", warm_start: bool = False,
                 history: bool = False):
        if method not in VARIANTS:
            raise ValueError("method must be 'ti', 'plain' or 'g'")
        self.spec = spec
        dev = spec.a.device
        self._pr = spec.struct()
        self.history = (torch.full((max_iter + 1,), float("nan"), dtype=torch.float32, device=dev)
                        if history else None)
        self._opt = Options(int(max_iter), int(check_every), float(tol), 1 if warm_start else 0,
                            LSE_REFERENCE[lse_reference], None if self.history is None else self.history.data_ptr(),
                            0, 0.0, None)
        h = C.c_void_p()
        _check(lib().uot_plan_create(C.byref(self._pr), C.byref(self._opt), VARIANTS[method], C.byref(h)))
        self._h = h
        nbytes = int(lib().uot_plan_workspace_size(h))
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.f = torch.zeros(spec.n, dtype=torch.float32, device=dev)
        self.g = torch.zeros(spec.m, dtype=torch.float32, device=dev)
        self.res = torch.zeros(C.sizeof(Result), dtype=torch.uint8, device=dev)

    def solve(self):
        """Enqueue the solve on the current stream (f is read first when warm_start was set)."""
        _check(lib().uot_plan_solve(self._h, _ptr(self.f), _ptr(self.g), _ptr(self.res), _ptr(self.ws),
                                    self.ws.numel(), _stream()))
        return self

    def result(self) -> Result:
        """The device-side uot_result of the latest solve (synchronises with it)."""
        return Result.from_buffer_copy(bytes(self.res.cpu().numpy()))

    def close(self):
        if getattr(self, "_h", None):
            torch.cuda.synchronize(self.spec.a.device)  # no solve of this plan is still running
            lib().uot_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dual_value(spec: Spec, f: torch.Tensor, g: torch.Tensor, primal: bool = False,
               ws: torch.Tensor | None = None) -> torch.Tensor:
    """F_eps(f, g) (and, with primal=True, the primal value of the induced plan and its mass), FP64."""
    pr = spec.struct()
    _dev_f32(f, "f", (spec.n,))
    _dev_f32(g, "g", (spec.m,))
    out = torch.zeros(3, dtype=torch.float64, device=spec.a.device)
    ws = spec.workspace() if ws is None else ws
    _check(lib().uot_dual_value(C.byref(pr), _ptr(f), _ptr(g), _ptr(out), 1 if primal else 0, _ptr(ws),
                                ws.numel(), _stream()))
    return out if primal else out[:1]


def grad(spec: Spec, f: torch.Tensor, g: torch.Tensor, wrt=("a", "b", "x", "y"),
         ws: torch.Tensor | None = None) -> dict:
    """Envelope gradients of UOT at the optimal pair (f, g) with respect to a, b, x, y."""
    pr = spec.struct()
    _dev_f32(f, "f", (spec.n,))
    _dev_f32(g, "g", (spec.m,))
    dev = spec.a.device
    out = {}
    if "a" in wrt:
        out["a"] = torch.empty(spec.n, dtype=torch.float32, device=dev)
    if "b" in wrt:
        out["b"] = torch.empty(spec.m, dtype=torch.float32, device=dev)
    if "x" in wrt and spec.C is None:
        out["x"] = torch.empty_like(spec.x)
    if "y" in wrt and spec.C is None:
        out["y"] = torch.empty_like(spec.y)
    ws = spec.workspace() if ws is None else ws
    _check(lib().uot_grad(C.byref(pr), _ptr(f), _ptr(g), _ptr(out.get("a")), _ptr(out.get("b")),
                          _ptr(out.get("x")), _ptr(out.get("y")), _ptr(ws), ws.numel(), _stream()))
    return out


def grad_unrolled(spec: Spec, T: int = 200, ckpt_every: int = 20):
    """Value F_eps(f_T, g_T) after T TI iterations from zero and its exact (unrolled) gradient
    with respect to a, b, x, y.  Returns (value (FP64 tensor [1]), dict of gradients)."""
    pr = spec.struct()
    nbytes = lib().uot_unrolled_workspace_size(C.byref(pr), int(T), int(ckpt_every))
    if nbytes == 0:
        raise UOTError(1, lib().uot_last_error().decode())
    dev = spec.a.device
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    val = torch.zeros(1, dtype=torch.float64, device=dev)
    out = {"a": torch.empty(spec.n, dtype=torch.float32, device=dev),
           "b": torch.empty(spec.m, dtype=torch.float32, device=dev),
           "x": torch.empty_like(spec.x), "y": torch.empty_like(spec.y)}
    _check(lib().uot_grad_unrolled(C.byref(pr), int(T), int(ckpt_every), _ptr(val), _ptr(out["a"]),
                                   _ptr(out["b"]), _ptr(out["x"]), _ptr(out["y"]), _ptr(ws), ws.numel(), _stream()))
    return val, out


class UOTLoss(torch.autograd.Function):
    """UOT(a, b; x, y) as a differentiable scalar.

    Forward: TI-Sinkhorn to `tol`, then the FP64 dual value at the returned pair.
    Backward: envelope gradients (uot_grad) scaled by the incoming gradient.
    """

    @staticmethod
    def forward(ctx, x, y, a, b, eps, rho1, rho2, max_iter=10000, tol=1e-6, check_every=10):
        spec = Spec(a.detach().contiguous(), b.detach().contiguous(), eps, rho1, rho2,
                    x=x.detach().contiguous(), y=y.detach().contiguous())
        ws = spec.workspace()
        r = solve(spec, "ti", max_iter=max_iter, tol=tol, check_every=check_every, ws=ws)
        val = dual_value(spec, r.f, r.g, ws=ws)[0]
        ctx.spec, ctx.f, ctx.g = spec, r.f, r.g
        return val.to(torch.float32)

    @staticmethod
    def backward(ctx, gout):
        gr = grad(ctx.spec, ctx.f, ctx.g)
        s = gout.to(torch.float32)
        return (gr["x"] * s, gr["y"] * s, gr["a"] * s, gr["b"] * s, None, None, None, None, None, None)


def kernel_launches() -> int:
    """Kernels launched by libuot in this process so far."""
    return int(lib().uot_kernel_launches())


class SweepProfile:
    """Context manager bracketing every sweep launch of this thread with CUDA events.

    After exit: .sweep_ms (summed device time), .timed, .launches.
    """

    def __enter__(self):
        _check(lib().uot_profile_begin())
        return self

    def __exit__(self, *exc):
        ms, timed, n = C.c_double(), C.c_int64(), C.c_int64()
        _check(lib().uot_profile_end(C.byref(ms), C.byref(timed), C.byref(n)))
        self.sweep_ms, self.timed, self.launches = ms.value, timed.value, n.value
        return False


@dataclass
class BatchOut:
    f: list            # per-problem f (device tensors, views into one packed buffer)
    g: list
    iters: list
    converged: list
    residual: list
    lam: list
    status: int
    device_s: float | None = None   # CUDA-event time of the library call on its stream (timing=True)


_side_streams = {}


def _graph_stream(dev):
    """A non-default stream for calls that capture CUDA graphs (capture is impossible on the legacy
    default stream): the current stream if it is not the default one, else one side stream per device."""
    cur = torch.cuda.current_stream(dev)
    if cur.cuda_stream != 0:
        return cur
    key = dev.index if dev.index is not None else torch.cuda.current_device()
    if key not in _side_streams:
        _side_streams[key] = torch.cuda.Stream(device=dev)
    return _side_streams[key]


def solve_batched(problems, method: str = "ti", max_iter: int = 20000, tol: float = 1e-6,
                  check_every: int = 10, device="cuda:0", graph: bool = True, timing: bool = False) -> BatchOut:
    """Solve many independent point-cloud problems in one batched call.

    `problems`: sequence of objects with numpy/torch arrays x (n x d), y (m x d), a (n), b (m) and floats
    eps, rho1, rho2 (d in 1..3, p = 2).  Inputs are packed into device arrays here (marshalling only).
    graph=True runs the call on a non-default stream, where the library captures each chunk of
    check_every iterations once as a CUDA graph and replays it; graph=False passes the legacy default
    stream, on which the library launches every half-step itself (same kernels, same results).
    """
    import numpy as np
    dev = torch.device(device)
    cnt = len(problems)
    n = np.array([p.x.shape[0] for p in problems], dtype=np.int32)
    m = np.array([p.y.shape[0] for p in problems], dtype=np.int32)
    d = np.array([p.x.shape[1] for p in problems], dtype=np.int32)
    eps = np.array([p.eps for p in problems], dtype=np.float64)
    r1 = np.array([p.rho1 for p in problems], dtype=np.float64)
    r2 = np.array([p.rho2 for p in problems], dtype=np.float64)
    xo = np.concatenate([[0], np.cumsum(n.astype(np.int64) * d)[:-1]]).astype(np.int64)
    yo = np.concatenate([[0], np.cumsum(m.astype(np.int64) * d)[:-1]]).astype(np.int64)
    ao = np.concatenate([[0], np.cumsum(n.astype(np.int64))[:-1]]).astype(np.int64)
    bo = np.concatenate([[0], np.cumsum(m.astype(np.int64))[:-1]]).astype(np.int64)
    cat = lambda vs: torch.from_numpy(np.ascontiguousarray(np.concatenate(
        [np.asarray(v, dtype=np.float32).ravel() for v in vs]))).to(dev)
    X, Y = cat([p.x for p in problems]), cat([p.y for p in problems])
    A, B = cat([p.a for p in problems]), cat([p.b for p in problems])
    host = [n, m, d, eps, r1, r2, xo, yo, ao, bo]
    bt = Batch(cnt, 0, *[h.ctypes.data for h in host], X.data_ptr(), Y.data_ptr(), A.data_ptr(), B.data_ptr())
    nbytes = lib().uot_batch_workspace_size(C.byref(bt))
    if nbytes == 0:
        raise UOTError(1, lib().uot_last_error().decode())
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    F = torch.empty(A.numel(), dtype=torch.float32, device=dev)
    G = torch.empty(B.numel(), dtype=torch.float32, device=dev)
    res = (Result * cnt)()
    opt = Options(int(max_iter), int(check_every), float(tol), 0, 0, None)
    cur = torch.cuda.current_stream(dev)
    if graph:
        side = _graph_stream(dev)
        side.wait_stream(cur)
        handle = C.c_void_p(side.cuda_stream)
    else:
        side = torch.cuda.default_stream(dev)
        handle = C.c_void_p(0)
    if timing:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(side)
    st = lib().uot_sinkhorn_batched(C.byref(bt), C.byref(opt), 1 if method == "ti" else 0, _ptr(F), _ptr(G),
                                    res, _ptr(ws), ws.numel(), handle)
    if timing:
        ev1.record(side)
    if side is not cur:
        cur.wait_stream(side)
    _check(st, allow=(UOT_OK, UOT_NOT_CONVERGED))
    fs = [F[ao[k]:ao[k] + n[k]] for k in range(cnt)]
    gs = [G[bo[k]:bo[k] + m[k]] for k in range(cnt)]
    dsec = None
    if timing:
        ev1.synchronize()
        dsec = ev0.elapsed_time(ev1) * 1e-3
    return BatchOut(fs, gs, [r.iters for r in res], [bool(r.converged) for r in res],
                    [r.residual for r in res], [r.lambda_ for r in res], st, dsec)


@dataclass
class FW1DOut:
    f: list            # per-problem translated potentials (device FP64 views into one packed buffer)
    g: list
    status: list       # per-problem status codes
    code: int          # return code of the call


def fw1d_batched(problems, n_iter: int, p: float = 2.0, device="cuda:0", check: bool = True) -> FW1DOut:
    """1-D unregularised UOT by Frank-Wolfe on H_0 (Sec. 4, Alg. 2) for many problems in one call.

    `problems`: sequence of objects with 1-D arrays x (n, ascending), a (n), y (m, ascending), b (m) and
    floats rho1, rho2.  Inputs are packed into device arrays here (marshalling only).  With check=False a
    failing problem is reported in `status` instead of raising.
    """
    import numpy as np
    dev = torch.device(device)
    cnt = len(problems)
    n = np.array([np.asarray(q.x).size for q in problems], dtype=np.int32)
    m = np.array([np.asarray(q.y).size for q in problems], dtype=np.int32)
    xo = np.concatenate([[0], np.cumsum(n.astype(np.int64))[:-1]]).astype(np.int64)
    yo = np.concatenate([[0], np.cumsum(m.astype(np.int64))[:-1]]).astype(np.int64)
    r1 = np.array([q.rho1 for q in problems], dtype=np.float64)
    r2 = np.array([q.rho2 for q in problems], dtype=np.float64)
    cat = lambda vs: torch.from_numpy(np.ascontiguousarray(np.concatenate(
        [np.asarray(v, dtype=np.float32).ravel() for v in vs]))).to(dev)
    X, A = cat([q.x for q in problems]), cat([q.a for q in problems])
    Y, B = cat([q.y for q in problems]), cat([q.b for q in problems])
    host = [n, m, xo, yo, r1, r2]
    bt = FW1DBatch(cnt, int(n_iter), float(p), *[h.ctypes.data for h in host],
                   X.data_ptr(), A.data_ptr(), Y.data_ptr(), B.data_ptr())
    nbytes = lib().uot_fw1d_workspace_size(C.byref(bt))
    if nbytes == 0:
        raise UOTError(1, lib().uot_last_error().decode())
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    F = torch.empty(X.numel(), dtype=torch.float64, device=dev)
    G = torch.empty(Y.numel(), dtype=torch.float64, device=dev)
    stat = (C.c_int32 * cnt)()
    code = lib().uot_fw1d_batched(C.byref(bt), _ptr(F), _ptr(G), stat, _ptr(ws), ws.numel(), _stream())
    if check:
        _check(code)
    fs = [F[xo[k]:xo[k] + n[k]] for k in range(cnt)]
    gs = [G[yo[k]:yo[k] + m[k]] for k in range(cnt)]
    return FW1DOut(fs, gs, list(stat), code)


@dataclass
class MMOT1DOut:
    f: list            # per problem, per measure: translated potentials (device FP64 views)
    bary_x: list       # per problem: barycenter points (device FP64 views)
    bary_w: list       # per problem: barycenter weights
    status: list
    code: int


def mmot1d_batched(problems, n_iter: int, device="cuda:0", check: bool = True) -> MMOT1DOut:
    """1-D unbalanced multi-marginal OT and barycenters (Sec. 5) by Frank-Wolfe, many problems in one call.

    `problems`: sequence of objects with lists xs (K ascending 1-D arrays), alphas (K weight arrays),
    omega (K barycentric weights summing to one) and a float rho; every problem has the same K.
    Inputs are packed into device arrays here (marshalling only).
    """
    import numpy as np
    dev = torch.device(device)
    cnt = len(problems)
    K = len(problems[0].xs)
    n = np.array([[np.asarray(xk).size for xk in q.xs] for q in problems], dtype=np.int32).reshape(-1)
    off = np.concatenate([[0], np.cumsum(n.astype(np.int64))[:-1]]).astype(np.int64)
    rho = np.array([q.rho for q in problems], dtype=np.float64)
    om = np.array([list(q.omega) for q in problems], dtype=np.float64).reshape(-1)
    cat = lambda vs: torch.from_numpy(np.ascontiguousarray(np.concatenate(
        [np.asarray(v, dtype=np.float32).ravel() for v in vs]))).to(dev)
    X = cat([xk for q in problems for xk in q.xs])
    A = cat([ak for q in problems for ak in q.alphas])
    host = [n, off, rho, om]
    bt = MMOT1DBatch(cnt, int(n_iter), K, 0, *[h.ctypes.data for h in host], X.data_ptr(), A.data_ptr())
    nbytes = lib().uot_mmot1d_workspace_size(C.byref(bt))
    if nbytes == 0:
        raise UOTError(1, lib().uot_last_error().decode())
    nb = int(lib().uot_mmot1d_barycenter_size(C.byref(bt)))
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    F = torch.empty(X.numel(), dtype=torch.float64, device=dev)
    BX = torch.zeros(nb, dtype=torch.float64, device=dev)
    BW = torch.zeros(nb, dtype=torch.float64, device=dev)
    blen = (C.c_int32 * cnt)()
    stat = (C.c_int32 * cnt)()
    code = lib().uot_mmot1d_batched(C.byref(bt), _ptr(F), _ptr(BX), _ptr(BW), blen, stat, _ptr(ws), ws.numel(),
                                    _stream())
    if check:
        _check(code)
    fs, bxs, bws = [], [], []
    bo = 0
    for p in range(cnt):
        fs.append([F[off[p * K + k]:off[p * K + k] + n[p * K + k]] for k in range(K)])
        bxs.append(BX[bo:bo + blen[p]])
        bws.append(BW[bo:bo + blen[p]])
        bo += int(n[p * K:(p + 1) * K].sum())
    return MMOT1DOut(fs, bxs, bws, list(stat), code)


def tune_set(knob: str, value: int, dim: int = -1, bucket: int = -1) -> None:
    """Sets (value != 0) or clears (value 0) one entry of the launch-shape table."""
    _check(lib().uot_tune_set(knob.encode(), int(dim), int(bucket), int(value)))


def tune_get(knob: str, dim: int = -1, entries: int = 0) -> int:
    """The entry that applies to a sweep of `entries` cost entries, 0 for the built-in rule."""
    v = C.c_int64(0)
    _check(lib().uot_tune_get(knob.encode(), int(dim), int(entries), C.byref(v)))
    return int(v.value)


def tune_bucket(entries: int) -> int:
    return int(lib().uot_tune_bucket(int(entries)))


def tune_clear() -> None:
    _check(lib().uot_tune_clear())


def tune_load(path: str) -> None:
    """Adds the entries of a JSON tuning cache (see autotune.py)."""
    _check(lib().uot_tune_load(os.fspath(path).encode()))


def version() -> str:
    return lib().uot_version().decode()
