"""Thin ctypes binding of libsaa (include/saa.h).

Argument marshalling only: tensors are passed as raw device pointers with
torch's current CUDA stream; every step of the estimator runs in libsaa's
kernels.  There is no CPU or eager-PyTorch fallback: if the library is not
built, or no CUDA device is present, calls raise.

Names follow the C ABI: :func:`saa_eval`, :func:`saa_grad`,
:func:`saa_solve`, :func:`saa_generate`, plus :class:`Problem` for the
``saa_problem`` struct (the law of the samples R_i of Sec. 3.1,
arXiv 2404.11631).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import torch

from . import build as _build

SAA_OK, SAA_EINVAL, SAA_ENOMEM, SAA_ECUDA, SAA_ETIMEOUT, SAA_EDEVICE, SAA_EUNSUPPORTED = range(7)
LAW_GAUSS, LAW_LOGN_STD, LAW_STUDENT_T, LAW_MIX = range(4)
PRECS = {"fp64": 0, "fp32": 1, "bf16x3": 2, "fp8x": 3, "f16x3": 4}


class SAAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libsaa status {status}: {msg}")
        self.status = status


class _CProblem(C.Structure):
    _fields_ = [
        ("d", C.c_int32),
        ("law", C.c_int32),
        ("N", C.c_int64),
        ("nu", C.c_int32),
        ("reserved", C.c_int32),
        ("lam", C.c_double),
        ("seed", C.c_uint64),
        ("instance", C.c_uint32),
        ("epoch", C.c_uint32),
        ("mu", C.c_void_p),
        ("chol", C.c_void_p),
        ("sd", C.c_void_p),
    ]


class _CNewsvendor(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("S", C.c_int64),
        ("seed", C.c_uint64),
        ("instance", C.c_uint32),
        ("epoch", C.c_uint32),
        ("mu", C.c_void_p),
        ("sigma", C.c_void_p),
        ("k", C.c_void_p),
        ("h", C.c_void_p),
        ("v", C.c_void_p),
    ]


_lock = threading.Lock()
_lib = None
_ctx: dict[int, C.c_void_p] = {}


def lib():
    """Loads libsaa.so (building it in-tree first if it is missing).  With
    SAA_BOUNDS_CHECK=1 in the environment it loads the index-checked build,
    libsaa_bounds.so, building or refreshing it first."""
    global _lib
    with _lock:
        if _lib is None:
            if os.environ.get("SAA_BOUNDS_CHECK") == "1":
                path = _build.build(bounds=True)
            else:
                path = _build.LIB
                if not os.path.exists(path):
                    path = _build.build()
            L = C.CDLL(path)
            vp, sz = C.c_void_p, C.c_size_t
            pp = C.POINTER(_CProblem)
            L.saa_ctx_create.argtypes = [C.POINTER(vp), C.c_int]
            L.saa_ctx_create.restype = C.c_int
            L.saa_ctx_destroy.argtypes = [vp]
            L.saa_ctx_sync.argtypes = [vp, vp]
            L.saa_ctx_sync.restype = C.c_int
            L.saa_workspace_size.argtypes = [vp, pp, C.c_int32, C.c_int, C.c_int]
            L.saa_workspace_size.restype = sz
            L.saa_eval.argtypes = [vp, pp, C.c_int32, vp, C.c_int, vp, vp, vp, vp, sz, vp]
            L.saa_eval.restype = C.c_int
            L.saa_eval_host_workspace_size.argtypes = [vp, pp, C.c_int32, C.c_int]
            L.saa_eval_host_workspace_size.restype = sz
            L.saa_eval_host.argtypes = [vp, pp, C.c_int32, vp, C.c_int, vp, vp, vp, vp, sz, vp]
            L.saa_eval_host.restype = C.c_int
            L.saa_partials_workspace_size.argtypes = [vp, pp, C.c_int64, C.c_int32, C.c_int, C.c_int]
            L.saa_partials_workspace_size.restype = sz
            L.saa_partials.argtypes = [vp, pp, C.c_int64, C.c_int64, C.c_int32, vp, C.c_int, C.c_int, vp, vp, sz, vp]
            L.saa_partials.restype = C.c_int
            L.saa_partials_merge.argtypes = [vp, C.c_int32, C.c_int64, vp, vp, vp]
            L.saa_partials_merge.restype = C.c_int
            L.saa_finalize_partials.argtypes = [vp, pp, C.c_int32, vp, vp, vp, vp, vp, vp, vp]
            L.saa_finalize_partials.restype = C.c_int
            L.saa_grad.argtypes = [vp, pp, C.c_int32, vp, C.c_int, vp, vp, vp, sz, vp]
            L.saa_grad.restype = C.c_int
            L.saa_solve.argtypes = [vp, pp, vp, C.c_int32, C.c_int32, C.c_int64, C.c_int, vp, vp, vp, vp, sz, vp]
            L.saa_solve.restype = C.c_int
            L.saa_generate.argtypes = [vp, pp, C.c_int64, C.c_int64, C.c_int, vp, vp, vp, vp]
            L.saa_generate.restype = C.c_int
            L.saa_profile_enable.argtypes = [vp, C.c_int]
            L.saa_profile_enable.restype = C.c_int
            L.saa_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.saa_profile_read.restype = C.c_int
            L.saa_workspace_size_batched.argtypes = [vp, C.c_int32, pp, C.POINTER(C.c_int32), C.c_int]
            L.saa_workspace_size_batched.restype = sz
            L.saa_eval_batched.argtypes = [vp, C.c_int32, pp, C.POINTER(C.c_int32), vp, C.c_int, vp, vp, vp, vp, sz,
                                           vp]
            L.saa_eval_batched.restype = C.c_int
            L.saa_generate_moments_workspace_size.argtypes = [vp, pp, C.c_int64, C.c_int64, C.c_int]
            L.saa_generate_moments_workspace_size.restype = sz
            L.saa_generate_moments.argtypes = [vp, pp, C.c_int64, C.c_int64, C.c_int, vp, vp, vp, sz, vp]
            L.saa_generate_moments.restype = C.c_int
            nvp = C.POINTER(_CNewsvendor)
            L.saa_newsvendor_workspace_size.argtypes = [nvp, C.c_int32]
            L.saa_newsvendor_workspace_size.restype = sz
            L.saa_newsvendor_grad.argtypes = [vp, nvp, C.c_int32, vp, vp, vp, sz, vp]
            L.saa_newsvendor_grad.restype = C.c_int
            L.saa_moments_workspace_size.argtypes = [vp, pp, C.c_int]
            L.saa_moments_workspace_size.restype = sz
            L.saa_moments.argtypes = [vp, pp, C.c_int, vp, vp, vp, sz, vp]
            L.saa_moments.restype = C.c_int
            L.saa_eval_moments_workspace_size.argtypes = [pp, C.c_int32]
            L.saa_eval_moments_workspace_size.restype = sz
            L.saa_eval_moments.argtypes = [vp, pp, C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
            L.saa_eval_moments.restype = C.c_int
            lgp = C.POINTER(_CLogistic)
            L.saa_logistic_pitch.argtypes = [C.c_int32]
            L.saa_logistic_pitch.restype = C.c_int32
            L.saa_logistic_generate.argtypes = [vp, lgp, C.c_int64, C.c_int64, vp, vp, vp]
            L.saa_logistic_generate.restype = C.c_int
            L.saa_logistic_workspace_size.argtypes = [vp, C.c_int32, C.c_int64, C.c_int32, C.c_int]
            L.saa_logistic_workspace_size.restype = sz
            L.saa_logistic_eval.argtypes = [vp, C.c_int32, C.c_int64, vp, vp, vp, C.c_int64, C.c_int32, vp, vp, vp,
                                            vp, vp, vp, sz, vp]
            L.saa_logistic_eval.restype = C.c_int
            L.saa_solve_adaptive_workspace_size.argtypes = [vp, pp, C.POINTER(C.c_int64), C.c_int32, C.c_int]
            L.saa_solve_adaptive_workspace_size.restype = sz
            L.saa_solve_adaptive.argtypes = [vp, pp, vp, C.POINTER(C.c_int64), C.c_int32, C.c_int32, C.c_int32,
                                             C.c_int, vp, vp, vp, vp, sz, vp]
            L.saa_solve_adaptive.restype = C.c_int
            L.saa_eval_samples_workspace_size.argtypes = [vp, C.c_int64, C.c_int32, C.c_int32, C.c_int]
            L.saa_eval_samples_workspace_size.restype = sz
            L.saa_eval_samples.argtypes = [vp, C.c_int64, C.c_int32, vp, vp, vp, C.c_int32, vp, C.c_double, C.c_int,
                                           vp, vp, vp, vp, sz, vp]
            L.saa_eval_samples.restype = C.c_int
            L.saa_cholesky.argtypes = [vp, C.c_int32, vp, vp, vp]
            L.saa_cholesky.restype = C.c_int
            L.saa_batch_workspace_size.argtypes = [vp, C.c_int32, pp, C.POINTER(C.c_int32), C.c_int, C.c_int]
            L.saa_batch_workspace_size.restype = sz
            L.saa_batch_create.argtypes = [vp, C.c_int32, pp, C.POINTER(C.c_int32), vp, C.c_int, vp, vp, vp, vp, vp,
                                           sz, vp, C.POINTER(vp)]
            L.saa_batch_create.restype = C.c_int
            L.saa_batch_launch.argtypes = [vp, vp]
            L.saa_batch_launch.restype = C.c_int
            L.saa_batch_destroy.argtypes = [vp]
            L.saa_batch_destroy.restype = None
            L.saa_selftest_timeout.argtypes = [vp, C.c_uint32, vp]
            L.saa_selftest_timeout.restype = C.c_int
            L.saa_bounds_check_enabled.argtypes = []
            L.saa_bounds_check_enabled.restype = C.c_int32
            L.saa_selftest_bounds.argtypes = [vp, vp]
            L.saa_selftest_bounds.restype = C.c_int
            L.saa_selftest_arith.argtypes = [vp, vp, vp]
            L.saa_selftest_arith.restype = C.c_int
            L.saa_ctx_set_autotune.argtypes = [vp, C.c_int]
            L.saa_ctx_set_autotune.restype = C.c_int
            L.saa_ctx_set_sample_store.argtypes = [vp, sz]
            L.saa_ctx_set_sample_store.restype = C.c_int
            L.saa_plan_info.argtypes = [vp, pp, C.c_int32, C.c_int, C.c_int, C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
            L.saa_plan_info.restype = C.c_int
            L.saa_max_dim.argtypes = [C.c_int]
            L.saa_max_dim.restype = C.c_int32
            L.saa_status_string.argtypes = [C.c_int]
            L.saa_status_string.restype = C.c_char_p
            L.saa_last_error.restype = C.c_char_p
            _lib = L
    return _lib


def _check(status: int):
    if status != SAA_OK:
        raise SAAError(status, lib().saa_last_error().decode())


def context(device: int | None = None) -> C.c_void_p:
    """The libsaa context of a CUDA device (created once per process)."""
    if not torch.cuda.is_available():
        raise RuntimeError("libsaa needs a CUDA device; there is no CPU path")
    dev = torch.cuda.current_device() if device is None else int(device)
    with _lock:
        ctx = _ctx.get(dev)
    if ctx is None:
        ctx = C.c_void_p()
        _check(lib().saa_ctx_create(C.byref(ctx), dev))
        with _lock:
            _ctx[dev] = ctx
    return ctx


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(device) -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


@dataclass
class Problem:
    """Law of the samples R_i = mu + s_i C zhat_i (Sec. 3.1) and estimator options.

    mu   -- [d] float64 CUDA tensor, the mean of R
    chol -- [d, d] float64 CUDA tensor, lower Cholesky factor C of Sigma, or
            None with ``sd`` -- [d] float64 CUDA tensor: Sigma = diag(sd^2),
            the independent assets of Sec. 4.1 at any dimension (FP32, K <= 4)
    N    -- samples per resample; law -- LAW_*; nu -- t-law degrees of freedom
    lam  -- weight of the variance term (0.5 reproduces Eq. 3)
    seed, instance, epoch -- Philox key and counter words
    """

    mu: torch.Tensor
    chol: torch.Tensor | None
    N: int
    law: int = LAW_GAUSS
    nu: int = 4
    lam: float = 0.5
    seed: int = 0
    instance: int = 0
    epoch: int = 0
    sd: torch.Tensor | None = None

    @property
    def d(self) -> int:
        return int(self.mu.shape[0])

    @property
    def device(self):
        return self.mu.device

    def c_struct(self, host: bool = False) -> _CProblem:
        where = "CPU" if host else "CUDA"
        for name, t in (("mu", self.mu), ("chol", self.chol), ("sd", self.sd)):
            if t is not None and not (t.is_cuda != host and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous float64 {where} tensor")
        if self.chol is None and self.sd is None:
            raise ValueError("give chol, or sd for a diagonal covariance")
        if self.chol is not None and self.chol.shape != (self.d, self.d):
            raise ValueError("chol must be [d, d]")
        if self.sd is not None and self.sd.shape != (self.d,):
            raise ValueError("sd must be [d]")
        return _CProblem(self.d, self.law, self.N, self.nu, 0, self.lam, self.seed, self.instance, self.epoch,
                         self.mu.data_ptr(), None if self.chol is None else self.chol.data_ptr(),
                         None if self.sd is None else self.sd.data_ptr())


def _prec(prec) -> int:
    return PRECS[prec] if isinstance(prec, str) else int(prec)


def _decisions(X: torch.Tensor, prob: Problem) -> torch.Tensor:
    if X.dim() == 1:
        X = X.unsqueeze(0)
    if not (X.is_cuda and X.dtype == torch.float64 and X.is_contiguous() and X.shape[1] == prob.d):
        raise ValueError("X must be a contiguous float64 CUDA tensor [K, d]")
    return X


def workspace_size(prob: Problem, K: int, prec="fp32", want_grad: int = 0) -> int:
    cp = prob.c_struct()
    n = lib().saa_workspace_size(context(prob.device.index), C.byref(cp), K, _prec(prec), want_grad)
    if n == 0:
        raise SAAError(SAA_EINVAL, "no workspace size for these arguments: " + lib().saa_last_error().decode())
    return int(n)


def _workspace(prob, K, prec, want_grad, ws):
    need = workspace_size(prob, K, prec, want_grad)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=prob.device)
    return ws


def saa_eval(prob: Problem, X: torch.Tensor, prec="fp32", pbar: bool = True, var: bool = True,
             ws: torch.Tensor | None = None) -> dict:
    """Eq. 4 for the K decisions in X: {'f', 'pbar', 'var'} as float64 CUDA tensors."""
    X = _decisions(X, prob)
    K = X.shape[0]
    dev = prob.device
    f = torch.empty(K, dtype=torch.float64, device=dev)
    pb = torch.empty(K, dtype=torch.float64, device=dev) if pbar else None
    vr = torch.empty(K, dtype=torch.float64, device=dev) if var else None
    ws = _workspace(prob, K, prec, 0, ws)
    cp = prob.c_struct()
    _check(lib().saa_eval(context(dev.index), C.byref(cp), K, _ptr(X), _prec(prec), _ptr(f), _ptr(pb), _ptr(vr),
                          _ptr(ws), ws.numel(), _stream(dev)))
    out = {"f": f}
    if pbar:
        out["pbar"] = pb
    if var:
        out["var"] = vr
    return out


def saa_eval_host_workspace_size(prob: Problem, K: int, prec="fp32", device: int | None = None) -> int:
    """Device scratch bytes of saa_eval_host (prob's tensors on the host)."""
    cp = prob.c_struct(host=True)
    n = lib().saa_eval_host_workspace_size(context(device), C.byref(cp), K, _prec(prec))
    if n == 0:
        raise SAAError(SAA_EINVAL, "no workspace size for these arguments: " + lib().saa_last_error().decode())
    return int(n)


def saa_eval_host(prob: Problem, X: torch.Tensor, prec="fp32", out: dict | None = None,
                  ws: torch.Tensor | None = None, device: int | None = None) -> dict:
    """Eq. 4 with mu, chol (or sd), X and the outputs in host memory (pinned
    tensors copy by DMA): the library copies in, evaluates, copies out and
    waits, so {'f', 'pbar', 'var'} (float64 CPU tensors) are ready on return."""
    if X.dim() == 1:
        X = X.unsqueeze(0)
    if X.is_cuda or X.dtype != torch.float64 or not X.is_contiguous() or X.shape[1] != prob.d:
        raise ValueError("X must be a contiguous float64 CPU tensor [K, d]")
    K = X.shape[0]
    dev = torch.cuda.current_device() if device is None else int(device)
    if out is None:
        out = {k: torch.empty(K, dtype=torch.float64).pin_memory() for k in ("f", "pbar", "var")}
    need = saa_eval_host_workspace_size(prob, K, prec, dev)
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=torch.device("cuda", dev))
    cp = prob.c_struct(host=True)
    _check(lib().saa_eval_host(context(dev), C.byref(cp), K, _ptr(X), _prec(prec), _ptr(out["f"]),
                               _ptr(out.get("pbar")), _ptr(out.get("var")), _ptr(ws), ws.numel(),
                               _stream(torch.device("cuda", dev))))
    return out


def saa_grad(prob: Problem, X: torch.Tensor, prec="fp32", want_f: bool = True,
             ws: torch.Tensor | None = None) -> dict:
    """Eq. 4 and its gradient in w: {'f', 'grad' [K, d]}."""
    X = _decisions(X, prob)
    K = X.shape[0]
    dev = prob.device
    f = torch.empty(K, dtype=torch.float64, device=dev) if want_f else None
    g = torch.empty(K, prob.d, dtype=torch.float64, device=dev)
    ws = _workspace(prob, K, prec, 1, ws)
    cp = prob.c_struct()
    _check(lib().saa_grad(context(dev.index), C.byref(cp), K, _ptr(X), _prec(prec), _ptr(f), _ptr(g), _ptr(ws),
                          ws.numel(), _stream(dev)))
    out = {"grad": g}
    if want_f:
        out["f"] = f
    return out


def partials_len(d: int, K: int, grad: bool) -> int:
    """Length of saa_partials' FP64 vector: P1 [K], P2 [K], P3 [d], P4 [K*d]."""
    return 2 * K + d + (K * d if grad else 0)


def saa_partials(prob: Problem, i0: int, n: int, X: torch.Tensor, prec="fp32", grad: bool = False,
                 ws: torch.Tensor | None = None) -> torch.Tensor:
    """Partial sums of Eq. 4 / Eq. 5 over scenarios [i0, i0 + n) (see
    saa.h): a float64 CUDA vector [P1 | P2 | P3 | P4] that adds across
    disjoint ranges."""
    X = _decisions(X, prob)
    K = X.shape[0]
    dev = prob.device
    cp = prob.c_struct()
    ctx = context(dev.index)
    need = lib().saa_partials_workspace_size(ctx, C.byref(cp), n, K, _prec(prec), int(grad))
    if need == 0:
        raise SAAError(SAA_EINVAL, "no workspace size for these arguments: " + lib().saa_last_error().decode())
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    part = torch.empty(partials_len(prob.d, K, grad), dtype=torch.float64, device=dev)
    _check(lib().saa_partials(ctx, C.byref(cp), int(i0), int(n), K, _ptr(X), _prec(prec), int(grad), _ptr(part),
                              _ptr(ws), ws.numel(), _stream(dev)))
    return part


def saa_partials_merge(parts: torch.Tensor) -> torch.Tensor:
    """Totals of the rows of ``parts`` ([R, len] float64 CUDA), added in row
    order with compensation (bitwise independent of who produced the rows)."""
    if not (parts.is_cuda and parts.dtype == torch.float64 and parts.is_contiguous() and parts.dim() == 2):
        raise ValueError("parts must be a contiguous [R, len] float64 CUDA tensor")
    dev = parts.device
    total = torch.empty(parts.shape[1], dtype=torch.float64, device=dev)
    _check(lib().saa_partials_merge(context(dev.index), parts.shape[0], parts.shape[1], _ptr(parts), _ptr(total),
                                    _stream(dev)))
    return total


def saa_finalize_partials(prob: Problem, X: torch.Tensor, part: torch.Tensor, grad: bool = False) -> dict:
    """Eq. 4, Eq. 5 (and the gradient) from the whole sample's partial sums:
    {'f', 'pbar', 'var'} (+ 'grad' [K, d]) as float64 CUDA tensors."""
    X = _decisions(X, prob)
    K = X.shape[0]
    dev = prob.device
    if not (part.is_cuda and part.dtype == torch.float64 and part.is_contiguous()
            and part.numel() == partials_len(prob.d, K, grad)):
        raise ValueError("part must be a contiguous float64 CUDA vector of partials_len(d, K, grad)")
    out = {k: torch.empty(K, dtype=torch.float64, device=dev) for k in ("f", "pbar", "var")}
    if grad:
        out["grad"] = torch.empty(K, prob.d, dtype=torch.float64, device=dev)
    cp = prob.c_struct()
    _check(lib().saa_finalize_partials(context(dev.index), C.byref(cp), K, _ptr(X), _ptr(part), _ptr(out["f"]),
                                       _ptr(out["pbar"]), _ptr(out["var"]), _ptr(out.get("grad")), _stream(dev)))
    return out


def saa_solve(prob: Problem, w0: torch.Tensor, T: int, M: int = 1, t0: int = 0, prec="fp32",
              ws: torch.Tensor | None = None) -> dict:
    """Algorithm 1 for T iterations from t0: {'w', 'f_trace', 'gap_trace'}."""
    dev = prob.device
    if not (w0.is_cuda and w0.dtype == torch.float64 and w0.is_contiguous() and w0.shape == (prob.d,)):
        raise ValueError("w0 must be a contiguous float64 CUDA tensor [d]")
    w = torch.empty(prob.d, dtype=torch.float64, device=dev)
    ft = torch.empty(max(T, 1), dtype=torch.float64, device=dev)
    gt = torch.empty(max(T, 1), dtype=torch.float64, device=dev)
    ws = _workspace(prob, 1, prec, 2, ws)
    cp = prob.c_struct()
    _check(lib().saa_solve(context(dev.index), C.byref(cp), _ptr(w0), T, M, t0, _prec(prec), _ptr(w), _ptr(ft),
                           _ptr(gt), _ptr(ws), ws.numel(), _stream(dev)))
    return {"w": w, "f_trace": ft[:T], "gap_trace": gt[:T]}


def saa_solve_adaptive(prob: Problem, w0: torch.Tensor, N_sched, M: int = 1, k0: int = 0, prec="fp32",
                       ws: torch.Tensor | None = None) -> dict:
    """Algorithm 1 with N_sched[k] samples in epoch k0 + k (M iterations
    each): {'w', 'f_trace', 'gap_trace'}; prob.N is not used."""
    dev = prob.device
    if not (w0.is_cuda and w0.dtype == torch.float64 and w0.is_contiguous() and w0.shape == (prob.d,)):
        raise ValueError("w0 must be a contiguous float64 CUDA tensor [d]")
    sched = (C.c_int64 * len(N_sched))(*[int(n) for n in N_sched])
    n = len(N_sched)
    cp = prob.c_struct()
    ctx = context(dev.index)
    need = lib().saa_solve_adaptive_workspace_size(ctx, C.byref(cp), sched, n, _prec(prec))
    if need == 0:
        raise SAAError(SAA_EINVAL, "saa_solve_adaptive: invalid schedule or problem")
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    w = torch.empty(prob.d, dtype=torch.float64, device=dev)
    ft = torch.empty(n * M, dtype=torch.float64, device=dev)
    gt = torch.empty(n * M, dtype=torch.float64, device=dev)
    _check(lib().saa_solve_adaptive(ctx, C.byref(cp), _ptr(w0), sched, n, M, k0, _prec(prec), _ptr(w), _ptr(ft),
                                    _ptr(gt), _ptr(ws), ws.numel(), _stream(dev)))
    return {"w": w, "f_trace": ft, "gap_trace": gt}


def saa_generate(prob: Problem, i0: int, n: int, prec="fp32", want_xi: bool = False) -> dict:
    """Innovations zhat [n, d], scales s [n] and optionally samples xi [n, d]."""
    dev = prob.device
    dt = torch.float64 if _prec(prec) == 0 else torch.float32
    z = torch.empty(n, prob.d, dtype=dt, device=dev)
    s = torch.empty(n, dtype=dt, device=dev)
    xi = torch.empty(n, prob.d, dtype=dt, device=dev) if want_xi else None
    cp = prob.c_struct()
    _check(lib().saa_generate(context(dev.index), C.byref(cp), i0, n, _prec(prec), _ptr(z), _ptr(s), _ptr(xi),
                              _stream(dev)))
    out = {"z": z, "s": s}
    if want_xi:
        out["xi"] = xi
    return out


def saa_generate_moments(prob: Problem, i0: int, n: int, prec="fp32", out: dict | None = None) -> dict:
    """Per-dimension sums of the innovations and of their squares over
    scenarios i0 .. i0+n-1: {'sum': [d], 'sumsq': [d]} float64 tensors.
    ``out`` (a previous result, with its 'ws') is reused instead of
    allocating."""
    dev = prob.device
    cp = prob.c_struct()
    ctx = context(dev.index)
    need = lib().saa_generate_moments_workspace_size(ctx, C.byref(cp), i0, n, _prec(prec))
    if need == 0:
        raise SAAError(SAA_EINVAL, lib().saa_last_error().decode())
    if out is not None and out["ws"].numel() >= need and out["sum"].numel() == prob.d:
        ws, s1, s2 = out["ws"], out["sum"], out["sumsq"]
    else:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
        s1 = torch.empty(prob.d, dtype=torch.float64, device=dev)
        s2 = torch.empty(prob.d, dtype=torch.float64, device=dev)
    _check(lib().saa_generate_moments(ctx, C.byref(cp), i0, n, _prec(prec), _ptr(s1), _ptr(s2), _ptr(ws),
                                      ws.numel(), _stream(dev)))
    return {"sum": s1, "sumsq": s2, "ws": ws}


class _CLogistic(C.Structure):
    _fields_ = [("n", C.c_int32), ("reserved", C.c_int32), ("N", C.c_int64), ("seed", C.c_uint64),
                ("instance", C.c_uint32), ("flip", C.c_uint32), ("wstar", C.c_void_p)]


LABEL_NOISE_10PCT = 429496730   # round(0.1 * 2^32): the paper's 10 % label noise


def saa_logistic_generate(n: int, N: int, wstar: torch.Tensor, seed: int = 0, instance: int = 0,
                          flip: int = LABEL_NOISE_10PCT, i0: int = 0, rows: int | None = None) -> dict:
    """Synthetic binary-classification data (Sec. 4.1's setup) on the device:
    {'X': int32 [rows, pitch] feature bits, 'z': uint8 [rows] labels}."""
    if not (wstar.is_cuda and wstar.dtype == torch.int32 and wstar.is_contiguous() and wstar.numel() == n):
        raise ValueError("wstar must be a contiguous int32 CUDA tensor [n]")
    dev = wstar.device
    rows = N - i0 if rows is None else rows
    pitch = int(lib().saa_logistic_pitch(n))
    X = torch.empty(rows, pitch, dtype=torch.int32, device=dev)
    z = torch.empty(rows, dtype=torch.uint8, device=dev)
    cp = _CLogistic(n, 0, N, seed, instance, flip, wstar.data_ptr())
    _check(lib().saa_logistic_generate(context(dev.index), C.byref(cp), i0, rows, _ptr(X), _ptr(z), _stream(dev)))
    return {"X": X, "z": z}


def saa_logistic_eval(X: torch.Tensor, z: torch.Tensor, n: int, W: torch.Tensor, V: torch.Tensor | None = None,
                      idx: torch.Tensor | None = None, want_grad: bool = True, want_hvp: bool | None = None,
                      ws: torch.Tensor | None = None) -> dict:
    """F [K], grad [K, n] and (with V) hvp [K, n] of the logistic objective
    over the rows idx (int64, repeats allowed; all rows when None) of the
    bit matrix X [N, pitch] with labels z [N], for omega = W [K, n]."""
    if W.dim() == 1:
        W = W.unsqueeze(0)
    if V is not None and V.dim() == 1:
        V = V.unsqueeze(0)
    N = int(X.shape[0])
    if not (X.is_cuda and X.dtype == torch.int32 and X.is_contiguous() and X.shape[1] == lib().saa_logistic_pitch(n)):
        raise ValueError("X must be the contiguous int32 CUDA bit matrix [N, saa_logistic_pitch(n)]")
    if not (z.is_cuda and z.dtype == torch.uint8 and z.numel() == N):
        raise ValueError("z must be a uint8 CUDA tensor [N]")
    for name, t in (("W", W), ("V", V)):
        if t is not None and not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.shape[1] == n):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor [K, n]")
    if idx is not None and not (idx.is_cuda and idx.dtype == torch.int64 and idx.is_contiguous()):
        raise ValueError("idx must be a contiguous int64 CUDA tensor")
    want_hvp = (V is not None) if want_hvp is None else want_hvp
    K = int(W.shape[0])
    b = N if idx is None else int(idx.numel())
    dev = X.device
    ctx = context(dev.index)
    has_v = 1 if (V is not None and want_hvp) else 0
    need = lib().saa_logistic_workspace_size(ctx, n, b, K, has_v)
    if need == 0:
        raise SAAError(SAA_EINVAL, lib().saa_last_error().decode())
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    F = torch.empty(K, dtype=torch.float64, device=dev)
    g = torch.empty(K, n, dtype=torch.float64, device=dev) if want_grad else None
    h = torch.empty(K, n, dtype=torch.float64, device=dev) if has_v else None
    _check(lib().saa_logistic_eval(ctx, n, N, _ptr(X), _ptr(z), _ptr(idx), b, K, _ptr(W), _ptr(V), _ptr(F), _ptr(g),
                                   _ptr(h), _ptr(ws), ws.numel(), _stream(dev)))
    out = {"F": F, "ws": ws}
    if g is not None:
        out["grad"] = g
    if h is not None:
        out["hvp"] = h
    return out


@dataclass
class Newsvendor:
    """Newsvendor problem of Sec. 3.2 with normal demands: n products, S
    demand samples each; mu, sigma, k (ordering), h (holding), v (shortage)
    are [n] float64 CUDA tensors."""

    mu: torch.Tensor
    sigma: torch.Tensor
    k: torch.Tensor
    h: torch.Tensor
    v: torch.Tensor
    S: int
    seed: int = 0
    instance: int = 0
    epoch: int = 0

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    def c_struct(self) -> _CNewsvendor:
        ts = (self.mu, self.sigma, self.k, self.h, self.v)
        for t in ts:
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.shape == (self.n,)):
                raise ValueError("newsvendor arrays must be contiguous float64 CUDA tensors of shape [n]")
        return _CNewsvendor(self.n, self.S, self.seed, self.instance, self.epoch, *[t.data_ptr() for t in ts])


def saa_newsvendor_grad(prob: Newsvendor, X: torch.Tensor, return_counts: bool = False):
    """Monte Carlo gradient of the newsvendor cost at K decision vectors X [K, n]."""
    dev = prob.mu.device
    X = X if X.dim() == 2 else X.unsqueeze(0)
    if not (X.is_cuda and X.dtype == torch.float64 and X.is_contiguous() and X.shape[1] == prob.n):
        raise ValueError("X must be a contiguous float64 CUDA tensor [K, n]")
    K = int(X.shape[0])
    cp = prob.c_struct()
    need = lib().saa_newsvendor_workspace_size(C.byref(cp), K)
    if need == 0:
        raise SAAError(SAA_EINVAL, lib().saa_last_error().decode())
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    g = torch.empty(K, prob.n, dtype=torch.float64, device=dev)
    _check(lib().saa_newsvendor_grad(context(dev.index), C.byref(cp), K, _ptr(X), _ptr(g), _ptr(ws), ws.numel(),
                                     _stream(dev)))
    if return_counts:
        return g, ws.view(torch.int32).view(K, prob.n)
    return g


def saa_moments(prob: Problem, prec="f16x3", ws: torch.Tensor | None = None) -> dict:
    """Covariance-first sums of the whitened samples of resample prob.epoch:
    {'M': [d, d] = sum_i a_i a_i', 'mt': [d] = sum_i a_i} (float64)."""
    dev = prob.device
    cp = prob.c_struct()
    ctx = context(dev.index)
    need = lib().saa_moments_workspace_size(ctx, C.byref(cp), _prec(prec))
    if need == 0:
        raise SAAError(SAA_EINVAL, lib().saa_last_error().decode())
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    M = torch.empty(prob.d, prob.d, dtype=torch.float64, device=dev)
    mt = torch.empty(prob.d, dtype=torch.float64, device=dev)
    _check(lib().saa_moments(ctx, C.byref(cp), _prec(prec), _ptr(M), _ptr(mt), _ptr(ws), ws.numel(), _stream(dev)))
    return {"M": M, "mt": mt}


def saa_eval_moments(prob: Problem, X: torch.Tensor, moments: dict, want_grad: bool = True,
                     ws: torch.Tensor | None = None) -> dict:
    """Eq. 4 (f, pbar, var) and, with want_grad, its gradient for the K
    decisions X [K, d] from the moments of saa_moments."""
    X = _decisions(X, prob)
    K = int(X.shape[0])
    dev = prob.device
    cp = prob.c_struct()
    need = lib().saa_eval_moments_workspace_size(C.byref(cp), K)
    if need == 0:
        raise SAAError(SAA_EINVAL, "saa_eval_moments: invalid problem size")
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    f = torch.empty(K, dtype=torch.float64, device=dev)
    pb = torch.empty_like(f)
    var = torch.empty_like(f)
    g = torch.empty(K, prob.d, dtype=torch.float64, device=dev) if want_grad else None
    _check(lib().saa_eval_moments(context(dev.index), C.byref(cp), K, _ptr(X), _ptr(moments["M"]),
                                  _ptr(moments["mt"]), _ptr(f), _ptr(pb), _ptr(var), _ptr(g), _ptr(ws), ws.numel(),
                                  _stream(dev)))
    out = {"f": f, "pbar": pb, "var": var}
    if want_grad:
        out["grad"] = g
    return out


def saa_eval_samples(R: torch.Tensor, X: torch.Tensor, lam: float, prec="f16x3",
                     center: torch.Tensor | None = None, sigma: torch.Tensor | None = None,
                     ws: torch.Tensor | None = None) -> dict:
    """Streamed mode: Eq. 4 (f, pbar, var) over samples held in device
    memory, R [N, d] float32 (scenario i = row i), for the decisions X [K, d]
    float64.  ``center`` [d] float64 (e.g. the samples' mean) is subtracted
    before the split-precision contraction and ``sigma`` [d] float64 (e.g.
    per-column standard deviations) sets the exact power-of-two column
    scaling; neither changes the result beyond rounding.  ``prec`` "fp8x"
    (E4M3 products) needs both."""
    if not (R.is_cuda and R.dtype == torch.float32 and R.is_contiguous() and R.dim() == 2):
        raise ValueError("R must be a contiguous float32 CUDA tensor [N, d]")
    N, d = int(R.shape[0]), int(R.shape[1])
    if X.dim() == 1:
        X = X.unsqueeze(0)
    if not (X.is_cuda and X.dtype == torch.float64 and X.is_contiguous() and X.shape[1] == d):
        raise ValueError("X must be a contiguous float64 CUDA tensor [K, d]")
    for name, v in (("center", center), ("sigma", sigma)):
        if v is not None and not (v.is_cuda and v.dtype == torch.float64 and v.is_contiguous() and v.numel() == d):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor [d]")
    K = int(X.shape[0])
    dev = R.device
    ctx = context(dev.index)
    need = lib().saa_eval_samples_workspace_size(ctx, N, d, K, _prec(prec))
    if need == 0:
        raise SAAError(SAA_EINVAL, lib().saa_last_error().decode())
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    f = torch.empty(K, dtype=torch.float64, device=dev)
    pb = torch.empty_like(f)
    var = torch.empty_like(f)
    _check(lib().saa_eval_samples(ctx, N, d, _ptr(R), _ptr(center), _ptr(sigma), K, _ptr(X), float(lam), _prec(prec),
                                  _ptr(f), _ptr(pb), _ptr(var), _ptr(ws), ws.numel(), _stream(dev)))
    return {"f": f, "pbar": pb, "var": var, "ws": ws}


def saa_cholesky(sigma: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """Lower Cholesky factor C of Sigma (C C' = Sigma) on the device, the
    ``chol`` of :class:`Problem`; ``out`` may be ``sigma`` itself (in place)."""
    if not (sigma.is_cuda and sigma.dtype == torch.float64 and sigma.is_contiguous() and sigma.dim() == 2
            and sigma.shape[0] == sigma.shape[1]):
        raise ValueError("sigma must be a contiguous square float64 CUDA tensor")
    d = int(sigma.shape[0])
    if out is None:
        out = torch.empty_like(sigma)
    elif not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.shape == sigma.shape):
        raise ValueError("out must be a contiguous float64 CUDA tensor shaped like sigma")
    dev = sigma.device
    _check(lib().saa_cholesky(context(dev.index), d, _ptr(sigma), _ptr(out), _stream(dev)))
    return out


class Batch:
    """A ragged batch of problems, marshalled once.  With ``graph=True`` (the
    default) it is a saa_batch: planned once and replayed as a CUDA graph by
    :meth:`run`, optionally with gradients.  With ``graph=False`` every run
    is one saa_eval_batched call (values only).  The decision tensors, mu and
    chol are bound by address: update them in place between runs."""

    def __init__(self, problems: list, Xs: list, prec="fp32", want_pbar=True, want_var=True, want_grad=False,
                 graph=True):
        self.problems, self.Xs, self.prec = problems, [_decisions(X, p) for X, p in zip(Xs, problems)], prec
        if want_grad and not graph:
            raise ValueError("gradients of a batch need graph=True (saa_batch)")
        B = len(problems)
        dev = problems[0].device
        self.B, self.device, self.handle = B, dev, None
        self.cprobs = (_CProblem * B)(*[p.c_struct() for p in problems])
        self.K = (C.c_int32 * B)(*[int(X.shape[0]) for X in self.Xs])
        self.f = [torch.empty(int(X.shape[0]), dtype=torch.float64, device=dev) for X in self.Xs]
        self.pbar = [torch.empty_like(t) for t in self.f] if want_pbar else None
        self.var = [torch.empty_like(t) for t in self.f] if want_var else None
        self.grad = [torch.empty(int(X.shape[0]), p.d, dtype=torch.float64, device=dev)
                     for X, p in zip(self.Xs, problems)] if want_grad else None
        ptrs = lambda ts: (C.c_void_p * B)(*[t.data_ptr() for t in ts]) if ts is not None else None  # noqa: E731
        self.pX, self.pf, self.pp, self.pv = ptrs(self.Xs), ptrs(self.f), ptrs(self.pbar), ptrs(self.var)
        self.pg = ptrs(self.grad)
        ctx = context(dev.index)
        if graph:
            need = lib().saa_batch_workspace_size(ctx, B, self.cprobs, self.K, _prec(prec), int(want_grad))
        else:
            need = lib().saa_workspace_size_batched(ctx, B, self.cprobs, self.K, _prec(prec))
        if need == 0:
            raise SAAError(SAA_EINVAL, lib().saa_last_error().decode())
        self.ws = torch.empty(need, dtype=torch.uint8, device=dev)
        if graph:
            h = C.c_void_p()
            _check(lib().saa_batch_create(ctx, B, self.cprobs, self.K, self.pX, _prec(prec), self.pf, self.pp,
                                          self.pv, self.pg, _ptr(self.ws), self.ws.numel(), _stream(dev),
                                          C.byref(h)))
            self.handle = h

    def run(self) -> dict:
        if self.handle is not None:
            _check(lib().saa_batch_launch(self.handle, _stream(self.device)))
        else:
            _check(lib().saa_eval_batched(context(self.device.index), self.B, self.cprobs, self.K, self.pX,
                                          _prec(self.prec), self.pf, self.pp, self.pv, _ptr(self.ws),
                                          self.ws.numel(), _stream(self.device)))
        out = {"f": self.f}
        if self.pbar is not None:
            out["pbar"] = self.pbar
        if self.var is not None:
            out["var"] = self.var
        if self.grad is not None:
            out["grad"] = self.grad
        return out

    def close(self):
        if self.handle is not None and _lib is not None:
            lib().saa_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def saa_eval_batched(problems: list, Xs: list, prec="fp32") -> dict:
    """Eq. 4 for a ragged batch (one saa_eval_batched call): lists of
    per-problem f, pbar and var tensors."""
    return Batch(problems, Xs, prec, graph=False).run()


def saa_grad_batched(problems: list, Xs: list, prec="fp32") -> dict:
    """Eq. 4 and its gradient for a ragged batch (a saa_batch, launched once):
    lists of per-problem f, pbar, var and grad [K_b, d_b] tensors."""
    b = Batch(problems, Xs, prec, want_grad=True)
    out = b.run()
    torch.cuda.current_stream(b.device).synchronize()
    b.close()
    return out


def saa_selftest_arith(device: int | None = None) -> tuple[int, int]:
    """(quotient, root) mismatch counts of the generator's Markstein-corrected
    arithmetic against IEEE over all 2^23 FP32 uniforms (both 0 when exact)."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    out = torch.empty(2, dtype=torch.int64, device=dev)
    _check(lib().saa_selftest_arith(context(dev.index), _ptr(out), _stream(dev)))
    c = out.cpu()
    return int(c[0]), int(c[1])


def saa_selftest_timeout(budget_us: int = 1000, device: int | None = None):
    """Runs the bounded-wait self-test (see saa.h); saa_ctx_sync then raises SAA_ETIMEOUT."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    _check(lib().saa_selftest_timeout(context(dev.index), budget_us, _stream(dev)))


def saa_bounds_check_enabled() -> bool:
    """True when the loaded library is the index-checked build (see saa.h)."""
    return bool(lib().saa_bounds_check_enabled())


def saa_selftest_bounds(device: int | None = None):
    """Runs the index-check self-test (see saa.h): in the checked build the
    next saa_ctx_sync raises SAA_EDEVICE; the normal build raises
    SAA_EUNSUPPORTED here."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    _check(lib().saa_selftest_bounds(context(dev.index), _stream(dev)))


def saa_ctx_sync(device: int | None = None):
    """Waits for the current stream and raises if a device-side check fired."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    _check(lib().saa_ctx_sync(context(dev.index), _stream(dev)))


def saa_ctx_set_sample_store(max_bytes: int, device: int | None = None):
    """Most bytes of FP32 samples the diagonal-covariance gradient keeps
    between its forward and adjoint passes (0: draw them twice)."""
    _check(lib().saa_ctx_set_sample_store(context(device), int(max_bytes)))


def saa_profile_enable(enable: bool = True, device: int | None = None):
    """Starts / stops event timing of the main sample kernel (see saa.h)."""
    _check(lib().saa_profile_enable(context(device), int(enable)))


def saa_profile_read(device: int | None = None) -> tuple[float, int, int]:
    """(summed main-kernel ms, main-kernel launches, kernels launched) since the last read."""
    ms, n, k = C.c_double(), C.c_int64(), C.c_int64()
    _check(lib().saa_profile_read(context(device), C.byref(ms), C.byref(n), C.byref(k)))
    return ms.value, n.value, k.value


def saa_plan_info(prob: Problem, K: int, prec="fp32", want_grad: bool = False) -> dict:
    """Launch shape of saa_eval / saa_grad for this problem: {'grid', 'cluster', 'tiles'}."""
    g, c, t = C.c_int32(), C.c_int32(), C.c_int64()
    cp = prob.c_struct()
    _check(lib().saa_plan_info(context(prob.device.index), C.byref(cp), K, _prec(prec), int(want_grad), C.byref(g),
                               C.byref(c), C.byref(t)))
    return {"grid": g.value, "cluster": c.value, "tiles": t.value}


def max_dim(prec) -> int:
    return int(lib().saa_max_dim(_prec(prec)))


EXPORTED = ["saa_ctx_create", "saa_ctx_destroy", "saa_ctx_sync", "saa_workspace_size", "saa_eval", "saa_grad",
            "saa_solve", "saa_generate", "saa_max_dim", "saa_status_string", "saa_last_error",
            "saa_profile_enable", "saa_profile_read", "saa_eval_batched", "saa_workspace_size_batched",
            "saa_ctx_set_autotune", "saa_selftest_timeout", "saa_cholesky", "saa_generate_moments",
            "saa_generate_moments_workspace_size", "saa_batch_workspace_size", "saa_batch_create",
            "saa_batch_launch", "saa_batch_destroy", "saa_newsvendor_workspace_size", "saa_newsvendor_grad",
            "saa_moments_workspace_size", "saa_moments", "saa_eval_moments_workspace_size", "saa_eval_moments",
            "saa_eval_samples_workspace_size", "saa_eval_samples", "saa_solve_adaptive_workspace_size",
            "saa_solve_adaptive", "saa_logistic_pitch", "saa_logistic_generate", "saa_logistic_workspace_size",
            "saa_logistic_eval", "saa_ctx_set_sample_store", "saa_selftest_arith", "saa_eval_host_workspace_size",
            "saa_eval_host", "saa_partials_workspace_size", "saa_partials", "saa_finalize_partials",
            "saa_partials_merge", "saa_plan_info", "saa_bounds_check_enabled", "saa_selftest_bounds"]
