"""Plain FP64 CPU oracle for the SAA hot path (arXiv 2404.11631, Sec. 3.1).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2404_11631_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``saa_oracle.c`` (plain C, compiled with
``-ffp-contract=off``); this module only builds it with gcc and marshals
numpy arrays through ctypes.

Functions and the passages they follow:

* :func:`philox` -- Philox4x32-10 (Salmon et al., SC'11), the counter-based
  generator of the samples R_i.
* :func:`generate` -- the scenario generator (normals, law transforms) and
  the samples at scenario precision.
* :func:`saa` / :func:`saa_explicit` -- Eq. 4 with Eq. 5 and its gradient in w.
* :func:`fw` / :func:`fw_step` -- Algorithm 1.
* :func:`rse` -- the relative squared error of Table 2's notes.
* :func:`cholesky` -- the lower Cholesky factor C of Sigma used by the
  normal law of Sec. 3.1 (R = mu + C z).
* :func:`newsvendor_grad`, :func:`newsvendor_demands` -- the newsvendor's
  Monte Carlo gradient (Sec. 3.2, the approximated gradient) and the
  standardised demand samples it counts.

Parity status: every function is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force and independent library routines; the
paper prints no worked example, so no value is pinned to a printed number.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "saa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

LAW_GAUSS, LAW_LOGN_STD, LAW_STUDENT_T, LAW_MIX = 0, 1, 2, 3

CFLAGS = ["-O3", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile ``saa_oracle.c`` into ``_build/liboracle.so`` (gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Problem(C.Structure):
    """Mirror of the oracle's own problem struct (see saa_oracle.c)."""

    _fields_ = [
        ("d", C.c_int32),
        ("N", C.c_int64),
        ("law", C.c_int32),
        ("nu", C.c_int32),
        ("lam", C.c_double),
        ("seed", C.c_uint64),
        ("instance", C.c_uint32),
        ("epoch", C.c_uint32),
        ("mu", C.POINTER(C.c_double)),
        ("chol", C.POINTER(C.c_double)),
        ("sd", C.POINTER(C.c_double)),
    ]


class Newsvendor(C.Structure):
    """Mirror of the oracle's newsvendor struct (see saa_oracle.c)."""

    _fields_ = [
        ("n", C.c_int64),
        ("S", C.c_int64),
        ("seed", C.c_uint64),
        ("instance", C.c_uint32),
        ("epoch", C.c_uint32),
        ("mu", C.POINTER(C.c_double)),
        ("sigma", C.POINTER(C.c_double)),
        ("k", C.POINTER(C.c_double)),
        ("h", C.POINTER(C.c_double)),
        ("v", C.POINTER(C.c_double)),
    ]


class Logistic(C.Structure):
    """Mirror of the oracle's binary-classification data set (saa_oracle.c)."""

    _fields_ = [
        ("n", C.c_int32),
        ("N", C.c_int64),
        ("seed", C.c_uint64),
        ("instance", C.c_uint32),
        ("flip", C.c_uint32),
        ("wstar", C.POINTER(C.c_int32)),
    ]


def _p(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, fp = C.POINTER(C.c_double), C.POINTER(C.c_float)
            u32p, u64p = C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)
            L.oracle_philox_batch.argtypes = [C.c_int64, u32p, u32p, u32p]
            L.oracle_log_f32.argtypes = [C.c_int64, fp, fp]
            L.oracle_log_f64.argtypes = [C.c_int64, dp, dp]
            L.oracle_exp_f32.argtypes = [C.c_int64, fp, fp]
            L.oracle_exp_f64.argtypes = [C.c_int64, dp, dp]
            L.oracle_sincos2pi_f32.argtypes = [C.c_int64, u32p, fp, fp]
            L.oracle_sincos2pi_f64.argtypes = [C.c_int64, u64p, dp, dp]
            L.oracle_constants.argtypes = [C.c_int, dp, C.c_int]
            L.oracle_constants.restype = C.c_int
            pp = C.POINTER(Problem)
            L.oracle_generate.argtypes = [pp, C.c_int, C.c_uint32, C.c_int64, C.c_int64, dp, dp, dp]
            L.oracle_generate.restype = C.c_int
            L.oracle_saa_explicit.argtypes = [C.c_int64, C.c_int, dp, C.c_int, dp, C.c_double, dp, dp, dp, dp]
            L.oracle_saa_explicit.restype = C.c_int
            L.oracle_saa.argtypes = [pp, C.c_int, C.c_uint32, C.c_int, dp, dp, dp, dp, dp]
            L.oracle_saa.restype = C.c_int
            L.oracle_partials.argtypes = [pp, C.c_int, C.c_uint32, C.c_int64, C.c_int64, C.c_int, dp, C.c_int, dp]
            L.oracle_partials.restype = C.c_int
            L.oracle_finalize_partials.argtypes = [C.c_int64, C.c_int, C.c_int, dp, dp, C.c_double, dp, dp, dp, dp,
                                                   dp]
            L.oracle_finalize_partials.restype = C.c_int
            L.oracle_fw_step.argtypes = [C.c_int, dp, dp, C.c_int64, dp, dp]
            L.oracle_fw_step.restype = C.c_int
            L.oracle_fw.argtypes = [pp, C.c_int, dp, C.c_int, C.c_int, C.c_int64, dp, dp, dp, dp]
            L.oracle_fw.restype = C.c_int
            nvp = C.POINTER(Newsvendor)
            L.oracle_newsvendor_demands.argtypes = [nvp, C.c_int64, fp]
            L.oracle_newsvendor_demands.restype = C.c_int
            L.oracle_newsvendor_grad.argtypes = [nvp, C.c_int, dp, dp, C.POINTER(C.c_int64)]
            L.oracle_newsvendor_grad.restype = C.c_int
            L.oracle_newsvendor_grad_range.argtypes = [nvp, C.c_int, dp, C.c_int64, C.c_int64, dp,
                                                       C.POINTER(C.c_int64)]
            L.oracle_newsvendor_grad_range.restype = C.c_int
            lgp = C.POINTER(Logistic)
            u8p = C.POINTER(C.c_uint8)
            L.oracle_logistic_data.argtypes = [lgp, C.c_int64, C.c_int64, u8p, u8p]
            L.oracle_logistic_data.restype = C.c_int
            L.oracle_logistic_eval.argtypes = [lgp, C.POINTER(C.c_int64), C.c_int64, C.c_int, dp, dp, dp, dp, dp]
            L.oracle_logistic_eval.restype = C.c_int
            L.oracle_cholesky.argtypes = [C.c_int, dp, dp]
            L.oracle_cholesky.restype = C.c_int
            L.oracle_rse.argtypes = [C.c_double, C.c_double]
            L.oracle_rse.restype = C.c_double
            L.oracle_max_threads.restype = C.c_int
            _lib = L
    return _lib


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


# --- Philox and elementary functions -------------------------------------

def philox(ctr, key):
    """Philox4x32-10 of counters ``ctr`` [n,4] under keys ``key`` [n,2] (uint32)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, dtype=np.uint32), (ctr.shape[0], 2)))
    out = np.empty_like(ctr)
    lib().oracle_philox_batch(ctr.shape[0], _p(ctr, C.c_uint32), _p(key, C.c_uint32), _p(out, C.c_uint32))
    return out


def log_f32(u):
    u = np.ascontiguousarray(u, dtype=np.float32)
    out = np.empty_like(u)
    lib().oracle_log_f32(u.size, _p(u, C.c_float), _p(out, C.c_float))
    return out


def log_f64(u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    lib().oracle_log_f64(u.size, _p(u), _p(out))
    return out


def exp_f32(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty_like(x)
    lib().oracle_exp_f32(x.size, _p(x, C.c_float), _p(out, C.c_float))
    return out


def exp_f64(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    lib().oracle_exp_f64(x.size, _p(x), _p(out))
    return out


def sincos2pi_f32(num):
    """sin/cos(2 pi n 2^-24) for odd integers n in [1, 2^24)."""
    num = np.ascontiguousarray(num, dtype=np.uint32)
    s = np.empty(num.shape, np.float32)
    c = np.empty(num.shape, np.float32)
    lib().oracle_sincos2pi_f32(num.size, _p(num, C.c_uint32), _p(s, C.c_float), _p(c, C.c_float))
    return s, c


def sincos2pi_f64(num):
    """sin/cos(2 pi n 2^-53) for odd integers n in [1, 2^53)."""
    num = np.ascontiguousarray(num, dtype=np.uint64)
    s = np.empty(num.shape, np.float64)
    c = np.empty(num.shape, np.float64)
    lib().oracle_sincos2pi_f64(num.size, _p(num, C.c_uint64), _p(s), _p(c))
    return s, c


def constants(which: int) -> np.ndarray:
    buf = np.zeros(32, np.float64)
    n = lib().oracle_constants(which, _p(buf), 32)
    if n < 0:
        raise ValueError(which)
    return buf[:n].copy()


# --- problem marshalling ---------------------------------------------------

def make_problem(d, N, mu, chol, law=LAW_GAUSS, nu=4, lam=0.5, seed=0, instance=0, epoch=0, sd=None):
    """Returns (Problem, keepalive) for the given law parameters; chol None
    with ``sd`` [d] gives Sigma = diag(sd^2)."""
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    assert mu.shape == (d,)
    if chol is not None:
        chol = np.ascontiguousarray(chol, dtype=np.float64)
        assert chol.shape == (d, d)
    if sd is not None:
        sd = np.ascontiguousarray(sd, dtype=np.float64)
        assert sd.shape == (d,)
    assert chol is not None or sd is not None
    P = Problem(d, N, law, nu, lam, seed, instance, epoch, _p(mu), _p(chol), _p(sd))
    return P, (mu, chol, sd)


def generate(prob, prec, i0, n, epoch=None, want_xi=False):
    """Innovations zhat [n,d] (promoted to float64), scales s [n], and, when
    ``want_xi``, samples xi [n,d] at scenario precision (promoted)."""
    P, keep = prob
    d = P.d
    z = np.empty((n, d), np.float64)
    s = np.empty(n, np.float64)
    xi = np.empty((n, d), np.float64) if want_xi else None
    ep = P.epoch if epoch is None else epoch
    _check(lib().oracle_generate(C.byref(P), prec, ep, i0, n, _p(z), _p(s), _p(xi)), "generate")
    return z, s, xi


def saa(prob, prec, W, grad=False, epoch=None):
    """Eq. 4 on the generated samples: dict with f, pbar, var (and grad)."""
    P, keep = prob
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    K = W.shape[0]
    f, pb, var = np.empty(K), np.empty(K), np.empty(K)
    g = np.empty((K, P.d)) if grad else None
    ep = P.epoch if epoch is None else epoch
    _check(lib().oracle_saa(C.byref(P), prec, ep, K, _p(W), _p(f), _p(pb), _p(var), _p(g)), "saa")
    out = {"f": f, "pbar": pb, "var": var}
    if grad:
        out["grad"] = g
    return out


def partials(prob, prec, i0, n, W, grad=False, epoch=None):
    """Partial sums over scenarios [i0, i0 + n) with D_i = R_i - mu and
    p_ik = w_k'D_i: [P1 = sum p (K) | P2 = sum p^2 (K) | P3 = sum D (d) |
    P4 = sum D p (K*d, with grad)], float64."""
    P, keep = prob
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    K, d = W.shape[0], P.d
    out = np.empty(2 * K + d + (K * d if grad else 0))
    ep = P.epoch if epoch is None else epoch
    _check(lib().oracle_partials(C.byref(P), prec, ep, i0, n, K, _p(W), int(grad), _p(out)), "partials")
    return out


def finalize_partials(N, W, mu, lam, part, grad=False):
    """Eq. 4, Eq. 5 (and the gradient) from the whole sample's partial sums."""
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    part = np.ascontiguousarray(part, dtype=np.float64)
    K, d = W.shape
    f, pb, var = np.empty(K), np.empty(K), np.empty(K)
    g = np.empty((K, d)) if grad else None
    _check(lib().oracle_finalize_partials(N, d, K, _p(W), _p(mu), lam, _p(part), _p(f), _p(pb), _p(var), _p(g)),
           "finalize_partials")
    out = {"f": f, "pbar": pb, "var": var}
    if grad:
        out["grad"] = g
    return out


def saa_explicit(R, W, lam=0.5, grad=False):
    """Eq. 4 on an explicit sample matrix R [N,d]."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    N, d = R.shape
    K = W.shape[0]
    f, pb, var = np.empty(K), np.empty(K), np.empty(K)
    g = np.empty((K, d)) if grad else None
    _check(lib().oracle_saa_explicit(N, d, _p(R), K, _p(W), lam, _p(f), _p(pb), _p(var), _p(g)), "saa_explicit")
    out = {"f": f, "pbar": pb, "var": var}
    if grad:
        out["grad"] = g
    return out


def fw_step(g, w, t):
    """One Frank-Wolfe step (Algorithm 1): returns (j*, gap, w_next)."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    wn = np.empty_like(w)
    gap = C.c_double()
    js = lib().oracle_fw_step(w.size, _p(g), _p(w), t, _p(wn), C.byref(gap))
    return js, gap.value, wn


def fw(prob, prec, w0, T, M, t0=0, want_w_trace=False):
    """Algorithm 1 for T iterations from t0: dict w, f_trace, gap_trace (w_trace)."""
    P, keep = prob
    w0 = np.ascontiguousarray(w0, dtype=np.float64)
    w = np.empty(P.d)
    ft, gt = np.empty(T), np.empty(T)
    wt = np.empty((T, P.d)) if want_w_trace else None
    _check(lib().oracle_fw(C.byref(P), prec, _p(w0), T, M, t0, _p(w), _p(ft), _p(gt), _p(wt)), "fw")
    out = {"w": w, "f_trace": ft, "gap_trace": gt}
    if want_w_trace:
        out["w_trace"] = wt
    return out


def fw_adaptive(probs, prec, w0, M, k0=0, want_w_trace=False):
    """Algorithm 1 with a sample size per epoch (the resampling step's
    N_k "adapted to k"): epoch k0 + k draws its N samples from probs[k]
    (one problem per epoch, equal but for N) and runs M iterations from the
    global iteration (k0 + k) M, so the step size and the resample index
    follow the global count.  Returns dict w, f_trace, gap_trace (w_trace)."""
    w = np.ascontiguousarray(w0, dtype=np.float64)
    ft, gt, wt = [], [], []
    for k, prob in enumerate(probs):
        out = fw(prob, prec, w, T=M, M=M, t0=(k0 + k) * M, want_w_trace=want_w_trace)
        w = out["w"]
        ft.append(out["f_trace"])
        gt.append(out["gap_trace"])
        if want_w_trace:
            wt.append(out["w_trace"])
    res = {"w": w, "f_trace": np.concatenate(ft), "gap_trace": np.concatenate(gt)}
    if want_w_trace:
        res["w_trace"] = np.concatenate(wt)
    return res


# --- binary classification (Sec. 3.3) --------------------------------------

LABEL_NOISE_10PCT = 429496730   # round(0.1 * 2^32): a label flips when its noise word is below this


def make_logistic(n, N, wstar, seed=0, instance=0, flip=LABEL_NOISE_10PCT):
    """Returns (Logistic, keepalive) for N points with n binary features and
    the integer labelling weights ``wstar`` [n]."""
    w = np.ascontiguousarray(wstar, dtype=np.int32)
    assert w.shape == (n,)
    P = Logistic(n, N, seed, instance, flip, _p(w, C.c_int32))
    return P, w


def logistic_data(prob, i0=0, rows=None):
    """(features uint8 [rows, n], labels uint8 [rows]) of points i0 .. i0+rows-1."""
    P, keep = prob
    rows = P.N - i0 if rows is None else rows
    x = np.empty((rows, P.n), np.uint8)
    z = np.empty(rows, np.uint8)
    _check(lib().oracle_logistic_data(C.byref(P), i0, rows, _p(x, C.c_uint8), _p(z, C.c_uint8)), "logistic_data")
    return x, z


def logistic_eval(prob, W, V=None, idx=None, want=("F", "grad", "hvp")):
    """F [K], grad [K, n] and (with V) hvp [K, n] over the sample idx (all
    points when None), for the parameter vectors W [K, n]."""
    P, keep = prob
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    K = W.shape[0]
    V = None if V is None else np.ascontiguousarray(np.atleast_2d(V), dtype=np.float64)
    ix = None if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
    b = P.N if ix is None else ix.size
    F = np.empty(K) if "F" in want else None
    g = np.empty((K, P.n)) if "grad" in want else None
    h = np.empty((K, P.n)) if ("hvp" in want and V is not None) else None
    _check(lib().oracle_logistic_eval(C.byref(P), _p(ix, C.c_int64), b, K, _p(W), _p(V), _p(F), _p(g), _p(h)),
           "logistic_eval")
    out = {}
    if F is not None:
        out["F"] = F
    if g is not None:
        out["grad"] = g
    if h is not None:
        out["hvp"] = h
    return out


def rse(y_t, y_star):
    """Relative squared error in percent (Table 2 notes)."""
    return float(lib().oracle_rse(float(y_t), float(y_star)))


def cholesky(S):
    """Lower Cholesky factor of the symmetric positive definite S (lower
    triangle read); raises ValueError when a pivot is not positive."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    d = S.shape[0]
    out = np.empty_like(S)
    _check(lib().oracle_cholesky(d, _p(S), _p(out)), "cholesky")
    return out


def make_newsvendor(mu, sigma, k, h, v, S, seed=0, instance=0, epoch=0):
    """Returns (Newsvendor, keepalive) for n products with S demand samples each."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (mu, sigma, k, h, v)]
    n = arrs[0].shape[0]
    P = Newsvendor(n, S, seed, instance, epoch, *[_p(a) for a in arrs])
    return P, arrs


def newsvendor_demands(prob, j):
    """Standardised demand samples z_j0 .. z_j(S-1) of product j (float32)."""
    P, keep = prob
    z = np.empty(P.S, np.float32)
    _check(lib().oracle_newsvendor_demands(C.byref(P), j, _p(z, C.c_float)), "newsvendor_demands")
    return z


def newsvendor_grad(prob, X, products=None):
    """Monte Carlo gradient estimates [K, m] at decisions X [K, n], and the
    counts, for all products or for the range products = (j0, j1)."""
    P, keep = prob
    X = np.ascontiguousarray(np.atleast_2d(X), dtype=np.float64)
    K = X.shape[0]
    j0, j1 = (0, P.n) if products is None else products
    g = np.empty((K, j1 - j0))
    cnt = np.empty((K, j1 - j0), np.int64)
    _check(lib().oracle_newsvendor_grad_range(C.byref(P), K, _p(X), j0, j1, _p(g), _p(cnt, C.c_int64)),
           "newsvendor_grad")
    return g, cnt
