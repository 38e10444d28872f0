"""Thin ctypes binding of the C ABI declared in include/ttgb.h.

Argument marshalling only: every step of TT sums, dots, rounding and the
orthogonalization schemes runs in the CUDA library (libttgb.so).  There is no
CPU fallback: if the library is missing or no sm_103 GPU is present, the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

TT_OK = 0
STATUS = {0: "TT_OK", 1: "TT_ERR_ARG", 2: "TT_ERR_SHAPE", 3: "TT_ERR_OOM", 4: "TT_ERR_NOT_SPD",
          5: "TT_ERR_BREAKDOWN", 6: "TT_ERR_NONFINITE", 7: "TT_ERR_TIMEOUT", 8: "TT_ERR_CUDA",
          9: "TT_ERR_CANCELLED"}
PRECISION = {"fp64": 0, "mixed_tf32": 1, "fp32": 2}
SCHEME = {"cgs": 0, "mgs": 1, "cgs2": 2, "mgs2": 3, "gram": 4, "householder": 5}
POLICY = {"paper": 0, "every_update": 1}
SIGN = {"stable": 0, "literal": 1}
DTYPE_F64, DTYPE_F32 = 0, 1


class TTError(RuntimeError):
    def __init__(self, status, where, msg=""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__("%s: %s %s" % (where, self.name, msg))


class _Stats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("kernel_launches", "roundings", "host_syncs", "bytes_in_use",
                                           "peak_bytes", "svd_calls", "certified_bonds", "fallback_orth", "svd_sweeps",
                                           "series_passes", "series_retries",
                                           "second_pass_skips", "fallback_fp32")]


class _Prof(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_uint64), ("total_ms", C.c_double),
                ("flops", C.c_double), ("bytes", C.c_double)]


_lib = None
_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_PI = C.POINTER(C.c_int)
_PD = C.POINTER(C.c_double)
_PP = C.POINTER(C.c_void_p)

_SIGS = {
    "tt_ctx_create": (_I, [C.POINTER(_P), _I, _I, _P, C.c_size_t]),
    "tt_ctx_destroy": (None, [_P]),
    "tt_ctx_get_stats": (_I, [_P, C.POINTER(_Stats)]),
    "tt_ctx_reset_stats": (None, [_P]),
    "tt_ctx_precision": (_I, [_P]),
    "tt_ctx_set_profiling": (_I, [_P, _I]),
    "tt_ctx_set_profiling_family": (_I, [_P, C.c_char_p]),
    "tt_ctx_set_tc_wait_limit": (_I, [_P, C.c_longlong]),
    "tt_ctx_set_pipeline": (_I, [_P, _I]),
    "tt_ctx_get_profile": (_I, [_P, C.POINTER(_Prof), _I, _PI]),
    "tt_ctx_reset_profile": (None, [_P]),
    "tt_tensor_create": (_I, [_P, _I, _PI, _PI, C.POINTER(_PD), C.POINTER(_P)]),
    "tt_tensor_wrap_device": (_I, [_P, _I, _PI, _PI, _PP, _I, C.POINTER(_P)]),
    "tt_tensor_shape": (_I, [_P, _PI, _PI, _PI]),
    "tt_tensor_core_ptr": (_I, [_P, _I, _PP]),
    "tt_tensor_download": (_I, [_P, _P, C.POINTER(_PD)]),
    "tt_tensor_create_storage": (_I, [_P, _I, _PI, _PI, C.POINTER(_P), C.POINTER(_P)]),
    "tt_tensor_download_storage": (_I, [_P, _P, C.POINTER(_P)]),
    "tt_tensor_free": (None, [_P]),
    "tt_add": (_I, [_P, _I, _PD, _PP, C.POINTER(_P)]),
    "tt_scale": (_I, [_P, _P, _D, C.POINTER(_P)]),
    "tt_dot": (_I, [_P, _P, _P, _PD]),
    "tt_dot_many": (_I, [_P, _P, _I, _PP, _PD]),
    "tt_norm": (_I, [_P, _P, _PD]),
    "tt_round": (_I, [_P, _P, _D, C.POINTER(_P), _PD]),
    "tt_round_to_host": (_I, [_P, _P, _D, C.POINTER(_P), _PD, C.POINTER(_P)]),
    "tt_round_capped": (_I, [_P, _P, _D, _I, C.POINTER(_P), _PD]),
    "tt_operator_create": (_I, [_P, _I, _PI, _PI, _PI, C.POINTER(_PD), C.POINTER(_P)]),
    "tt_operator_laplacian": (_I, [_P, _I, _I, C.POINTER(_P)]),
    "tt_operator_shape": (_I, [_P, _PI, _PI, _PI, _PI]),
    "tt_operator_download": (_I, [_P, _P, C.POINTER(_PD)]),
    "tt_operator_free": (None, [_P]),
    "tt_matvec": (_I, [_P, _P, _P, C.POINTER(_P)]),
    "tt_krylov_basis": (_I, [_P, _P, _P, _I, _D, _I, _PP]),
    "tt_round_gram_svd": (_I, [_P, _P, _D, _I, C.POINTER(_P), _PD]),
    "tt_round_randomized": (_I, [_P, _P, _P, _D, C.POINTER(_P)]),
    "tt_canonical": (_I, [_P, _I, _PI, C.c_long, C.POINTER(_P)]),
    "tt_householder_vectors": (_I, [_P, _D, _I, _I, _PP, _PP, _PD, _PI]),
    "tt_householder_apply": (_I, [_P, _I, _PP, _P, _I, _D, C.POINTER(_P)]),
    "tt_round_batched": (_I, [_P, _I, _PP, _PD, _PP]),
    "tt_ctx_set_concurrency": (_I, [_P, _I]),
    "tt_ctx_get_concurrency": (_I, [_P]),
    "tt_orthogonalize": (_I, [_P, _I, _D, _I, _I, _PP, _PP, _PD, _PI]),
    "tt_set_sign_rule": (_I, [_P, _I]),
    "tt_gram_f32": (_I, [_P, _I, C.c_long, _P, C.c_long, _P, _I]),
    "tt_cholesky_inverse": (_I, [_P, _I, _P, _P, _P, _D, _D, _PI]),
    "tt_gemm_f32": (_I, [_P, _I, _I, _I, _I, _P, C.c_long, _P, C.c_long, _P, C.c_long, _I]),
    "tt_dot_f64_noalloc": (_I, [_P, _I, _PI, _PI, _PI, _PP, _PP, _P]),
    "tt_server_create": (_I, [_P, _I, C.c_size_t, C.POINTER(_P)]),
    "tt_server_add_basis": (_I, [_P, _I, _PP, _PI]),
    "tt_server_submit": (_I, [_P, _I, _P, _D, _I, _I, _I, C.POINTER(C.c_uint64)]),
    "tt_server_wait": (_I, [_P, C.c_uint64, _I, C.POINTER(_P), _PD, _I, _PD]),
    "tt_server_cancel": (_I, [_P, C.c_uint64]),
    "tt_server_get_stats": (_I, [_P, C.c_void_p]),
    "tt_server_destroy": (None, [_P]),
    "tt_status_str": (C.c_char_p, [_I]),
    "tt_last_error": (C.c_char_p, []),
}


def lib_path():
    return _build.LIB


def lib():
    """Loads libttgb.so (built in-tree by ``build.build()``); raises if absent."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("libttgb.so is not built (%s); call paper_2211_08770_gb300.build.build()" % path)
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st, where):
    if st != TT_OK:
        msg = lib().tt_last_error()
        raise TTError(st, where, msg.decode() if msg else "")


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover - torch is optional plumbing
        pass
    return 0


class Ctx:
    """A tt_ctx: device, arithmetic (fp64 / mixed_tf32 / fp32), CUDA stream
    (an integer cudaStream_t; default: torch's current stream) and HBM budget
    in bytes (0 = none)."""

    def __init__(self, device=0, precision="fp64", stream=None, hbm_budget=0):
        self._h = _P()
        self.precision = precision
        self.stream = _default_stream() if stream is None else int(stream)
        _check(lib().tt_ctx_create(C.byref(self._h), device, PRECISION[precision], _P(self.stream or None),
                                   hbm_budget), "tt_ctx_create")

    @property
    def handle(self):
        return self._h

    def stats(self):
        s = _Stats()
        _check(lib().tt_ctx_get_stats(self._h, C.byref(s)), "tt_ctx_get_stats")
        return {k: int(getattr(s, k)) for k, _ in _Stats._fields_}

    def reset_stats(self):
        lib().tt_ctx_reset_stats(self._h)

    def set_profiling(self, on=True, family=None):
        """Event timing of the library's launches; family: time only that
        kernel family (None: all)."""
        _check(lib().tt_ctx_set_profiling(self._h, 1 if on else 0), "tt_ctx_set_profiling")
        _check(lib().tt_ctx_set_profiling_family(self._h, family.encode() if family else None),
               "tt_ctx_set_profiling_family")

    def reset_profile(self):
        lib().tt_ctx_reset_profile(self._h)

    def profile(self):
        """{family: dict(launches, total_ms, flops, bytes)} since the last reset."""
        buf = (_Prof * 64)()
        k = C.c_int()
        _check(lib().tt_ctx_get_profile(self._h, buf, 64, C.byref(k)), "tt_ctx_get_profile")
        return {buf[i].name.decode(): dict(launches=int(buf[i].launches), total_ms=buf[i].total_ms,
                                           flops=buf[i].flops, bytes=buf[i].bytes) for i in range(min(64, k.value))}

    def set_tc_wait_limit(self, cycles):
        """SM-cycle limit of the tensor-core row Gram's bounded waits (0: the
        default, about 2 s)."""
        _check(lib().tt_ctx_set_tc_wait_limit(self._h, int(cycles)), "tt_ctx_set_tc_wait_limit")

    def set_pipeline(self, on=True):
        """Pipelined (speculative two-stream) sweeps of TT-round on this
        context (on by default); off: every sweep on the context's stream."""
        _check(lib().tt_ctx_set_pipeline(self._h, 1 if on else 0), "tt_ctx_set_pipeline")

    def set_sign_rule(self, rule):
        _check(lib().tt_set_sign_rule(self._h, SIGN[rule]), "tt_set_sign_rule")

    @property
    def concurrency(self):
        """Lanes used by tt_round_batched."""
        return int(lib().tt_ctx_get_concurrency(self._h))

    @concurrency.setter
    def concurrency(self, lanes):
        _check(lib().tt_ctx_set_concurrency(self._h, int(lanes)), "tt_ctx_set_concurrency")

    def close(self):
        if self._h:
            lib().tt_ctx_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TT:
    """Handle of a device TT tensor (tt_tensor*) owned by the library."""

    def __init__(self, ctx, handle, keepalive=None):
        self.ctx = ctx
        self._h = handle
        self._keep = keepalive

    @property
    def handle(self):
        return self._h

    def shape(self):
        d = C.c_int()
        _check(lib().tt_tensor_shape(self._h, C.byref(d), None, None), "tt_tensor_shape")
        n = (C.c_int * d.value)()
        r = (C.c_int * (d.value + 1))()
        _check(lib().tt_tensor_shape(self._h, None, n, r), "tt_tensor_shape")
        return d.value, list(n), list(r)

    @property
    def ranks(self):
        return self.shape()[2]

    def core_ptr(self, k):
        p = _P()
        _check(lib().tt_tensor_core_ptr(self._h, k, C.byref(p)), "tt_tensor_core_ptr")
        return p.value

    def cores(self):
        """Downloads the cores as float64 numpy arrays (r_{k-1}, n_k, r_k)."""
        d, n, r = self.shape()
        out = [np.empty((r[k], n[k], r[k + 1]), dtype=np.float64) for k in range(d)]
        ptrs = (_PD * d)(*[o.ctypes.data_as(_PD) for o in out])
        _check(lib().tt_tensor_download(self.ctx.handle, self._h, ptrs), "tt_tensor_download")
        return out

    def download_storage(self, out):
        """Copies the cores into the given host arrays (numpy, the context's
        storage dtype, at least r_{k-1} n_k r_k elements each; page-locked
        memory gives full-bandwidth copies) without conversion; returns views
        of the right shapes."""
        d, n, r = self.shape()
        views = []
        for k in range(d):
            v = out[k].reshape(-1)[: r[k] * n[k] * r[k + 1]]
            if not v.flags["C_CONTIGUOUS"]:
                raise ValueError("host buffer %d is not contiguous" % k)
            views.append(v.reshape(r[k], n[k], r[k + 1]))
        ptrs = (_P * d)(*[v.ctypes.data for v in views])
        _check(lib().tt_tensor_download_storage(self.ctx.handle, self._h, ptrs), "tt_tensor_download_storage")
        return views

    def free(self):
        if self._h:
            lib().tt_tensor_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _handles(xs):
    return (_P * len(xs))(*[x.handle for x in xs])


def tt_tensor_create(ctx, cores):
    cores = [np.ascontiguousarray(c, dtype=np.float64) for c in cores]
    d = len(cores)
    n = (C.c_int * d)(*[c.shape[1] for c in cores])
    r = (C.c_int * (d + 1))(*([c.shape[0] for c in cores] + [cores[-1].shape[2]]))
    ptrs = (_PD * d)(*[c.ctypes.data_as(_PD) for c in cores])
    h = _P()
    _check(lib().tt_tensor_create(ctx.handle, d, n, r, ptrs, C.byref(h)), "tt_tensor_create")
    return TT(ctx, h)


def tt_tensor_create_storage(ctx, cores):
    """tt_tensor_create from host arrays already in the context's storage
    dtype (float32 for mixed_tf32 / fp32, float64 for fp64), copied without
    conversion.  From page-locked memory the copies are asynchronous: keep
    the arrays unchanged until a later synchronizing call returns."""
    want = np.float64 if ctx.precision == "fp64" else np.float32
    for c in cores:
        if c.dtype != want or not c.flags["C_CONTIGUOUS"]:
            raise ValueError("cores must be C-contiguous %s arrays" % np.dtype(want).name)
    d = len(cores)
    n = (C.c_int * d)(*[c.shape[1] for c in cores])
    r = (C.c_int * (d + 1))(*([c.shape[0] for c in cores] + [cores[-1].shape[2]]))
    ptrs = (_P * d)(*[c.ctypes.data for c in cores])
    h = _P()
    _check(lib().tt_tensor_create_storage(ctx.handle, d, n, r, ptrs, C.byref(h)), "tt_tensor_create_storage")
    return TT(ctx, h)


def tt_tensor_wrap_device(ctx, n, r, dev_ptrs, dtype, keepalive=None):
    d = len(n)
    nn = (C.c_int * d)(*n)
    rr = (C.c_int * (d + 1))(*r)
    pp = (_P * d)(*dev_ptrs)
    h = _P()
    _check(lib().tt_tensor_wrap_device(ctx.handle, d, nn, rr, pp, dtype, C.byref(h)), "tt_tensor_wrap_device")
    return TT(ctx, h, keepalive)


def tt_add(ctx, alphas, xs):
    al = (C.c_double * len(xs))(*[float(a) for a in alphas])
    h = _P()
    _check(lib().tt_add(ctx.handle, len(xs), al, _handles(xs), C.byref(h)), "tt_add")
    return TT(ctx, h)


def tt_scale(ctx, x, alpha):
    h = _P()
    _check(lib().tt_scale(ctx.handle, x.handle, float(alpha), C.byref(h)), "tt_scale")
    return TT(ctx, h)


def tt_dot(ctx, x, y):
    v = C.c_double()
    _check(lib().tt_dot(ctx.handle, x.handle, y.handle, C.byref(v)), "tt_dot")
    return v.value


def tt_dot_many(ctx, x, ys):
    out = (C.c_double * max(1, len(ys)))()
    _check(lib().tt_dot_many(ctx.handle, x.handle, len(ys), _handles(ys), out), "tt_dot_many")
    return np.array(out[: len(ys)])


def tt_norm(ctx, x):
    v = C.c_double()
    _check(lib().tt_norm(ctx.handle, x.handle, C.byref(v)), "tt_norm")
    return v.value


def tt_round(ctx, x, delta):
    h = _P()
    e = C.c_double()
    _check(lib().tt_round(ctx.handle, x.handle, float(delta), C.byref(h), C.byref(e)), "tt_round")
    return TT(ctx, h), e.value


def tt_round_capped(ctx, x, delta, max_rank):
    h = _P()
    e = C.c_double()
    _check(lib().tt_round_capped(ctx.handle, x.handle, float(delta), int(max_rank), C.byref(h), C.byref(e)),
           "tt_round_capped")
    return TT(ctx, h), e.value


class Operator:
    """Handle of a device TT-matrix (tt_operator*) owned by the library."""

    def __init__(self, ctx, handle):
        self.ctx = ctx
        self._h = handle

    @property
    def handle(self):
        return self._h

    def shape(self):
        d = C.c_int()
        _check(lib().tt_operator_shape(self._h, C.byref(d), None, None, None), "tt_operator_shape")
        m = (C.c_int * d.value)()
        n = (C.c_int * d.value)()
        R = (C.c_int * (d.value + 1))()
        _check(lib().tt_operator_shape(self._h, None, m, n, R), "tt_operator_shape")
        return d.value, list(m), list(n), list(R)

    def cores(self):
        """Downloads the cores as float64 arrays (R_{k-1}, m_k, n_k, R_k)."""
        d, m, n, R = self.shape()
        out = [np.empty((R[k], m[k], n[k], R[k + 1])) for k in range(d)]
        ptrs = (_PD * d)(*[o.ctypes.data_as(_PD) for o in out])
        _check(lib().tt_operator_download(self.ctx.handle, self._h, ptrs), "tt_operator_download")
        return out

    def free(self):
        if self._h:
            lib().tt_operator_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def tt_operator_create(ctx, cores):
    cores = [np.ascontiguousarray(c, dtype=np.float64) for c in cores]
    d = len(cores)
    m = (C.c_int * d)(*[c.shape[1] for c in cores])
    n = (C.c_int * d)(*[c.shape[2] for c in cores])
    R = (C.c_int * (d + 1))(*([c.shape[0] for c in cores] + [cores[-1].shape[3]]))
    ptrs = (_PD * d)(*[c.ctypes.data_as(_PD) for c in cores])
    h = _P()
    _check(lib().tt_operator_create(ctx.handle, d, m, n, R, ptrs, C.byref(h)), "tt_operator_create")
    return Operator(ctx, h)


def tt_operator_laplacian(ctx, d, n):
    h = _P()
    _check(lib().tt_operator_laplacian(ctx.handle, int(d), int(n), C.byref(h)), "tt_operator_laplacian")
    return Operator(ctx, h)


def tt_matvec(ctx, op, x):
    h = _P()
    _check(lib().tt_matvec(ctx.handle, op.handle, x.handle, C.byref(h)), "tt_matvec")
    return TT(ctx, h)


def tt_krylov_basis(ctx, op, x1, m, delta=0.0, max_rank=1):
    out = (_P * m)()
    _check(lib().tt_krylov_basis(ctx.handle, op.handle, x1.handle, int(m), float(delta), int(max_rank), out),
           "tt_krylov_basis")
    return [TT(ctx, _P(out[j])) for j in range(m)]


def tt_round_gram_svd(ctx, x, delta, max_rank=0):
    h = _P()
    e = C.c_double()
    _check(lib().tt_round_gram_svd(ctx.handle, x.handle, float(delta), int(max_rank), C.byref(h), C.byref(e)),
           "tt_round_gram_svd")
    return TT(ctx, h), e.value


def tt_round_randomized(ctx, x, omega, delta=0.0):
    h = _P()
    _check(lib().tt_round_randomized(ctx.handle, x.handle, omega.handle, float(delta), C.byref(h)),
           "tt_round_randomized")
    return TT(ctx, h)


def tt_canonical(ctx, n, j):
    """e_j (0-based j, i_1 fastest) as a rank-1 TT."""
    d = len(n)
    nn = (C.c_int * d)(*n)
    h = _P()
    _check(lib().tt_canonical(ctx.handle, d, nn, int(j), C.byref(h)), "tt_canonical")
    return TT(ctx, h)


def tt_householder_vectors(ctx, A, delta, policy="paper"):
    m = len(A)
    U = (_P * m)()
    R = (C.c_double * (m * m))()
    nr = C.c_int()
    _check(lib().tt_householder_vectors(ctx.handle, float(delta), POLICY[policy], m, _handles(A), U, R,
                                        C.byref(nr)), "tt_householder_vectors")
    Rm = np.array(R[:]).reshape(m, m).T.copy()
    return [TT(ctx, _P(U[i])) for i in range(m)], Rm, nr.value


def tt_householder_apply(ctx, U, x, transpose=False, delta=-1.0):
    h = _P()
    _check(lib().tt_householder_apply(ctx.handle, len(U), _handles(U) if U else None, x.handle,
                                      1 if transpose else 0, float(delta), C.byref(h)), "tt_householder_apply")
    return TT(ctx, h)


def tt_round_to_host(ctx, x, delta, out):
    """tt_round that also copies the rounded cores into the host arrays
    `out` (numpy, the context's storage dtype, each at least as large as x's
    core; page-locked memory lets the copies overlap the sweep).  Returns
    (TT, err_est, views of out with the rounded shapes)."""
    want = np.float64 if ctx.precision == "fp64" else np.float32
    d, n, r = x.shape()
    for k in range(d):
        if out[k].dtype != want or not out[k].flags["C_CONTIGUOUS"] or out[k].size < r[k] * n[k] * r[k + 1]:
            raise ValueError("host buffer %d: C-contiguous %s with at least %d elements" %
                             (k, np.dtype(want).name, r[k] * n[k] * r[k + 1]))
    ptrs = (_P * d)(*[o.ctypes.data for o in out])
    h = _P()
    e = C.c_double()
    _check(lib().tt_round_to_host(ctx.handle, x.handle, float(delta), C.byref(h), C.byref(e), ptrs),
           "tt_round_to_host")
    y = TT(ctx, h)
    _, _, ry = y.shape()
    views = [out[k].reshape(-1)[: ry[k] * n[k] * ry[k + 1]].reshape(ry[k], n[k], ry[k + 1]) for k in range(d)]
    return y, e.value, views


def tt_round_batched(ctx, xs, deltas):
    k = len(xs)
    dl = (C.c_double * k)(*[float(v) for v in deltas])
    out = (_P * k)()
    _check(lib().tt_round_batched(ctx.handle, k, _handles(xs), dl, out), "tt_round_batched")
    return [TT(ctx, _P(out[i])) for i in range(k)]


def tt_orthogonalize(ctx, scheme, A, delta, policy="paper"):
    m = len(A)
    Q = (_P * m)()
    R = (C.c_double * (m * m))()
    nr = C.c_int()
    _check(lib().tt_orthogonalize(ctx.handle, SCHEME[scheme], float(delta), POLICY[policy], m, _handles(A), Q, R,
                                  C.byref(nr)), "tt_orthogonalize")
    Rm = np.array(R[:]).reshape(m, m).T.copy()  # column-major -> R[j, i]
    return [TT(ctx, _P(Q[i])) for i in range(m)], Rm, nr.value


def tt_gram_f32(ctx, n, K, x_ptr, ldx, g_ptr, use_tensor_cores=1):
    """G = X X^T for device FP32 pointers (see include/ttgb.h); mode 0
    CUDA cores, 1 tensor cores, 2 the column Gram X^T X on tensor cores."""
    mode = int(use_tensor_cores)
    if mode not in (0, 1, 2):
        raise ValueError("use_tensor_cores must be 0, 1 or 2")
    _check(lib().tt_gram_f32(ctx.handle, n, K, _P(x_ptr), ldx, _P(g_ptr), mode), "tt_gram_f32")


def tt_dot_f64_noalloc(stream, n, rx, ry, x_ptrs, y_ptrs, result_ptr):
    """<x, y> of FP64 device cores into the device double at result_ptr,
    allocating nothing (see include/ttgb.h); asynchronous on `stream`."""
    d = len(n)
    nn = (C.c_int * d)(*n)
    a = (C.c_int * (d + 1))(*rx)
    b = (C.c_int * (d + 1))(*ry)
    xs = (_P * d)(*x_ptrs)
    ys = (_P * d)(*y_ptrs)
    _check(lib().tt_dot_f64_noalloc(_P(stream or None), d, nn, a, b, xs, ys, _P(result_ptr)), "tt_dot_f64_noalloc")


def tt_gemm_f32(ctx, trans_b, M, N, K, a_ptr, lda, b_ptr, ldb, c_ptr, ldc, use_tensor_cores=True):
    """C = A op(B) on device FP32 pointers (see include/ttgb.h)."""
    mode = int(use_tensor_cores) if not isinstance(use_tensor_cores, bool) else (1 if use_tensor_cores else 0)
    _check(lib().tt_gemm_f32(ctx.handle, 1 if trans_b else 0, M, N, K, _P(a_ptr), lda, _P(b_ptr), ldb, _P(c_ptr),
                             ldc, mode), "tt_gemm_f32")


def tt_cholesky_inverse(ctx, n, g_ptr, l_ptr, t_ptr, shift_rel=0.0, drop_rel=0.0):
    """G + s I = L L^T, T = L^{-1} on device pointers (see include/ttgb.h);
    returns the number of dropped pivots."""
    nd = C.c_int()
    _check(lib().tt_cholesky_inverse(ctx.handle, n, _P(g_ptr), _P(l_ptr), _P(t_ptr), float(shift_rel),
                                     float(drop_rel), C.byref(nd)), "tt_cholesky_inverse")
    return nd.value


def loss_of_orthogonality(ctx, Q):
    """||I - Q^T Q||_2 with (Q^T Q)(i,j) = <q_i, q_j> from GPU TT dots
    (Section 3.4, eq. LOO); the m x m spectral norm is a host metric."""
    m = len(Q)
    G = np.zeros((m, m))
    for i in range(m):
        v = tt_dot_many(ctx, Q[i], Q[: i + 1])
        G[i, : i + 1] = v
        G[: i + 1, i] = v
    return float(np.max(np.abs(np.linalg.eigvalsh(np.eye(m) - G))))


class _ServerStats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in (
        "submitted", "completed", "failed", "cancelled", "refused", "queued", "running",
        "footprint_in_use", "footprint_peak", "footprint_budget", "roundings", "kernel_launches", "host_syncs")]


class Server:
    """A tt_server over ctx: requests run concurrently on `workers` lanes,
    admitted by device footprint (bytes, 0 = the context's budget)."""

    def __init__(self, ctx, workers=8, footprint_budget=0):
        self.ctx = ctx
        self._h = _P()
        _check(lib().tt_server_create(ctx.handle, int(workers), int(footprint_budget), C.byref(self._h)),
               "tt_server_create")
        self._basis_k = {}
        self._inputs = {}  # ticket -> input TT, kept alive until its wait returns

    def add_basis(self, tensors):
        """Copies orthonormal TT tensors (TT objects) into a resident basis; returns its id."""
        bid = C.c_int()
        _check(lib().tt_server_add_basis(self._h, len(tensors), _handles(tensors), C.byref(bid)),
               "tt_server_add_basis")
        self._basis_k[bid.value] = len(tensors)
        return bid.value

    def submit_round(self, x, delta):
        t = C.c_uint64()
        _check(lib().tt_server_submit(self._h, 0, x.handle, float(delta), -1, 0, 0, C.byref(t)), "tt_server_submit")
        self._inputs[t.value] = x
        return t.value

    def submit_orth(self, x, basis_id, k, scheme, delta):
        t = C.c_uint64()
        _check(lib().tt_server_submit(self._h, 1, x.handle, float(delta), int(basis_id), int(k), SCHEME[scheme],
                                      C.byref(t)), "tt_server_submit")
        self._inputs[t.value] = x
        return t.value

    def wait(self, ticket, timeout_ms=-1, coef_cap=0):
        """(TT result, coefficients (list), (t_submit, t_start, t_done))."""
        h = _P()
        cf = (C.c_double * max(coef_cap, 1))()
        tm = (C.c_double * 3)()
        st = lib().tt_server_wait(self._h, C.c_uint64(ticket), int(timeout_ms), C.byref(h), cf, int(coef_cap), tm)
        if st != TT_OK and STATUS.get(st) == "TT_ERR_TIMEOUT":
            _check(st, "tt_server_wait")  # the request is still pending: keep its input
        self._inputs.pop(ticket, None)
        _check(st, "tt_server_wait")
        return TT(self.ctx, h), [cf[i] for i in range(coef_cap)], (tm[0], tm[1], tm[2])

    def cancel(self, ticket):
        _check(lib().tt_server_cancel(self._h, C.c_uint64(ticket)), "tt_server_cancel")

    def stats(self):
        s = _ServerStats()
        _check(lib().tt_server_get_stats(self._h, C.byref(s)), "tt_server_get_stats")
        return {k: int(getattr(s, k)) for k, _ in _ServerStats._fields_}

    def close(self):
        if self._h:
            lib().tt_server_destroy(self._h)
            self._h = _P()
        self._inputs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
