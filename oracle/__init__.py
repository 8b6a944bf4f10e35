"""CPU oracle -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.

ctypes marshalling around ``hc_oracle.c``: a plain serial C reference of the
HSZp-style compressor, the multi-stage decompressor (Algorithm 2) and the
homomorphic operations of Section V of the paper.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference arm of
``bench.py`` may import this package.  It shares nothing with the CUDA
library and never calls it.

Status codes: 0 ok, 1 invalid argument, 2 range (|q| >= 2^30 or a non-finite
input), 3 corrupt stream, 4 unsupported.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

KIND_DERIV, KIND_GRADMAG, KIND_LAPLACIAN = 0, 1, 2
# predictors: delta inside the block (HSZp with block heads), block mean
# (HSZx), Lorenzo over the field's axes (HSZp-nd), delta across blocks over
# the flattened field (HSZp), block mean over multidimensional boxes (HSZx-nd)
PRED_DELTA, PRED_MEAN, PRED_LORENZO, PRED_GLOBAL, PRED_MEAN_ND = 0, 1, 2, 3, 4


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile hc_oracle.c with gcc into oracle/liboracle.so (no -march flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        # HC_ORACLE_LIB: a build of a modified copy of hc_oracle.c, loaded in
        # place of oracle/liboracle.so (the planted-mistake runs of
        # tests/test_oracle_mutants.py)
        L = ctypes.CDLL(os.environ.get("HC_ORACLE_LIB") or build())
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        P = ctypes.POINTER
        L.orc_eps.argtypes = [vp, i32, i64, dbl, i32, P(dbl)]
        L.orc_quantize.argtypes = [vp, i32, i64, dbl, vp]
        L.orc_compress_bound.argtypes = [i64, i32]
        L.orc_compress_bound.restype = i64
        L.orc_compress.argtypes = [vp, i32, i32, vp, dbl, i32, i32, vp, i64, P(i64), P(dbl)]
        L.orc_compress_codes.argtypes = [vp, i32, i32, vp, dbl, dbl, i32, i32, vp, i64, P(i64)]
        L.orc_compress_pred.argtypes = [vp, i32, i32, vp, dbl, i32, i32, i32, vp, i64, P(i64), P(dbl)]
        L.orc_compress_codes_pred.argtypes = [vp, i32, i32, vp, dbl, dbl, i32, i32, i32, vp, i64, P(i64)]
        L.orc_mean_m_sum.argtypes = [vp, i64, i32, i64, P(i64)]
        L.orc_mean_p_sum_x.argtypes = [vp, vp, i64, i32, P(i64)]
        L.orc_std_p_x.argtypes = [vp, vp, i64, i32, dbl, P(i64), P(ctypes.c_uint64), P(ctypes.c_uint64), P(dbl)]
        L.orc_divergence_q.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.orc_curl2_q.argtypes = [vp, vp, vp, i32, i32, dbl, dbl, vp, vp]
        L.orc_read_header.argtypes = [vp, i64, vp, vp]
        for name in ("orc_decode_p", "orc_decode_q", "orc_decode_m", "orc_decode_f"):
            getattr(L, name).argtypes = [vp, i64, vp]
        L.orc_dequantize.argtypes = [vp, i64, dbl, i32, vp]
        L.orc_sums_q.argtypes = [vp, i64, P(i64), P(ctypes.c_uint64), P(ctypes.c_uint64)]
        L.orc_mean_p_sum.argtypes = [vp, i64, i32, P(i64)]
        L.orc_var_p_sums.argtypes = [vp, i64, i32, P(i64), P(ctypes.c_uint64), P(ctypes.c_uint64)]
        L.orc_finalize.argtypes = [i64, i64, ctypes.c_uint64, ctypes.c_uint64, dbl, P(dbl), P(dbl), P(dbl)]
        L.orc_stats_f.argtypes = [vp, i32, i64, P(dbl), P(dbl)]
        L.orc_deriv_q.argtypes = [vp, vp, i32, vp]
        L.orc_lap_q.argtypes = [vp, vp, vp]
        L.orc_stencil_q.argtypes = [vp, vp, i32, i32, dbl, vp]
        L.orc_stencil_f.argtypes = [vp, i32, vp, i32, i32, vp]
        L.orc_stencil_at.argtypes = [vp, vp, i32, i32, dbl, vp, i64, vp, vp]
        L.orc_lorenzo_mean_p.argtypes = [vp, vp, P(i64)]
        L.orc_compress_bound_nd.argtypes = [i32, vp, vp]
        L.orc_compress_bound_nd.restype = i64
        L.orc_compress_codes_nd.argtypes = [vp, i32, i32, vp, vp, dbl, dbl, i32, vp, i64, P(i64)]
        L.orc_compress_nd.argtypes = [vp, i32, i32, vp, vp, dbl, i32, vp, i64, P(i64), P(dbl)]
        L.orc_xnd_mean_m.argtypes = [vp, vp, vp, P(i64)]
        L.orc_xnd_mean_p.argtypes = [vp, vp, vp, vp, P(i64)]
        L.orc_xnd_std_p.argtypes = [vp, vp, vp, vp, dbl, P(i64), P(ctypes.c_uint64), P(ctypes.c_uint64), P(dbl)]
        L.orc_xnd_deriv_p.argtypes = [vp, vp, vp, vp, i32, vp]
        L.orc_xnd_lap_p.argtypes = [vp, vp, vp, vp, vp]
        L.orc_lorenzo_var_p.argtypes = [vp, vp, P(i64), P(ctypes.c_uint64), P(ctypes.c_uint64)]
        L.orc_lorenzo_deriv_p.argtypes = [vp, vp, i32, vp]
        L.orc_lorenzo_lap_p.argtypes = [vp, vp, vp]
        for f in (L.orc_eps, L.orc_quantize, L.orc_compress, L.orc_compress_codes, L.orc_read_header,
                  L.orc_decode_p, L.orc_decode_q, L.orc_decode_m, L.orc_decode_f, L.orc_dequantize,
                  L.orc_sums_q, L.orc_mean_p_sum, L.orc_var_p_sums, L.orc_finalize, L.orc_stats_f,
                  L.orc_deriv_q, L.orc_lap_q, L.orc_stencil_q, L.orc_stencil_f, L.orc_stencil_at,
                  L.orc_compress_pred, L.orc_compress_codes_pred, L.orc_mean_m_sum, L.orc_mean_p_sum_x,
                  L.orc_std_p_x, L.orc_divergence_q, L.orc_curl2_q, L.orc_lorenzo_mean_p, L.orc_lorenzo_var_p,
                  L.orc_lorenzo_deriv_p, L.orc_lorenzo_lap_p, L.orc_compress_codes_nd, L.orc_compress_nd,
                  L.orc_xnd_mean_m, L.orc_xnd_mean_p, L.orc_xnd_std_p, L.orc_xnd_deriv_p, L.orc_xnd_lap_p):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(st: int, what: str):
    if st != 0:
        raise OracleError(st, what)


def _dtype_code(x: np.ndarray) -> int:
    if x.dtype == np.float32:
        return 0
    if x.dtype == np.float64:
        return 1
    raise TypeError("fields are float32 or float64")


def dims3(shape) -> np.ndarray:
    """Shape padded with leading ones to (n0, n1, n2)."""
    shape = tuple(int(s) for s in shape)
    return np.array((1,) * (3 - len(shape)) + shape, dtype=np.int64)


# ---------------------------------------------------------------- compression
def eps_for(x: np.ndarray, eb: float, rel: bool) -> float:
    x = np.ascontiguousarray(x)
    out = ctypes.c_double()
    _check(lib().orc_eps(_ptr(x), _dtype_code(x), x.size, eb, int(rel), ctypes.byref(out)), "eps")
    return out.value


def quantize(x: np.ndarray, eps: float) -> np.ndarray:
    x = np.ascontiguousarray(x)
    q = np.empty(x.shape, np.int32)
    _check(lib().orc_quantize(_ptr(x), _dtype_code(x), x.size, eps, _ptr(q)), "quantize")
    return q


def compress_bound(n: int, S: int) -> int:
    return int(lib().orc_compress_bound(n, S))


def compress(x: np.ndarray, eb: float, rel: bool = True, S: int = 32, pred: int = 0):
    """Algorithm 1 on a float32/float64 array -> (stream bytes as uint8 array, eps).
    pred 0: delta inside each block (HSZp, block heads); 1: block means (HSZx);
    2: Lorenzo over the field's axes (HSZp-nd); 3: delta across blocks (HSZp)."""
    x = np.ascontiguousarray(x)
    d = np.array(x.shape, np.int64)
    cap = compress_bound(x.size, S)
    if cap < 0:
        raise OracleError(1, "compress_bound")
    out = np.zeros(cap, np.uint8)
    nbytes = ctypes.c_int64()
    eps = ctypes.c_double()
    _check(lib().orc_compress_pred(_ptr(x), _dtype_code(x), x.ndim, _ptr(d), eb, int(rel), S, pred, _ptr(out),
                                   cap, ctypes.byref(nbytes), ctypes.byref(eps)), "compress")
    return out[: nbytes.value].copy(), eps.value


def compress_codes(q: np.ndarray, eps: float, S: int = 32, dtype=np.float32, eb=None, rel=False, pred: int = 0):
    """Encode given integer codes (the steps of Algorithm 1 after quantization)."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    d = np.array(q.shape, np.int64)
    cap = compress_bound(q.size, S)
    out = np.zeros(cap, np.uint8)
    nbytes = ctypes.c_int64()
    code = 0 if np.dtype(dtype) == np.float32 else 1
    _check(lib().orc_compress_codes_pred(_ptr(q), code, q.ndim, _ptr(d), eps, eps if eb is None else eb,
                                         int(rel), S, pred, _ptr(out), cap, ctypes.byref(nbytes)),
           "compress_codes")
    return out[: nbytes.value].copy()


HEADER_KEYS = ("dtype", "ndim", "n0", "n1", "n2", "S", "G", "eb_mode", "qmax", "N", "nb", "nchunks",
               "payload_words", "total_bytes", "wmax", "off_payload", "pred", "b0", "b1", "b2")


def read_header(stream: np.ndarray) -> dict:
    s = np.ascontiguousarray(stream, dtype=np.uint8)
    ints = np.zeros(20, np.int64)
    dbls = np.zeros(2, np.float64)
    _check(lib().orc_read_header(_ptr(s), s.size, _ptr(ints), _ptr(dbls)), "read_header")
    h = {k: int(v) for k, v in zip(HEADER_KEYS, ints)}
    h["eps"], h["eb"] = float(dbls[0]), float(dbls[1])
    h["shape"] = (h["n0"], h["n1"], h["n2"])[3 - h["ndim"]:]
    h["block"] = (h["b0"], h["b1"], h["b2"])[3 - h["ndim"]:]
    return h


# ------------------------------------------------------------- decompression
def decode(stream: np.ndarray, stage: str) -> np.ndarray:
    """Algorithm 2: stage 'm' (heads), 'p' (D_p), 'q' (D_q) or 'f' (D_f)."""
    s = np.ascontiguousarray(stream, dtype=np.uint8)
    h = read_header(s)
    if stage == "m":
        out = np.empty(h["nb"], np.int32)
        _check(lib().orc_decode_m(_ptr(s), s.size, _ptr(out)), "decode_m")
        return out
    if stage in ("p", "q"):
        out = np.empty(h["shape"], np.int32)
        fn = lib().orc_decode_p if stage == "p" else lib().orc_decode_q
        _check(fn(_ptr(s), s.size, _ptr(out)), "decode_" + stage)
        return out
    if stage == "f":
        out = np.empty(h["shape"], np.float32 if h["dtype"] == 0 else np.float64)
        _check(lib().orc_decode_f(_ptr(s), s.size, _ptr(out)), "decode_f")
        return out
    raise ValueError(stage)


def dequantize(q: np.ndarray, eps: float, dtype=np.float32) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.int32)
    out = np.empty(q.shape, dtype)
    code = 0 if np.dtype(dtype) == np.float32 else 1
    _check(lib().orc_dequantize(_ptr(q), q.size, eps, code, _ptr(out)), "dequantize")
    return out


# --------------------------------------------------------------- statistics
def sums_q(q: np.ndarray):
    """Exact (sum q, sum q^2) as Python ints."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    s1, lo, hi = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().orc_sums_q(_ptr(q), q.size, ctypes.byref(s1), ctypes.byref(lo), ctypes.byref(hi)), "sums_q")
    return s1.value, (hi.value << 64) | lo.value


def mean_p_sum(dp: np.ndarray, S: int) -> int:
    """Stage-2 block-weighted sum of D_p (equals sum q)."""
    dp = np.ascontiguousarray(dp, dtype=np.int32)
    s1 = ctypes.c_int64()
    _check(lib().orc_mean_p_sum(_ptr(dp), dp.size, S, ctypes.byref(s1)), "mean_p_sum")
    return s1.value


def var_p_sums(dp: np.ndarray, S: int):
    """Stage-2 eta-accumulator sums (sum q, sum q^2) from D_p."""
    dp = np.ascontiguousarray(dp, dtype=np.int32)
    s1, lo, hi = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().orc_var_p_sums(_ptr(dp), dp.size, S, ctypes.byref(s1), ctypes.byref(lo),
                                ctypes.byref(hi)), "var_p_sums")
    return s1.value, (hi.value << 64) | lo.value


def mean_m_sum(M: np.ndarray, S: int, n: int) -> int:
    """Stage-1 sum of the HSZx block means weighted by the true block sizes (Eq. mean_m)."""
    M = np.ascontiguousarray(M, dtype=np.int32)
    t = ctypes.c_int64()
    _check(lib().orc_mean_m_sum(_ptr(M), M.size, S, n, ctypes.byref(t)), "mean_m_sum")
    return t.value


def mean_p_sum_x(dp: np.ndarray, M: np.ndarray, S: int) -> int:
    """Stage-2 HSZx sum of q: sum p + M_b S_b."""
    dp = np.ascontiguousarray(dp, dtype=np.int32)
    M = np.ascontiguousarray(M, dtype=np.int32)
    s1 = ctypes.c_int64()
    _check(lib().orc_mean_p_sum_x(_ptr(dp), _ptr(M), dp.size, S, ctypes.byref(s1)), "mean_p_sum_x")
    return s1.value


def std_p_x(dp: np.ndarray, M: np.ndarray, S: int, eps: float):
    """Stage-2 HSZx standard deviation about the integer mean mu~:
    (mu~, exact sum (p + M_b - mu~)^2, sigma)."""
    dp = np.ascontiguousarray(dp, dtype=np.int32)
    M = np.ascontiguousarray(M, dtype=np.int32)
    mt, lo, hi, sg = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
    _check(lib().orc_std_p_x(_ptr(dp), _ptr(M), dp.size, S, eps, ctypes.byref(mt), ctypes.byref(lo),
                             ctypes.byref(hi), ctypes.byref(sg)), "std_p_x")
    return mt.value, (hi.value << 64) | lo.value, sg.value


def finalize(n: int, s1: int, s2: int, eps: float):
    """(mean, variance, std) from the exact sums, scaled by 2 eps at the end."""
    m, v, sd = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().orc_finalize(n, s1, s2 & ((1 << 64) - 1), s2 >> 64, eps, ctypes.byref(m),
                              ctypes.byref(v), ctypes.byref(sd)), "finalize")
    return m.value, v.value, sd.value


def stats_f(f: np.ndarray):
    """Generic flow on D_f: (mean, sample variance) in compensated double."""
    f = np.ascontiguousarray(f)
    m, v = ctypes.c_double(), ctypes.c_double()
    _check(lib().orc_stats_f(_ptr(f), _dtype_code(f), f.size, ctypes.byref(m), ctypes.byref(v)), "stats_f")
    return m.value, v.value


# ----------------------------------------------------------------- stencils
def deriv_q(q: np.ndarray, axis: int) -> np.ndarray:
    """Integer derivative numerators along a user axis (0 = slowest)."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    d = dims3(q.shape)
    out = np.empty(q.shape, np.int64)
    _check(lib().orc_deriv_q(_ptr(q), _ptr(d), axis + 3 - q.ndim, _ptr(out)), "deriv_q")
    return out


def lap_q(q: np.ndarray) -> np.ndarray:
    """Integer Laplacian numerators (replicated edges)."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    d = dims3(q.shape)
    out = np.empty(q.shape, np.int64)
    _check(lib().orc_lap_q(_ptr(q), _ptr(d), _ptr(out)), "lap_q")
    return out


def stencil_q(q: np.ndarray, kind: int, eps: float, axis: int = 0) -> np.ndarray:
    """Homomorphic stage-3 result in double: eps*D, eps*|D|, or 2 eps*L."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    d = dims3(q.shape)
    out = np.empty(q.shape, np.float64)
    _check(lib().orc_stencil_q(_ptr(q), _ptr(d), kind, axis + 3 - q.ndim, eps, _ptr(out)), "stencil_q")
    return out


def divergence_q(qs, eps):
    """Divergence of the vector field whose components (same shape, ndim
    components) are the code arrays qs, component c differentiated along user
    axis c: (integer numerators, values)."""
    qs = [np.ascontiguousarray(q, dtype=np.int32) for q in qs]
    nd = qs[0].ndim
    d = dims3(qs[0].shape)
    axes = np.array([c + 3 - nd for c in range(len(qs))], np.int32)
    ptrs = (ctypes.c_void_p * len(qs))(*[q.ctypes.data for q in qs])
    e = np.ascontiguousarray(eps, dtype=np.float64)
    num = np.empty(qs[0].shape, np.int64)
    val = np.empty(qs[0].shape, np.float64)
    _check(lib().orc_divergence_q(ptrs, len(qs), _ptr(d), _ptr(axes), _ptr(e), _ptr(num), _ptr(val)),
           "divergence_q")
    return num, val


def curl2_q(qu, qv, eps_u, eps_v):
    """Curl of a 2-D field (u, v): (integer numerators, values)."""
    qu = np.ascontiguousarray(qu, dtype=np.int32)
    qv = np.ascontiguousarray(qv, dtype=np.int32)
    assert qu.ndim == 2 and qu.shape == qv.shape
    d = dims3(qu.shape)
    num = np.empty(qu.shape, np.int64)
    val = np.empty(qu.shape, np.float64)
    _check(lib().orc_curl2_q(_ptr(qu), _ptr(qv), _ptr(d), 1, 2, eps_u, eps_v, _ptr(num), _ptr(val)), "curl2_q")
    return num, val


def stencil_f(f: np.ndarray, kind: int, axis: int = 0) -> np.ndarray:
    """Generic flow on D_f in double (derivative, gradient magnitude, Laplacian)."""
    f = np.ascontiguousarray(f)
    d = dims3(f.shape)
    out = np.empty(f.shape, np.float64)
    _check(lib().orc_stencil_f(_ptr(f), _dtype_code(f), _ptr(d), kind, axis + 3 - f.ndim, _ptr(out)),
           "stencil_f")
    return out


def stencil_at(q: np.ndarray, kind: int, eps: float, idx, axis: int = 0):
    """(integer numerators, scaled values) at flat indices idx only."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    d = dims3(q.shape)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    num = np.empty(idx.size, np.int64)
    val = np.empty(idx.size, np.float64)
    _check(lib().orc_stencil_at(_ptr(q), _ptr(d), kind, axis + 3 - q.ndim, eps, _ptr(idx), idx.size, _ptr(num),
                                _ptr(val)), "stencil_at")
    return num, val


# ------------------------------------------------- global predictors, stage 2
def global_dims(shape, pred: int) -> np.ndarray:
    """Prediction shape: the field's (n0, n1, n2) for HSZp-nd, (1, 1, N) for HSZp."""
    d = dims3(shape)
    if pred == PRED_GLOBAL:
        return np.array((1, 1, int(np.prod(d))), np.int64)
    return d


def lorenzo_mean_p(dp: np.ndarray, pred: int) -> int:
    """Stage-2 sum q of a global-predictor D_p: sum p (L0-z)(L1-y)(L2-x)."""
    dp = np.ascontiguousarray(dp, dtype=np.int32)
    L = global_dims(dp.shape, pred)
    s1 = ctypes.c_int64()
    _check(lib().orc_lorenzo_mean_p(_ptr(dp), _ptr(L), ctypes.byref(s1)), "lorenzo_mean_p")
    return s1.value


def lorenzo_var_p(dp: np.ndarray, pred: int):
    """Stage-2 (sum q, sum q^2) of a global-predictor D_p (Algorithm 4 extended)."""
    dp = np.ascontiguousarray(dp, dtype=np.int32)
    L = global_dims(dp.shape, pred)
    s1, lo, hi = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().orc_lorenzo_var_p(_ptr(dp), _ptr(L), ctypes.byref(s1), ctypes.byref(lo), ctypes.byref(hi)),
           "lorenzo_var_p")
    return s1.value, (hi.value << 64) | lo.value


def lorenzo_deriv_p(dp: np.ndarray, axis: int) -> np.ndarray:
    """Stage-2 derivative numerators of an HSZp-nd D_p along a user axis."""
    dp = np.ascontiguousarray(dp, dtype=np.int32)
    d = dims3(dp.shape)
    out = np.empty(dp.shape, np.int64)
    _check(lib().orc_lorenzo_deriv_p(_ptr(dp), _ptr(d), axis + 3 - dp.ndim, _ptr(out)), "lorenzo_deriv_p")
    return out


def lorenzo_lap_p(dp: np.ndarray) -> np.ndarray:
    """Stage-2 Laplacian numerators of an HSZp-nd D_p (replicated edges)."""
    dp = np.ascontiguousarray(dp, dtype=np.int32)
    d = dims3(dp.shape)
    out = np.empty(dp.shape, np.int64)
    _check(lib().orc_lorenzo_lap_p(_ptr(dp), _ptr(d), _ptr(out)), "lorenzo_lap_p")
    return out


# ------------------------------------------------------ HSZx-nd (boxes of codes)
def compress_nd(x: np.ndarray, block, eb: float, rel: bool = True):
    """Algorithm 1 with block means over boxes of `block` codes (HSZx-nd)."""
    x = np.ascontiguousarray(x)
    d = np.array(x.shape, np.int64)
    b = np.array(block, np.int64)
    cap = int(lib().orc_compress_bound_nd(x.ndim, _ptr(d), _ptr(b)))
    if cap < 0:
        raise OracleError(1, "compress_bound_nd")
    out = np.zeros(cap, np.uint8)
    nbytes, eps = ctypes.c_int64(), ctypes.c_double()
    _check(lib().orc_compress_nd(_ptr(x), _dtype_code(x), x.ndim, _ptr(d), _ptr(b), eb, int(rel), _ptr(out), cap,
                                 ctypes.byref(nbytes), ctypes.byref(eps)), "compress_nd")
    return out[: nbytes.value].copy(), eps.value


def compress_codes_nd(q: np.ndarray, block, eps: float, dtype=np.float32, eb=None, rel=False):
    """Encode given codes with block means over boxes of `block` codes."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    d = np.array(q.shape, np.int64)
    b = np.array(block, np.int64)
    cap = int(lib().orc_compress_bound_nd(q.ndim, _ptr(d), _ptr(b)))
    if cap < 0:
        raise OracleError(1, "compress_bound_nd")
    out = np.zeros(cap, np.uint8)
    nbytes = ctypes.c_int64()
    code = 0 if np.dtype(dtype) == np.float32 else 1
    _check(lib().orc_compress_codes_nd(_ptr(q), code, q.ndim, _ptr(d), _ptr(b), eps, eps if eb is None else eb,
                                       int(rel), _ptr(out), cap, ctypes.byref(nbytes)), "compress_codes_nd")
    return out[: nbytes.value].copy()


def _bd3(shape, block):
    return dims3(shape), np.array((1,) * (3 - len(block)) + tuple(int(v) for v in block), np.int64)


def xnd_mean_m(M: np.ndarray, shape, block) -> int:
    """Stage-1 sum of the box means times the true box sizes (Eq. mean_m)."""
    M = np.ascontiguousarray(M, dtype=np.int32)
    d, b = _bd3(shape, block)
    t = ctypes.c_int64()
    _check(lib().orc_xnd_mean_m(_ptr(M), _ptr(d), _ptr(b), ctypes.byref(t)), "xnd_mean_m")
    return t.value


def xnd_mean_p(dp: np.ndarray, M: np.ndarray, block) -> int:
    """Stage-2 sum q of HSZx-nd: sum p + M_b S_b."""
    dp = np.ascontiguousarray(dp, dtype=np.int32)
    M = np.ascontiguousarray(M, dtype=np.int32)
    d, b = _bd3(dp.shape, block)
    s1 = ctypes.c_int64()
    _check(lib().orc_xnd_mean_p(_ptr(dp), _ptr(M), _ptr(d), _ptr(b), ctypes.byref(s1)), "xnd_mean_p")
    return s1.value


def xnd_std_p(dp: np.ndarray, M: np.ndarray, block, eps: float):
    """Stage-2 HSZx-nd standard deviation about mu~: (mu~, exact sum of squares, sigma)."""
    dp = np.ascontiguousarray(dp, dtype=np.int32)
    M = np.ascontiguousarray(M, dtype=np.int32)
    d, b = _bd3(dp.shape, block)
    mt, lo, hi, sg = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
    _check(lib().orc_xnd_std_p(_ptr(dp), _ptr(M), _ptr(d), _ptr(b), eps, ctypes.byref(mt), ctypes.byref(lo),
                               ctypes.byref(hi), ctypes.byref(sg)), "xnd_std_p")
    return mt.value, (hi.value << 64) | lo.value, sg.value


def xnd_deriv_p(dp: np.ndarray, M: np.ndarray, block, axis: int) -> np.ndarray:
    """Stage-2 HSZx-nd derivative numerators along a user axis."""
    dp = np.ascontiguousarray(dp, dtype=np.int32)
    M = np.ascontiguousarray(M, dtype=np.int32)
    d, b = _bd3(dp.shape, block)
    out = np.empty(dp.shape, np.int64)
    _check(lib().orc_xnd_deriv_p(_ptr(dp), _ptr(M), _ptr(d), _ptr(b), axis + 3 - dp.ndim, _ptr(out)),
           "xnd_deriv_p")
    return out


def xnd_lap_p(dp: np.ndarray, M: np.ndarray, block) -> np.ndarray:
    """Stage-2 HSZx-nd Laplacian numerators (replicated edges)."""
    dp = np.ascontiguousarray(dp, dtype=np.int32)
    M = np.ascontiguousarray(M, dtype=np.int32)
    d, b = _bd3(dp.shape, block)
    out = np.empty(dp.shape, np.int64)
    _check(lib().orc_xnd_lap_p(_ptr(dp), _ptr(M), _ptr(d), _ptr(b), _ptr(out)), "xnd_lap_p")
    return out
