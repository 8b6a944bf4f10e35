"""ctypes binding of libhc.so (include/hc.h).

Argument marshalling only: torch provides device memory and the current CUDA
stream; every step of compression, decompression and the homomorphic
operations runs in the library's CUDA kernels.  There is no fallback: if the
library or a GPU is missing, loading fails with an error.

Two layers:
* ``lib()`` returns the raw ctypes functions named exactly as in hc.h
  (``hc_compress``, ``hc_decompress_to_stage``, ``hc_op_mean`` ...).
* ``compress`` / ``decompress`` / ``mean`` / ``variance`` / ``derivative`` /
  ``gradmag`` / ``laplacian`` allocate outputs with torch and call them.

Streams: every call takes ``stream=`` (default: torch's current stream) and
queues its kernels there.  The operation workspace is allocated and zeroed on
that stream.  Outputs are allocated the torch way, on the current stream: a
caller that passes another stream runs the call inside
``torch.cuda.stream(s)``, or orders the streams itself, as with any torch
tensor that is used on a side stream.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhc.so")

HC_OK, HC_ERR_INVALID_ARG, HC_ERR_RANGE, HC_ERR_CORRUPT, HC_ERR_UNSUPPORTED = 0, 1, 2, 3, 4
HC_ERR_CUDA, HC_ERR_NOMEM, HC_ERR_TIMEOUT = 5, 6, 7
HC_F32, HC_F64, HC_I32, HC_I64 = 0, 1, 2, 3
HC_EB_ABS, HC_EB_REL = 0, 1
HC_STAGE_COMPRESSED, HC_STAGE_M, HC_STAGE_P, HC_STAGE_Q, HC_STAGE_F = 0, 1, 2, 3, 4
HC_OP_MEAN, HC_OP_VARIANCE, HC_OP_DERIVATIVE, HC_OP_GRADMAG, HC_OP_LAPLACIAN = 0, 1, 2, 3, 4
HC_OP_MULTI = 5
OPS = {"multi": HC_OP_MULTI, "mean": HC_OP_MEAN, "variance": HC_OP_VARIANCE, "derivative": HC_OP_DERIVATIVE, "gradmag": HC_OP_GRADMAG,
       "laplacian": HC_OP_LAPLACIAN}

STAGES = {"m": HC_STAGE_M, "p": HC_STAGE_P, "q": HC_STAGE_Q, "f": HC_STAGE_F}

# Names of every function declared in include/hc.h (checked by the tests).
ABI_FUNCTIONS = (
    "hc_status_str", "hc_last_error", "hc_version", "hc_compress_bound", "hc_compress_workspace_bytes",
    "hc_workspace_bytes", "hc_stage_bytes", "hc_compress", "hc_compress_codes", "hc_read_header",
    "hc_decompress_to_stage", "hc_workspace_status", "hc_op_mean", "hc_op_variance", "hc_op_std",
    "hc_op_derivative", "hc_op_gradmag", "hc_op_laplacian", "hc_op_variance_noalloc", "hc_autotune",
    "hc_batch_plan_bytes", "hc_batch_workspace_bytes", "hc_batch_plan", "hc_batch_run", "hc_batch_graph_create",
    "hc_batch_graph_launch", "hc_batch_graph_destroy", "hc_batch_status", "hc_op_multi", "hc_compress_ex",
    "hc_compress_codes_ex", "hc_op_divergence", "hc_op_curl", "hc_workspace_bytes_for", "hc_compress_bound_nd",
    "hc_compress_workspace_bytes_nd", "hc_compress_nd", "hc_compress_codes_nd", "hc_vector_workspace_bytes",
    "hc_shard_plan", "hc_read_header_host", "hc_finalize", "hc_autotune_export", "hc_autotune_import",
)
HC_PRED_DELTA, HC_PRED_MEAN, HC_PRED_LORENZO, HC_PRED_GLOBAL_DELTA, HC_PRED_MEAN_ND = 0, 1, 2, 3, 4
# "delta": HSZp with block heads; "mean": HSZx; "lorenzo": HSZp-nd (Lorenzo over
# the field's axes); "global": HSZp (delta across blocks, flattened field);
# "mean-nd": HSZx-nd (box means, boxes given by `block`)
PREDICTORS = {"delta": HC_PRED_DELTA, "mean": HC_PRED_MEAN, "lorenzo": HC_PRED_LORENZO,
              "global": HC_PRED_GLOBAL_DELTA, "mean-nd": HC_PRED_MEAN_ND}
HC_BATCH_MEAN, HC_BATCH_VARIANCE, HC_BATCH_DERIVATIVE, HC_BATCH_GRADMAG, HC_BATCH_LAPLACIAN = 1, 2, 4, 8, 16
HC_BATCH_DIVERGENCE, HC_BATCH_CURL = 32, 64
BATCH_OPS = {"mean": HC_BATCH_MEAN, "variance": HC_BATCH_VARIANCE, "derivative": HC_BATCH_DERIVATIVE,
             "gradmag": HC_BATCH_GRADMAG, "laplacian": HC_BATCH_LAPLACIAN, "divergence": HC_BATCH_DIVERGENCE,
             "curl": HC_BATCH_CURL}


class HcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libhc status {status}: {msg}")
        self.status = status


class HcHeader(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("ndim", ctypes.c_int32), ("dims", ctypes.c_int64 * 3),
                ("S", ctypes.c_int32), ("G", ctypes.c_int32), ("eps", ctypes.c_double), ("eb", ctypes.c_double),
                ("eb_mode", ctypes.c_int32), ("qmax", ctypes.c_uint32), ("N", ctypes.c_int64),
                ("nb", ctypes.c_int64), ("nchunks", ctypes.c_int64), ("payload_words", ctypes.c_int64),
                ("off_widths", ctypes.c_int64), ("off_heads", ctypes.c_int64), ("off_chunks", ctypes.c_int64),
                ("off_payload", ctypes.c_int64), ("total_bytes", ctypes.c_int64), ("wmax", ctypes.c_uint32),
                ("pred", ctypes.c_uint32), ("block", ctypes.c_uint32 * 3)]

    @property
    def shape(self):
        return tuple(int(d) for d in self.dims)[3 - self.ndim:]


class HcStage(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("d_data", ctypes.c_void_p),
                ("hdr", ctypes.POINTER(HcHeader)), ("dtype", ctypes.c_int32), ("S", ctypes.c_int32),
                ("n", ctypes.c_int64), ("qmax", ctypes.c_uint32), ("pred", ctypes.c_uint32)]


class HcBatchItem(ctypes.Structure):
    _fields_ = [("d_stream", ctypes.c_void_p), ("hdr", HcHeader), ("ops", ctypes.c_uint32), ("axis", ctypes.c_int32),
                ("d_scalar", ctypes.c_void_p), ("d_field", ctypes.c_void_p), ("field_dtype", ctypes.c_int32),
                ("ncomp", ctypes.c_int32), ("comps", ctypes.c_void_p)]


class HcMultiOut(ctypes.Structure):
    _fields_ = [("d_derivative", ctypes.c_void_p * 3), ("d_gradmag", ctypes.c_void_p),
                ("d_laplacian", ctypes.c_void_p), ("d_stats", ctypes.c_void_p), ("out_dtype", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class HcShard(ctypes.Structure):
    _fields_ = [("hdr", HcHeader), ("header_bytes", ctypes.c_uint8 * 256), ("src_off", ctypes.c_int64 * 3),
                ("dst_off", ctypes.c_int64 * 3), ("nbytes", ctypes.c_int64 * 3), ("chunks_off", ctypes.c_int64),
                ("first", ctypes.c_int64)]


class HcBatchTune(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ty", ctypes.c_int32), ("unit_elems", ctypes.c_int64),
                ("ctas_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32)]


SCALAR_BYTES = 64
_SCALAR_DTYPE = np.dtype([("mean", "<f8"), ("variance", "<f8"), ("std", "<f8"), ("n", "<i8"), ("s1", "<i8"),
                          ("s2_lo", "<u8"), ("s2_hi", "<u8"), ("status", "<i4"), ("exact", "<i4")])

_lib = None
_lock = threading.Lock()


def lib():
    """Load libhc.so (build it first with paper_2603_25206_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, sz, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
        P = ctypes.POINTER
        sig = {
            "hc_status_str": ([i32], ctypes.c_char_p),
            "hc_last_error": ([], ctypes.c_char_p),
            "hc_version": ([], i32),
            "hc_compress_bound": ([i64, i32], sz),
            "hc_compress_workspace_bytes": ([i64, i32], sz),
            "hc_workspace_bytes": ([], sz),
            "hc_workspace_bytes_for": ([P(HcHeader)], sz),
            "hc_compress_bound_nd": ([i32, P(ctypes.c_int64), P(ctypes.c_int32)], sz),
            "hc_vector_workspace_bytes": ([P(HcStage), i32], sz),
            "hc_shard_plan": ([P(HcHeader), vp, i64, i64, P(HcShard), vp], i32),
            "hc_read_header_host": ([vp, sz, P(HcHeader)], i32),
            "hc_finalize": ([i64, i64, ctypes.c_uint64, ctypes.c_uint64, dbl, vp], i32),
            "hc_compress_workspace_bytes_nd": ([i32, P(ctypes.c_int64), P(ctypes.c_int32)], sz),
            "hc_compress_nd": ([vp, i32, i32, P(ctypes.c_int64), P(ctypes.c_int32), dbl, i32, vp, sz, vp, sz, P(sz),
                                P(HcHeader), vp], i32),
            "hc_compress_codes_nd": ([vp, i32, i32, P(ctypes.c_int64), P(ctypes.c_int32), dbl, dbl, i32, vp, sz, vp,
                                      sz, P(sz), P(HcHeader), vp], i32),
            "hc_stage_bytes": ([P(HcHeader), i32], sz),
            "hc_compress": ([vp, i32, i32, P(ctypes.c_int64), dbl, i32, i32, vp, sz, vp, sz, P(sz), P(HcHeader), vp],
                            i32),
            "hc_compress_codes": ([vp, i32, i32, P(ctypes.c_int64), dbl, dbl, i32, i32, vp, sz, vp, sz, P(sz),
                                   P(HcHeader), vp], i32),
            "hc_compress_ex": ([vp, i32, i32, P(ctypes.c_int64), dbl, i32, i32, i32, vp, sz, vp, sz, P(sz),
                                P(HcHeader), vp], i32),
            "hc_compress_codes_ex": ([vp, i32, i32, P(ctypes.c_int64), dbl, dbl, i32, i32, i32, vp, sz, vp, sz,
                                      P(sz), P(HcHeader), vp], i32),
            "hc_read_header": ([vp, sz, P(HcHeader), vp], i32),
            "hc_decompress_to_stage": ([P(HcHeader), vp, i32, vp, i32, vp, sz, vp], i32),
            "hc_workspace_status": ([vp, vp], i32),
            "hc_op_mean": ([P(HcStage), dbl, i32, P(ctypes.c_int64), vp, vp, sz, vp], i32),
            "hc_op_variance": ([P(HcStage), dbl, i32, P(ctypes.c_int64), vp, vp, sz, vp], i32),
            "hc_op_std": ([P(HcStage), dbl, i32, P(ctypes.c_int64), vp, vp, sz, vp], i32),
            "hc_op_variance_noalloc": ([P(HcStage), dbl, i32, P(ctypes.c_int64), vp, vp], i32),
            "hc_op_derivative": ([P(HcStage), dbl, i32, P(ctypes.c_int64), i32, vp, i32, vp, sz, vp], i32),
            "hc_op_gradmag": ([P(HcStage), dbl, i32, P(ctypes.c_int64), vp, i32, vp, sz, vp], i32),
            "hc_op_laplacian": ([P(HcStage), dbl, i32, P(ctypes.c_int64), vp, i32, vp, sz, vp], i32),
            "hc_autotune": ([P(HcStage), i32, i32, vp, vp, sz, vp, P(ctypes.c_int)], i32),
            "hc_autotune_export": ([ctypes.c_char_p, sz, P(sz)], i32),
            "hc_autotune_import": ([ctypes.c_char_p, P(ctypes.c_int)], i32),
            "hc_op_multi": ([P(HcStage), dbl, i32, P(ctypes.c_int64), P(HcMultiOut), vp, sz, vp], i32),
            "hc_op_divergence": ([P(HcStage), i32, i32, P(ctypes.c_int64), vp, i32, vp, sz, vp], i32),
            "hc_op_curl": ([P(HcStage), i32, i32, P(ctypes.c_int64), vp, i32, vp, sz, vp], i32),
            "hc_batch_plan_bytes": ([i32], sz),
            "hc_batch_workspace_bytes": ([i32], sz),
            "hc_batch_plan": ([P(HcBatchItem), i32, P(HcBatchTune), vp, sz, P(sz)], i32),
            "hc_batch_run": ([vp, vp, vp, sz, vp], i32),
            "hc_batch_graph_create": ([vp, vp, vp, sz, P(vp)], i32),
            "hc_batch_graph_launch": ([vp, vp], i32),
            "hc_batch_graph_destroy": ([vp], i32),
            "hc_batch_status": ([vp, vp], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc: int):
    if rc != HC_OK:
        raise HcError(rc, lib().hc_last_error().decode())


# ------------------------------------------------------------ torch plumbing
def _torch():
    import torch

    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dims(shape):
    arr = (ctypes.c_int64 * 3)()
    for i, d in enumerate(shape):
        arr[i] = int(d)
    return arr


_ws_cache: dict = {}


def workspace(device=None, stream=None, nbytes: int = 0):
    """Zero-initialised operation workspace, one per (device, stream), of at
    least hc_workspace_bytes() and `nbytes` bytes (grown on demand)."""
    torch = _torch()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    key = (dev.index, s.cuda_stream)
    ws = _ws_cache.get(key)
    need = max(int(lib().hc_workspace_bytes()), int(nbytes))
    if ws is None or ws.numel() < need:
        if ws is not None:
            s.synchronize()  # the old buffer may still be in use by queued work
        # allocated and zero-filled on the stream it serves, so the fill is
        # ordered before the first kernel that reads it even when that stream
        # is not torch's current one
        with torch.cuda.stream(s):
            ws = torch.zeros(need, dtype=torch.uint8, device=dev)
        _ws_cache[key] = ws
    return ws


def _workspace_for(inp, dev, stream):
    """The workspace a call on `inp` needs (global-predictor streams need scratch)."""
    if isinstance(inp, Compressed):
        return workspace(dev, stream, int(lib().hc_workspace_bytes_for(ctypes.byref(inp.header))))
    return workspace(dev, stream)


@dataclass
class Compressed:
    """A device-resident stream with its host-side header."""
    stream: "object"  # torch.uint8 tensor (possibly larger than nbytes)
    header: HcHeader
    nbytes: int

    @property
    def shape(self):
        return self.header.shape

    @property
    def eps(self):
        return self.header.eps

    @property
    def dtype(self):
        return "float64" if self.header.dtype == HC_F64 else "float32"

    def stage(self, level: str = "q") -> HcStage:
        st = HcStage()
        st.kind = HC_STAGE_COMPRESSED
        st.level = STAGES[level]
        st.d_data = self.stream.data_ptr()
        st.hdr = ctypes.pointer(self.header)
        return st


@dataclass
class StageArray:
    """A materialized stage: kind 'm', 'p', 'q' or 'f' (torch tensor on the GPU)."""
    kind: str
    data: "object"
    shape: tuple
    eps: float
    S: int = 0
    qmax: int = 0
    pred: int = HC_PRED_DELTA

    def stage(self) -> HcStage:
        torch = _torch()
        st = HcStage()
        st.kind = STAGES[self.kind]
        st.d_data = self.data.data_ptr()
        st.dtype = HC_F64 if self.data.dtype == torch.float64 else HC_F32
        st.S = self.S
        st.n = int(np.prod(self.shape))
        st.qmax = self.qmax
        st.pred = self.pred
        return st


def _block(block, ndim):
    if block is None or len(block) != ndim:
        raise ValueError("predictor 'mean-nd' needs block: one box extent per axis")
    arr = (ctypes.c_int32 * 3)()
    for i, b in enumerate(block):
        arr[i] = int(b)
    return arr


def compress(x, eb: float, rel: bool = True, S: int = 32, stream=None, predictor: str = "delta",
             block=None) -> Compressed:
    """C (Algorithm 1) of a float32/float64 CUDA tensor.  predictor "delta"
    (HSZp with block heads), "mean" (HSZx: block means), "lorenzo" (HSZp-nd),
    "global" (HSZp, delta across blocks) or "mean-nd" (HSZx-nd: box means,
    boxes of `block` codes, one extent per axis; S is then their product)."""
    torch = _torch()
    if predictor == "mean-nd":
        return _compress_nd(x, None, eb, rel, block, stream)
    if not x.is_cuda:
        raise ValueError("compress expects a CUDA tensor")
    x = x.contiguous()
    dtype = HC_F64 if x.dtype == torch.float64 else HC_F32
    if x.dtype not in (torch.float32, torch.float64):
        raise TypeError("fields are float32 or float64")
    L = lib()
    cap = int(L.hc_compress_bound(x.numel(), S))
    out = torch.empty(cap, dtype=torch.uint8, device=x.device)
    ws = torch.empty(int(L.hc_compress_workspace_bytes(x.numel(), S)), dtype=torch.uint8, device=x.device)
    nbytes = ctypes.c_size_t()
    hdr = HcHeader()
    _check(L.hc_compress_ex(ctypes.c_void_p(x.data_ptr()), dtype, x.dim(), _dims(x.shape), eb,
                            HC_EB_REL if rel else HC_EB_ABS, S, PREDICTORS[predictor],
                            ctypes.c_void_p(out.data_ptr()), cap, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                            ctypes.byref(nbytes), ctypes.byref(hdr), _stream_ptr(stream)))
    return Compressed(out, hdr, nbytes.value)


def _compress_nd(x, codes_eps, eb, rel, block, stream, dtype="float32"):
    torch = _torch()
    src = x.contiguous()
    shape = tuple(src.shape)
    L = lib()
    bl = _block(block, len(shape))
    cap = int(L.hc_compress_bound_nd(len(shape), _dims(shape), bl))
    wsn = int(L.hc_compress_workspace_bytes_nd(len(shape), _dims(shape), bl))
    if not cap or not wsn:
        raise HcError(HC_ERR_INVALID_ARG, "bad shape or box extents")
    out = torch.empty(cap, dtype=torch.uint8, device=src.device)
    ws = torch.empty(wsn, dtype=torch.uint8, device=src.device)
    nbytes = ctypes.c_size_t()
    hdr = HcHeader()
    if codes_eps is None:
        dt = HC_F64 if src.dtype == torch.float64 else HC_F32
        _check(L.hc_compress_nd(ctypes.c_void_p(src.data_ptr()), dt, len(shape), _dims(shape), bl, eb,
                                HC_EB_REL if rel else HC_EB_ABS, ctypes.c_void_p(out.data_ptr()), cap,
                                ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.byref(nbytes), ctypes.byref(hdr),
                                _stream_ptr(stream)))
    else:
        _check(L.hc_compress_codes_nd(ctypes.c_void_p(src.data_ptr()), HC_F64 if dtype == "float64" else HC_F32,
                                      len(shape), _dims(shape), bl, codes_eps, codes_eps if eb is None else eb,
                                      HC_EB_REL if rel else HC_EB_ABS, ctypes.c_void_p(out.data_ptr()), cap,
                                      ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.byref(nbytes),
                                      ctypes.byref(hdr), _stream_ptr(stream)))
    return Compressed(out, hdr, nbytes.value)


def compress_codes(q, eps: float, S: int = 32, dtype: str = "float32", eb=None, rel=False, stream=None,
                   predictor: str = "delta", block=None) -> Compressed:
    """Encode given int32 codes (CUDA tensor)."""
    torch = _torch()
    if predictor == "mean-nd":
        return _compress_nd(q, eps, eb, rel, block, stream, dtype)
    q = q.contiguous()
    L = lib()
    cap = int(L.hc_compress_bound(q.numel(), S))
    out = torch.empty(cap, dtype=torch.uint8, device=q.device)
    ws = torch.empty(int(L.hc_compress_workspace_bytes(q.numel(), S)), dtype=torch.uint8, device=q.device)
    nbytes = ctypes.c_size_t()
    hdr = HcHeader()
    _check(L.hc_compress_codes_ex(ctypes.c_void_p(q.data_ptr()), HC_F64 if dtype == "float64" else HC_F32,
                                  q.dim(), _dims(q.shape), eps, eps if eb is None else eb,
                                  HC_EB_REL if rel else HC_EB_ABS, S, PREDICTORS[predictor],
                                  ctypes.c_void_p(out.data_ptr()), cap, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                  ctypes.byref(nbytes), ctypes.byref(hdr), _stream_ptr(stream)))
    return Compressed(out, hdr, nbytes.value)


def from_stream(stream_tensor, stream=None) -> Compressed:
    """Wrap a device-resident stream (uint8 tensor): reads and checks its header."""
    hdr = HcHeader()
    _check(lib().hc_read_header(ctypes.c_void_p(stream_tensor.data_ptr()), stream_tensor.numel(),
                                ctypes.byref(hdr), _stream_ptr(stream)))
    return Compressed(stream_tensor, hdr, int(hdr.total_bytes))


def header_of(data) -> HcHeader:
    """The checked header of a stream held in host memory (bytes, bytearray,
    memoryview or a numpy array holding the whole stream, read as its raw
    bytes whatever its dtype): hc_read_header_host."""
    if isinstance(data, np.ndarray):
        arr = np.ascontiguousarray(data).reshape(-1).view(np.uint8)
    else:
        arr = np.frombuffer(memoryview(data).cast("B"), np.uint8)
    hdr = HcHeader()
    _check(lib().hc_read_header_host(ctypes.c_void_p(arr.ctypes.data), arr.size, ctypes.byref(hdr)))
    return hdr


def save(c: Compressed, path: str) -> int:
    """Write the stream of c (its total_bytes, header first) to `path`; the
    file is the persistent form of the compressed field.  Returns the bytes
    written."""
    data = c.stream[: c.nbytes].cpu().numpy()
    with open(path, "wb") as f:
        f.write(data.tobytes())
    return int(data.size)


def load(path: str, device=None) -> Compressed:
    """Read a stream written by save (or by any producer of the same format),
    check its header on the host, and put it on `device` (default: the current
    CUDA device)."""
    torch = _torch()
    data = np.fromfile(path, dtype=np.uint8)
    hdr = header_of(data)
    n = int(hdr.total_bytes)
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    t = torch.from_numpy(data[:n].copy()).to(dev)
    return Compressed(t, hdr, n)


def shard_range(nchunks: int, rank: int, world: int):
    """Chunks [c0, c1) of rank `rank` of `world`: contiguous, balanced, in
    rank order (empty when there are more ranks than chunks)."""
    if not (0 <= rank < world):
        raise ValueError("rank must be in [0, world)")
    return rank * nchunks // world, (rank + 1) * nchunks // world


def shard_plan(header: HcHeader, chunks, c0: int, c1: int):
    """hc_shard_plan on a host copy of the chunk index (uint64 array of
    nchunks + 1 words): the shard's HcShard and its rebased chunk index."""
    chunks = np.ascontiguousarray(chunks, dtype=np.uint64)
    if chunks.size != int(header.nchunks) + 1:
        raise ValueError("the chunk index has nchunks + 1 words")
    plan = HcShard()
    out = np.empty(c1 - c0 + 1 if c1 > c0 else 1, np.uint64)
    _check(lib().hc_shard_plan(ctypes.byref(header), ctypes.c_void_p(chunks.ctypes.data), int(c0), int(c1),
                               ctypes.byref(plan), ctypes.c_void_p(out.ctypes.data)))
    return plan, out


def shard(c: Compressed, rank: int, world: int, stream=None):
    """The part of c that rank `rank` of `world` reduces: a stream of its own
    made of contiguous whole chunks (hc_shard_plan), built on c's device with
    copies only.  None when the rank has no chunk.  The statistics of the
    ranks' shards add up exactly to those of c (paper_2603_25206_gb300.shard
    combines them across ranks)."""
    torch = _torch()
    c0, c1 = shard_range(int(c.header.nchunks), rank, world)
    if c1 <= c0:
        return None
    off = int(c.header.off_chunks)
    n_idx = int(c.header.nchunks) + 1
    s = torch.cuda.current_stream(c.stream.device) if stream is None else stream
    with torch.cuda.stream(s):
        chunks = c.stream[off:off + 8 * n_idx].cpu().numpy().view(np.uint64)
        plan, rebased = shard_plan(c.header, chunks, c0, c1)
        total = int(plan.hdr.total_bytes)
        out = torch.zeros(total, dtype=torch.uint8, device=c.stream.device)
        out[:256] = torch.from_numpy(np.frombuffer(bytes(plan.header_bytes), np.uint8).copy()).to(out.device)
        for k in range(3):
            n = int(plan.nbytes[k])
            if n:
                so, do = int(plan.src_off[k]), int(plan.dst_off[k])
                out[do:do + n].copy_(c.stream[so:so + n])
        co = int(plan.chunks_off)
        out[co:co + 8 * rebased.size] = torch.from_numpy(rebased.view(np.uint8).copy()).to(out.device)
    hdr = HcHeader()
    ctypes.memmove(ctypes.byref(hdr), ctypes.byref(plan.hdr), ctypes.sizeof(HcHeader))
    return Compressed(out, hdr, total)


def decompress(c: Compressed, stage: str = "f", out=None, out_dtype=None, stream=None):
    """D_i..D_1 (Algorithm 2) to stage 'm', 'p', 'q' or 'f'."""
    torch = _torch()
    kind = STAGES[stage]
    if stage == "m":
        shape, tdt = (c.header.nb,), torch.int32
    elif stage in ("p", "q"):
        shape, tdt = c.shape, torch.int32
    else:
        f64 = (out_dtype == "float64") if out_dtype else (c.header.dtype == HC_F64)
        shape, tdt = c.shape, (torch.float64 if f64 else torch.float32)
    if out is None:
        out = torch.empty(shape, dtype=tdt, device=c.stream.device)
    odt = HC_F64 if out.dtype == torch.float64 else HC_F32
    ws = _workspace_for(c, c.stream.device, stream)
    _check(lib().hc_decompress_to_stage(ctypes.byref(c.header), ctypes.c_void_p(c.stream.data_ptr()), kind,
                                        ctypes.c_void_p(out.data_ptr()), odt, ctypes.c_void_p(ws.data_ptr()),
                                        ws.numel(), _stream_ptr(stream)))
    return out


def as_stage(c: Compressed, stage: str, data) -> StageArray:
    """Describe a materialized stage of c for the operations."""
    return StageArray(stage, data, c.shape, c.eps, c.header.S, int(c.header.qmax), int(c.header.pred))


def _input(inp, level):
    if isinstance(inp, Compressed):
        return inp.stage(level), inp.eps, inp.shape, inp.stream.device
    return inp.stage(), inp.eps, inp.shape, inp.data.device


def parse_scalar(buf) -> dict:
    """hc_scalar (64 bytes, any tensor/bytes) -> dict with exact s2 as a Python int."""
    raw = np.frombuffer(bytes(buf.cpu().numpy().tobytes()) if hasattr(buf, "cpu") else bytes(buf),
                        dtype=_SCALAR_DTYPE, count=1)[0]
    d = {k: raw[k].item() for k in _SCALAR_DTYPE.names}
    d["s2"] = (int(d.pop("s2_hi")) << 64) | int(d.pop("s2_lo"))
    return d


def finalize(n: int, s1: int, s2: int, eps: float) -> dict:
    """Eq. var_q's final scaling of exact sums (s1 = sum q, s2 = sum q^2 as a
    Python int below 2^128) over n codes, computed by the library on the host
    (hc_finalize: the device finish's arithmetic and roundings); returns the
    parsed hc_scalar."""
    if not (0 <= s2 < (1 << 128)):
        raise ValueError("s2 must be a non-negative 128-bit integer")
    buf = ctypes.create_string_buffer(SCALAR_BYTES)
    _check(lib().hc_finalize(int(n), int(s1), s2 & ((1 << 64) - 1), s2 >> 64, float(eps),
                             ctypes.cast(buf, ctypes.c_void_p)))
    return parse_scalar(buf.raw)


def _stat(fn_name, inp, level, out, stream):
    torch = _torch()
    st, eps, shape, dev = _input(inp, level)
    if out is None:
        out = torch.empty(SCALAR_BYTES, dtype=torch.uint8, device=dev)
    ws = _workspace_for(inp, dev, stream)
    _check(getattr(lib(), fn_name)(ctypes.byref(st), eps, len(shape), _dims(shape), ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
    return out


def mean(inp, level: str = "p", out=None, stream=None):
    """Homomorphic mean; returns the 64-byte device hc_scalar (see parse_scalar)."""
    return _stat("hc_op_mean", inp, level, out, stream)


def variance(inp, level: str = "q", out=None, stream=None):
    return _stat("hc_op_variance", inp, level, out, stream)


def std(inp, level: str = "q", out=None, stream=None):
    return _stat("hc_op_std", inp, level, out, stream)


def variance_noalloc(c: Compressed, level: str = "q", out=None, stream=None):
    """Fused variance without a workspace (static scratch inside libhc.so)."""
    torch = _torch()
    st = c.stage(level)
    if out is None:
        out = torch.empty(SCALAR_BYTES, dtype=torch.uint8, device=c.stream.device)
    _check(lib().hc_op_variance_noalloc(ctypes.byref(st), c.eps, len(c.shape), _dims(c.shape),
                                        ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


_OUT = {"float32": HC_F32, "float64": HC_F64, "int64": HC_I64}


def _field_out(shape, out_dtype, dev, out):
    torch = _torch()
    if out is None:
        tdt = {"float32": torch.float32, "float64": torch.float64, "int64": torch.int64}[out_dtype]
        out = torch.empty(shape, dtype=tdt, device=dev)
    return out


def derivative(inp, axis: int, out_dtype: str = "float32", out=None, level: str = "q", stream=None):
    st, eps, shape, dev = _input(inp, level)
    out = _field_out(shape, out_dtype, dev, out)
    ws = _workspace_for(inp, dev, stream)
    _check(lib().hc_op_derivative(ctypes.byref(st), eps, len(shape), _dims(shape), axis,
                                  ctypes.c_void_p(out.data_ptr()), _OUT[out_dtype], ctypes.c_void_p(ws.data_ptr()),
                                  ws.numel(), _stream_ptr(stream)))
    return out


def gradmag(inp, out_dtype: str = "float32", out=None, level: str = "q", stream=None):
    st, eps, shape, dev = _input(inp, level)
    out = _field_out(shape, out_dtype, dev, out)
    ws = _workspace_for(inp, dev, stream)
    _check(lib().hc_op_gradmag(ctypes.byref(st), eps, len(shape), _dims(shape), ctypes.c_void_p(out.data_ptr()),
                               _OUT[out_dtype], ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
    return out


def laplacian(inp, out_dtype: str = "float32", out=None, level: str = "q", stream=None):
    st, eps, shape, dev = _input(inp, level)
    out = _field_out(shape, out_dtype, dev, out)
    ws = _workspace_for(inp, dev, stream)
    _check(lib().hc_op_laplacian(ctypes.byref(st), eps, len(shape), _dims(shape), ctypes.c_void_p(out.data_ptr()),
                                 _OUT[out_dtype], ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
    return out


def multi(inp, derivative=True, gradmag=True, laplacian=True, stats=True, out_dtype: str = "float32",
          outs=None, level: str = "q", stream=None) -> dict:
    """Every operation of one field from one decode (hc_op_multi).  Returns a
    dict with "derivative" (list per axis), "gradmag", "laplacian" (tensors)
    and "stats" (the 64-byte hc_scalar), each present when requested.
    `outs` may hold preallocated tensors under the same keys."""
    torch = _torch()
    st, eps, shape, dev = _input(inp, level)
    outs = dict(outs or {})
    mo = HcMultiOut()
    mo.out_dtype = _OUT[out_dtype]
    if derivative:
        ds = outs.get("derivative") or [None] * len(shape)
        ds = [_field_out(shape, out_dtype, dev, d) for d in ds]
        outs["derivative"] = ds
        for a, d in enumerate(ds):
            mo.d_derivative[a] = d.data_ptr()
    for key, flag in (("gradmag", gradmag), ("laplacian", laplacian)):
        if flag:
            t = _field_out(shape, out_dtype, dev, outs.get(key))
            outs[key] = t
            setattr(mo, "d_" + key, t.data_ptr())
    if stats:
        t = outs.get("stats")
        if t is None:
            t = torch.empty(SCALAR_BYTES, dtype=torch.uint8, device=dev)
        outs["stats"] = t
        mo.d_stats = t.data_ptr()
    ws = _workspace_for(inp, dev, stream)
    _check(lib().hc_op_multi(ctypes.byref(st), eps, len(shape), _dims(shape), ctypes.byref(mo),
                             ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
    return outs


def _vector(fn, comps, out_dtype, out, stream, level="q"):
    torch = _torch()
    arr = (HcStage * len(comps))()
    for k, c in enumerate(comps):
        arr[k] = c.stage(level)
    shape = comps[0].shape
    dev = comps[0].stream.device
    out = _field_out(shape, out_dtype, dev, out)
    ws = workspace(dev, stream, int(lib().hc_vector_workspace_bytes(arr, len(comps))))
    _check(getattr(lib(), fn)(arr, len(comps), len(shape), _dims(shape), ctypes.c_void_p(out.data_ptr()),
                              _OUT[out_dtype], ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
    return out


def divergence(comps, out_dtype: str = "float32", out=None, stream=None, level: str = "q"):
    """Divergence of the vector field whose components are the compressed
    fields `comps` (one per axis, same shape); level "p" for HSZp-nd and
    HSZx-nd components (Section V-C's stage-2 form)."""
    return _vector("hc_op_divergence", comps, out_dtype, out, stream, level)


def curl(comps, out_dtype: str = "float32", out=None, stream=None, level: str = "q"):
    """Curl of a 2-D vector field (u, v) given as two compressed fields;
    level "p" for HSZp-nd and HSZx-nd components."""
    return _vector("hc_op_curl", comps, out_dtype, out, stream, level)


def workspace_status(stream=None) -> int:
    ws = workspace(None, stream)
    return int(lib().hc_workspace_status(ctypes.c_void_p(ws.data_ptr()), _stream_ptr(stream)))


def autotune(c: Compressed, op: str, out_dtype: str = "float32", out=None, stream=None) -> int:
    """Time the fused stencil's tile heights, each with a one- and a two-wave
    grid, for this field and op ("derivative", "gradmag", "laplacian", or
    "multi" for hc_op_multi's one-pass kernel); later calls use the fastest.
    Returns the chosen tile height."""
    torch = _torch()
    st = c.stage("q")
    if op == "multi" and out is None:
        out = _field_out((len(c.shape) + 2,) + tuple(c.shape), out_dtype, c.stream.device, None)
    out = _field_out(c.shape, out_dtype, c.stream.device, out)
    ws = workspace(c.stream.device, stream)
    chosen = ctypes.c_int()
    _check(lib().hc_autotune(ctypes.byref(st), OPS[op], _OUT[out_dtype], ctypes.c_void_p(out.data_ptr()),
                             ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream), ctypes.byref(chosen)))
    return chosen.value


def autotune_export() -> str:
    """The autotuner's kept choices as JSON text (hc_autotune_export)."""
    n = ctypes.c_size_t()
    _check(lib().hc_autotune_export(None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(lib().hc_autotune_export(buf, n.value + 1, ctypes.byref(n)))
    return buf.value.decode("ascii")


def autotune_import(text: str) -> int:
    """Keep the choices of an exported text for later calls of this process
    (hc_autotune_import); returns the number of entries read."""
    count = ctypes.c_int()
    _check(lib().hc_autotune_import(text.encode("ascii"), ctypes.byref(count)))
    return count.value


def save_autotune(path) -> None:
    """Write the autotuner's kept choices to a JSON file."""
    with open(path, "w") as f:
        f.write(autotune_export())


def load_autotune(path) -> int:
    """Read a file written by save_autotune; returns the number of choices read."""
    with open(path) as f:
        return autotune_import(f.read())


# ------------------------------------------------------------ batched launch
class Batch:
    """Many compressed fields and their operations in one persistent fused
    launch (hc_batch_*).

    ``items``: a list of (Compressed, ops) where ops is a string such as
    "mean|variance|laplacian" (at most one of derivative / gradmag /
    laplacian), or (tuple of component Compressed, "divergence" / "curl")
    for a vector field.  Field outputs are allocated here (``field_dtype``); the
    statistics land in one 64-byte hc_scalar per item.  ``run()`` launches
    the kernel; ``capture()`` records it in a CUDA graph that ``replay()``
    relaunches.  The plan is built once (host) and copied to the device; the
    workspace is zeroed once and left zeroed by every launch.
    """

    def __init__(self, items, field_dtype: str = "float32", axis: int = 0, threads: int = 0, ty: int = 0,
                 unit_elems: int = 0, ctas_per_sm: int = 0, device=None):
        torch = _torch()
        if not items:
            raise ValueError("empty batch")
        L = lib()
        self.comps = [c for c, _ in items]
        first = self.comps[0][0] if isinstance(self.comps[0], (tuple, list)) else self.comps[0]
        dev = device if device is not None else first.stream.device
        n = len(items)
        self.n = n
        self.scalars = torch.zeros((n, SCALAR_BYTES), dtype=torch.uint8, device=dev)
        self.fields = [None] * n
        arr = (HcBatchItem * n)()
        self._vec = []  # the component stage arrays of vector items (read by hc_batch_plan)
        for i, (c, ops) in enumerate(items):
            mask = 0
            for name in ops.split("|"):
                mask |= BATCH_OPS[name.strip()]
            it = arr[i]
            if isinstance(c, (tuple, list)):
                comps = (HcStage * len(c))()
                for k, ck in enumerate(c):
                    comps[k] = ck.stage("q")
                self._vec.append((comps, c))
                it.ncomp = len(c)
                it.comps = ctypes.cast(comps, ctypes.c_void_p)
                c = c[0]
            else:
                it.d_stream = c.stream.data_ptr()
                it.hdr = c.header
            it.ops = mask
            it.axis = axis
            if mask & (HC_BATCH_MEAN | HC_BATCH_VARIANCE):
                it.d_scalar = self.scalars[i].data_ptr()
            if mask & (HC_BATCH_DERIVATIVE | HC_BATCH_GRADMAG | HC_BATCH_LAPLACIAN | HC_BATCH_DIVERGENCE |
                       HC_BATCH_CURL):
                f = _field_out(c.shape, field_dtype, dev, None)
                self.fields[i] = f
                it.d_field = f.data_ptr()
                it.field_dtype = _OUT[field_dtype]
        self._items = arr
        tune = HcBatchTune(threads, ty, unit_elems, ctas_per_sm, 0)
        cap = int(L.hc_batch_plan_bytes(n))
        self.h_plan = torch.empty(cap, dtype=torch.uint8).pin_memory()
        used = ctypes.c_size_t()
        _check(L.hc_batch_plan(arr, n, ctypes.byref(tune), ctypes.c_void_p(self.h_plan.data_ptr()), cap,
                               ctypes.byref(used)))
        self.d_plan = self.h_plan.to(dev, non_blocking=False)
        self.ws = torch.zeros(int(L.hc_batch_workspace_bytes(n)), dtype=torch.uint8, device=dev)
        self.graph = None
        self.plan_info = np.frombuffer(self.h_plan[:24].numpy().tobytes(), dtype=np.int32).tolist()

    @property
    def threads(self):
        return self.plan_info[2]

    @property
    def grid(self):
        return self.plan_info[3]

    @property
    def smem(self):
        return self.plan_info[4]

    def run(self, stream=None):
        _check(lib().hc_batch_run(ctypes.c_void_p(self.h_plan.data_ptr()), ctypes.c_void_p(self.d_plan.data_ptr()),
                                  ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), _stream_ptr(stream)))

    def capture(self):
        if self.graph is None:
            g = ctypes.c_void_p()
            _check(lib().hc_batch_graph_create(ctypes.c_void_p(self.h_plan.data_ptr()),
                                               ctypes.c_void_p(self.d_plan.data_ptr()),
                                               ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), ctypes.byref(g)))
            self.graph = g
        return self.graph

    def replay(self, stream=None):
        _check(lib().hc_batch_graph_launch(self.capture(), _stream_ptr(stream)))

    def status(self, stream=None) -> int:
        return int(lib().hc_batch_status(ctypes.c_void_p(self.ws.data_ptr()), _stream_ptr(stream)))

    def results(self):
        """Per item: the parsed hc_scalar (or None) and the field tensor (or None)."""
        raw = self.scalars.cpu().numpy()
        out = []
        for i in range(self.n):
            sc = parse_scalar(raw[i].tobytes()) if self._items[i].d_scalar else None
            out.append((sc, self.fields[i]))
        return out

    def close(self):
        if self.graph is not None:
            lib().hc_batch_graph_destroy(self.graph)
            self.graph = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _trim(c: Compressed) -> Compressed:
    """Keep only the stream bytes resident (drop the bound-sized buffer)."""
    return Compressed(c.stream[: c.nbytes].clone(), c.header, c.nbytes)


def time_batch(b: Batch, reps: int = 5, flush=None) -> float:
    """Median CUDA-event time (ms) of a graph replay of the batch."""
    torch = _torch()
    b.replay()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.replay()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def batch_autotune(fields, eb: float, rel: bool = True, ops: str = "mean|variance|laplacian",
                   S_list=(16, 32, 64, 128), threads_list=(128, 256, 512), ty_list=(0, 16, 8),
                   field_dtype: str = "float32", reps: int = 5, flush=None):
    """Autotuner of the batched launch: block size S, threads per CTA and
    stencil tile height.

    For every S the fields (CUDA tensors) are compressed at that block size;
    for every (threads, tile height) the batch is planned, captured in a CUDA
    graph and timed (median of `reps` replays).  Returns (best, table): best
    is a dict with the chosen S, threads, ty (the largest tile height a field
    may take; 0: no limit), the compressed fields at that S and the planned
    Batch; table lists every (S, threads, ty, ms, compressed bytes).
    The block size changes the stream (and its compression ratio), not the
    results: the codes q, and so every integer result, are the same for all S.
    """
    table = []
    best = None
    for S in S_list:
        comps = [_trim(compress(x, eb, rel=rel, S=S)) for x in fields]
        cbytes = sum(c.nbytes for c in comps)
        for th in threads_list:
            for ty in ty_list:
                b = Batch([(c, ops) for c in comps], field_dtype=field_dtype, threads=th, ty=ty)
                ms = time_batch(b, reps=reps, flush=flush)
                table.append({"S": S, "threads": th, "ty": ty, "ms": ms, "compressed_bytes": cbytes,
                              "grid": b.grid, "smem": b.smem})
                if best is None or ms < best["ms"]:
                    if best is not None:
                        best["batch"].close()
                    best = {"S": S, "threads": th, "ty": ty, "ms": ms, "comps": comps, "batch": b}
                else:
                    b.close()
    return best, table
