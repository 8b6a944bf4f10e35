"""Host-side checks of the C ABI (no GPU needed, no kernel is launched).

* libhc.so loads and exports every function include/hc.h declares, and the
  Python binding names exactly those functions.
* The structs of hc.h have the sizes and field offsets the binding assumes
  (checked against a C program compiled with gcc from hc.h).
* Sizing queries agree with the oracle's layout arithmetic.
* Argument errors are caught on the host before any CUDA call.
"""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from conftest import ROOT

HC_H = os.path.join(ROOT, "include", "hc.h")


def _declared():
    return re.findall(r"HC_API [^(]*?(hc_\w+)\(", open(HC_H).read())


@pytest.fixture(scope="module")
def hc():
    from paper_2603_25206_gb300 import build as b

    b.build()
    from paper_2603_25206_gb300 import hc as mod

    mod.lib()
    return mod


def test_exports_every_declared_symbol(hc):
    names = _declared()
    assert len(names) >= 18
    lib = ctypes.CDLL(hc.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(names) == sorted(hc.ABI_FUNCTIONS)


def test_struct_layout_matches_c(hc):
    src = r"""
#include <stddef.h>
#include <stdio.h>
#include "hc.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(hc_header), sizeof(hc_stage), sizeof(hc_scalar));
  printf("%zu %zu %zu %zu\n", offsetof(hc_header, eps), offsetof(hc_header, N), offsetof(hc_header, wmax),
         offsetof(hc_header, total_bytes));
  printf("%zu %zu %zu %zu\n", offsetof(hc_stage, d_data), offsetof(hc_stage, hdr), offsetof(hc_stage, n),
         offsetof(hc_stage, qmax));
  printf("%zu %zu %zu\n", offsetof(hc_scalar, s1), offsetof(hc_scalar, status), offsetof(hc_scalar, exact));
  printf("%zu %zu %zu %zu %zu\n", sizeof(hc_batch_item), offsetof(hc_batch_item, hdr), offsetof(hc_batch_item, ops),
         offsetof(hc_batch_item, d_scalar), offsetof(hc_batch_item, field_dtype));
  printf("%zu %zu %zu\n", sizeof(hc_batch_tune), offsetof(hc_batch_tune, unit_elems), offsetof(hc_batch_tune, ctas_per_sm));
  printf("%zu %zu %zu\n", sizeof(hc_multi_out), offsetof(hc_multi_out, d_stats), offsetof(hc_multi_out, out_dtype));
  printf("%zu %zu %zu\n", offsetof(hc_header, pred), offsetof(hc_header, block), offsetof(hc_stage, pred));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(hc_shard), offsetof(hc_shard, header_bytes), offsetof(hc_shard, src_off),
         offsetof(hc_shard, nbytes), offsetof(hc_shard, chunks_off), offsetof(hc_shard, first));
  printf("%zu %zu\n", offsetof(hc_batch_item, ncomp), offsetof(hc_batch_item, comps));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HC_H), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    vals = [int(v) for v in out]
    H, St = hc.HcHeader, hc.HcStage
    assert vals[:3] == [ctypes.sizeof(H), ctypes.sizeof(St), hc.SCALAR_BYTES]
    assert vals[3:7] == [H.eps.offset, H.N.offset, H.wmax.offset, H.total_bytes.offset]
    assert vals[7:11] == [St.d_data.offset, St.hdr.offset, St.n.offset, St.qmax.offset]
    assert vals[11:14] == [hc._SCALAR_DTYPE.fields["s1"][1], hc._SCALAR_DTYPE.fields["status"][1],
                           hc._SCALAR_DTYPE.fields["exact"][1]]
    B, T = hc.HcBatchItem, hc.HcBatchTune
    assert vals[14:19] == [ctypes.sizeof(B), B.hdr.offset, B.ops.offset, B.d_scalar.offset, B.field_dtype.offset]
    assert vals[19:22] == [ctypes.sizeof(T), T.unit_elems.offset, T.ctas_per_sm.offset]
    M = hc.HcMultiOut
    assert vals[22:25] == [ctypes.sizeof(M), M.d_stats.offset, M.out_dtype.offset]
    assert vals[25:28] == [H.pred.offset, H.block.offset, St.pred.offset]
    Sh = hc.HcShard
    assert vals[28:34] == [ctypes.sizeof(Sh), Sh.header_bytes.offset, Sh.src_off.offset, Sh.nbytes.offset,
                           Sh.chunks_off.offset, Sh.first.offset]
    assert vals[34:36] == [B.ncomp.offset, B.comps.offset]


def test_plain_c_program_links_and_calls_the_library(hc, orc):
    """A C11 program that includes only hc.h links libhc.so and calls its host
    entry points: version, status strings, the size queries of a stream and of
    a box stream (the same values as the oracle's layout), and a refused call
    whose message comes back through hc_last_error.  No GPU is touched."""
    src = r"""
#include <stdio.h>
#include <string.h>
#include "hc.h"
int main(void) {
  int64_t dims[3] = {20, 24, 32};
  int32_t block[3] = {4, 4, 8};
  printf("%d\n", hc_version());
  printf("%s|%s\n", hc_status_str(HC_ERR_CORRUPT), hc_status_str(HC_ERR_UNSUPPORTED));
  printf("%zu %zu\n", hc_compress_bound(1000, 32), hc_compress_bound_nd(3, dims, block));
  printf("%zu\n", hc_workspace_bytes());
  hc_header h;
  memset(&h, 0, sizeof h);
  int rc = hc_decompress_to_stage(&h, (const void*)16, HC_STAGE_Q, (void*)16, HC_F32, (void*)16,
                                  hc_workspace_bytes(), NULL);
  printf("%d %s\n", rc, hc_last_error());
  return 0;
}
"""
    lib_dir = os.path.dirname(hc.LIB_PATH)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.dirname(HC_H), c, "-o", exe,
                               "-L", lib_dir, "-lhc", "-Wl,-rpath," + lib_dir])
        lines = subprocess.check_output([exe]).decode().splitlines()
    assert int(lines[0]) == hc.lib().hc_version()
    assert lines[1] == "corrupt stream|unsupported"
    bound, bound_nd = (int(v) for v in lines[2].split())
    assert bound == orc.compress_bound(1000, 32)
    import numpy as np

    assert bound_nd == int(orc.lib().orc_compress_bound_nd(3, orc._ptr(np.array((20, 24, 32), np.int64)),
                                                           orc._ptr(np.array((4, 4, 8), np.int64))))
    assert int(lines[3]) == int(hc.lib().hc_workspace_bytes())
    rc, msg = lines[4].split(" ", 1)
    assert int(rc) == hc.HC_ERR_CORRUPT and msg == "bad ndim"


@pytest.mark.parametrize("S", [1, 2, 3, 16, 32, 33, 64, 100, 128, 4096])
def test_compress_bound_matches_oracle_layout(hc, orc, S):
    for n in (1, 7, 31, 32, 33, 1000, 4096 * 3 + 5, 10**6 + 3):
        assert int(hc.lib().hc_compress_bound(n, S)) == orc.compress_bound(n, S)


def test_status_strings_and_version(hc):
    L = hc.lib()
    assert L.hc_status_str(0) == b"ok"
    assert L.hc_status_str(3) == b"corrupt stream"
    assert L.hc_version() == 1
    assert L.hc_workspace_bytes() >= 64
    assert L.hc_compress_bound(0, 32) == 0
    assert L.hc_compress_bound(10, 0) == 0
    assert L.hc_compress_bound(10, 4097) == 0


def test_argument_errors_before_any_cuda_call(hc):
    L = hc.lib()
    dims = (ctypes.c_int64 * 3)(10, 1, 1)
    n = ctypes.c_size_t()
    # S out of range -> rejected by the layout check on the host
    rc = L.hc_compress(ctypes.c_void_p(16), 0, 1, dims, 1e-3, 1, 0, ctypes.c_void_p(16), 10**6,
                       ctypes.c_void_p(16), 10**6, ctypes.byref(n), None, None)
    assert rc == hc.HC_ERR_INVALID_ARG
    assert b"block size" in L.hc_last_error()
    # null stage
    rc = L.hc_op_mean(None, 1e-3, 1, dims, ctypes.c_void_p(16), ctypes.c_void_p(16), 10**6, None)
    assert rc == hc.HC_ERR_INVALID_ARG
    # workspace too small
    st = hc.HcStage()
    st.kind = hc.HC_STAGE_Q
    st.d_data = 16
    st.n = 10
    rc = L.hc_op_variance(ctypes.byref(st), 1e-3, 1, dims, ctypes.c_void_p(16), ctypes.c_void_p(16), 8, None)
    assert rc == hc.HC_ERR_NOMEM
    # stage-2 differentiation of a 1-D block partition is not defined (Section V-B)
    st.kind = hc.HC_STAGE_P
    st.S = 32
    rc = L.hc_op_laplacian(ctypes.byref(st), 1e-3, 1, dims, ctypes.c_void_p(16), 0, ctypes.c_void_p(16),
                           L.hc_workspace_bytes(), None)
    assert rc == hc.HC_ERR_UNSUPPORTED
    # metadata of an HSZp-style stream supports no operation
    st.kind = hc.HC_STAGE_M
    rc = L.hc_op_mean(ctypes.byref(st), 1e-3, 1, dims, ctypes.c_void_p(16), ctypes.c_void_p(16),
                      L.hc_workspace_bytes(), None)
    assert rc == hc.HC_ERR_UNSUPPORTED
    # axis out of range
    st.kind = hc.HC_STAGE_Q
    rc = L.hc_op_derivative(ctypes.byref(st), 1e-3, 1, dims, 1, ctypes.c_void_p(16), 0, ctypes.c_void_p(16),
                            L.hc_workspace_bytes(), None)
    assert rc == hc.HC_ERR_INVALID_ARG


def test_binding_fails_loudly_without_library(hc, monkeypatch, tmp_path):
    monkeypatch.setattr(hc, "_lib", None)
    monkeypatch.setattr(hc, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        hc.lib()


def test_batch_argument_errors_before_any_cuda_call(hc):
    L = hc.lib()
    assert L.hc_batch_plan_bytes(0) == 0 and L.hc_batch_workspace_bytes(0) == 0
    assert L.hc_batch_plan_bytes(4) > L.hc_batch_plan_bytes(1) > 0
    assert L.hc_batch_workspace_bytes(3) == 64 + 3 * 32
    cap = L.hc_batch_plan_bytes(1)
    buf = ctypes.create_string_buffer(cap)
    used = ctypes.c_size_t()
    items = (hc.HcBatchItem * 1)()
    # empty batch / null items
    assert L.hc_batch_plan(items, 0, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_INVALID_ARG
    assert L.hc_batch_plan(None, 1, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_INVALID_ARG
    # plan buffer too small
    assert L.hc_batch_plan(items, 1, None, buf, cap - 1, ctypes.byref(used)) == hc.HC_ERR_NOMEM
    # a zero header is inconsistent
    assert L.hc_batch_plan(items, 1, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_CORRUPT
    # a consistent header (block 32, 1-D, 100 elements) with bad ops / pointers
    h = items[0].hdr
    h.dtype, h.ndim, h.S, h.G = hc.HC_F32, 1, 32, 128
    h.dims[0], h.dims[1], h.dims[2] = 1, 1, 100
    h.eps, h.eb, h.eb_mode, h.qmax = 1e-3, 1e-3, hc.HC_EB_ABS, 10
    h.N, h.nb, h.nchunks, h.payload_words, h.wmax = 100, 4, 1, 0, 0
    h.off_widths = 256
    h.off_heads = 256 + 16
    h.off_chunks = h.off_heads + 16
    h.off_payload = h.off_chunks + 16
    h.total_bytes = h.off_payload + 16
    items[0].d_stream = 16
    items[0].ops = 0
    assert L.hc_batch_plan(items, 1, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_INVALID_ARG
    assert b"ops" in L.hc_last_error()
    items[0].ops = hc.HC_BATCH_LAPLACIAN | hc.HC_BATCH_GRADMAG
    assert L.hc_batch_plan(items, 1, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_INVALID_ARG
    items[0].ops = hc.HC_BATCH_VARIANCE  # statistics without an output pointer
    assert L.hc_batch_plan(items, 1, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_INVALID_ARG
    items[0].ops = hc.HC_BATCH_GRADMAG
    items[0].d_field = 16
    items[0].field_dtype = hc.HC_I64
    assert L.hc_batch_plan(items, 1, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_UNSUPPORTED
    items[0].ops = hc.HC_BATCH_DERIVATIVE
    items[0].axis = 1
    assert L.hc_batch_plan(items, 1, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_INVALID_ARG
    tune = hc.HcBatchTune(100, 0, 0, 0, 0)
    items[0].axis = 0
    assert L.hc_batch_plan(items, 1, ctypes.byref(tune), buf, cap, ctypes.byref(used)) == hc.HC_ERR_INVALID_ARG
    # vector items (divergence / curl): components without the operation, the
    # operation without components or with a second operation, a component
    # whose header is inconsistent, a divergence with ncomp != ndim
    items[0].ops = hc.HC_BATCH_LAPLACIAN
    items[0].ncomp = 1
    assert L.hc_batch_plan(items, 1, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_INVALID_ARG
    assert b"components" in L.hc_last_error()
    items[0].ops = hc.HC_BATCH_DIVERGENCE
    assert L.hc_batch_plan(items, 1, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_INVALID_ARG
    comps = (hc.HcStage * 2)()
    items[0].comps = ctypes.cast(comps, ctypes.c_void_p)
    items[0].ops = hc.HC_BATCH_DIVERGENCE | hc.HC_BATCH_MEAN
    assert L.hc_batch_plan(items, 1, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_INVALID_ARG
    items[0].ops = hc.HC_BATCH_DIVERGENCE
    bad = hc.HcHeader()  # all zero: inconsistent
    for k in range(2):
        comps[k].kind, comps[k].level, comps[k].d_data = hc.HC_STAGE_COMPRESSED, hc.HC_STAGE_Q, 16
        comps[k].hdr = ctypes.pointer(bad)
    assert L.hc_batch_plan(items, 1, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_CORRUPT
    for k in range(2):
        comps[k].hdr = ctypes.pointer(h)  # a 1-D field: a divergence takes 1 component
    items[0].ncomp = 2
    assert L.hc_batch_plan(items, 1, None, buf, cap, ctypes.byref(used)) == hc.HC_ERR_INVALID_ARG
    items[0].ops, items[0].ncomp, items[0].comps = hc.HC_BATCH_DERIVATIVE, 0, None
    # run / graph with something that is not a plan
    ws = ctypes.c_void_p(16)
    assert L.hc_batch_run(buf, ctypes.c_void_p(16), ws, 1 << 20, None) == hc.HC_ERR_INVALID_ARG
    g = ctypes.c_void_p()
    assert L.hc_batch_graph_create(buf, ctypes.c_void_p(16), ws, 1 << 20, ctypes.byref(g)) == hc.HC_ERR_INVALID_ARG
    assert L.hc_batch_graph_launch(None, None) == hc.HC_ERR_INVALID_ARG
    assert L.hc_batch_graph_destroy(None) == hc.HC_OK


def test_multi_argument_errors_before_any_cuda_call(hc):
    L = hc.lib()
    dims = (ctypes.c_int64 * 3)(10, 1, 1)
    st = hc.HcStage()
    st.kind = hc.HC_STAGE_Q
    st.d_data = 16
    st.n = 10
    mo = hc.HcMultiOut()
    mo.out_dtype = hc.HC_F32
    ws = ctypes.c_void_p(16)
    assert L.hc_op_multi(ctypes.byref(st), 1e-3, 1, dims, None, ws, L.hc_workspace_bytes(), None) == hc.HC_ERR_INVALID_ARG
    mo.out_dtype = hc.HC_I64
    assert L.hc_op_multi(ctypes.byref(st), 1e-3, 1, dims, ctypes.byref(mo), ws, L.hc_workspace_bytes(),
                         None) == hc.HC_ERR_INVALID_ARG
    mo.out_dtype = hc.HC_F32
    mo.d_derivative[1] = 16  # axis 1 of a 1-D field
    assert L.hc_op_multi(ctypes.byref(st), 1e-3, 1, dims, ctypes.byref(mo), ws, L.hc_workspace_bytes(),
                         None) == hc.HC_ERR_INVALID_ARG
    mo.d_derivative[1] = None
    mo.d_laplacian = 20  # unaligned
    assert L.hc_op_multi(ctypes.byref(st), 1e-3, 1, dims, ctypes.byref(mo), ws, L.hc_workspace_bytes(),
                         None) == hc.HC_ERR_INVALID_ARG


def test_vector_argument_errors_before_any_cuda_call(hc):
    L = hc.lib()
    dims = (ctypes.c_int64 * 3)(10, 12, 1)
    comps = (hc.HcStage * 2)()
    ws = ctypes.c_void_p(16)
    assert L.hc_op_divergence(None, 2, 2, dims, ctypes.c_void_p(16), hc.HC_F32, ws, L.hc_workspace_bytes(),
                              None) == hc.HC_ERR_INVALID_ARG
    assert L.hc_op_divergence(comps, 1, 2, dims, ctypes.c_void_p(16), hc.HC_F32, ws, L.hc_workspace_bytes(),
                              None) == hc.HC_ERR_INVALID_ARG
    assert L.hc_op_curl(comps, 2, 3, dims, ctypes.c_void_p(16), hc.HC_F32, ws, L.hc_workspace_bytes(),
                        None) == hc.HC_ERR_UNSUPPORTED
    # arrays instead of streams
    comps[0].kind = comps[1].kind = hc.HC_STAGE_Q
    assert L.hc_op_divergence(comps, 2, 2, dims, ctypes.c_void_p(16), hc.HC_F32, ws, L.hc_workspace_bytes(),
                              None) == hc.HC_ERR_UNSUPPORTED


@pytest.mark.parametrize("shape,block", [((7, 10), (2, 3)), ((5, 6, 7), (2, 2, 4)), ((9,), (4,)),
                                         ((13, 17, 19), (4, 4, 4)), ((3, 5, 6), (8, 8, 8))])
def test_box_compress_bound_matches_oracle_layout(hc, orc, shape, block):
    """HSZx-nd sizing: the stream bound follows the box grid exactly as the
    oracle lays it out; bad extents give 0."""
    import numpy as np

    L = hc.lib()
    d = (ctypes.c_int64 * 3)(*shape)
    b = (ctypes.c_int32 * 3)(*block)
    want = int(orc.lib().orc_compress_bound_nd(len(shape), orc._ptr(np.array(shape, np.int64)),
                                               orc._ptr(np.array(block, np.int64))))
    assert int(L.hc_compress_bound_nd(len(shape), d, b)) == want
    assert int(L.hc_compress_workspace_bytes_nd(len(shape), d, b)) > 64
    for bad in ((0,) * len(shape), (4096,) + (2,) * (len(shape) - 1)):
        if len(bad) == len(shape) and (0 in bad or np.prod(bad) > 4096):
            assert int(L.hc_compress_bound_nd(len(shape), d, (ctypes.c_int32 * 3)(*bad))) == 0


def _fake_header(hc, shape, pred, S=32, block=(0, 0, 0)):
    h = hc.HcHeader()
    h.ndim = len(shape)
    dims = (1,) * (3 - len(shape)) + tuple(shape)
    for a in range(3):
        h.dims[a] = dims[a]
        h.block[a] = block[a]
    h.N = int(dims[0] * dims[1] * dims[2])
    h.S = S
    h.pred = pred
    return h


def test_workspace_sizes_per_predictor(hc):
    """hc_workspace_bytes_for: the common size for block streams; + 4 bytes
    per element for HSZx-nd; + a rebuilt D_q (4), an int64 accumulator (8)
    and the scan totals for the global predictors (the totals vanish when no
    axis is longer than 32 and grow with a long flattened row)."""
    L = hc.lib()
    base = int(L.hc_workspace_bytes())
    r16 = lambda v: (v + 15) & ~15  # noqa: E731
    for pred in (hc.HC_PRED_DELTA, hc.HC_PRED_MEAN):
        assert int(L.hc_workspace_bytes_for(ctypes.byref(_fake_header(hc, (64, 64, 64), pred)))) == base
    hb = _fake_header(hc, (20, 33, 64), hc.HC_PRED_MEAN_ND, 64, (4, 4, 4))
    assert int(L.hc_workspace_bytes_for(ctypes.byref(hb))) == r16(base) + r16(4 * hb.N)
    small = _fake_header(hc, (8, 20, 24), hc.HC_PRED_LORENZO)
    assert int(L.hc_workspace_bytes_for(ctypes.byref(small))) == r16(base) + 12 * small.N
    big = _fake_header(hc, (256, 384, 384), hc.HC_PRED_LORENZO)
    flat = _fake_header(hc, (256, 384, 384), hc.HC_PRED_GLOBAL_DELTA)
    nb = int(L.hc_workspace_bytes_for(ctypes.byref(big)))
    nf = int(L.hc_workspace_bytes_for(ctypes.byref(flat)))
    assert r16(base) + 12 * big.N <= nb < r16(base) + 13 * big.N
    assert nf > r16(base) + 12 * flat.N  # one long row: chunk totals
    assert int(L.hc_workspace_bytes_for(None)) == 0


def test_vector_workspace_sizes(hc):
    """hc_vector_workspace_bytes: the common size when one fused kernel
    applies (block streams of one block size at stage Q), else the largest
    component workspace plus 16 bytes per element."""
    L = hc.lib()
    base = int(L.hc_workspace_bytes())
    heads = [_fake_header(hc, (8, 20, 24), hc.HC_PRED_DELTA) for _ in range(3)]
    arr = (hc.HcStage * 3)()
    for k in range(3):
        arr[k].kind = hc.HC_STAGE_COMPRESSED
        arr[k].level = hc.HC_STAGE_Q
        arr[k].hdr = ctypes.pointer(heads[k])
    assert int(L.hc_vector_workspace_bytes(arr, 3)) == base
    heads[1].pred = hc.HC_PRED_LORENZO
    arr[1].hdr = ctypes.pointer(heads[1])
    comp = int(L.hc_workspace_bytes_for(ctypes.byref(heads[1])))
    assert int(L.hc_vector_workspace_bytes(arr, 3)) == ((comp + 15) & ~15) + 16 * heads[0].N
    for k in range(3):
        arr[k].level = hc.HC_STAGE_P
    heads[1].pred = hc.HC_PRED_DELTA
    arr[1].hdr = ctypes.pointer(heads[1])
    assert int(L.hc_vector_workspace_bytes(arr, 3)) == ((base + 15) & ~15) + 16 * heads[0].N
    assert int(L.hc_vector_workspace_bytes(arr, 0)) == 0


def _header_from_oracle_stream(hc, orc, s):
    """A host hc_header filled from an oracle stream's header (the section
    offsets follow the stream layout: widths at 256, heads and the chunk
    index each on the next 16-byte boundary)."""
    g = orc.read_header(s)
    r16 = lambda v: (v + 15) & ~15  # noqa: E731
    h = hc.HcHeader()
    h.dtype, h.ndim = g["dtype"], g["ndim"]
    for a, k in enumerate(("n0", "n1", "n2")):
        h.dims[a] = g[k]
    for a, k in enumerate(("b0", "b1", "b2")):
        h.block[a] = g[k]
    h.S, h.G, h.eps, h.eb, h.eb_mode, h.qmax = g["S"], g["G"], g["eps"], g["eb"], g["eb_mode"], g["qmax"]
    h.N, h.nb, h.nchunks, h.payload_words = g["N"], g["nb"], g["nchunks"], g["payload_words"]
    h.off_widths = 256
    h.off_heads = r16(256 + g["nb"])
    h.off_chunks = r16(h.off_heads + 4 * g["nb"])
    h.off_payload, h.total_bytes, h.wmax, h.pred = g["off_payload"], g["total_bytes"], g["wmax"], g["pred"]
    assert h.off_payload == r16(h.off_chunks + 8 * (g["nchunks"] + 1))
    return h


def _copy_header(hc, h):
    c = hc.HcHeader()
    ctypes.memmove(ctypes.byref(c), ctypes.byref(h), ctypes.sizeof(h))
    return c


def test_host_header_checked_before_any_cuda_call(hc, orc, rng):
    """Every entry point that takes the caller's host copy of a header checks
    it on the host first: a header whose fields contradict one another is
    refused with HC_ERR_CORRUPT before anything reaches the GPU.  The
    unmodified header passes that check; each call with it is stopped by a
    later argument check instead (an invalid stage kind, a null output, an
    invalid level), so no kernel is launched."""
    import numpy as np

    L = hc.lib()
    p16 = ctypes.c_void_p(16)
    wsn = L.hc_workspace_bytes()
    x = rng.standard_normal((6, 10, 40)).astype(np.float32)
    s0, _ = orc.compress(x, 1e-3, True, 32)
    x2 = rng.standard_normal((12, 20)).astype(np.float32)
    s4, _ = orc.compress_nd(x2, (4, 4), 1e-3, True)

    def entries(h, base):
        # the call's own ndim, dims and eps are the valid stream's: only the header differs
        dims = (ctypes.c_int64 * 3)(*[int(v) for v in base.dims][3 - base.ndim:])
        nd, eps = base.ndim, base.eps
        st = hc.HcStage()
        st.kind, st.level, st.d_data, st.hdr = hc.HC_STAGE_COMPRESSED, hc.HC_STAGE_Q, 16, ctypes.pointer(h)
        st.n = h.N
        bad_level = hc.HcStage()
        ctypes.memmove(ctypes.byref(bad_level), ctypes.byref(st), ctypes.sizeof(st))
        bad_level.level = hc.HC_STAGE_F
        chosen = ctypes.c_int()
        return {
            "decompress": lambda: L.hc_decompress_to_stage(ctypes.byref(h), p16, 99, p16, 0, p16, wsn, None),
            "mean": lambda: L.hc_op_mean(ctypes.byref(st), eps, nd, dims, None, p16, wsn, None),
            "laplacian": lambda: L.hc_op_laplacian(ctypes.byref(st), eps, nd, dims, None, 0, p16, wsn, None),
            "multi": lambda: L.hc_op_multi(ctypes.byref(st), eps, nd, dims, None, p16, wsn, None),
            "noalloc": lambda: L.hc_op_variance_noalloc(ctypes.byref(bad_level), eps, nd, dims, p16, None),
            "autotune": lambda: L.hc_autotune(ctypes.byref(st), hc.HC_OP_LAPLACIAN, 0, None, p16, wsn, None,
                                              ctypes.byref(chosen)),
        }

    corruptions = [
        ("dtype", lambda h: setattr(h, "dtype", 2), b"bad dtype"),
        ("ndim", lambda h: setattr(h, "ndim", 0), b"bad ndim"),
        ("N", lambda h: setattr(h, "N", h.N + 1), b"section offsets"),
        ("nb", lambda h: setattr(h, "nb", h.nb + 1), b"section offsets"),
        ("off_payload", lambda h: setattr(h, "off_payload", h.off_payload + 16), b"section offsets"),
        ("total_bytes", lambda h: setattr(h, "total_bytes", h.total_bytes + 16), b"total size"),
        ("payload_words", lambda h: (setattr(h, "payload_words", h.payload_words + (1 << 30)),
                                     setattr(h, "total_bytes", h.total_bytes + (4 << 30))), b"larger than any"),
        ("wmax", lambda h: setattr(h, "wmax", 32), b"max width"),
        ("pred", lambda h: setattr(h, "pred", 5), (b"unknown predictor", b"box extents on")),
        ("eps_zero", lambda h: setattr(h, "eps", 0.0), b"bad eps"),
        ("eps_inf", lambda h: setattr(h, "eps", float("inf")), b"bad eps"),
        ("qmax", lambda h: setattr(h, "qmax", 1 << 30), b"max |q|"),
    ]
    h0 = _header_from_oracle_stream(hc, orc, s0)
    h4 = _header_from_oracle_stream(hc, orc, s4)
    assert (h0.pred, h4.pred, tuple(h4.block), tuple(h0.block)) == (0, 4, (1, 4, 4), (0, 0, 0))
    after_check = {"decompress": b"kind must be", "mean": b"null output", "laplacian": b"output must be",
                   "multi": b"null output set", "noalloc": b"fused level", "autotune": b"16-byte aligned"}
    for h in (h0, h4):
        for name, call in entries(h, h).items():
            assert call() == hc.HC_ERR_INVALID_ARG, name
            assert after_check[name] in L.hc_last_error(), (name, L.hc_last_error())
    box_corruptions = [
        ("block_on_delta", h0, lambda h: setattr(h, "block", (ctypes.c_uint32 * 3)(0, 0, 4)), b"box extents on"),
        ("box_product", h4, lambda h: setattr(h, "block", (ctypes.c_uint32 * 3)(1, 4, 8)), b"box extents and S"),
        ("box_leading", h4, lambda h: setattr(h, "block", (ctypes.c_uint32 * 3)(2, 4, 2)), b"leading box"),
        ("leading_dim", h4, lambda h: h.dims.__setitem__(0, 2), b"leading dims"),
    ]
    cases = [(n, base, f, m) for base in (h0, h4) for n, f, m in corruptions] + box_corruptions
    for name, base, corrupt, msg in cases:
        h = _copy_header(hc, base)
        corrupt(h)
        for entry, call in entries(h, base).items():
            rc = call()
            assert rc == hc.HC_ERR_CORRUPT, (name, entry, rc, L.hc_last_error())
            msgs = msg if isinstance(msg, tuple) else (msg,)
            assert any(m in L.hc_last_error() for m in msgs), (name, entry, L.hc_last_error())


def test_workspace_size_of_real_and_invalid_headers(hc, orc, rng):
    """hc_workspace_bytes_for on the headers of real streams of every
    predictor (1-D, 2-D and 3-D fields, ragged boxes) gives the documented
    size; a header whose ndim, extents, N, box extents or predictor are
    invalid gives 0, and so does a vector of components holding one."""
    import numpy as np

    L = hc.lib()
    base = int(L.hc_workspace_bytes())
    r16 = lambda v: (v + 15) & ~15  # noqa: E731
    for shape in ((300,), (17, 23), (5, 9, 40)):
        x = rng.standard_normal(shape).astype(np.float32)
        for pred in (0, 1, 2, 3):
            s, _ = orc.compress(x, 1e-3, True, 16, pred=pred)
            h = _header_from_oracle_stream(hc, orc, s)
            got = int(L.hc_workspace_bytes_for(ctypes.byref(h)))
            if pred < 2:
                assert got == base
            else:
                assert r16(base) + 12 * h.N <= got < r16(base) + 13 * h.N + 4096, (shape, pred)
        block = (7,) * len(shape) if len(shape) < 3 else (2, 3, 8)
        s4, _ = orc.compress_nd(x, block, 1e-3, True)
        h4 = _header_from_oracle_stream(hc, orc, s4)
        assert int(L.hc_workspace_bytes_for(ctypes.byref(h4))) == r16(base) + r16(4 * h4.N)
    s, _ = orc.compress(rng.standard_normal((6, 8, 10)).astype(np.float32), 1e-3, True, 32, pred=2)
    good = _header_from_oracle_stream(hc, orc, s)
    s4, _ = orc.compress_nd(rng.standard_normal((6, 8, 10)).astype(np.float32), (2, 2, 4), 1e-3, True)
    good4 = _header_from_oracle_stream(hc, orc, s4)
    bad = [
        (good, lambda h: setattr(h, "ndim", 0)),
        (good, lambda h: setattr(h, "ndim", 4)),
        (good, lambda h: h.dims.__setitem__(1, 0)),
        (good, lambda h: h.dims.__setitem__(2, -8)),
        (good, lambda h: setattr(h, "N", h.N + 1)),
        (good, lambda h: setattr(h, "pred", 5)),
        (good, lambda h: (h.dims.__setitem__(0, 1 << 20), h.dims.__setitem__(1, 1 << 20),
                          setattr(h, "N", (1 << 40) * h.dims[2]))),
        (good4, lambda h: h.block.__setitem__(2, 0)),
    ]
    for base_h, corrupt in bad:
        h = _copy_header(hc, base_h)
        corrupt(h)
        assert int(L.hc_workspace_bytes_for(ctypes.byref(h))) == 0
        st = hc.HcStage()
        st.kind, st.level, st.d_data, st.hdr = hc.HC_STAGE_COMPRESSED, hc.HC_STAGE_Q, 16, ctypes.pointer(h)
        assert int(L.hc_vector_workspace_bytes(ctypes.byref(st), 1)) == 0
    st = hc.HcStage()
    st.kind, st.level, st.d_data, st.hdr = hc.HC_STAGE_COMPRESSED, hc.HC_STAGE_Q, 16, ctypes.pointer(good)
    assert int(L.hc_vector_workspace_bytes(ctypes.byref(st), 1)) >= int(L.hc_workspace_bytes_for(ctypes.byref(good)))


def test_empty_and_oversized_fields_refused_on_the_host(hc):
    """An empty field (an axis of length 0), a negative extent, more than
    2^40 elements, or an empty or oversized box is refused with
    HC_ERR_INVALID_ARG before any device memory is touched, by compression,
    box compression, the size queries and an operation on a stage array."""
    L = hc.lib()
    p16 = ctypes.c_void_p(16)
    n = ctypes.c_size_t()
    big = 1 << 21
    for nd, dims, msg in ((1, (0,), b"every dimension"), (2, (7, 0), b"every dimension"),
                          (3, (4, -2, 9), b"every dimension"), (3, (big, big, 2), b"too large")):
        d = (ctypes.c_int64 * 3)(*dims, *([1] * (3 - len(dims))))
        rc = L.hc_compress(p16, 0, nd, d, 1e-3, 1, 32, p16, 1 << 30, p16, 1 << 30, ctypes.byref(n), None, None)
        assert rc == hc.HC_ERR_INVALID_ARG and msg in L.hc_last_error(), dims
        rc = L.hc_compress_codes_ex(p16, 0, nd, d, 0.5, 1e-3, 0, 32, 0, p16, 1 << 30, p16, 1 << 30,
                                    ctypes.byref(n), None, None)
        assert rc == hc.HC_ERR_INVALID_ARG and msg in L.hc_last_error(), dims
        blk = (ctypes.c_int32 * 3)(4, 4, 4)
        rc = L.hc_compress_nd(p16, 0, nd, d, blk, 1e-3, 1, p16, 1 << 30, p16, 1 << 30, ctypes.byref(n), None, None)
        assert rc == hc.HC_ERR_INVALID_ARG and msg in L.hc_last_error(), dims
        assert int(L.hc_compress_bound_nd(nd, d, blk)) == 0
        st = hc.HcStage()
        st.kind, st.d_data, st.n = hc.HC_STAGE_Q, 16, 0
        rc = L.hc_op_mean(ctypes.byref(st), 1e-3, nd, d, p16, p16, L.hc_workspace_bytes(), None)
        assert rc == hc.HC_ERR_INVALID_ARG and msg in L.hc_last_error(), dims
    d = (ctypes.c_int64 * 3)(8, 8, 8)
    for blk, msg in (((0, 4, 4), b"box extents"), ((16, 16, 32), b"box size")):
        rc = L.hc_compress_nd(p16, 0, 3, d, (ctypes.c_int32 * 3)(*blk), 1e-3, 1, p16, 1 << 30, p16, 1 << 30,
                              ctypes.byref(n), None, None)
        assert rc == hc.HC_ERR_INVALID_ARG and msg in L.hc_last_error(), blk
    assert int(L.hc_compress_bound(0, 32)) == 0 and int(L.hc_compress_bound(-5, 32)) == 0
    assert int(L.hc_compress_bound(1 << 41, 32)) == 0


def test_host_header_reader_and_save_load(hc, orc, rng, tmp_path):
    """hc_read_header_host (the parser hc_read_header shares) reads every
    predictor's stream header as the oracle writes it, refuses corrupt and
    truncated images, and save / load round-trip a stream through a file
    (here on CPU tensors: the file format is the stream itself)."""
    import numpy as np
    import torch

    x = rng.standard_normal((9, 20, 48)).astype(np.float32)
    streams = [orc.compress(x, 1e-3, True, 32, pred=p)[0] for p in (0, 1, 2, 3)]
    streams.append(orc.compress_nd(x, (3, 4, 8), 1e-3, True)[0])
    streams.append(orc.compress(x.astype(np.float64).reshape(-1), 1e-4, False, 100)[0])
    for s in streams:
        want = _header_from_oracle_stream(hc, orc, s)
        got = hc.header_of(s)
        for name, _ in hc.HcHeader._fields_:
            a, b = getattr(got, name), getattr(want, name)
            if hasattr(a, "_length_"):
                a, b = list(a), list(b)
            assert a == b, name
        assert hc.header_of(bytes(s)).total_bytes == s.size
        assert hc.header_of(memoryview(bytearray(s))).total_bytes == s.size
        padded = np.concatenate([s, np.zeros((-s.size) % 8, np.uint8)])
        assert bytes(hc.header_of(padded.view(np.uint64))) == bytes(got)  # raw bytes, not converted values
        for bad, why in ((s[:255], "shorter than its header"), (s[:-16], "truncated")):
            with pytest.raises(hc.HcError) as e:
                hc.header_of(bad)
            assert e.value.status == hc.HC_ERR_CORRUPT and why in str(e.value)
        for off in (0, 72, 128):  # magic, nb, total size
            bad = s.copy()
            bad[off] ^= 0x01
            with pytest.raises(hc.HcError) as e:
                hc.header_of(bad)
            assert e.value.status == hc.HC_ERR_CORRUPT
        c = hc.Compressed(torch.from_numpy(np.concatenate([s, np.zeros(48, np.uint8)])), got, int(s.size))
        path = str(tmp_path / "field.hcz")
        assert hc.save(c, path) == s.size
        assert open(path, "rb").read() == s.tobytes()
        back = hc.load(path, device="cpu")
        assert back.nbytes == s.size and np.array_equal(back.stream.numpy(), s)
        assert bytes(back.header) == bytes(got)
    # a shard's header image is a stream header the library itself accepts
    s = streams[0]
    h = hc.header_of(s)
    r16 = lambda v: (v + 15) & ~15  # noqa: E731
    off = r16(r16(256 + h.nb) + 4 * h.nb)
    chunks = np.frombuffer(s[off:off + 8 * (h.nchunks + 1)].tobytes(), np.uint64)
    plan, _ = hc.shard_plan(h, chunks, 0, int(h.nchunks))
    img = np.zeros(int(plan.hdr.total_bytes), np.uint8)
    img[:256] = np.frombuffer(bytes(plan.header_bytes), np.uint8)
    assert bytes(hc.header_of(img)) == bytes(plan.hdr)


def test_finalize_on_the_host_matches_the_oracle(hc, orc):
    """hc_finalize (host code, no device access) applies Eq. var_q's final
    scaling to exact sums: bit-equal to the oracle's finish for s2 below and
    above 2^64, NaN variance for N = 1, the sums copied through; null output,
    N < 1 and a non-positive or non-finite eps are refused."""
    import math

    import numpy as np

    rng = np.random.default_rng(2026)
    cases = [(1, 7, 49, 0.25), (2, -3, 5, 1e-3), (8, 18, 740, 0.1)]
    for _ in range(40):
        k = int(rng.integers(2, 64))
        q = [int(v) for v in rng.integers(-(1 << 29), 1 << 29, size=k)]
        rep = int(rng.choice([1, 1 << 10, 1 << 20]))
        cases.append((k * rep, sum(q) * rep, sum(v * v for v in q) * rep, float(rng.choice([1e-6, 3.3e-3, 17.0]))))
    saw_wide = False
    for n, s1, s2, eps in cases:
        r = hc.finalize(n, s1, s2, eps)
        m, v, sd = orc.finalize(n, s1, s2, eps)
        assert r["n"] == n and r["s1"] == s1 and r["s2"] == s2 and r["exact"] == 1 and r["status"] == 0
        assert r["mean"] == m
        if n < 2:
            assert math.isnan(r["variance"]) and math.isnan(r["std"])
        else:
            assert r["variance"] == v and r["std"] == sd
        saw_wide |= s2 >= (1 << 64)
    assert saw_wide
    L = hc.lib()
    buf = ctypes.create_string_buffer(hc.SCALAR_BYTES)
    out = ctypes.cast(buf, ctypes.c_void_p)
    assert L.hc_finalize(4, 1, 1, 0, 1e-3, None) == hc.HC_ERR_INVALID_ARG
    assert L.hc_finalize(0, 1, 1, 0, 1e-3, out) == hc.HC_ERR_INVALID_ARG
    for eps in (0.0, -1.0, float("inf"), float("nan")):
        assert L.hc_finalize(4, 1, 1, 0, eps, out) == hc.HC_ERR_INVALID_ARG
