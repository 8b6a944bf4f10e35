// hc_launch.h -- host-side declarations shared by the translation units of
// libhc.so (argument checking, layout arithmetic, launch helpers and the
// per-file entry points the C ABI dispatches to).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/hc.h"

namespace hc {

// Geometry of a stream for a given shape and block size.
struct Layout {
  int64_t dims[3];  // padded to 3 axes with leading ones
  int64_t N, nb, nchunks;
  int S, G;
  int64_t off_widths, off_heads, off_chunks, off_payload;
  size_t bound;  // stream bytes with every block at width 31
  int64_t bd[3];  // HSZx-nd box extents (leading ones); 0 for 1-D blocks
};

// Record a failure message (thread-local) and return `code`.
int fail(int code, const char* msg);
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int make_layout(int ndim, const int64_t* dims, int S, Layout* L);
// Layout of an HSZx-nd stream: boxes of block[0..ndim) codes, S their product,
// nb the box grid.
int make_layout_nd(int ndim, const int64_t* dims, const int32_t* block, Layout* L);
size_t compress_ws_bytes(const Layout& L);

int device_sms();
int check_launch(const char* what);
// Like check_launch, with the launch configuration in the error message.
int check_launch_cfg(const char* what, const void* kernel, long long grid, int smem);
// Raise a kernel's dynamic shared-memory limit to at least `bytes` (never lowers it).
int ensure_smem(const void* kernel, int bytes);

// Consistency checks of a header (no device access).
int check_header(const hc_header& h);
int read_header_impl(const void* d_stream, size_t bytes, hc_header* out, cudaStream_t st);

// block: the box extents of an HSZx-nd stream (pred HC_PRED_MEAN_ND), else NULL
int compress_impl(const void* d_x, int src_kind, int dtype, int ndim, const int64_t* dims, double eb,
                  double eps_given, int eb_mode, int S, int pred, const int32_t* block, void* d_stream, size_t cap,
                  void* d_ws, size_t ws_bytes, size_t* out_bytes, hc_header* hdr_out, cudaStream_t st);

// Workspace of decompression and operations: a status word, the
// last-block ticket of the reductions and the per-CTA partial results.
struct Partial {
  long long s1;
  unsigned long long s2_lo, s2_hi;
  int err;
  int pad;
};
struct OpWs {
  int status;
  unsigned int ticket;
  int pad[14];  // pad[0..1]: the integer mean of a stage-2 HSZx deviation (8-byte aligned)
};
constexpr int kMaxGrid = 4096;
constexpr size_t kOpWsBytes = sizeof(OpWs) + sizeof(Partial) * kMaxGrid;

inline Partial* ws_partials(void* d_ws) {
  return reinterpret_cast<Partial*>(reinterpret_cast<char*>(d_ws) + sizeof(OpWs));
}

// Per-file entry points (inputs already validated by the ABI layer).
int decode_impl(const hc_header* h, const void* d_stream, int kind, void* d_out, int out_dtype, void* d_ws,
                cudaStream_t st);
// The residuals D_p of every slot (block-mean and global-predictor streams),
// int32[N] into d_out (hc_decode.cu).
int decode_residuals_impl(const hc_header* h, const void* d_stream, void* d_out, void* d_ws, cudaStream_t st);
// Stage 1: a copy of the heads section (hc_decode.cu).
int decode_heads_impl(const hc_header* h, const void* d_stream, void* d_out, cudaStream_t st);

// Global-predictor streams (hc_global.cu): workspace they need (any call),
// decompression, statistics and stencils at a level.
size_t global_workspace_bytes(const hc_header* h);
int global_decode_impl(const hc_header* h, const void* d_stream, int kind, void* d_out, int out_dtype, void* d_ws,
                       size_t ws_bytes, cudaStream_t st);
int global_stats_impl(const hc_header* h, const void* d_stream, int level, int what, hc_scalar* d_out, void* d_ws,
                      size_t ws_bytes, cudaStream_t st);
int global_stencil_impl(const hc_header* h, const void* d_stream, int level, int op, int axis3, void* d_out,
                        int out_dtype, void* d_ws, size_t ws_bytes, cudaStream_t st);

// HSZx-nd streams (hc_xnd.cu): the same four entry points.
size_t xnd_workspace_bytes(const hc_header* h);
int xnd_decode_impl(const hc_header* h, const void* d_stream, int kind, void* d_out, int out_dtype, void* d_ws,
                    size_t ws_bytes, cudaStream_t st);
int xnd_stats_impl(const hc_header* h, const void* d_stream, int level, int what, hc_scalar* d_out, void* d_ws,
                   size_t ws_bytes, cudaStream_t st);
int xnd_stencil_impl(const hc_header* h, const void* d_stream, int level, int op, int axis3, void* d_out,
                     int out_dtype, void* d_ws, size_t ws_bytes, cudaStream_t st);
// One-pass HSZx-nd stencils at stage 2 or 3 (hc_xnd_march.cu): d_scratch
// holds the box offsets (4 nb bytes).  HC_ERR_UNSUPPORTED (nothing recorded)
// when the tile plan does not apply.
int xnd_march_impl(const hc_header* h, const void* d_stream, int level, int op, int axis3, void* d_out, int out_dtype,
                   void* d_ws, void* d_scratch, size_t scratch_bytes, cudaStream_t st);

enum ReduceWhat { RED_MEAN = 0, RED_VAR = 1 };
int reduce_stream_impl(const hc_header* h, const void* d_stream, int level, int what, hc_scalar* d_out,
                       void* d_ws, cudaStream_t st);
int reduce_array_impl(const hc_stage* in, double eps, int what, hc_scalar* d_out, void* d_ws, cudaStream_t st);
// Stage-1 mean of HSZx from a block-means array (Eq. mean_m).
int mean_m_array_impl(const int32_t* means, int64_t nb, int S, int64_t n, double eps, hc_scalar* d_out, void* d_ws,
                      cudaStream_t st);
// Fused statistics of block-size-32 streams (block heads or block means,
// widths <= 16, |q| < 2^26; hc_reduce32.cu): warp-autonomous chunks with bulk
// copies.  reduce32_applies says whether a stream qualifies; max_parts bounds
// the grid (partial slots); shift: the stage-2 HSZx deviation's integer mean.
bool reduce32_applies(const hc_header* h);
// The same kernel on HSZx-nd streams of 64- or 128-slot boxes (widths <= 16,
// |q| < 2^26): the mean (what RED_MEAN) and the sums about `shift` (NULL:
// the exact stage-3 variance).
bool reduce32_box_applies(const hc_header* h);
// The stage-2 mean of a global-predictor stream (HSZp-nd with rows of at
// least 32 codes, HSZp) of block size 32, widths <= 16 and N below
// 2^32 - 256, on the same kernel.
bool reduce32_global_mean_applies(const hc_header* h);
int reduce32_global_mean_impl(const hc_header* h, const void* d_stream, hc_scalar* d_out, Partial* parts,
                              unsigned* ticket, int max_parts, cudaStream_t st);
int reduce32_box_impl(const hc_header* h, const void* d_stream, int what, hc_scalar* d_out, Partial* parts,
                      unsigned* ticket, int max_parts, const long long* shift, cudaStream_t st);
int reduce32_impl(const hc_header* h, const void* d_stream, int level, int what, hc_scalar* d_out, Partial* parts,
                  unsigned* ticket, int max_parts, const long long* shift, cudaStream_t st);
// Fused stage-3 variance with its scratch (per-CTA partials + ticket) at given device addresses.
int variance_stream_scratch_impl(const hc_header* h, const void* d_stream, hc_scalar* d_out, Partial* parts,
                                 unsigned* ticket, int max_parts, cudaStream_t st);

enum StencilOp { ST_DERIV = 0, ST_GRADMAG = 1, ST_LAPLACIAN = 2, ST_MULTI = 3 };
int stencil_stream_impl(const hc_header* h, const void* d_stream, int op, int axis3, void* d_out, int out_dtype,
                        void* d_ws, cudaStream_t st);
// Pipelined fused stencil (block size 32, rows of a multiple of 8, |q| < 2^15);
// HC_ERR_UNSUPPORTED when it does not apply.  d3 is the (possibly remapped) shape.
int stencil_pipe_impl(const hc_header* h, const void* d_stream, const int64_t* d3, int op, int axis3, void* d_out,
                      int out_dtype, void* d_ws, cudaStream_t st);
// All operations of one field in one pass (pipelined tile, ST_MULTI):
// outputs by internal axis, NULL where not wanted; d_stats (exact stage-3
// statistics) or NULL.  HC_ERR_UNSUPPORTED when the pipelined tile does not
// apply (nothing recorded).
int stencil_multi_impl(const hc_header* h, const void* d_stream, void* const deriv3[3], void* d_grad, void* d_lap,
                       hc_scalar* d_stats, int out_dtype, void* d_ws, cudaStream_t st);
// Divergence (op 0) or 2-D curl (op 1) of nc component streams (hc_vector.cu).
int vector_stream_impl(const hc_header* const* hs, const void* const* streams, int nc, int op, void* d_out,
                       int out_dtype, void* d_ws, cudaStream_t st);
// The same on streams of any predictor and at stage 2 or 3, component by
// component (each component's own derivative path, exact integer sums).
size_t vector_any_workspace_bytes(const hc_header* const* hs, int nc);
int vector_any_impl(const hc_header* const* hs, const void* const* streams, int nc, int op, int level, void* d_out,
                    int out_dtype, void* d_ws, size_t ws_bytes, cudaStream_t st);
// Shape the fused stencils walk: a 2-D field (1, n1, n2) is walked as (n1, 1, n2).
void stencil_walk_dims(const hc_header* h, int64_t d3[3], int* axis3);
// Time the pipelined kernel's tile heights for this field/op and cache the best.
int stencil_pipe_autotune(const hc_header* h, const void* d_stream, const int64_t* d3, int op, void* d_out,
                          int out_dtype, void* d_ws, cudaStream_t st, int* chosen);
// The tuner's choices as JSON text (hc_autotune_export / hc_autotune_import).
int autotune_export_impl(char* buf, size_t cap, size_t* len);
int autotune_import_impl(const char* text, int* count);
int stencil_array_impl(const hc_stage* in, const int64_t* dims3, double eps, int op, int axis3, void* d_out,
                       int out_dtype, void* d_ws, cudaStream_t st);

// Batched fused launch (hc_batch.cu).
int64_t batch_plan_bytes(int n);
int64_t batch_ws_bytes(int n);
int batch_plan_impl(const hc_batch_item* items, int n, const hc_batch_tune* tune, void* h_plan, size_t cap,
                    size_t* used);
int batch_run_impl(const void* h_plan, const void* d_plan, void* d_ws, size_t ws_bytes, cudaStream_t st);
int batch_graph_impl(const void* h_plan, const void* d_plan, void* d_ws, size_t ws_bytes, void** out);
int batch_graph_launch_impl(void* graph, cudaStream_t st);
int batch_graph_destroy_impl(void* graph);
int batch_status_impl(void* d_ws, cudaStream_t st);

}  // namespace hc
