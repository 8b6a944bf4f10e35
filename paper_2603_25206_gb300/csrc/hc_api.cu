// hc_api.cu -- the extern "C" entry points of libhc.so (declared in
// include/hc.h): argument checking, header parsing, dispatch to the kernels.
// Nothing here allocates device memory.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <map>
#include <utility>

#include "hc_internal.cuh"
#include "hc_launch.h"

namespace hc {

static thread_local char g_last_error[512] = "";

int fail(int code, const char* msg) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg ? msg : "");
  return code;
}

static int64_t align16(int64_t x) { return (x + 15) & ~(int64_t)15; }

int make_layout(int ndim, const int64_t* dims, int S, Layout* L) {
  if (ndim < 1 || ndim > 3 || !dims) return fail(HC_ERR_INVALID_ARG, "ndim must be 1..3 with dims given");
  if (S < 1 || S > kMaxS) return fail(HC_ERR_INVALID_ARG, "block size S must be in 1..4096");
  L->dims[0] = L->dims[1] = L->dims[2] = 1;
  int64_t n = 1;
  for (int a = 0; a < ndim; ++a) {
    if (dims[a] < 1) return fail(HC_ERR_INVALID_ARG, "every dimension must be >= 1");
    if (n > ((int64_t)1 << 40) / dims[a]) return fail(HC_ERR_INVALID_ARG, "field too large");
    n *= dims[a];
    L->dims[3 - ndim + a] = dims[a];
  }
  L->N = n;
  L->S = S;
  L->bd[0] = L->bd[1] = L->bd[2] = 0;
  L->nb = (n + S - 1) / S;
  L->G = std::max(1, kChunkElems / S);
  L->nchunks = (L->nb + L->G - 1) / L->G;
  L->off_widths = kHeaderBytes;
  L->off_heads = align16(L->off_widths + L->nb);
  L->off_chunks = align16(L->off_heads + 4 * L->nb);
  L->off_payload = align16(L->off_chunks + 8 * (L->nchunks + 1));
  const int64_t nseg = (S + 31) / 32;
  const int64_t wmax_words = nseg + ((int64_t)S * 31 + 31) / 32;
  L->bound = (size_t)align16(L->off_payload + 4 * L->nb * wmax_words + 16);
  return HC_OK;
}

int make_layout_nd(int ndim, const int64_t* dims, const int32_t* block, Layout* L) {
  if (ndim < 1 || ndim > 3 || !dims || !block) return fail(HC_ERR_INVALID_ARG, "ndim must be 1..3 with dims and block");
  int64_t S = 1;
  for (int a = 0; a < ndim; ++a) {
    if (block[a] < 1 || block[a] > kMaxS) return fail(HC_ERR_INVALID_ARG, "box extents must be >= 1");
    S *= block[a];
    if (S > kMaxS) return fail(HC_ERR_INVALID_ARG, "box size (product of the extents) must be <= 4096");
  }
  int rc = make_layout(ndim, dims, (int)S, L);
  if (rc) return rc;
  int64_t nb = 1;
  for (int a = 0; a < 3; ++a) {
    L->bd[a] = a < 3 - ndim ? 1 : block[a - (3 - ndim)];
    nb *= (L->dims[a] + L->bd[a] - 1) / L->bd[a];
  }
  L->nb = nb;
  L->nchunks = (L->nb + L->G - 1) / L->G;
  L->off_heads = align16(L->off_widths + L->nb);
  L->off_chunks = align16(L->off_heads + 4 * L->nb);
  L->off_payload = align16(L->off_chunks + 8 * (L->nchunks + 1));
  const int64_t nseg = (S + 31) / 32;
  const int64_t wmax_words = nseg + (S * 31 + 31) / 32;
  L->bound = (size_t)align16(L->off_payload + 4 * L->nb * wmax_words + 16);
  return HC_OK;
}

size_t compress_ws_bytes(const Layout& L) { return 64 + 8 * (size_t)(L.nchunks + 1); }

int device_sms() {
  static int sms[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (!sms[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = v > 0 ? v : 148;
  }
  return sms[dev];
}

int check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char buf[400];
    std::snprintf(buf, sizeof(buf), "%s: kernel launch failed: %s", what, cudaGetErrorString(e));
    return fail(HC_ERR_CUDA, buf);
  }
  return HC_OK;
}

int check_launch_cfg(const char* what, const void* kernel, long long grid, int smem) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFuncAttributes fa;
    std::memset(&fa, 0, sizeof fa);
    cudaFuncGetAttributes(&fa, kernel);
    cudaGetLastError();
    char buf[480];
    std::snprintf(buf, sizeof(buf),
                  "%s: kernel launch failed: %s (grid %lld, block %d, dynamic smem %d, static smem %zu, "
                  "max dynamic smem %d, regs %d)",
                  what, cudaGetErrorString(e), grid, kThreads, smem, fa.sharedSizeBytes,
                  fa.maxDynamicSharedSizeBytes, fa.numRegs);
    return fail(HC_ERR_CUDA, buf);
  }
  return HC_OK;
}

int ensure_smem(const void* kernel, int bytes) {
  // Per (kernel, device): the largest dynamic shared-memory size set so far.
  // The limit is only ever raised, so launches of the same kernel with
  // smaller tiles stay valid.
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> limit;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(kernel, dev);
  auto it = limit.find(key);
  if (it != limit.end() && it->second >= bytes) return HC_OK;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return fail(HC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  if ((size_t)bytes + fa.sharedSizeBytes > (size_t)optin)
    return fail(HC_ERR_UNSUPPORTED, "kernel needs more shared memory than the device offers");
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
    return fail(HC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  limit[key] = bytes;
  return HC_OK;
}

static uint64_t le(const uint8_t* b, int off, int n) {
  uint64_t v = 0;
  for (int i = 0; i < n; ++i) v |= (uint64_t)b[off + i] << (8 * i);
  return v;
}

// Consistency of a header's fields with one another (the checks that need no
// device access).
int check_header(const hc_header& h) {
  if (h.dtype != HC_F32 && h.dtype != HC_F64) return fail(HC_ERR_CORRUPT, "bad dtype");
  if (h.ndim < 1 || h.ndim > 3) return fail(HC_ERR_CORRUPT, "bad ndim");
  for (int a = 0; a < 3 - h.ndim; ++a)
    if (h.dims[a] != 1) return fail(HC_ERR_CORRUPT, "leading dims must be 1");
  Layout L;
  int64_t d[3];
  for (int a = 0; a < h.ndim; ++a) d[a] = h.dims[3 - h.ndim + a];
  if (h.pred == HC_PRED_MEAN_ND) {
    int32_t bl[3];
    for (int a = 0; a < 3 - h.ndim; ++a)
      if (h.block[a] != 1) return fail(HC_ERR_CORRUPT, "leading box extents must be 1");
    for (int a = 0; a < h.ndim; ++a) bl[a] = (int32_t)h.block[3 - h.ndim + a];
    if ((int64_t)h.block[0] * h.block[1] * h.block[2] != h.S) return fail(HC_ERR_CORRUPT, "box extents and S disagree");
    if (make_layout_nd(h.ndim, d, bl, &L) != HC_OK) return fail(HC_ERR_CORRUPT, "bad shape or box extents");
  } else {
    if (h.block[0] || h.block[1] || h.block[2]) return fail(HC_ERR_CORRUPT, "box extents on a 1-D block stream");
    if (make_layout(h.ndim, d, h.S, &L) != HC_OK) return fail(HC_ERR_CORRUPT, "bad shape or block size");
  }
  if (L.N != h.N || L.nb != h.nb || L.G != h.G || L.nchunks != h.nchunks || L.off_widths != h.off_widths ||
      L.off_heads != h.off_heads || L.off_chunks != h.off_chunks || L.off_payload != h.off_payload)
    return fail(HC_ERR_CORRUPT, "section offsets do not follow from the shape");
  if (h.payload_words < 0 || h.total_bytes != align16(h.off_payload + 4 * h.payload_words + 16))
    return fail(HC_ERR_CORRUPT, "payload size and total size disagree");
  if ((size_t)h.total_bytes > L.bound) return fail(HC_ERR_CORRUPT, "payload larger than any valid stream");
  if (h.wmax > 31) return fail(HC_ERR_CORRUPT, "max width above 31");
  if (h.pred > HC_PRED_MEAN_ND) return fail(HC_ERR_CORRUPT, "unknown predictor");
  if (!(h.eps > 0.0) || !std::isfinite(h.eps)) return fail(HC_ERR_CORRUPT, "bad eps");
  if (h.qmax >= (1u << 30)) return fail(HC_ERR_CORRUPT, "max |q| out of range");
  return HC_OK;
}

// The header image b (kHeaderBytes bytes, host memory) of a stream of `bytes`
// bytes: parsed field by field, checked, and refused if the stream is shorter
// than the header says.
static int parse_header_image(const uint8_t* b, size_t bytes, hc_header* out) {
  if (le(b, 0, 4) != kMagic || le(b, 4, 2) != (uint64_t)kVersion) return fail(HC_ERR_CORRUPT, "bad magic or version");
  hc_header h;
  std::memset(&h, 0, sizeof h);
  h.dtype = (int32_t)le(b, 6, 1);
  h.ndim = (int32_t)le(b, 7, 1);
  for (int a = 0; a < 3; ++a) h.dims[a] = (int64_t)le(b, 8 + 8 * a, 8);
  h.S = (int32_t)le(b, 32, 4);
  h.G = (int32_t)le(b, 36, 4);
  const uint64_t eps_bits = le(b, 40, 8), eb_bits = le(b, 48, 8);
  std::memcpy(&h.eps, &eps_bits, 8);
  std::memcpy(&h.eb, &eb_bits, 8);
  h.eb_mode = (int32_t)le(b, 56, 4);
  h.qmax = (uint32_t)le(b, 60, 4);
  h.N = (int64_t)le(b, 64, 8);
  h.nb = (int64_t)le(b, 72, 8);
  h.nchunks = (int64_t)le(b, 80, 8);
  h.payload_words = (int64_t)le(b, 88, 8);
  h.off_widths = (int64_t)le(b, 96, 8);
  h.off_heads = (int64_t)le(b, 104, 8);
  h.off_chunks = (int64_t)le(b, 112, 8);
  h.off_payload = (int64_t)le(b, 120, 8);
  h.total_bytes = (int64_t)le(b, 128, 8);
  h.wmax = (uint32_t)le(b, 136, 4);
  h.pred = (uint32_t)le(b, 140, 4);
  for (int a = 0; a < 3; ++a) h.block[a] = (uint32_t)le(b, 144 + 4 * a, 4);
  int rc = check_header(h);
  if (rc) return rc;
  if ((size_t)h.total_bytes > bytes) return fail(HC_ERR_CORRUPT, "stream truncated");
  *out = h;
  return HC_OK;
}

int read_header_impl(const void* d_stream, size_t bytes, hc_header* out, cudaStream_t st) {
  if (!d_stream || !out) return fail(HC_ERR_INVALID_ARG, "null pointer");
  if (bytes < (size_t)kHeaderBytes) return fail(HC_ERR_CORRUPT, "stream shorter than its header");
  uint8_t b[kHeaderBytes];
  if (cudaMemcpyAsync(b, d_stream, kHeaderBytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(HC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  return parse_header_image(b, bytes, out);
}

static int read_header_host_impl(const void* h_stream, size_t bytes, hc_header* out) {
  if (!h_stream || !out) return fail(HC_ERR_INVALID_ARG, "null pointer");
  if (bytes < (size_t)kHeaderBytes) return fail(HC_ERR_CORRUPT, "stream shorter than its header");
  return parse_header_image(reinterpret_cast<const uint8_t*>(h_stream), bytes, out);
}

}  // namespace hc

using namespace hc;

static cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Checks shared by every operation: workspace, shape and the stage view.
static int check_op(const hc_stage* in, double eps, int ndim, const int64_t* dims, void* d_ws, size_t ws_bytes,
                    int64_t dims3[3]) {
  if (!in || !in->d_data) return fail(HC_ERR_INVALID_ARG, "null stage");
  if (!d_ws || ws_bytes < kOpWsBytes) return fail(HC_ERR_NOMEM, "workspace smaller than hc_workspace_bytes()");
  if (!aligned16(d_ws) || !aligned16(in->d_data)) return fail(HC_ERR_INVALID_ARG, "device buffers must be 16-byte aligned");
  Layout L;
  int rc = make_layout(ndim, dims, 1, &L);
  if (rc) return rc;
  for (int a = 0; a < 3; ++a) dims3[a] = L.dims[a];
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(HC_ERR_INVALID_ARG, "eps must be positive");
  if (in->kind == HC_STAGE_COMPRESSED) {
    const hc_header* h = in->hdr;
    if (!h) return fail(HC_ERR_INVALID_ARG, "a stream input needs its header (hc_read_header)");
    rc = check_header(*h);  // the caller's host copy: its sections must follow from its shape
    if (rc) return rc;
    if (h->ndim != ndim || h->eps != eps) return fail(HC_ERR_INVALID_ARG, "eps / ndim differ from the stream header");
    for (int a = 0; a < 3; ++a)
      if (h->dims[a] != dims3[a]) return fail(HC_ERR_INVALID_ARG, "dims differ from the stream header");
    if (in->level != HC_STAGE_M && in->level != HC_STAGE_P && in->level != HC_STAGE_Q)
      return fail(HC_ERR_INVALID_ARG, "fused level must be HC_STAGE_M, HC_STAGE_P or HC_STAGE_Q");
    return HC_OK;
  }
  if (in->n != L.N) return fail(HC_ERR_INVALID_ARG, "stage length differs from prod(dims)");
  if ((in->kind == HC_STAGE_P || in->kind == HC_STAGE_M) && (in->S < 1 || in->S > kMaxS))
    return fail(HC_ERR_INVALID_ARG, "M / P input needs S");
  if (in->kind == HC_STAGE_F && in->dtype != HC_F32 && in->dtype != HC_F64)
    return fail(HC_ERR_INVALID_ARG, "F input dtype");
  if (in->kind == HC_STAGE_M && in->pred != HC_PRED_MEAN)
    return fail(HC_ERR_UNSUPPORTED, "HSZp-style metadata supports no operation (Section V)");
  if (in->kind == HC_STAGE_P && in->pred == HC_PRED_MEAN)
    return fail(HC_ERR_UNSUPPORTED, "a block-mean D_p array needs its block means: operate on the stream");
  if ((in->kind == HC_STAGE_P || in->kind == HC_STAGE_M) && in->pred >= HC_PRED_LORENZO)
    return fail(HC_ERR_UNSUPPORTED, "a global-predictor or box D_p array: operate on the stream");
  if (in->kind < HC_STAGE_M || in->kind > HC_STAGE_F) return fail(HC_ERR_INVALID_ARG, "unknown stage kind");
  return HC_OK;
}

extern "C" {

const char* hc_status_str(int status) {
  switch (status) {
    case HC_OK:
      return "ok";
    case HC_ERR_INVALID_ARG:
      return "invalid argument";
    case HC_ERR_RANGE:
      return "value out of range";
    case HC_ERR_CORRUPT:
      return "corrupt stream";
    case HC_ERR_UNSUPPORTED:
      return "unsupported";
    case HC_ERR_CUDA:
      return "CUDA error";
    case HC_ERR_NOMEM:
      return "buffer too small";
    case HC_ERR_TIMEOUT:
      return "timeout";
    default:
      return "unknown status";
  }
}

const char* hc_last_error(void) { return g_last_error; }

int hc_version(void) { return kVersion; }

size_t hc_compress_bound(int64_t n, int S) {
  Layout L;
  if (make_layout(1, &n, S, &L) != HC_OK) return 0;
  return L.bound;
}

size_t hc_compress_workspace_bytes(int64_t n, int S) {
  Layout L;
  if (make_layout(1, &n, S, &L) != HC_OK) return 0;
  return compress_ws_bytes(L);
}

size_t hc_workspace_bytes(void) { return kOpWsBytes; }

size_t hc_workspace_bytes_for(const hc_header* hdr) {
  if (!hdr || hdr->ndim < 1 || hdr->ndim > 3 || hdr->pred > HC_PRED_MEAN_ND) return 0;
  // the fields the size depends on must agree: extents >= 1 whose product is N
  __int128 n = 1;
  for (int a = 0; a < 3; ++a) {
    if (hdr->dims[a] < 1 || (hdr->pred == HC_PRED_MEAN_ND && hdr->block[a] < 1)) return 0;
    n *= hdr->dims[a];
    if (n > ((__int128)1 << 40)) return 0;
  }
  if (n != hdr->N) return 0;
  if (hdr->pred == HC_PRED_MEAN_ND) return xnd_workspace_bytes(hdr);
  return global_workspace_bytes(hdr);
}

size_t hc_stage_bytes(const hc_header* hdr, int kind) {
  if (!hdr) return 0;
  switch (kind) {
    case HC_STAGE_COMPRESSED:
      return (size_t)hdr->total_bytes;
    case HC_STAGE_M:
      return 4 * (size_t)hdr->nb;
    case HC_STAGE_P:
    case HC_STAGE_Q:
      return 4 * (size_t)hdr->N;
    case HC_STAGE_F:
      return (hdr->dtype == HC_F64 ? 8 : 4) * (size_t)hdr->N;
    default:
      return 0;
  }
}

int hc_compress_ex(const void* d_x, int dtype, int ndim, const int64_t* dims, double eb, int eb_mode, int S,
                   int predictor, void* d_stream, size_t cap, void* d_ws, size_t ws_bytes, size_t* out_bytes,
                   hc_header* hdr_out, void* stream) {
  if (predictor == HC_PRED_MEAN_ND) return fail(HC_ERR_INVALID_ARG, "HSZx-nd streams are written by hc_compress_nd");
  return compress_impl(d_x, dtype == HC_F64 ? 1 : 0, dtype, ndim, dims, eb, 0.0, eb_mode, S, predictor, nullptr, d_stream,
                       cap, d_ws, ws_bytes, out_bytes, hdr_out, as_stream(stream));
}

int hc_compress(const void* d_x, int dtype, int ndim, const int64_t* dims, double eb, int eb_mode, int S,
                void* d_stream, size_t cap, void* d_ws, size_t ws_bytes, size_t* out_bytes, hc_header* hdr_out,
                void* stream) {
  return hc_compress_ex(d_x, dtype, ndim, dims, eb, eb_mode, S, HC_PRED_DELTA, d_stream, cap, d_ws, ws_bytes,
                        out_bytes, hdr_out, stream);
}

int hc_compress_codes_ex(const int32_t* d_q, int dtype, int ndim, const int64_t* dims, double eps, double eb,
                         int eb_mode, int S, int predictor, void* d_stream, size_t cap, void* d_ws, size_t ws_bytes,
                         size_t* out_bytes, hc_header* hdr_out, void* stream) {
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(HC_ERR_INVALID_ARG, "eps must be positive and finite");
  if (predictor == HC_PRED_MEAN_ND) return fail(HC_ERR_INVALID_ARG, "HSZx-nd streams are written by hc_compress_codes_nd");
  return compress_impl(d_q, 2, dtype, ndim, dims, eb, eps, eb_mode, S, predictor, nullptr, d_stream, cap, d_ws, ws_bytes,
                       out_bytes, hdr_out, as_stream(stream));
}

int hc_compress_codes(const int32_t* d_q, int dtype, int ndim, const int64_t* dims, double eps, double eb,
                      int eb_mode, int S, void* d_stream, size_t cap, void* d_ws, size_t ws_bytes, size_t* out_bytes,
                      hc_header* hdr_out, void* stream) {
  return hc_compress_codes_ex(d_q, dtype, ndim, dims, eps, eb, eb_mode, S, HC_PRED_DELTA, d_stream, cap, d_ws,
                              ws_bytes, out_bytes, hdr_out, stream);
}

size_t hc_compress_bound_nd(int ndim, const int64_t* dims, const int32_t* block) {
  Layout L;
  if (make_layout_nd(ndim, dims, block, &L) != HC_OK) return 0;
  return L.bound;
}

size_t hc_compress_workspace_bytes_nd(int ndim, const int64_t* dims, const int32_t* block) {
  Layout L;
  if (make_layout_nd(ndim, dims, block, &L) != HC_OK) return 0;
  return compress_ws_bytes(L);
}

int hc_compress_nd(const void* d_x, int dtype, int ndim, const int64_t* dims, const int32_t* block, double eb,
                   int eb_mode, void* d_stream, size_t cap, void* d_ws, size_t ws_bytes, size_t* out_bytes,
                   hc_header* hdr_out, void* stream) {
  return compress_impl(d_x, dtype == HC_F64 ? 1 : 0, dtype, ndim, dims, eb, 0.0, eb_mode, 0, HC_PRED_MEAN_ND, block,
                       d_stream, cap, d_ws, ws_bytes, out_bytes, hdr_out, as_stream(stream));
}

int hc_compress_codes_nd(const int32_t* d_q, int dtype, int ndim, const int64_t* dims, const int32_t* block,
                         double eps, double eb, int eb_mode, void* d_stream, size_t cap, void* d_ws, size_t ws_bytes,
                         size_t* out_bytes, hc_header* hdr_out, void* stream) {
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(HC_ERR_INVALID_ARG, "eps must be positive and finite");
  return compress_impl(d_q, 2, dtype, ndim, dims, eb, eps, eb_mode, 0, HC_PRED_MEAN_ND, block, d_stream, cap, d_ws,
                       ws_bytes, out_bytes, hdr_out, as_stream(stream));
}

int hc_read_header(const void* d_stream, size_t bytes, hc_header* hdr_out, void* stream) {
  return read_header_impl(d_stream, bytes, hdr_out, as_stream(stream));
}

int hc_read_header_host(const void* h_stream, size_t bytes, hc_header* hdr_out) {
  return read_header_host_impl(h_stream, bytes, hdr_out);
}

int hc_decompress_to_stage(const hc_header* hdr, const void* d_stream, int kind, void* d_out, int out_dtype,
                           void* d_ws, size_t ws_bytes, void* stream) {
  if (!hdr || !d_stream || !d_out) return fail(HC_ERR_INVALID_ARG, "null pointer");
  int rc = check_header(*hdr);
  if (rc) return rc;
  if (!d_ws || ws_bytes < kOpWsBytes) return fail(HC_ERR_NOMEM, "workspace smaller than hc_workspace_bytes()");
  if (!aligned16(d_stream) || !aligned16(d_out) || !aligned16(d_ws))
    return fail(HC_ERR_INVALID_ARG, "device buffers must be 16-byte aligned");
  if (kind < HC_STAGE_M || kind > HC_STAGE_F) return fail(HC_ERR_INVALID_ARG, "kind must be M, P, Q or F");
  if (kind == HC_STAGE_F && out_dtype != HC_F32 && out_dtype != HC_F64)
    return fail(HC_ERR_INVALID_ARG, "F output is HC_F32 or HC_F64");
  if (hdr->pred == HC_PRED_MEAN_ND)
    return xnd_decode_impl(hdr, d_stream, kind, d_out, out_dtype, d_ws, ws_bytes, as_stream(stream));
  if (hdr->pred >= HC_PRED_LORENZO)
    return global_decode_impl(hdr, d_stream, kind, d_out, out_dtype, d_ws, ws_bytes, as_stream(stream));
  return decode_impl(hdr, d_stream, kind, d_out, out_dtype, d_ws, as_stream(stream));
}

int hc_workspace_status(void* d_ws, void* stream) {
  if (!d_ws) return fail(HC_ERR_INVALID_ARG, "null workspace");
  int v = 0, zero = 0;
  cudaStream_t st = as_stream(stream);
  if (cudaMemcpyAsync(&v, d_ws, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(d_ws, &zero, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(HC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  return v;
}

static int stats(const hc_stage* in, double eps, int ndim, const int64_t* dims, hc_scalar* d_out, void* d_ws,
                 size_t ws_bytes, void* stream, int what) {
  int64_t dims3[3];
  int rc = check_op(in, eps, ndim, dims, d_ws, ws_bytes, dims3);
  if (rc) return rc;
  if (!d_out) return fail(HC_ERR_INVALID_ARG, "null output");
  if (in->kind == HC_STAGE_COMPRESSED) {
    if (in->hdr->pred == HC_PRED_MEAN_ND)
      return xnd_stats_impl(in->hdr, in->d_data, in->level, what, d_out, d_ws, ws_bytes, as_stream(stream));
    if (in->hdr->pred >= HC_PRED_LORENZO)
      return global_stats_impl(in->hdr, in->d_data, in->level, what, d_out, d_ws, ws_bytes, as_stream(stream));
    return reduce_stream_impl(in->hdr, in->d_data, in->level, what, d_out, d_ws, as_stream(stream));
  }
  if (in->kind == HC_STAGE_M) {
    // block means of an HSZx stream (Eq. mean_m): the mean only
    if (what != RED_MEAN) return fail(HC_ERR_UNSUPPORTED, "stage 1 gives the mean only (Eq. mean_m)");
    return mean_m_array_impl(reinterpret_cast<const int32_t*>(in->d_data), ceil_div(in->n, in->S), in->S, in->n, eps,
                             d_out, d_ws, as_stream(stream));
  }
  return reduce_array_impl(in, eps, what, d_out, d_ws, as_stream(stream));
}

int hc_op_mean(const hc_stage* in, double eps, int ndim, const int64_t* dims, hc_scalar* d_out, void* d_ws,
               size_t ws_bytes, void* stream) {
  return stats(in, eps, ndim, dims, d_out, d_ws, ws_bytes, stream, RED_MEAN);
}

int hc_op_variance(const hc_stage* in, double eps, int ndim, const int64_t* dims, hc_scalar* d_out, void* d_ws,
                   size_t ws_bytes, void* stream) {
  return stats(in, eps, ndim, dims, d_out, d_ws, ws_bytes, stream, RED_VAR);
}

int hc_op_std(const hc_stage* in, double eps, int ndim, const int64_t* dims, hc_scalar* d_out, void* d_ws,
              size_t ws_bytes, void* stream) {
  return stats(in, eps, ndim, dims, d_out, d_ws, ws_bytes, stream, RED_VAR);
}

static int stencil(const hc_stage* in, double eps, int ndim, const int64_t* dims, int op, int axis, void* d_out,
                   int out_dtype, void* d_ws, size_t ws_bytes, void* stream) {
  int64_t dims3[3];
  int rc = check_op(in, eps, ndim, dims, d_ws, ws_bytes, dims3);
  if (rc) return rc;
  if (!d_out || !aligned16(d_out)) return fail(HC_ERR_INVALID_ARG, "output must be a 16-byte aligned device buffer");
  if (op == ST_DERIV && (axis < 0 || axis >= ndim)) return fail(HC_ERR_INVALID_ARG, "axis out of range");
  const int axis3 = axis + 3 - ndim;
  if (in->kind == HC_STAGE_COMPRESSED) {
    if (in->level == HC_STAGE_M) return fail(HC_ERR_UNSUPPORTED, "stage 1 holds no point values to differentiate");
    if (in->hdr->pred == HC_PRED_MEAN_ND)
      return xnd_stencil_impl(in->hdr, in->d_data, in->level, op, axis3, d_out, out_dtype, d_ws, ws_bytes,
                              as_stream(stream));
    if (in->hdr->pred >= HC_PRED_LORENZO)
      return global_stencil_impl(in->hdr, in->d_data, in->level, op, axis3, d_out, out_dtype, d_ws, ws_bytes,
                                 as_stream(stream));
    if (in->level == HC_STAGE_P)
      return fail(HC_ERR_UNSUPPORTED,
                  "stage-2 differentiation is not defined for a 1-D block partition (Section V-B)");
    return stencil_stream_impl(in->hdr, in->d_data, op, axis3, d_out, out_dtype, d_ws, as_stream(stream));
  }
  return stencil_array_impl(in, dims3, eps, op, axis3, d_out, out_dtype, d_ws, as_stream(stream));
}

int hc_op_derivative(const hc_stage* in, double eps, int ndim, const int64_t* dims, int axis, void* d_out,
                     int out_dtype, void* d_ws, size_t ws_bytes, void* stream) {
  return stencil(in, eps, ndim, dims, ST_DERIV, axis, d_out, out_dtype, d_ws, ws_bytes, stream);
}

int hc_op_gradmag(const hc_stage* in, double eps, int ndim, const int64_t* dims, void* d_out, int out_dtype,
                  void* d_ws, size_t ws_bytes, void* stream) {
  return stencil(in, eps, ndim, dims, ST_GRADMAG, 0, d_out, out_dtype, d_ws, ws_bytes, stream);
}

int hc_op_laplacian(const hc_stage* in, double eps, int ndim, const int64_t* dims, void* d_out, int out_dtype,
                    void* d_ws, size_t ws_bytes, void* stream) {
  return stencil(in, eps, ndim, dims, ST_LAPLACIAN, 0, d_out, out_dtype, d_ws, ws_bytes, stream);
}

int hc_autotune(const hc_stage* in, int op, int out_dtype, void* d_out, void* d_ws, size_t ws_bytes, void* stream,
                int* chosen) {
  if (!in || !chosen) return fail(HC_ERR_INVALID_ARG, "null argument");
  *chosen = 0;
  if (in->kind != HC_STAGE_COMPRESSED || !in->hdr || !in->d_data)
    return fail(HC_ERR_INVALID_ARG, "hc_autotune takes a compressed stream with its header");
  if (int rc = check_header(*in->hdr)) return rc;
  if (!d_ws || ws_bytes < kOpWsBytes) return fail(HC_ERR_NOMEM, "workspace smaller than hc_workspace_bytes()");
  if (!d_out || !aligned16(d_out) || !aligned16(in->d_data) || !aligned16(d_ws))
    return fail(HC_ERR_INVALID_ARG, "device buffers must be 16-byte aligned");
  int sop;
  switch (op) {
    case HC_OP_DERIVATIVE:
      sop = ST_DERIV;
      break;
    case HC_OP_GRADMAG:
      sop = ST_GRADMAG;
      break;
    case HC_OP_LAPLACIAN:
      sop = ST_LAPLACIAN;
      break;
    case HC_OP_MULTI:
      sop = ST_MULTI;
      if (out_dtype == HC_I64) return fail(HC_ERR_INVALID_ARG, "out_dtype must be F32 or F64");
      break;
    default:
      return HC_OK;  // statistics have no tunable tile
  }
  if (out_dtype != HC_F32 && out_dtype != HC_F64 && out_dtype != HC_I64) return fail(HC_ERR_INVALID_ARG, "out_dtype");
  if (in->hdr->pred >= HC_PRED_LORENZO) return HC_OK;  // global predictors: no tiled kernel to tune
  int64_t d3[3];
  stencil_walk_dims(in->hdr, d3, nullptr);
  return stencil_pipe_autotune(in->hdr, in->d_data, d3, sop, d_out, out_dtype, d_ws, as_stream(stream), chosen);
}

int hc_autotune_export(char* buf, size_t cap, size_t* len) { return autotune_export_impl(buf, cap, len); }

int hc_autotune_import(const char* text, int* count) { return autotune_import_impl(text, count); }

int hc_op_multi(const hc_stage* in, double eps, int ndim, const int64_t* dims, const hc_multi_out* out, void* d_ws,
                size_t ws_bytes, void* stream) {
  int64_t dims3[3];
  int rc = check_op(in, eps, ndim, dims, d_ws, ws_bytes, dims3);
  if (rc) return rc;
  if (!out) return fail(HC_ERR_INVALID_ARG, "null output set");
  if (out->out_dtype != HC_F32 && out->out_dtype != HC_F64) return fail(HC_ERR_INVALID_ARG, "out_dtype must be F32 or F64");
  void* fields[5] = {out->d_derivative[0], out->d_derivative[1], out->d_derivative[2], out->d_gradmag,
                     out->d_laplacian};
  for (int a = ndim; a < 3; ++a)
    if (out->d_derivative[a]) return fail(HC_ERR_INVALID_ARG, "derivative output for an axis >= ndim");
  for (void* f : fields)
    if (f && !aligned16(f)) return fail(HC_ERR_INVALID_ARG, "outputs must be 16-byte aligned device buffers");
  if (in->kind == HC_STAGE_COMPRESSED && in->hdr->pred < HC_PRED_LORENZO) {
    if (in->level == HC_STAGE_P && (out->d_derivative[0] || out->d_derivative[1] || out->d_derivative[2] ||
                                    out->d_gradmag || out->d_laplacian))
      return fail(HC_ERR_UNSUPPORTED, "stage-2 differentiation is not defined for a 1-D block partition (Section V-B)");
    if (in->level == HC_STAGE_Q) {
      // the user's derivative axes in the shape the kernel walks
      void* deriv3[3] = {nullptr, nullptr, nullptr};
      for (int a = 0; a < ndim; ++a) {
        int axis3 = a + 3 - ndim;
        int64_t d3[3];
        stencil_walk_dims(in->hdr, d3, &axis3);
        deriv3[axis3] = out->d_derivative[a];
      }
      rc = stencil_multi_impl(in->hdr, in->d_data, deriv3, out->d_gradmag, out->d_laplacian, out->d_stats,
                              out->out_dtype, d_ws, as_stream(stream));
      if (rc != HC_ERR_UNSUPPORTED) return rc;
    }
  }
  // one operation at a time
  for (int a = 0; a < ndim; ++a)
    if (out->d_derivative[a] &&
        (rc = stencil(in, eps, ndim, dims, ST_DERIV, a, out->d_derivative[a], out->out_dtype, d_ws, ws_bytes, stream)))
      return rc;
  if (out->d_gradmag &&
      (rc = stencil(in, eps, ndim, dims, ST_GRADMAG, 0, out->d_gradmag, out->out_dtype, d_ws, ws_bytes, stream)))
    return rc;
  if (out->d_laplacian &&
      (rc = stencil(in, eps, ndim, dims, ST_LAPLACIAN, 0, out->d_laplacian, out->out_dtype, d_ws, ws_bytes, stream)))
    return rc;
  if (out->d_stats) return stats(in, eps, ndim, dims, out->d_stats, d_ws, ws_bytes, stream, RED_VAR);
  return HC_OK;
}

static int vector_op(const hc_stage* comps, int ncomp, int ndim, const int64_t* dims, void* d_out, int out_dtype,
                     void* d_ws, size_t ws_bytes, void* stream, int op) {
  if (!comps || !d_out) return fail(HC_ERR_INVALID_ARG, "null pointer");
  if (op == 0 && ncomp != ndim) return fail(HC_ERR_INVALID_ARG, "divergence takes ndim components");
  if (op == 1 && (ndim != 2 || ncomp != 2)) return fail(HC_ERR_UNSUPPORTED, "curl is defined here for 2-D fields");
  if (ncomp < 1 || ncomp > 3) return fail(HC_ERR_INVALID_ARG, "ncomp");
  if (!aligned16(d_out)) return fail(HC_ERR_INVALID_ARG, "output must be a 16-byte aligned device buffer");
  if (out_dtype != HC_F32 && out_dtype != HC_F64 && out_dtype != HC_I64) return fail(HC_ERR_INVALID_ARG, "out_dtype");
  const hc_header* hs[3];
  const void* ds[3];
  const int level = comps[0].level;
  bool fused = level == HC_STAGE_Q;  // 1-D block streams of one block size at stage Q: one fused kernel
  for (int c = 0; c < ncomp; ++c) {
    const hc_stage& in = comps[c];
    if (in.kind != HC_STAGE_COMPRESSED || !in.hdr)
      return fail(HC_ERR_UNSUPPORTED, "vector operations take compressed streams");
    if (in.level != level) return fail(HC_ERR_INVALID_ARG, "every component at the same level");
    if (level != HC_STAGE_P && level != HC_STAGE_Q)
      return fail(HC_ERR_UNSUPPORTED, "vector operations run at stage P or Q (Section V-C)");
    int64_t dims3[3];
    int rc = check_op(&in, in.hdr->eps, ndim, dims, d_ws, ws_bytes, dims3);
    if (rc) return rc;
    if (in.hdr->pred >= HC_PRED_LORENZO || in.hdr->S != comps[0].hdr->S) fused = false;
    hs[c] = in.hdr;
    ds[c] = in.d_data;
  }
  if (fused) return vector_stream_impl(hs, ds, ncomp, op, d_out, out_dtype, d_ws, as_stream(stream));
  return vector_any_impl(hs, ds, ncomp, op, level, d_out, out_dtype, d_ws, ws_bytes, as_stream(stream));
}

size_t hc_vector_workspace_bytes(const hc_stage* comps, int ncomp) {
  if (!comps || ncomp < 1 || ncomp > 3) return 0;
  const hc_header* hs[3];
  bool fused = comps[0].level == HC_STAGE_Q;
  for (int c = 0; c < ncomp; ++c) {
    if (comps[c].kind != HC_STAGE_COMPRESSED || !comps[c].hdr || !hc_workspace_bytes_for(comps[c].hdr)) return 0;
    hs[c] = comps[c].hdr;
    if (hs[c]->pred >= HC_PRED_LORENZO || hs[c]->S != hs[0]->S || comps[c].level != HC_STAGE_Q) fused = false;
  }
  return fused ? kOpWsBytes : vector_any_workspace_bytes(hs, ncomp);
}

int hc_op_divergence(const hc_stage* comps, int ncomp, int ndim, const int64_t* dims, void* d_out, int out_dtype,
                     void* d_ws, size_t ws_bytes, void* stream) {
  return vector_op(comps, ncomp, ndim, dims, d_out, out_dtype, d_ws, ws_bytes, stream, 0);
}

int hc_op_curl(const hc_stage* comps, int ncomp, int ndim, const int64_t* dims, void* d_out, int out_dtype,
               void* d_ws, size_t ws_bytes, void* stream) {
  return vector_op(comps, ncomp, ndim, dims, d_out, out_dtype, d_ws, ws_bytes, stream, 1);
}

// ------------------------------------------------------------------ shards
static void put_le(uint8_t* b, int off, uint64_t v, int n) {
  for (int i = 0; i < n; ++i) b[off + i] = (uint8_t)(v >> (8 * i));
}
// The 256-byte image of a header, field by field as read_header_impl reads it.
static void header_image(const hc_header& h, uint8_t* b) {
  std::memset(b, 0, kHeaderBytes);
  put_le(b, 0, kMagic, 4);
  put_le(b, 4, (uint64_t)kVersion, 2);
  put_le(b, 6, (uint64_t)h.dtype, 1);
  put_le(b, 7, (uint64_t)h.ndim, 1);
  for (int a = 0; a < 3; ++a) put_le(b, 8 + 8 * a, (uint64_t)h.dims[a], 8);
  put_le(b, 32, (uint64_t)h.S, 4);
  put_le(b, 36, (uint64_t)h.G, 4);
  uint64_t u;
  std::memcpy(&u, &h.eps, 8);
  put_le(b, 40, u, 8);
  std::memcpy(&u, &h.eb, 8);
  put_le(b, 48, u, 8);
  put_le(b, 56, (uint64_t)h.eb_mode, 4);
  put_le(b, 60, h.qmax, 4);
  put_le(b, 64, (uint64_t)h.N, 8);
  put_le(b, 72, (uint64_t)h.nb, 8);
  put_le(b, 80, (uint64_t)h.nchunks, 8);
  put_le(b, 88, (uint64_t)h.payload_words, 8);
  put_le(b, 96, (uint64_t)h.off_widths, 8);
  put_le(b, 104, (uint64_t)h.off_heads, 8);
  put_le(b, 112, (uint64_t)h.off_chunks, 8);
  put_le(b, 120, (uint64_t)h.off_payload, 8);
  put_le(b, 128, (uint64_t)h.total_bytes, 8);
  put_le(b, 136, h.wmax, 4);
  put_le(b, 140, h.pred, 4);
  for (int a = 0; a < 3; ++a) put_le(b, 144 + 4 * a, h.block[a], 4);
}

int hc_shard_plan(const hc_header* full, const uint64_t* h_chunks, int64_t c0, int64_t c1, hc_shard* out,
                  uint64_t* chunks_out) {
  if (!full || !h_chunks || !out || !chunks_out) return fail(HC_ERR_INVALID_ARG, "null pointer");
  int rc = check_header(*full);
  if (rc) return rc;
  if (full->pred != HC_PRED_DELTA && full->pred != HC_PRED_MEAN)
    return fail(HC_ERR_UNSUPPORTED, "only block-head and block-mean streams shard: their blocks decode alone");
  if (c0 < 0 || c1 <= c0 || c1 > full->nchunks) return fail(HC_ERR_INVALID_ARG, "chunk range must be 0 <= c0 < c1 <= nchunks");
  if (h_chunks[0] != 0 || h_chunks[full->nchunks] != (uint64_t)full->payload_words)
    return fail(HC_ERR_CORRUPT, "chunk index does not run from 0 to the payload size");
  for (int64_t c = 0; c < full->nchunks; ++c)
    if (h_chunks[c] > h_chunks[c + 1]) return fail(HC_ERR_CORRUPT, "chunk index not ascending");
  const int64_t G = full->G, S = full->S;
  const int64_t b0 = c0 * G, b1 = std::min<int64_t>(c1 * G, full->nb);
  const int64_t first = b0 * S, n = std::min<int64_t>(b1 * S, full->N) - first;
  Layout L;
  rc = make_layout(1, &n, (int)S, &L);
  if (rc) return rc;
  if (L.nb != b1 - b0 || L.nchunks != c1 - c0 || L.G != G) return fail(HC_ERR_CORRUPT, "shard layout mismatch");
  const uint64_t w0 = h_chunks[c0], w1 = h_chunks[c1];
  hc_header h = *full;
  h.ndim = 1;
  h.dims[0] = h.dims[1] = 1;
  h.dims[2] = n;
  h.N = n;
  h.nb = L.nb;
  h.nchunks = L.nchunks;
  h.off_widths = L.off_widths;
  h.off_heads = L.off_heads;
  h.off_chunks = L.off_chunks;
  h.off_payload = L.off_payload;
  h.payload_words = (int64_t)(w1 - w0);
  h.total_bytes = align16(L.off_payload + 4 * h.payload_words + 16);
  h.block[0] = h.block[1] = h.block[2] = 0;
  rc = check_header(h);
  if (rc) return rc;
  out->hdr = h;
  header_image(h, out->header_bytes);
  out->src_off[0] = full->off_widths + b0;
  out->dst_off[0] = h.off_widths;
  out->nbytes[0] = b1 - b0;
  out->src_off[1] = full->off_heads + 4 * b0;
  out->dst_off[1] = h.off_heads;
  out->nbytes[1] = 4 * (b1 - b0);
  out->src_off[2] = full->off_payload + 4 * (int64_t)w0;
  out->dst_off[2] = h.off_payload;
  out->nbytes[2] = 4 * h.payload_words;
  out->chunks_off = h.off_chunks;
  out->first = first;
  for (int64_t k = 0; k <= c1 - c0; ++k) chunks_out[k] = h_chunks[c0 + k] - w0;
  return HC_OK;
}

// Eq. var_q on the host: the same integer arithmetic and the same rounding
// steps as finalize_int, the device finish of every exact statistic (each
// integer converted to double once, round to nearest even; the 128-bit
// numerator N s2 - s1^2 formed with the same wrapping 128-bit products).
int hc_finalize(int64_t n, int64_t s1, uint64_t s2_lo, uint64_t s2_hi, double eps, hc_scalar* out) {
  if (!out) return fail(HC_ERR_INVALID_ARG, "null output");
  if (n < 1) return fail(HC_ERR_INVALID_ARG, "N must be at least 1");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(HC_ERR_INVALID_ARG, "eps must be positive and finite");
  typedef unsigned __int128 u128h;
  typedef __int128 i128h;
  const u128h s2 = ((u128h)s2_hi << 64) | (u128h)s2_lo;
  const double two_eps = 2.0 * eps;
  hc_scalar r;
  r.n = n;
  r.s1 = s1;
  r.s2_lo = s2_lo;
  r.s2_hi = s2_hi;
  r.status = HC_OK;
  r.exact = 1;
  r.mean = ((double)s1 / (double)n) * two_eps;
  double v = std::nan("");
  if (n >= 2) {
    const i128h num = (i128h)((u128h)(i128h)n * s2 - (u128h)((i128h)s1 * (i128h)s1));
    const double den = (double)n * (double)(n - 1);
    v = ((double)num / den) * (two_eps * two_eps);
  }
  r.variance = v;
  r.std = std::sqrt(v);
  *out = r;
  return HC_OK;
}

size_t hc_batch_plan_bytes(int n_items) { return (size_t)batch_plan_bytes(n_items); }
size_t hc_batch_workspace_bytes(int n_items) { return (size_t)batch_ws_bytes(n_items); }
int hc_batch_plan(const hc_batch_item* items, int n_items, const hc_batch_tune* tune, void* h_plan, size_t cap,
                  size_t* used) {
  return batch_plan_impl(items, n_items, tune, h_plan, cap, used);
}
int hc_batch_run(const void* h_plan, const void* d_plan, void* d_ws, size_t ws_bytes, void* stream) {
  return batch_run_impl(h_plan, d_plan, d_ws, ws_bytes, as_stream(stream));
}
int hc_batch_graph_create(const void* h_plan, const void* d_plan, void* d_ws, size_t ws_bytes, void** graph_exec) {
  return batch_graph_impl(h_plan, d_plan, d_ws, ws_bytes, graph_exec);
}
int hc_batch_graph_launch(void* graph_exec, void* stream) {
  return batch_graph_launch_impl(graph_exec, as_stream(stream));
}
int hc_batch_graph_destroy(void* graph_exec) { return batch_graph_destroy_impl(graph_exec); }
int hc_batch_status(void* d_ws, void* stream) { return batch_status_impl(d_ws, as_stream(stream)); }

}  // extern "C"
