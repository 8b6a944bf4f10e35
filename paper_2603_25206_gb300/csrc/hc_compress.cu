// hc_compress.cu -- the compressor C of the paper (Algorithm 1, Section IV),
// on the GPU.  The stream it writes is byte-identical to the layout described
// in hc_internal.cuh.
//
//   k_ws_init      clear the workspace accumulators
//   k_minmax       value range of the field (value-range-relative bound)
//   k_eps          eps = eb or eb * (max - min)
//   k_blocks       quantize, block metadata (first code, or the block mean
//                  for HSZx, or none for the global predictors), block
//                  width, words per chunk, max |q|, max width    (one thread / block)
//   k_chunk_scan   exclusive scan of the words per chunk -> chunk index
//   k_pack         sign words + w-bit magnitudes of every block  (one thread / block)
//   k_header       header and the zero padding between sections
#include <cstdint>
#include <cstring>

#include "hc_internal.cuh"
#include "hc_launch.h"

namespace hc {

// Workspace of the compressor (caller-provided device memory).
struct CompWs {
  int status;
  uint32_t qmax;
  uint32_t wmax;
  uint32_t pad0;
  unsigned long long min_key;
  unsigned long long max_key;
  double eps;
  unsigned long long total_words;
  unsigned long long pad1[2];
  // followed by unsigned long long chunk_words[nchunks] (offset 64)
};
static_assert(sizeof(CompWs) == 64, "workspace header is 64 bytes");

__device__ __forceinline__ unsigned long long* chunk_words(CompWs* ws) {
  return reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ws) + sizeof(CompWs));
}

// Order-preserving map of a double to an unsigned 64-bit key.
__device__ __forceinline__ unsigned long long order_key(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(unsigned long long k) {
  unsigned long long b = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

// Input sources ---------------------------------------------------------
struct SrcF32 {
  const float* x;
  __device__ double get(int64_t i) const { return (double)__ldg(x + i); }
};
struct SrcF64 {
  const double* x;
  __device__ double get(int64_t i) const { return __ldg(x + i); }
};

// Quantization (Section IV): q = floor(x / (2 eps) + 0.5) with an IEEE double
// division.  Returns false when |q| >= 2^30 or x is not finite.
template <class Src>
__device__ __forceinline__ bool quantize_at(const Src& src, int64_t i, double two_eps, int32_t& q) {
  const double t = src.get(i) / two_eps;
  const double r = floor(t + 0.5);
  if (!(fabs(r) < (double)kQLimit)) {
    q = 0;
    return false;
  }
  q = (int32_t)r;
  return true;
}

struct SrcCodes {
  const int32_t* q;
};
__device__ __forceinline__ bool quantize_at(const SrcCodes& src, int64_t i, double, int32_t& q) {
  const int32_t v = __ldg(src.q + i);
  if (!(v > -kQLimit && v < kQLimit)) {
    q = 0;
    return false;
  }
  q = v;
  return true;
}

__global__ void k_ws_init(CompWs* ws, int64_t nchunks) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    ws->status = 0;
    ws->qmax = 0;
    ws->wmax = 0;
    ws->min_key = ~0ull;
    ws->max_key = 0ull;
    ws->eps = 0.0;
    ws->total_words = 0;
  }
  for (int64_t c = i; c < nchunks; c += (int64_t)gridDim.x * blockDim.x) chunk_words(ws)[c] = 0;
}

template <class Src>
__global__ void __launch_bounds__(kThreads) k_minmax(Src src, int64_t n, CompWs* ws) {
  __shared__ unsigned long long s_min, s_max;
  __shared__ int s_bad;
  if (threadIdx.x == 0) {
    s_min = ~0ull;
    s_max = 0ull;
    s_bad = 0;
  }
  __syncthreads();
  unsigned long long lo = ~0ull, hi = 0ull;
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = src.get(i);
    if (!isfinite(v)) {
      bad = 1;
      continue;
    }
    const unsigned long long k = order_key(v);
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
  }
  atomicMin(&s_min, lo);
  atomicMax(&s_max, hi);
  if (bad) s_bad = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMin(&ws->min_key, s_min);
    atomicMax(&ws->max_key, s_max);
    if (s_bad) set_error(&ws->status, HC_ERR_RANGE);
  }
}

// eps = eb (absolute) or eb * (max - min) (value-range relative); a constant
// field keeps eps = eb.
__global__ void k_eps(CompWs* ws, double eb, int rel) {
  double eps = eb;
  if (rel && ws->max_key >= ws->min_key && ws->status == 0) {
    const double mn = key_value(ws->min_key), mx = key_value(ws->max_key);
    if (mx > mn) eps = eb * (mx - mn);
  }
  if (!(eps > 0.0) || !isfinite(eps)) set_error(&ws->status, HC_ERR_INVALID_ARG);
  ws->eps = eps;
}

struct OutStream {
  uint8_t* base;
  uint8_t* widths;
  int32_t* heads;
  uint64_t* chunks;
  uint32_t* payload;
  int64_t N, nb, nchunks;
  int S, G, nseg;
  int pred;      // hc_predictor
  int64_t L[3];  // prediction shape of the global predictors: (n0, n1, n2), or (1, 1, N) for HSZp
  int64_t bd[3];  // HSZx-nd: box extents along (n0, n1, n2)
  int64_t gd[3];  // HSZx-nd: box grid ceil(n_a / b_a)
};

// HSZx-nd: field index of slot k of box b (row-major inside the box, boxes
// row-major over the grid), or -1 for a slot outside the field.
__device__ __forceinline__ int64_t box_slot_index(const OutStream& o, int64_t b, int64_t k) {
  const int64_t k2 = b % o.gd[2], r = b / o.gd[2];
  const int64_t k1 = r % o.gd[1], k0 = r / o.gd[1];
  const int64_t s2 = k % o.bd[2], t = k / o.bd[2];
  const int64_t s1 = t % o.bd[1], s0 = t / o.bd[1];
  const int64_t z = k0 * o.bd[0] + s0, y = k1 * o.bd[1] + s1, x = k2 * o.bd[2] + s2;
  if (z >= o.L[0] || y >= o.L[1] || x >= o.L[2]) return -1;
  return (z * o.L[1] + y) * o.L[2] + x;
}

// Residual of the global predictors at flat index i (Section IV, HSZp and
// HSZp-nd): the Lorenzo residual over the prediction shape L, with codes
// outside the field taken as 0 -- sum over the corners d of {0,1}^3 of
// (-1)^(d0+d1+d2) q(i - d).  With leading axes of length 1 it is the 2-D
// four-term or the 1-D two-term form.  The neighbours are quantized again
// here (the same rule, so the same codes).  Returns false when a code is out
// of range or the residual does not fit the encoder's 31-bit magnitude.
template <class Src>
__device__ __forceinline__ bool global_residual(const Src& src, const OutStream& o, int64_t i, double two_eps,
                                                int32_t& p) {
  const int64_t x = i % o.L[2], r = i / o.L[2];
  const int64_t y = r % o.L[1], z = r / o.L[1];
  long long acc = 0;
  bool ok = true;
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const int dz = d >> 2, dy = (d >> 1) & 1, dx = d & 1;
    if ((dz && z == 0) || (dy && y == 0) || (dx && x == 0)) continue;
    int32_t q;
    ok &= quantize_at(src, i - dz * o.L[1] * o.L[2] - dy * o.L[2] - dx, two_eps, q);
    acc += ((dz + dy + dx) & 1) ? -(long long)q : (long long)q;
  }
  if (!ok || acc <= -(1ll << 31) || acc >= (1ll << 31)) {
    p = 0;
    return false;
  }
  p = (int32_t)acc;
  return true;
}

// Integer block mean of HSZx: the integer nearest to a / d (d > 0), ties
// toward zero (Section V-D bounds the rounding by 1/2; the worked example of
// Section IV rounds 5.5 down to 5).
__device__ __forceinline__ int32_t nearest_ratio(long long a, long long d) {
  const unsigned long long m = (unsigned long long)(a < 0 ? -a : a);
  const long long r = (long long)((2ull * m + (unsigned long long)d - 1ull) / (2ull * (unsigned long long)d));
  return (int32_t)(a < 0 ? -r : r);
}

// One thread per block: codes, deltas, width, head; per-chunk word counts.
template <class Src>
__global__ void __launch_bounds__(kThreads) k_blocks(Src src, OutStream o, CompWs* ws) {
  __shared__ unsigned long long s_cw[kThreads + 2];
  __shared__ uint32_t s_qmax, s_wmax;
  __shared__ int s_bad;
  const int64_t bfirst = (int64_t)blockIdx.x * blockDim.x;
  const int64_t cfirst = bfirst / o.G;
  for (int i = threadIdx.x; i < kThreads + 2; i += blockDim.x) s_cw[i] = 0;
  if (threadIdx.x == 0) {
    s_qmax = 0;
    s_wmax = 0;
    s_bad = 0;
  }
  __syncthreads();
  const int64_t b = bfirst + threadIdx.x;
  const double two_eps = 2.0 * ws->eps;
  if (b < o.nb) {
    const int64_t first = b * o.S;
    const int64_t Sb = min((int64_t)o.S, o.N - first);
    int32_t prev = 0, q;
    uint32_t maxmag = 0, qm = 0;
    bool ok = true;
    if (o.pred == HC_PRED_MEAN_ND) {
      // HSZx-nd: the box mean over the slots inside the field, then the
      // widest |q - M_b| over them
      long long sum = 0;
      int64_t nin = 0;
      for (int64_t k = 0; k < o.S; ++k) {
        const int64_t i = box_slot_index(o, b, k);
        if (i < 0) continue;
        ok &= quantize_at(src, i, two_eps, q);
        sum += q;
        ++nin;
        const uint32_t aq = (uint32_t)(q < 0 ? -q : q);
        qm = aq > qm ? aq : qm;
      }
      const int32_t mb = ok ? nearest_ratio(sum, nin) : 0;
      o.heads[b] = mb;
      for (int64_t k = 0; k < o.S && ok; ++k) {
        const int64_t i = box_slot_index(o, b, k);
        if (i < 0) continue;
        quantize_at(src, i, two_eps, q);
        const int32_t p = q - mb;
        const uint32_t m = (uint32_t)(p < 0 ? -(long long)p : (long long)p);
        maxmag = m > maxmag ? m : maxmag;
      }
    } else if (o.pred >= HC_PRED_LORENZO) {
      // global predictors: no block metadata, the widest residual
      o.heads[b] = 0;
      for (int64_t k = 0; k < Sb; ++k) {
        ok &= quantize_at(src, first + k, two_eps, q);
        const uint32_t aq = (uint32_t)(q < 0 ? -q : q);
        qm = aq > qm ? aq : qm;
        int32_t p;
        ok &= global_residual(src, o, first + k, two_eps, p);
        const uint32_t m = (uint32_t)(p < 0 ? -(long long)p : (long long)p);
        maxmag = m > maxmag ? m : maxmag;
      }
    } else if (o.pred == HC_PRED_MEAN) {
      // HSZx: M_b from the block's code sum, then the widest |q - M_b|
      long long sum = 0;
      for (int64_t k = 0; k < Sb; ++k) {
        ok &= quantize_at(src, first + k, two_eps, q);
        sum += q;
        const uint32_t aq = (uint32_t)(q < 0 ? -q : q);
        qm = aq > qm ? aq : qm;
      }
      const int32_t mb = ok ? nearest_ratio(sum, Sb) : 0;
      o.heads[b] = mb;
      for (int64_t k = 0; k < Sb && ok; ++k) {
        quantize_at(src, first + k, two_eps, q);
        const int32_t p = q - mb;
        const uint32_t m = (uint32_t)(p < 0 ? -p : p);
        maxmag = m > maxmag ? m : maxmag;
      }
    } else {
      for (int64_t k = 0; k < Sb; ++k) {
        ok &= quantize_at(src, first + k, two_eps, q);
        if (k == 0) {
          o.heads[b] = q;
        } else {
          const int32_t p = q - prev;
          const uint32_t m = (uint32_t)(p < 0 ? -p : p);
          maxmag = m > maxmag ? m : maxmag;
        }
        const uint32_t aq = (uint32_t)(q < 0 ? -q : q);
        qm = aq > qm ? aq : qm;
        prev = q;
      }
    }
    const uint32_t w = maxmag ? 32u - (uint32_t)__clz(maxmag) : 0u;
    o.widths[b] = (uint8_t)w;
    const uint32_t words = w ? (uint32_t)o.nseg + (((uint32_t)o.S * w + 31u) >> 5) : 0u;
    atomicAdd(&s_cw[b / o.G - cfirst], (unsigned long long)words);
    atomicMax(&s_qmax, qm);
    atomicMax(&s_wmax, w);
    if (!ok) s_bad = 1;
  }
  __syncthreads();
  const int64_t clast = min(o.nb, bfirst + (int64_t)blockDim.x) - 1;
  for (int64_t c = cfirst + threadIdx.x; c <= clast / o.G; c += blockDim.x)
    if (s_cw[c - cfirst]) atomicAdd(&chunk_words(ws)[c], s_cw[c - cfirst]);
  if (threadIdx.x == 0) {
    atomicMax(&ws->qmax, s_qmax);
    atomicMax(&ws->wmax, s_wmax);
    if (s_bad) set_error(&ws->status, HC_ERR_RANGE);
  }
}

// Exclusive scan of the per-chunk word counts into the chunk index (one CTA).
__global__ void __launch_bounds__(1024) k_chunk_scan(CompWs* ws, uint64_t* chunks, int64_t nchunks) {
  __shared__ unsigned long long s_warp[32];
  __shared__ unsigned long long s_carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nt = blockDim.x;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  const unsigned long long* cw = chunk_words(ws);
  for (int64_t base = 0; base < nchunks; base += nt) {
    const int64_t c = base + tid;
    const unsigned long long v = c < nchunks ? cw[c] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
      unsigned long long t = lane < (nt >> 5) ? s_warp[lane] : 0ull;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      s_warp[lane] = t;
    }
    __syncthreads();
    const unsigned long long excl = s_carry + x - v + (wid ? s_warp[wid - 1] : 0ull);
    if (c < nchunks) chunks[c] = excl;
    __syncthreads();
    if (tid == 0) s_carry += s_warp[(nt >> 5) - 1];
    __syncthreads();
  }
  if (tid == 0) {
    chunks[nchunks] = s_carry;
    ws->total_words = s_carry;
  }
}

// One CTA per two chunks; one thread per block writes the block's words.
template <class Src>
__global__ void __launch_bounds__(kThreads) k_pack(Src src, OutStream o, CompWs* ws) {
  extern __shared__ uint32_t s_dyn[];
  __shared__ uint32_t s_warp[32];
  const int64_t b0 = (int64_t)blockIdx.x * kTileChunks * o.G;
  const int nblk = (int)min((int64_t)kTileChunks * o.G, o.nb - b0);
  uint32_t* s_off = s_dyn;  // nblk + 1
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    const uint32_t w = o.widths[b0 + i];
    s_off[i] = w ? (uint32_t)o.nseg + (((uint32_t)o.S * w + 31u) >> 5) : 0u;
  }
  __syncthreads();
  cta_exclusive_scan(s_off, nblk, s_warp);
  const uint64_t base = o.chunks[b0 / o.G];
  const double two_eps = 2.0 * ws->eps;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    const int64_t b = b0 + i;
    const uint32_t w = o.widths[b];
    if (w == 0) continue;
    const int64_t first = b * o.S;
    const int64_t Sb = min((int64_t)o.S, o.N - first);
    uint32_t* out = o.payload + base + s_off[i];
    uint32_t* mag = out + o.nseg;
    uint32_t sign = 0;
    unsigned long long acc = 0;
    uint32_t nbits = 0;
    int32_t prev = 0, q;
    const bool mean_pred = o.pred == HC_PRED_MEAN;
    const bool box_pred = o.pred == HC_PRED_MEAN_ND;
    const bool global_pred = o.pred == HC_PRED_LORENZO || o.pred == HC_PRED_GLOBAL_DELTA;
    const int32_t mb = mean_pred ? o.heads[b] : 0;
    for (int64_t k = 0; k < o.S; ++k) {
      int32_t p = 0;
      if (box_pred) {
        const int64_t i = box_slot_index(o, b, k);
        if (i >= 0) {
          quantize_at(src, i, two_eps, q);
          p = q - o.heads[b];
        }
      } else if (k < Sb) {
        if (global_pred) {
          global_residual(src, o, first + k, two_eps, p);
        } else {
          quantize_at(src, first + k, two_eps, q);
          p = mean_pred ? q - mb : ((k == 0) ? 0 : q - prev);
          prev = q;
        }
      }
      if (p < 0) sign |= 1u << (k & 31);
      if ((k & 31) == 31 || k == o.S - 1) {
        out[k >> 5] = sign;
        sign = 0;
      }
      const uint32_t m = (uint32_t)(p < 0 ? -(long long)p : (long long)p);
      acc |= (unsigned long long)m << nbits;
      nbits += w;
      if (nbits >= 32) {
        *mag++ = (uint32_t)acc;
        acc >>= 32;
        nbits -= 32;
      }
    }
    if (nbits > 0) *mag = (uint32_t)acc;
  }
}

struct HeaderArgs {
  int dtype, ndim, S, G, eb_mode, pred;
  int64_t bd[3];  // HSZx-nd box extents (0 otherwise)
  int64_t dims[3];
  double eb;
  int64_t N, nb, nchunks, off_widths, off_heads, off_chunks, off_payload;
};

__device__ __forceinline__ void put_le(uint8_t* b, int off, unsigned long long v, int nbytes) {
  for (int i = 0; i < nbytes; ++i) b[off + i] = (uint8_t)(v >> (8 * i));
}

// Header (256 bytes) and the zero bytes between sections and after the payload.
__global__ void k_header(HeaderArgs a, uint8_t* stream, CompWs* ws) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned long long pw = ws->total_words;
  const int64_t total = ((a.off_payload + 4 * (int64_t)pw + 16) + 15) & ~(int64_t)15;
  for (int i = 0; i < kHeaderBytes; ++i) stream[i] = 0;
  put_le(stream, 0, kMagic, 4);
  put_le(stream, 4, kVersion, 2);
  put_le(stream, 6, (unsigned long long)a.dtype, 1);
  put_le(stream, 7, (unsigned long long)a.ndim, 1);
  for (int d = 0; d < 3; ++d) put_le(stream, 8 + 8 * d, (unsigned long long)a.dims[d], 8);
  put_le(stream, 32, (unsigned long long)a.S, 4);
  put_le(stream, 36, (unsigned long long)a.G, 4);
  put_le(stream, 40, (unsigned long long)__double_as_longlong(ws->eps), 8);
  put_le(stream, 48, (unsigned long long)__double_as_longlong(a.eb), 8);
  put_le(stream, 56, (unsigned long long)a.eb_mode, 4);
  put_le(stream, 60, ws->qmax, 4);
  put_le(stream, 64, (unsigned long long)a.N, 8);
  put_le(stream, 72, (unsigned long long)a.nb, 8);
  put_le(stream, 80, (unsigned long long)a.nchunks, 8);
  put_le(stream, 88, pw, 8);
  put_le(stream, 96, (unsigned long long)a.off_widths, 8);
  put_le(stream, 104, (unsigned long long)a.off_heads, 8);
  put_le(stream, 112, (unsigned long long)a.off_chunks, 8);
  put_le(stream, 120, (unsigned long long)a.off_payload, 8);
  put_le(stream, 128, (unsigned long long)total, 8);
  put_le(stream, 136, ws->wmax, 4);
  put_le(stream, 140, (unsigned long long)a.pred, 4);
  for (int d = 0; d < 3; ++d) put_le(stream, 144 + 4 * d, (unsigned long long)a.bd[d], 4);
  for (int64_t i = a.off_widths + a.nb; i < a.off_heads; ++i) stream[i] = 0;
  for (int64_t i = a.off_heads + 4 * a.nb; i < a.off_chunks; ++i) stream[i] = 0;
  for (int64_t i = a.off_chunks + 8 * (a.nchunks + 1); i < a.off_payload; ++i) stream[i] = 0;
  for (int64_t i = a.off_payload + 4 * (int64_t)pw; i < total; ++i) stream[i] = 0;
}

// ------------------------------------------------------------------ host
int compress_impl(const void* d_x, int src_kind, int dtype, int ndim, const int64_t* dims, double eb,
                  double eps_given, int eb_mode, int S, int pred, const int32_t* block, void* d_stream, size_t cap,
                  void* d_ws, size_t ws_bytes, size_t* out_bytes, hc_header* hdr_out, cudaStream_t st) {
  Layout L;
  int rc = pred == HC_PRED_MEAN_ND ? make_layout_nd(ndim, dims, block, &L) : make_layout(ndim, dims, S, &L);
  if (rc) return rc;
  S = L.S;
  if (!d_x || !d_stream || !d_ws || !out_bytes) return fail(HC_ERR_INVALID_ARG, "null pointer");
  if (!aligned16(d_stream) || !aligned16(d_ws) || !aligned16(d_x)) return fail(HC_ERR_INVALID_ARG, "device buffers must be 16-byte aligned");
  if (dtype != HC_F32 && dtype != HC_F64) return fail(HC_ERR_INVALID_ARG, "dtype must be HC_F32 or HC_F64");
  if (eb_mode != HC_EB_ABS && eb_mode != HC_EB_REL) return fail(HC_ERR_INVALID_ARG, "eb_mode");
  if (pred < HC_PRED_DELTA || pred > HC_PRED_MEAN_ND) return fail(HC_ERR_INVALID_ARG, "predictor");
  if (!(eb > 0.0) || !std::isfinite(eb)) return fail(HC_ERR_INVALID_ARG, "eb must be positive and finite");
  if (cap < L.bound) return fail(HC_ERR_NOMEM, "stream buffer smaller than hc_compress_bound");
  if (ws_bytes < compress_ws_bytes(L)) return fail(HC_ERR_NOMEM, "workspace smaller than hc_compress_workspace_bytes");

  CompWs* ws = reinterpret_cast<CompWs*>(d_ws);
  uint8_t* base = reinterpret_cast<uint8_t*>(d_stream);
  OutStream o;
  o.base = base;
  o.widths = base + L.off_widths;
  o.heads = reinterpret_cast<int32_t*>(base + L.off_heads);
  o.chunks = reinterpret_cast<uint64_t*>(base + L.off_chunks);
  o.payload = reinterpret_cast<uint32_t*>(base + L.off_payload);
  o.N = L.N;
  o.nb = L.nb;
  o.nchunks = L.nchunks;
  o.S = S;
  o.G = L.G;
  o.nseg = (S + 31) / 32;
  o.pred = pred;
  for (int d = 0; d < 3; ++d) {
    o.L[d] = pred == HC_PRED_GLOBAL_DELTA ? (d == 2 ? L.N : 1) : L.dims[d];
    o.bd[d] = L.bd[d] ? L.bd[d] : 1;
    o.gd[d] = (L.dims[d] + o.bd[d] - 1) / o.bd[d];
  }

  const int sms = device_sms();
  k_ws_init<<<(unsigned)std::min<int64_t>(ceil_div(L.nchunks, kThreads) + 1, 4096), kThreads, 0, st>>>(ws, L.nchunks);
  const unsigned gblocks = (unsigned)ceil_div(L.nb, kThreads);
  const int pack_smem = (kTileChunks * L.G + 1) * 4;
  const unsigned ptiles = (unsigned)ceil_div(L.nchunks, kTileChunks);
  if (pack_smem > 48 * 1024) return fail(HC_ERR_INVALID_ARG, "block size too small for the packer");
  if (src_kind == 2) {
    SrcCodes src{reinterpret_cast<const int32_t*>(d_x)};
    // eps is given: write it through the min/max-free path
    k_eps<<<1, 1, 0, st>>>(ws, eps_given, 0);
    k_blocks<<<gblocks, kThreads, 0, st>>>(src, o, ws);
    k_chunk_scan<<<1, 1024, 0, st>>>(ws, o.chunks, L.nchunks);
    k_pack<<<ptiles, kThreads, pack_smem, st>>>(src, o, ws);
  } else if (dtype == HC_F32) {
    SrcF32 src{reinterpret_cast<const float*>(d_x)};
    if (eb_mode == HC_EB_REL) k_minmax<<<sms * 4, kThreads, 0, st>>>(src, L.N, ws);
    k_eps<<<1, 1, 0, st>>>(ws, eb, eb_mode == HC_EB_REL);
    k_blocks<<<gblocks, kThreads, 0, st>>>(src, o, ws);
    k_chunk_scan<<<1, 1024, 0, st>>>(ws, o.chunks, L.nchunks);
    k_pack<<<ptiles, kThreads, pack_smem, st>>>(src, o, ws);
  } else {
    SrcF64 src{reinterpret_cast<const double*>(d_x)};
    if (eb_mode == HC_EB_REL) k_minmax<<<sms * 4, kThreads, 0, st>>>(src, L.N, ws);
    k_eps<<<1, 1, 0, st>>>(ws, eb, eb_mode == HC_EB_REL);
    k_blocks<<<gblocks, kThreads, 0, st>>>(src, o, ws);
    k_chunk_scan<<<1, 1024, 0, st>>>(ws, o.chunks, L.nchunks);
    k_pack<<<ptiles, kThreads, pack_smem, st>>>(src, o, ws);
  }
  HeaderArgs a;
  a.dtype = dtype;
  a.ndim = ndim;
  a.S = S;
  a.G = L.G;
  a.eb_mode = eb_mode;
  a.pred = pred;
  for (int d = 0; d < 3; ++d) {
    a.dims[d] = L.dims[d];
    a.bd[d] = L.bd[d];
  }
  a.eb = eb;
  a.N = L.N;
  a.nb = L.nb;
  a.nchunks = L.nchunks;
  a.off_widths = L.off_widths;
  a.off_heads = L.off_heads;
  a.off_chunks = L.off_chunks;
  a.off_payload = L.off_payload;
  k_header<<<1, 32, 0, st>>>(a, base, ws);
  rc = check_launch("compress");
  if (rc) return rc;

  CompWs h;
  if (cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(HC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  if (h.status == HC_ERR_RANGE)
    return fail(HC_ERR_RANGE, "a code |q| >= 2^30, a residual |p| >= 2^31 or a non-finite value");
  if (h.status) return fail(h.status, "compression failed on the device");
  const int64_t total = ((L.off_payload + 4 * (int64_t)h.total_words + 16) + 15) & ~(int64_t)15;
  *out_bytes = (size_t)total;
  if (hdr_out) {
    rc = read_header_impl(d_stream, (size_t)total, hdr_out, st);
    if (rc) return rc;
  }
  return HC_OK;
}

}  // namespace hc
