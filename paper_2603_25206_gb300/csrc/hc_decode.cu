// hc_decode.cu -- multi-stage partial decompression (Algorithm 2) of a whole
// stream to a materialized stage: D_m (heads), D_p, D_q or D_f.
//
// A persistent grid walks the stream two chunks (about 8192 elements) at a
// time.  Per tile the CTA stages the widths, scans them into word offsets and
// copies the tile's payload into shared memory with 16-byte loads; each thread
// then decodes one 32-element segment serially (bit unpack, sign, in-block
// prefix sum -- or, for block-mean (HSZx) streams, the block mean added to
// each value) into a padded shared tile, which is written out with coalesced
// 16-byte stores.
#include <cstdint>

#include "hc_internal.cuh"
#include "hc_launch.h"

namespace hc {

__device__ __forceinline__ int pidx(int r) { return r + (r >> 5); }
// padded output tile: 33 words per 32 elements (conflict-free serial writes)
__host__ __device__ inline int decode_out_words(int tb, int S) { return round4(((tb * S + 31) / 32) * 33 + 4); }

template <class OutT>
struct Conv;
template <>
struct Conv<int32_t> {
  __device__ static int32_t f(int32_t q, float, double) { return q; }
};
template <>
struct Conv<float> {
  // float32 reconstruction: (float)q * (float)(2 eps) in float32 arithmetic
  __device__ static float f(int32_t q, float te, double) { return __fmul_rn(__int2float_rn(q), te); }
};
template <>
struct Conv<double> {
  __device__ static double f(int32_t q, float, double te) { return __dmul_rn((double)q, te); }
};

// KIND: HC_STAGE_P, HC_STAGE_Q or HC_STAGE_F.  SMALL: S <= 32 (one segment per block).
template <int KIND, class OutT, bool SMALL, int PRED>
__global__ void __launch_bounds__(kThreads) k_decode(DevStream s, OutT* __restrict__ out, float te_f, double te_d,
                                                      int64_t ntiles, int stage_words, int* err) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_warp[32];
  __shared__ int s_flag;
  const int tb = kTileChunks * s.G;  // blocks per tile
  const int out_words = decode_out_words(tb, s.S);
  const int nsegmax = SMALL ? tb : tb * s.nseg;
  const PipeTileSmem L =
      pipe_tile_smem(tb, stage_words, out_words + (SMALL ? 0 : nsegmax));
  uint32_t* s_off = smem + L.off;
  int32_t* s_out = reinterpret_cast<int32_t*>(smem + L.extra);
  int32_t* s_tot = s_out + out_words;
  const int tid = threadIdx.x, nt = blockDim.x;

  // two tile buffers: tile t is decoded while tile t + gridDim.x is copied in
  int64_t t = blockIdx.x;
  int bi = 0;
  TileCopy cur{}, nxt{};
  bool cur_ok = false, have_nxt = false;
  if (t < ntiles) {
    cur = tile_bounds(s, t, tb);
    cur_ok = tile_issue(s, cur, stage_words, L.w(smem, 0), L.h(smem, 0), L.words(smem, 0));
  }
  if (t + gridDim.x < ntiles) {
    nxt = tile_bounds(s, t + gridDim.x, tb);
    have_nxt = true;
  }
  for (; t < ntiles; t += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();
    bool nxt_ok = false;
    if (have_nxt) nxt_ok = tile_issue(s, nxt, stage_words, L.w(smem, bi ^ 1), L.h(smem, bi ^ 1), L.words(smem, bi ^ 1));
    TileCopy nn{};
    const bool have_nn = t + 2 * (int64_t)gridDim.x < ntiles;
    if (have_nn) nn = tile_bounds(s, t + 2 * (int64_t)gridDim.x, tb);
    const int64_t b0 = cur.b0;
    const int nblk = cur.nblk;
    const int64_t e0 = b0 * s.S;
    const int elems = (int)min((int64_t)nblk * s.S, s.N - e0);
    const int32_t* hb = L.h(smem, bi) + (int)(b0 & 3);
    TileView tv;
    const bool ok = tile_ready(s, cur, cur_ok, L.w(smem, bi), s_off, L.words(smem, bi), s_warp, &s_flag, err, tv);
    cur = nxt;
    cur_ok = nxt_ok;
    nxt = nn;
    have_nxt = have_nn;
    bi ^= 1;
    if (!ok) continue;

    const int nsegs = SMALL ? nblk : nblk * s.nseg;
    for (int seg = tid; seg < nsegs; seg += nt) {
      const int bl = SMALL ? seg : seg / s.nseg;
      const int j = SMALL ? 0 : seg - bl * s.nseg;
      const int64_t b = b0 + bl;
      const int Sb = (int)min((int64_t)s.S, s.N - b * s.S);
      const int cnt = min(32, Sb - 32 * j);
      if (cnt <= 0) continue;
      const uint32_t w = tv.w[bl];
      const int32_t head = hb[bl];
      const int r0 = bl * s.S + 32 * j;
      if constexpr (PRED == HC_PRED_MEAN) {
        // HSZx: q = M_b + p in every slot, no prefix sum (D_p holds p)
        const int32_t base = (KIND == HC_STAGE_P) ? 0 : head;
        if (w == 0) {
          for (int i = 0; i < cnt; ++i) s_out[pidx(r0 + i)] = base;
        } else {
          const uint32_t* blk = tv.words + tv.off[bl];
          unpack_any(blk + s.nseg + j * w, blk[j], w, cnt,
                     [&](int i, int32_t p) { s_out[pidx(r0 + i)] = base + p; });
        }
        continue;
      }
      int32_t acc = (KIND == HC_STAGE_P) ? 0 : (SMALL ? head : 0);
      if (w == 0) {
        for (int i = 0; i < cnt; ++i)
          s_out[pidx(r0 + i)] = (KIND == HC_STAGE_P) ? ((j == 0 && i == 0) ? head : 0) : acc;
      } else {
        const uint32_t* blk = tv.words + tv.off[bl];
        const uint32_t sw = blk[j];
        unpack_any(blk + s.nseg + j * w, sw, w, cnt, [&](int i, int32_t p) {
          if (KIND == HC_STAGE_P) {
            s_out[pidx(r0 + i)] = (j == 0 && i == 0) ? head : p;
          } else {
            acc += p;
            s_out[pidx(r0 + i)] = acc;
          }
        });
      }
      if (!SMALL && KIND != HC_STAGE_P) s_tot[seg] = acc;
    }
    __syncthreads();
    if (!SMALL && KIND != HC_STAGE_P && PRED != HC_PRED_MEAN) {
      // carry of segment j: head + totals of the block's earlier segments
      for (int seg = tid; seg < nsegs; seg += nt) {
        const int bl = seg / s.nseg, j = seg - bl * s.nseg;
        const int64_t b = b0 + bl;
        const int Sb = (int)min((int64_t)s.S, s.N - b * s.S);
        const int cnt = min(32, Sb - 32 * j);
        if (cnt <= 0) continue;
        int32_t c = hb[bl];
        for (int jj = 0; jj < j; ++jj) c += s_tot[bl * s.nseg + jj];
        const int r0 = bl * s.S + 32 * j;
        for (int i = 0; i < cnt; ++i) s_out[pidx(r0 + i)] += c;
      }
      __syncthreads();
    }
    // coalesced write-out
    OutT* dst = out + e0;
    constexpr int V = 16 / sizeof(OutT);
    int done = 0;
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
      const int nv = elems / V;
      for (int v = tid; v < nv; v += nt) {
        union {
          uint4 u;
          OutT e[V];
        } pk;
#pragma unroll
        for (int k = 0; k < V; ++k) pk.e[k] = Conv<OutT>::f(s_out[pidx(v * V + k)], te_f, te_d);
        reinterpret_cast<uint4*>(dst)[v] = pk.u;
      }
      done = nv * V;
    }
    for (int i = done + tid; i < elems; i += nt) dst[i] = Conv<OutT>::f(s_out[pidx(i)], te_f, te_d);
  }
  cp_async_wait_all();
}

__global__ void k_copy_heads(const int32_t* __restrict__ heads, int32_t* __restrict__ out, int64_t nb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __ldg(heads + i);
}

DevStream dev_stream(const hc_header* h, const void* d_stream) {
  const uint8_t* b = reinterpret_cast<const uint8_t*>(d_stream);
  DevStream s;
  s.widths = b + h->off_widths;
  s.heads = reinterpret_cast<const int32_t*>(b + h->off_heads);
  s.chunks = reinterpret_cast<const uint64_t*>(b + h->off_chunks);
  s.payload = reinterpret_cast<const uint32_t*>(b + h->off_payload);
  s.N = h->N;
  s.nb = h->nb;
  s.nchunks = h->nchunks;
  s.payload_words = h->payload_words;
  s.S = h->S;
  s.G = h->G;
  s.nseg = (h->S + 31) / 32;
  s.wmax = (int)h->wmax;
  s.gshift = (h->G & (h->G - 1)) == 0 ? __builtin_ctz((unsigned)h->G) : -1;
  s.pred = (int)h->pred;
  return s;
}

static PipeTileSmem decode_layout(const hc_header* h, bool small, int stage) {
  const int tb = kTileChunks * h->G;
  const int nseg = (h->S + 31) / 32;
  const int nsegmax = small ? tb : tb * nseg;
  return pipe_tile_smem(tb, stage, decode_out_words(tb, h->S) + (small ? 0 : nsegmax));
}

template <int KIND, class OutT, bool SMALL, int PRED>
static int launch_decode(const hc_header* h, const void* d_stream, void* d_out, int* err, cudaStream_t st) {
  const DevStream s = dev_stream(h, d_stream);
  const int stage = stage_words_for(kTileChunks * h->G, h->S, (int)h->wmax);
  const PipeTileSmem L = decode_layout(h, SMALL, stage);
  const int smem = 4 * L.total;
  auto kern = k_decode<KIND, OutT, SMALL, PRED>;
  int rc = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (rc) return rc;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  per_sm = std::max(per_sm, 1);
  const int64_t ntiles = ceil_div(h->nchunks, kTileChunks);
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)device_sms() * per_sm);
  const double te = 2.0 * h->eps;
  kern<<<grid, kThreads, smem, st>>>(s, reinterpret_cast<OutT*>(d_out), (float)te, te, ntiles, stage, err);
  return check_launch_cfg("decompress_to_stage", reinterpret_cast<const void*>(kern), grid, smem);
}

template <int KIND, class OutT, int PRED>
static int launch_decode_sp(const hc_header* h, const void* d_stream, void* d_out, int* err, cudaStream_t st) {
  if (h->S <= 32) return launch_decode<KIND, OutT, true, PRED>(h, d_stream, d_out, err, st);
  return launch_decode<KIND, OutT, false, PRED>(h, d_stream, d_out, err, st);
}

template <int KIND, class OutT>
static int launch_decode_s(const hc_header* h, const void* d_stream, void* d_out, int* err, cudaStream_t st) {
  if (h->pred == HC_PRED_MEAN) return launch_decode_sp<KIND, OutT, HC_PRED_MEAN>(h, d_stream, d_out, err, st);
  return launch_decode_sp<KIND, OutT, HC_PRED_DELTA>(h, d_stream, d_out, err, st);
}

// Every slot of a block-mean or global-predictor stream holds a residual, so
// the block-mean decoder at stage P (which adds no base) writes D_p.
int decode_residuals_impl(const hc_header* h, const void* d_stream, void* d_out, void* d_ws, cudaStream_t st) {
  if (h->pred == HC_PRED_DELTA) return fail(HC_ERR_INVALID_ARG, "delta streams keep the head in the first slot");
  int* err = &reinterpret_cast<OpWs*>(d_ws)->status;
  return launch_decode_sp<HC_STAGE_P, int32_t, HC_PRED_MEAN>(h, d_stream, d_out, err, st);
}

// Stage 1: the heads section as it is (first codes, block means or box means).
int decode_heads_impl(const hc_header* h, const void* d_stream, void* d_out, cudaStream_t st) {
  const uint8_t* b = reinterpret_cast<const uint8_t*>(d_stream);
  const int grid = (int)std::min<int64_t>(ceil_div(h->nb, kThreads), 4096);
  k_copy_heads<<<grid, kThreads, 0, st>>>(reinterpret_cast<const int32_t*>(b + h->off_heads),
                                          reinterpret_cast<int32_t*>(d_out), h->nb);
  return check_launch("decompress_to_stage(M)");
}

int decode_impl(const hc_header* h, const void* d_stream, int kind, void* d_out, int out_dtype, void* d_ws,
                cudaStream_t st) {
  if (h->pred >= HC_PRED_LORENZO) return fail(HC_ERR_INVALID_ARG, "global-predictor stream on the block decoder");
  int* err = &reinterpret_cast<OpWs*>(d_ws)->status;
  switch (kind) {
    case HC_STAGE_M:
      return decode_heads_impl(h, d_stream, d_out, st);
    case HC_STAGE_P:
      return launch_decode_s<HC_STAGE_P, int32_t>(h, d_stream, d_out, err, st);
    case HC_STAGE_Q:
      return launch_decode_s<HC_STAGE_Q, int32_t>(h, d_stream, d_out, err, st);
    case HC_STAGE_F:
      if (out_dtype == HC_F64) return launch_decode_s<HC_STAGE_F, double>(h, d_stream, d_out, err, st);
      return launch_decode_s<HC_STAGE_F, float>(h, d_stream, d_out, err, st);
    default:
      return fail(HC_ERR_INVALID_ARG, "unknown stage");
  }
}

}  // namespace hc
