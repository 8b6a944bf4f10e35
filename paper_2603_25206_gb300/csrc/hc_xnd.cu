// hc_xnd.cu -- HSZx-nd streams (Section IV, "HSZx-nd"): the field is cut
// into boxes of b0 x b1 x b2 codes, stored in row-major order of the box grid
// (the S = b0 b1 b2 slots of a box row-major inside it), each decorrelated by
// its integer mean, p = q - M_b; slots of a box outside the field hold 0.
//
//   k_decode_box     stages 2-4 in field order: a tile's boxes are unpacked
//                    into shared memory, then written out row by row along
//                    runs of boxes (p, M_b + p, or the dequantized value)
//   k_mean_m_box     stage 1: sum_b M_b S_b with the true box sizes (Eq. mean_m)
//   k_stats_box      stages 2 and 3: per segment sum p and sum p^2, per box
//                    the S_b terms -- s1 = sum p + S_b M_b, and about a shift
//                    c0 (0, or mu~ for the stage-2 deviation) s2 = sum p^2 +
//                    2 c sum p + S_b c^2 with c = M_b - c0 (padding slots hold
//                    p = 0, so only S_b needs the true size)
//   k_box_stencil    stage-2 stencils (Section V-B, HSZx-2d, every axis): the
//                    differences of D_p plus the box means' difference where a
//                    neighbour lies in another box -- the stage-3 numerators
//                    exactly, scaled by the stage-3 stencils' own emit
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "hc_finish.cuh"
#include "hc_internal.cuh"
#include "hc_launch.h"
#include "hc_stencil_tile.cuh"

namespace hc {

DevStream dev_stream(const hc_header* h, const void* d_stream);

namespace {

// Field shape, box extents and box grid.
struct BoxGeo {
  int64_t n[3];
  int b[3];
  int64_t g[3];
};

BoxGeo box_geo(const hc_header* h) {
  BoxGeo bg;
  for (int a = 0; a < 3; ++a) {
    bg.n[a] = h->dims[a];
    bg.b[a] = (int)h->block[a];
    bg.g[a] = (bg.n[a] + bg.b[a] - 1) / bg.b[a];
  }
  return bg;
}

__device__ __forceinline__ int64_t box_true_size(const BoxGeo& bg, int64_t box) {
  const int64_t k2 = box % bg.g[2], r = box / bg.g[2];
  const int64_t k1 = r % bg.g[1], k0 = r / bg.g[1];
  return min((int64_t)bg.b[0], bg.n[0] - k0 * bg.b[0]) * min((int64_t)bg.b[1], bg.n[1] - k1 * bg.b[1]) *
         min((int64_t)bg.b[2], bg.n[2] - k2 * bg.b[2]);
}

template <int KIND, class OutT>
__device__ __forceinline__ OutT box_value(int32_t head, int32_t p, float te_f, double te) {
  if constexpr (KIND == HC_STAGE_P) {
    return (OutT)p;
  } else if constexpr (KIND == HC_STAGE_Q) {
    return (OutT)(head + p);
  } else if constexpr (sizeof(OutT) == 4) {
    return __fmul_rn(__int2float_rn(head + p), te_f);
  } else {
    return __dmul_rn((double)(head + p), te);
  }
}

// The tile walk shared by the box kernels: chunk-aligned tiles of two
// chunks, the next tile copied with cp.async while this one is processed;
// seg(b, j, cnt, w, blk, head) is called once per 32-slot segment of a box
// (w > 0: blk points at the box's staged payload).
template <bool SMALL, class F>
__device__ __forceinline__ void box_tiles(const DevStream& s, int64_t ntiles, int stage_words, int* err, F&& seg) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_warp[32];
  __shared__ int s_flag;
  const int tb = kTileChunks * s.G;
  const PipeTileSmem Lm = pipe_tile_smem(tb, stage_words, 0);
  uint32_t* s_off = smem + Lm.off;
  const int tid = threadIdx.x, nt = blockDim.x;
  int64_t t = blockIdx.x;
  int bi = 0;
  TileCopy cur{}, nxt{};
  bool cur_ok = false, have_nxt = false;
  if (t < ntiles) {
    cur = tile_bounds(s, t, tb);
    cur_ok = tile_issue(s, cur, stage_words, Lm.w(smem, 0), Lm.h(smem, 0), Lm.words(smem, 0));
  }
  if (t + gridDim.x < ntiles) {
    nxt = tile_bounds(s, t + gridDim.x, tb);
    have_nxt = true;
  }
  for (; t < ntiles; t += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();
    bool nxt_ok = false;
    if (have_nxt)
      nxt_ok = tile_issue(s, nxt, stage_words, Lm.w(smem, bi ^ 1), Lm.h(smem, bi ^ 1), Lm.words(smem, bi ^ 1));
    TileCopy nn{};
    const bool have_nn = t + 2 * (int64_t)gridDim.x < ntiles;
    if (have_nn) nn = tile_bounds(s, t + 2 * (int64_t)gridDim.x, tb);
    const int64_t b0 = cur.b0;
    const int nblk = cur.nblk;
    const int32_t* hb = Lm.h(smem, bi) + (int)(b0 & 3);
    TileView tv;
    const bool ok = tile_ready(s, cur, cur_ok, Lm.w(smem, bi), s_off, Lm.words(smem, bi), s_warp, &s_flag, err, tv);
    cur = nxt;
    cur_ok = nxt_ok;
    nxt = nn;
    have_nxt = have_nn;
    bi ^= 1;
    if (!ok) continue;
    const int nsegs = SMALL ? nblk : nblk * s.nseg;
    for (int sg = tid; sg < nsegs; sg += nt) {
      const int bl = SMALL ? sg : sg / s.nseg;
      const int j = SMALL ? 0 : sg - bl * s.nseg;
      const int cnt = min(32, s.S - 32 * j);
      const uint32_t w = tv.w[bl];
      seg(b0 + bl, j, cnt, w, w ? tv.words + tv.off[bl] : nullptr, hb[bl]);
    }
  }
  cp_async_wait_all();
  __syncthreads();
}

template <bool SMALL>
int box_tile_smem(const hc_header* h, int* stage) {
  *stage = stage_words_for(kTileChunks * h->G, h->S, (int)h->wmax);
  return 4 * pipe_tile_smem(kTileChunks * h->G, *stage, 0).total;
}

// Stages 2-4 in field order.  A tile's boxes are decoded into a staging
// buffer in shared memory (box by box, slot order, one pad word per box), then
// written out row by row: the tile's boxes form runs along x of one box row
// (k0, k1), and for each layer (s0, s1) of such a run the field codes are one
// contiguous segment, so consecutive threads store consecutive codes.
template <int KIND, class OutT, bool SMALL>
__global__ void __launch_bounds__(kThreads) k_decode_box(DevStream s, BoxGeo bg, OutT* __restrict__ out, float te_f,
                                                          double te, int64_t ntiles, int stage_words, int xshift,
                                                          int* err) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_warp[32];
  __shared__ int s_flag;
  const int tb = kTileChunks * s.G;
  const PipeTileSmem Lm = pipe_tile_smem(tb, stage_words, tb * (s.S + 1));
  uint32_t* s_off = smem + Lm.off;
  int32_t* stg = reinterpret_cast<int32_t*>(smem + Lm.extra);  // box bl, slot k at bl (S + 1) + k
  const int tid = threadIdx.x, nt = blockDim.x;
  const int S1 = s.S + 1;
  int64_t t = blockIdx.x;
  int bi = 0;
  TileCopy cur{}, nxt{};
  bool cur_ok = false, have_nxt = false;
  if (t < ntiles) {
    cur = tile_bounds(s, t, tb);
    cur_ok = tile_issue(s, cur, stage_words, Lm.w(smem, 0), Lm.h(smem, 0), Lm.words(smem, 0));
  }
  if (t + gridDim.x < ntiles) {
    nxt = tile_bounds(s, t + gridDim.x, tb);
    have_nxt = true;
  }
  for (; t < ntiles; t += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();
    bool nxt_ok = false;
    if (have_nxt)
      nxt_ok = tile_issue(s, nxt, stage_words, Lm.w(smem, bi ^ 1), Lm.h(smem, bi ^ 1), Lm.words(smem, bi ^ 1));
    TileCopy nn{};
    const bool have_nn = t + 2 * (int64_t)gridDim.x < ntiles;
    if (have_nn) nn = tile_bounds(s, t + 2 * (int64_t)gridDim.x, tb);
    const int64_t b0 = cur.b0;
    const int nblk = cur.nblk;
    const int32_t* hb = Lm.h(smem, bi) + (int)(b0 & 3);
    TileView tv;
    const bool ok = tile_ready(s, cur, cur_ok, Lm.w(smem, bi), s_off, Lm.words(smem, bi), s_warp, &s_flag, err, tv);
    cur = nxt;
    cur_ok = nxt_ok;
    nxt = nn;
    have_nxt = have_nn;
    bi ^= 1;
    if (!ok) continue;
    // decode into the staging buffer
    const int nsegs = SMALL ? nblk : nblk * s.nseg;
    for (int sg = tid; sg < nsegs; sg += nt) {
      const int bl = SMALL ? sg : sg / s.nseg;
      const int j = SMALL ? 0 : sg - bl * s.nseg;
      const int cnt = min(32, s.S - 32 * j);
      const uint32_t w = tv.w[bl];
      const int32_t head = hb[bl];
      int32_t* dst = stg + bl * S1 + 32 * j;
      if (w == 0) {
        for (int i = 0; i < cnt; ++i) dst[i] = KIND == HC_STAGE_P ? 0 : head;
      } else {
        const uint32_t* blk = tv.words + tv.off[bl];
        unpack_any(blk + s.nseg + j * w, blk[j], w, cnt,
                   [&](int i, int32_t p) { dst[i] = KIND == HC_STAGE_P ? p : head + p; });
      }
    }
    __syncthreads();
    // write out: runs of boxes along x within one box row
    int64_t b = b0;
    const int64_t bend = b0 + nblk;
    while (b < bend) {
      const int64_t k2 = b % bg.g[2], r = b / bg.g[2];
      const int64_t k1 = r % bg.g[1], k0 = r / bg.g[1];
      const int64_t run = min(bg.g[2] - k2, bend - b);  // boxes in this run
      const int64_t x0 = k2 * bg.b[2];
      const int xlen = (int)(min(bg.n[2], (k2 + run) * bg.b[2]) - x0);
      const int blr = (int)(b - b0);
      for (int s0 = 0; s0 < bg.b[0]; ++s0) {
        const int64_t z = k0 * bg.b[0] + s0;
        if (z >= bg.n[0]) break;
        for (int s1 = 0; s1 < bg.b[1]; ++s1) {
          const int64_t y = k1 * bg.b[1] + s1;
          if (y >= bg.n[1]) break;
          OutT* row = out + (z * bg.n[1] + y) * bg.n[2] + x0;
          const int lrow = (s0 * bg.b[1] + s1) * bg.b[2];
          for (int xo = tid; xo < xlen; xo += nt) {
            const int kb = xshift >= 0 ? (xo >> xshift) : xo / bg.b[2];
            const int32_t v = stg[(blr + kb) * S1 + lrow + (xo - kb * bg.b[2])];
            row[xo] = box_value<KIND == HC_STAGE_P ? HC_STAGE_Q : KIND, OutT>(0, v, te_f, te);
          }
        }
      }
      b += run;
    }
  }
  cp_async_wait_all();
}

// stage 1: T = sum_b M_b S_b; mean (T / N) 2 eps (exact = 0); mu~ = nearest(T / N)
__global__ void __launch_bounds__(kThreads) k_mean_m_box(const int32_t* __restrict__ means, BoxGeo bg, int64_t nb,
                                                          int64_t n, Partial* parts, unsigned* ticket, hc_scalar* out,
                                                          double two_eps, long long* mu) {
  long long t = 0;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x)
    t += (long long)__ldg(means + b) * box_true_size(bg, b);
  reduce_and_finish(t, (u128)0, 0, parts, ticket, [&](long long a, u128, int e) {
    out->n = n;
    out->s1 = a;
    out->s2_lo = 0;
    out->s2_hi = 0;
    out->status = e;
    out->exact = 0;
    out->mean = (__ll2double_rn(a) / (double)n) * two_eps;
    out->variance = __longlong_as_double(0x7ff8000000000000ll);
    out->std = out->variance;
    if (mu) {
      const unsigned long long m = (unsigned long long)(a < 0 ? -a : a);
      const long long r = (long long)((2ull * m + (unsigned long long)n - 1ull) / (2ull * (unsigned long long)n));
      *mu = a < 0 ? -r : r;
    }
  });
}

// stages 2 and 3.  MODE 0: mean (s1); 1: exact variance (s2 = sum q^2);
// 2: the stage-2 deviation about mu~ (s2 = sum (q - mu~)^2, read from *shift).
// NARROW: widths <= 26, so a segment's sum of p^2 fits 64 bits.
template <int MODE, bool SMALL, bool NARROW>
__global__ void __launch_bounds__(kThreads) k_stats_box(DevStream s, BoxGeo bg, int64_t ntiles, int stage_words,
                                                         Partial* parts, unsigned* ticket, hc_scalar* out,
                                                         double two_eps, const long long* shift) {
  __shared__ int s_err;
  if (threadIdx.x == 0) s_err = 0;
  const long long c0 = (MODE == 2 && shift) ? __ldcg(shift) : 0ll;
  long long S1 = 0;
  i128 S2 = 0;
  box_tiles<SMALL>(s, ntiles, stage_words, &s_err,
                   [&](int64_t b, int j, int cnt, uint32_t w, const uint32_t* blk, int32_t head) {
                     long long a1 = 0;
                     using Sq = typename std::conditional<NARROW, unsigned long long, u128>::type;
                     Sq a2 = 0;
                     if (w)
                       unpack_any(blk + s.nseg + j * w, blk[j], w, cnt, [&](int, int32_t p) {
                         a1 += p;
                         if (MODE != 0) a2 += (Sq)((long long)p * p);
                       });
                     const long long c = (long long)head - c0;
                     S1 += a1;
                     if (MODE != 0) S2 += (i128)(u128)a2 + (i128)2 * c * a1;
                     if (j == 0) {
                       const long long sb = box_true_size(bg, b);
                       S1 += sb * head;
                       if (MODE != 0) S2 += (i128)sb * c * c;
                     }
                   });
  const int64_t n = s.N;
  reduce_and_finish(S1, (u128)S2, s_err, parts, ticket, [&](long long a, u128 b2, int e) {
    if (MODE == 2)
      finalize_about(out, n, a, b2, c0, two_eps, e);
    else
      finalize_int(out, n, a, b2, MODE == 1, two_eps, e);
  });
}

// Stage-2 stencils on D_p in field order (W) and the box means (M): per
// axis, D = W[hi] - W[lo] + (M[box hi] - M[box lo] when the two neighbours
// lie in different boxes), one-sided and doubled at a domain edge, 0 on an
// axis of length 1; the Laplacian adds, per existing neighbour,
// W[nb] - W[c] + (M[box nb] - M[box c] across a box border).  A CTA walks
// whole rows (its threads along x): one thread forms the row's coordinates and
// box coordinates once per row and shares them, the box along x comes from a
// shift when its extent is a power of two, and a neighbour crosses into the
// next box only from a box's first or last layer, so no neighbour needs a
// division.
template <int OP, int OUT>
__global__ void __launch_bounds__(kThreads) k_box_stencil(const int32_t* __restrict__ W, const int32_t* __restrict__ M,
                                                           BoxGeo bg, Geo g, int xshift,
                                                           typename OutType<OUT>::T* __restrict__ out) {
  const int64_t rows = bg.n[0] * bg.n[1];
  const int n2 = (int)bg.n[2];
  const int64_t st[3] = {bg.n[1] * bg.n[2], bg.n[2], 1};   // element strides
  const int64_t gs[3] = {bg.g[1] * bg.g[2], bg.g[2], 1};   // box-index strides
  __shared__ long long s_row[4];  // z, y, box index of x = 0, (ry << 32) | rz
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    if (threadIdx.x == 0) {
      const int64_t zz = row / bg.n[1], yy = row - zz * bg.n[1];
      const int64_t kz = zz / bg.b[0], ky = yy / bg.b[1];
      s_row[0] = zz;
      s_row[1] = yy;
      s_row[2] = kz * gs[0] + ky * gs[1];
      s_row[3] = ((long long)(yy - ky * bg.b[1]) << 32) | (long long)(zz - kz * bg.b[0]);
    }
    __syncthreads();
    const int64_t z = s_row[0], y = s_row[1], brow = s_row[2];
    const int rz = (int)(s_row[3] & 0xffffffffll), ry = (int)(s_row[3] >> 32);
    __syncthreads();  // every thread has read the row before thread 0 moves on
    const int64_t i0 = row * n2;
    for (int x = threadIdx.x; x < n2; x += blockDim.x) {
      const int kx = xshift >= 0 ? (x >> xshift) : x / bg.b[2];
      const int64_t c[3] = {z, y, x};
      const int r[3] = {rz, ry, x - kx * bg.b[2]};
      const int64_t bc = brow + kx;
      const int64_t i = i0 + x;
      if constexpr (OP == ST_LAPLACIAN) {
        const long long wc = __ldg(W + i), mc = __ldg(M + bc);
        long long v = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (c[a] > 0) {  // lower neighbour (a missing one replicates the edge: term 0)
            v += (long long)__ldg(W + i - st[a]) - wc;
            if (r[a] == 0) v += (long long)__ldg(M + bc - gs[a]) - mc;
          }
          if (c[a] + 1 < bg.n[a]) {
            v += (long long)__ldg(W + i + st[a]) - wc;
            if (r[a] == bg.b[a] - 1) v += (long long)__ldg(M + bc + gs[a]) - mc;
          }
        }
        out[i] = emit<OP, OUT>(v, 0, 0, g);
      } else {
        long long d[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (OP == ST_DERIV && a != g.axis) continue;
          const int64_t len = bg.n[a], k = c[a];
          if (len == 1) continue;
          const bool lo_step = k > 0, hi_step = k + 1 < len;  // one-sided at an edge
          long long v = (long long)__ldg(W + i + (hi_step ? st[a] : 0)) - __ldg(W + i - (lo_step ? st[a] : 0));
          const bool lo_cross = lo_step && r[a] == 0, hi_cross = hi_step && r[a] == bg.b[a] - 1;
          if (lo_cross || hi_cross)
            v += (long long)__ldg(M + bc + (hi_cross ? gs[a] : 0)) - __ldg(M + bc - (lo_cross ? gs[a] : 0));
          d[a] = (lo_step && hi_step) ? v : 2 * v;
        }
        if constexpr (OP == ST_DERIV)
          out[i] = emit<OP, OUT>(d[g.axis], 0, 0, g);
        else
          out[i] = emit<OP, OUT>(d[0], d[1], d[2], g);
      }
    }
  }
}

int tile_grid(const void* kern, int smem, int64_t ntiles) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  per_sm = std::max(per_sm, 1);
  return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(ntiles, (int64_t)device_sms() * per_sm),
                                                     kMaxGrid));
}

template <int KIND, class OutT, bool SMALL>
int launch_decode_box(const hc_header* h, const void* d_stream, void* d_out, int* err, cudaStream_t st) {
  const int stage = stage_words_for(kTileChunks * h->G, h->S, (int)h->wmax);
  const int tb = kTileChunks * h->G;
  const int smem = 4 * pipe_tile_smem(tb, stage, tb * (h->S + 1)).total;
  const int xshift = (h->block[2] & (h->block[2] - 1)) == 0 ? __builtin_ctz(h->block[2]) : -1;
  auto kern = k_decode_box<KIND, OutT, SMALL>;
  int rc = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (rc) return rc;
  const int64_t ntiles = ceil_div(h->nchunks, kTileChunks);
  const int grid = tile_grid(reinterpret_cast<const void*>(kern), smem, ntiles);
  const double te = 2.0 * h->eps;
  kern<<<grid, kThreads, smem, st>>>(dev_stream(h, d_stream), box_geo(h), reinterpret_cast<OutT*>(d_out),
                                     (float)te, te, ntiles, stage, xshift, err);
  return check_launch_cfg("decompress_to_stage (boxes)", reinterpret_cast<const void*>(kern), grid, smem);
}

template <int KIND, class OutT>
int launch_decode_box_s(const hc_header* h, const void* d_stream, void* d_out, int* err, cudaStream_t st) {
  if (h->S <= 32) return launch_decode_box<KIND, OutT, true>(h, d_stream, d_out, err, st);
  return launch_decode_box<KIND, OutT, false>(h, d_stream, d_out, err, st);
}

template <int MODE, bool SMALL, bool NARROW>
int launch_stats_box(const hc_header* h, const void* d_stream, hc_scalar* d_out, void* d_ws, const long long* shift,
                     cudaStream_t st) {
  int stage = 0;
  const int smem = box_tile_smem<SMALL>(h, &stage);
  auto kern = k_stats_box<MODE, SMALL, NARROW>;
  int rc = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (rc) return rc;
  const int64_t ntiles = ceil_div(h->nchunks, kTileChunks);
  const int grid = tile_grid(reinterpret_cast<const void*>(kern), smem, ntiles);
  OpWs* ws = reinterpret_cast<OpWs*>(d_ws);
  kern<<<grid, kThreads, smem, st>>>(dev_stream(h, d_stream), box_geo(h), ntiles, stage, ws_partials(d_ws),
                                     &ws->ticket, d_out, 2.0 * h->eps, shift);
  return check_launch_cfg("statistics (boxes)", reinterpret_cast<const void*>(kern), grid, smem);
}

template <int MODE>
int launch_stats_box_m(const hc_header* h, const void* d_stream, hc_scalar* d_out, void* d_ws,
                       const long long* shift, cudaStream_t st) {
  const bool small = h->S <= 32, narrow = h->wmax <= 26;
  if (small && narrow) return launch_stats_box<MODE, true, true>(h, d_stream, d_out, d_ws, shift, st);
  if (small) return launch_stats_box<MODE, true, false>(h, d_stream, d_out, d_ws, shift, st);
  if (narrow) return launch_stats_box<MODE, false, true>(h, d_stream, d_out, d_ws, shift, st);
  return launch_stats_box<MODE, false, false>(h, d_stream, d_out, d_ws, shift, st);
}

int launch_mean_m_box(const hc_header* h, const void* d_stream, hc_scalar* d_out, void* d_ws, long long* mu,
                      cudaStream_t st) {
  const int32_t* means = reinterpret_cast<const int32_t*>(reinterpret_cast<const uint8_t*>(d_stream) + h->off_heads);
  OpWs* ws = reinterpret_cast<OpWs*>(d_ws);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(h->nb, kThreads), 1024));
  k_mean_m_box<<<grid, kThreads, 0, st>>>(means, box_geo(h), h->nb, h->N, ws_partials(d_ws), &ws->ticket, d_out,
                                          2.0 * h->eps, mu);
  return check_launch("mean (stage 1, boxes)");
}

template <int OP>
int launch_box_stencil(const hc_header* h, const int32_t* W, const int32_t* M, int axis3, void* d_out, int out_dtype,
                       cudaStream_t st) {
  const Geo g = stencil_base_geo(h->dims, h->eps, axis3);
  const BoxGeo bg = box_geo(h);
  if (h->dims[2] > 0x7fffffff) return fail(HC_ERR_UNSUPPORTED, "rows longer than 2^31 codes");
  const int xshift = (bg.b[2] & (bg.b[2] - 1)) == 0 ? __builtin_ctz((unsigned)bg.b[2]) : -1;
  const unsigned grid =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>(bg.n[0] * bg.n[1], (int64_t)device_sms() * 16));
  switch (out_dtype) {
    case HC_F32:
      k_box_stencil<OP, HC_F32><<<grid, kThreads, 0, st>>>(W, M, bg, g, xshift, reinterpret_cast<float*>(d_out));
      break;
    case HC_F64:
      k_box_stencil<OP, HC_F64><<<grid, kThreads, 0, st>>>(W, M, bg, g, xshift, reinterpret_cast<double*>(d_out));
      break;
    case HC_I64:
      if (OP == ST_GRADMAG) return fail(HC_ERR_UNSUPPORTED, "the gradient magnitude has no integer form");
      k_box_stencil<OP, HC_I64><<<grid, kThreads, 0, st>>>(W, M, bg, g, xshift,
                                                           reinterpret_cast<long long*>(d_out));
      break;
    default:
      return fail(HC_ERR_INVALID_ARG, "out_dtype");
  }
  return check_launch("stage-2 stencil (boxes)");
}

size_t align16z(size_t x) { return (x + 15) & ~(size_t)15; }
int32_t* box_scratch(void* d_ws) { return reinterpret_cast<int32_t*>(reinterpret_cast<char*>(d_ws) + align16z(kOpWsBytes)); }

}  // namespace

size_t xnd_workspace_bytes(const hc_header* h) { return align16z(kOpWsBytes) + align16z(4 * (size_t)h->N); }

int xnd_decode_impl(const hc_header* h, const void* d_stream, int kind, void* d_out, int out_dtype, void* d_ws,
                    size_t ws_bytes, cudaStream_t st) {
  (void)ws_bytes;
  int* err = &reinterpret_cast<OpWs*>(d_ws)->status;
  switch (kind) {
    case HC_STAGE_M:
      return decode_heads_impl(h, d_stream, d_out, st);
    case HC_STAGE_P:
      return launch_decode_box_s<HC_STAGE_P, int32_t>(h, d_stream, d_out, err, st);
    case HC_STAGE_Q:
      return launch_decode_box_s<HC_STAGE_Q, int32_t>(h, d_stream, d_out, err, st);
    case HC_STAGE_F:
      if (out_dtype == HC_F64) return launch_decode_box_s<HC_STAGE_F, double>(h, d_stream, d_out, err, st);
      return launch_decode_box_s<HC_STAGE_F, float>(h, d_stream, d_out, err, st);
    default:
      return fail(HC_ERR_INVALID_ARG, "unknown stage");
  }
}

int xnd_stats_impl(const hc_header* h, const void* d_stream, int level, int what, hc_scalar* d_out, void* d_ws,
                   size_t ws_bytes, cudaStream_t st) {
  (void)ws_bytes;
  if (level == HC_STAGE_M) {
    if (what != RED_MEAN) return fail(HC_ERR_UNSUPPORTED, "stage 1 gives the mean only (Eq. mean_m)");
    return launch_mean_m_box(h, d_stream, d_out, d_ws, nullptr, st);
  }
  // boxes of 64 or 128 slots with narrow widths: the warp-autonomous
  // statistics kernel of hc_reduce32.cu; else the tile kernel k_stats_box
  OpWs* ws = reinterpret_cast<OpWs*>(d_ws);
  const bool r32 = reduce32_box_applies(h);
  Partial* parts = ws_partials(d_ws);
  if (what == RED_MEAN)
    return r32 ? reduce32_box_impl(h, d_stream, RED_MEAN, d_out, parts, &ws->ticket, kMaxGrid, nullptr, st)
               : launch_stats_box_m<0>(h, d_stream, d_out, d_ws, nullptr, st);
  if (level == HC_STAGE_P) {
    // Section V-A: the deviations about the integer mean mu~ of stage 1
    long long* mu = reinterpret_cast<long long*>(&ws->pad[0]);
    int rc = launch_mean_m_box(h, d_stream, d_out, d_ws, mu, st);
    if (rc) return rc;
    return r32 ? reduce32_box_impl(h, d_stream, RED_VAR, d_out, parts, &ws->ticket, kMaxGrid, mu, st)
               : launch_stats_box_m<2>(h, d_stream, d_out, d_ws, mu, st);
  }
  return r32 ? reduce32_box_impl(h, d_stream, RED_VAR, d_out, parts, &ws->ticket, kMaxGrid, nullptr, st)
             : launch_stats_box_m<1>(h, d_stream, d_out, d_ws, nullptr, st);
}

int xnd_stencil_impl(const hc_header* h, const void* d_stream, int level, int op, int axis3, void* d_out,
                     int out_dtype, void* d_ws, size_t ws_bytes, cudaStream_t st) {
  if (level == HC_STAGE_M) return fail(HC_ERR_UNSUPPORTED, "stage 1 holds no point values to differentiate");
  if (ws_bytes < xnd_workspace_bytes(h)) return fail(HC_ERR_NOMEM, "workspace smaller than hc_workspace_bytes_for");
  int32_t* W = box_scratch(d_ws);
  int* err = &reinterpret_cast<OpWs*>(d_ws)->status;
  // one pass when the march tile applies; else decode to an array, then the stencil
  const int rc1 = xnd_march_impl(h, d_stream, level, op, axis3, d_out, out_dtype, d_ws, W,
                                 ws_bytes - align16z(kOpWsBytes), st);
  if (rc1 != HC_ERR_UNSUPPORTED) return rc1;
  if (level == HC_STAGE_Q) {
    int rc = launch_decode_box_s<HC_STAGE_Q, int32_t>(h, d_stream, W, err, st);
    if (rc) return rc;
    hc_stage q{};
    q.kind = HC_STAGE_Q;
    q.d_data = W;
    q.n = h->N;
    q.qmax = h->qmax;
    return stencil_array_impl(&q, h->dims, h->eps, op, axis3, d_out, out_dtype, d_ws, st);
  }
  int rc = launch_decode_box_s<HC_STAGE_P, int32_t>(h, d_stream, W, err, st);
  if (rc) return rc;
  const int32_t* M = reinterpret_cast<const int32_t*>(reinterpret_cast<const uint8_t*>(d_stream) + h->off_heads);
  switch (op) {
    case ST_DERIV:
      return launch_box_stencil<ST_DERIV>(h, W, M, axis3, d_out, out_dtype, st);
    case ST_GRADMAG:
      return launch_box_stencil<ST_GRADMAG>(h, W, M, axis3, d_out, out_dtype, st);
    default:
      return launch_box_stencil<ST_LAPLACIAN>(h, W, M, axis3, d_out, out_dtype, st);
  }
}

}  // namespace hc
