// hc_global.cu -- streams of the global predictors (Section IV, "HSZp" and
// "HSZp-nd"): the prediction runs across block boundaries, so the codes are
// the prefix sums of the residuals D_p along every prediction axis,
//   q(z, y, x) = sum of p over the box [0..z] x [0..y] x [0..x]
// in the prediction shape L = (L0, L1, L2): the field's (n0, n1, n2) for the
// Lorenzo predictor (HSZp-nd), (1, 1, N) for the delta across blocks (HSZp).
//
//   stage 2 mean       k_global_mean: sum q = sum p (L0-z)(L1-y)(L2-x) while
//                      the stream is decoded (Section V-A's weighted sums),
//                      from running sums of each segment; no prefix sum
//   stage 2 derivative prefix sums of D_p over the axes other than a, then
//                      D = u(i) + u(i+e_a) (Eq. derivative_Dp as a box sum)
//   stage 2 Laplacian  per axis the same prefix sums, then the difference
//                      u(i+e_a) - u(i) accumulated (Eq. laplacian_Dp)
//   stages 3 and 4     D_q rebuilt by prefix sums along every axis
//
// The prefix sums run along one axis of an array seen as (A, L, B): element
// (a, l, b) at (a L + l) B + b -- one pass per column or per row where the
// shape allows, else chunk totals scanned by the same routine (recursion)
// and each chunk rescanned from its carry.  No kernel waits on another CTA.  The
// arithmetic is unsigned (wrapping): every value a caller reads back -- a
// code, a difference of codes -- fits 32 bits, and a wrapping sum of exact
// terms is exact modulo 2^32 whatever the intermediate sums are.
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

constexpr int kScanChunk = 32;
constexpr int64_t kScanGridCap = 152 * 32;

void global_dims(const hc_header* h, int64_t L[3]) {
  if (h->pred == HC_PRED_GLOBAL_DELTA) {
    L[0] = 1;
    L[1] = 1;
    L[2] = h->N;
  } else {
    for (int a = 0; a < 3; ++a) L[a] = h->dims[a];
  }
}

unsigned scan_grid(int64_t threads) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(threads, kThreads), kScanGridCap));
}

// ------------------------------------------------------------------ scans
// Plans, by the shape (A, L, B) of the scan:
//   L <= 32, or B > 1 with many columns: one thread per column (a, b) walks
//     l, loads coalesced across b -- one pass;
//   B == 1 (rows): one warp per chunk of 1024 codes of a row, coalesced
//     loads and a warp-shuffle scan; a row of up to 1024 codes is one pass,
//     longer rows first sum their chunks (then the same scan on the totals);
//   otherwise (few long columns): chunks of 32 along l, totals, recursion,
//     rescan from the carries.
constexpr int kRowChunk = 1024;
constexpr int64_t kColumnThreads = 152 * 256;
enum { SCAN_NONE, SCAN_COLUMN, SCAN_ROWS, SCAN_CHUNKED };

int scan_mode(int64_t A, int64_t L, int64_t B) {
  if (L <= 1 || A * B == 0) return SCAN_NONE;
  if (B == 1) return L <= kScanChunk ? SCAN_COLUMN : SCAN_ROWS;
  if (L <= kScanChunk || A * B >= kColumnThreads) return SCAN_COLUMN;
  return SCAN_CHUNKED;
}

// Walk codes [l0, l1) of one column with stride B from `run`, eight loads
// issued before their stores (the loads are independent of the running sum,
// and B >= 1 keeps every address distinct).
__device__ __forceinline__ void scan_walk(uint32_t* p, int64_t l0, int64_t l1, int64_t B, uint32_t run) {
  int64_t l = l0;
  for (; l + 8 <= l1; l += 8) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = p[(l + k) * B];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      run += v[k];
      p[(l + k) * B] = run;
    }
  }
  for (; l < l1; ++l) {
    run += p[l * B];
    p[l * B] = run;
  }
}

// one thread per column (a, b) walks l
__global__ void __launch_bounds__(kThreads) k_scan_column(uint32_t* x, int64_t A, int64_t L, int64_t B) {
  const int64_t n = A * B;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = t / B, b = t - a * B;
    scan_walk(x + a * L * B + b, 0, L, B, 0u);
  }
}

// rows: totals of the 1024-code chunks, one warp per chunk
__global__ void __launch_bounds__(kThreads) k_row_sums(const uint32_t* __restrict__ x, uint32_t* __restrict__ cs,
                                                        int64_t A, int64_t L, int64_t nc) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < A * nc; t += nw) {
    const int64_t a = t / nc, c = t - a * nc;
    const uint32_t* p = x + a * L + c * kRowChunk;
    const int len = (int)min((int64_t)kRowChunk, L - c * kRowChunk);
    uint32_t v = 0;
    for (int l = lane; l < len; l += 32) v += __ldg(p + l);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) cs[t] = v;
  }
}

// rows: each chunk scanned 32 codes at a time with warp shuffles, from the
// inclusive total of the chunks before it (cs NULL: one chunk per row)
__global__ void __launch_bounds__(kThreads) k_row_apply(uint32_t* __restrict__ x, const uint32_t* __restrict__ cs,
                                                         int64_t A, int64_t L, int64_t nc) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < A * nc; t += nw) {
    const int64_t a = t / nc, c = t - a * nc;
    uint32_t* p = x + a * L + c * kRowChunk;
    const int len = (int)min((int64_t)kRowChunk, L - c * kRowChunk);
    uint32_t carry = (cs && c > 0) ? cs[t - 1] : 0u;
    for (int j = 0; j < len; j += 32) {
      const int l = j + lane;
      uint32_t v = l < len ? p[l] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      if (l < len) p[l] = v + carry;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
  }
}

// chunk totals: cs[(a nc + c) B + b] = sum of chunk c of column (a, b)
__global__ void __launch_bounds__(kThreads) k_chunk_sums(const uint32_t* __restrict__ x, uint32_t* __restrict__ cs,
                                                          int64_t A, int64_t L, int64_t B, int64_t nc) {
  const int64_t n = A * nc * B;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t % B, r = t / B;
    const int64_t c = r % nc, a = r / nc;
    const int64_t l0 = c * kScanChunk, l1 = min(L, l0 + kScanChunk);
    const uint32_t* p = x + (a * L + l0) * B + b;
    uint32_t s = 0;
    for (int64_t l = l0; l < l1; ++l, p += B) s += __ldg(p);
    cs[t] = s;
  }
}

// rescan each chunk from the inclusive total of the chunks before it
__global__ void __launch_bounds__(kThreads) k_chunk_apply(uint32_t* __restrict__ x, const uint32_t* __restrict__ cs,
                                                           int64_t A, int64_t L, int64_t B, int64_t nc) {
  const int64_t n = A * nc * B;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t % B, r = t / B;
    const int64_t c = r % nc, a = r / nc;
    const int64_t l0 = c * kScanChunk, l1 = min(L, l0 + kScanChunk);
    scan_walk(x + a * L * B + b, l0, l1, B, c > 0 ? cs[t - B] : 0u);
  }
}

// elements of scratch a scan of (A, L, B) uses (every level rounded to 4)
int64_t scan_scratch_elems(int64_t A, int64_t L, int64_t B) {
  switch (scan_mode(A, L, B)) {
    case SCAN_ROWS: {
      const int64_t nc = ceil_div(L, kRowChunk);
      return nc == 1 ? 0 : ((A * nc + 3) & ~(int64_t)3) + scan_scratch_elems(A, nc, 1);
    }
    case SCAN_CHUNKED: {
      const int64_t nc = ceil_div(L, kScanChunk);
      return ((A * nc * B + 3) & ~(int64_t)3) + scan_scratch_elems(A, nc, B);
    }
    default:
      return 0;
  }
}

unsigned warp_grid(int64_t warps) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(warps * 32, kThreads), kScanGridCap));
}

// inclusive prefix sums along l of x seen as (A, L, B), in place
int scan_axis(uint32_t* x, int64_t A, int64_t L, int64_t B, uint32_t* scratch, cudaStream_t st) {
  switch (scan_mode(A, L, B)) {
    case SCAN_NONE:
      return HC_OK;
    case SCAN_COLUMN:
      k_scan_column<<<scan_grid(A * B), kThreads, 0, st>>>(x, A, L, B);
      return check_launch("prefix sum (columns)");
    case SCAN_ROWS: {
      const int64_t nc = ceil_div(L, kRowChunk);
      if (nc == 1) {
        k_row_apply<<<warp_grid(A), kThreads, 0, st>>>(x, nullptr, A, L, 1);
        return check_launch("prefix sum (rows)");
      }
      uint32_t* cs = scratch;
      uint32_t* next = scratch + ((A * nc + 3) & ~(int64_t)3);
      k_row_sums<<<warp_grid(A * nc), kThreads, 0, st>>>(x, cs, A, L, nc);
      int rc = check_launch("prefix sum (row chunk totals)");
      if (rc) return rc;
      if ((rc = scan_axis(cs, A, nc, 1, next, st))) return rc;
      k_row_apply<<<warp_grid(A * nc), kThreads, 0, st>>>(x, cs, A, L, nc);
      return check_launch("prefix sum (row chunks)");
    }
    default: {
      const int64_t nc = ceil_div(L, kScanChunk);
      uint32_t* cs = scratch;
      uint32_t* next = scratch + ((A * nc * B + 3) & ~(int64_t)3);
      k_chunk_sums<<<scan_grid(A * nc * B), kThreads, 0, st>>>(x, cs, A, L, B, nc);
      int rc = check_launch("prefix sum (chunk totals)");
      if (rc) return rc;
      if ((rc = scan_axis(cs, A, nc, B, next, st))) return rc;
      k_chunk_apply<<<scan_grid(A * nc * B), kThreads, 0, st>>>(x, cs, A, L, B, nc);
      return check_launch("prefix sum (chunks)");
    }
  }
}

// prefix sums along internal axis ax of an array of shape L
int scan_along(uint32_t* x, const int64_t L[3], int ax, uint32_t* scratch, cudaStream_t st) {
  if (ax == 2) return scan_axis(x, L[0] * L[1], L[2], 1, scratch, st);
  if (ax == 1) return scan_axis(x, L[0], L[1], L[2], scratch, st);
  return scan_axis(x, 1, L[0], L[1] * L[2], scratch, st);
}

int64_t max_scan_scratch_elems(const int64_t L[3]) {
  return std::max({scan_scratch_elems(L[0] * L[1], L[2], 1), scan_scratch_elems(L[0], L[1], L[2]),
                   scan_scratch_elems(1, L[0], L[1] * L[2])});
}

// Workspace carve-up after the common op workspace: the rebuilt / partial
// array W (uint32[N]), the Laplacian accumulator (int64[N]), scan scratch.
struct GlobalWs {
  uint32_t* W;
  long long* acc;
  uint32_t* scan;
};
size_t align16z(size_t x) { return (x + 15) & ~(size_t)15; }
size_t global_extra_bytes(const hc_header* h) {
  int64_t L[3];
  global_dims(h, L);
  return align16z(4 * (size_t)h->N) + align16z(8 * (size_t)h->N) + align16z(4 * (size_t)max_scan_scratch_elems(L));
}
GlobalWs global_ws(const hc_header* h, void* d_ws) {
  char* p = reinterpret_cast<char*>(d_ws) + align16z(kOpWsBytes);
  GlobalWs g;
  g.W = reinterpret_cast<uint32_t*>(p);
  p += align16z(4 * (size_t)h->N);
  g.acc = reinterpret_cast<long long*>(p);
  p += align16z(8 * (size_t)h->N);
  g.scan = reinterpret_cast<uint32_t*>(p);
  return g;
}

// ------------------------------------------------------- stage-2 mean
// Fused decode + weighted sum: tiles of two chunks, the next tile copied with
// cp.async while this one is decoded; one thread per 32-code segment adds
// p (L0 - z)(L1 - y)(L2 - x) over its positions (z, y, x) in the prediction
// shape, modulo 2^64 (the total, sum q, fits 63 bits).  A segment inside one
// row needs no per-code product: with P_j the running sums of its codes,
// sum_k p_k (L2 - x0 - k) = (L2 - x0 - cnt) P_last + sum_j P_j, two additions
// per code (32-bit when the widest block is at most 20 bits: |P| <= 2^25,
// |sum P| <= 2^30).  A segment that crosses a row end walks its positions.
template <bool SMALL, bool NARROW>
__global__ void __launch_bounds__(kThreads) k_global_mean(DevStream s, int64_t L0, int64_t L1, int64_t L2,
                                                           int64_t ntiles, int stage_words, Partial* parts,
                                                           unsigned* ticket, hc_scalar* out, double two_eps) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_warp[32];
  __shared__ int s_flag;
  __shared__ int s_err;
  const int tb = kTileChunks * s.G;
  const PipeTileSmem Lm = pipe_tile_smem(tb, stage_words, 0);
  uint32_t* s_off = smem + Lm.off;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_err = 0;
  unsigned long long acc = 0;

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
    TileView tv;
    const bool ok =
        tile_ready(s, cur, cur_ok, Lm.w(smem, bi), s_off, Lm.words(smem, bi), s_warp, &s_flag, &s_err, tv);
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
      const uint32_t w = tv.w[bl];
      if (cnt <= 0 || w == 0) continue;
      const int64_t e0 = b * s.S + 32 * j;
      int64_t x, y, z;
      if (s.N <= 0xffffffffll) {
        // 32-bit divisions (the 64-bit ones cost several times more per segment)
        const uint32_t e = (uint32_t)e0, l2 = (uint32_t)L2, l1 = (uint32_t)L1;
        const uint32_t r = e / l2, zz = r / l1;
        x = e - r * l2;
        y = r - zz * l1;
        z = zz;
      } else {
        const int64_t r = e0 / L2;
        x = e0 - r * L2;
        y = r % L1;
        z = r / L1;
      }
      unsigned long long wzy = (unsigned long long)(L0 - z) * (unsigned long long)(L1 - y);
      const uint32_t* blk = tv.words + tv.off[bl];
      if (L2 - x >= cnt) {
        using Acc = typename std::conditional<NARROW, int, long long>::type;
        Acc P = 0, R = 0;
        unpack_any(blk + s.nseg + j * w, blk[j], w, cnt, [&](int, int32_t p) {
          P += p;
          R += P;
        });
        acc += wzy * ((unsigned long long)(L2 - x - cnt) * (unsigned long long)(long long)P +
                      (unsigned long long)(long long)R);
        continue;
      }
      unpack_any(blk + s.nseg + j * w, blk[j], w, cnt, [&](int, int32_t p) {
        acc += wzy * (unsigned long long)(L2 - x) * (unsigned long long)(long long)p;
        if (++x == L2) {
          x = 0;
          if (++y == L1) {
            y = 0;
            ++z;
          }
          wzy = (unsigned long long)(L0 - z) * (unsigned long long)(L1 - y);
        }
      });
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int64_t n = s.N;
  reduce_and_finish((long long)acc, (u128)0, s_err, parts, ticket, [&](long long a, u128, int e) {
    finalize_int(out, n, a, (u128)0, false, two_eps, e);
  });
}

// ---------------------------------------------- stage-2 stencils on D_p
// Both kernels walk whole rows (CTA per row, threads along x): one thread
// splits the row index into (z, y) and shares it, so a point's position along
// the axis is the row's z or y, or x, with no division per point.
__device__ __forceinline__ void row_zy(const Geo& g, int64_t row, long long* s_zy, int64_t& z, int64_t& y) {
  if (threadIdx.x == 0) {
    s_zy[0] = row / g.n1;
    s_zy[1] = row - s_zy[0] * g.n1;
  }
  __syncthreads();
  z = s_zy[0];
  y = s_zy[1];
  __syncthreads();
}
__device__ __forceinline__ int64_t axis_pos(int ax, int64_t z, int64_t y, int x) {
  return ax == 0 ? z : (ax == 1 ? y : (int64_t)x);
}

// Derivative along internal axis ax from u = prefix sums of D_p over the
// other axes (u(i) = q(i) - q(i - e_ax) for i_ax > 0, q(i) at i_ax = 0):
// interior u(i) + u(i + e), first slice 2 u(i + e), last slice 2 u(i), an
// axis of length 1 gives 0 -- the same numerators as the stage-3 stencil.
template <int OUT>
__global__ void __launch_bounds__(kThreads) k_deriv_from_u(const uint32_t* __restrict__ u,
                                                            typename OutType<OUT>::T* __restrict__ out, Geo g,
                                                            int ax) {
  const int64_t rows = g.n0 * g.n1;
  const int n2 = (int)g.n2;
  const int64_t len = ax == 0 ? g.n0 : (ax == 1 ? g.n1 : g.n2);
  const int64_t stride = ax == 2 ? 1 : (ax == 1 ? g.n2 : g.n1 * g.n2);
  __shared__ long long s_zy[2];
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    int64_t z, y;
    row_zy(g, row, s_zy, z, y);
    for (int x = threadIdx.x; x < n2; x += blockDim.x) {
      const int64_t i = row * n2 + x, k = axis_pos(ax, z, y, x);
      long long d = 0;
      if (len > 1) {
        const long long here = (int32_t)__ldg(u + i);
        if (k == 0)
          d = 2ll * (int32_t)__ldg(u + i + stride);
        else if (k == len - 1)
          d = 2ll * here;
        else
          d = here + (int32_t)__ldg(u + i + stride);
      }
      out[i] = emit<ST_DERIV, OUT>(d, 0, 0, g);
    }
  }
}

// Laplacian term of axis ax: [i_ax < len - 1] u(i + e) - [i_ax > 0] u(i)
// (q(i+e) - q(i) minus q(i) - q(i-e), a missing neighbour replicating the
// edge), added to acc; the last axis writes the scaled result instead.
template <int OUT, bool FIRST, bool LAST>
__global__ void __launch_bounds__(kThreads) k_lap_from_u(const uint32_t* __restrict__ u, long long* __restrict__ acc,
                                                          typename OutType<OUT>::T* __restrict__ out, Geo g, int ax) {
  const int64_t rows = g.n0 * g.n1;
  const int n2 = (int)g.n2;
  const int64_t len = ax == 0 ? g.n0 : (ax == 1 ? g.n1 : g.n2);
  const int64_t stride = ax == 2 ? 1 : (ax == 1 ? g.n2 : g.n1 * g.n2);
  __shared__ long long s_zy[2];
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    int64_t z, y;
    row_zy(g, row, s_zy, z, y);
    for (int x = threadIdx.x; x < n2; x += blockDim.x) {
      const int64_t i = row * n2 + x, k = axis_pos(ax, z, y, x);
      long long v = FIRST ? 0ll : acc[i];
      if (k < len - 1) v += (int32_t)__ldg(u + i + stride);
      if (k > 0) v -= (int32_t)__ldg(u + i);
      if (LAST)
        out[i] = emit<ST_LAPLACIAN, OUT>(v, 0, 0, g);
      else
        acc[i] = v;
    }
  }
}

// Laplacian of a field with every axis of length 1: 0
template <int OUT>
__global__ void k_zero_out(typename OutType<OUT>::T* out, int64_t n, Geo g) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = emit<ST_LAPLACIAN, OUT>(0, 0, 0, g);
}

// D_f from a rebuilt D_q: (float)q * (float)(2 eps) or (double)q * 2 eps
template <class T>
__global__ void __launch_bounds__(kThreads) k_dequantize(const uint32_t* __restrict__ q, T* __restrict__ out,
                                                          int64_t n, float te_f, double te) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = (int32_t)__ldg(q + i);
    if constexpr (sizeof(T) == 4)
      out[i] = __fmul_rn(__int2float_rn(v), te_f);
    else
      out[i] = __dmul_rn((double)v, te);
  }
}

// D_q of a global-predictor stream into x (uint32[N]): residuals, then prefix
// sums along every prediction axis.
int rebuild_q(const hc_header* h, const void* d_stream, uint32_t* x, const GlobalWs& g, void* d_ws, cudaStream_t st) {
  int rc = decode_residuals_impl(h, d_stream, x, d_ws, st);
  if (rc) return rc;
  int64_t L[3];
  global_dims(h, L);
  for (int ax = 2; ax >= 0; --ax)
    if ((rc = scan_along(x, L, ax, g.scan, st))) return rc;
  return HC_OK;
}

// u = D_p with prefix sums over every internal axis but `keep` (field shape)
int partial_sums(const hc_header* h, const void* d_stream, int keep, const GlobalWs& g, void* d_ws, cudaStream_t st) {
  int rc = decode_residuals_impl(h, d_stream, g.W, d_ws, st);
  if (rc) return rc;
  const int64_t* L = h->dims;
  for (int ax = 2; ax >= 0; --ax)
    if (ax != keep && (rc = scan_along(g.W, L, ax, g.scan, st))) return rc;
  return HC_OK;
}

unsigned elem_grid(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kThreads), (int64_t)device_sms() * 16));
}

// one CTA per row (grid-stride), for the row-walking kernels
unsigned row_grid(const Geo& g) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g.n0 * g.n1, (int64_t)device_sms() * 16));
}

template <int OUT>
int stencil_p_typed(const hc_header* h, const void* d_stream, int op, int axis3, void* d_out, const GlobalWs& gw,
                    void* d_ws, cudaStream_t st) {
  using T = typename OutType<OUT>::T;
  T* out = reinterpret_cast<T*>(d_out);
  const Geo g = stencil_base_geo(h->dims, h->eps, axis3);
  const int64_t n = h->N;
  int rc;
  if (op == ST_DERIV) {
    if ((rc = partial_sums(h, d_stream, axis3, gw, d_ws, st))) return rc;
    k_deriv_from_u<OUT><<<row_grid(g), kThreads, 0, st>>>(gw.W, out, g, axis3);
    return check_launch("stage-2 derivative");
  }
  // Laplacian: one term per axis longer than 1
  int axes[3], na = 0;
  for (int ax = 0; ax < 3; ++ax)
    if (h->dims[ax] > 1) axes[na++] = ax;
  if (na == 0) {
    k_zero_out<OUT><<<elem_grid(n), kThreads, 0, st>>>(out, n, g);
    return check_launch("stage-2 Laplacian");
  }
  for (int k = 0; k < na; ++k) {
    const int ax = axes[k];
    if ((rc = partial_sums(h, d_stream, ax, gw, d_ws, st))) return rc;
    const bool first = k == 0, last = k == na - 1;
    if (first && last)
      k_lap_from_u<OUT, true, true><<<row_grid(g), kThreads, 0, st>>>(gw.W, gw.acc, out, g, ax);
    else if (first)
      k_lap_from_u<OUT, true, false><<<row_grid(g), kThreads, 0, st>>>(gw.W, gw.acc, out, g, ax);
    else if (last)
      k_lap_from_u<OUT, false, true><<<row_grid(g), kThreads, 0, st>>>(gw.W, gw.acc, out, g, ax);
    else
      k_lap_from_u<OUT, false, false><<<row_grid(g), kThreads, 0, st>>>(gw.W, gw.acc, out, g, ax);
    if ((rc = check_launch("stage-2 Laplacian"))) return rc;
  }
  return HC_OK;
}

}  // namespace

size_t global_workspace_bytes(const hc_header* h) {
  if (h->pred < HC_PRED_LORENZO) return kOpWsBytes;
  return align16z(kOpWsBytes) + global_extra_bytes(h);
}

int global_decode_impl(const hc_header* h, const void* d_stream, int kind, void* d_out, int out_dtype, void* d_ws,
                       size_t ws_bytes, cudaStream_t st) {
  if (kind == HC_STAGE_M) return fail(HC_ERR_UNSUPPORTED, "a global-predictor stream keeps no block metadata");
  if (kind == HC_STAGE_P) return decode_residuals_impl(h, d_stream, d_out, d_ws, st);
  if (ws_bytes < global_workspace_bytes(h)) return fail(HC_ERR_NOMEM, "workspace smaller than hc_workspace_bytes_for");
  const GlobalWs g = global_ws(h, d_ws);
  if (kind == HC_STAGE_Q) return rebuild_q(h, d_stream, reinterpret_cast<uint32_t*>(d_out), g, d_ws, st);
  int rc = rebuild_q(h, d_stream, g.W, g, d_ws, st);
  if (rc) return rc;
  const double te = 2.0 * h->eps;
  if (out_dtype == HC_F64)
    k_dequantize<double><<<elem_grid(h->N), kThreads, 0, st>>>(g.W, reinterpret_cast<double*>(d_out), h->N,
                                                              (float)te, te);
  else
    k_dequantize<float><<<elem_grid(h->N), kThreads, 0, st>>>(g.W, reinterpret_cast<float*>(d_out), h->N,
                                                             (float)te, te);
  return check_launch("decompress_to_stage(F)");
}

int global_stats_impl(const hc_header* h, const void* d_stream, int level, int what, hc_scalar* d_out, void* d_ws,
                      size_t ws_bytes, cudaStream_t st) {
  if (level == HC_STAGE_M) return fail(HC_ERR_UNSUPPORTED, "a global-predictor stream keeps no block metadata");
  OpWs* ws = reinterpret_cast<OpWs*>(d_ws);
  if (level == HC_STAGE_P && what == RED_MEAN && reduce32_global_mean_applies(h))
    return reduce32_global_mean_impl(h, d_stream, d_out, ws_partials(d_ws), &ws->ticket, kMaxGrid, st);
  if (level == HC_STAGE_P && what == RED_MEAN) {
    const DevStream s = dev_stream(h, d_stream);
    int64_t L[3];
    global_dims(h, L);
    const int stage = stage_words_for(kTileChunks * h->G, h->S, (int)h->wmax);
    const int smem = 4 * pipe_tile_smem(kTileChunks * h->G, stage, 0).total;
    const bool small = h->S <= 32, narrow = h->wmax <= 20;
    const void* kern = small ? (narrow ? reinterpret_cast<const void*>(k_global_mean<true, true>)
                                       : reinterpret_cast<const void*>(k_global_mean<true, false>))
                             : (narrow ? reinterpret_cast<const void*>(k_global_mean<false, true>)
                                       : reinterpret_cast<const void*>(k_global_mean<false, false>));
    int rc = ensure_smem(kern, smem);
    if (rc) return rc;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    per_sm = std::max(per_sm, 1);
    const int64_t ntiles = ceil_div(h->nchunks, kTileChunks);
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(ntiles, (int64_t)device_sms() * per_sm), kMaxGrid));
#define HC_GMEAN(SM, NA)                                                                                 \
  k_global_mean<SM, NA><<<grid, kThreads, smem, st>>>(s, L[0], L[1], L[2], ntiles, stage, ws_partials(d_ws), \
                                                      &ws->ticket, d_out, 2.0 * h->eps)
    if (small && narrow)
      HC_GMEAN(true, true);
    else if (small)
      HC_GMEAN(true, false);
    else if (narrow)
      HC_GMEAN(false, true);
    else
      HC_GMEAN(false, false);
#undef HC_GMEAN
    return check_launch_cfg("stage-2 mean (global predictor)", kern, grid, smem);
  }
  // Algorithm 4 (and level Q): q rebuilt by prefix sums, then exact s1, s2
  if (ws_bytes < global_workspace_bytes(h)) return fail(HC_ERR_NOMEM, "workspace smaller than hc_workspace_bytes_for");
  const GlobalWs g = global_ws(h, d_ws);
  int rc = rebuild_q(h, d_stream, g.W, g, d_ws, st);
  if (rc) return rc;
  hc_stage q{};
  q.kind = HC_STAGE_Q;
  q.d_data = g.W;
  q.n = h->N;
  q.qmax = h->qmax;
  return reduce_array_impl(&q, h->eps, what, d_out, d_ws, st);
}

int global_stencil_impl(const hc_header* h, const void* d_stream, int level, int op, int axis3, void* d_out,
                        int out_dtype, void* d_ws, size_t ws_bytes, cudaStream_t st) {
  if (level == HC_STAGE_M) return fail(HC_ERR_UNSUPPORTED, "stage 1 holds no point values to differentiate");
  if (ws_bytes < global_workspace_bytes(h)) return fail(HC_ERR_NOMEM, "workspace smaller than hc_workspace_bytes_for");
  const GlobalWs g = global_ws(h, d_ws);
  if (level == HC_STAGE_Q) {
    int rc = rebuild_q(h, d_stream, g.W, g, d_ws, st);
    if (rc) return rc;
    hc_stage q{};
    q.kind = HC_STAGE_Q;
    q.d_data = g.W;
    q.n = h->N;
    q.qmax = h->qmax;
    return stencil_array_impl(&q, h->dims, h->eps, op, axis3, d_out, out_dtype, d_ws, st);
  }
  if (h->pred != HC_PRED_LORENZO)
    return fail(HC_ERR_UNSUPPORTED, "stage-2 differentiation is not defined for a 1-D partition (Section V-B)");
  if (op == ST_GRADMAG)
    return fail(HC_ERR_UNSUPPORTED, "stage-2 gradient magnitude: take the derivatives at stage 2 or it at stage 3");
  switch (out_dtype) {
    case HC_F32:
      return stencil_p_typed<HC_F32>(h, d_stream, op, axis3, d_out, g, d_ws, st);
    case HC_F64:
      return stencil_p_typed<HC_F64>(h, d_stream, op, axis3, d_out, g, d_ws, st);
    case HC_I64:
      return stencil_p_typed<HC_I64>(h, d_stream, op, axis3, d_out, g, d_ws, st);
    default:
      return fail(HC_ERR_INVALID_ARG, "out_dtype");
  }
}

}  // namespace hc
