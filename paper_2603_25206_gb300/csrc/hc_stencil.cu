// hc_stencil.cu -- numerical differentiation on the integer codes
// (Section V-B, "Operation with D_q"): derivative along one axis, gradient
// magnitude and Laplacian.
//
// Integer numerators (exact):
//   derivative  D = q[i+e] - q[i-e] inside, D = 2 (q[1] - q[0]) at an edge
//               (one-sided), 0 along an axis of length 1;   value eps * D
//   gradient    |grad| = eps * sqrt(D0^2 + D1^2 + D2^2)
//   Laplacian   L = sum_a (q[i-e_a] + q[i+e_a]) - 2 ndim q[i], edge values
//               replicated;                                   value 2 eps * L
// Fields are (n0, n1, n2) row-major with leading ones for ndim < 3, so the
// same 3-D code serves 1-D and 2-D fields (an axis of length 1 adds 0).
//
// Fused form (stream -> field, no materialized stage).  The 1-D block
// partition does not follow the rows (Section V-B), so every CTA decodes what
// it needs: a CTA owns TY rows of all x (or of an x-range when rows are very
// long) for a range of planes.  It marches along the slowest axis with a ring
// of three decoded plane slabs in shared memory (the paper's Algorithm 3
// sliding window, one plane per step instead of one block); each slab is the
// TY rows plus one halo row on each side, decoded from the stream through the
// chunk index.  The stencil reads only shared memory and writes each output
// once.
//
// Array form: the same stencils on a materialized D_q (exact) or D_f (the
// plain path, in the field's floating-point type).
#include <cstdint>
#include <cstdlib>
#include <type_traits>

#include "hc_internal.cuh"
#include "hc_launch.h"

namespace hc {

DevStream dev_stream(const hc_header* h, const void* d_stream);

__device__ __forceinline__ int pidx(int r) { return r + (r >> 5); }
__host__ __device__ inline int padded_elems_words(int elems) { return round4(((elems + 31) / 32) * 33 + 4); }

struct Geo {
  int64_t n0, n1, n2;
  int ty;      // rows per tile
  int tz;      // planes per tile
  int tx;      // x extent per tile (n2 when rows are whole)
  int nyt, nxt, nzt;
  int nslot;   // 3 (n0 > 1) or 1
  int nblk_max;  // blocks of one decoded range
  int range_elems;  // elements one range may hold (nblk_max * S)
  int ranges;  // ranges per slab: 1 with whole rows, ty + 2 otherwise
  int slot_words;
  int axis;    // derivative axis (internal, 0..2)
  float eps_f, te_f;
  double eps, te;
};

template <int OUT>
struct OutType;
template <>
struct OutType<HC_F32> {
  using T = float;
};
template <>
struct OutType<HC_F64> {
  using T = double;
};
template <>
struct OutType<HC_I64> {
  using T = long long;
};

// Scaled output of one stencil result.
template <int OP, int OUT>
__device__ __forceinline__ typename OutType<OUT>::T emit(long long a, long long b, long long c, const Geo& g) {
  if constexpr (OP == ST_DERIV) {
    if constexpr (OUT == HC_F32) return __fmul_rn(__ll2float_rn(a), g.eps_f);
    if constexpr (OUT == HC_F64) return __dmul_rn(__ll2double_rn(a), g.eps);
    if constexpr (OUT == HC_I64) return a;
  } else if constexpr (OP == ST_LAPLACIAN) {
    if constexpr (OUT == HC_F32) return __fmul_rn(__ll2float_rn(a), g.te_f);
    if constexpr (OUT == HC_F64) return __dmul_rn(__ll2double_rn(a), g.te);
    if constexpr (OUT == HC_I64) return a;
  } else {
    if constexpr (OUT == HC_F32) {
      const float x = __ll2float_rn(a), y = __ll2float_rn(b), z = __ll2float_rn(c);
      return __fmul_rn(__fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z))), g.eps_f);
    } else {
      const double x = (double)a, y = (double)b, z = (double)c;
      return sqrt(x * x + y * y + z * z) * g.eps;
    }
  }
  return 0;
}

// Decode the blocks covering elements [e0, e1) into dst (padded layout,
// element e at pidx(e - base)); returns base = first block * S.
template <bool SMALL>
__device__ inline int64_t decode_range(const DevStream& s, int64_t e0, int64_t e1, int32_t* dst, uint8_t* s_w,
                                       uint32_t* s_off, uint32_t* s_stage, int stage_words, int32_t* s_tot,
                                       uint32_t* s_warp, int* s_flag, int* err) {
  const int64_t b0 = e0 / s.S, b1 = (e1 - 1) / s.S;
  const int nblk = (int)(b1 - b0 + 1);
  TileView tv;
  if (!load_blocks(s, b0, nblk, s_w, s_off, s_stage, stage_words, s_warp, s_flag, err, tv)) return b0 * s.S;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nsegs = SMALL ? nblk : nblk * s.nseg;
  for (int seg = tid; seg < nsegs; seg += nt) {
    const int bl = SMALL ? seg : seg / s.nseg;
    const int j = SMALL ? 0 : seg - bl * s.nseg;
    const int64_t b = b0 + bl;
    const int Sb = (int)min((int64_t)s.S, s.N - b * s.S);
    const int cnt = min(32, Sb - 32 * j);
    if (cnt <= 0) continue;
    const uint32_t w = tv.w[bl];
    const int32_t head = __ldg(s.heads + b);
    const int r0 = bl * s.S + 32 * j;
    int32_t acc = SMALL ? head : 0;
    if (w == 0) {
      for (int i = 0; i < cnt; ++i) dst[pidx(r0 + i)] = acc;
    } else {
      // the general kernel keeps the compact sliding-window unpacker (the
      // pipelined kernel carries the width-specialised one)
      const uint32_t* blk = tv.words + tv.off[bl];
      unpack_segment<false>(blk + s.nseg + j * w, blk[j], w, cnt, [&](int i, int32_t p) {
        acc += p;
        dst[pidx(r0 + i)] = acc;
      });
    }
    if (!SMALL) s_tot[seg] = acc;
  }
  __syncthreads();
  if (!SMALL) {
    for (int seg = tid; seg < nsegs; seg += nt) {
      const int bl = seg / s.nseg, j = seg - bl * s.nseg;
      const int64_t b = b0 + bl;
      const int Sb = (int)min((int64_t)s.S, s.N - b * s.S);
      const int cnt = min(32, Sb - 32 * j);
      if (cnt <= 0) continue;
      int32_t c = __ldg(s.heads + b);
      for (int jj = 0; jj < j; ++jj) c += s_tot[bl * s.nseg + jj];
      const int r0 = bl * s.S + 32 * j;
      for (int i = 0; i < cnt; ++i) dst[pidx(r0 + i)] += c;
    }
    __syncthreads();
  }
  return b0 * s.S;
}

__device__ __forceinline__ int ring_slot(const Geo& g, int64_t z) { return g.nslot == 3 ? (int)(z % 3) : 0; }

// Decode plane z of the CTA's slab (rows [ylo, yhi), x range [xlo, xhi) when
// rows are split) into its ring slot.
template <bool SMALL>
__device__ inline void load_slab(const DevStream& s, const Geo& g, int64_t z, int64_t ylo, int64_t yhi, int64_t xlo,
                                 int64_t xhi, bool whole, int32_t* ring, int range_words, long long (*s_base)[66],
                                 uint8_t* s_w, uint32_t* s_off, uint32_t* s_stage, int stage_words, int32_t* s_tot,
                                 uint32_t* s_warp, int* s_flag, int* err) {
  const int slot = ring_slot(g, z);
  int32_t* dst = ring + slot * g.slot_words;
  if (whole) {
    const int64_t e0 = (z * g.n1 + ylo) * g.n2, e1 = (z * g.n1 + yhi) * g.n2;
    const int64_t base = decode_range<SMALL>(s, e0, e1, dst, s_w, s_off, s_stage, stage_words, s_tot, s_warp,
                                             s_flag, err);
    if (threadIdx.x == 0) s_base[slot][0] = base;
  } else {
    for (int64_t y = ylo; y < yhi; ++y) {
      const int ri = (int)(y - ylo);
      const int64_t row = (z * g.n1 + y) * g.n2;
      const int64_t base = decode_range<SMALL>(s, row + xlo, row + xhi, dst + ri * range_words, s_w, s_off,
                                               s_stage, stage_words, s_tot, s_warp, s_flag, err);
      if (threadIdx.x == 0) s_base[slot][ri] = base;
    }
  }
  __syncthreads();
}

// Integer stencil of one output point from its neighbours (clamped indices
// already applied by the caller) and its scaled output.
template <int OP, int OUT>
__device__ __forceinline__ typename OutType<OUT>::T point(const Geo& g, int32_t c, int32_t zm, int32_t zp,
                                                          int32_t ym, int32_t yp, int32_t xm, int32_t xp, int ez,
                                                          int ey, int ex) {
  if constexpr (OP == ST_LAPLACIAN) {
    const long long sum = (long long)zm + zp + ym + yp + xm + xp - 6ll * c;
    return emit<OP, OUT>(sum, 0, 0, g);
  } else {
    // one-sided differences at an edge are doubled: (q1 - q0) * 2
    const long long d0 = (long long)(zp - zm) * ez;
    const long long d1 = (long long)(yp - ym) * ey;
    const long long d2 = (long long)(xp - xm) * ex;
    if constexpr (OP == ST_DERIV)
      return emit<OP, OUT>(g.axis == 0 ? d0 : (g.axis == 1 ? d1 : d2), 0, 0, g);
    else
      return emit<OP, OUT>(d0, d1, d2, g);
  }
}

// Whole rows: every slot holds one contiguous decoded range; all offsets
// are 32-bit element offsets into the padded slot.
template <int OP, int OUT>
__device__ inline void stencil_plane_whole(const Geo& g, int64_t z, int64_t y0, int64_t y1, const int32_t* ring,
                                           long long (*s_base)[66], typename OutType<OUT>::T* out) {
  const int64_t zm = z > 0 ? z - 1 : 0, zp = z + 1 < g.n0 ? z + 1 : z;
  const int sc = ring_slot(g, z), sm = ring_slot(g, zm), sp = ring_slot(g, zp);
  const int32_t* pc = ring + sc * g.slot_words;
  const int32_t* pm = ring + sm * g.slot_words;
  const int32_t* pp = ring + sp * g.slot_words;
  const int n2 = (int)g.n2;
  const int ez = (z == 0 || z == g.n0 - 1) ? 2 : 1;
  for (int64_t y = y0; y < y1; ++y) {
    const int64_t erow = (z * g.n1 + y) * g.n2;
    const int rc = (int)(erow - s_base[sc][0]);
    const int rzm = (int)((zm * g.n1 + y) * g.n2 - s_base[sm][0]);
    const int rzp = (int)((zp * g.n1 + y) * g.n2 - s_base[sp][0]);
    const int rym = y > 0 ? rc - n2 : rc;
    const int ryp = y + 1 < g.n1 ? rc + n2 : rc;
    const int ey = (y == 0 || y == g.n1 - 1) ? 2 : 1;
    typename OutType<OUT>::T* orow = out + erow;
    for (int x = threadIdx.x; x < n2; x += blockDim.x) {
      const int xm = x > 0 ? x - 1 : 0, xp = x + 1 < n2 ? x + 1 : x;
      const int ex = (x == 0 || x == n2 - 1) ? 2 : 1;
      const int32_t c = pc[pidx(rc + x)];
      int32_t vzm = 0, vzp = 0, vym = 0, vyp = 0, vxm = 0, vxp = 0;
      if (OP != ST_DERIV || g.axis == 0) {
        vzm = pm[pidx(rzm + x)];
        vzp = pp[pidx(rzp + x)];
      }
      if (OP != ST_DERIV || g.axis == 1) {
        vym = pc[pidx(rym + x)];
        vyp = pc[pidx(ryp + x)];
      }
      if (OP != ST_DERIV || g.axis == 2) {
        vxm = pc[pidx(rc + xm)];
        vxp = pc[pidx(rc + xp)];
      }
      orow[x] = point<OP, OUT>(g, c, vzm, vzp, vym, vyp, vxm, vxp, ez, ey, ex);
    }
  }
}

// Rows split along x: every row of a slot is its own decoded range.
template <int OP, int OUT>
__device__ inline void stencil_plane_tiled(const Geo& g, int64_t z, int64_t y0, int64_t y1, int64_t x0, int64_t x1,
                                           int64_t ylo, const int32_t* ring, int range_words, long long (*s_base)[66],
                                           typename OutType<OUT>::T* out) {
  const int64_t zm = z > 0 ? z - 1 : 0, zp = z + 1 < g.n0 ? z + 1 : z;
  const int sc = ring_slot(g, z), sm = ring_slot(g, zm), sp = ring_slot(g, zp);
  const int ez = (z == 0 || z == g.n0 - 1) ? 2 : 1;
  for (int64_t y = y0; y < y1; ++y) {
    const int64_t ym = y > 0 ? y - 1 : 0, yp = y + 1 < g.n1 ? y + 1 : y;
    const int ey = (y == 0 || y == g.n1 - 1) ? 2 : 1;
    auto row = [&](int slot, int64_t zz, int64_t yy) -> const int32_t* {
      const int ri = (int)(yy - ylo);
      return ring + slot * g.slot_words + ri * range_words;
    };
    auto rel = [&](int slot, int64_t zz, int64_t yy) -> int64_t {
      return (zz * g.n1 + yy) * g.n2 - s_base[slot][(int)(yy - ylo)];
    };
    const int32_t *pc = row(sc, z, y), *pym = row(sc, z, ym), *pyp = row(sc, z, yp);
    const int32_t *pzm = row(sm, zm, y), *pzp = row(sp, zp, y);
    const int64_t rc = rel(sc, z, y), rym = rel(sc, z, ym), ryp = rel(sc, z, yp), rzm = rel(sm, zm, y),
                  rzp = rel(sp, zp, y);
    typename OutType<OUT>::T* orow = out + (z * g.n1 + y) * g.n2;
    for (int64_t x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
      const int64_t xm = x > 0 ? x - 1 : 0, xp = x + 1 < g.n2 ? x + 1 : x;
      const int ex = (x == 0 || x == g.n2 - 1) ? 2 : 1;
      orow[x] = point<OP, OUT>(g, pc[pidx((int)(rc + x))], pzm[pidx((int)(rzm + x))], pzp[pidx((int)(rzp + x))],
                               pym[pidx((int)(rym + x))], pyp[pidx((int)(ryp + x))], pc[pidx((int)(rc + xm))],
                               pc[pidx((int)(rc + xp))], ez, ey, ex);
    }
  }
}

template <int OP, int OUT, bool SMALL>
__global__ void __launch_bounds__(kThreads) k_stencil_stream(DevStream s, Geo g, typename OutType<OUT>::T* out,
                                                              int* err) {
  using T = typename OutType<OUT>::T;
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_warp[32];
  __shared__ int s_flag;
  __shared__ long long s_base[3][66];  // per slot, per range: base element
  const int nsegmax = SMALL ? g.nblk_max : g.nblk_max * s.nseg;
  const TileSmem L =
      tile_smem(g.nblk_max, s.G - 1, s.S, s.wmax, g.nslot * g.slot_words + (SMALL ? 0 : round4(nsegmax)));
  uint32_t* s_stage = smem;
  uint32_t* s_off = smem + L.off;
  int32_t* ring = reinterpret_cast<int32_t*>(smem + L.extra);
  int32_t* s_tot = ring + g.nslot * g.slot_words;
  uint8_t* s_w = reinterpret_cast<uint8_t*>(smem + L.w);
  const int range_words = padded_elems_words(g.range_elems);

  // tile coordinates
  int64_t t = blockIdx.x;
  const int xt = (int)(t % g.nxt);
  t /= g.nxt;
  const int yt = (int)(t % g.nyt);
  const int zt = (int)(t / g.nyt);
  const int64_t x0 = (int64_t)xt * g.tx, x1 = min(x0 + g.tx, g.n2);
  const int64_t y0 = (int64_t)yt * g.ty, y1 = min(y0 + g.ty, g.n1);
  const int64_t z0 = (int64_t)zt * g.tz, z1 = min(z0 + g.tz, g.n0);
  const int64_t ylo = max(y0 - 1, (int64_t)0), yhi = min(y1 + 1, g.n1);
  const int64_t xlo = max(x0 - 1, (int64_t)0), xhi = min(x1 + 1, g.n2);
  const bool whole = (g.ranges == 1);

  // prime the ring with planes z0 - 1 and z0, then march: load z + 1, compute z
  if (z0 > 0)
    load_slab<SMALL>(s, g, z0 - 1, ylo, yhi, xlo, xhi, whole, ring, range_words, s_base, s_w, s_off, s_stage,
                     L.stage_words, s_tot, s_warp, &s_flag, err);
  load_slab<SMALL>(s, g, z0, ylo, yhi, xlo, xhi, whole, ring, range_words, s_base, s_w, s_off, s_stage,
                   L.stage_words, s_tot, s_warp, &s_flag, err);
  for (int64_t z = z0; z < z1; ++z) {
    if (z + 1 < g.n0)
      load_slab<SMALL>(s, g, z + 1, ylo, yhi, xlo, xhi, whole, ring, range_words, s_base, s_w, s_off, s_stage,
                       L.stage_words, s_tot, s_warp, &s_flag, err);
    if (whole)
      stencil_plane_whole<OP, OUT>(g, z, y0, y1, ring, s_base, out);
    else
      stencil_plane_tiled<OP, OUT>(g, z, y0, y1, x0, x1, ylo, ring, range_words, s_base, out);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- arrays
template <class In>
struct ArrAcc {
  const In* a;
  __device__ __forceinline__ In operator()(int64_t i) const { return __ldg(a + i); }
};

// D_q input: exact integer numerators.  D_f input: the plain path computes the
// generic-flow formulas of Eq. derivatives / Eq. laplacian in the field's type.
// One CTA walks whole rows (x fastest) so no per-element division is needed.
template <int OP, int OUT, class In>
__global__ void __launch_bounds__(kThreads) k_stencil_array(const In* __restrict__ a, Geo g,
                                                             typename OutType<OUT>::T* __restrict__ out) {
  const int64_t rows = g.n0 * g.n1, pl = g.n1 * g.n2;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int64_t z = r / g.n1, y = r - z * g.n1;
    const int64_t rb = r * g.n2;
    const int64_t ym = y > 0 ? -g.n2 : 0, yp = y + 1 < g.n1 ? g.n2 : 0;
    const int64_t zm = z > 0 ? -pl : 0, zp = z + 1 < g.n0 ? pl : 0;
    const bool yedge = (y == 0 || y == g.n1 - 1), zedge = (z == 0 || z == g.n0 - 1);
    for (int64_t x = threadIdx.x; x < g.n2; x += blockDim.x) {
      const int64_t i = rb + x;
      const int64_t xm = x > 0 ? -1 : 0, xp = x + 1 < g.n2 ? 1 : 0;
      const bool xedge = (x == 0 || x == g.n2 - 1);
      if constexpr (std::is_integral<In>::value) {
        // integer codes
        if constexpr (OP == ST_LAPLACIAN) {
          const long long sum = (long long)__ldg(a + i + xm) + __ldg(a + i + xp) + __ldg(a + i + ym) +
                                __ldg(a + i + yp) + __ldg(a + i + zm) + __ldg(a + i + zp) - 6ll * __ldg(a + i);
          out[i] = emit<OP, OUT>(sum, 0, 0, g);
        } else {
          long long d0 = 0, d1 = 0, d2 = 0;
          if (OP == ST_GRADMAG || g.axis == 0) d0 = ((long long)__ldg(a + i + zp) - __ldg(a + i + zm)) * (zedge ? 2 : 1);
          if (OP == ST_GRADMAG || g.axis == 1) d1 = ((long long)__ldg(a + i + yp) - __ldg(a + i + ym)) * (yedge ? 2 : 1);
          if (OP == ST_GRADMAG || g.axis == 2) d2 = ((long long)__ldg(a + i + xp) - __ldg(a + i + xm)) * (xedge ? 2 : 1);
          if constexpr (OP == ST_DERIV)
            out[i] = emit<OP, OUT>(g.axis == 0 ? d0 : (g.axis == 1 ? d1 : d2), 0, 0, g);
          else
            out[i] = emit<OP, OUT>(d0, d1, d2, g);
        }
      } else {
        using R = typename OutType<OUT>::T;
        // floating point: (d+ - d-) / 2 inside, d1 - d0 at an edge
        auto der = [&](int64_t m, int64_t p, bool edge) -> In {
          const In v = __ldg(a + i + p) - __ldg(a + i + m);
          return edge ? v : v * In(0.5);
        };
        if constexpr (OP == ST_LAPLACIAN) {
          const In c = __ldg(a + i);
          const In v = ((__ldg(a + i + zm) + __ldg(a + i + zp)) - In(2) * c) +
                       ((__ldg(a + i + ym) + __ldg(a + i + yp)) - In(2) * c) +
                       ((__ldg(a + i + xm) + __ldg(a + i + xp)) - In(2) * c);
          out[i] = (R)v;
        } else {
          In d0 = 0, d1 = 0, d2 = 0;
          if (OP == ST_GRADMAG || g.axis == 0) d0 = g.n0 > 1 ? der(zm, zp, zedge) : In(0);
          if (OP == ST_GRADMAG || g.axis == 1) d1 = g.n1 > 1 ? der(ym, yp, yedge) : In(0);
          if (OP == ST_GRADMAG || g.axis == 2) d2 = g.n2 > 1 ? der(xm, xp, xedge) : In(0);
          if constexpr (OP == ST_DERIV)
            out[i] = (R)(g.axis == 0 ? d0 : (g.axis == 1 ? d1 : d2));
          else
            out[i] = (R)sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        }
      }
    }
  }
}

// Plain path, 4 outputs per thread (rows a multiple of 4, 16-byte aligned
// arrays): the same formulas as k_stencil_array with vector loads and stores.
template <int OP, int OUT, class In>
__global__ void __launch_bounds__(kThreads) k_stencil_array4(const In* __restrict__ a, Geo g,
                                                              typename OutType<OUT>::T* __restrict__ out) {
  using R = typename OutType<OUT>::T;
  using V4 = typename std::conditional<sizeof(In) == 4, int4, longlong4>::type;
  const int64_t rows = g.n0 * g.n1, pl = g.n1 * g.n2;
  const int nq = (int)(g.n2 / 4);
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int64_t z = r / g.n1, y = r - z * g.n1;
    const int64_t rb = r * g.n2;
    const int64_t ym = y > 0 ? -g.n2 : 0, yp = y + 1 < g.n1 ? g.n2 : 0;
    const int64_t zm = z > 0 ? -pl : 0, zp = z + 1 < g.n0 ? pl : 0;
    const bool yedge = (y == 0 || y == g.n1 - 1), zedge = (z == 0 || z == g.n0 - 1);
    for (int xq = threadIdx.x; xq < nq; xq += blockDim.x) {
      const int64_t i = rb + 4 * xq;
      In c[4], vym[4], vyp[4], vzm[4], vzp[4];
      *reinterpret_cast<V4*>(c) = *reinterpret_cast<const V4*>(a + i);
      *reinterpret_cast<V4*>(vym) = *reinterpret_cast<const V4*>(a + i + ym);
      *reinterpret_cast<V4*>(vyp) = *reinterpret_cast<const V4*>(a + i + yp);
      *reinterpret_cast<V4*>(vzm) = *reinterpret_cast<const V4*>(a + i + zm);
      *reinterpret_cast<V4*>(vzp) = *reinterpret_cast<const V4*>(a + i + zp);
      const In xl = xq > 0 ? __ldg(a + i - 1) : c[0];
      const In xr = 4 * xq + 4 < g.n2 ? __ldg(a + i + 4) : c[3];
      R res[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t x = 4 * xq + k;
        const In cm = k == 0 ? xl : c[k - 1];
        const In cp = k == 3 ? xr : c[k + 1];
        const bool xedge = (x == 0 || x == g.n2 - 1);
        if constexpr (OP == ST_LAPLACIAN) {
          const In v = ((vzm[k] + vzp[k]) - In(2) * c[k]) + ((vym[k] + vyp[k]) - In(2) * c[k]) +
                       ((cm + cp) - In(2) * c[k]);
          res[k] = (R)v;
        } else {
          auto der = [&](In m, In p, bool edge) -> In {
            const In v = p - m;
            return edge ? v : v * In(0.5);
          };
          In d0 = 0, d1 = 0, d2 = 0;
          if (OP == ST_GRADMAG || g.axis == 0) d0 = g.n0 > 1 ? der(vzm[k], vzp[k], zedge) : In(0);
          if (OP == ST_GRADMAG || g.axis == 1) d1 = g.n1 > 1 ? der(vym[k], vyp[k], yedge) : In(0);
          if (OP == ST_GRADMAG || g.axis == 2) d2 = g.n2 > 1 ? der(cm, cp, xedge) : In(0);
          if constexpr (OP == ST_DERIV)
            res[k] = (R)(g.axis == 0 ? d0 : (g.axis == 1 ? d1 : d2));
          else
            res[k] = (R)sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        }
      }
      R* o = out + i;
#pragma unroll
      for (int v = 0; v < (int)(4 * sizeof(R) / 16); ++v) reinterpret_cast<uint4*>(o)[v] = reinterpret_cast<const uint4*>(res)[v];
    }
  }
}

// ------------------------------------------------------------------ host
static Geo base_geo(const int64_t* dims3, double eps, int axis3) {
  Geo g{};
  g.n0 = dims3[0];
  g.n1 = dims3[1];
  g.n2 = dims3[2];
  g.axis = axis3;
  g.eps = eps;
  g.te = 2.0 * eps;
  g.eps_f = (float)eps;
  g.te_f = (float)(2.0 * eps);
  return g;
}

static int stream_smem_bytes(const hc_header* h, const Geo& g) {
  const bool small = h->S <= 32;
  const int nseg = (h->S + 31) / 32;
  const int nsegmax = small ? g.nblk_max : g.nblk_max * nseg;
  const TileSmem L = tile_smem(g.nblk_max, h->G - 1, h->S, (int)h->wmax,
                               g.nslot * g.slot_words + (small ? 0 : round4(nsegmax)));
  return 4 * L.words;
}

// Pick rows per tile (whole rows when they fit), planes per tile and the
// resulting shared-memory footprint.
static int plan_stream(const hc_header* h, Geo& g, int* smem_out) {
  const int S = h->S;
  const int64_t budget = 110 * 1024;  // two CTAs per SM
  const int64_t hard = 220 * 1024;
  g.nslot = g.n0 > 1 ? 3 : 1;
  auto try_plan = [&](int ty, int64_t tx) -> int {
    g.ty = ty;
    g.tx = (int)tx;
    const bool whole = (tx == g.n2);
    const int64_t rows = std::min<int64_t>(ty + 2, g.n1);
    g.ranges = whole ? 1 : (int)rows;
    const int64_t span = whole ? rows * g.n2 : std::min<int64_t>(tx + 2, g.n2);
    g.nblk_max = (int)((span + S - 1) / S + 1);
    g.range_elems = g.nblk_max * S;
    g.slot_words = g.ranges * padded_elems_words(g.range_elems);
    return stream_smem_bytes(h, g);
  };
  int bytes = 0;
  bool ok = false;
  // whole rows: largest ty in {16, 8, 4, 2, 1} within the budget, capped by n1
  for (int ty : {16, 8, 4, 2, 1}) {
    if (ty > g.n1 && ty != 1) continue;
    bytes = try_plan(ty, g.n2);
    if (bytes <= budget && g.range_elems <= (1 << 24)) {
      ok = true;
      break;
    }
  }
  if (!ok) {
    // long rows: one row per tile and an x-range per CTA
    int64_t tx = 8192;
    while (tx > 64) {
      bytes = try_plan(1, std::min<int64_t>(tx, g.n2));
      if (bytes <= budget) break;
      tx /= 2;
    }
    if (bytes > hard) return fail(HC_ERR_UNSUPPORTED, "stencil tile does not fit in shared memory");
  }
  if (g.ty > 64) return fail(HC_ERR_UNSUPPORTED, "tile too tall");
  g.nxt = (int)ceil_div(g.n2, g.tx);
  g.nyt = (int)ceil_div(g.n1, g.ty);
  const int64_t target = (int64_t)device_sms() * 4;
  const int64_t per_plane = (int64_t)g.nxt * g.nyt;
  const int64_t nzt = std::max<int64_t>(1, std::min<int64_t>(g.n0, ceil_div(target, per_plane)));
  g.tz = (int)ceil_div(g.n0, nzt);
  g.nzt = (int)ceil_div(g.n0, g.tz);
  *smem_out = bytes;
  return HC_OK;
}

template <int OP, int OUT, bool SMALL>
static int launch_stream_st(const hc_header* h, const void* d_stream, Geo g, void* d_out, int* err, cudaStream_t st) {
  int smem = 0;
  int rc = plan_stream(h, g, &smem);
  if (rc) return rc;
  auto kern = k_stencil_stream<OP, OUT, SMALL>;
  rc = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (rc) return rc;
  const int64_t grid = (int64_t)g.nxt * g.nyt * g.nzt;
  if (grid > 0x7fffffff) return fail(HC_ERR_UNSUPPORTED, "field too large");
  kern<<<(unsigned)grid, kThreads, smem, st>>>(dev_stream(h, d_stream), g,
                                                reinterpret_cast<typename OutType<OUT>::T*>(d_out), err);
  return check_launch_cfg("stencil (fused)", reinterpret_cast<const void*>(kern), grid, smem);
}

template <int OP, int OUT>
static int launch_stream_s(const hc_header* h, const void* d_stream, const Geo& g, void* d_out, int* err,
                           cudaStream_t st) {
  if (h->S <= 32) return launch_stream_st<OP, OUT, true>(h, d_stream, g, d_out, err, st);
  return launch_stream_st<OP, OUT, false>(h, d_stream, g, d_out, err, st);
}

template <int OP>
static int launch_stream_o(const hc_header* h, const void* d_stream, const Geo& g, void* d_out, int out_dtype,
                           int* err, cudaStream_t st) {
  switch (out_dtype) {
    case HC_F32:
      return launch_stream_s<OP, HC_F32>(h, d_stream, g, d_out, err, st);
    case HC_F64:
      return launch_stream_s<OP, HC_F64>(h, d_stream, g, d_out, err, st);
    case HC_I64:
      if (OP == ST_GRADMAG) return fail(HC_ERR_UNSUPPORTED, "the gradient magnitude has no integer form");
      return launch_stream_s<OP, HC_I64>(h, d_stream, g, d_out, err, st);
    default:
      return fail(HC_ERR_INVALID_ARG, "out_dtype");
  }
}

int stencil_stream_impl(const hc_header* h, const void* d_stream, int op, int axis3, void* d_out, int out_dtype,
                        void* d_ws, cudaStream_t st) {
  int* err = &reinterpret_cast<OpWs*>(d_ws)->status;
  // a 2-D field marches along its rows: (1, n1, n2) is walked as (n1, 1, n2)
  int64_t d3[3];
  stencil_walk_dims(h, d3, &axis3);
  // the pipelined kernel covers block size 32 with rows of a multiple of 8
  // codes and |q| < 2^15; everything else takes the general kernel below
  static const bool force_general = std::getenv("HC_FORCE_GENERAL_STENCIL") != nullptr;
  if (!force_general) {
    const int rc = stencil_pipe_impl(h, d_stream, d3, op, axis3, d_out, out_dtype, d_ws, st);
    if (rc != HC_ERR_UNSUPPORTED) return rc;
  }
  const Geo g = base_geo(d3, h->eps, axis3);
  switch (op) {
    case ST_DERIV:
      return launch_stream_o<ST_DERIV>(h, d_stream, g, d_out, out_dtype, err, st);
    case ST_GRADMAG:
      return launch_stream_o<ST_GRADMAG>(h, d_stream, g, d_out, out_dtype, err, st);
    default:
      return launch_stream_o<ST_LAPLACIAN>(h, d_stream, g, d_out, out_dtype, err, st);
  }
}

template <int OP, int OUT, class In>
static int launch_array(const void* d_in, const Geo& g, void* d_out, cudaStream_t st) {
  const int64_t rows = g.n0 * g.n1;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(rows, (int64_t)device_sms() * 16));
  if constexpr (!std::is_integral<In>::value) {
    if (g.n2 % 4 == 0 && aligned16(d_in) && aligned16(d_out)) {
      k_stencil_array4<OP, OUT, In><<<grid, kThreads, 0, st>>>(reinterpret_cast<const In*>(d_in), g,
                                                               reinterpret_cast<typename OutType<OUT>::T*>(d_out));
      return check_launch("stencil (array, 4-wide)");
    }
  }
  k_stencil_array<OP, OUT, In><<<grid, kThreads, 0, st>>>(reinterpret_cast<const In*>(d_in), g,
                                                          reinterpret_cast<typename OutType<OUT>::T*>(d_out));
  return check_launch("stencil (array)");
}

template <int OP, class In>
static int launch_array_o(const void* d_in, const Geo& g, void* d_out, int out_dtype, bool integer, cudaStream_t st) {
  switch (out_dtype) {
    case HC_F32:
      return launch_array<OP, HC_F32, In>(d_in, g, d_out, st);
    case HC_F64:
      return launch_array<OP, HC_F64, In>(d_in, g, d_out, st);
    case HC_I64:
      if (!integer || OP == ST_GRADMAG) return fail(HC_ERR_UNSUPPORTED, "integer output needs integer input");
      return launch_array<OP, HC_I64, In>(d_in, g, d_out, st);
    default:
      return fail(HC_ERR_INVALID_ARG, "out_dtype");
  }
}

template <class In>
static int launch_array_op(const void* d_in, const Geo& g, int op, void* d_out, int out_dtype, bool integer,
                           cudaStream_t st) {
  switch (op) {
    case ST_DERIV:
      return launch_array_o<ST_DERIV, In>(d_in, g, d_out, out_dtype, integer, st);
    case ST_GRADMAG:
      return launch_array_o<ST_GRADMAG, In>(d_in, g, d_out, out_dtype, integer, st);
    default:
      return launch_array_o<ST_LAPLACIAN, In>(d_in, g, d_out, out_dtype, integer, st);
  }
}

int stencil_array_impl(const hc_stage* in, const int64_t* dims3, double eps, int op, int axis3, void* d_out,
                       int out_dtype, void* d_ws, cudaStream_t st) {
  (void)d_ws;
  const Geo g = base_geo(dims3, eps, axis3);
  if (in->kind == HC_STAGE_Q) return launch_array_op<int32_t>(in->d_data, g, op, d_out, out_dtype, true, st);
  if (in->kind == HC_STAGE_F) {
    if (in->dtype == HC_F64) return launch_array_op<double>(in->d_data, g, op, d_out, out_dtype, false, st);
    return launch_array_op<float>(in->d_data, g, op, d_out, out_dtype, false, st);
  }
  if (in->kind == HC_STAGE_P)
    return fail(HC_ERR_UNSUPPORTED,
                "stage-2 differentiation is not defined for a 1-D block partition (Section V-B)");
  return fail(HC_ERR_INVALID_ARG, "stencils take a stream or a Q or F array");
}

}  // namespace hc

namespace hc {
// The (possibly remapped) 3-D shape the fused stencil kernels walk.
void stencil_walk_dims(const hc_header* h, int64_t d3[3], int* axis3) {
  d3[0] = h->dims[0];
  d3[1] = h->dims[1];
  d3[2] = h->dims[2];
  if (d3[0] == 1 && d3[1] > 1) {
    d3[0] = d3[1];
    d3[1] = 1;
    if (axis3 && *axis3 == 1) *axis3 = 0;
  }
}
}  // namespace hc
