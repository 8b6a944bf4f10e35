// hc_stencil_tile.cuh -- the general fused stencil tile (stream -> field):
// decode the planes of a tile with their halos into a ring of shared-memory
// slabs and apply the derivative, gradient-magnitude or Laplacian stencil
// (Section V-B, "Operation with D_q") to the integer codes.  Shared by the
// single-field kernel and the batched persistent kernel.
//
// A tile owns TY rows of all x (or of an x-range when rows are very long) for
// a range of planes; it marches along the slowest axis with a ring of three
// decoded plane slabs (the paper's Algorithm 3 sliding window, one plane per
// step instead of one block).  Each slab is the TY rows plus one halo row on
// each side, decoded from the stream through the chunk index.
#pragma once

#include <cstdint>

#include "hc_internal.cuh"
#include "hc_launch.h"

namespace hc {

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
  int op;      // StencilOp and hc_dtype of the output, read at run time by
  int out;     // the ST_RUNTIME instantiation
  float eps_f, te_f;
  double eps, te;
};

// OP / OUT template value taking the operation and output type from Geo at
// run time (one instantiation serves every kind; the branch is uniform
// across the CTA).
constexpr int ST_RUNTIME = -1;

template <int OUT>
struct OutType;
template <>
struct OutType<ST_RUNTIME> {
  using T = void;
};
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
      // explicit roundings: the same value from every kernel (no contraction)
      const double x = __ll2double_rn(a), y = __ll2double_rn(b), z = __ll2double_rn(c);
      return __dmul_rn(__dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z))), g.eps);
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
    if (s.pred == HC_PRED_MEAN) {
      // block mean (HSZx): q = M_b + p, no prefix sum and no carry
      if (w == 0) {
        for (int i = 0; i < cnt; ++i) dst[pidx(r0 + i)] = head;
      } else {
        const uint32_t* blk = tv.words + tv.off[bl];
        unpack_segment<false>(blk + s.nseg + j * w, blk[j], w, cnt,
                              [&](int i, int32_t p) { dst[pidx(r0 + i)] = head + p; });
      }
      continue;
    }
    int32_t acc = SMALL ? head : 0;
    if (w == 0) {
      for (int i = 0; i < cnt; ++i) dst[pidx(r0 + i)] = acc;
    } else {
      // compact sliding-window unpacker: the general kernel is bound by its
      // barriers, not by the unpack
      const uint32_t* blk = tv.words + tv.off[bl];
      unpack_segment<false>(blk + s.nseg + j * w, blk[j], w, cnt, [&](int i, int32_t p) {
        acc += p;
        dst[pidx(r0 + i)] = acc;
      });
    }
    if (!SMALL) s_tot[seg] = acc;
  }
  __syncthreads();
  if (!SMALL && s.pred != HC_PRED_MEAN) {
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

// Store output point i (compile-time or run-time operation and type).
template <int OP, int OUT>
__device__ __forceinline__ void store_point(const Geo& g, typename OutType<OUT>::T* out, int64_t i, int32_t c,
                                            int32_t zm, int32_t zp, int32_t ym, int32_t yp, int32_t xm, int32_t xp,
                                            int ez, int ey, int ex) {
  if constexpr (OP == ST_RUNTIME) {
#define HC_RT_CASE(O, D)                                                                                   \
  case O * 4 + D:                                                                                          \
    reinterpret_cast<typename OutType<D>::T*>(out)[i] = point<O, D>(g, c, zm, zp, ym, yp, xm, xp, ez, ey, ex); \
    break;
    switch (g.op * 4 + g.out) {
      HC_RT_CASE(ST_DERIV, HC_F32)
      HC_RT_CASE(ST_DERIV, HC_F64)
      HC_RT_CASE(ST_DERIV, HC_I64)
      HC_RT_CASE(ST_GRADMAG, HC_F32)
      HC_RT_CASE(ST_GRADMAG, HC_F64)
      HC_RT_CASE(ST_LAPLACIAN, HC_F32)
      HC_RT_CASE(ST_LAPLACIAN, HC_F64)
      HC_RT_CASE(ST_LAPLACIAN, HC_I64)
      default:
        break;
    }
#undef HC_RT_CASE
  } else {
    out[i] = point<OP, OUT>(g, c, zm, zp, ym, yp, xm, xp, ez, ey, ex);
  }
}

// Per-thread exact moments of the codes a tile owns: sum q (64-bit) and
// sum q^2 (128-bit as two words; |q| < 2^30 so q^2 < 2^60).
struct Moments {
  long long s1 = 0;
  unsigned long long lo = 0, hi = 0;
  __device__ __forceinline__ void add(int32_t q) {
    s1 += q;
    const unsigned long long v = (unsigned long long)((long long)q * q);
    lo += v;
    hi += (lo < v) ? 1ull : 0ull;
  }
  // add a 64-bit partial sum of squares (and its sum) with one carry
  __device__ __forceinline__ void add_sums(long long a1, unsigned long long a2) {
    s1 += a1;
    lo += a2;
    hi += (lo < a2) ? 1ull : 0ull;
  }
};

// Whole rows: every slot holds one contiguous decoded range; all offsets
// are 32-bit element offsets into the padded slot.
template <int OP, int OUT, bool STATS>
__device__ inline void stencil_plane_whole(const Geo& g, int64_t z, int64_t y0, int64_t y1, const int32_t* ring,
                                           long long (*s_base)[66], typename OutType<OUT>::T* out, Moments& mo) {
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
    for (int x = threadIdx.x; x < n2; x += blockDim.x) {
      const int xm = x > 0 ? x - 1 : 0, xp = x + 1 < n2 ? x + 1 : x;
      const int ex = (x == 0 || x == n2 - 1) ? 2 : 1;
      const int32_t c = pc[pidx(rc + x)];
      int32_t vzm = 0, vzp = 0, vym = 0, vyp = 0, vxm = 0, vxp = 0;
      if (OP == ST_RUNTIME || OP != ST_DERIV || g.axis == 0) {
        vzm = pm[pidx(rzm + x)];
        vzp = pp[pidx(rzp + x)];
      }
      if (OP == ST_RUNTIME || OP != ST_DERIV || g.axis == 1) {
        vym = pc[pidx(rym + x)];
        vyp = pc[pidx(ryp + x)];
      }
      if (OP == ST_RUNTIME || OP != ST_DERIV || g.axis == 2) {
        vxm = pc[pidx(rc + xm)];
        vxp = pc[pidx(rc + xp)];
      }
      store_point<OP, OUT>(g, out, erow + x, c, vzm, vzp, vym, vyp, vxm, vxp, ez, ey, ex);
      if (STATS) mo.add(c);
    }
  }
}

// Rows split along x: every row of a slot is its own decoded range.
template <int OP, int OUT, bool STATS>
__device__ inline void stencil_plane_tiled(const Geo& g, int64_t z, int64_t y0, int64_t y1, int64_t x0, int64_t x1,
                                           int64_t ylo, const int32_t* ring, int range_words, long long (*s_base)[66],
                                           typename OutType<OUT>::T* out, Moments& mo) {
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
    const int64_t erow = (z * g.n1 + y) * g.n2;
    for (int64_t x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
      const int64_t xm = x > 0 ? x - 1 : 0, xp = x + 1 < g.n2 ? x + 1 : x;
      const int ex = (x == 0 || x == g.n2 - 1) ? 2 : 1;
      const int32_t c = pc[pidx((int)(rc + x))];
      store_point<OP, OUT>(g, out, erow + x, c, pzm[pidx((int)(rzm + x))], pzp[pidx((int)(rzp + x))],
                           pym[pidx((int)(rym + x))], pyp[pidx((int)(ryp + x))], pc[pidx((int)(rc + xm))],
                           pc[pidx((int)(rc + xp))], ez, ey, ex);
      if (STATS) mo.add(c);
    }
  }
}

// One output tile (xt, yt, zt) = t of a field: decode its planes with halos
// into the ring and write every output point of the tile once.  With STATS
// the codes the tile owns are added to `mo` (each point is owned by one tile).
// smem: the dynamic shared memory (stencil_tile_words); s_warp, s_flag and
// s_base: the caller's static shared scratch.
template <int OP, int OUT, bool SMALL, bool STATS>
__device__ inline void stencil_tile(const DevStream& s, const Geo& g, int64_t t, typename OutType<OUT>::T* out,
                                    int* err, uint32_t* smem, uint32_t* s_warp, int* s_flag,
                                    long long (*s_base)[66], Moments& mo) {
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
  const int xt = (int)(t % g.nxt);
  t /= g.nxt;
  const int yt = (int)(t % g.nyt);
  const int zt = (int)(t / g.nyt);
  const int64_t x0 = (int64_t)xt * g.tx, x1 = min(x0 + g.tx, g.n2);
  const int64_t y0 = (int64_t)yt * g.ty, y1 = min(y0 + g.ty, g.n1);
  const int64_t z0 = (int64_t)zt * g.tz, z1 = min(z0 + g.tz, g.n0);
  const int64_t ylo = max(y0 - 1, (int64_t)0), yhi = min(y1 + 1, g.n1);
  const int64_t xlo = max(x0 - 1, (int64_t)0), xhi = min(x1 + 1, g.n2);
  // whole rows exactly when a tile spans the row (a slab of one row split
  // along x also has one range per slot, but each range is the x window)
  const bool whole = (g.tx == g.n2);

  // prime the ring with planes z0 - 1 and z0, then march: load z + 1, compute z
  if (z0 > 0)
    load_slab<SMALL>(s, g, z0 - 1, ylo, yhi, xlo, xhi, whole, ring, range_words, s_base, s_w, s_off, s_stage,
                     L.stage_words, s_tot, s_warp, s_flag, err);
  load_slab<SMALL>(s, g, z0, ylo, yhi, xlo, xhi, whole, ring, range_words, s_base, s_w, s_off, s_stage,
                   L.stage_words, s_tot, s_warp, s_flag, err);
  for (int64_t z = z0; z < z1; ++z) {
    if (z + 1 < g.n0)
      load_slab<SMALL>(s, g, z + 1, ylo, yhi, xlo, xhi, whole, ring, range_words, s_base, s_w, s_off, s_stage,
                       L.stage_words, s_tot, s_warp, s_flag, err);
    if (whole)
      stencil_plane_whole<OP, OUT, STATS>(g, z, y0, y1, ring, s_base, out, mo);
    else
      stencil_plane_tiled<OP, OUT, STATS>(g, z, y0, y1, x0, x1, ylo, ring, range_words, s_base, out, mo);
    __syncthreads();
  }
}


// Dynamic shared memory (words) of stencil_tile for a stream and geometry.
__host__ __device__ inline int stencil_tile_words(int S, int G, int wmax, const Geo& g) {
  const bool small = S <= 32;
  const int nseg = (S + 31) / 32;
  const int nsegmax = small ? g.nblk_max : g.nblk_max * nseg;
  return tile_smem(g.nblk_max, G - 1, S, wmax, g.nslot * g.slot_words + (small ? 0 : round4(nsegmax))).words;
}

// Host planning (hc_stencil.cu): the geometry of a field in the (possibly
// remapped) walk shape dims3, and its tiles.
Geo stencil_base_geo(const int64_t* dims3, double eps, int axis3);
int stencil_plan(const hc_header* h, Geo& g, int* smem_bytes, int ty_force, int64_t unit_elems);

}  // namespace hc
