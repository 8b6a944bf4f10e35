// hc_stencil_pipe.cuh -- the pipelined fused stream -> stencil tile for the
// common case: block size 32 and codes |q| < 2^15 (the header's max |q| says
// so).  Same results as the general tile (Section V-B, "Operation with D_q").
// Shared by the one-field kernel and the batched persistent kernel.
//
// One CTA owns TY whole rows for a range of planes and marches along the
// slowest axis (the sliding window of Algorithm 3, one plane slab per step).
// Warp 0 is a loader; warps 1..7 decode and compute:
//   step k:  loader   wait for the copies issued two steps before, scan the
//                     widths of slab k+3, cp.async its payload and heads and
//                     the widths of slab k+5 (so every copy has two whole
//                     steps to land: a step is often shorter than a DRAM
//                     round trip);
//            workers  decode slab k into ring slot k % 4 and compute every
//                     output plane whose three slabs are ready (normally the
//                     plane of slab k-2);
//            one __syncthreads.
// Buffers: 4 ring slots, 4 payload and heads stages, 6 widths buffers.  A work item
// is V = 8 (rows a multiple of 8) or V = 4 (a multiple of 4) consecutive
// outputs of one row, or for rows of any length (V = 0) 8 outputs at any
// offset with unaligned loads, and the rows' last n2 % 8 outputs one by one.
// Decoded codes are stored as int16, a 32-code segment as 64 contiguous
// bytes: a decoding thread writes its segment with four 16-byte stores and a
// stencil thread reads V consecutive codes of a row with one load
// (consecutive threads read consecutive bytes: no bank conflicts).
#pragma once

#include <cstdint>
#include <type_traits>

#include "hc_group.cuh"
#include "hc_internal.cuh"
#include "hc_launch.h"
#include "hc_stencil_tile.cuh"

namespace hc {

constexpr int kWorkers = kThreads - 32;
constexpr int kSlots = 4;
constexpr int kWorkerWarps = kWorkers / 32;
// Estimated thread instructions per decoded code and per output point (from
// ncu instruction counts of the kernels): decoding with the grouped unpacker
// costs about 10 per code, a point about 25 for one operation, about 40 with
// the run-time operation dispatch and exact sums of the batched tiles, and
// about 100 for all operations.
constexpr int kDecodeCost = 10;
constexpr int kPointCost = 25;
constexpr int kPointCostRuntime = 40;  // run-time operation dispatch plus the exact sums (batched tiles)
constexpr int kPointCostMulti = 100;

struct PGeo {
  int64_t n0, n1, n2;
  int ty, tz, nyt, nzt;
  int nblk_max;     // blocks of one slab
  int pre_max;      // widths bytes staged per slab (G - 1 + nblk_max, rounded to 16)
  int heads_max;    // heads staged per slab (nblk_max + 4, rounded to 4)
  int stage_words;  // payload words per stage buffer
  int slot_bytes;   // nblk_max * 64
  int axis;
  int op, out;        // operation and output type for the ST_RUNTIME instantiation
  void* mout[5];      // ST_MULTI outputs (NULL: not wanted): the derivative along
                      // internal axes 0, 1, 2, the gradient magnitude, the Laplacian
  unsigned nq_magic;  // ceil(2^32 / nq) for the row/item split (unused when nq == 1)
  int nq;             // items per row: n2 / V
  int grp;            // group size of the grouped unpacker (group_for_width of the stream's max width)
  int waves;          // plane ranges for about this many waves of resident CTAs (1 or 2, tuned)
  float eps_f, te_f;
  double eps, te;
};

template <int OUT>
struct OT;
template <>
struct OT<ST_RUNTIME> {
  using T = void;
};
template <>
struct OT<HC_F32> {
  using T = float;
};
template <>
struct OT<HC_F64> {
  using T = double;
};
template <>
struct OT<HC_I64> {
  using T = long long;
};

template <int OP, int OUT>
__device__ __forceinline__ typename OT<OUT>::T emit1(int a, int b, int c, const PGeo& g) {
  if constexpr (OP == ST_DERIV) {
    if constexpr (OUT == HC_F32) return __fmul_rn(__int2float_rn(a), g.eps_f);
    if constexpr (OUT == HC_F64) return __dmul_rn((double)a, g.eps);
    if constexpr (OUT == HC_I64) return (long long)a;
  } else if constexpr (OP == ST_LAPLACIAN) {
    if constexpr (OUT == HC_F32) return __fmul_rn(__int2float_rn(a), g.te_f);
    if constexpr (OUT == HC_F64) return __dmul_rn((double)a, g.te);
    if constexpr (OUT == HC_I64) return (long long)a;
  } else {
    if constexpr (OUT == HC_F32) {
      const float x = __int2float_rn(a), y = __int2float_rn(b), z = __int2float_rn(c);
      return __fmul_rn(__fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z))), g.eps_f);
    } else {
      // explicit roundings: the same value from every kernel (no contraction)
      const double x = (double)a, y = (double)b, z = (double)c;
      return __dmul_rn(__dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z))), g.eps);
    }
  }
  return 0;
}

// Copy pipeline depth: the payload and heads of slab j are copied three
// steps before slab j is decoded (kStages buffers), its widths five steps
// before (kWidthBufs buffers: scanned two steps after they were copied), so
// every copy has at least two whole steps to land.
constexpr int kStages = 4;
constexpr int kWidthBufs = 6;

// Shared-memory carve-up (byte offsets), computed identically on both sides:
// the ring of decoded slots, the payload stages, the widths, heads and
// block offsets of the slabs in flight.
struct PSmem {
  int ring, stage, wb, hb, ob, total;
  int ob_bytes;  // one offsets buffer
};
__host__ __device__ inline PSmem psmem(const PGeo& g) {
  PSmem p;
  p.ring = 0;
  p.stage = p.ring + kSlots * g.slot_bytes;
  p.wb = p.stage + kStages * 4 * g.stage_words;
  p.hb = p.wb + kWidthBufs * g.pre_max;
  p.ob = p.hb + kStages * 4 * g.heads_max;
  p.ob_bytes = (4 * (g.nblk_max + 4) + 15) & ~15;
  p.total = p.ob + kStages * p.ob_bytes;
  return p;
}

struct SlabDesc {
  int64_t b0;   // first block
  int nblk;     // blocks
  int npre;     // widths before b0 in its chunk
  int64_t cs;   // chunk start block
};

__device__ __forceinline__ SlabDesc slab_desc(const DevStream& s, const PGeo& g, int64_t z, int64_t ylo,
                                              int64_t yhi) {
  SlabDesc d;
  const int64_t e0 = (z * g.n1 + ylo) * g.n2, e1 = (z * g.n1 + yhi) * g.n2;
  d.b0 = e0 >> 5;
  d.nblk = (int)(((e1 - 1) >> 5) - d.b0 + 1);
  d.cs = d.b0 & ~(int64_t)127;  // G = 128 blocks per chunk at S = 32
  d.npre = (int)(d.b0 - d.cs);
  return d;
}

// The V outputs of one work item from their neighbourhoods (compile-time
// operation O and output type D), written with vector stores when they fill
// 16 bytes and AL (the item's first output is aligned to its size).  cm / cp
// are the x neighbours of the first / last point.
template <int O, int D, int V, bool AL>
__device__ __forceinline__ void emit_items(const PGeo& g, typename OT<D>::T* o, const short* c, const short* a,
                                           const short* b, const short* zmv, const short* zpv, int xl, int xr,
                                           int ex0, int exn, int ez, int ey) {
  using T = typename OT<D>::T;
  T res[V];
#pragma unroll
  for (int i = 0; i < V; ++i) {
    const int cm = i == 0 ? xl : c[i - 1];
    const int cp = i == V - 1 ? xr : c[i + 1];
    if constexpr (O == ST_LAPLACIAN) {
      const int l = (int)zmv[i] + zpv[i] + a[i] + b[i] + cm + cp - 6 * (int)c[i];
      res[i] = emit1<O, D>(l, 0, 0, g);
    } else {
      int ex = 1;
      if (i == 0) ex = ex0;
      if (i == V - 1) ex = ex * exn;
      int d0 = 0, d1 = 0, d2 = 0;
      if (O == ST_GRADMAG || g.axis == 0) d0 = ((int)zpv[i] - zmv[i]) * ez;
      if (O == ST_GRADMAG || g.axis == 1) d1 = ((int)b[i] - a[i]) * ey;
      if (O == ST_GRADMAG || g.axis == 2) d2 = (cp - cm) * ex;
      if constexpr (O == ST_DERIV)
        res[i] = emit1<O, D>(g.axis == 0 ? d0 : (g.axis == 1 ? d1 : d2), 0, 0, g);
      else
        res[i] = emit1<O, D>(d0, d1, d2, g);
    }
  }
  if constexpr (AL && V * sizeof(T) >= 16) {
#pragma unroll
    for (int v = 0; v < (int)(V * sizeof(T) / 16); ++v)
      reinterpret_cast<uint4*>(o)[v] = reinterpret_cast<const uint4*>(res)[v];
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) o[i] = res[i];
  }
}

// ST_MULTI: every wanted output of the V points from one neighbourhood (one
// decode serves all operations).  The integer numerators of the V points are
// formed once; the outputs are then converted and stored one after the other.
template <int D, int V, bool AL>
__device__ __forceinline__ void emit_multi(const PGeo& g, int64_t i0, const short* c, const short* a,
                                           const short* b, const short* zmv, const short* zpv, int xl, int xr,
                                           int ex0, int exn, int ez, int ey) {
  using T = typename OT<D>::T;
  int n[4][V];  // derivative along axes 0, 1, 2 and the Laplacian
#pragma unroll
  for (int i = 0; i < V; ++i) {
    const int cm = i == 0 ? xl : c[i - 1];
    const int cp = i == V - 1 ? xr : c[i + 1];
    int ex = 1;
    if (i == 0) ex = ex0;
    if (i == V - 1) ex = ex * exn;
    n[0][i] = ((int)zpv[i] - zmv[i]) * ez;
    n[1][i] = ((int)b[i] - a[i]) * ey;
    n[2][i] = (cp - cm) * ex;
    n[3][i] = (int)zmv[i] + zpv[i] + a[i] + b[i] + cm + cp - 6 * (int)c[i];
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    T* o = reinterpret_cast<T*>(g.mout[k]);
    if (o == nullptr) continue;
    T res[V];
#pragma unroll
    for (int i = 0; i < V; ++i) {
      if (k < 3) res[i] = emit1<ST_DERIV, D>(n[k][i], 0, 0, g);
      if (k == 3) res[i] = emit1<ST_GRADMAG, D>(n[0][i], n[1][i], n[2][i], g);
      if (k == 4) res[i] = emit1<ST_LAPLACIAN, D>(n[3][i], 0, 0, g);
    }
    o += i0;
    if constexpr (AL && V * sizeof(T) >= 16) {
#pragma unroll
      for (int v = 0; v < (int)(V * sizeof(T) / 16); ++v)
        reinterpret_cast<uint4*>(o)[v] = reinterpret_cast<const uint4*>(res)[v];
    } else {
#pragma unroll
      for (int i = 0; i < V; ++i) o[i] = res[i];
    }
  }
}

// Compile-time operation and type, or (ST_RUNTIME) the run-time switch over
// both; out + i0 is the item's first output.
template <int OP, int OUT, int V, bool AL>
__device__ __forceinline__ void store_items(const PGeo& g, typename OT<OUT>::T* out, int64_t i0, const short* c,
                                            const short* a, const short* b, const short* zmv, const short* zpv,
                                            int xl, int xr, int ex0, int exn, int ez, int ey) {
  if constexpr (OP == ST_RUNTIME) {
#define HC_PIPE_RT(O, D)                                                                                            \
  case O * 4 + D:                                                                                                   \
    emit_items<O, D, V, AL>(g, reinterpret_cast<typename OT<D>::T*>(out) + i0, c, a, b, zmv, zpv, xl, xr, ex0, exn, \
                            ez, ey);                                                                                \
    break;
    switch (g.op * 4 + g.out) {
      HC_PIPE_RT(ST_DERIV, HC_F32)
      HC_PIPE_RT(ST_DERIV, HC_F64)
      HC_PIPE_RT(ST_DERIV, HC_I64)
      HC_PIPE_RT(ST_GRADMAG, HC_F32)
      HC_PIPE_RT(ST_GRADMAG, HC_F64)
      HC_PIPE_RT(ST_LAPLACIAN, HC_F32)
      HC_PIPE_RT(ST_LAPLACIAN, HC_F64)
      HC_PIPE_RT(ST_LAPLACIAN, HC_I64)
      default:
        break;
    }
#undef HC_PIPE_RT
  } else if constexpr (OP == ST_MULTI) {
    emit_multi<OUT, V, AL>(g, i0, c, a, b, zmv, zpv, xl, xr, ex0, exn, ez, ey);
  } else {
    emit_items<OP, OUT, V, AL>(g, out + i0, c, a, b, zmv, zpv, xl, xr, ex0, exn, ez, ey);
  }
}

// W consecutive int16 codes at element offset e of slot `base` (a 64-byte
// aligned shared-memory slot): one vector load when AL (e a multiple of W),
// else (W = 8, any e) five 32-bit loads from the word holding code e and a
// byte permute per output word.  The address stays a shared-memory pointer
// (base plus an offset), so the loads are shared-memory loads.  The reads may
// reach 4 bytes past the codes; the ring is followed by the staging and
// metadata buffers, so they stay inside the shared memory of the tile.
template <int W, bool AL>
__device__ __forceinline__ void load_codes(short* dst, const short* base, int e) {
  if constexpr (AL) {
    using Vec = typename std::conditional<W == 8, uint4, typename std::conditional<W == 4, uint2, unsigned short>::type>::type;
    *reinterpret_cast<Vec*>(dst) = *reinterpret_cast<const Vec*>(base + e);
  } else {
    static_assert(W == 8, "unaligned items are 8 codes wide");
    const uint32_t* wp = reinterpret_cast<const uint32_t*>(base) + (e >> 1);
    const uint32_t sel = (e & 1) ? 0x5432u : 0x3210u;
    uint32_t w[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) w[k] = wp[k];
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k] = __byte_perm(w[k], w[k + 1], sel);
  }
}

// One work item: the W outputs x .. x + W - 1 of row y0 + yr of plane z (slots
// pc / pm / pp hold planes z, z - 1, z + 1; rc0 / rm0 / rp0 are the element
// offsets of row y0 in them; row0 its element index in the field).
template <int OP, int OUT, int W, bool AL, bool STATS>
__device__ __forceinline__ void pipe_item(const PGeo& g, typename OT<OUT>::T* out, const short* pc, const short* pm,
                                          const short* pp, int rc0, int rm0, int rp0, int64_t row0, int64_t y0,
                                          int yr, int x, int n2, int ez, Moments& mo) {
  const int roff = yr * n2 + x;
  const int rc = rc0 + roff;
  const int64_t y = y0 + yr;
  const int ey = (y == 0 || y == g.n1 - 1) ? 2 : 1;
  const int eop = OP == ST_RUNTIME ? g.op : OP;
  short c[W], a[W], b[W], zmv[W], zpv[W];
  load_codes<W, AL>(c, pc, rc);
  if (eop != ST_DERIV || g.axis == 1) {
    load_codes<W, AL>(a, pc, y > 0 ? rc - n2 : rc);
    load_codes<W, AL>(b, pc, y + 1 < g.n1 ? rc + n2 : rc);
  }
  if (eop != ST_DERIV || g.axis == 0) {
    load_codes<W, AL>(zmv, pm, rm0 + roff);
    load_codes<W, AL>(zpv, pp, rp0 + roff);
  }
  int xl = c[0], xr = c[W - 1];
  if (eop != ST_DERIV || g.axis == 2) {
    if (x > 0) xl = pc[rc - 1];
    if (x + W < n2) xr = pc[rc + W];
  }
  // one-sided differences at the row ends are doubled
  const int ex0 = x == 0 ? 2 : 1, exn = x + W == n2 ? 2 : 1;
  if (STATS) {
    // int16 codes: q^2 < 2^30, so an item's sums fit 32 / 64 bits and go
    // into the 128-bit accumulator with one carry
    int a1 = 0;
    unsigned long long a2 = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      a1 += c[i];
      a2 += (unsigned long long)((int)c[i] * (int)c[i]);
    }
    mo.add_sums(a1, a2);
  }
  store_items<OP, OUT, W, AL>(g, out, row0 + roff, c, a, b, zmv, zpv, xl, xr, ex0, exn, ez, ey);
}

// One tile (row tile yt, plane range zt) of the pipelined stencil; needs
// blockDim.x == kThreads.  sm: the dynamic shared memory (psmem(g).total
// bytes).  With STATS the codes of the points the tile owns are added to mo.
// OP = OUT = ST_RUNTIME takes the operation and output type from g; OP =
// ST_MULTI writes every output of g.mout that is set (out is unused).  PRED:
// the stream's hc_predictor (s.pred), fixed at compile time so that each
// decoding loop stays as small as it can be.
template <int OP, int OUT, int V, bool STATS, int PRED>
__device__ inline void pipe_tile(const DevStream& s, const PGeo& g, int yt, int zt, typename OT<OUT>::T* out, int* err,
                                 unsigned char* sm, Moments& mo) {
  using T = typename OT<OUT>::T;
  // V = 8 / 4: items of V outputs, rows a multiple of V; V = 0: items of 8
  // outputs at any offset (unaligned loads, scalar stores) plus a scalar tail
  constexpr int VW = V == 0 ? 8 : V;
  const PSmem L = psmem(g);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const int64_t y0 = (int64_t)yt * g.ty, y1 = min(y0 + g.ty, g.n1);
  const int64_t z0 = (int64_t)zt * g.tz, z1 = min(z0 + g.tz, g.n0);
  // halo rows and planes: a derivative reads neighbours along its own axis
  // only, so the rows above and below the tile are decoded for axis 1 alone
  // and the planes around its range for axis 0 alone
  const bool hy = OP != ST_DERIV || g.axis == 1, hz = OP != ST_DERIV || g.axis == 0;
  const int64_t ylo = hy ? max(y0 - 1, (int64_t)0) : y0, yhi = hy ? min(y1 + 1, g.n1) : y1;
  const int64_t zs = hz ? max(z0 - 1, (int64_t)0) : z0, ze = hz ? min(z1 + 1, g.n0) : z1;  // slabs [zs, ze)
  const int nslab = (int)(ze - zs);

  auto meta_w = [&](int j) { return sm + L.wb + (j % kWidthBufs) * g.pre_max; };
  auto meta_h = [&](int j) { return reinterpret_cast<int32_t*>(sm + L.hb + (j % kStages) * 4 * g.heads_max); };
  auto meta_o = [&](int j) { return reinterpret_cast<uint32_t*>(sm + L.ob + (j % kStages) * L.ob_bytes); };
  auto stage = [&](int j) { return reinterpret_cast<uint32_t*>(sm + L.stage + (j % kStages) * 4 * g.stage_words); };
  auto slot = [&](int64_t z) { return sm + L.ring + (int)(z & 3) * g.slot_bytes; };

  // loader: copy widths [cs, b0 + nblk) of slab j
  auto load_widths = [&](int j) {
    const SlabDesc d = slab_desc(s, g, zs + j, ylo, yhi);
    const int nw = (d.npre + d.nblk + 15) & ~15;
    const uint8_t* wsrc = s.widths + d.cs;  // cs is a multiple of G = 128: 16-byte aligned
    uint8_t* wdst = meta_w(j);
    for (int i = lane * 16; i < nw; i += 32 * 16) cp_async16(wdst + i, wsrc + i);
  };
  // loader: copy heads [b0, b0 + nblk) of slab j
  auto load_heads = [&](int j) {
    const SlabDesc d = slab_desc(s, g, zs + j, ylo, yhi);
    const int64_t h0 = d.b0 & ~(int64_t)3;
    const int nh = (int)((d.b0 + d.nblk - h0 + 3) & ~3);
    int32_t* hdst = meta_h(j);
    for (int i = lane * 4; i < nh; i += 32 * 4) cp_async16(hdst + i, s.heads + h0 + i);
  };
  // loader: offsets of slab j from its widths, then cp.async of its payload.
  // Lane l sums the block sizes of its own run of consecutive widths, one warp
  // scan turns the run totals into run offsets, and a second pass over the
  // run writes the block offsets: two short independent passes instead of a
  // chain of dependent warp scans, one per 32 widths.
  auto scan_and_load_payload = [&](int j) {
    const SlabDesc d = slab_desc(s, g, zs + j, ylo, yhi);
    const uint8_t* w = meta_w(j);
    uint32_t* off = meta_o(j);
    const int n = d.npre + d.nblk;
    const int per = (n + 31) >> 5;
    const int r0 = min(lane * per, n), r1 = min(r0 + per, n);
    int bad = 0;
    uint32_t run = 0;
    for (int i = r0; i < r1; ++i) {
      uint32_t wi = w[i];
      if (wi > (uint32_t)s.wmax) {
        bad = 1;
        wi = 0;
      }
      run += wi ? 1u + wi : 0u;  // S = 32: one sign word + w magnitude words
    }
    uint32_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const uint32_t carry = __shfl_sync(0xffffffffu, x, 31);  // words of the whole range
    uint32_t at = x - run;                                     // exclusive, relative to chunk start
    for (int i = r0; i < r1; ++i) {
      const uint32_t wi = w[i];
      if (i >= d.npre) off[i - d.npre] = at;
      at += (wi && wi <= (uint32_t)s.wmax) ? 1u + wi : 0u;
    }
    // payload words [chunk base + off[0], chunk base + carry) plus one word
    __syncwarp();
    const uint32_t first = off[0];
    const uint64_t base = s.chunks[d.cs >> 7] + first;
    const uint32_t words = carry - first;
    bad |= (base + words > (uint64_t)s.payload_words) || ((int)words + 8 > g.stage_words);
    bad = __any_sync(0xffffffffu, bad);
    const uint64_t a0 = base & ~(uint64_t)3;
    const int lead = (int)(base - a0);
    if (!bad) {
      uint32_t* dst = stage(j);
      const int nvec = (lead + (int)words + 1 + 3) >> 2;
      for (int v = lane; v < nvec; v += 32) cp_async16(dst + 4 * v, s.payload + a0 + 4 * v);
    }
    __syncwarp();
    // offsets relative to the staging buffer (or all zero for a bad slab)
    for (int i = lane; i < d.nblk; i += 32) off[i] = bad ? 0u : off[i] - first + lead;
    if (bad && lane == 0) set_error(err, HC_ERR_CORRUPT);
  };

  // ---- prologue: widths of slabs 0..4; payload and heads of slabs 0..2
  if (warp == 0) {
    for (int j = 0; j < 5 && j < nslab; ++j) load_widths(j);
    cp_async_wait_all();
    __syncwarp();
    for (int j = 0; j < 3 && j < nslab; ++j) {
      scan_and_load_payload(j);
      load_heads(j);
    }
    cp_async_wait_all();
  }
  __syncthreads();

  int64_t znext = z0;  // next output plane
  for (int k = 0; k <= nslab; ++k) {
    if (warp == 0) {
      // One copy group per step: step k copies the payload and heads of slab
      // k + 3 and the widths of slab k + 5.  Waiting for all groups but the
      // newest (step k - 1's) completes step k - 2's group: the widths of
      // slab k + 3, scanned now, and (read after this step's barrier) the
      // payload of slab k + 1; every copy has two steps to land.
      cp_async_wait_group1();
      __syncwarp();
      if (k + 3 < nslab) {
        scan_and_load_payload(k + 3);
        load_heads(k + 3);
      }
      if (k + 5 < nslab) load_widths(k + 5);
      cp_async_commit();
    } else {
      // Split the 7 worker warps between decoding slab k and computing the
      // planes that are ready, in proportion to the estimated work (a segment
      // kDecodeCost / kPointCost above); a warp has one role, so no divergence.
      // (Giving every warp an equal share of both jobs was measured slower:
      // with separate roles the decoding warps' integer work overlaps the
      // computing warps' conversions and stores.)
      const int ww = warp - 1;
      const int64_t ready = zs + k - 1;  // last slab decoded in an earlier step
      int64_t zc1 = znext;
      // a plane is ready once its own slab (and, when planes are neighbours,
      // the next one) is decoded
      while (zc1 < z1 && min(zc1 + (hz ? 1 : 0), g.n0 - 1) <= ready) ++zc1;
      const int nplanes = (int)(zc1 - znext);
      const int nseg_k = k < nslab ? slab_desc(s, g, zs + k, ylo, yhi).nblk : 0;
      // full items of VW outputs, then (V = 0: rows of any length) the
      // n2 % 8 trailing outputs of every row one by one
      const int nfull = (int)(y1 - y0) * g.nq;
      const int tail = V == 0 ? (int)g.n2 - g.nq * VW : 0;
      const int items = nfull + (int)(y1 - y0) * tail;
      // (single-precision estimates: every worker warp forms the split once
      // per step, so it stays a handful of instructions)
      constexpr int point_cost =
          OP == ST_MULTI ? kPointCostMulti : (OP == ST_RUNTIME || STATS ? kPointCostRuntime : kPointCost);
      const float dec_cost = (float)(kDecodeCost * 32) * (float)nseg_k;
      const float comp_cost = (float)point_cost * (float)nplanes * (float)((int)(y1 - y0) * (int)g.n2);
      int ndw = kWorkerWarps;
      if (nplanes == 0)
        ndw = kWorkerWarps;
      else if (nseg_k == 0)
        ndw = 0;
      else
        ndw = min(kWorkerWarps - 1,
                  max(1, __float2int_rn(__fdividef((float)kWorkerWarps * dec_cost, dec_cost + comp_cost))));
      const bool decoder = ww < ndw;
      const int wt = decoder ? ww * 32 + lane : (ww - ndw) * 32 + lane;
      const int wstride = decoder ? ndw * 32 : (kWorkerWarps - ndw) * 32;
      // decode slab k into its slot
      if (decoder && k < nslab) {
        const int64_t z = zs + k;
        const SlabDesc d = slab_desc(s, g, z, ylo, yhi);
        const uint8_t* w = meta_w(k) + d.npre;
        const int32_t* hd = meta_h(k) + (int)(d.b0 & 3);
        const uint32_t* off = meta_o(k);
        const uint32_t* stg = stage(k);
        unsigned char* dst = slot(z);
        for (int seg = wt; seg < d.nblk; seg += wstride) {
          const uint32_t wi = min((uint32_t)w[seg], (uint32_t)s.wmax);
          int32_t q = hd[seg];
          short v[32];
          if (wi == 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = (short)q;
          } else if constexpr (PRED == HC_PRED_MEAN) {
            // block mean (HSZx): q = M_b + p
            const uint32_t* blk = stg + off[seg];
            decode32_grp(g.grp, blk + 1, blk[0], wi, [&](int i, int32_t x, int32_t neg) { v[i] = (short)(q + x - neg); });
          } else {
            const uint32_t* blk = stg + off[seg];
            decode32_grp(g.grp, blk + 1, blk[0], wi, [&](int i, int32_t x, int32_t neg) {
              q = q + x - neg;
              v[i] = (short)q;
            });
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            uint4 pk;
            pk.x = (uint32_t)(uint16_t)v[8 * j + 0] | ((uint32_t)(uint16_t)v[8 * j + 1] << 16);
            pk.y = (uint32_t)(uint16_t)v[8 * j + 2] | ((uint32_t)(uint16_t)v[8 * j + 3] << 16);
            pk.z = (uint32_t)(uint16_t)v[8 * j + 4] | ((uint32_t)(uint16_t)v[8 * j + 5] << 16);
            pk.w = (uint32_t)(uint16_t)v[8 * j + 6] | ((uint32_t)(uint16_t)v[8 * j + 7] << 16);
            *reinterpret_cast<uint4*>(dst + (seg << 6) + (j << 4)) = pk;
          }
        }
      }
      // compute every output plane whose slabs are all decoded before this step
      for (; znext < zc1; ++znext) {
        if (decoder) continue;
        const int64_t z = znext, zm = z > 0 ? z - 1 : 0, zp = z + 1 < g.n0 ? z + 1 : z;
        const short* pc = reinterpret_cast<const short*>(slot(z));
        const short* pm = reinterpret_cast<const short*>(slot(zm));
        const short* pp = reinterpret_cast<const short*>(slot(zp));
        // element offsets (inside each slot) of row y0 of planes z, z-1, z+1
        const int64_t row0 = (z * g.n1 + y0) * g.n2;
        // a slot starts at block (e0 >> 5) of its slab's first element e0 =
        // (z n1 + ylo) n2, so row y0 sits at (y0 - ylo) n2 + (e0 mod 32) in
        // it; e0 mod 32 needs only the low 32 bits of the product
        const int n2 = (int)g.n2;
        const int dy = (int)(y0 - ylo) * n2;
        const uint32_t pl = (uint32_t)g.n1 * (uint32_t)g.n2, yl = (uint32_t)ylo * (uint32_t)g.n2;
        const int rc0 = dy + (int)(((uint32_t)z * pl + yl) & 31u);
        const int rm0 = dy + (int)(((uint32_t)zm * pl + yl) & 31u);
        const int rp0 = dy + (int)(((uint32_t)zp * pl + yl) & 31u);
        const int ez = (z == 0 || z == g.n0 - 1) ? 2 : 1;
        for (int it = wt; it < items; it += wstride) {
          if (V != 0 || it < nfull) {
            const int yr = g.nq == 1 ? it : (int)__umulhi((unsigned)it, g.nq_magic);
            const int x = (it - yr * g.nq) * VW;
            pipe_item<OP, OUT, VW, (V != 0), STATS>(g, out, pc, pm, pp, rc0, rm0, rp0, row0, y0, yr, x, n2, ez, mo);
          } else {
            // the last n2 % 8 codes of every row, one at a time
            const int t2 = it - nfull;
            const int yr = t2 / (tail > 0 ? tail : 1);  // tail > 0 here (V = 0 only)
            const int x = g.nq * VW + (t2 - yr * tail);
            pipe_item<OP, OUT, 1, true, STATS>(g, out, pc, pm, pp, rc0, rm0, rp0, row0, y0, yr, x, n2, ez, mo);
          }
        }
      }
    }
    __syncthreads();
  }
  if (warp == 0) cp_async_wait_all();
}

// Tile heights tried by the autotuner (and, without tuning, the first that
// fits the shared-memory budget), largest first.  Small planes take tall
// tiles (up to the whole plane): a step then decodes and computes enough
// work to cover its fixed costs, and fewer halo rows are decoded twice.
constexpr int kPipeTileHeights[] = {128, 64, 32, 16, 8, 4, 2, 1};
// The heights to try for rows of n1 codes into out (at most 9): the whole
// plane first when n1 <= 128 is not itself in kPipeTileHeights, then those.
inline int pipe_heights(int64_t n1, int* out) {
  int k = 0;
  bool listed = false;
  for (int ty : kPipeTileHeights) listed |= ty == n1;
  if (n1 > 1 && n1 <= 128 && !listed) out[k++] = (int)n1;
  for (int ty : kPipeTileHeights) out[k++] = ty;
  return k;
}

// Geometry of the pipelined tile for a field walked as d3 (host).  False when
// the tile does not apply: S != 32, |q| >= 2^15, or no tile height fits.
// budget: shared-memory bytes a CTA may use (force_ty > 0 takes that height).
// max_ty > 0: no height above it (force_ty == 0 only).
bool plan_pipe_geometry(const hc_header* h, const int64_t* d3, PGeo& g, int* smem_out, int force_ty, int budget,
                        int max_ty = 0);
// Items per row and the magic divisor of the row/item split; false when
// the 32-bit magic division would not be exact for this tile.
bool plan_pipe_items(PGeo& g, int V);

}  // namespace hc
