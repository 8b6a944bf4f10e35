// hc_xnd_march.cu -- one-pass stencils of HSZx-nd streams (Section IV,
// "HSZx-nd"; Section V-B): the derivative, gradient magnitude and Laplacian
// straight from the stream, at stage 2 (D_p and the box means, with the
// means' difference added where two points lie in different boxes, Eq.
// derivative_Dp / laplacian_Dp on every axis) or stage 3 (D_q = M_b + p).
//
// A CTA owns a tile of R box rows x X box columns and marches through a
// range of box layers.  Each step decodes one layer into a ring of b0 + 2
// planes in shared memory (the tile's own boxes segment by segment with the
// grouped unpacker; the one-code halo around the tile -- the neighbouring
// row and column of codes -- run by run from the neighbouring boxes, whose
// codes are independent of each other: p_k = q_k - M_b), then computes every
// output plane whose three planes are decoded.  Box payload offsets come from
// one prefix pass over the widths (k_box_offsets), so any box is read
// directly.  The results equal the two-pass path's (decode to an array,
// then the array stencil) bit for bit.
#include <algorithm>
#include <cstdint>

#include "hc_group.cuh"
#include "hc_internal.cuh"
#include "hc_launch.h"
#include "hc_stencil_tile.cuh"

namespace hc {

DevStream dev_stream(const hc_header* h, const void* d_stream);

namespace {

constexpr int kOX = 4;  // ring column of the tile's first own code (16-byte aligned rows)

struct MGeo {
  int64_t n0, n1, n2;  // field (internal 3-D shape)
  int b0, b1, b2;      // box extents
  int l0, l1, l2;      // log2 of the extents when powers of two, else -1
  int64_t g0, g1, g2;  // box grid
  int R, X, L;         // tile: box rows, box columns, box layers
  int ntr, ntx;        // tiles along box rows and box columns
  int P;               // ring planes: b0 + 2 (1 for a single plane)
  int pitch, pw;       // ring row pitch and plane size (words)
  int grp;             // group size of the grouped unpacker
  int vec4;            // rows a multiple of 4 and a 16-byte aligned output: 4-wide stores
  unsigned nq_magic;   // ceil(2^32 / nq), nq = items (of 4 outputs) per tile row
  int nq;
  int mrow;            // stage 2: box means ring row length (X + 2)
  int sw;              // words of a thread's segment staging slot: wmax + 2 (rounded to 4)
};

// v / b for 0 <= v < 2^31: a shift when b is a power of two (l = log2 b)
__device__ __forceinline__ int div_b(int v, int b, int l) { return l >= 0 ? (v >> l) : v / b; }

// Residual p of slot sl of a box at payload word `off` with width w, every
// word read bounds-checked against the payload.
__device__ __forceinline__ int32_t box_code(const DevStream& s, uint64_t off, uint32_t w, int sl) {
  if (w == 0) return 0;
  const int j = sl >> 5, kk = sl & 31;
  const uint64_t pwds = (uint64_t)s.payload_words;
  const uint32_t bit = (uint32_t)kk * w;
  const uint64_t si = off + (uint64_t)j;
  const uint64_t wi = off + (uint64_t)s.nseg + (uint64_t)j * w + (bit >> 5);
  const uint32_t sw = si < pwds ? __ldg(s.payload + si) : 0u;
  const uint32_t lo = wi < pwds ? __ldg(s.payload + wi) : 0u;
  const uint32_t hi = wi + 1 < pwds ? __ldg(s.payload + wi + 1) : 0u;
  const uint32_t mag = __funnelshift_r(lo, hi, bit & 31u) & ((1u << w) - 1u);
  const int32_t neg = -(int32_t)((sw >> kk) & 1u);
  return ((int32_t)mag ^ neg) - neg;
}

// Scaled output of a 32-bit stencil numerator: the same value as emit() of
// the same integer (int -> float / double conversions of a value below 2^31
// round exactly as the 64-bit ones).
template <int OP, int OUT>
__device__ __forceinline__ typename OutType<OUT>::T emit_i(int a, int b, int c, const Geo& g) {
  if constexpr (OUT == HC_I64) {
    return (long long)a;
  } else if constexpr (OP == ST_DERIV) {
    if constexpr (OUT == HC_F32) return __fmul_rn(__int2float_rn(a), g.eps_f);
    if constexpr (OUT == HC_F64) return __dmul_rn(__int2double_rn(a), g.eps);
  } else if constexpr (OP == ST_LAPLACIAN) {
    if constexpr (OUT == HC_F32) return __fmul_rn(__int2float_rn(a), g.te_f);
    if constexpr (OUT == HC_F64) return __dmul_rn(__int2double_rn(a), g.te);
  } else {
    if constexpr (OUT == HC_F32) {
      const float x = __int2float_rn(a), y = __int2float_rn(b), z = __int2float_rn(c);
      return __fmul_rn(__fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z))), g.eps_f);
    } else {
      const double x = __int2double_rn(a), y = __int2double_rn(b), z = __int2double_rn(c);
      return __dmul_rn(__dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z))), g.eps);
    }
  }
  return 0;
}

// Payload word offset of every box: the chunk's offset plus the sizes of the
// boxes before it in the chunk.  One warp per chunk.  A width above the
// header's maximum, or a box ending past the payload, marks the stream
// corrupt (its offset is then set to the payload's end, where every read
// is skipped).
__global__ void __launch_bounds__(kThreads) k_box_offsets(DevStream s, uint32_t* __restrict__ boff, int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < s.nchunks; c += warps) {
    const int64_t b0 = c * s.G, b1 = min(b0 + s.G, s.nb);
    uint64_t run = __ldg(s.chunks + c);
    for (int64_t bb = b0; bb < b1; bb += 32) {
      const int64_t b = bb + lane;
      uint32_t words = 0;
      bool bad = false;
      if (b < b1) {
        const uint32_t w = __ldg(s.widths + b);
        bad = w > (uint32_t)s.wmax;
        words = bad ? 0u : block_words(s.S, s.nseg, w);
      }
      uint32_t x = words;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      const uint64_t at = run + (x - words);
      bad |= at + words > (uint64_t)s.payload_words;
      if (b < b1) boff[b] = bad ? (uint32_t)s.payload_words : (uint32_t)at;
      if (__any_sync(0xffffffffu, bad) && lane == 0) set_error(err, HC_ERR_CORRUPT);
      run += __shfl_sync(0xffffffffu, x, 31);
    }
  }
}

// One tile: box rows [k1a, k1a + R), box columns [k2a, k2a + X), box layers
// [ka, ka + L).  Shared memory: the ring (P planes of pw words: row ly =
// y - y0 + 1, column kOX + x - x0; the halo at row 0 / ny + 1 and column
// kOX - 1 / kOX + nx), the slot table (slot -> (s0 << 20) | s1 pitch + s2)
// and, at stage 2, the box means of three layers around the tile.
template <int OP, int OUT, bool ST2, int AX>
__global__ void __launch_bounds__(kThreads, 3)
    k_box_march(DevStream s, MGeo m, Geo g, const uint32_t* __restrict__ boff,
                typename OutType<OUT>::T* __restrict__ out, int* err) {
  using T = typename OutType<OUT>::T;
  extern __shared__ __align__(16) int32_t sm[];
  int32_t* ring = sm;
  uint32_t* tab = reinterpret_cast<uint32_t*>(sm + m.P * m.pw);
  int32_t* mr = reinterpret_cast<int32_t*>(tab + ((s.S + 3) & ~3));
  uint32_t* stg = reinterpret_cast<uint32_t*>(mr + 3 * (m.R + 2) * m.mrow);  // kThreads slots of sw words
  const int tid = threadIdx.x, nt = blockDim.x;

  const int64_t t = blockIdx.x;
  const int64_t tr = t % m.ntr, tx = (t / m.ntr) % m.ntx, tl = t / ((int64_t)m.ntr * m.ntx);
  const int64_t k1a = tr * m.R, k2a = tx * m.X, ka = tl * m.L;
  const int64_t kb = min(ka + m.L, m.g0);
  const int Rt = (int)min((int64_t)m.R, m.g1 - k1a), Xt = (int)min((int64_t)m.X, m.g2 - k2a);
  const int64_t y0 = k1a * m.b1, y1 = min(m.n1, (k1a + Rt) * m.b1);
  const int64_t x0 = k2a * m.b2, x1 = min(m.n2, (k2a + Xt) * m.b2);
  const int64_t z0 = ka * m.b0, z1 = min(m.n0, kb * m.b0);
  const int ny = (int)(y1 - y0), nx = (int)(x1 - x0);
  const int b12 = m.b1 * m.b2;

  for (int sl = tid; sl < s.S; sl += nt) {
    const int s0 = sl / b12, rr = sl - s0 * b12;
    const int s1 = rr / m.b2, s2 = rr - s1 * m.b2;
    tab[sl] = ((uint32_t)s0 << 20) | (uint32_t)(s1 * m.pitch + s2);
  }
  __syncthreads();

  int64_t znext = z0;  // next output plane
  // halos: a derivative reads neighbours along its own axis only (no plane
  // below / above the range unless AX = 0, no row / column halo unless AX =
  // 1 / 2); a plane is then ready once its own layer is decoded
  constexpr bool HZ = OP != ST_DERIV || AX == 0, HY = OP != ST_DERIV || AX == 1, HX = OP != ST_DERIV || AX == 2;
  const int64_t kfirst = HZ ? max(ka - 1, (int64_t)0) : ka;
  // (k b0) mod P and k mod 3 of the first layer the loop visits, then
  // advanced by one layer per iteration
  int zb = (int)((kfirst * m.b0) % m.P), k3 = (int)(kfirst % 3);
  for (int64_t k = kfirst; k <= (HZ ? kb : kb - 1); ++k) {
    if (k >= m.g0) break;  // uniform over the CTA
    // planes of layer k to decode: the whole layer inside the range, the
    // last plane of the layer below it, the first plane of the layer above
    int64_t zlo = k * m.b0, zhi = min(m.n0, zlo + m.b0) - 1;
    if (k == ka - 1) zlo = zhi;
    if (k == kb) zhi = zlo;
    const int s0lo = (int)(zlo - k * m.b0), s0hi = (int)(zhi - k * m.b0);
    const int slo = s0lo * b12, shi = (s0hi + 1) * b12;  // slots [slo, shi)
    const int jlo = slo >> 5, nj = ((shi - 1) >> 5) - jlo + 1;
    // ring slot of the layer's plane s0 = 0 (k b0 mod P, kept by steps of
    // b0 < P) and of any plane z in [k b0 - 2, k b0 + b0): 32-bit arithmetic
    // only (a 64-bit remainder per plane costs more than the plane's stencil)
    const int zbm = zb;
    auto ring_slot = [&](int64_t z) {
      int r = zbm + (int)(z - k * m.b0);
      if (r < 0) r += m.P;
      if (r >= m.P) r -= m.P;
      return r;
    };

    // Decode: the tile's own boxes one 32-slot segment per work item, and
    // the halo -- per plane the row below / above the tile (one run of b2
    // codes per box column) and the column left / right of it (one run of b1
    // codes, slot stride b2, per box row); only the planes the tile computes
    // read the halo (the planes below and above the range are read at the
    // tile's own positions only).  An item waits for two memory round trips:
    // the box's width, mean and offset, then its segment's words, copied to
    // the thread's staging slot with every load in flight together.
    {
      const int nown = Rt * Xt * nj;
      const bool hy0 = HY && y0 > 0, hy1 = HY && y1 < m.n1, hx0 = HX && x0 > 0, hx1 = HX && x1 < m.n2;
      const int runs = (hy0 + hy1) * Xt + (hx0 + hx1) * Rt;
      const int nhalo = (k != ka - 1 && k != kb) ? (int)(zhi - zlo + 1) * runs : 0;
      uint32_t* sb = stg + tid * m.sw;
      for (int i = tid; i < nown + nhalo; i += nt) {
        const bool own = i < nown;
        int64_t b;
        // own: segment j of the box at box row r, box column c (ring offset base)
        int j = 0, base = 0;
        // halo: slots sl0 + q st (q < cnth) into ring offsets d0 + q ds of plane s0h
        int sl0 = 0, st = 1, cnth = 0, d0 = 0, ds = 1, s0h = 0;
        if (own) {
          const int bi = i / nj, r = bi / Xt, c = bi - r * Xt;
          j = jlo + (i - bi * nj);
          b = (k * m.g1 + k1a + r) * m.g2 + k2a + c;
          base = (r * m.b1 + 1) * m.pitch + kOX + c * m.b2;
        } else {
          const int ih = i - nown;
          const int zi = ih / runs;
          int u = ih - zi * runs;
          s0h = (int)(zlo + zi - k * m.b0);
          int64_t by, bx;
          if (u < (hy0 + hy1) * Xt) {
            const bool hi = hy0 ? u >= Xt : true;
            const int c = hy0 && !hi ? u : u - (hy0 ? Xt : 0);
            const int y = (int)(hi ? y1 : y0 - 1);
            by = div_b(y, m.b1, m.l1);
            bx = k2a + c;
            sl0 = (s0h * m.b1 + (int)(y - by * m.b1)) * m.b2;
            cnth = (int)min((int64_t)m.b2, x1 - bx * m.b2);
            d0 = (hi ? ny + 1 : 0) * m.pitch + kOX + c * m.b2;
          } else {
            u -= (hy0 + hy1) * Xt;
            const bool hi = hx0 ? u >= Rt : true;
            const int r = hx0 && !hi ? u : u - (hx0 ? Rt : 0);
            const int x = (int)(hi ? x1 : x0 - 1);
            bx = div_b(x, m.b2, m.l2);
            by = k1a + r;
            sl0 = s0h * b12 + (int)(x - bx * m.b2);
            st = m.b2;
            cnth = (int)min((int64_t)m.b1, y1 - by * m.b1);
            d0 = (r * m.b1 + 1) * m.pitch + (hi ? kOX + nx : kOX - 1);
            ds = m.pitch;
          }
          b = (k * m.g1 + by) * m.g2 + bx;
          j = sl0 >> 5;
        }
        // first round trip: width, mean, offset
        const uint32_t w = __ldg(s.widths + b);
        const int32_t M = ST2 ? 0 : __ldg(s.heads + b);
        const uint64_t off = boff[b];
        if (w > (uint32_t)s.wmax) {
          set_error(err, HC_ERR_CORRUPT);
          continue;
        }
        // second round trip: the segment's sign word and w magnitude words,
        // plus the one word past them that the grouped unpacker may read
        // (staged only where all of it lies inside the payload and, for a
        // halo run, the run lies inside the segment; the rest is read code by
        // code with bounds checks)
        const uint64_t mi = off + (uint64_t)s.nseg + (uint64_t)j * w;
        const bool fast = w && mi + w < (uint64_t)s.payload_words &&
                          (own || ((sl0 + (cnth - 1) * st) >> 5) == j);
        if (fast) {
          sb[0] = __ldg(s.payload + off + j);
          const int n = (int)w + 1;
          for (int q0 = 0; q0 < n; q0 += 8) {
            uint32_t v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = q0 + q < n ? __ldg(s.payload + mi + q0 + q) : 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q)
              if (q0 + q < n) sb[1 + q0 + q] = v[q];
          }
        }
        if (own) {
          const int cnt = min(32, s.S - 32 * j);
          auto put = [&](int kk, int32_t v) {
            const int sl = 32 * j + kk;
            if (kk >= cnt || sl < slo || sl >= shi) return;
            const uint32_t e = tab[sl];
            int ps = zbm + (int)(e >> 20);
            if (ps >= m.P) ps -= m.P;
            ring[ps * m.pw + base + (int)(e & 0xfffffu)] = v;
          };
          // a whole segment inside the planes wanted: no per-code checks
          auto put_all = [&](int kk, int32_t v) {
            const uint32_t e = tab[32 * j + kk];
            int ps = zbm + (int)(e >> 20);
            if (ps >= m.P) ps -= m.P;
            ring[ps * m.pw + base + (int)(e & 0xfffffu)] = v;
          };
          const bool whole = cnt == 32 && 32 * j >= slo && 32 * j + 32 <= shi;
          if (w == 0) {
            for (int kk = 0; kk < cnt; ++kk) put(kk, M);
          } else if (fast && whole) {
            decode32_grp(m.grp, sb + 1, sb[0], w, [&](int kk, int32_t x, int32_t neg) { put_all(kk, M + x - neg); });
          } else if (fast) {
            decode32_grp(m.grp, sb + 1, sb[0], w, [&](int kk, int32_t x, int32_t neg) { put(kk, M + x - neg); });
          } else {
            for (int kk = 0; kk < cnt; ++kk) put(kk, M + box_code(s, off, w, 32 * j + kk));
          }
        } else {
          int32_t* dst = ring + ring_slot(k * m.b0 + s0h) * m.pw + d0;
          if (fast) {
            const uint32_t mask = (1u << w) - 1u, sw = sb[0];
            for (int q = 0; q < cnth; ++q) {
              const int kk = sl0 + q * st - 32 * j;
              const uint32_t bit = (uint32_t)kk * w, wi = bit >> 5;
              const uint32_t mag = __funnelshift_r(sb[1 + wi], sb[2 + wi], bit & 31u) & mask;
              const int32_t neg = -(int32_t)((sw >> kk) & 1u);
              dst[q * ds] = M + (((int32_t)mag ^ neg) - neg);
            }
          } else {
            for (int q = 0; q < cnth; ++q) dst[q * ds] = M + box_code(s, off, w, sl0 + q * st);
          }
        }
      }
    }

    // stage 2: the box means of layer k around the tile (rows -1..Rt,
    // columns -1..Xt), ring slot k mod 3
    if constexpr (ST2) {
      int32_t* ml = mr + k3 * (m.R + 2) * m.mrow;
      for (int i = tid; i < (Rt + 2) * (Xt + 2); i += nt) {
        const int r = i / (Xt + 2) - 1, c = i - (r + 1) * (Xt + 2) - 1;
        const int64_t by = k1a + r, bx = k2a + c;
        if (by < 0 || by >= m.g1 || bx < 0 || bx >= m.g2) continue;
        ml[(r + 1) * m.mrow + c + 1] = __ldg(s.heads + (k * m.g1 + by) * m.g2 + bx);
      }
    }
    __syncthreads();

    // every output plane whose neighbours are decoded: up to zhi - 1, or
    // up to the field's last plane once it is decoded
    const int64_t zc_end = min(z1, (zhi >= m.n0 - 1 || !HZ) ? zhi + 1 : zhi);
    for (; znext < zc_end; ++znext) {
      const int64_t z = znext;
      const int64_t zm = z > 0 ? z - 1 : z, zp = z + 1 < m.n0 ? z + 1 : z;
      const int32_t* pc = ring + ring_slot(z) * m.pw;
      const int32_t* pm = ring + ring_slot(zm) * m.pw;
      const int32_t* pp = ring + ring_slot(zp) * m.pw;
      const int ez = (z == 0 || z == m.n0 - 1) ? 2 : 1;
      // stage 2: the plane's place in its box and the layers of its z neighbours
      const int64_t kz = z >= k * m.b0 ? k : k - 1;  // planes computed now lie in layers k - 1 and k
      const int rz = (int)(z - kz * m.b0);
      const int kz3 = kz == k ? k3 : (k3 == 0 ? 2 : k3 - 1);  // kz mod 3
      const int32_t* mc = mr + kz3 * (m.R + 2) * m.mrow;
      const int32_t* mzm = mr + (kz3 == 0 ? 2 : kz3 - 1) * (m.R + 2) * m.mrow;
      const int32_t* mzp = mr + (kz3 == 2 ? 0 : kz3 + 1) * (m.R + 2) * m.mrow;
      const bool czm = ST2 && z > 0 && rz == 0, czp = ST2 && z + 1 < m.n0 && rz == m.b0 - 1;
      const int items = ny * m.nq;
      const int n2 = (int)m.n2, x0i = (int)x0, x1i = (int)x1;
      for (int it = tid; it < items; it += nt) {
        const int yr = m.nq == 1 ? it : (int)__umulhi((unsigned)it, m.nq_magic);
        const int xq = it - yr * m.nq;
        const int64_t y = y0 + yr;
        const int ly = yr + 1, lx = kOX + 4 * xq;
        const int rowc = ly * m.pitch + lx;
        const int rowm = (y > 0 ? ly - 1 : ly) * m.pitch + lx;
        const int rowp = (y + 1 < m.n1 ? ly + 1 : ly) * m.pitch + lx;
        // the neighbours the operation reads (a derivative: its axis only)
        constexpr bool NZ = OP != ST_DERIV || AX == 0, NY = OP != ST_DERIV || AX == 1;
        constexpr bool NX = OP != ST_DERIV || AX == 2;
        const int4 zero4 = make_int4(0, 0, 0, 0);
        const int4 C = *reinterpret_cast<const int4*>(pc + rowc);
        const int4 YM = NY ? *reinterpret_cast<const int4*>(pc + rowm) : zero4;
        const int4 YP = NY ? *reinterpret_cast<const int4*>(pc + rowp) : zero4;
        const int4 ZM = NZ ? *reinterpret_cast<const int4*>(pm + rowc) : zero4;
        const int4 ZP = NZ ? *reinterpret_cast<const int4*>(pp + rowc) : zero4;
        const int xb = x0i + 4 * xq;
        const int left = NX ? pc[rowc - 1] : 0, right = NX ? pc[rowc + 4] : 0;
        const int cv[4] = {C.x, C.y, C.z, C.w}, ymv[4] = {YM.x, YM.y, YM.z, YM.w}, ypv[4] = {YP.x, YP.y, YP.z, YP.w};
        const int zmv[4] = {ZM.x, ZM.y, ZM.z, ZM.w}, zpv[4] = {ZP.x, ZP.y, ZP.z, ZP.w};
        const int ey = (y == 0 || y == m.n1 - 1) ? 2 : 1;
        // stage 2: per point, the box means' difference toward each
        // neighbour that lies in another box (0 where it lies in the same one)
        int azm[4] = {0, 0, 0, 0}, azp[4] = {0, 0, 0, 0}, aym[4] = {0, 0, 0, 0}, ayp[4] = {0, 0, 0, 0};
        int axm[4] = {0, 0, 0, 0}, axp[4] = {0, 0, 0, 0};
        if constexpr (ST2) {
          const int ky = div_b((int)y, m.b1, m.l1);
          const int ry = (int)(y - ky * m.b1), rb = (int)(ky - k1a);
          const bool cym = y > 0 && ry == 0, cyp = y + 1 < m.n1 && ry == m.b1 - 1;
          if (m.b2 % 4 == 0) {
            // the item's four points share one box (items start at
            // multiples of 4 from the tile's first column, a box border):
            // its mean and its z / y neighbours' once, the x faces at the
            // item's first and last point only
            const int cb = (int)div_b(4 * xq, m.b2, m.l2), rx0 = 4 * xq - cb * m.b2;
            const int mi = (rb + 1) * m.mrow + cb + 1;
            const int Mc = mc[mi];
            const int tzm = NZ && czm ? mzm[mi] - Mc : 0, tzp = NZ && czp ? mzp[mi] - Mc : 0;
            const int tym = NY && cym ? mc[mi - m.mrow] - Mc : 0, typ = NY && cyp ? mc[mi + m.mrow] - Mc : 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              azm[i] = tzm;
              azp[i] = tzp;
              aym[i] = tym;
              ayp[i] = typ;
            }
            if (NX && xb > 0 && rx0 == 0) axm[0] = mc[mi - 1] - Mc;
            if (NX && xb + 4 < n2 && rx0 + 3 == m.b2 - 1) axp[3] = mc[mi + 1] - Mc;
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int xo = 4 * xq + i;  // column inside the tile
              const int cb = (int)div_b(xo, m.b2, m.l2), rx = xo - cb * m.b2;
              const int mi = (rb + 1) * m.mrow + cb + 1;
              const int Mc = mc[mi];
              if (NZ && czm) azm[i] = mzm[mi] - Mc;
              if (NZ && czp) azp[i] = mzp[mi] - Mc;
              if (NY && cym) aym[i] = mc[mi - m.mrow] - Mc;
              if (NY && cyp) ayp[i] = mc[mi + m.mrow] - Mc;
              if (NX && xb + i > 0 && rx == 0) axm[i] = mc[mi - 1] - Mc;
              if (NX && xb + i + 1 < n2 && rx == m.b2 - 1) axp[i] = mc[mi + 1] - Mc;
            }
          }
        }
        T res[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int x = xb + i;
          const int c = cv[i];
          const int xm = x == 0 ? c : (i == 0 ? left : cv[i - 1]);
          const int xp = x + 1 >= n2 ? c : (i == 3 ? right : cv[i + 1]);
          const int ex = (x == 0 || x == n2 - 1) ? 2 : 1;
          // neighbours as differences from c: the codes' own differences at
          // stage 3; at stage 2 the residuals' differences plus the box
          // means' difference where the neighbour lies in another box
          // (|q| < 2^27: every sum below fits 32 bits)
          const int dzm = zmv[i] - c + azm[i], dzp = zpv[i] - c + azp[i];
          const int dym = ymv[i] - c + aym[i], dyp = ypv[i] - c + ayp[i];
          const int dxm = xm - c + axm[i], dxp = xp - c + axp[i];
          if constexpr (OP == ST_LAPLACIAN) {
            res[i] = emit_i<OP, OUT>(dzm + dzp + dym + dyp + dxm + dxp, 0, 0, g);
          } else {
            const int d0 = (dzp - dzm) * ez, d1 = (dyp - dym) * ey, d2 = (dxp - dxm) * ex;
            if constexpr (OP == ST_DERIV)
              res[i] = emit_i<OP, OUT>(AX == 0 ? d0 : (AX == 1 ? d1 : d2), 0, 0, g);
            else
              res[i] = emit_i<OP, OUT>(d0, d1, d2, g);
          }
        }
        T* o = out + (z * m.n1 + y) * m.n2 + xb;
        if (m.vec4 && xb + 4 <= x1i) {
          if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<uint4*>(o) = *reinterpret_cast<const uint4*>(res);
          } else {
            reinterpret_cast<uint4*>(o)[0] = reinterpret_cast<const uint4*>(res)[0];
            reinterpret_cast<uint4*>(o)[1] = reinterpret_cast<const uint4*>(res)[1];
          }
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (xb + i < x1i) o[i] = res[i];
        }
      }
    }
    __syncthreads();
    zb += m.b0;
    if (zb >= m.P) zb -= m.P;
    k3 = k3 == 2 ? 0 : k3 + 1;
  }
}

int ilog2_or(int b) { return (b > 0 && (b & (b - 1)) == 0) ? __builtin_ctz((unsigned)b) : -1; }

// Tile plan: about 16 rows and 64 columns of codes, at least kThreads own
// segments per layer when the box grid allows, ring, tables and staging
// within a three-CTAs-per-SM shared-memory budget (the box layers per tile
// are set at launch).
bool plan_march(const hc_header* h, MGeo& m, int* smem_out) {
  m.n0 = h->dims[0];
  m.n1 = h->dims[1];
  m.n2 = h->dims[2];
  m.b0 = (int)h->block[0];
  m.b1 = (int)h->block[1];
  m.b2 = (int)h->block[2];
  if (m.b0 < 1 || m.b1 < 1 || m.b2 < 1) return false;
  m.l0 = ilog2_or(m.b0);
  m.l1 = ilog2_or(m.b1);
  m.l2 = ilog2_or(m.b2);
  m.g0 = ceil_div(m.n0, m.b0);
  m.g1 = ceil_div(m.n1, m.b1);
  m.g2 = ceil_div(m.n2, m.b2);
  if (m.n1 * m.n2 >= ((int64_t)1 << 31) || (uint64_t)h->payload_words >= 0xfffffff0ull) return false;
  const int nseg = (h->S + 31) / 32;
  m.P = m.n0 == 1 ? 1 : m.b0 + 2;  // a single plane needs no ring
  // box columns: about 64 codes (4-wide items need b2 X a multiple of 4)
  int X = std::max(1, 64 / m.b2);
  while ((X * m.b2) % 4) ++X;
  X = (int)std::min<int64_t>(X, m.g2);
  // box rows: about 16 rows of codes and enough segments to occupy the CTA
  int R = std::max(1, 16 / m.b1);
  while ((int64_t)R * X * nseg < kThreads && R < 64) R *= 2;
  R = (int)std::min<int64_t>(R, m.g1);
  if (m.b0 >= 4096) return false;  // slot table: s0 in the top 12 bits
  const int budget = 74 * 1024;  // three CTAs per SM
  for (;;) {
    m.R = R;
    m.X = X;
    // items of 4 codes cover ceil(X b2 / 4) * 4 columns (X b2 is a multiple
    // of 4 unless the tile is the field's only column of tiles)
    m.nq = (X * m.b2 + 3) / 4;
    m.pitch = (kOX + 4 * m.nq + 1 + 3) & ~3;
    m.pw = ((R * m.b1 + 2) * m.pitch + 3) & ~3;
    m.mrow = X + 2;
    m.sw = ((int)h->wmax + 2 + 3) & ~3;
    const int words = m.P * m.pw + ((h->S + 3) & ~3) + 3 * (R + 2) * m.mrow + kThreads * m.sw;
    *smem_out = 4 * words;
    // slot table: s1 pitch + s2 in the low 20 bits
    if (*smem_out <= budget && (int64_t)(m.b1 - 1) * m.pitch + m.b2 < (1 << 20)) break;
    if (R > 1)
      R = (R + 1) / 2;
    else if (X > 4 && ((X / 2) * m.b2) % 4 == 0)
      X /= 2;
    else
      return false;
  }
  m.ntr = (int)ceil_div(m.g1, m.R);
  m.ntx = (int)ceil_div(m.g2, m.X);
  m.L = (int)m.g0;  // set at launch from the kernel's occupancy (march_layers)
  m.grp = group_for_width(h->wmax);
  if (m.nq <= 1) {
    m.nq_magic = 0u;
  } else {
    const uint64_t mg = ((1ull << 32) + (uint64_t)m.nq - 1) / (uint64_t)m.nq;
    const uint64_t e = mg * (uint64_t)m.nq - (1ull << 32);
    const uint64_t it_max = (uint64_t)(m.R * m.b1) * (uint64_t)m.nq - 1;
    if (e != 0 && it_max >= ((1ull << 32) + e - 1) / e) return false;
    m.nq_magic = (unsigned)mg;
  }
  return true;
}

template <int OP, int OUT, bool ST2, int AX>
int launch_march_t(const hc_header* h, const void* d_stream, const MGeo& m0, int smem, const uint32_t* boff, int axis3,
                   void* d_out, int* err, cudaStream_t st) {
  MGeo m = m0;
  m.vec4 = (m.n2 % 4 == 0) && aligned16(d_out);
  auto kern = k_box_march<OP, OUT, ST2, AX>;
  int rc = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (rc) return rc;
  // layer ranges: one wave of resident CTAs (a tile marches through its
  // layers, so a second, partial wave would leave most SMs idle)
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  const int64_t cap = (int64_t)device_sms() * std::max(per_sm, 1);
  const int64_t cols = (int64_t)m.ntr * m.ntx;
  // layer ranges: the count whose waves x steps per tile is smallest (a tile
  // also decodes one plane of the layer below and above its range)
  int64_t nzt = 1;
  double best = 0.0;
  for (int64_t c = 1; c <= m.g0 && c <= 4096; ++c) {
    const double cost = (double)ceil_div(cols * c, cap) * ((double)ceil_div(m.g0, c) + 2.0 / m.b0);
    if (c == 1 || cost < best * 0.999) {
      best = cost;
      nzt = c;
    }
  }
  m.L = (int)ceil_div(m.g0, nzt);
  const Geo g = stencil_base_geo(h->dims, h->eps, axis3);
  const int64_t grid = (int64_t)m.ntr * m.ntx * ceil_div(m.g0, m.L);
  kern<<<(unsigned)grid, kThreads, smem, st>>>(dev_stream(h, d_stream), m, g, boff,
                                               reinterpret_cast<typename OutType<OUT>::T*>(d_out), err);
  return check_launch_cfg("stencil (boxes, one pass)", reinterpret_cast<const void*>(kern), grid, smem);
}

template <int OP, bool ST2, int AX>
int launch_march_o(const hc_header* h, const void* d_stream, const MGeo& m, int smem, const uint32_t* boff, int axis3,
                   void* d_out, int out_dtype, int* err, cudaStream_t st) {
  switch (out_dtype) {
    case HC_F32:
      return launch_march_t<OP, HC_F32, ST2, AX>(h, d_stream, m, smem, boff, axis3, d_out, err, st);
    case HC_F64:
      return launch_march_t<OP, HC_F64, ST2, AX>(h, d_stream, m, smem, boff, axis3, d_out, err, st);
    case HC_I64:
      if constexpr (OP == ST_GRADMAG) return fail(HC_ERR_UNSUPPORTED, "the gradient magnitude has no integer form");
      return launch_march_t<OP, HC_I64, ST2, AX>(h, d_stream, m, smem, boff, axis3, d_out, err, st);
    default:
      return fail(HC_ERR_INVALID_ARG, "out_dtype");
  }
}

template <bool ST2>
int launch_march_s(const hc_header* h, const void* d_stream, const MGeo& m, int smem, const uint32_t* boff, int op,
                   int axis3, void* d_out, int out_dtype, int* err, cudaStream_t st) {
  switch (op) {
    case ST_DERIV:
      // the derivative's axis fixed at compile time: only its neighbours are read
      if (axis3 == 0)
        return launch_march_o<ST_DERIV, ST2, 0>(h, d_stream, m, smem, boff, axis3, d_out, out_dtype, err, st);
      if (axis3 == 1)
        return launch_march_o<ST_DERIV, ST2, 1>(h, d_stream, m, smem, boff, axis3, d_out, out_dtype, err, st);
      return launch_march_o<ST_DERIV, ST2, 2>(h, d_stream, m, smem, boff, axis3, d_out, out_dtype, err, st);
    case ST_GRADMAG:
      return launch_march_o<ST_GRADMAG, ST2, -1>(h, d_stream, m, smem, boff, axis3, d_out, out_dtype, err, st);
    default:
      return launch_march_o<ST_LAPLACIAN, ST2, -1>(h, d_stream, m, smem, boff, axis3, d_out, out_dtype, err, st);
  }
}

}  // namespace

int xnd_march_impl(const hc_header* h, const void* d_stream, int level, int op, int axis3, void* d_out, int out_dtype,
                   void* d_ws, void* d_scratch, size_t scratch_bytes, cudaStream_t st) {
  // codes below 2^27 in magnitude: the tile's numerators are 32-bit sums
  if (h->pred != HC_PRED_MEAN_ND || (level != HC_STAGE_P && level != HC_STAGE_Q) || h->qmax >= (1u << 27))
    return HC_ERR_UNSUPPORTED;
  if (scratch_bytes < 4 * (size_t)h->nb) return HC_ERR_UNSUPPORTED;
  MGeo m{};
  int smem = 0;
  if (!plan_march(h, m, &smem)) return HC_ERR_UNSUPPORTED;
  int* err = &reinterpret_cast<OpWs*>(d_ws)->status;
  uint32_t* boff = reinterpret_cast<uint32_t*>(d_scratch);
  const DevStream s = dev_stream(h, d_stream);
  const unsigned ogrid =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(h->nchunks, kThreads / 32), (int64_t)device_sms() * 8));
  k_box_offsets<<<ogrid, kThreads, 0, st>>>(s, boff, err);
  int rc = check_launch("box offsets");
  if (rc) return rc;
  if (level == HC_STAGE_P)
    return launch_march_s<true>(h, d_stream, m, smem, boff, op, axis3, d_out, out_dtype, err, st);
  return launch_march_s<false>(h, d_stream, m, smem, boff, op, axis3, d_out, out_dtype, err, st);
}

}  // namespace hc
