// hc_group.cuh -- grouped bit-unpacking of a 32-code block segment and the
// 1-D bulk-copy (TMA) helpers of the warp-autonomous kernels.
//
// Decoding (Section IV, Algorithm 2 stage 2): code k of a segment of width w
// holds |p_k| at bits [k w, (k + 1) w) of the magnitude words and its sign at
// bit k of the sign word.  With G w <= 32 (G = 2, 3 or 4, chosen on the host
// from the stream's largest width), the G codes of a group lie inside one
// 32-bit funnel shift of a two-word window, so the window moves once per
// group instead of once per code, and each code costs a shift, a masked xor
// with its sign mask and a byte permute that spreads its sign bit:
//   x_k = |p_k| ^ neg_k,  neg_k = 0 or -1 (sign), so p_k = x_k - neg_k.
// Consumers fold the "- neg_k" into their own adds (IADD3) or, for weighted
// sums, into a per-segment popcount correction.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hc_internal.cuh"

namespace hc {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// 0xffffffff when bit 8 j + 7 of v is set, else 0: the byte permute's sign
// replication (selector nibbles 8 | j) of byte j into all four bytes.  j is a
// compile-time constant at every call site (unrolled loops).
__device__ __forceinline__ uint32_t byte_sign(uint32_t v, uint32_t j) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(v), "r"(0u), "r"(0x8888u + j * 0x1111u));
  return r;
}

// Decode one full 32-code segment of width 1 <= w <= 32 / G.  mw: the
// segment's first magnitude word in shared memory (the window reads up to
// two words past the segment's last magnitude word; callers leave that much
// readable slack after the staged payload).  f(k, x, neg) is called for
// k = 0..31 in order with x = |p_k| ^ neg and neg = 0 / -1.
//
// The window (lo, hi) slides one word when a group crosses a word boundary,
// with the next word already loaded (nx), so every payload word is read from
// shared memory once.  Measured on GB300 against a window read by index for
// each group (two loads per group, word index by multiply) and against
// moving the in-group shifts and sums to the multiply-add pipe: both moved
// work off the integer ALU pipe but were slower (more shared loads and
// longer dependency chains), so the sliding window stays.
template <int G, class F>
__device__ __forceinline__ void decode32(const uint32_t* __restrict__ mw, uint32_t sw, uint32_t w, F&& f) {
  static_assert(G >= 1 && G <= 4, "groups of 1 to 4 codes");
  constexpr int NG = (32 + G - 1) / G;
  const uint32_t mask = (1u << w) - 1u;
  uint32_t sh[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) sh[r] = sw << r;
  uint32_t lo = mw[0], hi = mw[1], nx = mw[2];
  const uint32_t* ptr = mw + 3;
  const uint32_t gw = (uint32_t)G * w;
  const uint32_t w2 = 2u * w, w3 = 3u * w;
  uint32_t o = 0;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const uint32_t y = __funnelshift_r(lo, hi, o);
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const int k = g * G + i;
      if (k < 32) {
        const uint32_t yi = i == 0 ? y : (i == 1 ? (y >> w) : (i == 2 ? (y >> w2) : (y >> w3)));
        // bit k of sw sits at bit 8 (k / 8) + 7 of sh[7 - k % 8]
        const uint32_t neg = byte_sign(sh[7 - (k & 7)], (uint32_t)(k >> 3));
        f(k, (int32_t)((yi & mask) ^ neg), (int32_t)neg);
      }
    }
    if (g + 1 < NG) {
      o += gw;
      if (o >= 32u) {
        o -= 32u;
        lo = hi;
        hi = nx;
        nx = *ptr++;
      }
    }
  }
}

// decode32 over two independent segments (a, b) side by side: the same
// sliding windows, one per segment, advanced in the same unrolled loop, so
// the two dependency chains (window moves, running sums in the callbacks)
// interleave instead of running one after the other.  fa(k, x, neg) and
// fb(k, x, neg) are called for k = 0..31 in order, as in decode32.  A
// segment of width 0 decodes to x = neg (p = 0); its sign word and window
// words are then whatever follows in shared memory, which callers must
// keep readable (three words past the segment's start).
template <int G, class FA, class FB>
__device__ __forceinline__ void decode32x2(const uint32_t* __restrict__ ma, uint32_t sa, uint32_t wa,
                                           const uint32_t* __restrict__ mb, uint32_t sb, uint32_t wb, FA&& fa,
                                           FB&& fb) {
  static_assert(G >= 1 && G <= 4, "groups of 1 to 4 codes");
  constexpr int NG = (32 + G - 1) / G;
  const uint32_t mska = (1u << wa) - 1u, mskb = (1u << wb) - 1u;
  uint32_t sha[8], shb[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    sha[r] = sa << r;
    shb[r] = sb << r;
  }
  uint32_t loa = ma[0], hia = ma[1], nxa = ma[2];
  uint32_t lob = mb[0], hib = mb[1], nxb = mb[2];
  const uint32_t* pa = ma + 3;
  const uint32_t* pb = mb + 3;
  const uint32_t gwa = (uint32_t)G * wa, gwb = (uint32_t)G * wb;
  uint32_t oa = 0, ob = 0;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const uint32_t ya = __funnelshift_r(loa, hia, oa);
    const uint32_t yb = __funnelshift_r(lob, hib, ob);
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const int k = g * G + i;
      if (k < 32) {
        const uint32_t yia = ya >> (i * wa), yib = yb >> (i * wb);
        const uint32_t nega = byte_sign(sha[7 - (k & 7)], (uint32_t)(k >> 3));
        const uint32_t negb = byte_sign(shb[7 - (k & 7)], (uint32_t)(k >> 3));
        fa(k, (int32_t)((yia & mska) ^ nega), (int32_t)nega);
        fb(k, (int32_t)((yib & mskb) ^ negb), (int32_t)negb);
      }
    }
    if (g + 1 < NG) {
      oa += gwa;
      if (oa >= 32u) {
        oa -= 32u;
        loa = hia;
        hia = nxa;
        nxa = *pa++;
      }
      ob += gwb;
      if (ob >= 32u) {
        ob -= 32u;
        lob = hib;
        hib = nxb;
        nxb = *pb++;
      }
    }
  }
}

// decode32 with each group's window read by index: group g's first bit is
// g G w, its word (g G w) / 32, both found with multiply-adds, and the two
// window words are loaded for every group.  Twice the shared loads of the
// sliding window, but no compares and predicated moves on the integer ALU
// pipe and no dependency from one group to the next.  Measured on GB300:
// faster inside the stencil tiles, whose stencil arithmetic keeps the ALU
// pipe busy (the one-pass kernel 0.77 -> 0.81 of HBM on 512^3), slower in
// the statistics kernel, where the extra shared loads dominate.  Reads at
// most one word past the segment's last magnitude word.
template <int G, class F>
__device__ __forceinline__ void decode32_ix(const uint32_t* __restrict__ mw, uint32_t sw, uint32_t w, F&& f) {
  static_assert(G >= 1 && G <= 4, "groups of 1 to 4 codes");
  constexpr int NG = (32 + G - 1) / G;
  const uint32_t mask = (1u << w) - 1u;
  uint32_t sh[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) sh[r] = sw << r;
  const uint32_t gw = (uint32_t)G * w;
  // multipliers of the in-group shifts by w, 2 w, 3 w: y >> s = hi32(y 2^(32 - s))
  const uint32_t m1 = 1u << (32u - w);
  const uint32_t m2 = G > 2 ? 1u << (32u - 2u * w) : 0u;
  const uint32_t m3 = G > 3 ? 1u << (32u - 3u * w) : 0u;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const uint32_t bp = (uint32_t)g * gw;       // first bit of the group
    const uint32_t j = __umulhi(bp, 1u << 27);  // its word: bp / 32
    const uint32_t y = __funnelshift_r(mw[j], mw[j + 1], bp);
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const int k = g * G + i;
      if (k < 32) {
        const uint32_t yi = i == 0 ? y : __umulhi(y, i == 1 ? m1 : (i == 2 ? m2 : m3));
        const uint32_t neg = byte_sign(sh[7 - (k & 7)], (uint32_t)(k >> 3));
        f(k, (int32_t)((yi & mask) ^ neg), (int32_t)neg);
      }
    }
  }
}

// Group size of the grouped unpacker for a stream whose widths are at most
// wmax: the most codes whose bits fit one 32-bit funnel shift (1 = the
// one-code sliding window of unpack_full).
__host__ __device__ inline int group_for_width(uint32_t wmax) {
  return wmax <= 8u ? 4 : (wmax <= 10u ? 3 : (wmax <= 16u ? 2 : 1));
}

// decode32_ix with the group size chosen at run time (uniform over a launch,
// so no divergence); grp = 1 falls back to the one-code window (any width).
// The stencil tiles' decoder.
template <class F>
__device__ __forceinline__ void decode32_grp(int grp, const uint32_t* __restrict__ mw, uint32_t sw, uint32_t w,
                                             F&& f) {
  if (grp == 4)
    decode32_ix<4>(mw, sw, w, f);
  else if (grp == 3)
    decode32_ix<3>(mw, sw, w, f);
  else if (grp == 2)
    decode32_ix<2>(mw, sw, w, f);
  else
    unpack_full(mw, sw, w, [&](int k, int32_t p) { f(k, p, 0); });
}

// sum_k (32 - k) b_k over the sign bits b_k of a full segment: with
// x_k = p_k + neg_k, sum_k (32 - k) p_k = sum_k (32 - k) x_k + this.
__device__ __forceinline__ int weighted_sign_count(uint32_t sw) {
  const int kb = __popc(sw & 0xAAAAAAAAu) + 2 * __popc(sw & 0xCCCCCCCCu) + 4 * __popc(sw & 0xF0F0F0F0u) +
                 8 * __popc(sw & 0xFF00FF00u) + 16 * __popc(sw & 0xFFFF0000u);
  return 32 * __popc(sw) - kb;
}

// ------------------------------------------------ 1-D bulk copies (TMA)
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Global -> shared bulk copy of `bytes` (a multiple of 16; both addresses
// 16-byte aligned), completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of `bar` to complete: false after
// `limit` polls (each poll may suspend the thread for a while).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned limit) {
  for (unsigned i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace hc
