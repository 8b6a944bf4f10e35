// hc_internal.cuh -- device-side building blocks shared by the kernels of
// libhc.so: the stream view, error reporting, a CTA-wide scan, the
// per-thread segment decoder and the tile loader.
//
// Stream layout (little-endian; the bytes are a parity target):
//   header 256 B | widths u8[nb] | heads i32[nb] | chunk index u64[nchunks+1]
//   | payload u32[payload_words] | >= 16 zero bytes.  Sections start on
//   16-byte boundaries.  A chunk is G = max(1, 4096/S) blocks; chunk[c] is the
//   payload word of its first block.  A block of width w > 0 holds
//   ceil(S/32) sign words (bit k%32 of word k/32 set iff p_k < 0) and then
//   ceil(S*w/32) magnitude words with |p_k| at bits [k*w, (k+1)*w),
//   least-significant bit first.  p_0 = 0: the block's first code (head) is
//   metadata (Section IV, SZp-style metadata).  Width-0 blocks have no words.
//
// Decoding works on 32-element "segments": segment j of a block covers
// elements [32j, 32j+32).  Its signs are sign word j and its magnitudes start
// exactly at magnitude word j*w (32 values of w bits are w words), so every
// segment decodes independently of the others.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hc.h"

namespace hc {

constexpr int kThreads = 256;
constexpr int kHeaderBytes = 256;
constexpr uint32_t kMagic = 0x315A4348u;
constexpr int kVersion = 1;
constexpr int kChunkElems = 4096;
constexpr int kMaxS = 4096;
constexpr int32_t kQLimit = 1 << 30;
constexpr int kTileChunks = 2;  // reductions and decompression walk the stream two chunks at a time

// Pointers into a device-resident stream plus the sizes a kernel needs.
struct DevStream {
  const uint8_t* widths;
  const int32_t* heads;
  const uint64_t* chunks;
  const uint32_t* payload;
  int64_t N, nb, nchunks, payload_words;
  int S, G, nseg;  // nseg = ceil(S/32): sign words and segments per block
  int wmax;        // largest block width recorded in the header (sizes the staging buffers)
};

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Payload words of a block of width w (0 for w = 0).
__device__ __forceinline__ uint32_t block_words(int S, int nseg, uint32_t w) {
  return w ? (uint32_t)nseg + (((uint32_t)S * w + 31u) >> 5) : 0u;
}

// First error wins; a NULL status pointer disables reporting only.
__device__ __forceinline__ void set_error(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// Exclusive scan of s_val[0..n) in shared memory, in place; s_val[n] receives
// the total, which is also returned.  s_warp: 32 words of shared scratch.
// Every thread of the CTA must call it.
__device__ inline uint32_t cta_exclusive_scan(uint32_t* s_val, int n, uint32_t* s_warp) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int ipt = (n + nt - 1) / nt;
  const int beg = min(tid * ipt, n), end = min(beg + ipt, n);
  uint32_t local = 0;
  for (int i = beg; i < end; ++i) local += s_val[i];
  uint32_t x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t v = lane < (nt >> 5) ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    s_warp[lane] = v;
  }
  __syncthreads();
  uint32_t run = x - local + (wid ? s_warp[wid - 1] : 0u);
  for (int i = beg; i < end; ++i) {
    uint32_t v = s_val[i];
    s_val[i] = run;
    run += v;
  }
  const uint32_t total = s_warp[(nt >> 5) - 1];
  __syncthreads();
  if (tid == 0) s_val[n] = total;
  __syncthreads();
  return total;
}

// Unpack one segment: count (<= 32) values of w bits (1 <= w <= 31) starting
// at mw[0] bit 0, signs in sw.  f(i, p) is called for i = 0..count-1 in order.
// The bit window (lo:hi) slides one word at a time, so each payload word is
// loaded once; at most one word past the segment's last magnitude word is
// read (the tile loader stages that word, and the stream is padded).
template <bool FULL, class F>
__device__ __forceinline__ void unpack_segment(const uint32_t* __restrict__ mw, uint32_t sw, uint32_t w,
                                               int count, F&& f) {
  const uint32_t mask = (1u << w) - 1u;
  uint32_t lo = mw[0], hi = mw[1];
  const uint32_t* ptr = mw + 2;
  uint32_t o = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    if (FULL || i < count) {
      const uint32_t m = __funnelshift_r(lo, hi, o) & mask;
      const int32_t neg = -(int32_t)((sw >> i) & 1u);
      f(i, ((int32_t)m ^ neg) - neg);
      if (i < 31) {
        o += w;
        if (o >= 32u) {
          o -= 32u;
          lo = hi;
          hi = *ptr++;
        }
      }
    }
  }
}

template <class F>
__device__ __forceinline__ void unpack_any(const uint32_t* mw, uint32_t sw, uint32_t w, int count, F&& f) {
  if (count == 32)
    unpack_segment<true>(mw, sw, w, 32, f);
  else
    unpack_segment<false>(mw, sw, w, count, f);
}

// Shared-memory description of a run of consecutive blocks [b0, b0 + nblk)
// whose payload has been staged: per block its width, its word offset inside
// the staging buffer and its head.
struct TileView {
  const uint8_t* w;     // widths (shared)
  const uint32_t* off;  // staging word offset of each block (shared)
  const uint32_t* words;  // staged payload (shared)
  int64_t b0;
  int nblk;
};

// Load widths / offsets / payload of blocks [b0, b0 + nblk) into shared
// memory.  The offsets are found from the chunk index entry of b0's chunk and
// a scan of the widths from that chunk's first block (at most G-1 extra
// widths).  Buffers (shared):
//   s_w      u8  [npre_max + nblk_max]   widths
//   s_off    u32 [npre_max + nblk_max + 1] word offsets
//   s_stage  u32 [stage_words]            payload (+1 word past the end)
// Returns false (and records HC_ERR_CORRUPT) if the stream is inconsistent;
// every thread gets the same answer.  Must be called by the whole CTA.
__device__ inline bool load_blocks(const DevStream& s, int64_t b0, int nblk, uint8_t* s_w, uint32_t* s_off,
                                   uint32_t* s_stage, int stage_words, uint32_t* s_warp, int* s_flag,
                                   int* err, TileView& tv) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t cs = (b0 / s.G) * s.G;
  const int npre = (int)(b0 - cs);
  const int n = npre + nblk;
  if (tid == 0) *s_flag = 0;
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    uint32_t w = s.widths[cs + i];
    if (w > 31u) {
      atomicOr(s_flag, 1);
      w = 31u;
    }
    s_w[i] = (uint8_t)w;
    s_off[i] = block_words(s.S, s.nseg, w);
  }
  __syncthreads();
  cta_exclusive_scan(s_off, n, s_warp);
  const uint64_t base = s.chunks[cs / s.G] + s_off[npre];
  const uint32_t first = s_off[npre];
  const uint32_t words = s_off[n] - first;
  if (tid == 0) {
    // every chunk start inside the run (and the run's end, when it is one)
    // must agree with the chunk index
    const uint64_t c0 = s.chunks[cs / s.G];
    for (int64_t cb = cs + s.G; cb <= b0 + nblk; cb += s.G) {
      const uint64_t expect = (cb >= s.nb) ? (uint64_t)s.payload_words : s.chunks[cb / s.G];
      if (c0 + s_off[cb - cs] != expect) *s_flag = 1;
    }
    if (b0 + nblk == s.nb && c0 + s_off[n] != (uint64_t)s.payload_words) *s_flag = 1;
  }
  __syncthreads();
  const bool bad = (*s_flag != 0) || base + words > (uint64_t)s.payload_words ||
                   (int64_t)words + 8 > (int64_t)stage_words;
  __syncthreads();
  if (bad) {
    if (tid == 0) set_error(err, HC_ERR_CORRUPT);
    return false;
  }
  // Stage words [base, base + words] (one extra word: the unpacker's window)
  // with 16-byte vector loads from a 16-byte aligned start.
  const uint64_t a0 = base & ~(uint64_t)3;
  const int lead = (int)(base - a0);
  const int nvec = (lead + (int)words + 1 + 3) >> 2;
  const uint4* src = reinterpret_cast<const uint4*>(s.payload + a0);
  uint4* dst = reinterpret_cast<uint4*>(s_stage);
  for (int i = tid; i < nvec; i += nt) dst[i] = __ldg(src + i);
  // offsets relative to the staging buffer
  for (int i = tid; i < nblk; i += nt) s_off[npre + i] = s_off[npre + i] - first + lead;
  __syncthreads();
  tv.w = s_w + npre;
  tv.off = s_off + npre;
  tv.words = s_stage;
  tv.b0 = b0;
  tv.nblk = nblk;
  return true;
}

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

// Size in words of the staging buffer for up to nblk blocks of width at most
// wmax (a multiple of 4).  A block wider than the header's wmax makes the
// loader report HC_ERR_CORRUPT instead of overflowing the buffer.
__host__ __device__ inline int stage_words_for(int nblk, int S, int wmax) {
  const int nseg = (S + 31) / 32;
  return round4(nblk * (wmax ? nseg + (S * wmax + 31) / 32 : 0) + 8);
}

// Dynamic shared-memory layout (32-bit word offsets) of a kernel that uses
// load_blocks for up to nblk_max blocks preceded by up to npre_max blocks of
// the same chunk, plus `extra_words` of its own (16-byte aligned):
//   [stage | off | extra | widths]
struct TileSmem {
  int stage_words;  // capacity of the staging buffer
  int off;          // offset of the block offsets
  int extra;        // offset of the kernel's own region
  int w;            // offset of the width bytes
  int words;        // total
};
__host__ __device__ inline TileSmem tile_smem(int nblk_max, int npre_max, int S, int wmax, int extra_words) {
  TileSmem t;
  t.stage_words = stage_words_for(nblk_max, S, wmax);
  t.off = t.stage_words;
  t.extra = t.off + round4(npre_max + nblk_max + 1);
  t.w = t.extra + round4(extra_words);
  t.words = t.w + round4((npre_max + nblk_max + 3) / 4 + 1);
  return t;
}

// 128-bit helpers ------------------------------------------------------
typedef unsigned __int128 u128;
typedef __int128 i128;

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int o) {
  uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
  lo = __shfl_down_sync(0xffffffffu, lo, o);
  hi = __shfl_down_sync(0xffffffffu, hi, o);
  return ((u128)hi << 64) | lo;
}

// Correctly rounded (round-to-nearest-even) conversion of a signed 128-bit
// integer to double: the top 64 significant bits are converted by the
// hardware with the discarded lower bits folded into a sticky bit.
__device__ inline double i128_to_double(i128 x) {
  const bool neg = x < 0;
  u128 u = neg ? (u128)(-x) : (u128)x;
  const uint64_t hi = (uint64_t)(u >> 64);
  double r;
  if (hi == 0) {
    r = __ull2double_rn((uint64_t)u);
  } else {
    const int shift = 64 - __clzll((long long)hi);  // 1..64
    uint64_t top = (uint64_t)(u >> shift);
    const u128 dropped = u & (((u128)1 << shift) - 1);
    top |= (dropped != 0) ? 1ull : 0ull;
    r = ldexp(__ull2double_rn(top), shift);
  }
  return neg ? -r : r;
}

}  // namespace hc
