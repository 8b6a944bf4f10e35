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
//   least-significant bit first.  Width-0 blocks have no words.  Header byte
//   140 names the predictor: delta (heads[b] = the block's first code, p_k =
//   q_k - q_{k-1}, p_0 = 0: Section IV, SZp-style metadata) or block mean
//   (HSZx: heads[b] = M_b, p_k = q_k - M_b for every k).
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
  int gshift;      // log2(G) when G is a power of two, else -1
  int pred;        // hc_predictor: heads are first codes (delta) or block means (HSZx)
};

// First block of the chunk that holds block b (a shift when G is a power of two).
__device__ __forceinline__ int64_t chunk_start(const DevStream& s, int64_t b) {
  return s.gshift >= 0 ? (b >> s.gshift) << s.gshift : (b / s.G) * s.G;
}
__device__ __forceinline__ int64_t chunk_of(const DevStream& s, int64_t b) {
  return s.gshift >= 0 ? (b >> s.gshift) : b / s.G;
}

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



// Full 32-element segment of any width 1..31 (width 0 is handled by callers).
// A width-specialised unpacker (compile-time shifts per width, with warps
// handed segments of one width by a per-tile sort) was measured slower in
// every kernel on GB300: the sort's padding idles lanes and adds barriers, and
// the specialised code strains the instruction cache.  The sliding window is
// the one unpacker.
template <class F>
__device__ __forceinline__ void unpack_full(const uint32_t* mw, uint32_t sw, uint32_t w, F&& f) {
  unpack_segment<true>(mw, sw, w, 32, f);
}

// Any segment: full ones skip the per-code count check.
template <class F>
__device__ __forceinline__ void unpack_any(const uint32_t* mw, uint32_t sw, uint32_t w, int count, F&& f) {
  if (count == 32)
    unpack_full(mw, sw, w, f);
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
  const int64_t cs = chunk_start(s, b0);
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
  const uint64_t base = s.chunks[chunk_of(s, cs)] + s_off[npre];
  const uint32_t first = s_off[npre];
  const uint32_t words = s_off[n] - first;
  if (tid == 0) {
    // every chunk start inside the run (and the run's end, when it is one)
    // must agree with the chunk index
    const uint64_t c0 = s.chunks[chunk_of(s, cs)];
    for (int64_t cb = cs + s.G; cb <= b0 + nblk; cb += s.G) {
      const uint64_t expect = (cb >= s.nb) ? (uint64_t)s.payload_words : s.chunks[chunk_of(s, cb)];
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

// cp.async 16-byte global -> shared copies (the caller waits with
// cp_async_wait_all; both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Close this thread's current group of cp.async copies; wait until at most
// its newest group is still in flight.
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_group1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }



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

// ----------------------------------------------------- chunk-aligned tiles
// Reductions and whole-stream decoding walk tiles of whole chunks.  A
// tile's payload range comes straight from the chunk index, so the next
// tile's widths, heads and payload are copied into shared memory with
// cp.async while the current tile is decoded.
struct TileCopy {
  int64_t b0;      // first block
  int nblk;        // blocks
  uint64_t p0, p1;  // payload words [p0, p1)
};

// tb: blocks per tile, a whole number of chunks (tb / G of them).
__device__ __forceinline__ TileCopy tile_bounds(const DevStream& s, int64_t t, int tb) {
  TileCopy c;
  c.b0 = t * tb;
  c.nblk = (int)min((int64_t)tb, s.nb - c.b0);
  const int64_t nch = tb / s.G;
  const int64_t c0 = t * nch;
  c.p0 = __ldg(s.chunks + c0);
  c.p1 = __ldg(s.chunks + min(c0 + nch, s.nchunks));
  return c;
}

// Issue the copies of one tile (every thread of the CTA takes a share).
// Buffers: w (tb + 32 bytes), h (tb + 8 ints), words (stage_words).  Returns
// false when the chunk index is inconsistent (nothing is copied then).
__device__ inline bool tile_issue(const DevStream& s, const TileCopy& c, int stage_words, uint8_t* w, int32_t* h,
                                  uint32_t* words) {
  if (c.p1 < c.p0 || c.p1 > (uint64_t)s.payload_words || (int64_t)(c.p1 - c.p0) + 8 > stage_words) return false;
  const int tid = threadIdx.x, nt = blockDim.x;
  // widths: bytes [b0, b0 + nblk), from a 16-byte aligned start
  const int64_t w0 = c.b0 & ~(int64_t)15;
  const int nw = (int)((c.b0 + c.nblk - w0 + 15) >> 4);
  for (int i = tid; i < nw; i += nt) cp_async16(w + 16 * i, s.widths + w0 + 16 * i);
  // heads: ints [b0, b0 + nblk)
  const int64_t h0 = c.b0 & ~(int64_t)3;
  const int nh = (int)((c.b0 + c.nblk - h0 + 3) >> 2);
  for (int i = tid; i < nh; i += nt) cp_async16(h + 4 * i, s.heads + h0 + 4 * i);
  // payload: words [p0, p1] (one word past the end for the unpacker)
  const uint64_t a0 = c.p0 & ~(uint64_t)3;
  const int np = (int)((c.p1 + 1 - a0 + 3) >> 2);
  for (int i = tid; i < np; i += nt) cp_async16(words + 4 * i, s.payload + a0 + 4 * i);
  return true;
}

// After the copies of tile c have landed: scan its widths into staging offsets.
// Fills tv (widths, offsets, payload views into the staged buffers).  Returns
// false (and records HC_ERR_CORRUPT) if the widths disagree with the chunk
// index.  Every thread of the CTA must call it.
__device__ inline bool tile_ready(const DevStream& s, const TileCopy& c, bool issued, const uint8_t* w,
                                  uint32_t* s_off, const uint32_t* words, uint32_t* s_warp, int* s_flag, int* err,
                                  TileView& tv) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int wlead = (int)(c.b0 & 15);
  if (tid == 0) *s_flag = issued ? 0 : 1;
  __syncthreads();
  for (int i = tid; i < c.nblk; i += nt) {
    uint32_t wi = w[wlead + i];
    if (wi > (uint32_t)s.wmax) {
      atomicOr(s_flag, 1);
      wi = 0;
    }
    s_off[i] = block_words(s.S, s.nseg, wi);
  }
  __syncthreads();
  const uint32_t total = cta_exclusive_scan(s_off, c.nblk, s_warp);
  const bool bad = (*s_flag != 0) || (uint64_t)total != c.p1 - c.p0;
  if (bad) {
    __syncthreads();
    if (tid == 0) set_error(err, HC_ERR_CORRUPT);
    return false;
  }
  const int lead = (int)(c.p0 & 3);
  for (int i = tid; i < c.nblk; i += nt) s_off[i] += lead;
  __syncthreads();
  tv.w = w + wlead;
  tv.off = s_off;
  tv.words = words;
  tv.b0 = c.b0;
  tv.nblk = c.nblk;
  return true;
}

// Shared-memory layout (32-bit word offsets) of a kernel walking
// chunk-aligned tiles with two copy buffers, each [widths | heads | payload],
// followed by the block offsets and `extra` words of the kernel's own.
struct PipeTileSmem {
  int wbuf, hbuf, pbuf, buf;  // offsets inside one buffer; buffer size
  int off, extra, total;
  __device__ uint8_t* w(uint32_t* sm, int b) const { return reinterpret_cast<uint8_t*>(sm + b * buf + wbuf); }
  __device__ int32_t* h(uint32_t* sm, int b) const { return reinterpret_cast<int32_t*>(sm + b * buf + hbuf); }
  __device__ uint32_t* words(uint32_t* sm, int b) const { return sm + b * buf + pbuf; }
};
__host__ __device__ inline PipeTileSmem pipe_tile_smem(int tb, int stage_words, int extra_words) {
  PipeTileSmem p;
  p.wbuf = 0;
  p.hbuf = round4((tb + 32 + 3) / 4);
  p.pbuf = p.hbuf + round4(tb + 8);
  p.buf = p.pbuf + round4(stage_words);
  p.off = 2 * p.buf;
  p.extra = p.off + round4(tb + 1);
  p.total = p.extra + round4(extra_words);
  return p;
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

// Final scaling of exact sums into a statistic result (Section V-A, Eq. var_q):
//   mean = (s1 / N) * 2 eps,
//   var  = ((N s2 - s1^2) / (N (N - 1))) * (2 eps)^2   (exact 128-bit numerator).
__device__ inline void finalize_int(hc_scalar* out, int64_t n, long long s1, u128 s2, bool var, double two_eps,
                                    int err) {
  out->n = n;
  out->s1 = s1;
  out->s2_lo = var ? (unsigned long long)s2 : 0ull;
  out->s2_hi = var ? (unsigned long long)(s2 >> 64) : 0ull;
  out->status = err;
  out->exact = 1;
  out->mean = (__ll2double_rn(s1) / (double)n) * two_eps;
  double v = __longlong_as_double(0x7ff8000000000000ll);  // NaN: not computed / undefined
  if (var && n >= 2) {
    const i128 num = (i128)n * (i128)s2 - (i128)s1 * (i128)s1;
    const double den = (double)n * (double)(n - 1);
    v = (i128_to_double(num) / den) * (two_eps * two_eps);
  }
  out->variance = v;
  out->std = sqrt(v);
}

// Stage-2 standard deviation of HSZx (Section V-A): s2 is the exact sum of
// squared deviations from the integer mean mu~; variance = s2 / (N - 1) *
// (2 eps)^2 (the paper's form, not Eq. var_q), mean from the exact s1.
__device__ inline void finalize_about(hc_scalar* out, int64_t n, long long s1, u128 s2, long long mu, double two_eps,
                                      int err) {
  (void)mu;
  out->n = n;
  out->s1 = s1;
  out->s2_lo = (unsigned long long)s2;
  out->s2_hi = (unsigned long long)(s2 >> 64);
  out->status = err;
  out->exact = 0;
  out->mean = (__ll2double_rn(s1) / (double)n) * two_eps;
  double v = __longlong_as_double(0x7ff8000000000000ll);
  if (n >= 2) v = (i128_to_double((i128)s2) / (double)(n - 1)) * (two_eps * two_eps);
  out->variance = v;
  out->std = sqrt(v);
}

}  // namespace hc
