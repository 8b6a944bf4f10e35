// hc_reduce32.cu -- fused homomorphic statistics (Section V-A) for the common
// stream shape: block size 32, block widths <= 16, codes |q| < 2^26.
//
// Same results as k_reduce_stream (exact s1 = sum q, s2 = sum q^2 and the
// final scaling of Eq. var_q); a different schedule:
//  * every warp works alone on whole chunks (128 blocks, 4096 codes): the
//    chunk index gives the chunk's payload range, so no warp waits for
//    another and there is no CTA barrier until the final sum;
//  * one lane copies the next chunk's payload into the warp's other shared
//    buffer with a 1-D bulk copy (TMA) completing on an mbarrier, while the
//    warp decodes the current chunk; widths and heads come straight into
//    registers (one coalesced 4-byte and one 16-byte load per lane, one
//    iteration ahead);
//  * lane l decodes blocks 4l .. 4l+3 of the chunk with the grouped unpacker
//    (hc_group.cuh: G codes per window step, G = 4, 3 or 2 from the stream's
//    largest width).
// Per code: stage 2 ("Operation with D_p") is one multiply-add of the
// block-weighted sum sum_k (32 - k) p_k, no prefix sum; stage 3 ("Operation
// with D_q") rebuilds q with the running (eta) accumulator and adds q (mean)
// and q^2 (variance).  Block-mean (HSZx) streams: q = M_b + p, so the sums
// follow from sum p and sum p^2 per block.  HSZx-nd streams of boxes of 64
// or 128 slots (BPL = 2 or 1 boxes per lane of a 4096-code chunk) take the
// same path: a box is 2 or 4 consecutive 32-slot segments, its mean M_b
// weighted by the box's true size S_b (padding slots hold p = 0).
#include <cstdint>
#include <type_traits>

#include "hc_finish.cuh"
#include "hc_group.cuh"
#include "hc_internal.cuh"
#include "hc_launch.h"

namespace hc {

DevStream dev_stream(const hc_header* h, const void* d_stream);

namespace {

constexpr int kWarps = 4;          // warps per CTA
constexpr int kChunkSegs = 128;    // 32-slot segments per chunk (4096 codes)
constexpr unsigned kWaitPolls = 1u << 22;

// What a launch sums: the stage-2 weighted sum (mean), the stage-3 sum
// (mean), or the stage-3 sums of q and q^2 (variance).
enum Op { OP_MEAN_P = 0, OP_MEAN_Q = 1, OP_VAR = 2, OP_MEAN_G = 3 };
// OP_MEAN_G: the stage-2 mean of a global-predictor stream (HSZp-nd Lorenzo
// residuals, or HSZp's delta across blocks), sum q = sum_i p_i (L0 - z)(L1 -
// y)(L2 - x) over the prediction shape L, modulo 2^64 (exact: sum q fits
// 63 bits).  For a block of 32 codes inside one row starting at x0, sum_k p_k
// (L2 - x0 - k) = (L2 - x0 - 32) sum_k p_k + sum_k (32 - k) p_k: two sums per
// block, the second the stage-2 weighted sum of the block-head streams.

// Words of one chunk buffer: 128 blocks of at most wmax + 1 words, the
// copy's 16-byte alignment on both ends and the decoder's read-ahead.
__host__ __device__ inline int chunk_buf_words(int wmax) { return round4(kChunkSegs * (wmax + 1) + 3 + 3 + 8); }
__host__ __device__ inline int smem_bytes(int buf_words) { return 128 + kWarps * 2 * buf_words * 4; }

// Widths and heads of the lane's BPL blocks (boxes) of a chunk, blocks
// BPL lane .. BPL lane + BPL - 1 (byte j of w4 and lane j of h4: block
// BPL lane + j): one load of widths and one of heads per lane, loaded one
// iteration before use.  (Interleaving the blocks over the lanes, block 32 j
// + lane, lowers shared-memory bank conflicts but needs eight narrow loads
// per lane; measured slower.)
struct ChunkData {
  uint32_t w4;
  int4 h4;
};
// Payload words [p0, p1) of a chunk, loaded two iterations before use (one
// iteration before its bulk copy is issued).
struct ChunkRange {
  uint64_t p0, p1;
};

template <int BPL>
__device__ __forceinline__ ChunkData load_data(const DevStream& s, int64_t c, int lane) {
  ChunkData m;
  const int64_t b = c * (32 * BPL) + BPL * lane;
  m.w4 = 0;
  m.h4 = make_int4(0, 0, 0, 0);
  if (c < s.nchunks && b < s.nb) {
    // b is a multiple of BPL: aligned widths and heads; a lane whose last
    // blocks lie past nb reads at most BPL - 1 bytes / 4 (BPL - 1) bytes
    // beyond the sections' ends, inside their 16-byte padding
    if constexpr (BPL == 4) {
      m.w4 = __ldg(reinterpret_cast<const uint32_t*>(s.widths + b));
      m.h4 = __ldg(reinterpret_cast<const int4*>(s.heads + b));
    } else if constexpr (BPL == 2) {
      m.w4 = __ldg(reinterpret_cast<const uint16_t*>(s.widths + b));
      const int2 h2 = __ldg(reinterpret_cast<const int2*>(s.heads + b));
      m.h4.x = h2.x;
      m.h4.y = h2.y;
    } else {
      m.w4 = __ldg(s.widths + b);
      m.h4.x = __ldg(s.heads + b);
    }
  }
  return m;
}

// Box geometry of an HSZx-nd stream, for the true sizes of ragged boxes at
// the field's far faces (unused for 1-D blocks and when every box is full);
// for OP_MEAN_G, (n0, n1, n2) is the prediction shape L and `ragged` says
// that blocks cross row ends.
struct BoxDims {
  int64_t n0, n1, n2, g1, g2;
  int b0, b1, b2;
  int ragged;
};
__device__ __forceinline__ long long box_size(const BoxDims& d, int64_t b, int S) {
  if (!d.ragged) return S;
  const int64_t k2 = b % d.g2, r = b / d.g2;
  const int64_t k1 = r % d.g1, k0 = r / d.g1;
  return min((int64_t)d.b0, d.n0 - k0 * d.b0) * min((int64_t)d.b1, d.n1 - k1 * d.b1) *
         min((int64_t)d.b2, d.n2 - k2 * d.b2);
}

__device__ __forceinline__ ChunkRange load_range(const DevStream& s, int64_t c) {
  ChunkRange r{0, 0};
  if (c < s.nchunks) {
    r.p0 = __ldg(s.chunks + c);
    r.p1 = __ldg(s.chunks + c + 1);
  }
  return r;
}

template <int G, int OP, int ACC, int PRED, int BPL>
__global__ void __launch_bounds__(kWarps * 32, 5) k_reduce32(DevStream s, int buf_words, Partial* parts,
                                                          unsigned* ticket, hc_scalar* out, double two_eps,
                                                          const long long* shift, BoxDims bd) {
  constexpr int SEGS = 4 / BPL;  // 32-slot segments per block (box)
  extern __shared__ __align__(128) unsigned char sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm) + 2 * warp;
  uint32_t* bufs = reinterpret_cast<uint32_t*>(sm + 128) + (size_t)(2 * warp) * buf_words;
  const long long c0 = shift ? __ldcg(shift) : 0ll;
  const int64_t stride = (int64_t)gridDim.x * kWarps;
  int err = 0;
  long long S1 = 0;
  u128 S2 = 0;
  unsigned long long G1 = 0;  // OP_MEAN_G: sum q modulo 2^64

  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    fence_mbar_init();
  }
  __syncwarp();

  // Copy of a chunk's payload into buffer b by lane 0: words [a0, end) with
  // a0 = p0 rounded down and end = p1 rounded up to 16 bytes (the stream keeps
  // >= 16 zero bytes after the payload).  False (nothing issued) when the
  // chunk index is inconsistent or the chunk holds no payload words.
  auto issue = [&](const ChunkRange& m, int b) -> bool {
    if (m.p1 < m.p0 || m.p1 > (uint64_t)s.payload_words) return false;
    const uint64_t a0 = m.p0 & ~(uint64_t)3, end = (m.p1 + 3) & ~(uint64_t)3;
    if ((int64_t)(end - a0) + 8 > (int64_t)buf_words || end == a0) return false;
    if (lane == 0) {
      const unsigned bytes = (unsigned)((end - a0) * 4);
      mbar_expect_tx(bar + b, bytes);
      bulk_g2s(bufs + (size_t)b * buf_words, s.payload + a0, bytes, bar + b);
    }
    return true;
  };

  // Software pipeline over the warp's chunks c, c + stride, ...: at the
  // iteration of chunk c the copy of c + stride is issued (its range was
  // loaded one iteration earlier), the widths and heads of c + stride and the
  // range of c + 2 stride are loaded, and chunk c is decoded.
  int64_t c = (int64_t)blockIdx.x * kWarps + warp;
  ChunkRange cur_r = load_range(s, c);
  ChunkData cur = load_data<BPL>(s, c, lane);
  ChunkRange nxt_r = load_range(s, c + stride);
  bool cur_issued = c < s.nchunks && issue(cur_r, 0);
  unsigned phase = 0;  // bit b: parity of buffer b's next completion
  for (int i = 0; c < s.nchunks; c += stride, ++i) {
    const int b = i & 1;
    const int64_t cn = c + stride;
    bool nxt_issued = false;
    if (cn < s.nchunks) {
      // every lane is done with buffer b ^ 1 (chunk c - stride) before the
      // bulk copy overwrites it
      __syncwarp();
      if (lane == 0) fence_proxy_async_smem();
      nxt_issued = issue(nxt_r, b ^ 1);
    }
    const ChunkData nxt = load_data<BPL>(s, cn, lane);
    const ChunkRange nn_r = load_range(s, cn + stride);
    // block offsets inside the chunk: exclusive scan of the block sizes
    // (SEGS sign words + SEGS w magnitude words, 0 for width 0)
    const int64_t bb = c * (32 * BPL) + BPL * lane;
    uint32_t wj[BPL], oj[BPL];
    uint32_t lsum = 0;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < BPL; ++j) {
      uint32_t w = (cur.w4 >> (8 * j)) & 0xffu;
      if (bb + j >= s.nb) w = 0;
      if (w > (uint32_t)s.wmax) {
        bad = true;
        w = 0;
      }
      wj[j] = w;
      oj[j] = lsum;
      lsum += w ? SEGS * (w + 1u) : 0u;
    }
    uint32_t incl = lsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    bad = __any_sync(0xffffffffu, bad) || (!cur_issued && total != 0) || (uint64_t)total != cur_r.p1 - cur_r.p0;
    if (cur_issued) {
      // every lane waits (each observes the copy's completion itself); the
      // outcome is made warp-uniform so the warp leaves together on a timeout
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar + b, (phase >> b) & 1u, kWaitPolls))) {
        err = HC_ERR_TIMEOUT;
        if (nxt_issued) mbar_wait_bounded(bar + (b ^ 1), (phase >> (b ^ 1)) & 1u, kWaitPolls);
        break;
      }
      phase ^= 1u << b;
    }
    if (bad) {
      err = HC_ERR_CORRUPT;
    } else {
      const uint32_t* base = bufs + (size_t)b * buf_words + (uint32_t)(cur_r.p0 & 3) + (incl - lsum);
      const int32_t hj[4] = {cur.h4.x, cur.h4.y, cur.h4.z, cur.h4.w};
      constexpr bool kPairs = BPL == 4 && PRED == HC_PRED_DELTA && (OP == OP_MEAN_P || OP == OP_MEAN_Q);
      // the lane's four blocks all full (every lane but the one holding the
      // stream's last blocks): decoded two at a time, side by side; a block
      // of width 0 goes through the same arithmetic (it decodes to p = 0)
      const bool pairs = kPairs && (bb + 4) * 32 <= s.N;
      if constexpr (kPairs) {
        if (pairs) {
#pragma unroll
          for (int j = 0; j < 4; j += 2) {
            const uint32_t* ba = base + oj[j];
            const uint32_t* bq = base + oj[j + 1];
            if constexpr (OP == OP_MEAN_P) {
              // Section V-A, stage 2: 32 head + sum_k (32 - k) p_k per block
              int32_t a = 0, c = 0;
              decode32x2<G>(
                  ba + 1, ba[0], wj[j], bq + 1, bq[0], wj[j + 1], [&](int k, int32_t x, int32_t) { a += (32 - k) * x; },
                  [&](int k, int32_t x, int32_t) { c += (32 - k) * x; });
              S1 += 32ll * ((long long)hj[j] + hj[j + 1]) + (long long)a + c + weighted_sign_count(ba[0]) +
                    weighted_sign_count(bq[0]);
            } else {
              // Section V-A, stage 3: q rebuilt from each block's head
              int32_t qa = hj[j], qc = hj[j + 1], a1 = 0, c1 = 0;
              using A2 = typename std::conditional<ACC == 0, uint32_t, unsigned long long>::type;
              A2 a2 = 0, c2 = 0;
              decode32x2<G>(
                  ba + 1, ba[0], wj[j], bq + 1, bq[0], wj[j + 1],
                  [&](int, int32_t x, int32_t neg) {
                    qa = qa + x - neg;
                    a1 += qa;
                    if (OP == OP_VAR) {
                      if constexpr (ACC == 0)
                        a2 += (uint32_t)(qa * qa);
                      else
                        a2 += (unsigned long long)((long long)qa * qa);
                    }
                  },
                  [&](int, int32_t x, int32_t neg) {
                    qc = qc + x - neg;
                    c1 += qc;
                    if (OP == OP_VAR) {
                      if constexpr (ACC == 0)
                        c2 += (uint32_t)(qc * qc);
                      else
                        c2 += (unsigned long long)((long long)qc * qc);
                    }
                  });
              S1 += (long long)a1 + c1;
              if (OP == OP_VAR) S2 += (u128)a2 + (u128)c2;
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < BPL; ++j) {
        if (pairs) break;
        const int64_t blk = bb + j;
        if (blk >= s.nb) break;
        const uint32_t w = wj[j];
        const int32_t head = hj[j];
        const uint32_t* bw = base + oj[j];
        const int cnt = (int)min((int64_t)32, s.N - blk * 32);
        if constexpr (OP == OP_MEAN_G) {
          // position of the block's first code in the prediction shape
          // (32-bit when N < 2^32, as the launch requires)
          const uint32_t e0 = (uint32_t)blk * 32u, l2 = (uint32_t)bd.n2, l1 = (uint32_t)bd.n1;
          const uint32_t r = e0 / l2, x0 = e0 - r * l2, zz = r / l1, yy = r - zz * l1;
          const unsigned long long wzy =
              (unsigned long long)((uint64_t)bd.n0 - zz) * (unsigned long long)((uint64_t)l1 - yy);
          if (w == 0 || cnt <= 0) continue;
          if (cnt == 32 && x0 + 32u <= l2) {
            // inside one row: sum p and sum (32 - k) p from the grouped unpacker
            int32_t a = 0, aw = 0;
            decode32<G>(bw + 1, bw[0], w, [&](int k, int32_t x, int32_t) {
              a += x;
              aw += (32 - k) * x;
            });
            const long long P = (long long)a + __popc(bw[0]);
            const long long R = (long long)aw + weighted_sign_count(bw[0]);
            G1 += wzy * ((unsigned long long)(l2 - x0 - 32u) * (unsigned long long)P + (unsigned long long)R);
          } else if (cnt == 32 && bd.ragged) {
            // across one row end (rows of at least 32 codes): codes k < kb end
            // row A, codes k >= kb start row B at x = k - kb; the same two sums
            // over each part (row B's from a predicated second pair), with
            // weights (L2 - x0 - 32) for A and (L2 + kb - 32) for B, modulo 2^64
            const uint32_t kb = l2 - x0;
            int32_t a = 0, aw = 0, b = 0, bw2 = 0;
            decode32<G>(bw + 1, bw[0], w, [&](int k, int32_t x, int32_t) {
              a += x;
              aw += (32 - k) * x;
              const int32_t xb = (uint32_t)k >= kb ? x : 0;
              b += xb;
              bw2 += (32 - k) * xb;
            });
            const uint32_t mb = ~0u << kb, sw = bw[0];
            const long long PB = (long long)b + __popc(sw & mb), RB = (long long)bw2 + weighted_sign_count(sw & mb);
            const long long PA = (long long)a + __popc(sw) - PB, RA = (long long)aw + weighted_sign_count(sw) - RB;
            const uint32_t yb = yy + 1u == l1 ? 0u : yy + 1u, zb = yy + 1u == l1 ? zz + 1u : zz;
            const unsigned long long wzyb =
                (unsigned long long)((uint64_t)bd.n0 - zb) * (unsigned long long)((uint64_t)l1 - yb);
            const unsigned long long wa = (unsigned long long)((long long)l2 - x0 - 32);  // negative: wraps
            G1 += wzy * (wa * (unsigned long long)PA + (unsigned long long)RA);
            G1 += wzyb * ((unsigned long long)(l2 + kb - 32u) * (unsigned long long)PB + (unsigned long long)RB);
          } else {
            // a block that crosses a row end (or the field's last one): code by code
            unsigned long long wz = wzy;
            uint32_t x = x0, y = yy, z = zz;
            unpack_segment<false>(bw + 1, bw[0], w, cnt, [&](int, int32_t p) {
              G1 += wz * (unsigned long long)(l2 - x) * (unsigned long long)(long long)p;
              if (++x == l2) {
                x = 0;
                if (++y == l1) {
                  y = 0;
                  ++z;
                }
                wz = (unsigned long long)((uint64_t)bd.n0 - z) * (unsigned long long)((uint64_t)l1 - y);
              }
            });
          }
        } else if constexpr (PRED == HC_PRED_MEAN_ND) {
          // q = M_b + p for every slot of the box's true size S_b (HSZx-nd;
          // padding slots hold p = 0): sums from sum p and sum p^2
          const long long sb = box_size(bd, blk, 32 * SEGS);
          long long sp = 0;
          unsigned long long sp2 = 0;
          if (w) {
#pragma unroll
            for (int t = 0; t < SEGS; ++t) {
              int32_t a = 0;
              unsigned long long a2 = 0;
              decode32<G>(bw + SEGS + t * w, bw[t], w, [&](int, int32_t x, int32_t neg) {
                const int32_t p = x - neg;
                a += p;
                if (OP == OP_VAR) a2 += (unsigned long long)((long long)p * p);
              });
              sp += a;
              sp2 += a2;
            }
          }
          S1 += sb * head + sp;
          if (OP == OP_VAR) {
            const long long cc = (long long)head - c0;
            S2 += (u128)((i128)sb * cc * cc + (i128)2 * cc * sp + (i128)sp2);
          }
        } else if constexpr (PRED == HC_PRED_MEAN) {
          // q = M_b + p for every slot (HSZx): sums from sum p and sum p^2
          long long sp = 0;
          unsigned long long sp2 = 0;
          if (w) {
            if (cnt == 32) {
              int32_t a = 0;
              unsigned long long a2 = 0;
              decode32<G>(bw + 1, bw[0], w, [&](int, int32_t x, int32_t neg) {
                const int32_t p = x - neg;
                a += p;
                if (OP == OP_VAR) a2 += (unsigned long long)((long long)p * p);
              });
              sp = a;
              sp2 = a2;
            } else {
              unpack_segment<false>(bw + 1, bw[0], w, cnt, [&](int, int32_t p) {
                sp += p;
                if (OP == OP_VAR) sp2 += (unsigned long long)((long long)p * p);
              });
            }
          }
          S1 += (long long)cnt * head + sp;
          if (OP == OP_VAR) {
            const long long cc = (long long)head - c0;
            S2 += (u128)((i128)cnt * cc * cc + (i128)2 * cc * sp + (i128)sp2);
          }
        } else if constexpr (OP == OP_MEAN_P) {
          // Section V-A, stage 2: S_b head + sum_k (S_b - k) p_k (p_0 = 0)
          long long c1 = (long long)cnt * head;
          if (w) {
            if (cnt == 32) {
              int32_t a = 0;
              decode32<G>(bw + 1, bw[0], w, [&](int k, int32_t x, int32_t) { a += (32 - k) * x; });
              c1 += (long long)a + weighted_sign_count(bw[0]);
            } else {
              long long a = 0;
              unpack_segment<false>(bw + 1, bw[0], w, cnt, [&](int k, int32_t p) { a += (long long)(cnt - k) * p; });
              c1 += a;
            }
          }
          S1 += c1;
        } else {
          // Section V-A, stage 3: q rebuilt from the head (eta accumulator)
          if (w == 0) {
            S1 += (long long)cnt * head;
            if (OP == OP_VAR) S2 += (u128)((unsigned long long)cnt * (unsigned long long)((long long)head * head));
          } else if (cnt == 32) {
            int32_t q = head, a1 = 0;
            using A2 = typename std::conditional<ACC == 0, uint32_t, unsigned long long>::type;
            A2 a2 = 0;
            decode32<G>(bw + 1, bw[0], w, [&](int, int32_t x, int32_t neg) {
              q = q + x - neg;
              a1 += q;
              if (OP == OP_VAR) {
                if constexpr (ACC == 0)
                  a2 += (uint32_t)(q * q);
                else
                  a2 += (unsigned long long)((long long)q * q);
              }
            });
            S1 += a1;
            if (OP == OP_VAR) S2 += (u128)a2;
          } else {
            int32_t q = head;
            long long a1 = 0;
            unsigned long long a2 = 0;
            unpack_segment<false>(bw + 1, bw[0], w, cnt, [&](int, int32_t p) {
              q += p;
              a1 += q;
              if (OP == OP_VAR) a2 += (unsigned long long)((long long)q * q);
            });
            S1 += a1;
            if (OP == OP_VAR) S2 += (u128)a2;
          }
        }
      }
    }
    cur = nxt;
    cur_r = nxt_r;
    nxt_r = nn_r;
    cur_issued = nxt_issued;
  }
  if constexpr (OP == OP_MEAN_G) S1 = (long long)G1;
  reduce_and_finish(S1, S2, err, parts, ticket, [&](long long a, u128 b2, int e) {
    if (shift)
      finalize_about(out, s.N, a, b2, c0, two_eps, e);
    else
      finalize_int(out, s.N, a, b2, OP == OP_VAR, two_eps, e);
  });
}

template <int G, int OP, int ACC, int PRED, int BPL>
int launch(const hc_header* h, const void* d_stream, hc_scalar* d_out, Partial* parts, unsigned* ticket,
           int max_parts, const long long* shift, cudaStream_t st) {
  const DevStream s = dev_stream(h, d_stream);
  const int bw = chunk_buf_words((int)h->wmax);
  const int bytes = smem_bytes(bw);
  auto kern = k_reduce32<G, OP, ACC, PRED, BPL>;
  BoxDims bd{};
  if (OP == OP_MEAN_G) {
    // the prediction shape: the field's for HSZp-nd, (1, 1, N) for HSZp
    const bool flat = h->pred == HC_PRED_GLOBAL_DELTA;
    bd.n0 = flat ? 1 : h->dims[0];
    bd.n1 = flat ? 1 : h->dims[1];
    bd.n2 = flat ? h->N : h->dims[2];
    bd.ragged = bd.n2 % 32 != 0;  // blocks across row ends (rows of >= 32 codes)
  } else if (PRED == HC_PRED_MEAN_ND) {
    bd.n0 = h->dims[0];
    bd.n1 = h->dims[1];
    bd.n2 = h->dims[2];
    bd.b0 = (int)h->block[0];
    bd.b1 = (int)h->block[1];
    bd.b2 = (int)h->block[2];
    bd.g1 = ceil_div(bd.n1, bd.b1);
    bd.g2 = ceil_div(bd.n2, bd.b2);
    bd.ragged = bd.n0 % bd.b0 || bd.n1 % bd.b1 || bd.n2 % bd.b2;
  }
  int rc = ensure_smem(reinterpret_cast<const void*>(kern), bytes);
  if (rc) return rc;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarps * 32, bytes);
  per_sm = std::max(per_sm, 1);
  int64_t grid = std::min<int64_t>((int64_t)device_sms() * per_sm, ceil_div(h->nchunks, kWarps));
  grid = std::max<int64_t>(1, std::min<int64_t>(grid, std::min<int64_t>(kMaxGrid, max_parts)));
  kern<<<(unsigned)grid, kWarps * 32, bytes, st>>>(s, bw, parts, ticket, d_out, 2.0 * h->eps, shift, bd);
  return check_launch_cfg("reduce (block size 32)", reinterpret_cast<const void*>(kern), grid, bytes);
}

template <int OP, int ACC, int PRED, int BPL = 4>
int launch_g(const hc_header* h, const void* d_stream, hc_scalar* d_out, Partial* parts, unsigned* ticket,
             int max_parts, const long long* shift, cudaStream_t st) {
  if (h->wmax <= 8)
    return launch<4, OP, ACC, PRED, BPL>(h, d_stream, d_out, parts, ticket, max_parts, shift, st);
  if (h->wmax <= 10)
    return launch<3, OP, ACC, PRED, BPL>(h, d_stream, d_out, parts, ticket, max_parts, shift, st);
  return launch<2, OP, ACC, PRED, BPL>(h, d_stream, d_out, parts, ticket, max_parts, shift, st);
}

template <int BPL>
int box_dispatch(const hc_header* h, const void* d_stream, int what, hc_scalar* d_out, Partial* parts,
                 unsigned* ticket, int max_parts, const long long* shift, cudaStream_t st) {
  if (what == RED_MEAN)
    return launch_g<OP_MEAN_Q, 1, HC_PRED_MEAN_ND, BPL>(h, d_stream, d_out, parts, ticket, max_parts, nullptr, st);
  return launch_g<OP_VAR, 1, HC_PRED_MEAN_ND, BPL>(h, d_stream, d_out, parts, ticket, max_parts, shift, st);
}

}  // namespace

bool reduce32_box_applies(const hc_header* h) {
  return h->pred == HC_PRED_MEAN_ND && (h->S == 64 || h->S == 128) && h->wmax <= 16 && h->qmax > 0 &&
         h->qmax < (1u << 26);
}

int reduce32_box_impl(const hc_header* h, const void* d_stream, int what, hc_scalar* d_out, Partial* parts,
                      unsigned* ticket, int max_parts, const long long* shift, cudaStream_t st) {
  // stages 2 and 3 have the same sums (sum q = sum p + M_b S_b); with
  // `shift` the squares are taken about the integer mean (stage-2 std)
  if (h->S == 64) return box_dispatch<2>(h, d_stream, what, d_out, parts, ticket, max_parts, shift, st);
  return box_dispatch<1>(h, d_stream, what, d_out, parts, ticket, max_parts, shift, st);
}

bool reduce32_global_mean_applies(const hc_header* h) {
  // rows of at least 32 codes (or HSZp's single row): a block then crosses
  // at most one row end, which the two-part sums handle without leaving
  // the grouped unpacker
  const bool rows32 = h->pred == HC_PRED_GLOBAL_DELTA || h->dims[2] >= 32;
  return h->S == 32 && (h->pred == HC_PRED_LORENZO || h->pred == HC_PRED_GLOBAL_DELTA) && h->wmax <= 16 &&
         h->N < 0xffffff00ll && rows32;
}

int reduce32_global_mean_impl(const hc_header* h, const void* d_stream, hc_scalar* d_out, Partial* parts,
                              unsigned* ticket, int max_parts, cudaStream_t st) {
  return launch_g<OP_MEAN_G, 1, HC_PRED_LORENZO>(h, d_stream, d_out, parts, ticket, max_parts, nullptr, st);
}

bool reduce32_applies(const hc_header* h) {
  return h->S == 32 && (h->pred == HC_PRED_DELTA || h->pred == HC_PRED_MEAN) && h->wmax <= 16 && h->qmax > 0 &&
         h->qmax < (1u << 26);
}

int reduce32_impl(const hc_header* h, const void* d_stream, int level, int what, hc_scalar* d_out, Partial* parts,
                  unsigned* ticket, int max_parts, const long long* shift, cudaStream_t st) {
  const bool narrow = h->qmax < (1u << 12);
  if (h->pred == HC_PRED_MEAN) {
    // stages 2 and 3 have the same sums (sum q = sum p + M_b S_b); with
    // `shift` the squares are taken about the integer mean (stage-2 std)
    if (what == RED_MEAN) return launch_g<OP_MEAN_Q, 1, HC_PRED_MEAN>(h, d_stream, d_out, parts, ticket, max_parts, nullptr, st);
    return narrow ? launch_g<OP_VAR, 0, HC_PRED_MEAN>(h, d_stream, d_out, parts, ticket, max_parts, shift, st)
                  : launch_g<OP_VAR, 1, HC_PRED_MEAN>(h, d_stream, d_out, parts, ticket, max_parts, shift, st);
  }
  if (what == RED_MEAN) {
    if (level == HC_STAGE_P)
      return launch_g<OP_MEAN_P, 1, HC_PRED_DELTA>(h, d_stream, d_out, parts, ticket, max_parts, nullptr, st);
    return launch_g<OP_MEAN_Q, 1, HC_PRED_DELTA>(h, d_stream, d_out, parts, ticket, max_parts, nullptr, st);
  }
  // the variance at stage 2 rebuilds q with the eta accumulator: stage 3's arithmetic
  return narrow ? launch_g<OP_VAR, 0, HC_PRED_DELTA>(h, d_stream, d_out, parts, ticket, max_parts, nullptr, st)
                : launch_g<OP_VAR, 1, HC_PRED_DELTA>(h, d_stream, d_out, parts, ticket, max_parts, nullptr, st);
}

}  // namespace hc
