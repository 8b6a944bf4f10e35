// hc_reduce.cu -- homomorphic statistics (Section V-A): mean, variance and
// standard deviation.
//
// Fused forms read the compressed stream and never materialize a stage:
//   level 2 (Operation with D_p):  sum q = sum_b sum_i (S_b - i + 1) p_i,
//                                  the block-weighted sum, no prefix sum;
//   level 3 (Operation with D_q):  q rebuilt in registers (the eta
//                                  accumulator of Section V-A), s1 = sum q,
//                                  s2 = sum q^2.
// Array forms read a materialized D_p, D_q or D_f (the unfused and the plain
// "decompress, then operate" paths).
//
// Integer sums are exact: int64 for s1, 128-bit for s2.  Each CTA writes one
// partial; the last CTA to finish (ticket counter in the workspace, reset by
// that CTA) adds the partials and applies the final scaling of Eq. var_q:
//   mean = (s1 / N) * 2 eps,
//   var  = ((N s2 - s1^2) / (N (N - 1))) * (2 eps)^2   (exact 128-bit numerator).
#include <cstdint>
#include <type_traits>

#include "hc_finish.cuh"
#include "hc_internal.cuh"
#include "hc_launch.h"

namespace hc {

DevStream dev_stream(const hc_header* h, const void* d_stream);

// Chunks per tile of the fused statistics: four (two for the stage decoder);
// the larger tile spreads the per-tile width scan and copy issue over twice
// the codes (about 10% faster reductions, measured).
constexpr int kRedTileChunks = 4;

__device__ __forceinline__ int pidx(int r) { return r + (r >> 5); }

// words of the per-segment moment arrays: totals (int32), sums (int64) and,
// for the variance, sums of squares (128-bit)
__host__ __device__ inline int seg_moment_words(int nsegmax, bool var) {
  return round4(nsegmax) + round4(2 * nsegmax) + (var ? 4 * nsegmax : 0);
}
// padded value tile (33 words per 32 elements)
__host__ __device__ inline int padded_words(int elems) { return round4(((elems + 31) / 32) * 33 + 4); }

// ---------------------------------------------------------------- finishing
// ------------------------------------------------------- fused, from stream
// ACC: 0 narrow (max |q| < 2^12: 32-bit per-segment sums), 1 mid (< 2^26:
// 64-bit per-segment sums), 2 wide (128-bit per element).
// Block-mean (HSZx) streams (PRED = HC_PRED_MEAN, its own instantiations):
// q = M_b + p, so the
// segment's sums follow from sum p and sum p^2 (no prefix sum): s1 += cnt M_b
// + sum p, and, about a shift c0 (0, or the integer mean mu~ of the stage-2
// form), s2 += cnt c^2 + 2 c sum p + sum p^2 with c = M_b - c0.  `shift`
// points at c0 in device memory (NULL: no shift).
template <int LEVEL, int ACC, bool VAR, bool SMALL, int PRED>
__global__ void __launch_bounds__(kThreads) k_reduce_stream(DevStream s, int64_t ntiles, int stage_words,
                                                             Partial* parts, unsigned* ticket, hc_scalar* out,
                                                             double two_eps, const long long* shift) {
  extern __shared__ __align__(16) uint32_t smem[];
  const long long c0 = shift ? __ldcg(shift) : 0ll;
  __shared__ uint32_t s_warp[32];
  __shared__ int s_flag;
  __shared__ int s_err;
  const int tb = kRedTileChunks * s.G;
  const int nsegmax = SMALL ? tb : tb * s.nseg;
  constexpr bool seg_arrays = (!SMALL && LEVEL == 3);
  const int segw = seg_arrays ? seg_moment_words(nsegmax, VAR) : 0;
  const PipeTileSmem L = pipe_tile_smem(tb, stage_words, segw);
  uint32_t* s_off = smem + L.off;
  // per-segment local moments for S > 32 at level 3
  int32_t* s_T = reinterpret_cast<int32_t*>(smem + L.extra);
  long long* s_a1 = reinterpret_cast<long long*>(smem + L.extra + round4(nsegmax));
  u128* s_a2 = reinterpret_cast<u128*>(smem + L.extra + round4(nsegmax) + round4(2 * nsegmax));
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_err = 0;
  long long S1 = 0;
  u128 S2 = 0;
  unsigned long long S2n = 0;  // narrow: 64-bit per-thread sum of q^2

  // two tile buffers: tile t is decoded while tile t + gridDim.x is copied in
  int64_t t = blockIdx.x;
  int bi = 0;
  TileCopy cur{}, nxt{};
  bool cur_ok = false, have_nxt = false;
  if (t < ntiles) {
    cur = tile_bounds(s, t, tb);
    cur_ok = tile_issue(s, cur, stage_words, L.w(smem, 0), L.h(smem, 0), L.words(smem, 0));
  }
  if (t + gridDim.x < ntiles) {
    nxt = tile_bounds(s, t + gridDim.x, tb);
    have_nxt = true;
  }
  for (; t < ntiles; t += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();
    bool nxt_ok = false;
    if (have_nxt) nxt_ok = tile_issue(s, nxt, stage_words, L.w(smem, bi ^ 1), L.h(smem, bi ^ 1), L.words(smem, bi ^ 1));
    TileCopy nn{};
    const bool have_nn = t + 2 * (int64_t)gridDim.x < ntiles;
    if (have_nn) nn = tile_bounds(s, t + 2 * (int64_t)gridDim.x, tb);
    const int64_t b0 = cur.b0;
    const int nblk = cur.nblk;
    const int32_t* hb = L.h(smem, bi) + (int)(b0 & 3);
    TileView tv;
    const bool ok = tile_ready(s, cur, cur_ok, L.w(smem, bi), s_off, L.words(smem, bi), s_warp, &s_flag, &s_err, tv);
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
      if (cnt <= 0) {
        if (seg_arrays) {
          s_T[seg] = 0;
          s_a1[seg] = 0;
          if (VAR) s_a2[seg] = 0;
        }
        continue;
      }
      const uint32_t w = tv.w[bl];
      const int32_t head = hb[bl];
      const uint32_t* blk = tv.words + tv.off[bl];
      if constexpr (PRED == HC_PRED_MEAN) {
        // HSZx (Section V-A): stage 2 mean sum p + M_b S_b, stage 3 / the
        // stage-2 deviation sums from sum p and sum p^2
        using P2 = typename std::conditional<ACC == 2, u128, unsigned long long>::type;
        long long sp = 0;
        P2 sp2 = 0;
        if (w) unpack_any(blk + s.nseg + j * w, blk[j], w, cnt, [&](int i, int32_t p) {
            sp += p;
            if (VAR) sp2 += (P2)(unsigned long long)((long long)p * p);
          });
        S1 += (long long)cnt * head + sp;
        if (VAR) {
          const long long c = (long long)head - c0;
          S2 += (u128)((i128)cnt * c * c + (i128)2 * c * sp + (i128)sp2);
        }
        if constexpr (!SMALL && LEVEL == 3) {
          s_T[seg] = 0;
          s_a1[seg] = 0;
          if (VAR) s_a2[seg] = 0;
        }
        continue;
      }
      if constexpr (LEVEL == 2) {
        // Section V-A, stage 2: sum_k (S_b - k) p_k with the head as p_0
        using A = typename std::conditional<ACC == 0, int32_t, long long>::type;
        A sa = 0, sb = 0;
        if (w) unpack_any(blk + s.nseg + j * w, blk[j], w, cnt, [&](int i, int32_t p) {
            sa += p;
            sb += (A)i * p;
          });
        long long c = (long long)(Sb - 32 * j) * (long long)sa - (long long)sb;
        if (j == 0) c += (long long)Sb * head;
        S1 += c;
      } else if constexpr (SMALL) {
        // Section V-A, stage 3 / eta accumulator: q rebuilt from the head
        if constexpr (ACC == 0) {
          int32_t q = head, a1 = 0;
          uint32_t a2 = 0;
          if (w) {
            unpack_any(blk + s.nseg, blk[0], w, cnt, [&](int i, int32_t p) {
              q += p;
              a1 += q;
              if (VAR) a2 += (uint32_t)(q * q);
            });
          } else {
            a1 = cnt * head;
            if (VAR) a2 = (uint32_t)cnt * (uint32_t)(head * head);
          }
          S1 += a1;
          if (VAR) S2n += a2;
        } else if constexpr (ACC == 1) {
          int32_t q = head;
          long long a1 = 0;
          unsigned long long a2 = 0;
          if (w) {
            unpack_any(blk + s.nseg, blk[0], w, cnt, [&](int i, int32_t p) {
              q += p;
              a1 += q;
              if (VAR) a2 += (unsigned long long)((long long)q * q);
            });
          } else {
            a1 = (long long)cnt * head;
            if (VAR) a2 = (unsigned long long)cnt * (unsigned long long)((long long)head * head);
          }
          S1 += a1;
          if (VAR) S2 += a2;
        } else {
          int32_t q = head;
          long long a1 = 0;
          u128 a2 = 0;
          if (w) {
            unpack_any(blk + s.nseg, blk[0], w, cnt, [&](int i, int32_t p) {
              q += p;
              a1 += q;
              if (VAR) a2 += (u128)(unsigned long long)((long long)q * q);
            });
          } else {
            a1 = (long long)cnt * head;
            if (VAR) a2 = (u128)cnt * (u128)(unsigned long long)((long long)head * head);
          }
          S1 += a1;
          if (VAR) S2 += a2;
        }
      } else {
        // S > 32: local prefix P (relative to the segment's carry), its sums
        // and the segment total; the carry is added once all totals are known.
        int32_t P = 0;
        long long a1 = 0;
        u128 a2 = 0;
        if (w) {
          if constexpr (ACC == 0) {
            int32_t l1 = 0;
            uint32_t l2 = 0;
            unpack_any(blk + s.nseg + j * w, blk[j], w, cnt, [&](int i, int32_t p) {
              P += p;
              l1 += P;
              if (VAR) l2 += (uint32_t)(P * P);
            });
            a1 = l1;
            a2 = l2;
          } else if constexpr (ACC == 1) {
            unsigned long long l2 = 0;
            unpack_any(blk + s.nseg + j * w, blk[j], w, cnt, [&](int i, int32_t p) {
              P += p;
              a1 += P;
              if (VAR) l2 += (unsigned long long)((long long)P * P);
            });
            a2 = l2;
          } else {
            unpack_any(blk + s.nseg + j * w, blk[j], w, cnt, [&](int i, int32_t p) {
              P += p;
              a1 += P;
              if (VAR) a2 += (u128)(unsigned long long)((long long)P * P);
            });
          }
        }
        s_T[seg] = P;
        s_a1[seg] = a1;
        if (VAR) s_a2[seg] = a2;
      }
    }
    if constexpr (!SMALL && LEVEL == 3) {
      __syncthreads();
      for (int seg = tid; seg < nsegs && PRED != HC_PRED_MEAN; seg += nt) {
        const int bl = seg / s.nseg, j = seg - bl * s.nseg;
        const int64_t b = b0 + bl;
        const int Sb = (int)min((int64_t)s.S, s.N - b * s.S);
        const int cnt = min(32, Sb - 32 * j);
        if (cnt <= 0) continue;
        long long c = hb[bl];
        for (int jj = 0; jj < j; ++jj) c += s_T[bl * s.nseg + jj];
        const long long a1 = s_a1[seg];
        S1 += (long long)cnt * c + a1;
        if (VAR) {
          const i128 v = (i128)cnt * c * c + (i128)2 * c * a1 + (i128)s_a2[seg];
          S2 += (u128)v;
        }
      }
    }
  }
  cp_async_wait_all();
  if (ACC == 0 && VAR) S2 += S2n;
  __syncthreads();
  const int err = s_err;
  reduce_and_finish(S1, S2, err, parts, ticket, [&](long long a, u128 b, int e) {
    if (shift)
      finalize_about(out, s.N, a, b, c0, two_eps, e);
    else
      finalize_int(out, s.N, a, b, VAR, two_eps, e);
  });
}

// ------------------------------------------------------ stage 1 (HSZx)
// Eq. mean_m: T = sum_b M_b S_b from the block means alone; mean = (T / N)
// 2 eps.  With mu != NULL the integer mean mu~ = round(T / N) (nearest, ties
// toward zero) is also stored for the stage-2 standard deviation.
__global__ void __launch_bounds__(kThreads) k_mean_m(const int32_t* __restrict__ means, int64_t nb, int S, int64_t n,
                                                      Partial* parts, unsigned* ticket, hc_scalar* out,
                                                      double two_eps, long long* mu) {
  long long t = 0;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    const long long Sb = min((long long)S, (long long)(n - b * S));
    t += (long long)__ldg(means + b) * Sb;
  }
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

// ------------------------------------------------------- materialized D_q
template <bool VAR>
__global__ void __launch_bounds__(kThreads) k_reduce_q_array(const int32_t* __restrict__ q, int64_t n,
                                                              Partial* parts, unsigned* ticket, hc_scalar* out,
                                                              double two_eps) {
  long long S1 = 0;
  u128 S2 = 0;
  const int64_t nv = ((reinterpret_cast<uintptr_t>(q) & 15u) == 0) ? n / 4 : 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
    const int4 x = __ldg(reinterpret_cast<const int4*>(q) + v);
    S1 += (long long)x.x + x.y + x.z + x.w;
    if (VAR)
      S2 += (u128)((unsigned long long)((long long)x.x * x.x) + (unsigned long long)((long long)x.y * x.y)) +
            (u128)((unsigned long long)((long long)x.z * x.z) + (unsigned long long)((long long)x.w * x.w));
  }
  for (int64_t i = nv * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const long long x = __ldg(q + i);
    S1 += x;
    if (VAR) S2 += (u128)(unsigned long long)(x * x);
  }
  reduce_and_finish(S1, S2, 0, parts, ticket, [&](long long a, u128 b, int e) {
    finalize_int(out, n, a, b, VAR, two_eps, e);
  });
}

// ------------------------------------------------------- materialized D_p
// Tile of 2 chunks' worth of blocks staged into shared memory; one thread per
// 32-element segment applies the stage-2 weights (mean) or rebuilds q with
// the running accumulator (variance).
template <bool VAR, bool SMALL>
__global__ void __launch_bounds__(kThreads) k_reduce_p_array(const int32_t* __restrict__ dp, int64_t n, int S,
                                                              int tb, Partial* parts, unsigned* ticket,
                                                              hc_scalar* out, double two_eps) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int nseg = (S + 31) / 32;
  const int nsegmax = SMALL ? tb : tb * nseg;
  int32_t* s_v = reinterpret_cast<int32_t*>(smem);
  const int vwords = padded_words(tb * S);
  int32_t* s_T = s_v + vwords;
  long long* s_a1 = reinterpret_cast<long long*>(smem + vwords + round4(nsegmax));
  u128* s_a2 = reinterpret_cast<u128*>(smem + vwords + round4(nsegmax) + round4(2 * nsegmax));
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t nb = (n + S - 1) / S;
  const int64_t ntiles = (nb + tb - 1) / tb;
  long long S1 = 0;
  u128 S2 = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t b0 = t * tb;
    const int nblk = (int)min((int64_t)tb, nb - b0);
    const int64_t e0 = b0 * S;
    const int elems = (int)min((int64_t)nblk * S, n - e0);
    for (int i = tid; i < elems; i += nt) s_v[pidx(i)] = __ldg(dp + e0 + i);
    __syncthreads();
    const int nsegs = SMALL ? nblk : nblk * nseg;
    for (int seg = tid; seg < nsegs; seg += nt) {
      const int bl = SMALL ? seg : seg / nseg;
      const int j = SMALL ? 0 : seg - bl * nseg;
      const int Sb = (int)min((int64_t)S, n - (b0 + bl) * S);
      const int cnt = min(32, Sb - 32 * j);
      const int r0 = bl * S + 32 * j;
      if (!VAR) {
        long long c = 0;
        for (int i = 0; i < cnt; ++i) c += (long long)(Sb - 32 * j - i) * s_v[pidx(r0 + i)];
        S1 += c;
        continue;
      }
      long long P = 0, a1 = 0;
      u128 a2 = 0;
      for (int i = 0; i < cnt; ++i) {
        P += s_v[pidx(r0 + i)];
        a1 += P;
        a2 += (u128)(unsigned long long)(P * P);
      }
      if (SMALL) {
        S1 += a1;
        S2 += a2;
      } else {
        s_T[seg] = cnt > 0 ? (int32_t)P : 0;
        s_a1[seg] = cnt > 0 ? a1 : 0;
        s_a2[seg] = cnt > 0 ? a2 : 0;
      }
    }
    if (VAR && !SMALL) {
      __syncthreads();
      for (int seg = tid; seg < nsegs; seg += nt) {
        const int bl = seg / nseg, j = seg - bl * nseg;
        const int Sb = (int)min((int64_t)S, n - (b0 + bl) * S);
        const int cnt = min(32, Sb - 32 * j);
        if (cnt <= 0) continue;
        long long c = 0;
        for (int jj = 0; jj < j; ++jj) c += s_T[bl * nseg + jj];
        const long long a1 = s_a1[seg];
        S1 += (long long)cnt * c + a1;
        S2 += (u128)((i128)cnt * c * c + (i128)2 * c * a1 + (i128)s_a2[seg]);
      }
    }
    __syncthreads();
  }
  reduce_and_finish(S1, S2, 0, parts, ticket, [&](long long a, u128 b, int e) {
    finalize_int(out, n, a, b, VAR, two_eps, e);
  });
}

// ------------------------------------------------------- materialized D_f
// The plain path: statistics of a float array in its own precision.  All
// threads use one shift c (the array's first value): each keeps compensated
// sums of d = x - c and d^2, warps add them in the array's type, CTAs in
// double, and the last CTA adds the per-CTA partials in parallel:
//   mean = c + S1 / N,   variance = (S2 - S1^2 / N) / (N - 1).
// No integer information is used.
template <class T>
__device__ __forceinline__ void kahan_add(T& s, T& c, T v) {
  const T y = v - c;
  const T t = s + y;
  c = (t - s) - y;
  s = t;
}

template <class T, bool VAR>
__global__ void __launch_bounds__(kThreads) k_reduce_f_array(const T* __restrict__ f, int64_t n, Partial* parts,
                                                              unsigned* ticket, hc_scalar* out) {
  __shared__ double r1[32], r2[32];
  __shared__ int s_last;
  constexpr int V = 16 / sizeof(T);
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const int64_t nv = ((reinterpret_cast<uintptr_t>(f) & 15u) == 0) ? n / V : 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const T c = f[0];
  T s = 0, cs = 0, s2 = 0, c2 = 0;
  for (int64_t v = i0; v < nv; v += stride) {
    const Vec x = reinterpret_cast<const Vec*>(f)[v];
    const T* xe = reinterpret_cast<const T*>(&x);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const T d = xe[k] - c;
      kahan_add(s, cs, d);
      if (VAR) kahan_add(s2, c2, d * d);
    }
  }
  for (int64_t i = nv * V + i0; i < n; i += stride) {
    const T d = f[i] - c;
    kahan_add(s, cs, d);
    if (VAR) kahan_add(s2, c2, d * d);
  }
  T a = s - cs, b = s2 - c2;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    r1[wid] = (double)a;
    r2[wid] = (double)b;
  }
  __syncthreads();
  if (tid == 0) {
    double A = 0, B = 0;
    for (int k = 0; k < nw; ++k) {
      A += r1[k];
      B += r2[k];
    }
    Partial p;
    p.s1 = __double_as_longlong(A);
    p.s2_lo = (unsigned long long)__double_as_longlong(B);
    p.s2_hi = 0;
    p.err = 0;
    p.pad = 0;
    parts[blockIdx.x] = p;
    __threadfence();
    s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double A = 0, B = 0;
  for (int k = tid; k < (int)gridDim.x; k += blockDim.x) {
    A += __longlong_as_double(__ldcg(&parts[k].s1));
    B += __longlong_as_double((long long)__ldcg(&parts[k].s2_lo));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    A += __shfl_down_sync(0xffffffffu, A, o);
    B += __shfl_down_sync(0xffffffffu, B, o);
  }
  __syncthreads();
  if (lane == 0) {
    r1[wid] = A;
    r2[wid] = B;
  }
  __syncthreads();
  if (tid != 0) return;
  A = 0;
  B = 0;
  for (int k = 0; k < nw; ++k) {
    A += r1[k];
    B += r2[k];
  }
  const double nd = (double)n;
  out->n = n;
  out->s1 = 0;
  out->s2_lo = 0;
  out->s2_hi = 0;
  out->status = 0;
  out->exact = 0;
  out->mean = (double)c + A / nd;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  out->variance = (VAR && n >= 2) ? (B - A * A / nd) / (nd - 1.0) : nan;
  out->std = sqrt(out->variance);
  *ticket = 0;
}

// --------------------------------------------------------------------- host
static int acc_class(uint32_t qmax) {
  if (qmax == 0) return 2;  // unknown bound: widest accumulators
  if (qmax < (1u << 12)) return 0;
  if (qmax < (1u << 26)) return 1;
  return 2;
}

template <int LEVEL, int ACC, bool VAR, bool SMALL, int PRED>
static int launch_stream_p(const hc_header* h, const void* d_stream, hc_scalar* d_out, void* d_ws, cudaStream_t st,
                           const long long* shift) {
  const DevStream s = dev_stream(h, d_stream);
  const int tb = kRedTileChunks * h->G;
  const int nseg = (h->S + 31) / 32;
  const int nsegmax = SMALL ? tb : tb * nseg;
  const int stage = stage_words_for(tb, h->S, (int)h->wmax);
  const PipeTileSmem L =
      pipe_tile_smem(tb, stage, (!SMALL && LEVEL == 3) ? seg_moment_words(nsegmax, VAR) : 0);
  const int bytes = 4 * L.total;
  auto kern = k_reduce_stream<LEVEL, ACC, VAR, SMALL, PRED>;
  int rc = ensure_smem(reinterpret_cast<const void*>(kern), bytes);
  if (rc) return rc;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, bytes);
  per_sm = std::max(per_sm, 1);
  const int64_t ntiles = ceil_div(h->nchunks, kRedTileChunks);
  const int grid = (int)std::min<int64_t>(std::min<int64_t>(ntiles, (int64_t)device_sms() * per_sm), kMaxGrid);
  OpWs* ws = reinterpret_cast<OpWs*>(d_ws);
  kern<<<grid, kThreads, bytes, st>>>(s, ntiles, stage, ws_partials(d_ws), &ws->ticket, d_out, 2.0 * h->eps, shift);
  return check_launch_cfg("reduce (fused)", reinterpret_cast<const void*>(kern), grid, bytes);
}

// Block-mean streams: the same sums at stages 2 and 3 (sum q = sum p + M_b
// S_b), one accumulator class for codes below 2^26 and one above.
template <int LEVEL, int ACC, bool VAR, bool SMALL>
static int launch_stream(const hc_header* h, const void* d_stream, hc_scalar* d_out, void* d_ws, cudaStream_t st,
                         const long long* shift = nullptr) {
  if (h->pred == HC_PRED_MEAN)
    return launch_stream_p<3, (ACC == 2 ? 2 : 1), VAR, SMALL, HC_PRED_MEAN>(h, d_stream, d_out, d_ws, st, shift);
  return launch_stream_p<LEVEL, ACC, VAR, SMALL, HC_PRED_DELTA>(h, d_stream, d_out, d_ws, st, shift);
}

template <int LEVEL, bool VAR, bool SMALL>
static int launch_stream_acc(const hc_header* h, const void* d_stream, hc_scalar* d_out, void* d_ws, cudaStream_t st,
                             const long long* shift = nullptr) {
  switch (acc_class(h->qmax)) {
    case 0:
      return launch_stream<LEVEL, 0, VAR, SMALL>(h, d_stream, d_out, d_ws, st, shift);
    case 1:
      return launch_stream<LEVEL, (LEVEL == 2 ? 2 : 1), VAR, SMALL>(h, d_stream, d_out, d_ws, st, shift);
    default:
      return launch_stream<LEVEL, 2, VAR, SMALL>(h, d_stream, d_out, d_ws, st, shift);
  }
}

// Stage 1 of HSZx: the block means alone (Eq. mean_m).
static int launch_mean_m(const int32_t* means, int64_t nb, int S, int64_t n, double eps, hc_scalar* d_out,
                         void* d_ws, long long* mu, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(ceil_div(nb, kThreads),
                                                                                   (int64_t)device_sms() * 4),
                                                                 kMaxGrid));
  OpWs* ws = reinterpret_cast<OpWs*>(d_ws);
  k_mean_m<<<grid, kThreads, 0, st>>>(means, nb, S, n, ws_partials(d_ws), &ws->ticket, d_out, 2.0 * eps, mu);
  return check_launch("mean (stage 1)");
}

int mean_m_array_impl(const int32_t* means, int64_t nb, int S, int64_t n, double eps, hc_scalar* d_out, void* d_ws,
                      cudaStream_t st) {
  return launch_mean_m(means, nb, S, n, eps, d_out, d_ws, nullptr, st);
}

int reduce_stream_impl(const hc_header* h, const void* d_stream, int level, int what, hc_scalar* d_out, void* d_ws,
                       cudaStream_t st) {
  if (h->pred >= HC_PRED_LORENZO) return fail(HC_ERR_INVALID_ARG, "global-predictor stream on the block reducer");
  const bool small = h->S <= 32;
  const bool hszx = h->pred == HC_PRED_MEAN;
  const int32_t* means = reinterpret_cast<const int32_t*>(reinterpret_cast<const uint8_t*>(d_stream) + h->off_heads);
  if (level == HC_STAGE_M) {
    if (!hszx) return fail(HC_ERR_UNSUPPORTED, "block heads of a delta-coded stream support no statistic");
    if (what != RED_MEAN) return fail(HC_ERR_UNSUPPORTED, "stage 1 gives the mean only (Eq. mean_m)");
    return launch_mean_m(means, h->nb, h->S, h->N, h->eps, d_out, d_ws, nullptr, st);
  }
  if (reduce32_applies(h)) {
    OpWs* ws = reinterpret_cast<OpWs*>(d_ws);
    long long* mu = nullptr;
    if (hszx && level == HC_STAGE_P && what == RED_VAR) {
      // Section V-A: the deviations about the integer mean mu~ of stage 1
      mu = reinterpret_cast<long long*>(&ws->pad[0]);
      int rc = launch_mean_m(means, h->nb, h->S, h->N, h->eps, d_out, d_ws, mu, st);
      if (rc) return rc;
    }
    return reduce32_impl(h, d_stream, level, what, d_out, ws_partials(d_ws), &ws->ticket, kMaxGrid, mu, st);
  }
  if (hszx && level == HC_STAGE_P && what == RED_VAR) {
    // Section V-A: the deviations about the integer mean mu~ of stage 1
    long long* mu = reinterpret_cast<long long*>(&reinterpret_cast<OpWs*>(d_ws)->pad[0]);
    int rc = launch_mean_m(means, h->nb, h->S, h->N, h->eps, d_out, d_ws, mu, st);
    if (rc) return rc;
    return small ? launch_stream_acc<3, true, true>(h, d_stream, d_out, d_ws, st, mu)
                 : launch_stream_acc<3, true, false>(h, d_stream, d_out, d_ws, st, mu);
  }
  if (level == HC_STAGE_P && what == RED_MEAN)
    return small ? launch_stream_acc<2, false, true>(h, d_stream, d_out, d_ws, st)
                 : launch_stream_acc<2, false, false>(h, d_stream, d_out, d_ws, st);
  // the stage-2 standard deviation of Section V-A rebuilds q with the eta
  // accumulator: the same arithmetic as stage 3
  if (what == RED_MEAN)
    return small ? launch_stream_acc<3, false, true>(h, d_stream, d_out, d_ws, st)
                 : launch_stream_acc<3, false, false>(h, d_stream, d_out, d_ws, st);
  return small ? launch_stream_acc<3, true, true>(h, d_stream, d_out, d_ws, st)
               : launch_stream_acc<3, true, false>(h, d_stream, d_out, d_ws, st);
}

template <class K>
static int persistent_grid(K kern, int smem, int64_t work) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  per_sm = std::max(per_sm, 1);
  return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(work, (int64_t)device_sms() * per_sm), kMaxGrid));
}

int reduce_array_impl(const hc_stage* in, double eps, int what, hc_scalar* d_out, void* d_ws, cudaStream_t st) {
  OpWs* ws = reinterpret_cast<OpWs*>(d_ws);
  Partial* parts = ws_partials(d_ws);
  const int64_t n = in->n;
  const bool var = what == RED_VAR;
  if (in->kind == HC_STAGE_Q) {
    const int32_t* q = reinterpret_cast<const int32_t*>(in->d_data);
    if (var) {
      const int grid = persistent_grid(k_reduce_q_array<true>, 0, ceil_div(n, kThreads * 4));
      k_reduce_q_array<true><<<grid, kThreads, 0, st>>>(q, n, parts, &ws->ticket, d_out, 2.0 * eps);
    } else {
      const int grid = persistent_grid(k_reduce_q_array<false>, 0, ceil_div(n, kThreads * 4));
      k_reduce_q_array<false><<<grid, kThreads, 0, st>>>(q, n, parts, &ws->ticket, d_out, 2.0 * eps);
    }
    return check_launch("reduce (D_q)");
  }
  if (in->kind == HC_STAGE_P) {
    const int S = in->S;
    const int G = std::max(1, kChunkElems / S);
    const int tb = kTileChunks * G;
    const int nseg = (S + 31) / 32;
    const bool small = S <= 32;
    const int nsegmax = small ? tb : tb * nseg;
    const int bytes = 4 * (padded_words(tb * S) + ((var && !small) ? seg_moment_words(nsegmax, true) : 0));
    const int32_t* dp = reinterpret_cast<const int32_t*>(in->d_data);
    const int64_t ntiles = ceil_div(ceil_div(n, S), tb);
    const void* kern;
    int rc;
#define HC_LAUNCH_P(VAR, SMALL)                                                                          \
  {                                                                                                      \
    kern = reinterpret_cast<const void*>(k_reduce_p_array<VAR, SMALL>);                                  \
    rc = ensure_smem(kern, bytes);                                                                       \
    if (rc) return rc;                                                                                   \
    const int grid = persistent_grid(k_reduce_p_array<VAR, SMALL>, bytes, ntiles);                       \
    k_reduce_p_array<VAR, SMALL><<<grid, kThreads, bytes, st>>>(dp, n, S, tb, parts, &ws->ticket, d_out, \
                                                                 2.0 * eps);                             \
  }
    if (var && small) HC_LAUNCH_P(true, true)
    else if (var) HC_LAUNCH_P(true, false)
    else if (small) HC_LAUNCH_P(false, true)
    else HC_LAUNCH_P(false, false)
#undef HC_LAUNCH_P
    return check_launch("reduce (D_p)");
  }
  if (in->kind == HC_STAGE_F) {
    if (in->dtype == HC_F64) {
      const double* f = reinterpret_cast<const double*>(in->d_data);
      if (var) {
        const int grid = persistent_grid(k_reduce_f_array<double, true>, 0, ceil_div(n, kThreads));
        k_reduce_f_array<double, true><<<grid, kThreads, 0, st>>>(f, n, parts, &ws->ticket, d_out);
      } else {
        const int grid = persistent_grid(k_reduce_f_array<double, false>, 0, ceil_div(n, kThreads));
        k_reduce_f_array<double, false><<<grid, kThreads, 0, st>>>(f, n, parts, &ws->ticket, d_out);
      }
    } else {
      const float* f = reinterpret_cast<const float*>(in->d_data);
      if (var) {
        const int grid = persistent_grid(k_reduce_f_array<float, true>, 0, ceil_div(n, kThreads));
        k_reduce_f_array<float, true><<<grid, kThreads, 0, st>>>(f, n, parts, &ws->ticket, d_out);
      } else {
        const int grid = persistent_grid(k_reduce_f_array<float, false>, 0, ceil_div(n, kThreads));
        k_reduce_f_array<float, false><<<grid, kThreads, 0, st>>>(f, n, parts, &ws->ticket, d_out);
      }
    }
    return check_launch("reduce (D_f)");
  }
  return fail(HC_ERR_INVALID_ARG, "statistics take a stream or a P, Q or F array");
}

}  // namespace hc

namespace hc {

// ------------------------------------------- fused variance, scratch given
// The fused stage-3 variance kernel above, launched with its per-CTA
// partials and last-block ticket at caller-given device addresses instead of
// the workspace.  Fails with HC_ERR_NOMEM when the launch would need more than
// max_parts partial slots.
template <int ACC, bool SMALL, int PRED>
static int launch_var_scratch_p(const hc_header* h, const void* d_stream, hc_scalar* d_out, Partial* parts,
                                unsigned* ticket, int max_parts, cudaStream_t st) {
  const DevStream s = dev_stream(h, d_stream);
  const int tb = kRedTileChunks * h->G;
  const int nseg = (h->S + 31) / 32;
  const int nsegmax = SMALL ? tb : tb * nseg;
  const int stage = stage_words_for(tb, h->S, (int)h->wmax);
  const PipeTileSmem L =
      pipe_tile_smem(tb, stage, !SMALL ? seg_moment_words(nsegmax, true) : 0);
  const int bytes = 4 * L.total;
  auto kern = k_reduce_stream<3, ACC, true, SMALL, PRED>;
  int rc = ensure_smem(reinterpret_cast<const void*>(kern), bytes);
  if (rc) return rc;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, bytes);
  per_sm = std::max(per_sm, 1);
  const int64_t ntiles = ceil_div(h->nchunks, kRedTileChunks);
  const int64_t grid = std::min<int64_t>(std::min<int64_t>(ntiles, (int64_t)device_sms() * per_sm), kMaxGrid);
  if (grid > max_parts) return fail(HC_ERR_NOMEM, "the static scratch of hc_op_variance_noalloc has too few partial slots for this GPU");
  kern<<<(unsigned)grid, kThreads, bytes, st>>>(s, ntiles, stage, parts, ticket, d_out, 2.0 * h->eps, nullptr);
  return check_launch_cfg("variance (static scratch)", reinterpret_cast<const void*>(kern), grid, bytes);
}

template <int ACC, bool SMALL>
static int launch_var_scratch(const hc_header* h, const void* d_stream, hc_scalar* d_out, Partial* parts,
                              unsigned* ticket, int max_parts, cudaStream_t st) {
  if (h->pred == HC_PRED_MEAN)
    return launch_var_scratch_p<(ACC == 2 ? 2 : 1), SMALL, HC_PRED_MEAN>(h, d_stream, d_out, parts, ticket,
                                                                          max_parts, st);
  return launch_var_scratch_p<ACC, SMALL, HC_PRED_DELTA>(h, d_stream, d_out, parts, ticket, max_parts, st);
}

int variance_stream_scratch_impl(const hc_header* h, const void* d_stream, hc_scalar* d_out, Partial* parts,
                                 unsigned* ticket, int max_parts, cudaStream_t st) {
  if (h->pred >= HC_PRED_LORENZO) return fail(HC_ERR_INVALID_ARG, "global-predictor stream on the block reducer");
  if (reduce32_applies(h))
    return reduce32_impl(h, d_stream, HC_STAGE_Q, RED_VAR, d_out, parts, ticket, max_parts, nullptr, st);
  const bool small = h->S <= 32;
  switch (acc_class(h->qmax)) {
    case 0:
      return small ? launch_var_scratch<0, true>(h, d_stream, d_out, parts, ticket, max_parts, st)
                   : launch_var_scratch<0, false>(h, d_stream, d_out, parts, ticket, max_parts, st);
    case 1:
      return small ? launch_var_scratch<1, true>(h, d_stream, d_out, parts, ticket, max_parts, st)
                   : launch_var_scratch<1, false>(h, d_stream, d_out, parts, ticket, max_parts, st);
    default:
      return small ? launch_var_scratch<2, true>(h, d_stream, d_out, parts, ticket, max_parts, st)
                   : launch_var_scratch<2, false>(h, d_stream, d_out, parts, ticket, max_parts, st);
  }
}

}  // namespace hc
