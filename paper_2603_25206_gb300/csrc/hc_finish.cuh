// hc_finish.cuh -- the end of every exact statistic: a CTA-wide sum of the
// per-thread (s1, s2, error) triple, one partial per CTA in the workspace, and
// the last CTA to finish (ticket counter, reset by that CTA) adding the
// partials and handing the totals to a finishing function.
#pragma once

#include <cstdint>

#include "hc_internal.cuh"
#include "hc_launch.h"

namespace hc {

// CTA sum of (s1, s2, err), one partial per CTA, and the last CTA's finish.
template <class Fin>
__device__ inline void reduce_and_finish(long long s1, u128 s2, int err, Partial* parts, unsigned* ticket,
                                         Fin&& fin) {
  __shared__ long long r_s1[32];
  __shared__ u128 r_s2[32];
  __shared__ int r_err[32];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += shfl_down_u128(s2, o);
    err |= __shfl_down_sync(0xffffffffu, err, o);
  }
  if (lane == 0) {
    r_s1[wid] = s1;
    r_s2[wid] = s2;
    r_err[wid] = err;
  }
  __syncthreads();
  if (tid == 0) {
    long long a = 0;
    u128 b = 0;
    int e = 0;
    for (int i = 0; i < nw; ++i) {
      a += r_s1[i];
      b += r_s2[i];
      e |= r_err[i];
    }
    Partial p;
    p.s1 = a;
    p.s2_lo = (unsigned long long)b;
    p.s2_hi = (unsigned long long)(b >> 64);
    p.err = e;
    p.pad = 0;
    parts[blockIdx.x] = p;
    __threadfence();
    s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  long long a = 0;
  u128 b = 0;
  int e = 0;
  for (int i = tid; i < (int)gridDim.x; i += blockDim.x) {
    a += __ldcg(&parts[i].s1);
    b += ((u128)__ldcg(&parts[i].s2_hi) << 64) | (u128)__ldcg(&parts[i].s2_lo);
    e |= __ldcg(&parts[i].err);
  }
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += shfl_down_u128(b, o);
    e |= __shfl_down_sync(0xffffffffu, e, o);
  }
  if (lane == 0) {
    r_s1[wid] = a;
    r_s2[wid] = b;
    r_err[wid] = e;
  }
  __syncthreads();
  if (tid == 0) {
    long long ta = 0;
    u128 tb = 0;
    int te = 0;
    for (int i = 0; i < nw; ++i) {
      ta += r_s1[i];
      tb += r_s2[i];
      te |= r_err[i];
    }
    fin(ta, tb, te);
    *ticket = 0;
  }
}

}  // namespace hc
