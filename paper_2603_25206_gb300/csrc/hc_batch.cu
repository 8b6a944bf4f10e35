// hc_batch.cu -- the batched fused launch: many compressed fields, each with
// its own operations, decoded and operated on by one persistent kernel.
//
// Work is cut into units.  A field with a stencil operation (derivative,
// gradient magnitude, Laplacian; Section V-B) contributes one unit per output
// tile (TY rows x the row length x TZ planes, decoded with halos into a
// shared-memory ring): a tile of the pipelined stencil (block size 32, |q| <
// 2^15, 256 threads per CTA: a loader warp prefetches the next slabs while
// seven warps decode and compute) or else of the general one; a field with statistics only
// (Section V-A) contributes one unit per two chunks of blocks, decoded to
// D_q in shared memory and summed; a vector field (divergence or curl,
// Section V-C) one unit per output tile of the fused multi-component tile.  Statistics are taken at stage 3 (the codes
// q): s1 = sum q (64-bit) and s2 = sum q^2 (128-bit), exact.  When a field has
// both a stencil and statistics, the stencil units add up the codes they own,
// so one pass over the stream serves both.
//
// Scheduling: every CTA takes the next unit from a counter in the workspace
// (atomicAdd), so fields of uneven size balance across the GPU.  A unit adds
// its CTA's exact sums to its field's accumulator with 64-bit atomics (a carry
// moves into the high word of s2); the field's last unit to finish applies the
// final scaling and zeroes the accumulator.  The last CTA to leave resets the
// counter, so the workspace is ready for the next launch and the launch can
// be replayed from a CUDA graph.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include "hc_internal.cuh"
#include "hc_launch.h"
#include "hc_stencil_pipe.cuh"
#include "hc_stencil_tile.cuh"
#include "hc_vector_tile.cuh"

namespace hc {

DevStream dev_stream(const hc_header* h, const void* d_stream);

namespace {

constexpr uint32_t kPlanMagic = 0x4E4C5042u;  // "BPLN"

enum { STATS_NONE = 0, STATS_MEAN = 1, STATS_VAR = 2 };

// One field of the batch as the kernel sees it.
enum { KIND_TILE = 0, KIND_PIPE = 1, KIND_STATS = 2, KIND_VECTOR = 3 };

struct BItem {
  DevStream s;
  Geo g;               // general stencil geometry (KIND_TILE)
  PGeo pg;             // pipelined stencil geometry (KIND_PIPE)
  void* field;         // stencil output
  hc_scalar* scalar;   // statistics output
  int64_t units;       // work units of this field
  int64_t rblocks;     // blocks per statistics unit (fop < 0)
  double two_eps;
  int fop;             // StencilOp, or -1 for statistics only
  int out;             // hc_dtype of the stencil output
  int stats;           // STATS_*
  int rwords;          // statistics unit: words of the decoded D_q tile
  int kind;            // KIND_*
  int vec;             // KIND_PIPE: outputs per work item of the pipelined tile (8, 4 or 1)
  VArgs va;            // KIND_VECTOR: the components, signs and output type (tile geometry in g)
};

// Unit kinds a launch's kernel carries: every kind, or (256 threads) only
// pipelined stencil tiles, with the operation at run time or the float32
// Laplacian at compile time.
enum { KSET_ALL = 0, KSET_PIPE = 1, KSET_PIPE_LAP = 2 };

struct BPlan {
  uint32_t magic;
  int32_t n;
  int32_t threads;
  int32_t grid;
  int32_t smem;
  int32_t kset;  // KSET_*
  int64_t total_units;
  int64_t items_off;   // byte offset of BItem[n]
  int64_t prefix_off;  // byte offset of int64 unit prefix[n + 1]
  int64_t bytes;
};

struct BWs {
  unsigned long long next;  // next unit to hand out
  unsigned int exited;      // CTAs that found no more work
  int status;               // first error of any field (sticky until hc_batch_status)
  int pad[12];
};
struct BAcc {
  unsigned long long s1, lo, hi;
  unsigned int done;  // units finished
  int err;            // first error of this field
};
static_assert(sizeof(BWs) == 64, "workspace header");
static_assert(sizeof(BAcc) == 32, "accumulator");

__host__ __device__ inline int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

inline int64_t plan_bytes_for(int n) {
  const int64_t items = align_up(sizeof(BPlan), 16);
  const int64_t prefix = items + align_up((int64_t)sizeof(BItem) * n, 16);
  return prefix + 8 * (int64_t)(n + 1);
}

// ---------------------------------------------------------------- device
// Statistics unit: blocks [b0, b0 + rblocks) decoded to q in shared memory,
// then summed by the CTA.
template <bool SMALL>
__device__ __noinline__ void stats_unit(const BItem& it, int64_t lu, int* err, uint32_t* smem, uint32_t* s_warp, int* s_flag,
                           Moments& mo) {
  const DevStream& s = it.s;
  const int nblk = (int)it.rblocks;
  const int nsegmax = SMALL ? nblk : nblk * s.nseg;
  const TileSmem L = tile_smem(nblk, s.G - 1, s.S, s.wmax, it.rwords + (SMALL ? 0 : round4(nsegmax)));
  uint32_t* s_stage = smem;
  uint32_t* s_off = smem + L.off;
  int32_t* dst = reinterpret_cast<int32_t*>(smem + L.extra);
  int32_t* s_tot = dst + it.rwords;
  uint8_t* s_w = reinterpret_cast<uint8_t*>(smem + L.w);
  const int64_t b0 = lu * it.rblocks;
  const int64_t b1 = min(b0 + it.rblocks, s.nb);
  const int64_t e0 = b0 * s.S, e1 = min(b1 * (int64_t)s.S, s.N);
  decode_range<SMALL>(s, e0, e1, dst, s_w, s_off, s_stage, L.stage_words, s_tot, s_warp, s_flag, err);
  const int n = (int)(e1 - e0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) mo.add(dst[pidx(i)]);
  __syncthreads();
}

template <bool SMALL>
__device__ __noinline__ void stencil_unit(const BItem& it, int64_t lu, int* err, uint32_t* smem, uint32_t* s_warp,
                                          int* s_flag, long long (*s_base)[66], Moments& mo) {
  stencil_tile<ST_RUNTIME, ST_RUNTIME, SMALL, true>(it.s, it.g, lu, it.field, err, smem, s_warp, s_flag, s_base, mo);
}

template <int V, int PRED>
__device__ __noinline__ void pipe_unit(const BItem& it, int64_t lu, int* err, unsigned char* smem, Moments& mo) {
  pipe_tile<ST_RUNTIME, ST_RUNTIME, V, true, PRED>(it.s, it.pg, (int)(lu % it.pg.nyt), (int)(lu / it.pg.nyt),
                                                  it.field, err, smem, mo);
}

// A divergence / curl output tile (operation and output type in the item's
// VArgs).
template <bool SMALL>
__device__ __noinline__ void vector_unit(const BItem& it, int64_t lu, int* err, uint32_t* smem, uint32_t* s_warp,
                                         int* s_flag, long long (*s_base)[3][66]) {
  vector_tile<SMALL>(it.va, it.g, lu, it.field, err, smem, s_warp, s_flag, s_base);
}

// The float32 Laplacian (the batched workload's field operation) with its
// operation and type fixed at compile time; other operations take the
// run-time switch of pipe_unit.
template <int V, int PRED>
__device__ __noinline__ void pipe_unit_lap(const BItem& it, int64_t lu, int* err, unsigned char* smem, Moments& mo) {
  pipe_tile<ST_LAPLACIAN, HC_F32, V, true, PRED>(it.s, it.pg, (int)(lu % it.pg.nyt), (int)(lu / it.pg.nyt),
                                                 reinterpret_cast<float*>(it.field), err, smem, mo);
}

template <int V>
__device__ __forceinline__ void pipe_unit_p(const BItem& it, int64_t lu, int* err, unsigned char* smem, Moments& mo) {
  const bool lap = it.pg.op == ST_LAPLACIAN && it.pg.out == HC_F32;
  if (it.s.pred == HC_PRED_MEAN) {
    if (lap)
      pipe_unit_lap<V, HC_PRED_MEAN>(it, lu, err, smem, mo);
    else
      pipe_unit<V, HC_PRED_MEAN>(it, lu, err, smem, mo);
  } else {
    if (lap)
      pipe_unit_lap<V, HC_PRED_DELTA>(it, lu, err, smem, mo);
    else
      pipe_unit<V, HC_PRED_DELTA>(it, lu, err, smem, mo);
  }
}

// CTA sum of the unit's moments into the field accumulator; the field's last
// unit finishes the statistic and zeroes the accumulator.
template <int THREADS>
__device__ void publish(const BItem& it, const Moments& mo, BAcc* a, int* status) {
  constexpr int NW = THREADS / 32;
  __shared__ long long r_s1[NW];
  __shared__ u128 r_s2[NW];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (it.stats != STATS_NONE) {
    long long s1 = mo.s1;
    u128 s2 = ((u128)mo.hi << 64) | (u128)mo.lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_down_sync(0xffffffffu, s1, o);
      s2 += shfl_down_u128(s2, o);
    }
    if (lane == 0) {
      r_s1[wid] = s1;
      r_s2[wid] = s2;
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (it.stats != STATS_NONE) {
      long long s1 = 0;
      u128 s2 = 0;
      for (int i = 0; i < NW; ++i) {
        s1 += r_s1[i];
        s2 += r_s2[i];
      }
      const unsigned long long lo = (unsigned long long)s2;
      unsigned long long hi = (unsigned long long)(s2 >> 64);
      atomicAdd(&a->s1, (unsigned long long)s1);
      const unsigned long long old = atomicAdd(&a->lo, lo);
      if (old + lo < old) ++hi;
      if (hi) atomicAdd(&a->hi, hi);
    }
    __threadfence();
    const unsigned done = atomicAdd(&a->done, 1u);
    if ((int64_t)done + 1 == it.units) {
      __threadfence();
      const long long s1 = (long long)atomicExch(&a->s1, 0ull);
      const unsigned long long lo = atomicExch(&a->lo, 0ull), hi = atomicExch(&a->hi, 0ull);
      const int err = atomicExch(&a->err, 0);
      atomicExch(&a->done, 0u);
      if (err) set_error(status, err);
      if (it.stats != STATS_NONE)
        finalize_int(it.scalar, it.s.N, s1, ((u128)hi << 64) | (u128)lo, it.stats == STATS_VAR, it.two_eps, err);
    }
  }
}

// The persistent scheduling loop: every CTA takes the next unit from the
// counter, copies its item into shared memory, runs the unit and publishes
// its sums.  KSET_ALL dispatches over every unit kind; the pipelined-only
// sets inline the one tile they carry, so their kernels keep the tile's own
// register budget.
template <int THREADS, int KSET>
__device__ __forceinline__ void batch_loop(const uint8_t* __restrict__ plan, BWs* ws, BAcc* acc) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_warp[32];
  __shared__ int s_flag;
  __shared__ long long s_base[3][3][66];  // ring-slot offsets: [0] for scalar stencils, all for vector tiles
  __shared__ __align__(16) BItem s_it;
  __shared__ long long s_unit;
  __shared__ int s_item;
  const BPlan* P = reinterpret_cast<const BPlan*>(plan);
  const bool valid = P->magic == kPlanMagic && P->threads == THREADS && P->kset == KSET;
  if (!valid && threadIdx.x == 0) set_error(&ws->status, HC_ERR_INVALID_ARG);
  const BItem* items = reinterpret_cast<const BItem*>(plan + (valid ? P->items_off : 0));
  const int64_t* prefix = reinterpret_cast<const int64_t*>(plan + (valid ? P->prefix_off : 0));
  const int n = valid ? P->n : 0;
  const int64_t total = valid ? P->total_units : 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const int64_t u = (int64_t)atomicAdd(&ws->next, 1ull);
      int it = -1;
      int64_t lu = 0;
      if (u < total) {
        int lo = 0, hi = n;  // prefix[lo] <= u < prefix[hi]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (prefix[mid] <= u)
            lo = mid;
          else
            hi = mid;
        }
        it = lo;
        lu = u - prefix[lo];
      }
      s_item = it;
      s_unit = lu;
    }
    __syncthreads();
    const int it = s_item;
    if (it < 0) break;
    {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(items + it);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&s_it);
      for (int i = threadIdx.x; i < (int)(sizeof(BItem) / 4); i += THREADS) dst[i] = src[i];
    }
    __syncthreads();
    const int64_t lu = s_unit;
    int* err = &acc[it].err;
    Moments mo;
    unsigned char* sm = reinterpret_cast<unsigned char*>(smem);
    if constexpr (KSET == KSET_PIPE_LAP) {
      float* f = reinterpret_cast<float*>(s_it.field);
      const int yt = (int)(lu % s_it.pg.nyt), zt = (int)(lu / s_it.pg.nyt);
      const bool mean = s_it.s.pred == HC_PRED_MEAN;
#define HC_LAP(VV)                                                                                     \
  if (mean)                                                                                            \
    pipe_tile<ST_LAPLACIAN, HC_F32, VV, true, HC_PRED_MEAN>(s_it.s, s_it.pg, yt, zt, f, err, sm, mo);  \
  else                                                                                                 \
    pipe_tile<ST_LAPLACIAN, HC_F32, VV, true, HC_PRED_DELTA>(s_it.s, s_it.pg, yt, zt, f, err, sm, mo);
      if (s_it.vec == 8) {
        HC_LAP(8)
      } else if (s_it.vec == 4) {
        HC_LAP(4)
      } else {
        HC_LAP(1)
      }
#undef HC_LAP
    } else if constexpr (KSET == KSET_PIPE) {
      if (s_it.vec == 8)
        pipe_unit_p<8>(s_it, lu, err, sm, mo);
      else if (s_it.vec == 4)
        pipe_unit_p<4>(s_it, lu, err, sm, mo);
      else
        pipe_unit_p<1>(s_it, lu, err, sm, mo);
    } else {
      if (s_it.kind == KIND_PIPE) {
        if constexpr (THREADS == kThreads) {
          if (s_it.vec == 8)
            pipe_unit_p<8>(s_it, lu, err, sm, mo);
          else if (s_it.vec == 4)
            pipe_unit_p<4>(s_it, lu, err, sm, mo);
          else
            pipe_unit_p<1>(s_it, lu, err, sm, mo);
        }
      } else if (s_it.kind == KIND_VECTOR) {
        if (s_it.va.s[0].S <= 32)
          vector_unit<true>(s_it, lu, err, smem, s_warp, &s_flag, s_base);
        else
          vector_unit<false>(s_it, lu, err, smem, s_warp, &s_flag, s_base);
      } else if (s_it.fop >= 0) {
        if (s_it.s.S <= 32)
          stencil_unit<true>(s_it, lu, err, smem, s_warp, &s_flag, s_base[0], mo);
        else
          stencil_unit<false>(s_it, lu, err, smem, s_warp, &s_flag, s_base[0], mo);
      } else {
        if (s_it.s.S <= 32)
          stats_unit<true>(s_it, lu, err, smem, s_warp, &s_flag, mo);
        else
          stats_unit<false>(s_it, lu, err, smem, s_warp, &s_flag, mo);
      }
    }
    publish<THREADS>(s_it, mo, acc + it, &ws->status);
    __syncthreads();
  }
  if (threadIdx.x == 0 && atomicAdd(&ws->exited, 1u) == gridDim.x - 1) {
    // every CTA has taken its last unit: ready the counter for the next launch
    ws->next = 0ull;
    ws->exited = 0u;
    __threadfence();
  }
}

// Resident CTAs per SM assumed for the register budget: the tiles' shared
// memory (tens of KB) allows about two 256-thread CTAs per SM, so more than
// that would only force spills.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS == 128 ? 4 : (THREADS == 256 ? 2 : 1)) k_batch(const uint8_t* __restrict__ plan, BWs* ws, BAcc* acc) {
  batch_loop<THREADS, KSET_ALL>(plan, ws, acc);
}

// Batches of pipelined tiles only: three 256-thread CTAs per SM (the tile's
// shared memory allows three), the tile inlined.
template <int KSET>
__global__ void __launch_bounds__(kThreads, 3) k_batch_pipe(const uint8_t* __restrict__ plan, BWs* ws, BAcc* acc) {
  batch_loop<kThreads, KSET>(plan, ws, acc);
}

template <int THREADS>
const void* batch_kernel() {
  return reinterpret_cast<const void*>(k_batch<THREADS>);
}

const void* kernel_for(int threads, int kset = KSET_ALL) {
  if (kset == KSET_PIPE) return reinterpret_cast<const void*>(k_batch_pipe<KSET_PIPE>);
  if (kset == KSET_PIPE_LAP) return reinterpret_cast<const void*>(k_batch_pipe<KSET_PIPE_LAP>);
  switch (threads) {
    case 128:
      return batch_kernel<128>();
    case 256:
      return batch_kernel<256>();
    case 512:
      return batch_kernel<512>();
    default:
      return nullptr;
  }
}

int launch(const BPlan* hp, const void* d_plan, void* d_ws, cudaStream_t st) {
  BWs* ws = reinterpret_cast<BWs*>(d_ws);
  BAcc* acc = reinterpret_cast<BAcc*>(reinterpret_cast<char*>(d_ws) + sizeof(BWs));
  const uint8_t* p = reinterpret_cast<const uint8_t*>(d_plan);
  if (hp->kset == KSET_PIPE) {
    k_batch_pipe<KSET_PIPE><<<hp->grid, kThreads, hp->smem, st>>>(p, ws, acc);
    return check_launch_cfg("batch (pipelined tiles)", kernel_for(hp->threads, hp->kset), hp->grid, hp->smem);
  }
  if (hp->kset == KSET_PIPE_LAP) {
    k_batch_pipe<KSET_PIPE_LAP><<<hp->grid, kThreads, hp->smem, st>>>(p, ws, acc);
    return check_launch_cfg("batch (pipelined Laplacian tiles)", kernel_for(hp->threads, hp->kset), hp->grid,
                            hp->smem);
  }
  switch (hp->threads) {
    case 128:
      k_batch<128><<<hp->grid, 128, hp->smem, st>>>(p, ws, acc);
      break;
    case 256:
      k_batch<256><<<hp->grid, 256, hp->smem, st>>>(p, ws, acc);
      break;
    default:
      k_batch<512><<<hp->grid, 512, hp->smem, st>>>(p, ws, acc);
      break;
  }
  return check_launch_cfg("batch", kernel_for(hp->threads), hp->grid, hp->smem);
}

int check_plan(const void* h_plan, const void* d_plan, void* d_ws, size_t ws_bytes, const BPlan** out) {
  if (!h_plan || !d_plan || !d_ws) return fail(HC_ERR_INVALID_ARG, "null pointer");
  const BPlan* hp = reinterpret_cast<const BPlan*>(h_plan);
  if (hp->magic != kPlanMagic || !kernel_for(hp->threads) || hp->n < 1 || hp->grid < 1 || hp->kset < KSET_ALL ||
      hp->kset > KSET_PIPE_LAP || (hp->kset != KSET_ALL && hp->threads != kThreads))
    return fail(HC_ERR_INVALID_ARG, "not a batch plan");
  if (!aligned16(d_plan) || !aligned16(d_ws)) return fail(HC_ERR_INVALID_ARG, "device buffers must be 16-byte aligned");
  if (ws_bytes < sizeof(BWs) + sizeof(BAcc) * (size_t)hp->n)
    return fail(HC_ERR_NOMEM, "workspace smaller than hc_batch_workspace_bytes()");
  *out = hp;
  return HC_OK;
}

}  // namespace

// ------------------------------------------------------------------ host
namespace {

int64_t unit_elems_hint(const hc_batch_tune* tune) { return tune ? tune->unit_elems : 0; }

// A divergence / curl item: the components' checks of hc_op_divergence /
// hc_op_curl for the fused stage-3 tile, the tile geometry and its shared
// memory.  The planes per unit are set with the other items' units.
int plan_vector_item(const hc_batch_item& x, BItem& b, int* smem, int64_t) {
  const bool div = (x.ops & HC_BATCH_DIVERGENCE) != 0;
  if (x.ops != (uint32_t)(div ? HC_BATCH_DIVERGENCE : HC_BATCH_CURL))
    return fail(HC_ERR_INVALID_ARG, "batch: a vector item has its one operation and no other");
  if (!x.comps || x.ncomp < 1 || x.ncomp > 3) return fail(HC_ERR_INVALID_ARG, "batch: vector item components");
  if (!x.d_field || !aligned16(x.d_field)) return fail(HC_ERR_INVALID_ARG, "batch: vector output");
  if (x.field_dtype != HC_F32 && x.field_dtype != HC_F64 && x.field_dtype != HC_I64)
    return fail(HC_ERR_INVALID_ARG, "batch: field_dtype");
  const hc_header* hs[3] = {nullptr, nullptr, nullptr};
  for (int c = 0; c < x.ncomp; ++c) {
    const hc_stage& in = x.comps[c];
    if (in.kind != HC_STAGE_COMPRESSED || !in.hdr || !in.d_data)
      return fail(HC_ERR_INVALID_ARG, "batch: vector components are compressed streams");
    if (in.level != HC_STAGE_Q) return fail(HC_ERR_UNSUPPORTED, "batch: vector items run at stage Q");
    int rc = check_header(*in.hdr);
    if (rc) return rc;
    if (!aligned16(in.d_data)) return fail(HC_ERR_INVALID_ARG, "batch: stream pointer");
    hs[c] = in.hdr;
    if (in.hdr->pred != HC_PRED_DELTA && in.hdr->pred != HC_PRED_MEAN)
      return fail(HC_ERR_UNSUPPORTED, "batch: vector components must be block-head or block-mean streams");
    if (in.hdr->S != hs[0]->S || in.hdr->ndim != hs[0]->ndim)
      return fail(HC_ERR_INVALID_ARG, "batch: vector components of one block size and shape");
    for (int a = 0; a < 3; ++a)
      if (in.hdr->dims[a] != hs[0]->dims[a]) return fail(HC_ERR_INVALID_ARG, "batch: vector components of one shape");
  }
  const int ndim = hs[0]->ndim;
  if (div && x.ncomp != ndim) return fail(HC_ERR_INVALID_ARG, "batch: divergence takes ndim components");
  if (!div && (ndim != 2 || x.ncomp != 2)) return fail(HC_ERR_UNSUPPORTED, "batch: curl is defined for 2-D fields");
  VArgs& va = b.va;
  va = VArgs{};
  va.ncomp = x.ncomp;
  va.same_eps = 1;
  va.gmax = 1;
  va.wmax = 0;
  for (int c = 0; c < x.ncomp; ++c) {
    va.s[c] = dev_stream(hs[c], x.comps[c].d_data);
    va.eps[c] = hs[c]->eps;
    if (hs[c]->eps != hs[0]->eps) va.same_eps = 0;
    va.gmax = std::max(va.gmax, (int)hs[c]->G);
    va.wmax = std::max(va.wmax, (int)hs[c]->wmax);
  }
  if (x.field_dtype == HC_I64 && !va.same_eps)
    return fail(HC_ERR_UNSUPPORTED, "an integer numerator needs one eps for every component");
  va.out = x.field_dtype;
  vector_axes(hs[0], div ? VEC_DIV : VEC_CURL, x.ncomp, va);
  int64_t d3[3];
  int axis3 = 0;
  stencil_walk_dims(hs[0], d3, &axis3);
  b.g = stencil_base_geo(d3, hs[0]->eps, 0);
  int rc = plan_vector(hs, x.ncomp, d3, b.g, va.gmax, va.wmax, smem);
  if (rc) return rc;
  b.kind = KIND_VECTOR;
  b.fop = -1;
  b.out = x.field_dtype;
  b.field = x.d_field;
  b.stats = STATS_NONE;
  b.scalar = nullptr;
  b.s = va.s[0];
  return HC_OK;
}

}  // namespace

int64_t batch_plan_bytes(int n) { return n < 1 ? 0 : plan_bytes_for(n); }
int64_t batch_ws_bytes(int n) { return n < 1 ? 0 : (int64_t)(sizeof(BWs) + sizeof(BAcc) * (size_t)n); }

int batch_plan_impl(const hc_batch_item* items, int n, const hc_batch_tune* tune, void* h_plan, size_t cap,
                    size_t* used) {
  if (!items || n < 1 || !h_plan) return fail(HC_ERR_INVALID_ARG, "batch: null or empty");
  const int64_t bytes = plan_bytes_for(n);
  if ((int64_t)cap < bytes) return fail(HC_ERR_NOMEM, "plan buffer smaller than hc_batch_plan_bytes()");
  const int threads = (tune && tune->threads) ? tune->threads : 256;
  const void* kern = kernel_for(threads);
  if (!kern) return fail(HC_ERR_INVALID_ARG, "threads per CTA must be 128, 256 or 512");
  const int ty_force = tune ? tune->ty : 0;
  if (ty_force < 0) return fail(HC_ERR_INVALID_ARG, "ty");
  uint8_t* base = reinterpret_cast<uint8_t*>(h_plan);
  std::memset(base, 0, (size_t)bytes);
  BPlan* P = reinterpret_cast<BPlan*>(base);
  BItem* it = reinterpret_cast<BItem*>(base + align_up(sizeof(BPlan), 16));
  int64_t* prefix = reinterpret_cast<int64_t*>(base + align_up(sizeof(BPlan), 16) + align_up((int64_t)sizeof(BItem) * n, 16));
  int smem = 0;
  int64_t field_points = 0;
  const uint32_t field_ops = HC_BATCH_DERIVATIVE | HC_BATCH_GRADMAG | HC_BATCH_LAPLACIAN;
  const uint32_t vec_ops = HC_BATCH_DIVERGENCE | HC_BATCH_CURL;
  for (int i = 0; i < n; ++i) {
    const hc_batch_item& x = items[i];
    if (x.ops & vec_ops) {
      int sm = 0;
      int rc = plan_vector_item(x, it[i], &sm, unit_elems_hint(tune));
      if (rc) return rc;
      smem = std::max(smem, sm);
      field_points += it[i].va.s[0].N;
      continue;
    }
    if (x.ncomp != 0 || x.comps) return fail(HC_ERR_INVALID_ARG, "batch: components given without a vector operation");
    const hc_header& h = x.hdr;
    int rc = check_header(h);
    if (!rc && h.pred >= HC_PRED_LORENZO)
      return fail(HC_ERR_UNSUPPORTED, "batch: global-predictor streams need hc_workspace_bytes_for scratch");
    if (rc) return rc;
    if (!x.d_stream || !aligned16(x.d_stream)) return fail(HC_ERR_INVALID_ARG, "batch: stream pointer");
    if (x.ops == 0 || (x.ops & ~(field_ops | HC_BATCH_MEAN | HC_BATCH_VARIANCE)))
      return fail(HC_ERR_INVALID_ARG, "batch: ops");
    const uint32_t f = x.ops & field_ops;
    if (f & (f - 1)) return fail(HC_ERR_INVALID_ARG, "batch: at most one field operation per item");
    BItem& b = it[i];
    b.s = dev_stream(&h, x.d_stream);
    b.two_eps = 2.0 * h.eps;
    b.scalar = x.d_scalar;
    b.field = x.d_field;
    b.stats = (x.ops & HC_BATCH_VARIANCE) ? STATS_VAR : ((x.ops & HC_BATCH_MEAN) ? STATS_MEAN : STATS_NONE);
    if (b.stats != STATS_NONE && !x.d_scalar) return fail(HC_ERR_INVALID_ARG, "batch: statistics need d_scalar");
    if (f) {
      if (!x.d_field) return fail(HC_ERR_INVALID_ARG, "batch: field operation needs d_field");
      b.fop = (f == HC_BATCH_DERIVATIVE) ? ST_DERIV : (f == HC_BATCH_GRADMAG ? ST_GRADMAG : ST_LAPLACIAN);
      b.out = x.field_dtype;
      if (b.out != HC_F32 && b.out != HC_F64 && b.out != HC_I64) return fail(HC_ERR_INVALID_ARG, "batch: field_dtype");
      if (b.fop == ST_GRADMAG && b.out == HC_I64)
        return fail(HC_ERR_UNSUPPORTED, "the gradient magnitude has no integer form");
      int axis3 = 0;
      if (b.fop == ST_DERIV) {
        if (x.axis < 0 || x.axis >= h.ndim) return fail(HC_ERR_INVALID_ARG, "batch: axis");
        axis3 = x.axis + (3 - h.ndim);
      }
      int64_t d3[3];
      stencil_walk_dims(&h, d3, &axis3);
      int sm = 0;
      // the pipelined tile when it applies (it needs kThreads threads per CTA)
      b.kind = KIND_TILE;
      if (threads == kThreads && aligned16(x.d_field) && d3[1] * d3[2] < ((int64_t)1 << 31) &&
          plan_pipe_geometry(&h, d3, b.pg, &sm, 0, 74 * 1024, ty_force)) {
        // rows of other lengths: one output per item (measured faster inside
        // the batched kernel than the unaligned 8-wide items, whose code and
        // registers the persistent kernel would carry for every unit)
        b.vec = d3[2] % 8 == 0 ? 8 : (d3[2] % 4 == 0 ? 4 : 1);
        if (plan_pipe_items(b.pg, b.vec)) {
          b.kind = KIND_PIPE;
          b.pg.axis = axis3;
          b.pg.op = b.fop;
          b.pg.out = b.out;
          b.pg.eps = h.eps;
          b.pg.te = 2.0 * h.eps;
          b.pg.eps_f = (float)h.eps;
          b.pg.te_f = (float)(2.0 * h.eps);
        }
      }
      if (b.kind == KIND_TILE) {
        b.g = stencil_base_geo(d3, h.eps, axis3);
        b.g.op = b.fop;
        b.g.out = b.out;
        rc = stencil_plan(&h, b.g, &sm, ty_force, 1);
        if (rc) return rc;
      }
      smem = std::max(smem, sm);
      field_points += h.N;
    } else {
      b.fop = -1;
      b.kind = KIND_STATS;
      b.rblocks = (int64_t)kTileChunks * h.G;
      const bool small = h.S <= 32;
      const int nseg = (h.S + 31) / 32;
      const int nsegmax = small ? (int)b.rblocks : (int)b.rblocks * nseg;
      b.rwords = padded_elems_words((int)b.rblocks * h.S);
      const TileSmem L = tile_smem((int)b.rblocks, h.G - 1, h.S, (int)h.wmax, b.rwords + (small ? 0 : round4(nsegmax)));
      smem = std::max(smem, 4 * L.words);
      b.units = ceil_div(h.nb, b.rblocks);
    }
  }
  // the narrowest kernel that carries every item's unit kind
  int kset = KSET_ALL;
  if (threads == kThreads) {
    bool all_pipe = true, all_lap = true;
    for (int i = 0; i < n; ++i) {
      all_pipe &= it[i].kind == KIND_PIPE;
      all_lap &= it[i].kind == KIND_PIPE && it[i].pg.op == ST_LAPLACIAN && it[i].pg.out == HC_F32;
    }
    kset = all_lap ? KSET_PIPE_LAP : (all_pipe ? KSET_PIPE : KSET_ALL);
  }
  kern = kernel_for(threads, kset);
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // static shared memory of the kernel plus the dynamic part must fit
  if (smem + 8 * 1024 > optin) return fail(HC_ERR_UNSUPPORTED, "batch: a field's tile does not fit in shared memory");
  int rc = ensure_smem(kern, smem);
  if (rc) return rc;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  per_sm = std::max(per_sm, 1);
  if (tune && tune->ctas_per_sm > 0) per_sm = std::min(per_sm, tune->ctas_per_sm);
  const int64_t grid_cap = (int64_t)device_sms() * per_sm;
  // stencil units of about equal size, several per CTA
  int64_t unit_elems = tune ? tune->unit_elems : 0;
  if (unit_elems <= 0) unit_elems = std::max<int64_t>(16384, field_points / std::max<int64_t>(1, grid_cap * 6));
  int64_t total = 0;
  for (int i = 0; i < n; ++i) {
    BItem& b = it[i];
    if (b.kind == KIND_TILE) {
      int sm = 0;
      rc = stencil_plan(&items[i].hdr, b.g, &sm, ty_force, unit_elems);
      if (rc) return rc;
      // the planes per tile do not change the tile's shared memory
      if (sm > smem) return fail(HC_ERR_UNSUPPORTED, "batch: inconsistent tile plan");
      b.units = (int64_t)b.g.nxt * b.g.nyt * b.g.nzt;
    } else if (b.kind == KIND_VECTOR) {
      // planes per unit from the unit size (whole rows of ty rows per plane)
      const int64_t plane = (int64_t)b.g.ty * b.g.n2;
      b.g.tz = (int)std::min<int64_t>(b.g.n0, std::max<int64_t>(1, ceil_div(unit_elems, plane)));
      b.g.nzt = (int)ceil_div(b.g.n0, b.g.tz);
      b.units = (int64_t)b.g.nyt * b.g.nzt;
    } else if (b.kind == KIND_PIPE) {
      // at least four planes per unit: a pipelined tile primes three slabs
      const int64_t plane = (int64_t)b.pg.ty * b.pg.n2;
      const int64_t tz = std::max<int64_t>(4, ceil_div(unit_elems, plane));
      b.pg.tz = (int)std::min<int64_t>(b.pg.n0, tz);
      b.pg.nzt = (int)ceil_div(b.pg.n0, b.pg.tz);
      b.units = (int64_t)b.pg.nyt * b.pg.nzt;
    }
    if (b.units >= (int64_t)0xffffffffu) return fail(HC_ERR_UNSUPPORTED, "batch: field too large");
    prefix[i] = total;
    total += b.units;
  }
  prefix[n] = total;
  P->magic = kPlanMagic;
  P->n = n;
  P->threads = threads;
  P->kset = kset;
  P->grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid_cap, total));
  P->smem = smem;
  P->total_units = total;
  P->items_off = align_up(sizeof(BPlan), 16);
  P->prefix_off = P->items_off + align_up((int64_t)sizeof(BItem) * n, 16);
  P->bytes = bytes;
  if (used) *used = (size_t)bytes;
  return HC_OK;
}

int batch_run_impl(const void* h_plan, const void* d_plan, void* d_ws, size_t ws_bytes, cudaStream_t st) {
  const BPlan* hp = nullptr;
  int rc = check_plan(h_plan, d_plan, d_ws, ws_bytes, &hp);
  if (rc) return rc;
  rc = ensure_smem(kernel_for(hp->threads, hp->kset), hp->smem);
  if (rc) return rc;
  return launch(hp, d_plan, d_ws, st);
}

int batch_graph_impl(const void* h_plan, const void* d_plan, void* d_ws, size_t ws_bytes, void** out) {
  if (!out) return fail(HC_ERR_INVALID_ARG, "null pointer");
  *out = nullptr;
  const BPlan* hp = nullptr;
  int rc = check_plan(h_plan, d_plan, d_ws, ws_bytes, &hp);
  if (rc) return rc;
  rc = ensure_smem(kernel_for(hp->threads, hp->kset), hp->smem);
  if (rc) return rc;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
    return fail(HC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaStreamDestroy(cs);
    return fail(HC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  }
  rc = launch(hp, d_plan, d_ws, cs);
  const cudaError_t e1 = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (rc || e1 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    return rc ? rc : fail(HC_ERR_CUDA, cudaGetErrorString(e1));
  }
  const cudaError_t e2 = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) return fail(HC_ERR_CUDA, cudaGetErrorString(e2));
  *out = reinterpret_cast<void*>(ge);
  return HC_OK;
}

int batch_graph_launch_impl(void* graph, cudaStream_t st) {
  if (!graph) return fail(HC_ERR_INVALID_ARG, "null graph");
  if (cudaGraphLaunch(reinterpret_cast<cudaGraphExec_t>(graph), st) != cudaSuccess)
    return fail(HC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  return HC_OK;
}

int batch_graph_destroy_impl(void* graph) {
  if (!graph) return HC_OK;
  if (cudaGraphExecDestroy(reinterpret_cast<cudaGraphExec_t>(graph)) != cudaSuccess)
    return fail(HC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  return HC_OK;
}

int batch_status_impl(void* d_ws, cudaStream_t st) {
  if (!d_ws) return fail(HC_ERR_INVALID_ARG, "null workspace");
  BWs* ws = reinterpret_cast<BWs*>(d_ws);
  int v = 0, zero = 0;
  if (cudaMemcpyAsync(&v, &ws->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&ws->status, &zero, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(HC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  return v;
}

}  // namespace hc
