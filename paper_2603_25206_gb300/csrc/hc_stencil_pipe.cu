// hc_stencil_pipe.cu -- the fused stream -> stencil kernel for the common
// case: block size 32, rows of a multiple of 8 elements that fit a tile, and
// codes |q| < 2^15 (the header's max |q| says so).  Same results as the
// general kernel in hc_stencil.cu (Section V-B, "Operation with D_q").
//
// One CTA owns TY whole rows for a range of planes and marches along the
// slowest axis (the sliding window of Algorithm 3, one plane slab per step).
// Warp 0 is a loader; warps 1..7 decode and compute:
//   step k:  loader   wait for the copies issued in step k-1, scan the widths
//                     of slab k+2, cp.async its payload and the widths + heads
//                     of slab k+3 (so every copy has a whole step to land);
//            workers  decode slab k into ring slot k % 4 and compute every
//                     output plane whose three slabs are ready (normally the
//                     plane of slab k-2);
//            one __syncthreads.
// Buffers: 4 ring slots, 3 payload stages, 4 metadata buffers.  A work item
// is V = 8 (rows a multiple of 8) or V = 4 (rows a multiple of 4) consecutive
// outputs of one row.
// Decoded codes are stored as int16, a 32-code segment as 64 contiguous
// bytes: a decoding thread writes its segment with four 16-byte stores and a
// stencil thread reads V consecutive codes of a row with one 16- or 8-byte
// load (consecutive threads read consecutive bytes: no bank conflicts).
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "hc_internal.cuh"
#include "hc_launch.h"

namespace hc {

DevStream dev_stream(const hc_header* h, const void* d_stream);

namespace {

constexpr int kWorkers = kThreads - 32;
constexpr int kSlots = 4;
constexpr int kWorkerWarps = kWorkers / 32;
constexpr int kSegCost = 4;  // decoding one 32-code segment ~ this many output items


struct PGeo {
  int64_t n0, n1, n2;
  int ty, tz, nyt, nzt;
  int nblk_max;     // blocks of one slab
  int pre_max;      // widths bytes staged per slab (G - 1 + nblk_max, rounded to 16)
  int heads_max;    // heads staged per slab (nblk_max + 4, rounded to 4)
  int stage_words;  // payload words per stage buffer
  int slot_bytes;   // nblk_max * 64
  int axis;
  unsigned nq_magic;  // ceil(2^32 / nq) for the row/item split (unused when nq == 1)
  int nq;             // items per row: n2 / V
  float eps_f, te_f;
  double eps, te;
};

template <int OUT>
struct OT;
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
      const double x = (double)a, y = (double)b, z = (double)c;
      return sqrt(x * x + y * y + z * z) * g.eps;
    }
  }
  return 0;
}

// Shared-memory carve-up (byte offsets), computed identically on both sides.
struct PSmem {
  int ring, stage, meta, total;
  int meta_bytes;  // one meta buffer: widths | heads | offsets
};
__host__ __device__ inline PSmem psmem(const PGeo& g) {
  PSmem p;
  p.ring = 0;
  p.stage = p.ring + kSlots * g.slot_bytes;
  p.meta = p.stage + 3 * 4 * g.stage_words;
  p.meta_bytes = g.pre_max + 4 * g.heads_max + 4 * (g.nblk_max + 4) + (kWidthSpecialize ? 2 * (g.nblk_max + 32 * 32 + 8) : 0);
  p.meta_bytes = (p.meta_bytes + 15) & ~15;
  p.total = p.meta + 4 * p.meta_bytes;
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

}  // namespace

template <int OP, int OUT, int V>
__global__ void __launch_bounds__(kThreads) k_stencil_pipe(DevStream s, PGeo g, typename OT<OUT>::T* __restrict__ out,
                                                            int* err) {
  using T = typename OT<OUT>::T;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int s_bad;
  const PSmem L = psmem(g);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const int yt = (int)(blockIdx.x % g.nyt), zt = (int)(blockIdx.x / g.nyt);
  const int64_t y0 = (int64_t)yt * g.ty, y1 = min(y0 + g.ty, g.n1);
  const int64_t z0 = (int64_t)zt * g.tz, z1 = min(z0 + g.tz, g.n0);
  const int64_t ylo = max(y0 - 1, (int64_t)0), yhi = min(y1 + 1, g.n1);
  const int64_t zs = max(z0 - 1, (int64_t)0), ze = min(z1 + 1, g.n0);  // slabs [zs, ze)
  const int nslab = (int)(ze - zs);
  if (tid == 0) s_bad = 0;

  auto meta_w = [&](int j) { return sm + L.meta + (j & 3) * L.meta_bytes; };
  auto meta_h = [&](int j) { return reinterpret_cast<int32_t*>(sm + L.meta + (j & 3) * L.meta_bytes + g.pre_max); };
  auto meta_o = [&](int j) {
    return reinterpret_cast<uint32_t*>(sm + L.meta + (j & 3) * L.meta_bytes + g.pre_max + 4 * g.heads_max);
  };
  auto meta_ord = [&](int j) {
    return reinterpret_cast<uint16_t*>(sm + L.meta + (j & 3) * L.meta_bytes + g.pre_max + 4 * g.heads_max +
                                       4 * (g.nblk_max + 4));
  };
  auto stage = [&](int j) { return reinterpret_cast<uint32_t*>(sm + L.stage + (j % 3) * 4 * g.stage_words); };
  __shared__ int s_whist[64];
  __shared__ int s_npad[4];  // padded order length per metadata buffer
  auto slot = [&](int64_t z) { return sm + L.ring + (int)(z & 3) * g.slot_bytes; };

  // loader: copy widths [cs, b0 + nblk) and heads [b0, b0 + nblk) of slab j
  auto load_meta = [&](int j) {
    const SlabDesc d = slab_desc(s, g, zs + j, ylo, yhi);
    const int nw = (d.npre + d.nblk + 15) & ~15;
    const uint8_t* wsrc = s.widths + d.cs;  // cs is a multiple of G = 128: 16-byte aligned
    uint8_t* wdst = meta_w(j);
    for (int i = lane * 16; i < nw; i += 32 * 16) cp_async16(wdst + i, wsrc + i);
    const int64_t h0 = d.b0 & ~(int64_t)3;
    const int nh = (int)((d.b0 + d.nblk - h0 + 3) & ~3);
    int32_t* hdst = meta_h(j);
    for (int i = lane * 4; i < nh; i += 32 * 4) cp_async16(hdst + i, s.heads + h0 + i);
  };
  // loader: offsets of slab j from its widths, then cp.async of its payload
  auto scan_and_load_payload = [&](int j) {
    const SlabDesc d = slab_desc(s, g, zs + j, ylo, yhi);
    const uint8_t* w = meta_w(j);
    uint32_t* off = meta_o(j);
    uint32_t carry = 0;
    const int n = d.npre + d.nblk;
    int bad = 0;
    for (int base = 0; base < n; base += 32) {
      const int i = base + lane;
      uint32_t wi = i < n ? w[i] : 0u;
      if (wi > (uint32_t)s.wmax) {
        bad = 1;
        wi = 0;
      }
      const uint32_t words = wi ? 1u + wi : 0u;  // S = 32: one sign word + w magnitude words
      uint32_t x = words;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (i >= d.npre && i < n) off[i - d.npre] = carry + x - words;  // exclusive, relative to chunk start
      carry += __shfl_sync(0xffffffffu, x, 31);
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
    if (bad && lane == 0) {
      s_bad = 1;
      set_error(err, HC_ERR_CORRUPT);
    }
    // counting sort of the slab's blocks by width: workers taking consecutive
    // entries run one width-specialised unpacker per warp
    uint16_t* ord = meta_ord(j);
    if (!kWidthSpecialize) return;
    s_whist[lane] = 0;
    __syncwarp();
    for (int i = lane; i < d.nblk; i += 32) atomicAdd(&s_whist[min((int)w[d.npre + i], 31)], 1);
    __syncwarp();
    {
      const int c = (s_whist[lane] + 31) & ~31;  // runs padded to whole warps
      int x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      s_whist[32 + lane] = x - c;
      const int padded = __shfl_sync(0xffffffffu, x, 31);
      if (lane == 0) s_npad[j & 3] = padded;
      for (int i = lane; i < padded; i += 32) ord[i] = 0xFFFFu;
    }
    __syncwarp();
    for (int i = lane; i < d.nblk; i += 32) ord[atomicAdd(&s_whist[32 + min((int)w[d.npre + i], 31)], 1)] = (uint16_t)i;
    __syncwarp();
  };

  // ---- prologue: metadata of slabs 0..2, payload of slabs 0 and 1
  if (warp == 0) {
    load_meta(0);
    if (nslab > 1) load_meta(1);
    cp_async_wait_all();
    __syncwarp();
    scan_and_load_payload(0);
    if (nslab > 1) scan_and_load_payload(1);
    if (nslab > 2) load_meta(2);
    cp_async_wait_all();
  }
  __syncthreads();

  int64_t znext = z0;  // next output plane
  for (int k = 0; k <= nslab; ++k) {
    if (warp == 0) {
      // copies issued in the previous step (payload k+1, metadata k+2) land here
      cp_async_wait_all();
      __syncwarp();
      if (k + 2 < nslab) scan_and_load_payload(k + 2);
      if (k + 3 < nslab) load_meta(k + 3);
    } else {
      // Split the 7 worker warps between decoding slab k and computing the
      // planes that are ready, in proportion to the estimated work (a segment
      // costs about kSegCost items); a warp has one role, so no divergence.
      const int ww = warp - 1;
      const int64_t ready = zs + k - 1;  // last slab decoded in an earlier step
      int64_t zc1 = znext;
      while (zc1 < z1 && min(zc1 + 1, g.n0 - 1) <= ready) ++zc1;
      const int nplanes = (int)(zc1 - znext);
      const int nseg_k = k < nslab ? slab_desc(s, g, zs + k, ylo, yhi).nblk : 0;
      const int items = (int)(y1 - y0) * g.nq;
      const int dec_cost = kSegCost * nseg_k, comp_cost = nplanes * items;
      int ndw = kWorkerWarps;
      if (comp_cost == 0)
        ndw = kWorkerWarps;
      else if (dec_cost == 0)
        ndw = 0;
      else
        ndw = min(kWorkerWarps - 1, max(1, (kWorkerWarps * dec_cost + (dec_cost + comp_cost) / 2) / (dec_cost + comp_cost)));
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
        const uint16_t* ord = meta_ord(k);
        const int nwork = kWidthSpecialize ? s_npad[k & 3] : d.nblk;
        for (int t = wt; t < nwork; t += wstride) {
          const int seg = kWidthSpecialize ? (int)ord[t] : t;
          if (seg == 0xFFFF) continue;
          const uint32_t wi = min((uint32_t)w[seg], (uint32_t)s.wmax);
          int32_t q = hd[seg];
          short v[32];
          if (wi == 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = (short)q;
          } else {
            const uint32_t* blk = stg + off[seg];
            unpack_full(blk + 1, blk[0], wi, [&](int i, int32_t p) {
              q += p;
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
        const int rc0 = (int)(row0 - (slab_desc(s, g, z, ylo, yhi).b0 << 5));
        const int rm0 = (int)((zm * g.n1 + y0) * g.n2 - (slab_desc(s, g, zm, ylo, yhi).b0 << 5));
        const int rp0 = (int)((zp * g.n1 + y0) * g.n2 - (slab_desc(s, g, zp, ylo, yhi).b0 << 5));
        T* const orow0 = out + row0;
        const int n2 = (int)g.n2;
        const int ez = (z == 0 || z == g.n0 - 1) ? 2 : 1;
        using Vec = typename std::conditional<V == 8, uint4, uint2>::type;
        for (int it = wt; it < items; it += wstride) {
          const int yr = g.nq == 1 ? it : (int)__umulhi((unsigned)it, g.nq_magic);
          const int x = (it - yr * g.nq) * V;
          const int roff = yr * n2 + x;
          const int rc = rc0 + roff;
          const int64_t y = y0 + yr;
          const int ey = (y == 0 || y == g.n1 - 1) ? 2 : 1;
          short c[V], a[V], b[V], zmv[V], zpv[V];
          *reinterpret_cast<Vec*>(c) = *reinterpret_cast<const Vec*>(pc + rc);
          if (OP != ST_DERIV || g.axis == 1) {
            *reinterpret_cast<Vec*>(a) = *reinterpret_cast<const Vec*>(pc + (y > 0 ? rc - n2 : rc));
            *reinterpret_cast<Vec*>(b) = *reinterpret_cast<const Vec*>(pc + (y + 1 < g.n1 ? rc + n2 : rc));
          }
          if (OP != ST_DERIV || g.axis == 0) {
            *reinterpret_cast<Vec*>(zmv) = *reinterpret_cast<const Vec*>(pm + rm0 + roff);
            *reinterpret_cast<Vec*>(zpv) = *reinterpret_cast<const Vec*>(pp + rp0 + roff);
          }
          int xl = c[0], xr = c[V - 1];
          if (OP != ST_DERIV || g.axis == 2) {
            if (x > 0) xl = pc[rc - 1];
            if (x + V < n2) xr = pc[rc + V];
          }
          // one-sided differences at the row ends are doubled
          const int ex0 = x == 0 ? 2 : 1, exn = x + V == n2 ? 2 : 1;
          T res[V];
#pragma unroll
          for (int i = 0; i < V; ++i) {
            const int cm = i == 0 ? xl : c[i - 1];
            const int cp = i == V - 1 ? xr : c[i + 1];
            if constexpr (OP == ST_LAPLACIAN) {
              const int l = (int)zmv[i] + zpv[i] + a[i] + b[i] + cm + cp - 6 * (int)c[i];
              res[i] = emit1<OP, OUT>(l, 0, 0, g);
            } else {
              int ex = 1;
              if (i == 0) ex = ex0;
              if (i == V - 1) ex = ex * exn;
              int d0 = 0, d1 = 0, d2 = 0;
              if (OP == ST_GRADMAG || g.axis == 0) d0 = ((int)zpv[i] - zmv[i]) * ez;
              if (OP == ST_GRADMAG || g.axis == 1) d1 = ((int)b[i] - a[i]) * ey;
              if (OP == ST_GRADMAG || g.axis == 2) d2 = (cp - cm) * ex;
              if constexpr (OP == ST_DERIV)
                res[i] = emit1<OP, OUT>(g.axis == 0 ? d0 : (g.axis == 1 ? d1 : d2), 0, 0, g);
              else
                res[i] = emit1<OP, OUT>(d0, d1, d2, g);
            }
          }
          T* o = orow0 + roff;
#pragma unroll
          for (int v = 0; v < (int)(V * sizeof(T) / 16); ++v)
            reinterpret_cast<uint4*>(o)[v] = reinterpret_cast<const uint4*>(res)[v];
        }
      }
    }
    __syncthreads();
  }
  if (warp == 0) cp_async_wait_all();
}

// ------------------------------------------------------------------ host
// The fast path applies when: S = 32, rows are a multiple of 4 codes, |q| <
// 2^15, the output is 16-byte aligned, and a tile of at least one row fits
// the shared-memory budget.  The tile height is the largest that keeps at
// least three CTAs per SM; the plane ranges are sized so that the grid fills
// whole waves of resident CTAs.
// Tile heights tried by the autotuner (and, without tuning, the first that
// fits the heuristic budget).
static const int kTileHeights[] = {16, 8, 4, 2, 1};

static bool plan_pipe_geometry(const hc_header* h, const int64_t* d3, PGeo& g, int* smem_out, int force_ty = 0) {
  if (h->S != 32 || h->qmax >= 32768u || d3[2] % 4 != 0) return false;
  g.n0 = d3[0];
  g.n1 = d3[1];
  g.n2 = d3[2];
  const int budget = force_ty ? 200 * 1024 : 74 * 1024;
  const int S = 32;
  int chosen = 0;
  for (int ty : kTileHeights) {
    if (force_ty && ty != force_ty) continue;
    if (ty > g.n1 && ty != 1) continue;
    const int64_t rows = std::min<int64_t>(ty + 2, g.n1);
    const int64_t span = rows * g.n2;
    if (span > (1 << 22)) continue;
    g.ty = ty;
    g.nblk_max = (int)((span + S - 1) / S + 1);
    g.pre_max = (h->G - 1 + g.nblk_max + 15 + 16) & ~15;
    g.heads_max = (g.nblk_max + 4 + 3 + 4) & ~3;
    g.stage_words = round4(g.nblk_max * (h->wmax ? 1 + (int)h->wmax : 0) + 16);
    g.slot_bytes = g.nblk_max * 64;
    const PSmem p = psmem(g);
    if (p.total <= budget || (ty == 1 && !force_ty)) {
      chosen = ty;
      *smem_out = p.total;
      break;
    }
  }
  if (!chosen || *smem_out > 200 * 1024) return false;
  g.nyt = (int)ceil_div(g.n1, g.ty);
  return true;
}

static void plan_pipe_grid(PGeo& g, int per_sm) {
  const int64_t capacity = (int64_t)device_sms() * std::max(per_sm, 1);
  // one wave when the rows allow it; never fewer than 4 planes per CTA
  int64_t nzt = std::max<int64_t>(1, capacity / g.nyt);
  nzt = std::min<int64_t>(nzt, std::max<int64_t>(1, g.n0 / 4));
  g.tz = (int)ceil_div(g.n0, nzt);
  g.nzt = (int)ceil_div(g.n0, g.tz);
}

template <int OP, int OUT, int V>
static int launch_pipe_o(const hc_header* h, const void* d_stream, PGeo g, int smem, void* d_out, int* err,
                         cudaStream_t st) {
  auto kern = k_stencil_pipe<OP, OUT, V>;
  int rc = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (rc) return rc;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  g.nq = (int)(g.n2 / V);
  g.nq_magic = g.nq > 1 ? (unsigned)(((1ull << 32) + (unsigned)g.nq - 1) / (unsigned)g.nq) : 0u;
  plan_pipe_grid(g, per_sm);
  const int64_t grid = (int64_t)g.nyt * g.nzt;
  kern<<<(unsigned)grid, kThreads, smem, st>>>(dev_stream(h, d_stream), g,
                                                reinterpret_cast<typename OT<OUT>::T*>(d_out), err);
  return check_launch_cfg("stencil (pipelined)", reinterpret_cast<const void*>(kern), grid, smem);
}

template <int OP, int OUT>
static int launch_pipe_v(const hc_header* h, const void* d_stream, const PGeo& g, int smem, void* d_out, int* err,
                         cudaStream_t st) {
  if (g.n2 % 8 == 0) return launch_pipe_o<OP, OUT, 8>(h, d_stream, g, smem, d_out, err, st);
  return launch_pipe_o<OP, OUT, 4>(h, d_stream, g, smem, d_out, err, st);
}

// Returns HC_ERR_UNSUPPORTED (without recording an error) when the fast path
// does not apply.
// Tile heights picked by hc_autotune, per (shape, max width, op, output type).
namespace {
struct TuneKey {
  int64_t n0, n1, n2;
  int wmax, op, out;
  bool operator<(const TuneKey& o) const {
    return std::tie(n0, n1, n2, wmax, op, out) < std::tie(o.n0, o.n1, o.n2, o.wmax, o.op, o.out);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;
}  // namespace

static int tuned_ty(const hc_header* h, const int64_t* d3, int op, int out_dtype) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(TuneKey{d3[0], d3[1], d3[2], (int)h->wmax, op, out_dtype});
  return it == g_tuned.end() ? 0 : it->second;
}

static int stencil_pipe_launch(const hc_header* h, const void* d_stream, const int64_t* d3, int op, int axis3,
                               void* d_out, int out_dtype, void* d_ws, cudaStream_t st, int force_ty);

int stencil_pipe_impl(const hc_header* h, const void* d_stream, const int64_t* d3, int op, int axis3, void* d_out,
                      int out_dtype, void* d_ws, cudaStream_t st) {
  return stencil_pipe_launch(h, d_stream, d3, op, axis3, d_out, out_dtype, d_ws, st, tuned_ty(h, d3, op, out_dtype));
}

// Time every tile height that fits on this field and remember the fastest.
// Returns the chosen height (0 when the pipelined kernel does not apply).
int stencil_pipe_autotune(const hc_header* h, const void* d_stream, const int64_t* d3, int op, void* d_out,
                          int out_dtype, void* d_ws, cudaStream_t st, int* chosen) {
  *chosen = 0;
  float best = 0.f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(HC_ERR_CUDA, "autotune: cudaEventCreate failed");
  for (int ty : kTileHeights) {
    PGeo g{};
    int smem = 0;
    if (!plan_pipe_geometry(h, d3, g, &smem, ty)) continue;
    float times[3];
    int rc = HC_OK;
    for (int r = -1; r < 3 && rc == HC_OK; ++r) {
      cudaEventRecord(e0, st);
      rc = stencil_pipe_launch(h, d_stream, d3, op, 0, d_out, out_dtype, d_ws, st, ty);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = HC_ERR_CUDA;
      if (r >= 0) cudaEventElapsedTime(&times[r], e0, e1);
    }
    if (rc != HC_OK) continue;
    std::sort(times, times + 3);
    if (*chosen == 0 || times[1] < best) {
      best = times[1];
      *chosen = ty;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  if (*chosen) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[TuneKey{d3[0], d3[1], d3[2], (int)h->wmax, op, out_dtype}] = *chosen;
  }
  return HC_OK;
}

static int stencil_pipe_launch(const hc_header* h, const void* d_stream, const int64_t* d3, int op, int axis3,
                               void* d_out, int out_dtype, void* d_ws, cudaStream_t st, int force_ty) {
  PGeo g{};
  int smem = 0;
  if (!aligned16(d_out) || !plan_pipe_geometry(h, d3, g, &smem, force_ty)) return HC_ERR_UNSUPPORTED;
  if (g.n1 * g.n2 >= ((int64_t)1 << 31)) return HC_ERR_UNSUPPORTED;
  g.axis = axis3;
  g.eps = h->eps;
  g.te = 2.0 * h->eps;
  g.eps_f = (float)h->eps;
  g.te_f = (float)(2.0 * h->eps);
  int* err = &reinterpret_cast<OpWs*>(d_ws)->status;
#define HC_PIPE_OUT(OPV)                                                                \
  switch (out_dtype) {                                                                  \
    case HC_F32:                                                                        \
      return launch_pipe_v<OPV, HC_F32>(h, d_stream, g, smem, d_out, err, st);          \
    case HC_F64:                                                                        \
      return launch_pipe_v<OPV, HC_F64>(h, d_stream, g, smem, d_out, err, st);          \
    case HC_I64:                                                                        \
      if (OPV == ST_GRADMAG) return HC_ERR_UNSUPPORTED;                                 \
      return launch_pipe_v<OPV, HC_I64>(h, d_stream, g, smem, d_out, err, st);          \
    default:                                                                            \
      return HC_ERR_UNSUPPORTED;                                                        \
  }
  if (op == ST_DERIV) {
    HC_PIPE_OUT(ST_DERIV)
  } else if (op == ST_GRADMAG) {
    HC_PIPE_OUT(ST_GRADMAG)
  } else {
    HC_PIPE_OUT(ST_LAPLACIAN)
  }
#undef HC_PIPE_OUT
}

}  // namespace hc
