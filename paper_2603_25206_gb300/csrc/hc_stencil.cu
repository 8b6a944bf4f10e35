// hc_stencil.cu -- numerical differentiation on the integer codes
// (Section V-B, "Operation with D_q"): derivative along one axis, gradient
// magnitude and Laplacian.
//
// Integer numerators (exact):
//   derivative  D = q[i+e] - q[i-e] inside, D = 2 (q[1] - q[0]) at an edge
//               (one-sided), 0 along an axis of length 1;   value eps * D
//   gradient    |grad| = eps * sqrt(D0^2 + D1^2 + D2^2)
//   Laplacian   L = sum_a (q[i-e_a] + q[i+e_a]) - 2 ndim q[i], edge values
//               replicated;                                   value 2 eps * L
// Fields are (n0, n1, n2) row-major with leading ones for ndim < 3, so the
// same 3-D code serves 1-D and 2-D fields (an axis of length 1 adds 0).
//
// Fused form (stream -> field, no materialized stage).  The 1-D block
// partition does not follow the rows (Section V-B), so every CTA decodes what
// it needs: a CTA owns TY rows of all x (or of an x-range when rows are very
// long) for a range of planes.  It marches along the slowest axis with a ring
// of three decoded plane slabs in shared memory (the paper's Algorithm 3
// sliding window, one plane per step instead of one block); each slab is the
// TY rows plus one halo row on each side, decoded from the stream through the
// chunk index.  The stencil reads only shared memory and writes each output
// once.
//
// Array form: the same stencils on a materialized D_q (exact) or D_f (the
// plain path, in the field's floating-point type).
#include <cstdint>
#include <cstdlib>
#include <type_traits>

#include "hc_internal.cuh"
#include "hc_launch.h"
#include "hc_stencil_tile.cuh"

namespace hc {

DevStream dev_stream(const hc_header* h, const void* d_stream);

template <int OP, int OUT, bool SMALL>
__global__ void __launch_bounds__(kThreads) k_stencil_stream(DevStream s, Geo g, typename OutType<OUT>::T* out,
                                                              int* err) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_warp[32];
  __shared__ int s_flag;
  __shared__ long long s_base[3][66];  // per slot, per range: base element
  Moments mo;
  stencil_tile<OP, OUT, SMALL, false>(s, g, blockIdx.x, out, err, smem, s_warp, &s_flag, s_base, mo);
}

// ---------------------------------------------------------------- arrays
template <class In>
struct ArrAcc {
  const In* a;
  __device__ __forceinline__ In operator()(int64_t i) const { return __ldg(a + i); }
};

// D_q input: exact integer numerators.  D_f input: the plain path computes the
// generic-flow formulas of Eq. derivatives / Eq. laplacian in the field's type.
// One CTA walks whole rows (x fastest) so no per-element division is needed.
template <int OP, int OUT, class In>
__global__ void __launch_bounds__(kThreads) k_stencil_array(const In* __restrict__ a, Geo g,
                                                             typename OutType<OUT>::T* __restrict__ out) {
  const int64_t rows = g.n0 * g.n1, pl = g.n1 * g.n2;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int64_t z = r / g.n1, y = r - z * g.n1;
    const int64_t rb = r * g.n2;
    const int64_t ym = y > 0 ? -g.n2 : 0, yp = y + 1 < g.n1 ? g.n2 : 0;
    const int64_t zm = z > 0 ? -pl : 0, zp = z + 1 < g.n0 ? pl : 0;
    const bool yedge = (y == 0 || y == g.n1 - 1), zedge = (z == 0 || z == g.n0 - 1);
    for (int64_t x = threadIdx.x; x < g.n2; x += blockDim.x) {
      const int64_t i = rb + x;
      const int64_t xm = x > 0 ? -1 : 0, xp = x + 1 < g.n2 ? 1 : 0;
      const bool xedge = (x == 0 || x == g.n2 - 1);
      if constexpr (std::is_integral<In>::value) {
        // integer codes
        if constexpr (OP == ST_LAPLACIAN) {
          const long long sum = (long long)__ldg(a + i + xm) + __ldg(a + i + xp) + __ldg(a + i + ym) +
                                __ldg(a + i + yp) + __ldg(a + i + zm) + __ldg(a + i + zp) - 6ll * __ldg(a + i);
          out[i] = emit<OP, OUT>(sum, 0, 0, g);
        } else {
          long long d0 = 0, d1 = 0, d2 = 0;
          if (OP == ST_GRADMAG || g.axis == 0) d0 = ((long long)__ldg(a + i + zp) - __ldg(a + i + zm)) * (zedge ? 2 : 1);
          if (OP == ST_GRADMAG || g.axis == 1) d1 = ((long long)__ldg(a + i + yp) - __ldg(a + i + ym)) * (yedge ? 2 : 1);
          if (OP == ST_GRADMAG || g.axis == 2) d2 = ((long long)__ldg(a + i + xp) - __ldg(a + i + xm)) * (xedge ? 2 : 1);
          if constexpr (OP == ST_DERIV)
            out[i] = emit<OP, OUT>(g.axis == 0 ? d0 : (g.axis == 1 ? d1 : d2), 0, 0, g);
          else
            out[i] = emit<OP, OUT>(d0, d1, d2, g);
        }
      } else {
        using R = typename OutType<OUT>::T;
        // floating point: (d+ - d-) / 2 inside, d1 - d0 at an edge
        auto der = [&](int64_t m, int64_t p, bool edge) -> In {
          const In v = __ldg(a + i + p) - __ldg(a + i + m);
          return edge ? v : v * In(0.5);
        };
        if constexpr (OP == ST_LAPLACIAN) {
          const In c = __ldg(a + i);
          const In v = ((__ldg(a + i + zm) + __ldg(a + i + zp)) - In(2) * c) +
                       ((__ldg(a + i + ym) + __ldg(a + i + yp)) - In(2) * c) +
                       ((__ldg(a + i + xm) + __ldg(a + i + xp)) - In(2) * c);
          out[i] = (R)v;
        } else {
          In d0 = 0, d1 = 0, d2 = 0;
          if (OP == ST_GRADMAG || g.axis == 0) d0 = g.n0 > 1 ? der(zm, zp, zedge) : In(0);
          if (OP == ST_GRADMAG || g.axis == 1) d1 = g.n1 > 1 ? der(ym, yp, yedge) : In(0);
          if (OP == ST_GRADMAG || g.axis == 2) d2 = g.n2 > 1 ? der(xm, xp, xedge) : In(0);
          if constexpr (OP == ST_DERIV)
            out[i] = (R)(g.axis == 0 ? d0 : (g.axis == 1 ? d1 : d2));
          else
            out[i] = (R)sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        }
      }
    }
  }
}

// Plain path, 4 outputs per thread (rows a multiple of 4, 16-byte aligned
// arrays): the same formulas as k_stencil_array with vector loads and stores.
template <int OP, int OUT, class In>
__global__ void __launch_bounds__(kThreads) k_stencil_array4(const In* __restrict__ a, Geo g,
                                                              typename OutType<OUT>::T* __restrict__ out) {
  using R = typename OutType<OUT>::T;
  using V4 = typename std::conditional<sizeof(In) == 4, int4, longlong4>::type;
  const int64_t rows = g.n0 * g.n1, pl = g.n1 * g.n2;
  const int nq = (int)(g.n2 / 4);
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int64_t z = r / g.n1, y = r - z * g.n1;
    const int64_t rb = r * g.n2;
    const int64_t ym = y > 0 ? -g.n2 : 0, yp = y + 1 < g.n1 ? g.n2 : 0;
    const int64_t zm = z > 0 ? -pl : 0, zp = z + 1 < g.n0 ? pl : 0;
    const bool yedge = (y == 0 || y == g.n1 - 1), zedge = (z == 0 || z == g.n0 - 1);
    for (int xq = threadIdx.x; xq < nq; xq += blockDim.x) {
      const int64_t i = rb + 4 * xq;
      In c[4], vym[4], vyp[4], vzm[4], vzp[4];
      *reinterpret_cast<V4*>(c) = *reinterpret_cast<const V4*>(a + i);
      *reinterpret_cast<V4*>(vym) = *reinterpret_cast<const V4*>(a + i + ym);
      *reinterpret_cast<V4*>(vyp) = *reinterpret_cast<const V4*>(a + i + yp);
      *reinterpret_cast<V4*>(vzm) = *reinterpret_cast<const V4*>(a + i + zm);
      *reinterpret_cast<V4*>(vzp) = *reinterpret_cast<const V4*>(a + i + zp);
      const In xl = xq > 0 ? __ldg(a + i - 1) : c[0];
      const In xr = 4 * xq + 4 < g.n2 ? __ldg(a + i + 4) : c[3];
      R res[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t x = 4 * xq + k;
        const In cm = k == 0 ? xl : c[k - 1];
        const In cp = k == 3 ? xr : c[k + 1];
        const bool xedge = (x == 0 || x == g.n2 - 1);
        if constexpr (OP == ST_LAPLACIAN) {
          const In v = ((vzm[k] + vzp[k]) - In(2) * c[k]) + ((vym[k] + vyp[k]) - In(2) * c[k]) +
                       ((cm + cp) - In(2) * c[k]);
          res[k] = (R)v;
        } else {
          auto der = [&](In m, In p, bool edge) -> In {
            const In v = p - m;
            return edge ? v : v * In(0.5);
          };
          In d0 = 0, d1 = 0, d2 = 0;
          if (OP == ST_GRADMAG || g.axis == 0) d0 = g.n0 > 1 ? der(vzm[k], vzp[k], zedge) : In(0);
          if (OP == ST_GRADMAG || g.axis == 1) d1 = g.n1 > 1 ? der(vym[k], vyp[k], yedge) : In(0);
          if (OP == ST_GRADMAG || g.axis == 2) d2 = g.n2 > 1 ? der(cm, cp, xedge) : In(0);
          if constexpr (OP == ST_DERIV)
            res[k] = (R)(g.axis == 0 ? d0 : (g.axis == 1 ? d1 : d2));
          else
            res[k] = (R)sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        }
      }
      R* o = out + i;
#pragma unroll
      for (int v = 0; v < (int)(4 * sizeof(R) / 16); ++v) reinterpret_cast<uint4*>(o)[v] = reinterpret_cast<const uint4*>(res)[v];
    }
  }
}

// ------------------------------------------------------------------ host
Geo stencil_base_geo(const int64_t* dims3, double eps, int axis3) {
  Geo g{};
  g.n0 = dims3[0];
  g.n1 = dims3[1];
  g.n2 = dims3[2];
  g.axis = axis3;
  g.eps = eps;
  g.te = 2.0 * eps;
  g.eps_f = (float)eps;
  g.te_f = (float)(2.0 * eps);
  return g;
}

static int stream_smem_bytes(const hc_header* h, const Geo& g) {
  return 4 * stencil_tile_words(h->S, h->G, (int)h->wmax, g);
}

// Pick rows per tile (whole rows when they fit), planes per tile and the
// resulting shared-memory footprint.  ty_force > 0 takes that tile height
// (capped by n1); unit_elems > 0 sizes the planes per tile so that a tile
// holds about that many output points (the batched launch), else the tiles
// are cut into about four per SM.
int stencil_plan(const hc_header* h, Geo& g, int* smem_out, int ty_force, int64_t unit_elems) {
  const int S = h->S;
  const int64_t budget = 110 * 1024;  // two CTAs per SM
  const int64_t hard = 220 * 1024;
  g.nslot = g.n0 > 1 ? 3 : 1;
  auto try_plan = [&](int ty, int64_t tx) -> int {
    g.ty = ty;
    g.tx = (int)tx;
    const bool whole = (tx == g.n2);
    const int64_t rows = std::min<int64_t>(ty + 2, g.n1);
    g.ranges = whole ? 1 : (int)rows;
    const int64_t span = whole ? rows * g.n2 : std::min<int64_t>(tx + 2, g.n2);
    g.nblk_max = (int)((span + S - 1) / S + 1);
    g.range_elems = g.nblk_max * S;
    g.slot_words = g.ranges * padded_elems_words(g.range_elems);
    return stream_smem_bytes(h, g);
  };
  int bytes = 0;
  bool ok = false;
  // whole rows: largest ty in {16, 8, 4, 2, 1} within the budget, capped by n1
  for (int ty : {16, 8, 4, 2, 1}) {
    if (ty > g.n1 && ty != 1) continue;
    if (ty_force > 0 && ty > ty_force) continue;
    bytes = try_plan(ty, g.n2);
    if (bytes <= budget && g.range_elems <= (1 << 24)) {
      ok = true;
      break;
    }
  }
  if (!ok) {
    // long rows: one row per tile and an x-range per CTA
    int64_t tx = 8192;
    while (tx > 64) {
      bytes = try_plan(1, std::min<int64_t>(tx, g.n2));
      if (bytes <= budget) break;
      tx /= 2;
    }
    if (bytes > hard) return fail(HC_ERR_UNSUPPORTED, "stencil tile does not fit in shared memory");
  }
  if (g.ty > 64) return fail(HC_ERR_UNSUPPORTED, "tile too tall");
  g.nxt = (int)ceil_div(g.n2, g.tx);
  g.nyt = (int)ceil_div(g.n1, g.ty);
  if (unit_elems > 0) {
    const int64_t plane = (int64_t)g.ty * g.tx;
    g.tz = (int)std::max<int64_t>(1, std::min<int64_t>(g.n0, ceil_div(unit_elems, plane)));
  } else {
    const int64_t target = (int64_t)device_sms() * 4;
    const int64_t per_plane = (int64_t)g.nxt * g.nyt;
    const int64_t nzt = std::max<int64_t>(1, std::min<int64_t>(g.n0, ceil_div(target, per_plane)));
    g.tz = (int)ceil_div(g.n0, nzt);
  }
  g.nzt = (int)ceil_div(g.n0, g.tz);
  *smem_out = bytes;
  return HC_OK;
}

template <int OP, int OUT, bool SMALL>
static int launch_stream_st(const hc_header* h, const void* d_stream, Geo g, void* d_out, int* err, cudaStream_t st) {
  int smem = 0;
  int rc = stencil_plan(h, g, &smem, 0, 0);
  if (rc) return rc;
  auto kern = k_stencil_stream<OP, OUT, SMALL>;
  rc = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (rc) return rc;
  const int64_t grid = (int64_t)g.nxt * g.nyt * g.nzt;
  if (grid > 0x7fffffff) return fail(HC_ERR_UNSUPPORTED, "field too large");
  kern<<<(unsigned)grid, kThreads, smem, st>>>(dev_stream(h, d_stream), g,
                                                reinterpret_cast<typename OutType<OUT>::T*>(d_out), err);
  return check_launch_cfg("stencil (fused)", reinterpret_cast<const void*>(kern), grid, smem);
}

template <int OP, int OUT>
static int launch_stream_s(const hc_header* h, const void* d_stream, const Geo& g, void* d_out, int* err,
                           cudaStream_t st) {
  if (h->S <= 32) return launch_stream_st<OP, OUT, true>(h, d_stream, g, d_out, err, st);
  return launch_stream_st<OP, OUT, false>(h, d_stream, g, d_out, err, st);
}

template <int OP>
static int launch_stream_o(const hc_header* h, const void* d_stream, const Geo& g, void* d_out, int out_dtype,
                           int* err, cudaStream_t st) {
  switch (out_dtype) {
    case HC_F32:
      return launch_stream_s<OP, HC_F32>(h, d_stream, g, d_out, err, st);
    case HC_F64:
      return launch_stream_s<OP, HC_F64>(h, d_stream, g, d_out, err, st);
    case HC_I64:
      if (OP == ST_GRADMAG) return fail(HC_ERR_UNSUPPORTED, "the gradient magnitude has no integer form");
      return launch_stream_s<OP, HC_I64>(h, d_stream, g, d_out, err, st);
    default:
      return fail(HC_ERR_INVALID_ARG, "out_dtype");
  }
}

int stencil_stream_impl(const hc_header* h, const void* d_stream, int op, int axis3, void* d_out, int out_dtype,
                        void* d_ws, cudaStream_t st) {
  if (h->pred >= HC_PRED_LORENZO) return fail(HC_ERR_INVALID_ARG, "global-predictor stream on the block stencil");
  int* err = &reinterpret_cast<OpWs*>(d_ws)->status;
  // a 2-D field marches along its rows: (1, n1, n2) is walked as (n1, 1, n2)
  int64_t d3[3];
  stencil_walk_dims(h, d3, &axis3);
  // the pipelined kernel covers block size 32 and |q| < 2^15 (rows of any
  // length); everything else takes the general kernel below
  static const bool force_general = std::getenv("HC_FORCE_GENERAL_STENCIL") != nullptr;
  if (!force_general) {
    const int rc = stencil_pipe_impl(h, d_stream, d3, op, axis3, d_out, out_dtype, d_ws, st);
    if (rc != HC_ERR_UNSUPPORTED) return rc;
  }
  const Geo g = stencil_base_geo(d3, h->eps, axis3);
  switch (op) {
    case ST_DERIV:
      return launch_stream_o<ST_DERIV>(h, d_stream, g, d_out, out_dtype, err, st);
    case ST_GRADMAG:
      return launch_stream_o<ST_GRADMAG>(h, d_stream, g, d_out, out_dtype, err, st);
    default:
      return launch_stream_o<ST_LAPLACIAN>(h, d_stream, g, d_out, out_dtype, err, st);
  }
}

template <int OP, int OUT, class In>
static int launch_array(const void* d_in, const Geo& g, void* d_out, cudaStream_t st) {
  const int64_t rows = g.n0 * g.n1;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(rows, (int64_t)device_sms() * 16));
  if constexpr (!std::is_integral<In>::value) {
    if (g.n2 % 4 == 0 && aligned16(d_in) && aligned16(d_out)) {
      k_stencil_array4<OP, OUT, In><<<grid, kThreads, 0, st>>>(reinterpret_cast<const In*>(d_in), g,
                                                               reinterpret_cast<typename OutType<OUT>::T*>(d_out));
      return check_launch("stencil (array, 4-wide)");
    }
  }
  k_stencil_array<OP, OUT, In><<<grid, kThreads, 0, st>>>(reinterpret_cast<const In*>(d_in), g,
                                                          reinterpret_cast<typename OutType<OUT>::T*>(d_out));
  return check_launch("stencil (array)");
}

template <int OP, class In>
static int launch_array_o(const void* d_in, const Geo& g, void* d_out, int out_dtype, bool integer, cudaStream_t st) {
  switch (out_dtype) {
    case HC_F32:
      return launch_array<OP, HC_F32, In>(d_in, g, d_out, st);
    case HC_F64:
      return launch_array<OP, HC_F64, In>(d_in, g, d_out, st);
    case HC_I64:
      if (!integer || OP == ST_GRADMAG) return fail(HC_ERR_UNSUPPORTED, "integer output needs integer input");
      return launch_array<OP, HC_I64, In>(d_in, g, d_out, st);
    default:
      return fail(HC_ERR_INVALID_ARG, "out_dtype");
  }
}

template <class In>
static int launch_array_op(const void* d_in, const Geo& g, int op, void* d_out, int out_dtype, bool integer,
                           cudaStream_t st) {
  switch (op) {
    case ST_DERIV:
      return launch_array_o<ST_DERIV, In>(d_in, g, d_out, out_dtype, integer, st);
    case ST_GRADMAG:
      return launch_array_o<ST_GRADMAG, In>(d_in, g, d_out, out_dtype, integer, st);
    default:
      return launch_array_o<ST_LAPLACIAN, In>(d_in, g, d_out, out_dtype, integer, st);
  }
}

int stencil_array_impl(const hc_stage* in, const int64_t* dims3, double eps, int op, int axis3, void* d_out,
                       int out_dtype, void* d_ws, cudaStream_t st) {
  (void)d_ws;
  const Geo g = stencil_base_geo(dims3, eps, axis3);
  if (in->kind == HC_STAGE_Q) return launch_array_op<int32_t>(in->d_data, g, op, d_out, out_dtype, true, st);
  if (in->kind == HC_STAGE_F) {
    if (in->dtype == HC_F64) return launch_array_op<double>(in->d_data, g, op, d_out, out_dtype, false, st);
    return launch_array_op<float>(in->d_data, g, op, d_out, out_dtype, false, st);
  }
  if (in->kind == HC_STAGE_P)
    return fail(HC_ERR_UNSUPPORTED,
                "stage-2 differentiation is not defined for a 1-D block partition (Section V-B)");
  return fail(HC_ERR_INVALID_ARG, "stencils take a stream or a Q or F array");
}

}  // namespace hc

namespace hc {
// The (possibly remapped) 3-D shape the fused stencil kernels walk: a field
// whose first axis has length 1, (1, n1, n2), is walked as (n1, 1, n2), so
// internal axes 0 and 1 trade places (the derivative along the length-1 axis
// stays 0, now along internal axis 1).
void stencil_walk_dims(const hc_header* h, int64_t d3[3], int* axis3) {
  d3[0] = h->dims[0];
  d3[1] = h->dims[1];
  d3[2] = h->dims[2];
  if (d3[0] == 1 && d3[1] > 1) {
    d3[0] = d3[1];
    d3[1] = 1;
    if (axis3 && *axis3 < 2) *axis3 = 1 - *axis3;
  }
}
}  // namespace hc
