// hc_vector.cu -- divergence and curl of a vector field stored as one
// compressed stream per component (Section V-C, "Multivariate Derivation"),
// on the codes (stage 3), fused: every component is decoded straight from its
// stream into its own ring of plane slabs in shared memory, and each output
// point combines the components' derivative numerators.
//
//   divergence  sum_c D_c, component c differentiated along axis c
//   curl (2-D)  D_u(along j) - D_v(along i), i the first and j the second index
//
// D is the derivative numerator of the scalar stencils (q[+1] - q[-1] inside,
// 2 (q[1] - q[0]) at an edge, 0 along an axis of length 1).  With one eps for
// every component the value is the integer sum times eps (the paper's form);
// with different eps each term is scaled by its own (in double, in component
// order, without contraction).
#include <algorithm>
#include <cstdint>

#include "hc_internal.cuh"
#include "hc_launch.h"
#include "hc_stencil_tile.cuh"
#include "hc_vector_tile.cuh"

namespace hc {

DevStream dev_stream(const hc_header* h, const void* d_stream);

namespace {

template <bool SMALL>
__global__ void __launch_bounds__(kThreads) k_vector_stream(VArgs va, Geo g, void* out, int* err) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_warp[32];
  __shared__ int s_flag;
  __shared__ long long s_base[3][3][66];
  vector_tile<SMALL>(va, g, (int64_t)blockIdx.x, out, err, smem, s_warp, &s_flag, s_base);
}

}  // namespace

int plan_vector(const hc_header* const* hs, int nc, const int64_t* d3, Geo& g, int gmax, int wmax, int* smem_out) {
  const int S = hs[0]->S;
  const bool small = S <= 32;
  const int nseg = (S + 31) / 32;
  g.nslot = g.n0 > 1 ? 3 : 1;
  g.ranges = 1;
  g.tx = (int)g.n2;
  const int64_t budget = 150 * 1024;
  for (int ty : {16, 8, 4, 2, 1}) {
    if (ty > g.n1 && ty != 1) continue;
    const int64_t rows = std::min<int64_t>(ty + 2, g.n1);
    const int64_t span = rows * g.n2;
    if (span > (1 << 22)) continue;
    g.ty = ty;
    g.nblk_max = (int)((span + S - 1) / S + 1);
    g.range_elems = g.nblk_max * S;
    g.slot_words = padded_elems_words(g.range_elems);
    const int nsegmax = small ? g.nblk_max : g.nblk_max * nseg;
    const int bytes = 4 * tile_smem(g.nblk_max, gmax - 1, S, wmax,
                                    nc * g.nslot * g.slot_words + (small ? 0 : round4(nsegmax))).words;
    if (bytes <= budget) {
      *smem_out = bytes;
      g.nxt = 1;
      g.nyt = (int)ceil_div(g.n1, g.ty);
      const int64_t target = (int64_t)device_sms() * 4;
      const int64_t nzt = std::max<int64_t>(1, std::min<int64_t>(g.n0, ceil_div(target, g.nyt)));
      g.tz = (int)ceil_div(g.n0, nzt);
      g.nzt = (int)ceil_div(g.n0, g.tz);
      return HC_OK;
    }
  }
  return fail(HC_ERR_UNSUPPORTED, "vector stencil: rows too long for a fused tile");
}

namespace {

template <bool SMALL>
int launch_vector(const VArgs& va, const Geo& g, int smem, void* d_out, int* err, cudaStream_t st) {
  auto kern = k_vector_stream<SMALL>;
  int rc = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (rc) return rc;
  const int64_t grid = (int64_t)g.nyt * g.nzt;
  if (grid > 0x7fffffff) return fail(HC_ERR_UNSUPPORTED, "field too large");
  kern<<<(unsigned)grid, kThreads, smem, st>>>(va, g, d_out, err);
  return check_launch_cfg("vector stencil", reinterpret_cast<const void*>(kern), grid, smem);
}

}  // namespace

namespace {

// acc (first component: =) += sign * T, integer numerators (one eps)
__global__ void __launch_bounds__(kThreads) k_vec_acc(const long long* __restrict__ T, long long* __restrict__ acc,
                                                       int64_t n, int sign, int first) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc[i] = (first ? 0ll : acc[i]) + sign * T[i];
}

// accd = accd + (sign * T) * eps_c in double, in component order (several eps)
__global__ void __launch_bounds__(kThreads) k_vec_acc_d(const long long* __restrict__ T, double* __restrict__ accd,
                                                         int64_t n, int sign, double eps, int first) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    accd[i] = __dadd_rn(first ? 0.0 : accd[i], __dmul_rn(__ll2double_rn(sign * T[i]), eps));
}

// the scaled output: num * eps (one eps), or the double sum (several)
template <int OUT>
__global__ void __launch_bounds__(kThreads) k_vec_emit(const long long* __restrict__ acc, int64_t n, double eps,
                                                        int same_eps, typename OutType<OUT>::T* __restrict__ out) {
  const double* accd = reinterpret_cast<const double*>(acc);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (OUT == HC_I64) {
      out[i] = acc[i];
    } else if (same_eps) {
      if constexpr (OUT == HC_F32)
        out[i] = __fmul_rn(__ll2float_rn(acc[i]), (float)eps);
      else
        out[i] = __dmul_rn(__ll2double_rn(acc[i]), eps);
    } else {
      out[i] = (typename OutType<OUT>::T)accd[i];
    }
  }
}

unsigned vec_grid(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kThreads), (int64_t)device_sms() * 16));
}

// derivative numerators of one component along internal axis axis3, at
// `level`, by its own predictor's path, into T (int64)
int component_derivative(const hc_header* h, const void* d_stream, int level, int axis3, long long* T, void* d_ws,
                         size_t ws_bytes, cudaStream_t st) {
  if (h->pred == HC_PRED_MEAN_ND)
    return xnd_stencil_impl(h, d_stream, level, ST_DERIV, axis3, T, HC_I64, d_ws, ws_bytes, st);
  if (h->pred >= HC_PRED_LORENZO)
    return global_stencil_impl(h, d_stream, level, ST_DERIV, axis3, T, HC_I64, d_ws, ws_bytes, st);
  if (level != HC_STAGE_Q)
    return fail(HC_ERR_UNSUPPORTED, "stage-2 differentiation is not defined for a 1-D block partition (Section V-B)");
  return stencil_stream_impl(h, d_stream, ST_DERIV, axis3, T, HC_I64, d_ws, st);
}

}  // namespace

size_t vector_any_workspace_bytes(const hc_header* const* hs, int nc) {
  size_t w = kOpWsBytes;
  for (int c = 0; c < nc; ++c) w = std::max(w, hc_workspace_bytes_for(hs[c]));
  return ((w + 15) & ~(size_t)15) + 16 * (size_t)hs[0]->N;
}

// Divergence / curl on streams of any predictor, component by component:
// each component's derivative numerators (its predictor's stage-2 or stage-3
// path) are summed exactly, then scaled as the fused kernel scales them.
int vector_any_impl(const hc_header* const* hs, const void* const* streams, int nc, int op, int level, void* d_out,
                    int out_dtype, void* d_ws, size_t ws_bytes, cudaStream_t st) {
  if (ws_bytes < vector_any_workspace_bytes(hs, nc))
    return fail(HC_ERR_NOMEM, "workspace smaller than hc_vector_workspace_bytes");
  size_t wsp = kOpWsBytes;
  for (int c = 0; c < nc; ++c) wsp = std::max(wsp, hc_workspace_bytes_for(hs[c]));
  wsp = (wsp + 15) & ~(size_t)15;
  const int64_t n = hs[0]->N;
  long long* T = reinterpret_cast<long long*>(reinterpret_cast<char*>(d_ws) + wsp);
  long long* acc = T + n;
  int same_eps = 1;
  for (int c = 1; c < nc; ++c) same_eps &= hs[c]->eps == hs[0]->eps;
  if (out_dtype == HC_I64 && !same_eps)
    return fail(HC_ERR_UNSUPPORTED, "an integer numerator needs one eps for every component");
  const int ndim = hs[0]->ndim;
  for (int c = 0; c < nc; ++c) {
    // divergence: component c along user axis c; curl: u along j, v along i (minus)
    const int user_axis = op == VEC_DIV ? c : (c == 0 ? 1 : 0);
    const int sign = (op == VEC_CURL && c == 1) ? -1 : 1;
    int rc = component_derivative(hs[c], streams[c], level, user_axis + 3 - ndim, T, d_ws, wsp, st);
    if (rc) return rc;
    if (same_eps)
      k_vec_acc<<<vec_grid(n), kThreads, 0, st>>>(T, acc, n, sign, c == 0);
    else
      k_vec_acc_d<<<vec_grid(n), kThreads, 0, st>>>(T, reinterpret_cast<double*>(acc), n, sign, hs[c]->eps, c == 0);
    if ((rc = check_launch("vector operation (sum)"))) return rc;
  }
  switch (out_dtype) {
    case HC_F32:
      k_vec_emit<HC_F32><<<vec_grid(n), kThreads, 0, st>>>(acc, n, hs[0]->eps, same_eps, reinterpret_cast<float*>(d_out));
      break;
    case HC_F64:
      k_vec_emit<HC_F64><<<vec_grid(n), kThreads, 0, st>>>(acc, n, hs[0]->eps, same_eps, reinterpret_cast<double*>(d_out));
      break;
    case HC_I64:
      k_vec_emit<HC_I64><<<vec_grid(n), kThreads, 0, st>>>(acc, n, hs[0]->eps, same_eps,
                                                           reinterpret_cast<long long*>(d_out));
      break;
    default:
      return fail(HC_ERR_INVALID_ARG, "out_dtype");
  }
  return check_launch("vector operation (scale)");
}

// comps: nc stream headers and device streams of the same shape and block
// size; op 0 divergence, 1 curl (2-D, two components).
int vector_stream_impl(const hc_header* const* hs, const void* const* streams, int nc, int op, void* d_out,
                       int out_dtype, void* d_ws, cudaStream_t st) {
  int* err = &reinterpret_cast<OpWs*>(d_ws)->status;
  VArgs va{};
  va.ncomp = nc;
  va.same_eps = 1;
  va.gmax = 1;
  va.wmax = 0;
  for (int c = 0; c < nc; ++c) {
    va.s[c] = dev_stream(hs[c], streams[c]);
    va.eps[c] = hs[c]->eps;
    if (hs[c]->eps != hs[0]->eps) va.same_eps = 0;
    va.gmax = std::max(va.gmax, (int)hs[c]->G);
    va.wmax = std::max(va.wmax, (int)hs[c]->wmax);
  }
  if (out_dtype == HC_I64 && !va.same_eps)
    return fail(HC_ERR_UNSUPPORTED, "an integer numerator needs one eps for every component");
  if (out_dtype != HC_F32 && out_dtype != HC_F64 && out_dtype != HC_I64) return fail(HC_ERR_INVALID_ARG, "out_dtype");
  va.out = out_dtype;
  vector_axes(hs[0], op, nc, va);
  int64_t d3[3];
  int axis3 = 0;
  stencil_walk_dims(hs[0], d3, &axis3);
  Geo g = stencil_base_geo(d3, hs[0]->eps, 0);
  int smem = 0;
  int rc = plan_vector(hs, nc, d3, g, va.gmax, va.wmax, &smem);
  if (rc) return rc;
  if (va.s[0].S <= 32) return launch_vector<true>(va, g, smem, d_out, err, st);
  return launch_vector<false>(va, g, smem, d_out, err, st);
}

}  // namespace hc
