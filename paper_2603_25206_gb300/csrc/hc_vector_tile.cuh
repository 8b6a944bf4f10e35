// hc_vector_tile.cuh -- the fused divergence / curl tile of a vector field
// stored as one compressed stream per component (Section V-C, "Multivariate
// Derivation"), at stage 3 (the codes).  Shared by the one-field kernel
// (hc_vector.cu) and the batched persistent kernel (hc_batch.cu).
//
//   divergence  sum_c D_c, component c differentiated along axis c
//   curl (2-D)  D_u(along j) - D_v(along i), i the first and j the second index
//
// D is the derivative numerator of the scalar stencils (q[+1] - q[-1] inside,
// 2 (q[1] - q[0]) at an edge, 0 along an axis of length 1).  With one eps for
// every component the value is the integer sum times eps (the paper's form);
// with different eps each term is scaled by its own (in double, in component
// order, without contraction).
#pragma once

#include <cstdint>

#include "hc_internal.cuh"
#include "hc_launch.h"
#include "hc_stencil_tile.cuh"

namespace hc {

enum { VEC_DIV = 0, VEC_CURL = 1 };

// The components of one vector operation.
struct VArgs {
  DevStream s[3];
  double eps[3];
  int axes[3];  // internal axis each component is differentiated along
  int sign[3];  // +1 / -1: the component's derivative is added or subtracted
                // (divergence: all +1; curl: u along j minus v along i)
  int ncomp;
  int out;      // hc_dtype of the output
  int same_eps;
  int gmax, wmax;  // staging buffer: largest G and block width over the components
};

// Axes and signs of the components of a divergence (op VEC_DIV: component c
// along user axis c) or 2-D curl (VEC_CURL: u along j minus v along i), in the
// internal axes of the shape the tiles walk (stencil_walk_dims).  Host.
inline void vector_axes(const hc_header* h0, int op, int nc, VArgs& va) {
  const int ndim = h0->ndim;
  int64_t d3[3];
  int amap[3] = {0, 0, 0};
  for (int a = 0; a < ndim; ++a) {
    int axis3 = a + 3 - ndim;
    stencil_walk_dims(h0, d3, &axis3);
    amap[a] = axis3;
  }
  for (int c = 0; c < 3; ++c) {
    va.axes[c] = 0;
    va.sign[c] = 0;
  }
  if (op == VEC_DIV) {
    for (int c = 0; c < nc; ++c) {
      va.axes[c] = amap[c];
      va.sign[c] = 1;
    }
  } else {
    va.axes[0] = amap[1];  // u along j
    va.sign[0] = 1;
    va.axes[1] = amap[0];  // v along i, subtracted
    va.sign[1] = -1;
  }
}

// derivative numerator of ring `ring` (one component) at (z, y, x) along axis a
__device__ __forceinline__ long long dnum(const Geo& g, const int32_t* ring, long long (*base)[66], int64_t z,
                                          int64_t y, int x, int a) {
  auto at = [&](int64_t zz, int64_t yy, int xx) -> int32_t {
    const int slot = ring_slot(g, zz);
    const int r = (int)((zz * g.n1 + yy) * g.n2 + xx - base[slot][0]);
    return ring[slot * g.slot_words + pidx(r)];
  };
  if (a == 0) {
    const int64_t zm = z > 0 ? z - 1 : 0, zp = z + 1 < g.n0 ? z + 1 : z;
    const int e = (z == 0 || z == g.n0 - 1) ? 2 : 1;
    return ((long long)at(zp, y, x) - at(zm, y, x)) * e;
  }
  if (a == 1) {
    const int64_t ym = y > 0 ? y - 1 : 0, yp = y + 1 < g.n1 ? y + 1 : y;
    const int e = (y == 0 || y == g.n1 - 1) ? 2 : 1;
    return ((long long)at(z, yp, x) - at(z, ym, x)) * e;
  }
  const int n2 = (int)g.n2;
  const int xm = x > 0 ? x - 1 : 0, xp = x + 1 < n2 ? x + 1 : x;
  const int e = (x == 0 || x == n2 - 1) ? 2 : 1;
  return ((long long)at(z, y, xp) - at(z, y, xm)) * e;
}

// One output tile t (row tile t % nyt, plane range t / nyt) of the
// divergence or curl: every component decoded straight from its stream into
// its own ring of plane slabs, each output point combining the components'
// signed derivative numerators (va.sign) and written in va.out's type.
// smem: the dynamic shared memory of plan_vector; s_base: per component and
// ring slot, the element offset of the slot.  Every thread of the CTA must
// call it.
template <bool SMALL>
__device__ inline void vector_tile(const VArgs& va, const Geo& g, int64_t t, void* out, int* err, uint32_t* smem,
                                   uint32_t* s_warp, int* s_flag, long long (*s_base)[3][66]) {
  const int nc = va.ncomp;
  const int S = va.s[0].S;
  const int nsegmax = SMALL ? g.nblk_max : g.nblk_max * va.s[0].nseg;
  const TileSmem L = tile_smem(g.nblk_max, va.gmax - 1, S, va.wmax,
                               nc * g.nslot * g.slot_words + (SMALL ? 0 : round4(nsegmax)));
  uint32_t* s_stage = smem;
  uint32_t* s_off = smem + L.off;
  int32_t* rings = reinterpret_cast<int32_t*>(smem + L.extra);
  int32_t* s_tot = rings + nc * g.nslot * g.slot_words;
  uint8_t* s_w = reinterpret_cast<uint8_t*>(smem + L.w);
  const int range_words = padded_elems_words(g.range_elems);

  const int yt = (int)(t % g.nyt);
  const int zt = (int)(t / g.nyt);
  const int64_t y0 = (int64_t)yt * g.ty, y1 = min(y0 + g.ty, g.n1);
  const int64_t z0 = (int64_t)zt * g.tz, z1 = min(z0 + g.tz, g.n0);
  const int64_t ylo = max(y0 - 1, (int64_t)0), yhi = min(y1 + 1, g.n1);

  auto load = [&](int c, int64_t z) {
    load_slab<SMALL>(va.s[c], g, z, ylo, yhi, 0, g.n2, true, rings + c * g.nslot * g.slot_words, range_words,
                     s_base[c], s_w, s_off, s_stage, L.stage_words, s_tot, s_warp, s_flag, err);
  };
  for (int c = 0; c < nc; ++c) {
    if (z0 > 0) load(c, z0 - 1);
    load(c, z0);
  }
  const int n2 = (int)g.n2;
  for (int64_t z = z0; z < z1; ++z) {
    if (z + 1 < g.n0)
      for (int c = 0; c < nc; ++c) load(c, z + 1);
    for (int64_t y = y0; y < y1; ++y) {
      const int64_t row = (z * g.n1 + y) * g.n2;
      for (int x = threadIdx.x; x < n2; x += blockDim.x) {
        long long D[3] = {0, 0, 0};
        for (int c = 0; c < nc; ++c)
          D[c] = va.sign[c] * dnum(g, rings + c * g.nslot * g.slot_words, s_base[c], z, y, x, va.axes[c]);
        const long long num = D[0] + D[1] + D[2];
        if (va.out == HC_I64) {
          reinterpret_cast<long long*>(out)[row + x] = num;
        } else if (va.same_eps) {
          if (va.out == HC_F32)
            reinterpret_cast<float*>(out)[row + x] = __fmul_rn(__ll2float_rn(num), (float)va.eps[0]);
          else
            reinterpret_cast<double*>(out)[row + x] = __dmul_rn(__ll2double_rn(num), va.eps[0]);
        } else {
          double v = 0.0;
          for (int c = 0; c < nc; ++c) v = __dadd_rn(v, __dmul_rn(__ll2double_rn(D[c]), va.eps[c]));
          if (va.out == HC_F32)
            reinterpret_cast<float*>(out)[row + x] = (float)v;
          else
            reinterpret_cast<double*>(out)[row + x] = v;
        }
      }
    }
    __syncthreads();
  }
}

// Geometry of the vector tile (host): whole rows, the largest tile height
// whose rings (one per component) fit the shared-memory budget; the plane
// ranges give about four tiles per SM.  *smem_out: dynamic shared memory.
int plan_vector(const hc_header* const* hs, int nc, const int64_t* d3, Geo& g, int gmax, int wmax, int* smem_out);

}  // namespace hc
