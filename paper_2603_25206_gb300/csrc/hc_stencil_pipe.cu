// hc_stencil_pipe.cu -- launch of the pipelined fused stencil tile
// (hc_stencil_pipe.cuh) for one field: grid planning, the tile-height
// autotuner and the dispatch over operation, output type and row width.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "hc_finish.cuh"
#include "hc_group.cuh"
#include "hc_internal.cuh"
#include "hc_launch.h"
#include "hc_stencil_pipe.cuh"

namespace hc {

DevStream dev_stream(const hc_header* h, const void* d_stream);

template <int OP, int OUT, int V, int PRED>
__global__ void __launch_bounds__(kThreads) k_stencil_pipe(DevStream s, PGeo g, typename OT<OUT>::T* __restrict__ out,
                                                            int* err) {
  extern __shared__ __align__(16) unsigned char sm[];
  Moments mo;
  pipe_tile<OP, OUT, V, false, PRED>(s, g, (int)(blockIdx.x % g.nyt), (int)(blockIdx.x / g.nyt), out, err, sm, mo);
}

// All operations of one field from one decode (ST_MULTI); with STATS the
// exact sums of the codes go through the per-CTA partials and the last CTA
// finishes the stage-3 statistics.
template <int OUT, int V, bool STATS, int PRED>
__global__ void __launch_bounds__(kThreads) k_stencil_multi(DevStream s, PGeo g, int* err, Partial* parts,
                                                             unsigned* ticket, hc_scalar* stats, double two_eps) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int s_err;
  if (threadIdx.x == 0) s_err = 0;
  __syncthreads();
  Moments mo;
  pipe_tile<ST_MULTI, OUT, V, STATS, PRED>(s, g, (int)(blockIdx.x % g.nyt), (int)(blockIdx.x / g.nyt), nullptr,
                                           &s_err, sm, mo);
  __syncthreads();
  const int e = s_err;
  if (threadIdx.x == 0 && e) set_error(err, e);
  if constexpr (STATS) {
    const u128 s2 = ((u128)mo.hi << 64) | (u128)mo.lo;
    reduce_and_finish(mo.s1, s2, e, parts, ticket,
                      [&](long long a, u128 b, int ee) { finalize_int(stats, s.N, a, b, true, two_eps, ee); });
  }
}

// ------------------------------------------------------------------ host
// The fast path applies when: S = 32, |q| < 2^15, the output is 16-byte
// aligned, and a tile of at least one row fits the shared-memory budget (rows
// of any length: 8-wide items, vector ones when the row length allows).  The
// tile height is the largest that keeps at least three CTAs per SM; the plane
// ranges are sized so that the grid fills whole waves of resident CTAs.
bool plan_pipe_geometry(const hc_header* h, const int64_t* d3, PGeo& g, int* smem_out, int force_ty, int budget,
                        int max_ty) {
  if (h->S != 32 || h->qmax >= 32768u) return false;
  g.n0 = d3[0];
  g.n1 = d3[1];
  g.n2 = d3[2];
  const int S = 32;
  int chosen = 0;
  int heights[10];
  const int nh = pipe_heights(g.n1, heights);
  for (int hi = 0; hi < nh; ++hi) {
    const int ty = heights[hi];
    if (force_ty && ty != force_ty) continue;
    if (!force_ty && max_ty > 0 && ty > max_ty) continue;
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
  g.grp = group_for_width(h->wmax);
  return true;
}

bool plan_pipe_items(PGeo& g, int V) {
  // V = 0: items of 8 at any offset plus a scalar tail (rows of any length)
  const int vw = V == 0 ? 8 : V;
  if (V != 0 && g.n2 % V != 0) return false;
  g.nq = (int)(g.n2 / vw);
  if (g.nq <= 1) {
    g.nq_magic = 0u;
    return true;
  }
  const uint64_t m = ((1ull << 32) + (uint64_t)g.nq - 1) / (uint64_t)g.nq;
  // floor(it * m / 2^32) == it / nq for every item index it < ty * nq when
  // (ty * nq - 1) * (m * nq - 2^32) < 2^32
  const uint64_t e = m * (uint64_t)g.nq - (1ull << 32);
  const uint64_t it_max = (uint64_t)g.ty * (uint64_t)g.nq - 1;
  if (e != 0 && it_max >= ((1ull << 32) + e - 1) / e) return false;
  g.nq_magic = (unsigned)m;
  return true;
}

static void plan_pipe_grid(PGeo& g, int per_sm) {
  const int64_t capacity = (int64_t)device_sms() * std::max(per_sm, 1) * std::max(g.waves, 1);
  // g.waves waves of resident CTAs when the rows allow it; never fewer than
  // 4 planes per CTA
  int64_t nzt = std::max<int64_t>(1, capacity / g.nyt);
  nzt = std::min<int64_t>(nzt, std::max<int64_t>(1, g.n0 / 4));
  g.tz = (int)ceil_div(g.n0, nzt);
  g.nzt = (int)ceil_div(g.n0, g.tz);
}

template <int OP, int OUT, int V, int PRED>
static int launch_pipe_p(const hc_header* h, const void* d_stream, PGeo g, int smem, void* d_out, int* err,
                         cudaStream_t st) {
  auto kern = k_stencil_pipe<OP, OUT, V, PRED>;
  if (!plan_pipe_items(g, V)) return HC_ERR_UNSUPPORTED;
  int rc = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (rc) return rc;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  plan_pipe_grid(g, per_sm);
  const int64_t grid = (int64_t)g.nyt * g.nzt;
  kern<<<(unsigned)grid, kThreads, smem, st>>>(dev_stream(h, d_stream), g,
                                                reinterpret_cast<typename OT<OUT>::T*>(d_out), err);
  return check_launch_cfg("stencil (pipelined)", reinterpret_cast<const void*>(kern), grid, smem);
}

template <int OP, int OUT, int V>
static int launch_pipe_o(const hc_header* h, const void* d_stream, const PGeo& g, int smem, void* d_out, int* err,
                         cudaStream_t st) {
  if (h->pred == HC_PRED_MEAN) return launch_pipe_p<OP, OUT, V, HC_PRED_MEAN>(h, d_stream, g, smem, d_out, err, st);
  return launch_pipe_p<OP, OUT, V, HC_PRED_DELTA>(h, d_stream, g, smem, d_out, err, st);
}

template <int OP, int OUT>
static int launch_pipe_v(const hc_header* h, const void* d_stream, const PGeo& g, int smem, void* d_out, int* err,
                         cudaStream_t st) {
  if (g.n2 % 8 == 0) return launch_pipe_o<OP, OUT, 8>(h, d_stream, g, smem, d_out, err, st);
  if (g.n2 % 4 == 0) return launch_pipe_o<OP, OUT, 4>(h, d_stream, g, smem, d_out, err, st);
  return launch_pipe_o<OP, OUT, 0>(h, d_stream, g, smem, d_out, err, st);
}

// Returns HC_ERR_UNSUPPORTED (without recording an error) when the fast path
// does not apply.
// Tile heights and grid waves picked by hc_autotune, per (shape, max width,
// op, output type); a choice is coded as ty | waves << 8 (0: untuned).
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

static int tuned_choice(const hc_header* h, const int64_t* d3, int op, int out_dtype) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(TuneKey{d3[0], d3[1], d3[2], (int)h->wmax, op, out_dtype});
  return it == g_tuned.end() ? 0 : it->second;
}

// ---------------------------------------------- the choices as JSON text
// {"format": "hc-autotune", "version": 1, "entries": [{"n0": .., "n1": ..,
// "n2": .., "wmax": .., "op": "derivative" | "gradmag" | "laplacian" |
// "multi", "out": "float32" | "float64" | "int64", "tile_rows": ..,
// "waves": ..}, ...]}: (n0, n1, n2) the shape the fused stencils walk.
namespace {
const char* const kTuneOps[] = {"derivative", "gradmag", "laplacian", "multi"};  // ST_DERIV .. ST_MULTI
const char* tune_out_name(int out) { return out == HC_F32 ? "float32" : (out == HC_F64 ? "float64" : "int64"); }

// A reader of exactly the export format: objects, arrays, strings without
// escapes, non-negative integers of at most 15 digits.
struct JsonIn {
  const char* p;
  void ws() {
    while (*p == ' ' || *p == '\n' || *p == '\t' || *p == '\r') ++p;
  }
  bool eat(char c) {
    ws();
    if (*p != c) return false;
    ++p;
    return true;
  }
  bool str(std::string& out) {
    ws();
    if (*p != '"') return false;
    ++p;
    out.clear();
    while (*p && *p != '"') {
      if (*p == '\\' || (unsigned char)*p < 0x20) return false;
      out += *p++;
    }
    if (*p != '"') return false;
    ++p;
    return true;
  }
  bool num(int64_t& v) {
    ws();
    if (*p < '0' || *p > '9') return false;
    v = 0;
    int digits = 0;
    while (*p >= '0' && *p <= '9') {
      if (++digits > 15) return false;
      v = v * 10 + (*p++ - '0');
    }
    return true;
  }
};

// One entry object; false when a key is missing, unknown or repeated, or a
// value is out of range.
bool read_entry(JsonIn& in, TuneKey& key, int& choice) {
  if (!in.eat('{')) return false;
  int64_t v[6] = {0, 0, 0, 0, 0, 0};  // n0, n1, n2, wmax, tile_rows, waves
  const char* names[6] = {"n0", "n1", "n2", "wmax", "tile_rows", "waves"};
  int op = -1, out = -1;
  unsigned seen = 0;
  for (;;) {
    std::string k;
    if (!in.str(k) || !in.eat(':')) return false;
    int slot = -1;
    for (int i = 0; i < 6; ++i)
      if (k == names[i]) slot = i;
    if (slot >= 0) {
      if (seen & (1u << slot) || !in.num(v[slot])) return false;
      seen |= 1u << slot;
    } else if (k == "op" || k == "out") {
      const unsigned bit = k == "op" ? 1u << 6 : 1u << 7;
      std::string val;
      if (seen & bit || !in.str(val)) return false;
      seen |= bit;
      if (k == "op") {
        for (int i = 0; i < 4; ++i)
          if (val == kTuneOps[i]) op = i;
        if (op < 0) return false;
      } else {
        out = val == "float32" ? HC_F32 : (val == "float64" ? HC_F64 : (val == "int64" ? HC_I64 : -1));
        if (out < 0) return false;
      }
    } else {
      return false;
    }
    if (in.eat(',')) continue;
    if (in.eat('}')) break;
    return false;
  }
  if (seen != 0xffu) return false;
  const int64_t kMaxDim = (int64_t)1 << 40;
  for (int i = 0; i < 3; ++i)
    if (v[i] < 1 || v[i] > kMaxDim) return false;
  if (v[3] > 32 || v[4] < 1 || v[4] > 255 || v[5] < 1 || v[5] > 2) return false;
  // combinations the tuner never records: no integer gradient magnitude, and
  // the one-pass kernel writes floating-point outputs only
  if (out == HC_I64 && (op == ST_GRADMAG || op == ST_MULTI)) return false;
  key = TuneKey{v[0], v[1], v[2], (int)v[3], op, out};
  choice = (int)v[4] | (int)(v[5] << 8);
  return true;
}
}  // namespace

int autotune_export_impl(char* buf, size_t cap, size_t* len) {
  if (!len) return fail(HC_ERR_INVALID_ARG, "null length");
  std::string t = "{\"format\": \"hc-autotune\", \"version\": 1, \"entries\": [";
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    bool first = true;
    for (const auto& kv : g_tuned) {
      char e[320];
      const TuneKey& k = kv.first;
      std::snprintf(e, sizeof(e),
                    "%s\n  {\"n0\": %lld, \"n1\": %lld, \"n2\": %lld, \"wmax\": %d, \"op\": \"%s\", \"out\": \"%s\", "
                    "\"tile_rows\": %d, \"waves\": %d}",
                    first ? "" : ",", (long long)k.n0, (long long)k.n1, (long long)k.n2, k.wmax,
                    kTuneOps[k.op], tune_out_name(k.out), kv.second & 0xff, std::max(1, kv.second >> 8));
      t += e;
      first = false;
    }
  }
  t += "]}\n";
  *len = t.size();
  if (!buf) return HC_OK;  // size query
  if (cap <= t.size()) return fail(HC_ERR_NOMEM, "buffer too small for the autotune text");
  std::memcpy(buf, t.c_str(), t.size() + 1);
  return HC_OK;
}

int autotune_import_impl(const char* text, int* count) {
  if (!text || !count) return fail(HC_ERR_INVALID_ARG, "null argument");
  *count = 0;
  JsonIn in{text};
  std::vector<std::pair<TuneKey, int>> got;
  bool fmt = false, ver = false, ents = false;
  auto bad = [](const char* why) { return fail(HC_ERR_INVALID_ARG, why); };
  if (!in.eat('{')) return bad("autotune text: not an object");
  for (;;) {
    std::string k;
    if (!in.str(k) || !in.eat(':')) return bad("autotune text: expected a key");
    if (k == "format" && !fmt) {
      std::string v;
      if (!in.str(v) || v != "hc-autotune") return bad("autotune text: format is not hc-autotune");
      fmt = true;
    } else if (k == "version" && !ver) {
      int64_t v;
      if (!in.num(v) || v != 1) return bad("autotune text: unsupported version");
      ver = true;
    } else if (k == "entries" && !ents) {
      if (!in.eat('[')) return bad("autotune text: entries is not an array");
      if (!in.eat(']')) {
        for (;;) {
          TuneKey key{};
          int choice = 0;
          if (!read_entry(in, key, choice)) return bad("autotune text: malformed or out-of-range entry");
          got.emplace_back(key, choice);
          if (in.eat(',')) continue;
          if (in.eat(']')) break;
          return bad("autotune text: expected , or ] in entries");
        }
      }
      ents = true;
    } else {
      return bad("autotune text: unknown or repeated key");
    }
    if (in.eat(',')) continue;
    if (in.eat('}')) break;
    return bad("autotune text: expected , or }");
  }
  in.ws();
  if (*in.p != '\0') return bad("autotune text: trailing characters");
  if (!fmt || !ver || !ents) return bad("autotune text: format, version and entries are required");
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (const auto& e : got) g_tuned[e.first] = e.second;
  *count = (int)got.size();
  return HC_OK;
}

static int stencil_pipe_launch(const hc_header* h, const void* d_stream, const int64_t* d3, int op, int axis3,
                               void* d_out, int out_dtype, void* d_ws, cudaStream_t st, int tune);

int stencil_pipe_impl(const hc_header* h, const void* d_stream, const int64_t* d3, int op, int axis3, void* d_out,
                      int out_dtype, void* d_ws, cudaStream_t st) {
  return stencil_pipe_launch(h, d_stream, d3, op, axis3, d_out, out_dtype, d_ws, st,
                             tuned_choice(h, d3, op, out_dtype));
}

static int stencil_multi_launch(const hc_header* h, const void* d_stream, void* const outs[5], hc_scalar* d_stats,
                                int out_dtype, void* d_ws, cudaStream_t st, int tune);

// Time every tile height that fits on this field, each with the plane
// ranges sized for one and for two waves of resident CTAs, and remember the
// fastest pair.  *chosen: the chosen height (0 when the pipelined kernel
// does not apply).
int stencil_pipe_autotune(const hc_header* h, const void* d_stream, const int64_t* d3, int op, void* d_out,
                          int out_dtype, void* d_ws, cudaStream_t st, int* chosen) {
  *chosen = 0;
  float best = 0.f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(HC_ERR_CUDA, "autotune: cudaEventCreate failed");
  int heights[10];
  int pick = 0;
  const int nh = pipe_heights(d3[1], heights);
  for (int hw = 0; hw < 2 * nh; ++hw) {
    const int ty = heights[hw >> 1], waves = 1 + (hw & 1);
    const int tune = ty | (waves << 8);
    PGeo g{};
    int smem = 0;
    if (!plan_pipe_geometry(h, d3, g, &smem, ty, 200 * 1024)) continue;
    float times[3];
    int rc = HC_OK;
    for (int r = -1; r < 3 && rc == HC_OK; ++r) {
      cudaEventRecord(e0, st);
      if (op == ST_MULTI) {
        // the one-pass kernel: (ndim + 2) output fields one after the other
        const size_t esz = out_dtype == HC_F64 ? 8 : 4;
        const size_t nb = esz * (size_t)h->N;
        char* o = reinterpret_cast<char*>(d_out);
        void* outs[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        int k = 0;
        // derivative outputs for the user axes, in the walk's internal axes
        for (int a = 0; a < h->ndim; ++a) {
          int axis3 = a + 3 - h->ndim;
          int64_t dd[3];
          stencil_walk_dims(h, dd, &axis3);
          outs[axis3] = o + (k++) * nb;
        }
        outs[3] = o + (k++) * nb;
        outs[4] = o + (k++) * nb;
        rc = stencil_multi_launch(h, d_stream, outs, nullptr, out_dtype, d_ws, st, tune);
      } else {
        rc = stencil_pipe_launch(h, d_stream, d3, op, 0, d_out, out_dtype, d_ws, st, tune);
      }
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = HC_ERR_CUDA;
      if (r >= 0) cudaEventElapsedTime(&times[r], e0, e1);
    }
    if (rc != HC_OK) continue;
    std::sort(times, times + 3);
    if (pick == 0 || times[1] < best) {
      best = times[1];
      pick = tune;
    }
  }
  *chosen = pick & 0xff;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  if (*chosen) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[TuneKey{d3[0], d3[1], d3[2], (int)h->wmax, op, out_dtype}] = pick;
  }
  return HC_OK;
}

static int stencil_pipe_launch(const hc_header* h, const void* d_stream, const int64_t* d3, int op, int axis3,
                               void* d_out, int out_dtype, void* d_ws, cudaStream_t st, int tune) {
  PGeo g{};
  int smem = 0;
  const int force_ty = tune & 0xff;
  if (!aligned16(d_out) || !plan_pipe_geometry(h, d3, g, &smem, force_ty, force_ty ? 200 * 1024 : 74 * 1024))
    return HC_ERR_UNSUPPORTED;
  g.waves = std::max(1, tune >> 8);
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

template <int OUT, int V, bool STATS, int PRED>
static int launch_multi_p(const hc_header* h, const void* d_stream, PGeo g, int smem, hc_scalar* d_stats, void* d_ws,
                          cudaStream_t st) {
  auto kern = k_stencil_multi<OUT, V, STATS, PRED>;
  if (!plan_pipe_items(g, V)) return HC_ERR_UNSUPPORTED;
  int rc = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (rc) return rc;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  plan_pipe_grid(g, per_sm);
  if (STATS && (int64_t)g.nyt * g.nzt > kMaxGrid) {
    // one partial per CTA: fewer, taller plane ranges
    if (g.nyt > kMaxGrid) return HC_ERR_UNSUPPORTED;
    const int64_t nzt = std::max<int64_t>(1, kMaxGrid / g.nyt);
    g.tz = (int)ceil_div(g.n0, nzt);
    g.nzt = (int)ceil_div(g.n0, g.tz);
  }
  const int64_t grid = (int64_t)g.nyt * g.nzt;
  OpWs* ws = reinterpret_cast<OpWs*>(d_ws);
  kern<<<(unsigned)grid, kThreads, smem, st>>>(dev_stream(h, d_stream), g, &ws->status, ws_partials(d_ws),
                                                &ws->ticket, d_stats, 2.0 * h->eps);
  return check_launch_cfg("stencil (all operations)", reinterpret_cast<const void*>(kern), grid, smem);
}

template <int OUT, int V, bool STATS>
static int launch_multi(const hc_header* h, const void* d_stream, const PGeo& g, int smem, hc_scalar* d_stats,
                        void* d_ws, cudaStream_t st) {
  if (h->pred == HC_PRED_MEAN) return launch_multi_p<OUT, V, STATS, HC_PRED_MEAN>(h, d_stream, g, smem, d_stats, d_ws, st);
  return launch_multi_p<OUT, V, STATS, HC_PRED_DELTA>(h, d_stream, g, smem, d_stats, d_ws, st);
}

int stencil_multi_impl(const hc_header* h, const void* d_stream, void* const deriv3[3], void* d_grad, void* d_lap,
                       hc_scalar* d_stats, int out_dtype, void* d_ws, cudaStream_t st) {
  int64_t d3[3];
  stencil_walk_dims(h, d3, nullptr);
  void* outs[5] = {deriv3[0], deriv3[1], deriv3[2], d_grad, d_lap};
  return stencil_multi_launch(h, d_stream, outs, d_stats, out_dtype, d_ws, st,
                              tuned_choice(h, d3, ST_MULTI, out_dtype));
}

static int stencil_multi_launch(const hc_header* h, const void* d_stream, void* const outs_in[5], hc_scalar* d_stats,
                                int out_dtype, void* d_ws, cudaStream_t st, int tune) {
  const int force_ty = tune & 0xff;
  if (out_dtype != HC_F32 && out_dtype != HC_F64) return HC_ERR_UNSUPPORTED;
  void* outs[5] = {outs_in[0], outs_in[1], outs_in[2], outs_in[3], outs_in[4]};
  for (void* o : outs)
    if (o && !aligned16(o)) return HC_ERR_UNSUPPORTED;
  int64_t d3[3];
  stencil_walk_dims(h, d3, nullptr);
  PGeo g{};
  int smem = 0;
  if (!plan_pipe_geometry(h, d3, g, &smem, force_ty, force_ty ? 200 * 1024 : 74 * 1024)) return HC_ERR_UNSUPPORTED;
  if (g.n1 * g.n2 >= ((int64_t)1 << 31)) return HC_ERR_UNSUPPORTED;
  g.waves = std::max(1, tune >> 8);
  g.axis = 0;
  g.op = ST_MULTI;
  g.out = out_dtype;
  for (int k = 0; k < 5; ++k) g.mout[k] = outs[k];
  g.eps = h->eps;
  g.te = 2.0 * h->eps;
  g.eps_f = (float)h->eps;
  g.te_f = (float)(2.0 * h->eps);
  const int v = g.n2 % 8 == 0 ? 8 : (g.n2 % 4 == 0 ? 4 : 0);
#define HC_MULTI(OUTT, VV)                                                                                  \
  return d_stats ? launch_multi<OUTT, VV, true>(h, d_stream, g, smem, d_stats, d_ws, st)                    \
                 : launch_multi<OUTT, VV, false>(h, d_stream, g, smem, d_stats, d_ws, st);
  if (out_dtype == HC_F32) {
    if (v == 8) {
      HC_MULTI(HC_F32, 8)
    } else if (v == 4) {
      HC_MULTI(HC_F32, 4)
    } else {
      HC_MULTI(HC_F32, 0)
    }
  } else {
    if (v == 8) {
      HC_MULTI(HC_F64, 8)
    } else if (v == 4) {
      HC_MULTI(HC_F64, 4)
    } else {
      HC_MULTI(HC_F64, 0)
    }
  }
#undef HC_MULTI
}

}  // namespace hc
