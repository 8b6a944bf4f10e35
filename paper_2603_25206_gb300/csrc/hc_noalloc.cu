// hc_noalloc.cu -- hc_op_variance_noalloc: the fused variance of a
// compressed stream for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or a framework allocator) at the point
// where they need a statistic: allocation-free real-time or embedded loops,
// whose latency budget leaves no room for an allocator call, and plugins that
// are handed a stream and a few pointers by a host application that owns all
// device memory and gives out no allocator.  For
// them this entry point needs no workspace argument: the kernel's scratch
// (one ticket counter and up to kNoAllocParts per-CTA partial sums) lives in a
// file-scope static device array of fixed size, which every GPU that loads
// the library holds until the process exits.  The caller still passes the
// input stream and the output hc_scalar.
#include <mutex>

#include "hc_internal.cuh"
#include "hc_launch.h"

namespace hc {

// Scratch layout: [ticket (unsigned) | pad to 256 B | partials[kNoAllocParts]].
constexpr int kNoAllocParts = 2048;
constexpr size_t kNoAllocHead = 256;
constexpr size_t kNoAllocBytes = kNoAllocHead + sizeof(Partial) * kNoAllocParts;  // 64 KiB + 256 B
// the launch caps its grid at kMaxGrid like the workspace launch, so both
// launches use the same grid whenever it fits the slots
static_assert(kNoAllocParts <= kMaxGrid, "the static partial slots must not exceed the workspace launch's grid cap");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the static scratch, looked up once per device with that
// device current (the host-side name of the array is not a device address).
static int scratch_for_current_device(unsigned char** out) {
  static std::mutex mu;
  static unsigned char* addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return fail(HC_ERR_CUDA, "hc_op_variance_noalloc: no usable current CUDA device");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(HC_ERR_CUDA, "hc_op_variance_noalloc: cudaGetSymbolAddress of the static scratch failed");
    }
    addr[dev] = reinterpret_cast<unsigned char*>(p);
  }
  *out = addr[dev];
  return HC_OK;
}

}  // namespace hc

using namespace hc;

extern "C" HC_API int hc_op_variance_noalloc(const hc_stage* in, double eps, int ndim, const int64_t* dims,
                                             hc_scalar* d_out, void* stream) {
  if (!in || !d_out) return fail(HC_ERR_INVALID_ARG, "null argument");
  if (in->kind != HC_STAGE_COMPRESSED)
    return fail(HC_ERR_UNSUPPORTED, "hc_op_variance_noalloc takes a compressed stream (HC_STAGE_COMPRESSED)");
  if (!in->d_data || !in->hdr) return fail(HC_ERR_INVALID_ARG, "a stream input needs its data and header");
  if (int hrc = check_header(*in->hdr)) return hrc;
  if (in->level != HC_STAGE_P && in->level != HC_STAGE_Q)
    return fail(HC_ERR_INVALID_ARG, "fused level must be HC_STAGE_P or HC_STAGE_Q");
  if (in->hdr && in->hdr->pred == HC_PRED_MEAN && in->level == HC_STAGE_P)
    return fail(HC_ERR_UNSUPPORTED, "the stage-2 block-mean deviation needs a workspace: use hc_op_variance");
  if (in->hdr && in->hdr->pred >= HC_PRED_LORENZO)
    return fail(HC_ERR_UNSUPPORTED, "a global-predictor stream rebuilds D_q in a workspace: use hc_op_variance");
  if (!aligned16(in->d_data)) return fail(HC_ERR_INVALID_ARG, "device buffers must be 16-byte aligned");
  const hc_header* h = in->hdr;
  Layout L;
  int rc = make_layout(ndim, dims, 1, &L);
  if (rc) return rc;
  if (h->ndim != ndim || h->eps != eps) return fail(HC_ERR_INVALID_ARG, "eps / ndim differ from the stream header");
  for (int a = 0; a < 3; ++a)
    if (h->dims[a] != L.dims[a]) return fail(HC_ERR_INVALID_ARG, "dims differ from the stream header");
  unsigned char* base = nullptr;
  rc = scratch_for_current_device(&base);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // The ticket must start at zero; clear it in stream order (no allocation).
  if (cudaMemsetAsync(base, 0, sizeof(unsigned), st) != cudaSuccess)
    return fail(HC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  return variance_stream_scratch_impl(h, in->d_data, d_out, reinterpret_cast<Partial*>(base + kNoAllocHead),
                                      reinterpret_cast<unsigned*>(base), kNoAllocParts, st);
}
