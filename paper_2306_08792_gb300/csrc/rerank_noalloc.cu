// Re-ranking for callers that cannot allocate device memory.
//
// gcr_rerank needs a scratch buffer (the query x gallery distance matrix plus row norms)
// that the caller normally allocates and passes in. Some callers cannot do that: a serving
// process that fixes its whole device-memory budget at start-up and must not allocate per
// request (an allocation can block, can synchronise the device and can fail once memory is
// fragmented), or a host application that embeds this library without giving it any
// allocator. For them gcr_rerank_noalloc runs the same computation with its scratch in a
// fixed array that is part of the library's device image, so the call itself allocates
// nothing.
//
// The array (GCR_RERANK_NOALLOC_SCRATCH_BYTES) is reserved on a device when the driver loads
// this library's device code there. Under CUDA's lazy module loading (the default) that is the
// cudaGetSymbolAddress call below, made during the first call of the entry point with the
// device current; from then on it stays reserved until the process exits. A process that fixes
// its memory budget at start-up should therefore make one call per device before doing so (with
// the device already full, the first call fails with GCR_E_CUDA), and before any stream capture.
// The address is cached per device; it stays valid until the device is reset (cudaDeviceReset,
// or a new primary context), after which the entry point must not be called on that device. All calls share the one array: calls whose work overlaps
// on the GPU (different streams, or different host threads without ordering) race on it and
// must be serialised by the caller. Nothing in it needs to start at zero: every byte the
// re-ranking reads is written earlier in the same call.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kScratchBytes = GCR_RERANK_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_rerank_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];  // device address of g_rerank_scratch, per device
std::mutex g_scratch_mu;

// Host code cannot use g_rerank_scratch directly: on the host that name denotes a shadow
// variable, not device memory. The device address comes from cudaGetSymbolAddress, taken
// with the device current.
int scratch_of_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GCR_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GCR_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_rerank_scratch) != cudaSuccess || p == nullptr) return GCR_E_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return GCR_OK;
}

}  // namespace

extern "C" int gcr_rerank_noalloc(const float* Xq, int64_t nq, const float* Xg, int64_t ng, int32_t d,
                                  const gcr_params* p, int32_t* idx_out, float* dist_out,
                                  gcr_stream_t stream) {
  const size_t need = gcr_rerank_workspace_size(nq, ng, d, p);
  if (need == 0)  // invalid or unsupported arguments: gcr_rerank reports which, launching nothing
    return gcr_rerank(Xq, nq, Xg, ng, d, p, idx_out, dist_out, nullptr, 0, stream);
  if (need > kScratchBytes) return GCR_E_WORKSPACE;
  void* ws = nullptr;
  const int s = scratch_of_current_device(&ws);
  if (s != GCR_OK) return s;
  return gcr_rerank(Xq, nq, Xg, ng, d, p, idx_out, dist_out, ws, kScratchBytes, stream);
}
