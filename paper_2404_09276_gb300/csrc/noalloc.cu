// Allocation-free Gram matrix for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running while a CUDA graph
// is being captured, allocators that own all device memory (a host framework
// with its own pool, an embedded or sandboxed runtime), or real-time paths
// that must not block on the driver's allocator. dashsvd_gram_noalloc
// computes the same G = C^T C as dashsvd_gram with no handle and no
// allocation: its per-chunk partial sums live in one fixed, file-scope device
// array that the library holds on every GPU that loads it, for as long as the
// process runs.
#include <mutex>

#include "internal.cuh"

namespace dsvd {
namespace {

constexpr size_t kNoAllocScratchFloats = (size_t)4 << 20;  // 16 MiB of FP32 partial sums
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float* g_scratch_ptr[kMaxDevices];  // device address of g_noalloc_scratch, per device
int g_num_sms[kMaxDevices];

}  // namespace
}  // namespace dsvd

using namespace dsvd;

extern "C" int dashsvd_gram_noalloc(const float* C, int64_t rows, int l, int64_t ldc, float* G, int64_t ldg,
                                    void* cuda_stream) {
  if (!C || !G || rows < 0 || l < 1 || l > DASHSVD_MAX_L || ldc < l || ldc % 4 || ldg < l ||
      ((uintptr_t)C & 15u) != 0)
    return DASHSVD_EINVAL;
  int dev = 0;
  DS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return DASHSVD_ENOTIMPL;
  {
    // once per device, with that device current: the host-side name of the
    // array is not a device address, so look the address up
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      DS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      int sms = 0;
      DS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      g_num_sms[dev] = sms;
      g_scratch_ptr[dev] = reinterpret_cast<float*>(p);
    }
  }
  // every partial block is written before it is read, so nothing needs clearing
  DS_CUDA(launch_gram_bounded(C, rows, l, ldc, G, ldg, g_scratch_ptr[dev], kNoAllocScratchFloats, g_num_sms[dev],
                              (cudaStream_t)cuda_stream));
  return DASHSVD_OK;
}
