// noalloc.cu - correlation matrices for callers that cannot allocate device
// memory.
//
// mraid_ccm_noalloc runs the same Gram and correlation kernels as
// mraid_ccm, but its int64 Gram sums and zero-variance counter live in one
// file-scope __device__ array instead of plan-owned allocations, and it
// needs no plan. The array is a fixed 8 MiB that every device which loads
// the library keeps until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>

#include "internal.h"

namespace mraid {
namespace {

constexpr size_t kNoAllocScratchBytes = 8u << 20;
constexpr size_t kNoAllocHeader = 256;  // zero-variance counter, padded
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once with that
// device current (the host-side symbol is only a stand-in) and kept for the
// life of the process: a context destroyed and recreated (cudaDeviceReset)
// may load the module elsewhere, so calls after that are not supported.
std::atomic<void*> g_noalloc_addr[kNoAllocMaxDevices];

mraid_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("mraid_ccm_noalloc: device %d beyond the %d supported", dev, kNoAllocMaxDevices);
    return MRAID_ERR_UNSUPPORTED;
  }
  void* p = g_noalloc_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_noalloc_addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return MRAID_OK;
}

}  // namespace
}  // namespace mraid

using namespace mraid;

extern "C" mraid_status mraid_ccm_noalloc(const mraid_params* p, const void* d_data, int32_t sub0,
                                          int32_t n_sub, float* d_corr, void* stream) {
  mraid_status st = mraid_validate(p);
  if (st != MRAID_OK) return st;
  if (p->bit_depth != 8) {
    set_error("mraid_ccm_noalloc: 8-bit samples only");
    return MRAID_ERR_UNSUPPORTED;
  }
  if (!d_data || !d_corr) {
    set_error("mraid_ccm_noalloc: d_data and d_corr are required");
    return MRAID_ERR_INVALID_ARG;
  }
  if (sub0 < 0 || n_sub < 1 || (int64_t)sub0 + n_sub > p->n_sub) {
    set_error("mraid_ccm_noalloc: sub-integrations [%d, %lld) outside [0, %d)", sub0,
              (long long)sub0 + n_sub, p->n_sub);
    return MRAID_ERR_INVALID_ARG;
  }
  const int64_t psum = (int64_t)(p->n_beam + 1) * (p->n_beam + 2) / 2;
  const int64_t cells = (int64_t)n_sub * p->n_chan;
  const int64_t max_cells = (int64_t)((kNoAllocScratchBytes - kNoAllocHeader) / (8 * psum));
  if (cells > max_cells) {
    set_error("mraid_ccm_noalloc: %lld cells exceed the %lld that the fixed %zu-byte scratch "
              "holds for %d beams; pass fewer sub-integrations per call",
              (long long)cells, (long long)max_cells, kNoAllocScratchBytes, p->n_beam);
    return MRAID_ERR_INVALID_ARG;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  void* scratch = nullptr;
  st = scratch_address(dev, &scratch);
  if (st != MRAID_OK) return st;

  // A stack plan that owns nothing: it only carries sizes, the stream and
  // the scratch pointers to the existing launchers.
  mraid_plan_s tmp;
  tmp.p = *p;
  tmp.p.keep = nullptr;
  tmp.device = dev;
  tmp.stream = static_cast<cudaStream_t>(stream);
  tmp.n_cells = cells;
  tmp.beam_stride = p->beam_stride ? p->beam_stride : (int64_t)p->n_sub * p->n_samp_sub * p->n_chan;
  tmp.np = p->n_beam * (p->n_beam + 1) / 2;
  tmp.psum = (int)psum;
  tmp.d_degenerate = static_cast<unsigned long long*>(scratch);
  int64_t* sums = reinterpret_cast<int64_t*>(static_cast<unsigned char*>(scratch) + kNoAllocHeader);

  e = cudaMemsetAsync(tmp.d_degenerate, 0, sizeof(unsigned long long), tmp.stream);
  if (e != cudaSuccess) return cuda_fail(e, "mraid_ccm_noalloc memset");
  e = launch_gram_u8(&tmp, static_cast<const uint8_t*>(d_data), sub0, n_sub, sums);
  if (e != cudaSuccess) return cuda_fail(e, "mraid_ccm_noalloc gram launch");
  e = launch_corr_from_sums(&tmp, sums, cells, d_corr);
  if (e != cudaSuccess) return cuda_fail(e, "mraid_ccm_noalloc corr launch");
  return MRAID_OK;
}
