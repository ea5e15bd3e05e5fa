// multires.cu - Gram sums of longer sub-intervals from shorter ones.
//
// Section 4.4 (Table 1, Fig. 7) runs the method at sub-interval lengths
// from 0.05 s to 10 s. The augmented Gram of Eq. 1 over a sub-interval made
// of m consecutive shorter ones is the sum of their Grams: every entry
// (sum x_a x_b, sum x_a, n) is a sum over samples, and int64 addition is
// exact, so the longer timescales cost no further pass over the samples.
// This kernel forms out[k] = sum_{j < m} in[k m + j] for every cell entry:
// a plain streaming reduction, coalesced along the (channel, entry) run of
// one sub-integration, bound by HBM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mraid {
namespace {

constexpr int kAggThreads = 256;

// per_sub: int64 entries of one sub-integration (n_chan * P); n_out_sub:
// output sub-intervals; m: input sub-integrations per output one.
template <int V>
__global__ void __launch_bounds__(kAggThreads)
gram_aggregate_kernel(const int64_t* __restrict__ src, int64_t* __restrict__ dst,
                      int64_t per_sub, int n_out_sub, int m) {
  const int64_t per_vec = per_sub / V;
  const int64_t n_out = per_vec * n_out_sub;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += stride) {
    const int64_t k = o / per_vec, e = o - k * per_vec;
    const int64_t* s = src + (k * m * per_vec + e) * V;
    if (V == 2) {
      longlong2 acc = make_longlong2(0, 0);
      for (int j = 0; j < m; ++j) {
        const longlong2 v = *reinterpret_cast<const longlong2*>(s + (int64_t)j * per_sub);
        acc.x += v.x;
        acc.y += v.y;
      }
      *reinterpret_cast<longlong2*>(dst + o * V) = acc;
    } else {
      int64_t acc = 0;
      for (int j = 0; j < m; ++j) acc += s[(int64_t)j * per_sub];
      dst[o] = acc;
    }
  }
}

}  // namespace

cudaError_t launch_gram_aggregate(const mraid_plan_s* pl, const int64_t* d_src, int64_t* d_dst,
                                  int n_out_sub, int m) {
  const int64_t per_sub = (int64_t)pl->p.n_chan * pl->psum;
  const bool vec2 = per_sub % 2 == 0 && (reinterpret_cast<uintptr_t>(d_src) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(d_dst) & 15) == 0;
  const int64_t n_out = per_sub / (vec2 ? 2 : 1) * n_out_sub;
  if (n_out <= 0) return cudaSuccess;
  int64_t blocks = (n_out + kAggThreads - 1) / kAggThreads;
  const int64_t cap = (int64_t)pl->sm_count * 8;  // 8 resident blocks per SM
  if (blocks > cap) blocks = cap;
  if (vec2)
    gram_aggregate_kernel<2><<<(unsigned)blocks, kAggThreads, 0, pl->stream>>>(d_src, d_dst, per_sub,
                                                                              n_out_sub, m);
  else
    gram_aggregate_kernel<1><<<(unsigned)blocks, kAggThreads, 0, pl->stream>>>(d_src, d_dst, per_sub,
                                                                              n_out_sub, m);
  return cudaGetLastError();
}

}  // namespace mraid
