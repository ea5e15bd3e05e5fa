// refine.cu - eigenvector refinement of the mask: which beams an RFI cell
// affects (Section 3.3 last paragraph; eigenvector threshold multiple t,
// Section 4.5).
//
// For every beam b a Gaussian fit (mean, population sigma) to |q1_b| over
// the cells the eigenvalue mask left unflagged (and not preserved); a
// flagged cell marks beam b when |q1_b| > mu_b + t sigma_b. Three launches:
// per-block partial sums (FP32 over 256-cell chunks, folded into FP64), one
// block that combines them in a fixed order, and a per-cell bit writer.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace mraid {
namespace {

constexpr int kRefThreads = 128;  // one thread per beam (N <= 128)

__global__ void __launch_bounds__(kRefThreads)
refine_partials(const float* __restrict__ q1, const uint8_t* __restrict__ flags, int64_t n_cells,
                int n_chan, const uint8_t* __restrict__ keep, int n_beam, double* __restrict__ part) {
  const int b = threadIdx.x;
  const int64_t per = (n_cells + gridDim.x - 1) / gridDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * per;
  const int64_t c1 = min(n_cells, c0 + per);
  double cnt = 0.0, s1 = 0.0, s2 = 0.0;
  float f1 = 0.f, f2 = 0.f;
  int fc = 0;
  for (int64_t c = c0; c < c1; ++c) {
    const bool use = !flags[c] && !(keep && keep[(uint32_t)c % (uint32_t)n_chan]);
    if (use && b < n_beam) {
      const float v = fabsf(q1[c * n_beam + b]);
      f1 += v;
      f2 = fmaf(v, v, f2);
      ++fc;
    }
    if (fc == 256 || c + 1 == c1) {  // fold the FP32 chunk into FP64
      cnt += fc;
      s1 += f1;
      s2 += f2;
      f1 = f2 = 0.f;
      fc = 0;
    }
  }
  if (b < n_beam) {
    double* o = part + ((size_t)blockIdx.x * n_beam + b) * 3;
    o[0] = cnt;
    o[1] = s1;
    o[2] = s2;
  }
}

__global__ void __launch_bounds__(kRefThreads)
refine_finalize(const double* __restrict__ part, int blocks, int n_beam, double t,
                double* __restrict__ mu_sigma, float* __restrict__ thresh) {
  const int b = threadIdx.x;
  if (b >= n_beam) return;
  double cnt = 0.0, s1 = 0.0, s2 = 0.0;
  for (int k = 0; k < blocks; ++k) {  // fixed order: deterministic
    const double* o = part + ((size_t)k * n_beam + b) * 3;
    cnt += o[0];
    s1 += o[1];
    s2 += o[2];
  }
  const double mu = cnt > 0.0 ? s1 / cnt : 0.0;
  const double sg = cnt > 0.0 ? sqrt(fmax(s2 / cnt - mu * mu, 0.0)) : 0.0;
  mu_sigma[2 * b] = mu;
  mu_sigma[2 * b + 1] = sg;
  thresh[b] = (float)(mu + t * sg);
}

__global__ void refine_bits(const float* __restrict__ q1, const uint8_t* __restrict__ flags,
                            int64_t n_cells, int n_beam, const float* __restrict__ thresh,
                            uint32_t* __restrict__ bits) {
  __shared__ float th[128];
  for (int b = threadIdx.x; b < n_beam; b += blockDim.x) th[b] = thresh[b];
  __syncthreads();
  const int W = (n_beam + 31) / 32;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells;
       c += (int64_t)gridDim.x * blockDim.x) {
    const bool f = flags[c] != 0;
    for (int w = 0; w < W; ++w) {
      uint32_t word = 0;
      if (f) {
        for (int k = 0; k < 32 && 32 * w + k < n_beam; ++k) {
          const int b = 32 * w + k;
          if (fabsf(q1[c * n_beam + b]) > th[b]) word |= 1u << k;
        }
      }
      bits[c * W + w] = word;
    }
  }
}

}  // namespace

cudaError_t launch_refine(mraid_plan_s* pl, const float* d_q1, const uint8_t* d_flags,
                          uint32_t* d_bits, double* d_mu_sigma) {
  const int blocks = pl->sm_count;
  refine_partials<<<blocks, kRefThreads, 0, pl->stream>>>(d_q1, d_flags, pl->n_cells, pl->p.n_chan,
                                                          pl->d_keep, pl->p.n_beam, pl->d_refine_part);
  refine_finalize<<<1, kRefThreads, 0, pl->stream>>>(pl->d_refine_part, blocks, pl->p.n_beam,
                                                      pl->p.vec_t, d_mu_sigma, pl->d_refine_thresh);
  const int64_t g = (pl->n_cells + 255) / 256;
  refine_bits<<<(unsigned)(g < (int64_t)pl->sm_count * 16 ? g : (int64_t)pl->sm_count * 16), 256, 0,
                pl->stream>>>(d_q1, d_flags, pl->n_cells, pl->p.n_beam, pl->d_refine_thresh, d_bits);
  return cudaGetLastError();
}

}  // namespace mraid
