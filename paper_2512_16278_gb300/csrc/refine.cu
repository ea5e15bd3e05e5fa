// refine.cu - eigenvector refinement of the mask: which beams an RFI cell
// affects (Section 3.3 last paragraph; eigenvector threshold multiple t,
// Section 4.5).
//
// For every beam b a Gaussian fit (mean, population sigma) to |q1_b| over
// the cells the eigenvalue mask left unflagged (and not preserved); a
// flagged cell marks beam b when |q1_b| > mu_b + t sigma_b. Three launches:
// per-block partial sums (FP32 over 256-cell chunks, folded into FP64), one
// warp per beam that combines them in a fixed order, and a per-cell bit
// writer.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace mraid {
namespace {

constexpr int kRefThreads = 128;  // groups of one thread per beam (N <= 128)

// Per-block partial sums over a contiguous run of cells. The block's
// threads form G = blockDim / N groups of N (one thread per beam); group g
// takes every G-th cell of the run, so a group reads one cell's q1 row per
// step and G rows are in flight. Groups are combined in a fixed order.
__global__ void __launch_bounds__(kRefThreads)
refine_partials(const float* __restrict__ q1, const uint8_t* __restrict__ flags, int64_t n_cells,
                int n_chan, const uint8_t* __restrict__ keep, int n_beam, double* __restrict__ part) {
  __shared__ double red[kRefThreads * 3];
  const int G = blockDim.x / n_beam;  // >= 1 (n_beam <= 128)
  const int g = threadIdx.x / n_beam, b = threadIdx.x % n_beam;
  const int64_t per = (n_cells + gridDim.x - 1) / gridDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * per;
  const int64_t c1 = min(n_cells, c0 + per);
  double cnt = 0.0, s1 = 0.0, s2 = 0.0;
  if (g < G) {
    float f1 = 0.f, f2 = 0.f;
    int fc = 0;
#pragma unroll 4
    for (int64_t c = c0 + g; c < c1; c += G) {
      const bool use = !flags[c] && !(keep && keep[(uint32_t)c % (uint32_t)n_chan]);
      if (use) {
        const float v = fabsf(q1[c * n_beam + b]);
        f1 += v;
        f2 = fmaf(v, v, f2);
        ++fc;
      }
      if (fc == 256) {  // fold the FP32 chunk into FP64
        cnt += fc;
        s1 += f1;
        s2 += f2;
        f1 = f2 = 0.f;
        fc = 0;
      }
    }
    cnt += fc;
    s1 += f1;
    s2 += f2;
  }
  red[3 * threadIdx.x] = cnt;
  red[3 * threadIdx.x + 1] = s1;
  red[3 * threadIdx.x + 2] = s2;
  __syncthreads();
  if (threadIdx.x < n_beam) {
    double a = 0.0, x = 0.0, y = 0.0;
    for (int k = 0; k < G; ++k) {  // fixed order
      const double* r = red + 3 * (k * n_beam + threadIdx.x);
      a += r[0];
      x += r[1];
      y += r[2];
    }
    double* o = part + ((size_t)blockIdx.x * n_beam + threadIdx.x) * 3;
    o[0] = a;
    o[1] = x;
    o[2] = y;
  }
}

// One warp per beam (a block of one warp each): lane l sums the partials of
// blocks l, l + 32, ... in order, then a fixed shuffle tree; deterministic
// for a given block count.
__global__ void __launch_bounds__(kRefThreads)
refine_finalize(const double* __restrict__ part, int blocks, int n_beam, double t,
                double* __restrict__ mu_sigma, float* __restrict__ thresh) {
  const int lane = threadIdx.x & 31, warps = (blockDim.x >> 5) * gridDim.x;
  for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < n_beam; b += warps) {
    double cnt = 0.0, s1 = 0.0, s2 = 0.0;
    for (int k = lane; k < blocks; k += 32) {
      const double* o = part + ((size_t)k * n_beam + b) * 3;
      cnt += o[0];
      s1 += o[1];
      s2 += o[2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      const double mu = cnt > 0.0 ? s1 / cnt : 0.0;
      const double sg = cnt > 0.0 ? sqrt(fmax(s2 / cnt - mu * mu, 0.0)) : 0.0;
      mu_sigma[2 * b] = mu;
      mu_sigma[2 * b + 1] = sg;
      thresh[b] = (float)(mu + t * sg);
    }
  }
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
  int64_t want = (pl->n_cells + 255) / 256;
  const int blocks = (int)(want < kRefBlocks ? (want < 1 ? 1 : want) : kRefBlocks);
  refine_partials<<<blocks, kRefThreads, 0, pl->stream>>>(d_q1, d_flags, pl->n_cells, pl->p.n_chan,
                                                          pl->d_keep, pl->p.n_beam, pl->d_refine_part);
  refine_finalize<<<pl->p.n_beam, 32, 0, pl->stream>>>(pl->d_refine_part, blocks, pl->p.n_beam,
                                                      pl->p.vec_t, d_mu_sigma, pl->d_refine_thresh);
  const int64_t g = (pl->n_cells + 255) / 256;
  refine_bits<<<(unsigned)(g < (int64_t)pl->sm_count * 16 ? g : (int64_t)pl->sm_count * 16), 256, 0,
                pl->stream>>>(d_q1, d_flags, pl->n_cells, pl->p.n_beam, pl->d_refine_thresh, d_bits);
  return cudaGetLastError();
}

}  // namespace mraid
