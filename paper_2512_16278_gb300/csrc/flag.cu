// flag.cu - iterative Gaussian-fit masking of the normalised dominant
// eigenvalue (Section 3.3 masking paragraph; threshold multiple k from
// Section 4.5; preserved channels from Section 4.3).
//
// One cooperative launch runs the whole iteration on the device: every pass
// masks the cells above the previous threshold, reduces (count, sum s,
// sum s^2) over the cells still unmasked and unpreserved (per thread in
// FP32 over its ~10 cells, then in FP64; the per-cell tests are FP32 and
// decide exactly as FP64 would), and
// derives mu, sigma (population) and mu + k sigma. The fit stops when a
// pass masks nothing new (the unmasked count is unchanged) or after
// max_clip_iter fits. Block partial sums are combined in a fixed order by
// every block, so the result is deterministic.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace mraid {
namespace {

constexpr int kFlagThreads = 512;

struct FlagArgs {
  const float* stat;
  int64_t n_cells;
  int n_chan;
  const uint8_t* keep;  // device [n_chan] or nullptr
  double k_sigma;
  int max_iter;
  uint8_t* flags;
  double* partials;     // [2][gridDim.x][3]
  mraid_flag_info* info;
};

// Block totals of (a, b, c): a fixed shuffle tree per warp, then the warps'
// totals in a fixed order. Only thread 0 receives the block totals (it alone
// publishes them); the other threads skip that FP64 loop, which GB300 would
// otherwise issue once per warp at a small fraction of the FP32 rate.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x / 32, nw = blockDim.x / 32;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[3 * w] = a;
    red[3 * w + 1] = b;
    red[3 * w + 2] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = c = 0.0;
    for (int i = 0; i < nw; ++i) {  // fixed order
      a += red[3 * i];
      b += red[3 * i + 1];
      c += red[3 * i + 2];
    }
  }
}

// Sum of the per-block partials [nb][3] in a fixed order: lane l takes
// blocks l, l+32, ... sequentially, then a fixed shuffle tree; every block
// computes the same bits. Result broadcast through shared memory.
__device__ __forceinline__ void grid_total3(const double* part, int nb, double* bcast, double& a,
                                            double& b, double& c) {
  if (threadIdx.x < 32) {
    double x = 0.0, y = 0.0, z = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) {
      x += part[3 * i];
      y += part[3 * i + 1];
      z += part[3 * i + 2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
      z += __shfl_xor_sync(0xffffffffu, z, o);
    }
    if (threadIdx.x == 0) {
      bcast[0] = x;
      bcast[1] = y;
      bcast[2] = z;
    }
  }
  __syncthreads();
  a = bcast[0];
  b = bcast[1];
  c = bcast[2];
  __syncthreads();
}

// Unroll of the per-cell loop: a thread issues the loads of kFlagUnroll
// cells before it uses them (and before any store), in its usual cell order.
constexpr int kFlagUnroll = 4;

__global__ void __launch_bounds__(kFlagThreads) flag_kernel(FlagArgs f) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double red[3 * (kFlagThreads / 32)];
  __shared__ double bcast[3];
  // the fit's state, kept by thread 0: mu, sigma, cells used, previous count
  __shared__ double fit_state[4];
  __shared__ double fit_thresh;
  __shared__ int fit_stop;
  const float* __restrict__ stat = f.stat;
  uint8_t* __restrict__ flags = f.flags;
  const uint8_t* __restrict__ keep = f.keep;
  const int64_t n = f.n_cells;
  const uint32_t n_chan = (uint32_t)f.n_chan;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += nthr) flags[i] = 0;

  double thresh = INFINITY;
  int fits = 0, converged = 0;
  if (threadIdx.x == 0) {
    fit_state[0] = 0.0;   // mu
    fit_state[1] = 0.0;   // sigma
    fit_state[2] = 0.0;   // cells in the last fit
    fit_state[3] = -1.0;  // unmasked count of the last fit
  }
  for (int pass = 0;; ++pass) {
    // The mask test v > thresh for a float v equals v > tf with tf the
    // largest float <= thresh: no float lies in (tf, thresh]. So the cells
    // need no FP64 (GB300 runs it at a small fraction of the FP32 rate).
    const float tf = __double2float_rd(thresh);
    // a thread's few cells sum in FP32 in a fixed order; blocks and the
    // grid combine in FP64, fixed order
    int cnt_t = 0;
    float s1_t = 0.f, s2_t = 0.f;
    for (int64_t i0 = tid; i0 < n; i0 += kFlagUnroll * nthr) {
      float v[kFlagUnroll];
      uint8_t m[kFlagUnroll];
#pragma unroll
      for (int u = 0; u < kFlagUnroll; ++u) {
        const int64_t i = i0 + u * nthr;
        const bool mine = i < n && !(keep && keep[(uint32_t)i % n_chan]);
        v[u] = mine ? stat[i] : 0.f;
        m[u] = mine ? flags[i] : (uint8_t)2;  // 2: past the end or preserved
      }
#pragma unroll
      for (int u = 0; u < kFlagUnroll; ++u) {
        if (m[u] == 0 && v[u] > tf) {
          m[u] = 1;
          flags[i0 + u * nthr] = 1;
        }
        if (m[u] == 0) {
          ++cnt_t;
          s1_t += v[u];
          s2_t = fmaf(v[u], v[u], s2_t);
        }
      }
    }
    double cnt = (double)cnt_t, s1 = (double)s1_t, s2 = (double)s2_t;
    block_sum3(cnt, s1, s2, red);
    double* part = f.partials + (size_t)(pass & 1) * gridDim.x * 3;
    if (threadIdx.x == 0) {
      part[3 * blockIdx.x] = cnt;
      part[3 * blockIdx.x + 1] = s1;
      part[3 * blockIdx.x + 2] = s2;
    }
    grid.sync();
    grid_total3(part, gridDim.x, bcast, cnt, s1, s2);
    // Thread 0 of every block makes the same decision and fit from the same
    // totals; its block takes the threshold and the decision from it. The
    // fit's state (fit_state, fits, converged) is thread 0's, and block 0's
    // thread 0 writes the report.
    if (threadIdx.x == 0) {
      int stop = 0;
      if (pass >= 1 && cnt == fit_state[3]) {  // the last threshold masked nothing
        converged = 1;
        stop = 1;
      } else if (fits == f.max_iter) {  // mask already holds max_iter markings
        stop = 1;
      } else if (cnt == 0.0) {  // nothing left to fit
        fit_state[0] = fit_state[1] = 0.0;
        thresh = INFINITY;
        fit_state[2] = 0.0;
        ++fits;
        converged = 1;
        stop = 1;
      } else {
        const double mu = s1 / cnt;
        const double sigma = sqrt(fmax(s2 / cnt - mu * mu, 0.0));
        thresh = mu + f.k_sigma * sigma;
        fit_state[0] = mu;
        fit_state[1] = sigma;
        fit_state[2] = cnt;
        fit_state[3] = cnt;
        ++fits;
      }
      fit_thresh = thresh;
      fit_stop = stop;
    }
    // the next pass writes these only after its own block barriers
    __syncthreads();
    thresh = fit_thresh;
    if (fit_stop) break;
  }
  // totals for the report. "Near" is |s - thresh| <= 2e-4 s, evaluated in
  // FP32 and redone in FP64 only within 1 % of the boundary: tfin is within
  // one float ulp (1.2e-7 relative) of thresh and the FP32 difference
  // carries a rounding error of the same order, far inside the 1 % band,
  // so every decision outside the band is the FP64 one.
  const float tfin = __double2float_rd(thresh);
  int nflag_t = 0, nnear_t = 0;
  for (int64_t i = tid; i < n; i += nthr) {
    nflag_t += flags[i];
    if (keep && keep[(uint32_t)i % n_chan]) continue;
    const float v = stat[i];
    const float a = fabsf(v - tfin), b = 2e-4f * v;
    bool near;
    if (!(b > 1e-30f) || fabsf(a - b) <= 1e-2f * b)
      near = fabs((double)v - thresh) <= 2e-4 * (double)v;
    else
      near = a < b;
    nnear_t += near;
  }
  double nflag = (double)nflag_t, nnear = (double)nnear_t, dummy = 0.0;
  block_sum3(nflag, nnear, dummy, red);
  grid.sync();  // everyone has read this pass's partials before they are reused
  double* part = f.partials;
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = nflag;
    part[3 * blockIdx.x + 1] = nnear;
    part[3 * blockIdx.x + 2] = 0.0;
  }
  grid.sync();
  if (blockIdx.x == 0) {
    double tf = 0.0, tn = 0.0, unused = 0.0;
    grid_total3(part, gridDim.x, bcast, tf, tn, unused);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double tf = bcast[0], tn = bcast[1];
    mraid_flag_info* o = f.info;
    o->mu = fit_state[0];
    o->sigma = fit_state[1];
    o->thresh = thresh;
    o->iterations = fits;
    o->converged = converged;
    o->n_flagged = (int64_t)tf;
    o->n_used = (int64_t)fit_state[2];
    o->n_near = (int64_t)tn;
  }
}

}  // namespace

int flag_grid_blocks(int device, int sm_count) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, flag_kernel, kFlagThreads, 0) !=
          cudaSuccess ||
      per_sm < 1)
    return 0;
  (void)device;
  return sm_count;  // one block per SM: fewer partials to combine
}

cudaError_t launch_flag(mraid_plan_s* pl, const float* d_stat, uint8_t* d_flags, int64_t n_cells,
                        mraid_flag_info* d_info) {
  FlagArgs f;
  f.stat = d_stat;
  f.n_cells = n_cells >= 0 ? n_cells : pl->n_cells;
  f.n_chan = pl->p.n_chan;
  f.keep = pl->d_keep;
  f.k_sigma = pl->p.eig_k;
  f.max_iter = pl->p.max_clip_iter;
  f.flags = d_flags;
  f.partials = pl->d_partials;
  f.info = d_info ? d_info : pl->d_info;
  // cooperative launch (all blocks co-resident for the grid barrier), in the
  // form that stream capture accepts
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl->flag_blocks);
  cfg.blockDim = dim3(kFlagThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = pl->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, flag_kernel, f);
}

}  // namespace mraid
