// bandpass.cu - Section 3.1 bandpass normalisation with ArPLS, and the CCM
// under the bandpass-centred reading of Eq. 1.
//
// For a fit interval of F sub-integrations the bandpass of beam a is its
// time-aggregated spectrum y_a(j), the mean of channel j over the
// interval's samples; here it comes exactly from the Gram sums already
// formed (sum of S_a over the interval's cells over the sum of their n).
// Its baseline z_a(j) is fitted over channels with ArPLS (asymmetrically
// reweighted penalized least squares; Baek, Park, Ahn and Ahn 2015, the
// method Section 3.1 names, with the lam / ratio / itermax parameters of
// Section 4.5): weights w start at 1; each step solves
// (W + lam D^T D) z = W y (D: second differences), takes the mean m and
// population deviation s of the negative residuals d = y - z, and moves to
// w_i = 1 / (1 + exp(2 (d_i - (2 s - m)) / s)) until the weights change by
// less than `ratio` (relative Euclidean norm) or itermax solves.
//
// The CCM of a cell about the bandpass is
//   C_ab = (1/n) sum_t (x_a - z_a)(x_b - z_b) = cov_ab / n^2 + d_a d_b,
// cov_ab = n S_ab - S_a S_b the exact int64 covariance numerator and
// d_a = S_a / n - z_a the cell mean's offset from the bandpass: no
// cancellation between large terms, so FP32 suffices for C.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace mraid {
namespace {

constexpr int kArThreads = 256;
constexpr int kArWarps = kArThreads / 32;
constexpr int kArArrays = 6;  // y, z, w, L[i][i-1], L[i][i-2], 1 / D_i

// Sum over the block in a fixed order; every thread gets the total.
__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < kArWarps; ++i) t += red[i];
  return t;
}

// Entries of D^T D for D the (n-2) x n second-difference matrix (rows
// 1, -2, 1): the contributions of the rows k that touch i.
__device__ __forceinline__ double dtd0(int i, int n) {  // (i, i)
  return (i >= 2 ? 1.0 : 0.0) + (i >= 1 && i - 1 <= n - 3 ? 4.0 : 0.0) + (i <= n - 3 ? 1.0 : 0.0);
}
__device__ __forceinline__ double dtd1(int i, int n) {  // (i, i + 1)
  return (i >= 1 && i - 1 <= n - 3 ? -2.0 : 0.0) + (i <= n - 3 ? -2.0 : 0.0);
}

struct ArplsArgs {
  const double* y;   // [sys][n]
  double* z;         // [sys][n]
  float* zf;         // [sys][n] float copy, or null
  int32_t* iters;    // [sys], or null
  double* work;      // [sys][6][n] when the arrays do not fit in shared memory
  int n, n_sys, itermax;
  double lam, ratio;
};

// One CTA per spectrum. Thread 0 factors and solves the pentadiagonal
// system (a sequential recurrence) from shared memory; all threads share
// the residual statistics and the reweighting.
__global__ void __launch_bounds__(kArThreads) arpls_kernel(ArplsArgs g) {
  extern __shared__ double ar_sm[];
  __shared__ double red[kArWarps];
  __shared__ int bad;
  const int sys = blockIdx.x, n = g.n;
  double* base = g.work ? g.work + (size_t)sys * kArArrays * n : ar_sm;
  double* ys = base;
  double* zs = ys + n;
  double* w = zs + n;
  double* l1 = w + n;   // L[i][i-1]; reused for the new weights
  double* l2 = l1 + n;  // L[i][i-2]
  double* idg = l2 + n;
  const double* y = g.y + (size_t)sys * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    ys[i] = y[i];
    w[i] = 1.0;
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const double lam = g.lam;
  int solves = 0;
  while (solves < g.itermax) {
    if (threadIdx.x == 0) {
      // A = W + lam D^T D = L diag(D) L^T; forward substitution L u = W y
      // along the factorisation (u kept in zs), then L^T z = u / D.
      double dm1 = 1.0, dm2 = 1.0, l1m1 = 0.0, um1 = 0.0, um2 = 0.0;
      for (int i = 0; i < n; ++i) {
        const double a0 = w[i] + lam * dtd0(i, n);
        double li2 = 0.0, li1 = 0.0;
        if (i >= 2) li2 = lam / dm2;  // A[i][i-2] = lam
        if (i >= 1) li1 = (lam * dtd1(i - 1, n) - li2 * dm2 * l1m1) / dm1;
        double di = a0;
        if (i >= 1) di -= li1 * li1 * dm1;
        if (i >= 2) di -= li2 * li2 * dm2;
        if (!(di > 0.0)) {
          bad = 1;
          break;
        }
        const double ui = w[i] * ys[i] - li1 * um1 - li2 * um2;
        l1[i] = li1;
        l2[i] = li2;
        idg[i] = 1.0 / di;
        zs[i] = ui;
        dm2 = dm1;
        dm1 = di;
        l1m1 = li1;
        um2 = um1;
        um1 = ui;
      }
      if (!bad) {
        double zp1 = 0.0, zp2 = 0.0;
        for (int i = n - 1; i >= 0; --i) {
          double zi = zs[i] * idg[i];
          if (i + 1 < n) zi -= l1[i + 1] * zp1;
          if (i + 2 < n) zi -= l2[i + 2] * zp2;
          zs[i] = zi;
          zp2 = zp1;
          zp1 = zi;
        }
      }
    }
    __syncthreads();
    if (bad) break;
    ++solves;
    // mean and population deviation of the negative residuals
    double sn = 0.0, cn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double d = ys[i] - zs[i];
      if (d < 0.0) {
        sn += d;
        cn += 1.0;
      }
    }
    sn = block_sum(sn, red);
    cn = block_sum(cn, red);
    if (cn == 0.0) break;
    const double m = sn / cn;
    double s2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double d = ys[i] - zs[i];
      if (d < 0.0) s2 += (d - m) * (d - m);
    }
    const double s = sqrt(block_sum(s2, red) / cn);
    if (!(s > 0.0)) break;
    // new weights (into l1) and how far they moved
    const double thr = 2.0 * s - m;
    double dw2 = 0.0, w2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double d = ys[i] - zs[i];
      const double wt = 1.0 / (1.0 + exp(2.0 * (d - thr) / s));
      dw2 += (w[i] - wt) * (w[i] - wt);
      w2 += w[i] * w[i];
      l1[i] = wt;
    }
    dw2 = block_sum(dw2, red);
    w2 = block_sum(w2, red);
    if (sqrt(dw2) / sqrt(w2) < g.ratio) break;
    for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = l1[i];
    __syncthreads();
  }
  __syncthreads();
  double* z = g.z + (size_t)sys * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    z[i] = zs[i];
    if (g.zf) g.zf[(size_t)sys * n + i] = (float)zs[i];
  }
  if (threadIdx.x == 0 && g.iters) g.iters[sys] = bad ? -1 : solves;
}

// y[(I * N + a) * n_chan + j]: mean of beam a, channel j over interval I,
// from the Gram sums (public [cell][P] or interleaved [cell/8][P][8]).
__global__ void bandpass_input_kernel(const int64_t* __restrict__ sums, int interleaved,
                                      int n_beam, int n_chan, int n_sub, int interval, int psum,
                                      double* __restrict__ y, int64_t total) {
  const int N1 = n_beam + 1;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx % n_chan);
    const int64_t ia = idx / n_chan;
    const int a = (int)(ia % n_beam);
    const int I = (int)(ia / n_beam);
    const int e_sa = a * N1 - a * (a - 1) / 2 + (n_beam - a);  // S_a
    const int e_n = psum - 1;                                   // n
    const int k0 = I * interval;
    const int k1 = k0 + interval < n_sub ? k0 + interval : n_sub;
    int64_t s = 0, nn = 0;
    for (int k = k0; k < k1; ++k) {
      const int64_t cell = (int64_t)k * n_chan + j;
      const int64_t* src = interleaved ? sums + (cell >> 3) * psum * 8 + (cell & 7) : sums + cell * psum;
      const int step = interleaved ? 8 : 1;
      s += src[(int64_t)e_sa * step];
      nn += src[(int64_t)e_n * step];
    }
    y[idx] = (double)s / (double)nn;
  }
}

// One warp per cell: C_ab = cov_ab / n^2 + d_a d_b, packed upper triangle.
__global__ void ccm_bandpass_kernel(const int64_t* __restrict__ sums, int interleaved,
                                    int64_t n_cells, int n_beam, int n_chan, int interval,
                                    int psum, int np, const double* __restrict__ z,
                                    float* __restrict__ ccm) {
  extern __shared__ unsigned char bp_raw[];
  const int warps = blockDim.x / 32;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  int64_t* S = reinterpret_cast<int64_t*>(bp_raw) + (size_t)warp * psum;
  float* dv = reinterpret_cast<float*>(reinterpret_cast<int64_t*>(bp_raw) + (size_t)warps * psum) +
              (size_t)warp * kMaxBeam;
  const int64_t cell = (int64_t)blockIdx.x * warps + warp;
  if (cell >= n_cells) return;
  const int N1 = n_beam + 1;
  if (interleaved) {
    const int64_t* src = sums + (cell >> 3) * psum * 8 + (cell & 7);
    for (int e = lane; e < psum; e += 32) S[e] = src[(int64_t)e * 8];
  } else {
    const int64_t* src = sums + cell * psum;
    for (int e = lane; e < psum; e += 32) S[e] = src[e];
  }
  __syncwarp();
  const int64_t n = S[psum - 1];
  const int k = (int)(cell / n_chan), j = (int)(cell % n_chan);
  const int I = k / interval;
  for (int a = lane; a < n_beam; a += 32) {
    const int64_t sa = S[a * N1 - a * (a - 1) / 2 + (n_beam - a)];
    dv[a] = (float)((double)sa / (double)n - z[((int64_t)I * n_beam + a) * n_chan + j]);
  }
  __syncwarp();
  const float inv_n2 = (float)(1.0 / ((double)n * (double)n));
  float* dst = ccm + cell * np;
  int a = 0, rowlen = n_beam, row_start = 0;
  for (int e = lane; e < np; e += 32) {
    while (e >= row_start + rowlen) {
      row_start += rowlen;
      --rowlen;
      ++a;
    }
    const int b = a + (e - row_start);
    const int64_t sa = S[a * N1 - a * (a - 1) / 2 + (n_beam - a)];
    const int64_t sb = S[b * N1 - b * (b - 1) / 2 + (n_beam - b)];
    const int64_t cov = n * S[a * N1 - a * (a - 1) / 2 + (b - a)] - sa * sb;
    dst[e] = fmaf(dv[a], dv[b], (float)cov * inv_n2);
  }
}

}  // namespace

size_t arpls_smem_bytes(int n) {
  const size_t b = (size_t)kArArrays * n * sizeof(double);
  return b <= 200 * 1024 ? b : 0;  // 0: the arrays live in global memory
}

size_t arpls_work_doubles(int n, int n_sys) {
  return arpls_smem_bytes(n) ? 0 : (size_t)kArArrays * n * n_sys;
}

cudaError_t launch_arpls(const mraid_plan_s* pl, const double* d_y, int n_sys, int n, double lam,
                         double ratio, int itermax, double* d_z, float* d_zf, int32_t* d_iters,
                         double* d_work) {
  if (n_sys <= 0) return cudaSuccess;
  ArplsArgs g;
  g.y = d_y;
  g.z = d_z;
  g.zf = d_zf;
  g.iters = d_iters;
  g.n = n;
  g.n_sys = n_sys;
  g.itermax = itermax;
  g.lam = lam;
  g.ratio = ratio;
  const size_t smem = arpls_smem_bytes(n);
  g.work = smem ? nullptr : d_work;
  if (!smem && !d_work) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(arpls_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  arpls_kernel<<<n_sys, kArThreads, smem, pl->stream>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_bandpass_input(const mraid_plan_s* pl, const int64_t* d_sums, bool interleaved,
                                  int interval, double* d_y) {
  const int n_int = (pl->p.n_sub + interval - 1) / interval;
  const int64_t total = (int64_t)n_int * pl->p.n_beam * pl->p.n_chan;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)pl->sm_count * 16) blocks = (int64_t)pl->sm_count * 16;
  if (blocks < 1) return cudaSuccess;
  bandpass_input_kernel<<<(unsigned)blocks, 256, 0, pl->stream>>>(
      d_sums, interleaved ? 1 : 0, pl->p.n_beam, pl->p.n_chan, pl->p.n_sub, interval, pl->psum,
      d_y, total);
  return cudaGetLastError();
}

cudaError_t launch_ccm_bandpass(const mraid_plan_s* pl, const int64_t* d_sums, bool interleaved,
                                int interval, const double* d_z, float* d_ccm) {
  const int psum = pl->psum;
  int warps = (int)(40960 / ((size_t)psum * 8 + kMaxBeam * 4));
  warps = warps < 1 ? 1 : (warps > 8 ? 8 : warps);
  const size_t smem = (size_t)warps * ((size_t)psum * 8 + kMaxBeam * 4);
  cudaError_t e = cudaFuncSetAttribute(ccm_bandpass_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (pl->n_cells + warps - 1) / warps;
  if (blocks > 0)
    ccm_bandpass_kernel<<<(unsigned)blocks, warps * 32, smem, pl->stream>>>(
        d_sums, interleaved ? 1 : 0, pl->n_cells, pl->p.n_beam, pl->p.n_chan, interval, psum,
        pl->np, d_z, d_ccm);
  return cudaGetLastError();
}

}  // namespace mraid
