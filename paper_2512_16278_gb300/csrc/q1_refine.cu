// q1_refine.cu - the FP64 final step of q1 on near-degenerate spectra.
//
// Section 3.3, Eq. 2 keeps, per cell, the unit eigenvector q1 of the
// largest eigenvalue. The FP32 eigensolvers fix q1 to about
// eps_32 ||r|| / (lambda_1 - lambda_2): well inside 1e-3 per element while
// the relative gap g = (lambda_1 - lambda_2) / lambda_1 is at least gap_hi
// (2e-3; 1e-2 behind the one-thread Jacobi solvers, whose lambda_1 and hence
// inverse-iteration shift are coarser), but not below it, where the first
// and second eigenvectors mix. For cells with kGapLo <= g < gap_hi this pass
// settles the mixing in FP64 on the same correlation matrix (its FP32
// entries are exact in FP64):
//   1. a plane holding q1 and q2: B = sigma I - r with sigma = lambda_1 +
//      delta just above lambda_1 (positive definite, smallest eigenvalues
//      delta and delta + lambda_1 - lambda_2), its FP32 Cholesky factor (a
//      pivot <= 0 means sigma fell below lambda_1: delta grows 4-fold and
//      the factor is redone), and x_s = B^-1 x_{s-1} / ||.|| three times
//      from x_0 = the FP32 q1. Each solve scales the q1 and q2 components by
//      1 / delta and 1 / (delta + lambda_1 - lambda_2) and every other one by
//      at most 1 / (delta + lambda_1 - lambda_3), far less, so span{x_2, x_3}
//      holds q1 and q2 whatever split of the two the FP32 solver returned
//      (at tiny gaps it can return mostly q2). The FP32 factor tilts that
//      plane by only ~eps_32 ||r|| / (lambda_2 - lambda_3), which does not
//      grow as lambda_1 - lambda_2 shrinks;
//   2. Rayleigh-Ritz on the plane in FP64: an orthonormal basis V (Gram-
//      Schmidt applied twice: the two vectors are nearly parallel), the 2x2
//      matrix V^T r V, and q1 = V y for its larger eigenvalue. Within the
//      plane the split of q1 and q2 is exact, so the small gap no longer
//      costs accuracy. The sign rule is applied last.
// The eigenvalues and the statistic are left as the FP32 solver wrote them
// (they already meet their bound); only q1 changes. Cells with g < kGapLo
// are degenerate to FP32 resolution (every vector of the cluster is an
// eigenvector of the rounded matrix) and keep the FP32 q1.
//
// FP64 pipes are few on this part (a warp-wide FP64 instruction holds one
// for many cycles): an all-FP64 factor and solves measured ~0.16 ms for the
// ~2000 selected cells of a 19-beam block, bound by the FP64 pipe, so only
// the step that needs the precision, the Ritz problem, runs in FP64. The
// selected cells are a small fraction of a block (~0.2 % of noise cells have
// g < 2e-3): a first kernel lists them, a second gives each listed cell its
// own warp, the factor in shared memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace mraid {
namespace {

constexpr float kGapLo = 1e-6f;
constexpr int kSolves = 3;
constexpr int kAttempts = 6;
constexpr int kRefineMaxWarps = 8;

// per warp: FP64 basis v1, v2 [N]; FP32 factor B [N][N + 1] (odd row
// stride), inverse pivots, current and previous vectors [N]; rounded up to
// 16 bytes so every warp's doubles stay aligned
__host__ __device__ inline size_t refine_warp_bytes(int N) {
  return (16 * (size_t)N + 4 * ((size_t)N * (N + 1) + 3 * (size_t)N) + 15) & ~(size_t)15;
}
// the (i, j) pairs of the lower triangle with j >= 1, ordered by j
// descending: the trailing triangle after pivot k (j > k) is the first
// m (m + 1) / 2 entries, m = N - 1 - k
__host__ __device__ inline size_t refine_table_entries(int N) {
  return (size_t)N * (N - 1) / 2;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 1 / sqrt(p) for p > 0 to FP64 precision: an FP32 estimate refined by two
// Newton steps r <- r (3 - p r^2) / 2 (each doubles the correct bits).
__device__ __forceinline__ double rsqrt64(double p) {
  double r = (double)rsqrtf((float)p);
  r = r * fma(-0.5 * p, r * r, 1.5);
  r = r * fma(-0.5 * p, r * r, 1.5);
  return r;
}

// Factor B = sigma I - r in FP32 (lower triangle, in place; inverse pivots
// in dinv); false if a pivot is not positive (all lanes agree).
__device__ bool load_and_factor(float* B, float* dinv, int N, const float* __restrict__ rp,
                                float sigma, const uint16_t* tab, int lane) {
  const int S = N + 1;
  int off = 0;  // packed offset of row a
  for (int a = 0; a < N; ++a) {
    for (int b = a + lane; b < N; b += 32) B[b * S + a] = (a == b ? sigma : 0.f) - rp[off + (b - a)];
    off += N - a;
  }
  __syncwarp();
  for (int k = 0; k < N; ++k) {
    const float pkk = B[k * S + k];
    if (!(pkk > 1e-30f)) return false;
    const float rk = rsqrtf(pkk);
    __syncwarp();
    if (lane == 0) {
      B[k * S + k] = pkk * rk;
      dinv[k] = rk;
    }
    for (int i = k + 1 + lane; i < N; i += 32) B[i * S + k] *= rk;
    __syncwarp();
    const int m = N - 1 - k;
    const int cnt = m * (m + 1) / 2;
    for (int e = lane; e < cnt; e += 32) {
      const int ij = tab[e];
      const int i = ij >> 8, j = ij & 255;
      B[i * S + j] = fmaf(-B[i * S + k], B[j * S + k], B[i * S + j]);
    }
    __syncwarp();
  }
  return true;
}

// x <- (L L^T)^-1 x in place (FP32), then normalised.
__device__ void solve_normalise(const float* B, const float* dinv, float* x, int N, int lane) {
  const int S = N + 1;
  for (int j = 0; j < N; ++j) {  // L z = x
    const float zj = x[j] * dinv[j];
    __syncwarp();
    if (lane == 0) x[j] = zj;
    for (int i = j + 1 + lane; i < N; i += 32) x[i] = fmaf(-B[i * S + j], zj, x[i]);
    __syncwarp();
  }
  for (int j = N - 1; j >= 0; --j) {  // L^T y = z
    const float yj = x[j] * dinv[j];
    __syncwarp();
    if (lane == 0) x[j] = yj;
    for (int i = lane; i < j; i += 32) x[i] = fmaf(-B[j * S + i], yj, x[i]);
    __syncwarp();
  }
  float nn = 0.f;
  for (int i = lane; i < N; i += 32) nn = fmaf(x[i], x[i], nn);
  nn = warp_sumf(nn);
  const float inv = nn > 0.f ? rsqrtf(nn) : 0.f;
  __syncwarp();
  for (int i = lane; i < N; i += 32) x[i] *= inv;
  __syncwarp();
}

// (r u)_i and (r v)_i for row i, r from the packed FP32 triangle
__device__ __forceinline__ void r_times(const float* __restrict__ rp, int N, int i,
                                        const double* u, const double* v, double& ru,
                                        double& rv) {
  ru = 0.0;
  rv = 0.0;
  for (int j = 0; j < N; ++j) {
    const int a = i < j ? i : j, b = i < j ? j : i;
    const double rij = (double)rp[a * N - a * (a - 1) / 2 + (b - a)];
    ru = fma(rij, u[j], ru);
    rv = fma(rij, v[j], rv);
  }
}

// The cells to refine: lane per cell, warp-aggregated appends to the list.
__global__ void q1_select_kernel(const float* __restrict__ evals, int64_t n_cells, int N,
                                 float gap_hi, uint32_t* __restrict__ list, int64_t list_cap,
                                 unsigned* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_cells;
       base += stride) {
    const int64_t cell = base + lane;
    bool near = false;
    if (cell < n_cells) {
      const float l1 = evals[cell * N];
      const float l2 = evals[cell * N + 1];
      const float gap = (l1 - l2) / l1;
      near = l1 > 0.f && gap >= kGapLo && gap < gap_hi;
    }
    const unsigned sel = __ballot_sync(0xffffffffu, near);
    if (!sel) continue;
    unsigned at = 0;
    if (lane == 0) at = atomicAdd(count, (unsigned)__popc(sel));
    at = __shfl_sync(0xffffffffu, at, 0);
    const int64_t slot = (int64_t)at + __popc(sel & ((1u << lane) - 1u));
    if (near && slot < list_cap) list[slot] = (uint32_t)cell;
  }
}

// One warp per listed cell.
__global__ void __launch_bounds__(32 * kRefineMaxWarps)
q1_refine_kernel(const float* __restrict__ corr, int64_t n_cells, int N,
                 const float* __restrict__ evals, float* __restrict__ q1,
                 const uint32_t* __restrict__ list, int64_t list_cap,
                 const unsigned* __restrict__ count, unsigned long long* __restrict__ refined) {
  extern __shared__ double rsm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warps = blockDim.x >> 5;
  unsigned char* wbase = reinterpret_cast<unsigned char*>(rsm) + (size_t)wib * refine_warp_bytes(N);
  uint16_t* tab = reinterpret_cast<uint16_t*>(reinterpret_cast<unsigned char*>(rsm) +
                                              (size_t)warps * refine_warp_bytes(N));
  {
    // row j from N - 1 down to 1, i = j .. N - 1 within each
    const int n_tab = (int)refine_table_entries(N);
    for (int e = threadIdx.x; e < n_tab; e += blockDim.x) {
      int j = N - 1, base = 0;
      while (e >= base + (N - j)) {
        base += N - j;
        --j;
      }
      const int i = j + (e - base);
      tab[e] = (uint16_t)((i << 8) | j);
    }
    __syncthreads();
  }
  double* v1 = reinterpret_cast<double*>(wbase);
  double* v2 = v1 + N;
  float* B = reinterpret_cast<float*>(v2 + N);
  float* dinv = B + (size_t)N * (N + 1);
  float* x = dinv + N;
  float* y = x + N;
  const int NP = N * (N + 1) / 2;
  const int64_t n_list = (int64_t)*count < list_cap ? (int64_t)*count : list_cap;
  for (int64_t w = (int64_t)blockIdx.x * warps + wib; w < n_list; w += (int64_t)gridDim.x * warps) {
    const int64_t cell = list[w];
    if (cell >= n_cells) continue;
    const float lambda1 = evals[cell * N];
    const float* rp = corr + cell * NP;
    float delta = 1e-5f * fabsf(lambda1);
    bool ok = false;
    for (int att = 0; att < kAttempts && !ok; ++att, delta *= 4.f)
      ok = load_and_factor(B, dinv, N, rp, lambda1 + delta, tab, lane);
    if (!ok) continue;  // keep the FP32 q1
    // x_0: the FP32 q1 (a fixed vector if it is not finite)
    bool finite = true;
    for (int i = lane; i < N; i += 32) {
      const float v = q1[cell * N + i];
      finite = finite && isfinite(v);
      x[i] = v;
    }
    finite = __all_sync(0xffffffffu, finite);
    __syncwarp();
    if (!finite)
      for (int i = lane; i < N; i += 32) x[i] = 1.f + 0.25f * (float)((i * 7) % 5);
    __syncwarp();
    for (int it = 0; it < kSolves; ++it) {
      if (it == kSolves - 1)  // keep x_{s-1} in y
        for (int i = lane; i < N; i += 32) y[i] = x[i];
      solve_normalise(B, dinv, x, N, lane);
    }
    // orthonormal FP64 basis of span{x_{s-1}, x_s}: v1 = x_s, v2 from x_{s-1}
    for (int i = lane; i < N; i += 32) {
      v1[i] = (double)x[i];
      v2[i] = (double)y[i];
    }
    __syncwarp();
    double nn1 = 0.0;
    for (int i = lane; i < N; i += 32) nn1 = fma(v1[i], v1[i], nn1);
    nn1 = warp_sum(nn1);
    const double s1 = rsqrt64(nn1);
    double c = 0.0;
    for (int i = lane; i < N; i += 32) {
      v1[i] *= s1;
      c = fma(v1[i], v2[i], c);
    }
    c = warp_sum(c);
    double n2 = 0.0;
    for (int i = lane; i < N; i += 32) {
      const double t = fma(-c, v1[i], v2[i]);
      v2[i] = t;
      n2 = fma(t, t, n2);
    }
    n2 = warp_sum(n2);
    __syncwarp();
    // else x_{s-1} and x_s are parallel to 1e-10 and q1 = x_s
    if (n2 > 1e-20) {
      // v2 - c v1 cancels most of v2, so its rounding leaves a component
      // along v1 of ~1e-16 / |v2 - c v1|: a second projection removes it (a
      // plane basis that is not orthogonal would tilt the Ritz vector)
      const double inv = rsqrt64(n2);
      double c2 = 0.0;
      for (int i = lane; i < N; i += 32) {
        v2[i] *= inv;
        c2 = fma(v1[i], v2[i], c2);
      }
      c2 = warp_sum(c2);
      double m2 = 0.0;
      for (int i = lane; i < N; i += 32) {
        const double t = fma(-c2, v1[i], v2[i]);
        v2[i] = t;
        m2 = fma(t, t, m2);
      }
      m2 = warp_sum(m2);
      const double inv2 = rsqrt64(m2);
      for (int i = lane; i < N; i += 32) v2[i] *= inv2;
      __syncwarp();
      // H = [v1 v2]^T r [v1 v2]
      double h11 = 0.0, h12 = 0.0, h22 = 0.0;
      for (int i = lane; i < N; i += 32) {
        double r1, r2;
        r_times(rp, N, i, v1, v2, r1, r2);
        h11 = fma(v1[i], r1, h11);
        h12 = fma(v1[i], r2, h12);
        h22 = fma(v2[i], r2, h22);
      }
      h11 = warp_sum(h11);
      h12 = warp_sum(h12);
      h22 = warp_sum(h22);
      // unit eigenvector (a, b) of the larger eigenvalue of [[h11 h12] [h12 h22]]
      const double hd = 0.5 * (h11 - h22);
      const double rad = sqrt(fma(hd, hd, h12 * h12));
      double a, b;
      if (hd >= 0.0) {  // theta - h22 = hd + rad >= rad: the better-conditioned form
        a = hd + rad;
        b = h12;
      } else {
        a = h12;
        b = rad - hd;
      }
      const double nab = fma(a, a, b * b);
      if (nab > 0.0) {
        const double s = rsqrt64(nab);
        a *= s;
        b *= s;
      } else {
        a = 1.0;
        b = 0.0;
      }
      __syncwarp();
      for (int i = lane; i < N; i += 32) v1[i] = fma(a, v1[i], b * v2[i]);
      __syncwarp();
    }
    // sign rule: largest magnitude positive, lowest index on ties
    double best = -1.0;
    int bi = N;
    for (int i = lane; i < N; i += 32) {
      const double mg = fabs(v1[i]);
      if (mg > best) {
        best = mg;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    const double sgn = v1[bi] < 0.0 ? -1.0 : 1.0;
    for (int i = lane; i < N; i += 32) q1[cell * N + i] = (float)(sgn * v1[i]);
    if (lane == 0 && refined) atomicAdd(refined, 1ull);
    __syncwarp();
  }
}

}  // namespace

float q1_refine_gap_hi(const mraid_plan_s* pl) {
  const int N = pl->p.n_beam;
  const bool reg = N == 2 || N == 3 || N == 4 || N == 13 || N == 19;
  return (reg && pl->eig_variant < 2) ? 1e-2f : 2e-3f;
}

cudaError_t launch_q1_refine(const mraid_plan_s* pl, const float* d_corr, int64_t n_cells,
                             const float* d_evals, float* d_q1, unsigned long long* d_count,
                             cudaStream_t stream) {
  const int N = pl->p.n_beam;
  if (n_cells <= 0 || !d_evals || !d_q1 || N < 2) return cudaSuccess;
  if (!pl->ws.q1_list || pl->ws.q1_list_cells < (size_t)n_cells) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(pl->ws.q1_list_n, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  {
    const int64_t want = (n_cells + 255) / 256;
    const int64_t cap = (int64_t)pl->sm_count * 8;
    q1_select_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, stream>>>(
        d_evals, n_cells, N, q1_refine_gap_hi(pl), pl->ws.q1_list,
        (int64_t)pl->ws.q1_list_cells, pl->ws.q1_list_n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t per_warp = refine_warp_bytes(N);
  int warps = (int)((48 * 1024) / per_warp);
  warps = warps < 1 ? 1 : (warps > kRefineMaxWarps ? kRefineMaxWarps : warps);
  const size_t smem = per_warp * warps + refine_table_entries(N) * sizeof(uint16_t);
  e = cudaFuncSetAttribute(q1_refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  // enough warps that a typical block's selected cells (~0.2 % of them)
  // get one warp each
  const int64_t blocks = (int64_t)pl->sm_count * (warps >= 4 ? 4 : 8);
  q1_refine_kernel<<<(unsigned)blocks, 32 * warps, smem, stream>>>(
      d_corr, n_cells, N, d_evals, d_q1, pl->ws.q1_list, (int64_t)pl->ws.q1_list_cells,
      pl->ws.q1_list_n, d_count);
  return cudaGetLastError();
}

}  // namespace mraid
