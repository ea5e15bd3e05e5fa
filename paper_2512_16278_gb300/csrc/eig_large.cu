// eig_large.cu - eigenvalues and q1 of larger correlation matrices (the
// 36- and 72-beam phased-array receivers, any N without a one-thread
// kernel), by reduction to tridiagonal form.
//
// Section 3.3, Eq. 2: C = Q Lambda Q^-1 per cell; eigenvalues largest first,
// s = lambda_1^2 / sum lambda_i^2, and the eigenvector q1 of lambda_1.
//
// Three passes:
//   1. one warp per matrix: Householder reduction r = Q T Q^T on the full
//      symmetric matrix in shared memory (row stride odd, so the lanes'
//      row accesses never share a bank); T (d, e) and the reflectors go to
//      a plan workspace;
//   2. one thread per matrix: every eigenvalue of T by implicit symmetric QR
//      steps with the Wilkinson shift (masked to the lowest unreduced block,
//      deflating from the bottom), the statistic, and the tridiagonal
//      eigenvector y of lambda_1 by inverse iteration (L D L^T of
//      sigma I - T, sigma just above lambda_1);
//   3. one warp per matrix: q1 = Q y with the stored reflectors, sign rule.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace mraid {
namespace {

constexpr int kRedWarps = 4;      // warps per block of pass 1 and pass 3
constexpr int kQrThreads = 64;    // threads per block of pass 2
constexpr int kMaxQrSteps = 32;   // QR steps per eigenvalue (cubic convergence)

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// sum over the LPM lanes of one matrix's group (LPM a power of two <= 32)
template <int LPM>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = LPM / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Offset of reflector k (length N-1-k) in a cell's packed reflector block.
__host__ __device__ __forceinline__ int64_t refl_off(int k, int N) {
  return (int64_t)k * (N - 1) - (int64_t)k * (k - 1) / 2;
}
// Reflector block per cell: the reflectors of steps 0..N-3, then their N-2
// scale factors beta.
__host__ __device__ __forceinline__ int64_t refl_floats(int N) {
  return N > 2 ? refl_off(N - 2, N) + (N - 2) : 1;
}
// Row stride of the full matrix in shared memory: a multiple of 4 floats
// (16-byte rows for vector accesses) with an odd quotient, so the rows of
// 8 consecutive lanes start in 8 different 4-bank groups and a warp's
// 16-byte accesses take the minimum 4 wavefronts.
__host__ __device__ __forceinline__ int row_stride(int N) {
  const int q = (N + 3) / 4;
  return 4 * ((q & 1) ? q : q + 1);
}

// ---------------------------------------------------------------- pass 1
// LPM lanes per matrix: 32, or 16 (two matrices per warp) where the
// trailing block has at most ~48 rows, so that fewer lanes sit idle in the
// row loops as the block shrinks.
template <int LPM>
__global__ void tri_reduce_kernel(const float* __restrict__ corr, int64_t n_cells, int N,
                                  float* __restrict__ de, float* __restrict__ refl) {
  extern __shared__ __align__(16) float rsm[];
  constexpr int MPW = 32 / LPM;  // matrices per warp
  const int lane32 = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int sub = lane32 / LPM, lane = lane32 % LPM;
  const int LD = row_stride(N);
  const int NP = N * (N + 1) / 2;
  float* A = rsm + ((size_t)w * MPW + sub) * ((size_t)N * LD + 2 * LD);
  float* V = A + (size_t)N * LD;   // current reflector, by absolute column (0 outside it)
  float* W = V + LD;               // p, then w = p - K v, by absolute column
  const uint32_t abase = static_cast<uint32_t>(__cvta_generic_to_shared(A));
  const int64_t RF = refl_floats(N);
  for (int64_t c0 = ((int64_t)blockIdx.x * nw + w) * MPW; c0 < n_cells;
       c0 += (int64_t)gridDim.x * nw * MPW) {
    // past the last cell a group repeats the warp's first matrix and writes nothing
    const bool valid = c0 + sub < n_cells;
    const int64_t cell = valid ? c0 + sub : c0;
    const float* src = corr + cell * NP;
    // packed upper triangle -> full symmetric matrix; padding columns zero
    for (int a = 0, off = 0; a < N; off += N - a, ++a)
      for (int b = a + lane; b < N; b += LPM) {
        cp_async4(abase + 4u * (uint32_t)(a * LD + b), src + off + (b - a));
        if (b != a) cp_async4(abase + 4u * (uint32_t)(b * LD + a), src + off + (b - a));
      }
    for (int a = 0; a < N; ++a)
      for (int b = N + lane; b < LD; b += LPM) A[a * LD + b] = 0.f;
    for (int j = lane; j < LD; j += LPM) V[j] = W[j] = 0.f;
    cp_async_wait_all();
    __syncwarp();
    float* dcell = de + cell * 2 * N;
    float* rcell = refl + cell * RF;
    for (int k = 0; k < N - 2; ++k) {
      const int m = N - 1 - k;
      const int j0 = (k + 1) & ~3;  // aligned start; V = W = 0 below column k + 1
      float s2 = 0.f;
      for (int i = lane; i < m; i += LPM) {
        const float x = A[(size_t)(k + 1 + i) * LD + k];
        s2 = fmaf(x, x, s2);
      }
      s2 = group_sum<LPM>(s2);
      const float x0 = A[(size_t)(k + 1) * LD + k];
      const float nx = sqrtf(s2);
      const float alpha = x0 >= 0.f ? -nx : nx;
      const float vtv = 2.f * nx * (nx + fabsf(x0));
      const bool reflect = vtv > 1e-30f;
      const float beta = reflect ? 2.f / vtv : 0.f;
      if (lane == 0) V[k] = 0.f;  // column k leaves the trailing block
      for (int i = lane; i < m; i += LPM) {
        const float v = i == 0 ? x0 - alpha : A[(size_t)(k + 1 + i) * LD + k];
        V[k + 1 + i] = v;
        if (valid) rcell[refl_off(k, N) + i] = v;
      }
      if (lane == 0 && valid) {
        rcell[refl_off(N - 2, N) + k] = beta;
        dcell[k] = A[(size_t)k * LD + k];
        dcell[N + k] = reflect ? alpha : x0;
      }
      __syncwarp();
      // p = beta A' v, one row per lane, 16-byte accesses
      for (int i = lane; i < m; i += LPM) {
        const float4* row = reinterpret_cast<const float4*>(A + (size_t)(k + 1 + i) * LD);
        const float4* v4 = reinterpret_cast<const float4*>(V);
        float a0 = 0.f, a1 = 0.f;
#pragma unroll 4
        for (int j = j0 >> 2; j < (LD >> 2); ++j) {
          const float4 r = row[j], v = v4[j];
          a0 = fmaf(r.x, v.x, a0);
          a1 = fmaf(r.y, v.y, a1);
          a0 = fmaf(r.z, v.z, a0);
          a1 = fmaf(r.w, v.w, a1);
        }
        W[k + 1 + i] = beta * (a0 + a1);
      }
      __syncwarp();
      float vp = 0.f;
      for (int i = lane; i < m; i += LPM) vp = fmaf(V[k + 1 + i], W[k + 1 + i], vp);
      const float kh = 0.5f * beta * group_sum<LPM>(vp);
      for (int i = lane; i < m; i += LPM) W[k + 1 + i] = fmaf(-kh, V[k + 1 + i], W[k + 1 + i]);
      __syncwarp();
      // A' -= v w^T + w v^T (columns below k + 1 see v = w = 0)
      for (int i = lane; i < m; i += LPM) {
        float4* row = reinterpret_cast<float4*>(A + (size_t)(k + 1 + i) * LD);
        const float4* v4 = reinterpret_cast<const float4*>(V);
        const float4* w4 = reinterpret_cast<const float4*>(W);
        const float vi = V[k + 1 + i], wi = W[k + 1 + i];
#pragma unroll 4
        for (int j = j0 >> 2; j < (LD >> 2); ++j) {
          float4 r = row[j];
          const float4 a = w4[j], b = v4[j];
          r.x = fmaf(-vi, a.x, fmaf(-wi, b.x, r.x));
          r.y = fmaf(-vi, a.y, fmaf(-wi, b.y, r.y));
          r.z = fmaf(-vi, a.z, fmaf(-wi, b.z, r.z));
          r.w = fmaf(-vi, a.w, fmaf(-wi, b.w, r.w));
          row[j] = r;
        }
      }
      __syncwarp();
      if (lane == 0) W[k] = 0.f;
    }
    if (lane == 0 && valid) {
      dcell[N - 2] = A[(size_t)(N - 2) * LD + (N - 2)];
      dcell[N - 1] = A[(size_t)(N - 1) * LD + (N - 1)];
      dcell[N + N - 2] = A[(size_t)(N - 2) * LD + (N - 1)];
      dcell[N + N - 1] = 0.f;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- pass 2
// One implicit QR step with the Wilkinson shift on the block [l, m] of the
// tridiagonal (d, e) held in this thread's shared-memory row.
__device__ void qr_step_mem(float* d, float* e, int l, int m) {
  const float dm1 = d[m - 1], dm = d[m], em = e[m - 1];
  const float dl = 0.5f * (dm1 - dm);
  const float r2s = fmaf(dl, dl, em * em);
  const float rr = r2s * rsqrtf(r2s);  // em != 0, so r2s > 0
  const float mu = dm - __fdividef(em * em, dl + (dl >= 0.f ? rr : -rr));
  // d[k] and e[k] of the current step travel in registers (each is
  // rewritten by the step before), so memory stays off the rotation chain
  float dk = d[l], ek = e[l];
  float x = dk - mu, z = ek;
  for (int k = l; k < m; ++k) {
    const float dk1 = d[k + 1];
    const float ek1 = (k < m - 1) ? e[k + 1] : 0.f;
    const float r2 = fmaf(x, x, z * z);
    const bool nz = r2 > 1e-37f;
    const float ri = nz ? rsqrtf(r2) : 0.f;
    const float c = nz ? x * ri : 1.f, s = nz ? z * ri : 0.f;
    if (k > l) e[k - 1] = r2 * ri;
    const float cc = c * c, ss = s * s, cs2 = 2.f * c * s * ek;
    d[k] = fmaf(cc, dk, fmaf(ss, dk1, cs2));
    const float dnext = fmaf(ss, dk, fmaf(cc, dk1, -cs2));
    const float ekn = fmaf(c * s, dk1 - dk, (cc - ss) * ek);
    if (k < m - 1) {
      z = s * ek1;
      ek = c * ek1;   // e[k+1] after this rotation: next step's e[k]
      e[k] = ekn;
    } else {
      e[k] = ekn;
      d[k + 1] = dnext;
    }
    dk = dnext;
    x = ekn;
  }
}

__global__ void __launch_bounds__(kQrThreads)
tri_qr_kernel(const float* __restrict__ de, int64_t n_cells, int N, float* __restrict__ evals,
              float* __restrict__ stat, float* __restrict__ y_out,
              unsigned long long* __restrict__ step_count) {
  extern __shared__ float qsm[];
  const int S = 4 * N + 1;  // odd row stride
  const int64_t cell = (int64_t)blockIdx.x * kQrThreads + threadIdx.x;
  const bool active = cell < n_cells;
  float* d = qsm + (size_t)threadIdx.x * S;
  float* e = d + N;
  float* td = e + N;  // T kept for the inverse iteration
  float* te = td + N;
  int steps = 0;
  if (active) {
    const float* src = de + cell * 2 * N;
    for (int i = 0; i < N; ++i) {
      d[i] = td[i] = src[i];
      e[i] = te[i] = src[N + i];
    }
    float an2 = 0.f;
    for (int i = 0; i < N; ++i) an2 = fmaf(d[i], d[i], fmaf(2.f * e[i], e[i], an2));
    const float thr2 = 1e-12f * an2;
    // |e| <= 1e-6 ||T||_F counts as zero (Weyl: eigenvalues move by less
    // than 1e-6 sqrt(N) lambda_max)
    for (int m = N - 1; m > 0;) {
      if (e[m - 1] * e[m - 1] <= thr2) {
        --m;
        continue;
      }
      int l = m - 1;
      while (l > 0 && e[l - 1] * e[l - 1] > thr2) --l;
      if (steps >= kMaxQrSteps * N) break;
      qr_step_mem(d, e, l, m);
      ++steps;
    }
    // descending order (insertion sort; N <= 128)
    for (int i = 1; i < N; ++i) {
      const float v = d[i];
      int j = i - 1;
      while (j >= 0 && d[j] < v) {
        d[j + 1] = d[j];
        --j;
      }
      d[j + 1] = v;
    }
    float ss = 0.f;
    for (int i = 0; i < N; ++i) ss = fmaf(d[i], d[i], ss);
    stat[cell] = ss > 0.f ? d[0] * d[0] / ss : 0.f;
    if (evals)
      for (int i = 0; i < N; ++i) evals[cell * N + i] = d[i];
  }
  if (step_count) {
    const unsigned ws = __reduce_add_sync(0xffffffffu, (unsigned)steps);
    const unsigned wm = __reduce_max_sync(0xffffffffu, (unsigned)steps);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&step_count[0], (unsigned long long)ws);
      atomicAdd(&step_count[1], (unsigned long long)wm);
    }
  }
  if (!active || !y_out) return;
  // inverse iteration on T: sigma I - T = L D L^T; d and e are free now
  // and hold 1/D and the subdiagonal of L
  const float lambda1 = d[0];
  float* dinv = d;
  float* lo = e;
  float delta = fmaxf(4e-5f * fabsf(lambda1), 1e-6f);
  bool ok = false;
  for (int attempt = 0; attempt < 4 && !ok; ++attempt, delta *= 16.f) {
    const float sig = lambda1 + delta;
    ok = true;
    float piv = sig - td[0];
    for (int i = 0; i < N; ++i) {
      if (i > 0) {
        const float l = -te[i - 1] * dinv[i - 1];
        lo[i] = l;
        piv = fmaf(-l * l, piv, sig - td[i]);
      }
      ok = ok && piv > 0.f;
      dinv[i] = __fdividef(1.f, fmaxf(piv, 1e-30f));
    }
  }
  float* y = td;  // T is no longer needed
  for (int i = 0; i < N; ++i) y[i] = 1.f + 0.25f * (float)((i * 7) % 5);
  for (int it = 0; it < 3; ++it) {
    for (int i = 1; i < N; ++i) y[i] = fmaf(-lo[i], y[i - 1], y[i]);
    for (int i = 0; i < N; ++i) y[i] *= dinv[i];
    for (int i = N - 2; i >= 0; --i) y[i] = fmaf(-lo[i + 1], y[i + 1], y[i]);
    float nn = 0.f;
    for (int i = 0; i < N; ++i) nn = fmaf(y[i], y[i], nn);
    const float inv = rsqrtf(fmaxf(nn, 1e-37f));
    for (int i = 0; i < N; ++i) y[i] *= inv;
  }
  const float bad = ok ? 0.f : __int_as_float(0x7fc00000);  // NaN marks a failed factor
  for (int i = 0; i < N; ++i) y_out[cell * N + i] = y[i] + bad;
}

// ---------------------------------------------------------------- pass 3
__global__ void __launch_bounds__(32 * kRedWarps)
tri_back_kernel(const float* __restrict__ refl, const float* __restrict__ y_in, int64_t n_cells,
                int N, float* __restrict__ q1) {
  extern __shared__ float bsm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* y = bsm + (size_t)w * N;
  const int64_t RF = refl_floats(N);
  for (int64_t cell = (int64_t)blockIdx.x * kRedWarps + w; cell < n_cells;
       cell += (int64_t)gridDim.x * kRedWarps) {
    for (int i = lane; i < N; i += 32) y[i] = y_in[cell * N + i];
    __syncwarp();
    const float* rc = refl + cell * RF;
    for (int k = N - 3; k >= 0; --k) {
      const int m = N - 1 - k;
      const float* v = rc + refl_off(k, N);
      float t = 0.f;
      for (int i = lane; i < m; i += 32) t = fmaf(v[i], y[k + 1 + i], t);
      t = warp_sum(t) * rc[refl_off(N - 2, N) + k];
      for (int i = lane; i < m; i += 32) y[k + 1 + i] = fmaf(-t, v[i], y[k + 1 + i]);
      __syncwarp();
    }
    // sign rule: largest magnitude positive, lowest index on ties
    float best = -1.f;
    int bi = N;
    for (int i = lane; i < N; i += 32) {
      const float a = fabsf(y[i]);
      if (a > best) {
        best = a;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    const float sgn = (bi < N && y[bi] < 0.f) ? -1.f : 1.f;
    for (int i = lane; i < N; i += 32) q1[cell * N + i] = sgn * y[i];
    __syncwarp();
  }
}

}  // namespace

size_t tri_workspace_floats(int n_beam) {
  return 2 * (size_t)n_beam + (size_t)refl_floats(n_beam) + (size_t)n_beam;
}

cudaError_t launch_eig_large(const mraid_plan_s* pl, const float* d_corr, int64_t n_cells,
                             float* d_evals, float* d_q1, float* d_stat, float* d_work,
                             cudaStream_t stream) {
  const int N = pl->p.n_beam;
  if (n_cells <= 0) return cudaSuccess;
  // workspace: [cell][2N] (d, e), then [cell][RF] reflectors, then [cell][N] y
  float* de = d_work;
  float* refl = de + (size_t)n_cells * 2 * N;
  float* y = refl + (size_t)n_cells * refl_floats(N);
  // pass 1: two matrices per warp up to 48 beams, else one; as many warps
  // per block (up to 4) as 200 KB of shared memory holds
  const int mpw = N <= 48 ? 2 : 1;
  const auto red = mpw == 2 ? tri_reduce_kernel<16> : tri_reduce_kernel<32>;
  const size_t per_warp =
      sizeof(float) * mpw * ((size_t)N * row_stride(N) + 2 * row_stride(N));
  int nw = (int)((200u << 10) / per_warp);
  nw = nw < 1 ? 1 : (nw > kRedWarps ? kRedWarps : nw);
  const size_t smem1 = per_warp * nw;
  cudaError_t e = cudaFuncSetAttribute(red, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
  if (e != cudaSuccess) return e;
  // one wave of resident blocks (they loop over the cells): a grid larger
  // than the GPU holds leaves a partial second wave
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, red, 32 * nw, smem1);
  if (e != cudaSuccess) return e;
  const int64_t wave1 = (int64_t)(per_sm > 0 ? per_sm : 1) * pl->sm_count;
  int64_t blocks = (n_cells + (int64_t)nw * mpw - 1) / ((int64_t)nw * mpw);
  if (blocks > wave1) blocks = wave1;
  red<<<(unsigned)blocks, 32 * nw, smem1, stream>>>(d_corr, n_cells, N, de, refl);
  const size_t smem2 = sizeof(float) * (size_t)kQrThreads * (4 * N + 1);
  e = cudaFuncSetAttribute(tri_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
  if (e != cudaSuccess) return e;
  const int64_t blocks2 = (n_cells + kQrThreads - 1) / kQrThreads;
  tri_qr_kernel<<<(unsigned)blocks2, kQrThreads, smem2, stream>>>(
      de, n_cells, N, d_evals, d_stat, d_q1 ? y : nullptr, pl->d_sweeps);
  if (d_q1) {
    const size_t smem3 = sizeof(float) * (size_t)kRedWarps * N;
    int per_sm3 = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm3, tri_back_kernel, 32 * kRedWarps,
                                                      smem3);
    if (e != cudaSuccess) return e;
    const int64_t wave3 = (int64_t)(per_sm3 > 0 ? per_sm3 : 1) * pl->sm_count;
    int64_t blocks3 = (n_cells + kRedWarps - 1) / kRedWarps;
    if (blocks3 > wave3) blocks3 = wave3;
    tri_back_kernel<<<(unsigned)blocks3, 32 * kRedWarps, smem3, stream>>>(refl, y, n_cells, N,
                                                                          d_q1);
  }
  return cudaGetLastError();
}

}  // namespace mraid
