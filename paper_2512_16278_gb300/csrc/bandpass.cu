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

constexpr int kArThreads = 512;
constexpr int kArWarps = kArThreads / 32;
constexpr int kCrArrays = 13;  // per block row: A (3), C (4), saved left coupling (4), F (2)

// Sum over the block in a fixed order; every thread gets the total.
__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll 8
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

struct M2 {  // [[a, b], [c, d]]
  double a, b, c, d;
};
__device__ __forceinline__ M2 mm(const M2& x, const M2& y) {
  return {fma(x.a, y.a, x.b * y.c), fma(x.a, y.b, x.b * y.d), fma(x.c, y.a, x.d * y.c),
          fma(x.c, y.b, x.d * y.d)};
}
__device__ __forceinline__ M2 tr(const M2& x) { return {x.a, x.c, x.b, x.d}; }

struct CrArrays {  // m block rows each
  double *aa, *ab, *ad;            // A_i = [[aa, ab], [ab, ad]]; the inverse once eliminated
  double *c00, *c01, *c10, *c11;   // C_i: coupling of row i to the next active row
  double *l00, *l01, *l10, *l11;   // left coupling of a row, saved when it is eliminated
  double *f0, *f1;                 // right side, then the solution
  __device__ CrArrays(double* p, int m)
      : aa(p), ab(p + m), ad(p + 2 * m), c00(p + 3 * m), c01(p + 4 * m), c10(p + 5 * m),
        c11(p + 6 * m), l00(p + 7 * m), l01(p + 8 * m), l10(p + 9 * m), l11(p + 10 * m),
        f0(p + 11 * m), f1(p + 12 * m) {}
  __device__ M2 C(int i) const { return {c00[i], c01[i], c10[i], c11[i]}; }
  __device__ M2 A(int i) const { return {aa[i], ab[i], ab[i], ad[i]}; }
};

// (W + lam D^T D) z = W y by block cyclic reduction. Unknowns in pairs
// X_i = (z_2i, z_2i+1) make the pentadiagonal matrix block tridiagonal with
// 2 x 2 blocks (row i: C_{i-1}^T X_{i-1} + A_i X_i + C_i X_{i+1}); m block
// rows, a power of two (rows past n are identity rows with no coupling).
// Each level eliminates the odd rows of the active set (stride s) into the
// even ones; then the single remaining row is solved and the eliminated
// rows are recovered level by level. It is Gaussian elimination of the
// symmetric positive definite matrix in an odd-even order, so it needs no
// pivoting, and every level is parallel over its rows.
__device__ void cr_solve(const CrArrays& r, int m, const double* w, const double* y, int n,
                         double lam) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int r0 = 2 * i, r1 = 2 * i + 1;
    const bool v0 = r0 < n, v1 = r1 < n;
    r.aa[i] = v0 ? w[r0] + lam * dtd0(r0, n) : 1.0;
    r.ab[i] = v1 ? lam * dtd1(r0, n) : 0.0;
    r.ad[i] = v1 ? w[r1] + lam * dtd0(r1, n) : 1.0;
    r.c00[i] = r0 + 2 < n ? lam : 0.0;                 // (r0, r0 + 2)
    r.c01[i] = 0.0;                                     // (r0, r0 + 3)
    r.c10[i] = r1 + 1 < n ? lam * dtd1(r1, n) : 0.0;    // (r1, r1 + 1)
    r.c11[i] = r1 + 2 < n ? lam : 0.0;                  // (r1, r1 + 2)
    r.f0[i] = v0 ? w[r0] * y[r0] : 0.0;
    r.f1[i] = v1 ? w[r1] * y[r1] : 0.0;
  }
  __syncthreads();
  for (int s = 1; s < m; s *= 2) {
    // rows leaving at this level: invert A_j, keep their left coupling
    for (int j = s + 2 * s * threadIdx.x; j < m; j += 2 * s * blockDim.x) {
      const double a = r.aa[j], b = r.ab[j], d = r.ad[j];
      const double inv = 1.0 / fma(a, d, -b * b);
      r.aa[j] = d * inv;
      r.ab[j] = -b * inv;
      r.ad[j] = a * inv;
      const M2 L = tr(r.C(j - s));
      r.l00[j] = L.a;
      r.l01[j] = L.b;
      r.l10[j] = L.c;
      r.l11[j] = L.d;
    }
    __syncthreads();
    // rows staying: take in both neighbours
    for (int i = 2 * s * threadIdx.x; i < m; i += 2 * s * blockDim.x) {
      M2 Ai = r.A(i);
      double g0 = r.f0[i], g1 = r.f1[i];
      if (i >= s) {
        const int j = i - s;
        const M2 Cj = r.C(j);
        M2 al = mm(tr(Cj), r.A(j));
        al = {-al.a, -al.b, -al.c, -al.d};
        const M2 t = mm(al, Cj);
        Ai = {Ai.a + t.a, Ai.b + t.b, Ai.c + t.c, Ai.d + t.d};
        g0 = fma(al.a, r.f0[j], fma(al.b, r.f1[j], g0));
        g1 = fma(al.c, r.f0[j], fma(al.d, r.f1[j], g1));
      }
      M2 Cn = {0.0, 0.0, 0.0, 0.0};
      if (i + s < m) {
        const int j = i + s;
        const M2 Ci = r.C(i);
        M2 ga = mm(Ci, r.A(j));
        ga = {-ga.a, -ga.b, -ga.c, -ga.d};
        const M2 t = mm(ga, tr(Ci));
        Ai = {Ai.a + t.a, Ai.b + t.b, Ai.c + t.c, Ai.d + t.d};
        g0 = fma(ga.a, r.f0[j], fma(ga.b, r.f1[j], g0));
        g1 = fma(ga.c, r.f0[j], fma(ga.d, r.f1[j], g1));
        Cn = mm(ga, r.C(j));
      }
      r.aa[i] = Ai.a;
      r.ab[i] = 0.5 * (Ai.b + Ai.c);
      r.ad[i] = Ai.d;
      r.c00[i] = Cn.a;
      r.c01[i] = Cn.b;
      r.c10[i] = Cn.c;
      r.c11[i] = Cn.d;
      r.f0[i] = g0;
      r.f1[i] = g1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double a = r.aa[0], b = r.ab[0], d = r.ad[0];
    const double inv = 1.0 / fma(a, d, -b * b);
    const double g0 = r.f0[0], g1 = r.f1[0];
    r.f0[0] = (d * g0 - b * g1) * inv;
    r.f1[0] = (a * g1 - b * g0) * inv;
  }
  __syncthreads();
  for (int s = m / 2; s >= 1; s /= 2) {
    for (int j = s + 2 * s * threadIdx.x; j < m; j += 2 * s * blockDim.x) {
      const double x0 = r.f0[j - s], x1 = r.f1[j - s];
      double g0 = r.f0[j] - fma(r.l00[j], x0, r.l01[j] * x1);
      double g1 = r.f1[j] - fma(r.l10[j], x0, r.l11[j] * x1);
      if (j + s < m) {
        const double y0 = r.f0[j + s], y1 = r.f1[j + s];
        g0 -= fma(r.c00[j], y0, r.c01[j] * y1);
        g1 -= fma(r.c10[j], y0, r.c11[j] * y1);
      }
      r.f0[j] = fma(r.aa[j], g0, r.ab[j] * g1);
      r.f1[j] = fma(r.ab[j], g0, r.ad[j] * g1);
    }
    __syncthreads();
  }
}

__host__ __device__ constexpr int cr_rows(int n) {  // block rows: a power of two >= n / 2
  int m = 1;
  while (2 * m < n) m *= 2;
  return m;
}

struct ArplsArgs {
  const double* y;   // [sys][n]
  double* z;         // [sys][n]
  float* zf;         // [sys][n] float copy, or null
  int32_t* iters;    // [sys], or null
  double* work;      // [sys][2][n] weights and new weights, then [sys][13 m] when the
                     // reduction arrays are not in shared memory
  int n, n_sys, itermax, in_smem;
  double lam, ratio;
};

// One CTA per spectrum: the weighted solves by block cyclic reduction,
// the residual statistics and the reweighting, all parallel over the CTA.
__global__ void __launch_bounds__(kArThreads, 1) arpls_kernel(ArplsArgs g) {
  extern __shared__ double ar_sm[];
  __shared__ double red[kArWarps];
  const int sys = blockIdx.x, n = g.n, m = cr_rows(n);
  double* w = g.work + (size_t)sys * 2 * n;
  double* wt = w + n;
  double* cr = g.in_smem ? ar_sm
                         : g.work + (size_t)g.n_sys * 2 * n + (size_t)sys * kCrArrays * m;
  const CrArrays r(cr, m);
  const double* y = g.y + (size_t)sys * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = 1.0;
  __syncthreads();
  int solves = 0;
  while (solves < g.itermax) {
    cr_solve(r, m, w, y, n, g.lam);
    ++solves;
    // z_i is f0 / f1 of block row i / 2
    double sn = 0.0, cn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double d = y[i] - ((i & 1) ? r.f1[i >> 1] : r.f0[i >> 1]);
      if (d < 0.0) {
        sn += d;
        cn += 1.0;
      }
    }
    sn = block_sum(sn, red);
    cn = block_sum(cn, red);
    if (cn == 0.0) break;
    const double mneg = sn / cn;
    double s2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double d = y[i] - ((i & 1) ? r.f1[i >> 1] : r.f0[i >> 1]);
      if (d < 0.0) s2 += (d - mneg) * (d - mneg);
    }
    const double sd = sqrt(block_sum(s2, red) / cn);
    if (!(sd > 0.0)) break;
    const double thr = 2.0 * sd - mneg;
    double dw2 = 0.0, w2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double d = y[i] - ((i & 1) ? r.f1[i >> 1] : r.f0[i >> 1]);
      const double wn = 1.0 / (1.0 + exp(2.0 * (d - thr) / sd));
      dw2 += (w[i] - wn) * (w[i] - wn);
      w2 += w[i] * w[i];
      wt[i] = wn;
    }
    dw2 = block_sum(dw2, red);
    w2 = block_sum(w2, red);
    if (sqrt(dw2) / sqrt(w2) < g.ratio) break;
    for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = wt[i];
    __syncthreads();
  }
  __syncthreads();
  double* z = g.z + (size_t)sys * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double zi = (i & 1) ? r.f1[i >> 1] : r.f0[i >> 1];
    z[i] = zi;
    if (g.zf) g.zf[(size_t)sys * n + i] = (float)zi;
  }
  if (threadIdx.x == 0 && g.iters) g.iters[sys] = solves;
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
  // FP32 throughout (this GPU's FP64 rate is low): S_a < 2^24 is exact
  // in float, and the offsets d_a are O(1), so rounding the mean and the
  // baseline to float costs ~1e-5 absolute in d_a, ~1e-7 of C
  const float inv_n = 1.f / (float)n;
  for (int a = lane; a < n_beam; a += 32) {
    const int64_t sa = S[a * N1 - a * (a - 1) / 2 + (n_beam - a)];
    dv[a] = fmaf((float)sa, inv_n, -(float)z[((int64_t)I * n_beam + a) * n_chan + j]);
  }
  __syncwarp();
  const float inv_n2 = inv_n * inv_n;
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
  const size_t b = (size_t)kCrArrays * cr_rows(n) * sizeof(double);
  return b <= 214 * 1024 ? b : 0;  // 0: the arrays live in global memory
}

size_t arpls_work_doubles(int n, int n_sys) {
  // the weights always; the reduction arrays when they are not in shared memory
  return (size_t)2 * n * n_sys +
         (arpls_smem_bytes(n) ? 0 : (size_t)kCrArrays * cr_rows(n) * n_sys);
}

cudaError_t launch_arpls(const mraid_plan_s* pl, const double* d_y, int n_sys, int n, double lam,
                         double ratio, int itermax, double* d_z, float* d_zf, int32_t* d_iters,
                         double* d_work) {
  if (n_sys <= 0) return cudaSuccess;
  if (!d_work) return cudaErrorInvalidValue;
  ArplsArgs g;
  g.y = d_y;
  g.z = d_z;
  g.zf = d_zf;
  g.iters = d_iters;
  g.work = d_work;
  g.n = n;
  g.n_sys = n_sys;
  g.itermax = itermax;
  g.lam = lam;
  g.ratio = ratio;
  const size_t smem = arpls_smem_bytes(n);
  g.in_smem = smem ? 1 : 0;
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

namespace mraid {
namespace {
mraid_status check_bandpass_params(const mraid_bandpass_params* bp) {
  if (!bp || !(bp->lam > 0.0) || !(bp->lam < 1e300) || !(bp->ratio > 0.0) || bp->itermax < 1 ||
      bp->itermax > 1000 || bp->interval < 1) {
    set_error("bandpass parameters: lam > 0, ratio > 0, itermax in 1..1000, interval >= 1");
    return MRAID_ERR_INVALID_ARG;
  }
  return MRAID_OK;
}

// ArPLS arrays in global memory for spectra too long for shared memory
mraid_status ensure_arpls_work(mraid_plan_s* pl, int n, int n_sys) {
  const size_t need = arpls_work_doubles(n, n_sys);
  if (need <= pl->ar_work_elems) return MRAID_OK;
  cudaFree(pl->ar_work);
  pl->ar_work = nullptr;
  pl->ar_work_elems = 0;
  cudaError_t e = cudaMalloc(&pl->ar_work, need * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "arpls work allocation");
  }
  pl->ar_work_elems = need;
  return MRAID_OK;
}
}  // namespace
}  // namespace mraid

// ---------------------------------------------------------------------------
// Entry points (include/mraid.h)

using namespace mraid;

void mraid_default_bandpass_params(mraid_bandpass_params* bp) {
  if (!bp) return;
  bp->lam = 1e5;
  bp->ratio = 1e-3;
  bp->itermax = 50;
  bp->interval = 20;
}

mraid_status mraid_arpls(mraid_plan_t pl, const double* d_y, int32_t n_sys, int32_t n,
                         const mraid_bandpass_params* bp, double* d_z, int32_t* d_iters) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  st = check_bandpass_params(bp);
  if (st != MRAID_OK) return st;
  if (!d_y || !d_z || n < 3 || n > (1 << 20) || n_sys < 0) {
    set_error("mraid_arpls: d_y and d_z are required, 3 <= n <= 2^20, n_sys >= 0");
    return MRAID_ERR_INVALID_ARG;
  }
  st = ensure_arpls_work(pl, n, n_sys);
  if (st != MRAID_OK) return st;
  cudaError_t e = MRAID_PROF(pl, K_ARPLS,
                             launch_arpls(pl, d_y, n_sys, n, bp->lam, bp->ratio, bp->itermax, d_z,
                                          nullptr, d_iters, pl->ar_work));
  return e == cudaSuccess ? MRAID_OK : cuda_fail(e, "arpls launch");
}

mraid_status mraid_run_bandpass(mraid_plan_t pl, const void* d_data,
                                const mraid_bandpass_params* bp, float* d_bandpass,
                                float* d_evals, float* d_q1, float* d_stat, uint8_t* d_flags,
                                mraid_flag_info* info) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  st = check_bandpass_params(bp);
  if (st != MRAID_OK) return st;
  if (!d_data || !d_stat || !d_flags) {
    set_error("mraid_run_bandpass: d_data, d_stat and d_flags are required");
    return MRAID_ERR_INVALID_ARG;
  }
  if (pl->p.bit_depth != 8 || pl->p.n_chan < 3 || pl->p.n_chan > (1 << 20)) {
    set_error("mraid_run_bandpass: 8-bit samples and 3 to 2^20 channels");
    return MRAID_ERR_UNSUPPORTED;
  }
  // an interval at least as long as the block is one interval of the
  // block: the same partition, and no int arithmetic on a huge interval
  const int interval = bp->interval < pl->p.n_sub ? bp->interval : pl->p.n_sub;
  const int n_int = (int)(((int64_t)pl->p.n_sub + interval - 1) / interval);
  if ((int64_t)n_int * pl->p.n_beam > INT32_MAX) {
    set_error("mraid_run_bandpass: %d intervals x %d beams exceed 2^31 - 1 spectra", n_int,
              pl->p.n_beam);
    return MRAID_ERR_UNSUPPORTED;
  }
  const int n_sys = n_int * pl->p.n_beam;
  const size_t elems = (size_t)n_sys * pl->p.n_chan;
  st = ensure_workspace(pl, (size_t)pl->n_cells);
  if (st != MRAID_OK) return st;
  cudaError_t e = cudaSuccess;
  if (elems > pl->bp_elems || (size_t)n_sys > pl->bp_sys) {
    cudaFree(pl->bp_y);
    cudaFree(pl->bp_z);
    cudaFree(pl->bp_iters);
    pl->bp_y = pl->bp_z = nullptr;
    pl->bp_iters = nullptr;
    pl->bp_elems = pl->bp_sys = 0;
    e = cudaMalloc(&pl->bp_y, elems * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&pl->bp_z, elems * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&pl->bp_iters, (size_t)n_sys * sizeof(int32_t));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "bandpass workspace allocation");
    }
    pl->bp_elems = elems;
    pl->bp_sys = (size_t)n_sys;
  }
  st = ensure_arpls_work(pl, pl->p.n_chan, n_sys);
  if (st != MRAID_OK) return st;
  if (d_q1) {
    st = evals_for_q1(pl, (size_t)pl->n_cells, &d_evals);
    if (st != MRAID_OK) return st;
  }
  e = cudaMemsetAsync(pl->d_sweeps, 0, 3 * sizeof(unsigned long long), pl->stream);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  bool inter = false;
  st = gram_sums_pass(pl, d_data, nullptr, &inter);
  if (st != MRAID_OK) return st;
  // the sums pass may count zero-variance beams; nothing is normalised here
  e = cudaMemsetAsync(pl->d_degenerate, 0, sizeof(unsigned long long), pl->stream);
  if (e == cudaSuccess)
    e = MRAID_PROF(pl, K_BP_INPUT,
                   launch_bandpass_input(pl, pl->ws.sums, inter, interval, pl->bp_y));
  if (e == cudaSuccess)
    e = MRAID_PROF(pl, K_ARPLS,
                   launch_arpls(pl, pl->bp_y, n_sys, pl->p.n_chan, bp->lam, bp->ratio,
                                bp->itermax, pl->bp_z, d_bandpass, pl->bp_iters, pl->ar_work));
  if (e == cudaSuccess)
    e = MRAID_PROF(pl, K_CCM_BP,
                   launch_ccm_bandpass(pl, pl->ws.sums, inter, interval, pl->bp_z, pl->ws.corr));
  if (e != cudaSuccess) return cuda_fail(e, "bandpass kernels");
  e = MRAID_PROF(pl, K_EIG, launch_eig(pl, pl->ws.corr, pl->n_cells, d_evals, d_q1, d_stat));
  if (e != cudaSuccess) return cuda_fail(e, "eig launch");
  e = MRAID_PROF(pl, K_FLAG, launch_flag(pl, d_stat, d_flags));
  if (e != cudaSuccess) return cuda_fail(e, "flag launch");
  e = cudaMemcpyAsync(&pl->d_info->n_degenerate, pl->d_degenerate, sizeof(int64_t),
                      cudaMemcpyDeviceToDevice, pl->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&pl->d_info->jacobi_sweeps, pl->d_sweeps, 2 * sizeof(int64_t),
                        cudaMemcpyDeviceToDevice, pl->stream);
  if (e == cudaSuccess)  // the FP64 q1 count (low half of the counter)
    e = cudaMemcpyAsync(&pl->d_info->q1_refined, pl->d_sweeps + 2, sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, pl->stream);
  if (e != cudaSuccess) return cuda_fail(e, "counter copy");
  return enqueue_info_copy(pl, info);
}
