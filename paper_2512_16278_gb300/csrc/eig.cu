// eig.cu - batched eigenvalues of small symmetric correlation matrices.
//
// Section 3.3, Eq. 2: C = Q Lambda Q^-1 for every cell's correlation
// matrix; eigenvalues ordered largest first and the dominant one
// normalised as s = lambda_1^2 / sum_i lambda_i^2. Only lambda_1's
// eigenvector q1 is kept (Section 3.3 stores the largest eigenvalue and
// its eigenvector per cell).
//
// Eigenvalues: two-sided parallel cyclic Jacobi in FP32. The rotations of
// one round act on disjoint index pairs (round-robin "circle" schedule), so
// one round is the block update A' = J^T A J over 2x2 blocks. For N <= 20
// one thread owns one matrix in registers: the pairs are always the slots
// (2i, 2i+1) and the round's results are written into circularly permuted
// slots, so every round runs the same register-indexed code. For larger N
// one thread block owns one matrix in shared memory.
// q1: inverse iteration with the Cholesky factor of (sigma I - r),
// sigma slightly above lambda_1, which is positive definite.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <utility>

#include "internal.h"

namespace mraid {
namespace {

// Compile-time loops: f(std::integral_constant<int, E>) for E = 0..K-1. The
// register-resident matrices below need every index to be a constant; fold
// expressions expand regardless of the optimiser's unrolling budget.
template <class F, int... E>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, E...>) {
  (f(std::integral_constant<int, E>{}), ...);
}
template <int K, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, K>{});
}

constexpr int kEigThreads = 64;
constexpr int kMaxSweeps = 16;
// Stop when off(A)_F^2 <= kTol2 * ||A||_F^2, i.e. off(A)_F <= 1e-5 ||A||_F.
// By Weyl's inequality every diagonal entry is then within off(A)_F of an
// eigenvalue: <= 1e-5 sqrt(N) lambda_max, inside the 1e-4 lambda_max bound
// (the actual error is second order in off(A) and far smaller).
constexpr float kTol2 = 1e-10f;

template <int N>
struct Slots {
  static constexpr bool kOdd = (N & 1) != 0;
  static constexpr int M = kOdd ? N + 1 : N;  // slots, incl. a fixed dummy for odd N
  static constexpr int H = M / 2;             // pair slots (2i, 2i+1)
  static constexpr int S0 = kOdd ? 1 : 0;     // first stored slot
  static constexpr int NP = N * (N + 1) / 2;
  // per-thread shared-memory row: the staged packed matrix, later the two
  // ping-pong scale vectors of M floats each; odd for conflict-free rows
  static constexpr int STR = ((NP > 2 * M) ? NP : 2 * M) | 1;
  static_assert(STR >= NP && STR >= 2 * M, "row too short");
  // packed upper triangle over stored slots (slot s holds beam s - S0 at start)
  __host__ __device__ static constexpr int idx(int k, int l) {
    return (k <= l) ? ((k - S0) * N - (k - S0) * (k - S0 - 1) / 2 + (l - k))
                    : ((l - S0) * N - (l - S0) * (l - S0 - 1) / 2 + (k - l));
  }
  // Circle schedule: top row T_i = slot 2i, bottom row B_i = slot 2i+1,
  // T_0 fixed; T_i -> T_{i+1}, T_{H-1} -> B_{H-1}, B_i -> B_{i-1}, B_0 -> T_1.
  // After M-1 rounds every pair of slots has shared a pair slot once.
  __host__ __device__ static constexpr int sigma(int s) {
    return (H == 1 || s == 0) ? s
           : (s % 2 == 0) ? ((s / 2 < H - 1) ? s + 2 : s + 1)
                          : ((s == 1) ? 2 : s - 2);
  }
  static constexpr int NB = H * (H - 1) / 2;  // off-diagonal 2x2 blocks (i < j)
  __host__ __device__ static constexpr int blk_i(int e) {
    int i = 0;
    while (e >= H - 1 - i) {
      e -= H - 1 - i;
      ++i;
    }
    return i;
  }
  __host__ __device__ static constexpr int blk_j(int e) {
    int i = 0;
    while (e >= H - 1 - i) {
      e -= H - 1 - i;
      ++i;
    }
    return i + 1 + e;
  }
  // packed (a <= b) index -> row / column
  __host__ __device__ static constexpr int row_of(int e) {
    int a = 0;
    while (e >= N - a) {
      e -= N - a;
      ++a;
    }
    return a;
  }
  __host__ __device__ static constexpr int col_of(int e) {
    int a = 0;
    while (e >= N - a) {
      e -= N - a;
      ++a;
    }
    return a + e;
  }
};

// Explicit shared-memory accesses (32-bit shared addresses), so the scale
// vectors never go through generic addressing.
__device__ __forceinline__ float lds(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts(uint32_t addr, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void rotation(float app, float aqq, float apq, float& c, float& s,
                                         float& t) {
  // t = tan(theta) of the rotation zeroing apq (smaller root of
  // t^2 + 2 tau t - 1 = 0, tau = (aqq - app) / (2 apq)), in division-free form
  // t = 2 apq sgn(d) / (|d| + sqrt(d^2 + 4 apq^2)), d = aqq - app, sgn(0) = +1.
  const float d = aqq - app;
  const float h2 = 2.f * apq;
  const float r2 = fmaf(d, d, h2 * h2);
  const float den = fmaxf(fabsf(d) + r2 * rsqrtf(fmaxf(r2, 1e-37f)), 1e-30f);
  t = __fdividef(d >= 0.f ? h2 : -h2, den);
  c = rsqrtf(fmaf(t, t, 1.f));
  s = t * c;
}

// One round of the scaled ("fast") two-sided Jacobi. The matrix is held as
// A = D A~ D with D = diag(d) per slot. For the pair (p, q) with rotation
// J (J_pp = J_qq = c, J_pq = s = t c, J_qp = -s) one has
// J^T D = D' M, D' = c D on p and q, M = [[1, alpha], [beta, 1]] with
// alpha = -t w, beta = t / w, w = d_q / d_p; so A~' = M A~ M^T, which costs
// one FMA per element and side instead of two multiplies and an add.
// The rotated pairs are the slots (2i, 2i+1); the results are written into
// circularly permuted slots (sigma), scales included.
template <int N>
__device__ __forceinline__ void jacobi_round(float (&a)[Slots<N>::NP], uint32_t dsrc,
                                             uint32_t ddst) {
  using S = Slots<N>;
  float al[S::H], be[S::H];
  static_for<S::H>([&](auto ii) {
    constexpr int i = decltype(ii)::value;
    if constexpr (i >= S::S0) {
      constexpr int p = 2 * i, q = 2 * i + 1;
      // tan(theta) from the true entries, scaled by 1 / (d_p d_q):
      // a_pp / (d_p d_q) = a~_pp / w, a_qq / (d_p d_q) = w a~_qq
      const float dp = lds(dsrc + 4 * p), dq = lds(dsrc + 4 * q);
      const float w = __fdividef(dq, dp), iw = __fdividef(dp, dq);
      const float app = a[S::idx(p, p)], aqq = a[S::idx(q, q)], apq = a[S::idx(p, q)];
      const float dd = fmaf(w, aqq, -iw * app);
      const float h2 = 2.f * apq;
      const float r2 = fmaf(dd, dd, h2 * h2);
      const float den = fmaxf(fabsf(dd) + r2 * rsqrtf(fmaxf(r2, 1e-37f)), 1e-30f);
      const float t = __fdividef(dd >= 0.f ? h2 : -h2, den);
      const float u = fmaf(t, t, 1.f);
      const float c = rsqrtf(u);
      al[i] = -t * w;
      be[i] = t * iw;
      sts(ddst + 4 * S::sigma(p), dp * c);  // scales move with their slots
      sts(ddst + 4 * S::sigma(q), dq * c);
    }
  });
  if constexpr (S::kOdd) sts(ddst + 4 * S::sigma(1), lds(dsrc + 4));  // idle slot keeps its scale
  float b[S::NP];
  // diagonal 2x2 blocks: A~' = M A~ M^T, off-diagonal entry annihilated
  static_for<S::H>([&](auto ii) {
    constexpr int i = decltype(ii)::value;
    if constexpr (i >= S::S0) {
      constexpr int p = 2 * i, q = 2 * i + 1;
      const float app = a[S::idx(p, p)], aqq = a[S::idx(q, q)], apq = a[S::idx(p, q)];
      const float h2 = 2.f * apq;
      b[S::idx(S::sigma(p), S::sigma(p))] = fmaf(al[i], fmaf(al[i], aqq, h2), app);
      b[S::idx(S::sigma(q), S::sigma(q))] = fmaf(be[i], fmaf(be[i], app, h2), aqq);
      b[S::idx(S::sigma(p), S::sigma(q))] = 0.f;
    }
  });
  if constexpr (S::kOdd) b[S::idx(S::sigma(1), S::sigma(1))] = a[S::idx(1, 1)];  // idle slot
  // off-diagonal blocks (i < j): B~' = M_i B~ M_j^T
  static_for<S::NB>([&](auto ee) {
    constexpr int i = S::blk_i(decltype(ee)::value), j = S::blk_j(decltype(ee)::value);
    constexpr int pi = 2 * i, qi = 2 * i + 1, pj = 2 * j, qj = 2 * j + 1;
    if constexpr (S::kOdd && i == 0) {
      // slot 0 is the dummy; slot 1 is idle this round: right factor only
      const float y0 = a[S::idx(qi, pj)], y1 = a[S::idx(qi, qj)];
      b[S::idx(S::sigma(qi), S::sigma(pj))] = fmaf(al[j], y1, y0);
      b[S::idx(S::sigma(qi), S::sigma(qj))] = fmaf(be[j], y0, y1);
    } else {
      const float x00 = a[S::idx(pi, pj)], x01 = a[S::idx(pi, qj)];
      const float x10 = a[S::idx(qi, pj)], x11 = a[S::idx(qi, qj)];
      const float l00 = fmaf(al[i], x10, x00), l01 = fmaf(al[i], x11, x01);
      const float l10 = fmaf(be[i], x00, x10), l11 = fmaf(be[i], x01, x11);
      b[S::idx(S::sigma(pi), S::sigma(pj))] = fmaf(al[j], l01, l00);
      b[S::idx(S::sigma(pi), S::sigma(qj))] = fmaf(be[j], l00, l01);
      b[S::idx(S::sigma(qi), S::sigma(pj))] = fmaf(al[j], l11, l10);
      b[S::idx(S::sigma(qi), S::sigma(qj))] = fmaf(be[j], l10, l11);
    }
  });
  static_for<S::NP>([&](auto ee) { a[decltype(ee)::value] = b[decltype(ee)::value]; });
}

// Cholesky-based inverse iteration for the eigenvector of lambda_1 of the
// packed matrix r (N x N), in registers. Returns false if the factor failed.
template <int N>
__device__ bool dominant_vector(const float* r, float lambda1, float (&x)[N]) {
  using S = Slots<N>;
  constexpr int NP = S::NP;
  auto pk = [](int a, int b) { return a * N - a * (a - 1) / 2 + (b - a); };  // a <= b
  float delta = fmaxf(4e-5f * fabsf(lambda1), 1e-6f);
  bool ok = false;
  float u[NP];
  float dinv[N];
  for (int attempt = 0; attempt < 4 && !ok; ++attempt, delta *= 16.f) {
    const float sig = lambda1 + delta;
    static_for<NP>([&](auto ee) {
      constexpr int e = decltype(ee)::value;
      u[e] = (S::row_of(e) == S::col_of(e)) ? sig - r[e] : -r[e];
    });
    ok = true;
    // right-looking Cholesky: u becomes U with sigma I - r = U^T U
    static_for<N>([&](auto aa) {
      constexpr int a = decltype(aa)::value;
      const float piv = u[pk(a, a)];
      ok = ok && (piv > 0.f);
      const float inv = rsqrtf(fmaxf(piv, 1e-30f));
      dinv[a] = inv;
      u[pk(a, a)] = piv * inv;
      static_for<N - a - 1>([&](auto bb) { u[pk(a, a + 1 + decltype(bb)::value)] *= inv; });
      static_for<N - a - 1>([&](auto bb) {
        constexpr int b = a + 1 + decltype(bb)::value;
        static_for<N - b>([&](auto cc) {
          constexpr int c = b + decltype(cc)::value;
          u[pk(b, c)] = fmaf(-u[pk(a, b)], u[pk(a, c)], u[pk(b, c)]);
        });
      });
    });
  }
  if (!ok) return false;
  static_for<N>([&](auto aa) {
    constexpr int a = decltype(aa)::value;
    x[a] = 1.f + 0.25f * (float)((a * 7) % 5);
  });
  for (int it = 0; it < 3; ++it) {
    // U^T z = x (forward), then U x = z (backward)
    static_for<N>([&](auto aa) {
      constexpr int a = decltype(aa)::value;
      float v = x[a];
      static_for<a>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        v = fmaf(-u[pk(k, a)], x[k], v);
      });
      x[a] = v * dinv[a];
    });
    static_for<N>([&](auto aa) {
      constexpr int a = N - 1 - decltype(aa)::value;
      float v = x[a];
      static_for<N - 1 - a>([&](auto kk) {
        constexpr int k = a + 1 + decltype(kk)::value;
        v = fmaf(-u[pk(a, k)], x[k], v);
      });
      x[a] = v * dinv[a];
    });
    float nn = 0.f;
    static_for<N>([&](auto aa) { nn = fmaf(x[decltype(aa)::value], x[decltype(aa)::value], nn); });
    const float inv = rsqrtf(fmaxf(nn, 1e-37f));
    static_for<N>([&](auto aa) { x[decltype(aa)::value] *= inv; });
  }
  return true;
}

template <int N>
__global__ void __launch_bounds__(kEigThreads)
eig_reg_kernel(const float* __restrict__ corr, int64_t n_cells, float* __restrict__ evals,
               float* __restrict__ stat, unsigned long long* __restrict__ sweep_count) {
  using S = Slots<N>;
  constexpr int NP = S::NP;
  constexpr int STR = S::STR;
  extern __shared__ float sm[];
  const int64_t cell0 = (int64_t)blockIdx.x * kEigThreads;
  const int ncell = (int)min((int64_t)kEigThreads, n_cells - cell0);
  const float* src = corr + cell0 * NP;
  for (int i = threadIdx.x; i < ncell * NP; i += blockDim.x) {
    const int c = i / NP;
    sm[c * STR + (i - c * NP)] = src[i];
  }
  __syncthreads();
  const bool active = (int)threadIdx.x < ncell;
  const float* my = sm + threadIdx.x * STR;
  float a[NP];
  // slot s holds beam s - S0, so packed slot order equals packed beam order
  static_for<NP>([&](auto ee) {
    constexpr int e = decltype(ee)::value;
    a[e] = active ? my[e] : (S::row_of(e) == S::col_of(e) ? 1.f : 0.f);
  });

  bool conv = !active;
  int sweeps = 0;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    if (!__any_sync(0xffffffffu, !conv)) break;
    // scales live in this thread's (now free) staging row of shared memory,
    // ping-ponged between two halves so a round reads the old ones
    const uint32_t d0 = static_cast<uint32_t>(__cvta_generic_to_shared(sm + threadIdx.x * STR));
    const uint32_t d1 = d0 + 4 * S::M;
    static_for<S::M>([&](auto kk) { sts(d0 + 4 * decltype(kk)::value, 1.f); });
    // two rounds per iteration: the scheduler can overlap the next round's
    // rotation chains with this round's block updates
#pragma unroll 2
    for (int r = 0; r < S::M - 1; ++r) jacobi_round<N>(a, (r & 1) ? d1 : d0, (r & 1) ? d0 : d1);
    const uint32_t dl = ((S::M - 1) & 1) ? d1 : d0;
    float d[S::M];
    static_for<S::M>([&](auto kk) { d[decltype(kk)::value] = lds(dl + 4 * decltype(kk)::value); });
    // back to true entries (a_kl = d_k a~_kl d_l), then the convergence test
    float off = 0.f, dia = 0.f;
    static_for<NP>([&](auto ee) {
      constexpr int e = decltype(ee)::value;
      constexpr int k = S::row_of(e) + S::S0, l = S::col_of(e) + S::S0;
      a[e] *= d[k] * d[l];
      if constexpr (k == l) dia = fmaf(a[e], a[e], dia);
      else off = fmaf(a[e], a[e], off);
    });
    if (!conv) ++sweeps;
    conv = conv || (off <= kTol2 * fmaf(2.f, off, dia));
  }
  if (sweep_count) {
    // executed sweeps of this warp (its slowest cell) and sweeps per cell
    const int wmax = __reduce_max_sync(0xffffffffu, sweeps);
    const unsigned wsum = __reduce_add_sync(0xffffffffu, (unsigned)sweeps);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&sweep_count[0], (unsigned long long)wsum);
      atomicAdd(&sweep_count[1], (unsigned long long)wmax);
    }
  }
  float ev[N];
  static_for<N>([&](auto kk) {
    constexpr int k = decltype(kk)::value;
    ev[k] = a[S::idx(k + S::S0, k + S::S0)];
  });
  // odd-even transposition sort, descending
  static_for<N>([&](auto pp) {
    constexpr int pass = decltype(pp)::value;
    static_for<(N - (pass & 1)) / 2>([&](auto kk) {
      constexpr int k = (pass & 1) + 2 * decltype(kk)::value;
      const float hi = fmaxf(ev[k], ev[k + 1]), lo = fminf(ev[k], ev[k + 1]);
      ev[k] = hi;
      ev[k + 1] = lo;
    });
  });
  if (!active) return;
  const int64_t cell = cell0 + threadIdx.x;
  float ss = 0.f;
  static_for<N>([&](auto kk) { ss = fmaf(ev[decltype(kk)::value], ev[decltype(kk)::value], ss); });
  stat[cell] = ss > 0.f ? ev[0] * ev[0] / ss : 0.f;
  if (evals) static_for<N>([&](auto kk) { evals[cell * N + decltype(kk)::value] = ev[decltype(kk)::value]; });
}

// q1 of every cell from its correlation and lambda_1 (evals[cell * N]): a
// separate pass so that the Jacobi sweeps keep all registers.
template <int N>
__global__ void __launch_bounds__(kEigThreads)
q1_reg_kernel(const float* __restrict__ corr, int64_t n_cells, const float* __restrict__ evals,
              float* __restrict__ q1) {
  constexpr int NP = Slots<N>::NP;
  constexpr int STR = Slots<N>::STR;
  extern __shared__ float sm[];
  const int64_t cell0 = (int64_t)blockIdx.x * kEigThreads;
  const int ncell = (int)min((int64_t)kEigThreads, n_cells - cell0);
  const float* src = corr + cell0 * NP;
  for (int i = threadIdx.x; i < ncell * NP; i += blockDim.x) {
    const int c = i / NP;
    sm[c * STR + (i - c * NP)] = src[i];
  }
  __syncthreads();
  if ((int)threadIdx.x >= ncell) return;
  const int64_t cell = cell0 + threadIdx.x;
  float x[N];
  const bool ok = dominant_vector<N>(sm + threadIdx.x * STR, evals[cell * N], x);
  // sign rule: largest-magnitude element positive (lowest index on ties)
  float best = 0.f, sgn = 1.f;
  static_for<N>([&](auto kk) {
    const float v = x[decltype(kk)::value];
    if (fabsf(v) > best) {
      best = fabsf(v);
      sgn = v < 0.f ? -1.f : 1.f;
    }
  });
  if (!ok) sgn = __int_as_float(0x7fc00000);  // NaN marks a failed factor
  static_for<N>([&](auto kk) { q1[cell * N + decltype(kk)::value] = sgn * x[decltype(kk)::value]; });
}

// ---------------------------------------------------------------------------
// Shared-memory Jacobi for larger N: one block per matrix, full N x N
// matrix, circle schedule with index pairs (k, partner) where
// k + partner = 2r (mod M-1) and index M-1 meets r.
constexpr int kBlkThreads = 256;

__global__ void __launch_bounds__(kBlkThreads)
eig_block_kernel(const float* __restrict__ corr, int64_t n_cells, int N, float* __restrict__ evals,
                 float* __restrict__ q1, float* __restrict__ stat) {
  extern __shared__ float sm[];
  const int ld = N + 1;
  const int M = (N & 1) ? N + 1 : N;
  float* A = sm;                     // N x ld
  float* B = A + N * ld;             // N x ld
  float* R0 = B + N * ld;            // N x ld: the input r
  float* jp = R0 + N * ld;           // [N] coefficient J[p_k][k]
  float* jq = jp + N;                // [N] coefficient J[q_k][k]
  int* pidx = reinterpret_cast<int*>(jq + N);  // [N] p_k
  int* qidx = pidx + N;                        // [N] q_k (== p_k if idle)
  float* red = reinterpret_cast<float*>(qidx + N);  // [2 * 32]
  float* x = red + 64;               // [N]
  float* y = x + N;                  // [N]
  const int np = N * (N + 1) / 2;
  const int tid = threadIdx.x;
  for (int64_t cell = blockIdx.x; cell < n_cells; cell += gridDim.x) {
    const float* src = corr + cell * np;
    for (int e = tid; e < np; e += blockDim.x) {
      // e -> (a, b), a <= b
      int a = 0, rem = e;
      while (rem >= N - a) {
        rem -= N - a;
        ++a;
      }
      const int b = a + rem;
      const float v = src[e];
      A[a * ld + b] = v;
      A[b * ld + a] = v;
      R0[a * ld + b] = v;
      R0[b * ld + a] = v;
    }
    __syncthreads();
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
      for (int r = 0; r < M - 1; ++r) {
        for (int k = tid; k < N; k += blockDim.x) {
          int partner = (k == M - 1) ? r : (k == r ? M - 1 : ((2 * r - k) % (M - 1) + (M - 1)) % (M - 1));
          if (partner >= N) {  // paired with the dummy: idle
            pidx[k] = k;
            qidx[k] = k;
            jp[k] = 1.f;
            jq[k] = 0.f;
          } else {
            const int p = min(k, partner), q = max(k, partner);
            float c, s, t;
            rotation(A[p * ld + p], A[q * ld + q], A[p * ld + q], c, s, t);
            pidx[k] = p;
            qidx[k] = q;
            // column k of J: J_pp = c, J_qp = -s; J_pq = s, J_qq = c
            jp[k] = (k == p) ? c : s;
            jq[k] = (k == p) ? -s : c;
          }
        }
        __syncthreads();
        for (int e = tid; e < N * N; e += blockDim.x) {
          const int k = e / N, l = e - k * N;
          const int pk = pidx[k], qk = qidx[k], pl = pidx[l], ql = qidx[l];
          const float ak = jp[k], bk = jq[k], al = jp[l], bl = jq[l];
          // B = J^T A J restricted to the pairs of k and l (idle: J column = e_k)
          const float v = ak * fmaf(A[pk * ld + pl], al, A[pk * ld + ql] * bl) +
                          bk * fmaf(A[qk * ld + pl], al, A[qk * ld + ql] * bl);
          B[k * ld + l] = v;
        }
        __syncthreads();
        for (int e = tid; e < N * N; e += blockDim.x) {
          const int k = e / N, l = e - k * N;
          A[k * ld + l] = (k == l) ? B[k * ld + l] : 0.5f * (B[k * ld + l] + B[l * ld + k]);
        }
        __syncthreads();
      }
      float off = 0.f, dia = 0.f;
      for (int e = tid; e < N * N; e += blockDim.x) {
        const int k = e / N, l = e - k * N;
        const float v = A[k * ld + l];
        if (k == l) dia = fmaf(v, v, dia);
        else off = fmaf(v, v, off);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        dia += __shfl_xor_sync(0xffffffffu, dia, o);
      }
      if ((tid & 31) == 0) {
        red[tid / 32] = off;
        red[32 + tid / 32] = dia;
      }
      __syncthreads();
      float to = 0.f, td = 0.f;
      for (int w = 0; w < (int)blockDim.x / 32; ++w) {
        to += red[w];
        td += red[32 + w];
      }
      __syncthreads();
      if (to <= kTol2 * (td + to)) break;
    }
    // eigenvalues: diagonal sorted descending (rank by counting)
    for (int k = tid; k < N; k += blockDim.x) {
      const float v = A[k * ld + k];
      int rank = 0;
      for (int m = 0; m < N; ++m) {
        const float w = A[m * ld + m];
        rank += (w > v) || (w == v && m < k);
      }
      y[rank] = v;
    }
    __syncthreads();
    const float lam1 = y[0];
    if (tid == 0) {
      float ss = 0.f;
      for (int k = 0; k < N; ++k) ss = fmaf(y[k], y[k], ss);
      stat[cell] = ss > 0.f ? lam1 * lam1 / ss : 0.f;
    }
    if (evals)
      for (int k = tid; k < N; k += blockDim.x) evals[cell * N + k] = y[k];
    __syncthreads();
    if (q1) {
      // B <- sigma I - r, then in-place right-looking Cholesky (upper)
      float delta = fmaxf(4e-5f * fabsf(lam1), 1e-6f);
      bool ok = false;
      for (int attempt = 0; attempt < 4 && !ok; ++attempt, delta *= 16.f) {
        for (int e = tid; e < N * N; e += blockDim.x) {
          const int k = e / N, l = e - k * N;
          B[k * ld + l] = (k == l ? lam1 + delta : 0.f) - R0[k * ld + l];
        }
        __syncthreads();
        ok = true;
        for (int a = 0; a < N; ++a) {
          const float piv = B[a * ld + a];
          ok = ok && piv > 0.f;
          const float inv = rsqrtf(fmaxf(piv, 1e-30f));
          __syncthreads();
          for (int b = a + 1 + tid; b < N; b += blockDim.x) B[a * ld + b] *= inv;
          if (tid == 0) B[a * ld + a] = piv * inv;
          __syncthreads();
          for (int e = tid; e < (N - a - 1) * (N - a - 1); e += blockDim.x) {
            const int b = a + 1 + e / (N - a - 1), c = a + 1 + e % (N - a - 1);
            if (c >= b) B[b * ld + c] = fmaf(-B[a * ld + b], B[a * ld + c], B[b * ld + c]);
          }
          __syncthreads();
        }
      }
      if (tid == 0) {
        for (int a = 0; a < N; ++a) x[a] = 1.f + 0.25f * (float)((a * 7) % 5);
        for (int it = 0; it < 3 && ok; ++it) {
          for (int a = 0; a < N; ++a) {
            float v = x[a];
            for (int k = 0; k < a; ++k) v = fmaf(-B[k * ld + a], x[k], v);
            x[a] = v / B[a * ld + a];
          }
          for (int a = N - 1; a >= 0; --a) {
            float v = x[a];
            for (int k = a + 1; k < N; ++k) v = fmaf(-B[a * ld + k], x[k], v);
            x[a] = v / B[a * ld + a];
          }
          float nn = 0.f;
          for (int a = 0; a < N; ++a) nn = fmaf(x[a], x[a], nn);
          const float inv = rsqrtf(fmaxf(nn, 1e-37f));
          for (int a = 0; a < N; ++a) x[a] *= inv;
        }
        int imax = 0;
        for (int a = 1; a < N; ++a)
          if (fabsf(x[a]) > fabsf(x[imax])) imax = a;
        const float sgn = (x[imax] < 0.f) ? -1.f : 1.f;
        for (int a = 0; a < N; ++a) x[a] = ok ? sgn * x[a] : __int_as_float(0x7fc00000);
      }
      __syncthreads();
      for (int k = tid; k < N; k += blockDim.x) q1[cell * N + k] = x[k];
    }
    __syncthreads();
  }
}

template <int N>
cudaError_t launch_reg(const float* d_corr, int64_t n_cells, float* d_evals, float* d_q1,
                       float* d_stat, unsigned long long* sweep_count, cudaStream_t stream) {
  constexpr int STR = Slots<N>::STR;
  const size_t smem = (size_t)kEigThreads * STR * sizeof(float);
  const int64_t blocks = (n_cells + kEigThreads - 1) / kEigThreads;
  cudaError_t e = cudaFuncSetAttribute(eig_reg_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (blocks > 0)
    eig_reg_kernel<N><<<(unsigned)blocks, kEigThreads, smem, stream>>>(d_corr, n_cells, d_evals,
                                                                          d_stat, sweep_count);
  if (d_q1) {
    e = cudaFuncSetAttribute(q1_reg_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (blocks > 0)
      q1_reg_kernel<N><<<(unsigned)blocks, kEigThreads, smem, stream>>>(d_corr, n_cells, d_evals,
                                                                           d_q1);
  }
  return cudaGetLastError();
}

}  // namespace

bool eig_supported(int n_beam) { return n_beam >= 2 && n_beam <= kMaxBeam; }

bool eig_q1_needs_evals(int n_beam) {
  return n_beam == 2 || n_beam == 3 || n_beam == 4 || n_beam == 13 || n_beam == 19;
}

cudaError_t launch_eig(const mraid_plan_s* pl, const float* d_corr, int64_t n_cells, float* d_evals,
                       float* d_q1, float* d_stat) {
  const int N = pl->p.n_beam;
  switch (N) {
    case 2: return launch_reg<2>(d_corr, n_cells, d_evals, d_q1, d_stat, pl->d_sweeps, pl->stream);
    case 3: return launch_reg<3>(d_corr, n_cells, d_evals, d_q1, d_stat, pl->d_sweeps, pl->stream);
    case 4: return launch_reg<4>(d_corr, n_cells, d_evals, d_q1, d_stat, pl->d_sweeps, pl->stream);
    case 13: return launch_reg<13>(d_corr, n_cells, d_evals, d_q1, d_stat, pl->d_sweeps, pl->stream);
    case 19: return launch_reg<19>(d_corr, n_cells, d_evals, d_q1, d_stat, pl->d_sweeps, pl->stream);
    default: break;
  }
  const int ld = N + 1;
  const size_t smem = sizeof(float) * (3 * (size_t)N * ld + 2 * N + 64 + 2 * N) + sizeof(int) * 2 * N;
  cudaError_t e = cudaFuncSetAttribute(eig_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int64_t blocks = n_cells < (int64_t)pl->sm_count * 8 ? n_cells : (int64_t)pl->sm_count * 8;
  if (blocks > 0)
    eig_block_kernel<<<(unsigned)blocks, kBlkThreads, smem, pl->stream>>>(d_corr, n_cells, N, d_evals,
                                                                           d_q1, d_stat);
  return cudaGetLastError();
}

}  // namespace mraid
