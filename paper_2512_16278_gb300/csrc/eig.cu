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

#include <type_traits>
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
  __host__ __device__ static constexpr int sigma_inv(int s) {
    int t = 0;
    while (sigma(t) != s) ++t;
    return t;
  }
  // Index held by slot s after r rounds of the circle schedule
  // (content(sigma(s), r + 1) = content(s, r), content(s, 0) = s).
  __host__ __device__ static constexpr int content(int s, int r) {
    for (int k = 0; k < r; ++k) s = sigma_inv(s);
    return s;
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

// Copy the packed matrices of a block's cells from global memory into
// per-thread shared-memory rows of STR floats. Asynchronous copies keep
// many loads in flight; a plain load-then-store loop waits out the memory
// latency once per element.
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
template <int NP, int STR>
__device__ __forceinline__ void stage_rows(float* sm, const float* __restrict__ src, int ncell) {
  const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(sm));
  for (int i = threadIdx.x; i < ncell * NP; i += blockDim.x) {
    const int c = i / NP;
    cp_async4(base + 4u * (uint32_t)(c * STR + (i - c * NP)), src + i);
  }
  cp_async_wait_all();
  __syncthreads();
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

// The same round with the data left in place: round r of a sweep rotates the
// index pairs (content(2i, r), content(2i+1, r)), known at compile time, so a
// fully unrolled sweep needs no register moves and no second array.
template <int N, int R>
__device__ __forceinline__ void jacobi_round_static(float (&a)[Slots<N>::NP], uint32_t dsm) {
  using S = Slots<N>;
  float al[S::H], be[S::H];
  static_for<S::H>([&](auto ii) {
    constexpr int i = decltype(ii)::value;
    if constexpr (i >= S::S0) {
      constexpr int p = S::content(2 * i, R), q = S::content(2 * i + 1, R);
      const float dp = lds(dsm + 4 * p), dq = lds(dsm + 4 * q);
      const float w = __fdividef(dq, dp), iw = __fdividef(dp, dq);
      const float app = a[S::idx(p, p)], aqq = a[S::idx(q, q)], apq = a[S::idx(p, q)];
      const float dd = fmaf(w, aqq, -iw * app);
      const float h2 = 2.f * apq;
      const float r2 = fmaf(dd, dd, h2 * h2);
      const float den = fmaxf(fabsf(dd) + r2 * rsqrtf(fmaxf(r2, 1e-37f)), 1e-30f);
      const float t = __fdividef(dd >= 0.f ? h2 : -h2, den);
      const float c = rsqrtf(fmaf(t, t, 1.f));
      al[i] = -t * w;
      be[i] = t * iw;
      sts(dsm + 4 * p, dp * c);
      sts(dsm + 4 * q, dq * c);
      // the pair's own 2x2 block
      a[S::idx(p, p)] = fmaf(al[i], fmaf(al[i], aqq, h2), app);
      a[S::idx(q, q)] = fmaf(be[i], fmaf(be[i], app, h2), aqq);
      a[S::idx(p, q)] = 0.f;
    }
  });
  static_for<S::NB>([&](auto ee) {
    constexpr int i = S::blk_i(decltype(ee)::value), j = S::blk_j(decltype(ee)::value);
    constexpr int pi = S::content(2 * i, R), qi = S::content(2 * i + 1, R);
    constexpr int pj = S::content(2 * j, R), qj = S::content(2 * j + 1, R);
    if constexpr (S::kOdd && i == 0) {
      // pair slot 0 holds the dummy and the idle index: right factor only
      const float y0 = a[S::idx(qi, pj)], y1 = a[S::idx(qi, qj)];
      a[S::idx(qi, pj)] = fmaf(al[j], y1, y0);
      a[S::idx(qi, qj)] = fmaf(be[j], y0, y1);
    } else {
      const float x00 = a[S::idx(pi, pj)], x01 = a[S::idx(pi, qj)];
      const float x10 = a[S::idx(qi, pj)], x11 = a[S::idx(qi, qj)];
      const float l00 = fmaf(al[i], x10, x00), l01 = fmaf(al[i], x11, x01);
      const float l10 = fmaf(be[i], x00, x10), l11 = fmaf(be[i], x01, x11);
      a[S::idx(pi, pj)] = fmaf(al[j], l01, l00);
      a[S::idx(pi, qj)] = fmaf(be[j], l00, l01);
      a[S::idx(qi, pj)] = fmaf(al[j], l11, l10);
      a[S::idx(qi, qj)] = fmaf(be[j], l10, l11);
    }
  });
}

// Cholesky-based inverse iteration for the eigenvector of lambda_1: the
// upper factor U of sigma I - r (sigma slightly above lambda_1, so the matrix
// is positive definite) is built in place in this thread's shared-memory row
// (packed upper triangle, which held r), then three solves U^T U x = x.
// src is r in global memory, reloaded if a shift proves too small.
template <int N>
__device__ bool dominant_vector(float* row, const float* __restrict__ src, float lambda1,
                                float (&x)[N]) {
  using S = Slots<N>;
  constexpr int NP = S::NP;
  auto pk = [](int a, int b) { return a * N - a * (a - 1) / 2 + (b - a); };  // a <= b
  float delta = fmaxf(4e-5f * fabsf(lambda1), 1e-6f);
  bool ok = false;
  float dinv[N];
  for (int attempt = 0; attempt < 4 && !ok; ++attempt, delta *= 16.f) {
    if (attempt > 0) static_for<NP>([&](auto ee) { row[decltype(ee)::value] = src[decltype(ee)::value]; });
    const float sig = lambda1 + delta;
    static_for<NP>([&](auto ee) {
      constexpr int e = decltype(ee)::value;
      row[e] = (S::row_of(e) == S::col_of(e)) ? sig - row[e] : -row[e];
    });
    ok = true;
    // right-looking Cholesky, in place: row becomes U with sigma I - r = U^T U
    static_for<N>([&](auto aa) {
      constexpr int a = decltype(aa)::value;
      const float piv = row[pk(a, a)];
      ok = ok && (piv > 0.f);
      const float inv = rsqrtf(fmaxf(piv, 1e-30f));
      dinv[a] = inv;
      row[pk(a, a)] = piv * inv;
      float ua[N];
      static_for<N - a - 1>([&](auto bb) {
        constexpr int b = a + 1 + decltype(bb)::value;
        ua[b] = row[pk(a, b)] * inv;
        row[pk(a, b)] = ua[b];
      });
      static_for<N - a - 1>([&](auto bb) {
        constexpr int b = a + 1 + decltype(bb)::value;
        static_for<N - b>([&](auto cc) {
          constexpr int c = b + decltype(cc)::value;
          row[pk(b, c)] = fmaf(-ua[b], ua[c], row[pk(b, c)]);
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
        v = fmaf(-row[pk(k, a)], x[k], v);
      });
      x[a] = v * dinv[a];
    });
    static_for<N>([&](auto aa) {
      constexpr int a = N - 1 - decltype(aa)::value;
      float v = x[a];
      static_for<N - 1 - a>([&](auto kk) {
        constexpr int k = a + 1 + decltype(kk)::value;
        v = fmaf(-row[pk(a, k)], x[k], v);
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

template <int N, bool kStatic>
__global__ void __launch_bounds__(kEigThreads)
eig_reg_kernel(const float* __restrict__ corr, int64_t n_cells, float* __restrict__ evals,
               float* __restrict__ stat, unsigned long long* __restrict__ sweep_count) {
  using S = Slots<N>;
  constexpr int NP = S::NP;
  constexpr int STR = S::STR;
  extern __shared__ float sm[];
  const int64_t cell0 = (int64_t)blockIdx.x * kEigThreads;
  const int ncell = (int)min((int64_t)kEigThreads, n_cells - cell0);
  stage_rows<NP, STR>(sm, corr + cell0 * NP, ncell);
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
    uint32_t dl = d0;
    if constexpr (kStatic) {
      // the whole sweep unrolled, data in place
      static_for<S::M - 1>([&](auto rr) { jacobi_round_static<N, decltype(rr)::value>(a, d0); });
    } else {
      // two rounds per iteration: the scheduler can overlap the next round's
      // rotation chains with this round's block updates
#pragma unroll 2
      for (int r = 0; r < S::M - 1; ++r) jacobi_round<N>(a, (r & 1) ? d1 : d0, (r & 1) ? d0 : d1);
      dl = ((S::M - 1) & 1) ? d1 : d0;
    }
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
  stage_rows<NP, STR>(sm, corr + cell0 * NP, ncell);
  if ((int)threadIdx.x >= ncell) return;
  const int64_t cell = cell0 + threadIdx.x;
  float x[N];
  const bool ok = dominant_vector<N>(sm + threadIdx.x * STR, corr + cell * NP, evals[cell * N], x);
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
// Tridiagonal route (same outputs): Householder reduction r = Q T Q^T in
// registers, all eigenvalues of T by implicit symmetric QR steps with the
// Wilkinson shift, deflating from the bottom, and q1 by inverse iteration on
// T followed by the back-transform with the stored reflectors. This costs
// about (4/3) N^3 flops for the reduction plus O(N^2) per QR pass, against
// ~3 N^3 flops per Jacobi sweep.
constexpr int kMaxQrIter = 24;  // QR steps per eigenvalue (the shift converges cubically)

// One implicit symmetric QR step with the Wilkinson shift on the unreduced
// block [l, m] of the tridiagonal (d, e); dm1, dm, em are d[m-1], d[m],
// e[m-1]. The bulge is chased down with plane rotations; steps outside
// [l, m) are skipped per lane. The code covers the rotation positions
// 0..K-1, so it serves every block with m <= K.
template <int N, int K = N - 1>
__device__ __forceinline__ void qr_step(float (&d)[N], float (&e)[N], int l, int m, float dm1,
                                        float dm, float em) {
  static_assert(K >= 1 && K <= N - 1, "rotation positions");
  // the eigenvalue of the trailing 2x2 nearer d[m]
  const float dl = 0.5f * (dm1 - dm);
  const float r2s = fmaf(dl, dl, em * em);
  const float rr = r2s * rsqrtf(r2s);  // em != 0 here, so r2s > 0
  const float mu = dm - __fdividef(em * em, dl + (dl >= 0.f ? rr : -rr));
  float x = 0.f, z = 0.f;
  static_for<K>([&](auto kk) {
    constexpr int k = decltype(kk)::value;
    if (k >= l && k < m) {
      if (k == l) {
        x = d[k] - mu;
        z = e[k];
      }
      // rotation in the (k, k+1) plane taking (x, z) to (r, 0)
      const float r2 = fmaf(x, x, z * z);
      const bool nz = r2 > 1e-37f;
      const float ri = nz ? rsqrtf(r2) : 0.f;
      const float c = nz ? x * ri : 1.f, s = nz ? z * ri : 0.f;
      if (k > l) e[k - 1] = r2 * ri;
      const float dk = d[k], ek = e[k], dk1 = d[k + 1];
      const float cc = c * c, ss = s * s, cs2 = 2.f * c * s * ek;
      d[k] = fmaf(cc, dk, fmaf(ss, dk1, cs2));
      d[k + 1] = fmaf(ss, dk, fmaf(cc, dk1, -cs2));
      e[k] = fmaf(c * s, dk1 - dk, (cc - ss) * ek);
      if constexpr (k + 1 < N - 1) {
        if (k < m - 1) {
          z = s * e[k + 1];
          e[k + 1] *= c;
        }
      }
      x = e[k];
    }
  });
}

// The same implicit QR step in root-free form for eigenvalues only (the
// Pal-Walker-Kahan variant, Parlett, The Symmetric Eigenvalue Problem,
// section 8-15): it carries the squared off-diagonals e2 = e^2 and the
// quantities gamma = c (d - mu) - s gamma' and p = gamma^2 / c of the
// rotation chase, so a rotation costs one division and no square root. The
// chase runs from the top of the unreduced block [l, m] down, deflating at
// its bottom, with the Wilkinson shift of the trailing 2x2 block.
template <int N, int K = N - 1>
__device__ __forceinline__ void qr_step_pwk(float (&d)[N], float (&e2)[N], int l, int m, float dm1,
                                            float dm, float e2m) {
  static_assert(K >= 1 && K <= N - 1, "rotation positions");
  const float dl = 0.5f * (dm1 - dm);
  const float r2s = fmaf(dl, dl, e2m);
  const float rr = r2s * rsqrtf(r2s);  // e2m > 0 here, so r2s > 0
  const float mu = dm - __fdividef(e2m, dl + (dl >= 0.f ? rr : -rr));
  float c = 1.f, s = 0.f, gamma = 0.f, p = 0.f;
  static_for<K>([&](auto kk) {
    constexpr int k = decltype(kk)::value;
    if (k >= l && k < m) {
      if (k == l) {
        gamma = d[k] - mu;
        p = gamma * gamma;
      }
      const float bb = e2[k];
      const float r = p + bb;
      if (k > l) e2[k - 1] = s * r;
      const float oldc = c;
      const float ri = r > 1e-37f ? __frcp_rn(r) : 0.f;
      c = r > 1e-37f ? p * ri : 1.f;
      s = bb * ri;
      const float oldgam = gamma, alpha = d[k + 1];
      gamma = fmaf(c, alpha - mu, -s * oldgam);
      d[k] = oldgam + (alpha - gamma);
      p = c != 0.f ? __fdividef(gamma * gamma, c) : oldc * bb;
      if (k == m - 1) {
        e2[k] = s * p;
        d[k + 1] = mu + gamma;
      }
    }
  });
}

template <int N, bool kCompact>
__global__ void __launch_bounds__(kEigThreads)
eig_tri_kernel(const float* __restrict__ corr, int64_t n_cells, float* __restrict__ evals,
               float* __restrict__ q1, float* __restrict__ stat,
               unsigned long long* __restrict__ step_count) {
  constexpr int NP = Slots<N>::NP;
  constexpr int STR = Slots<N>::STR;
  extern __shared__ float sm[];
  const int64_t cell0 = (int64_t)blockIdx.x * kEigThreads;
  const int ncell = (int)min((int64_t)kEigThreads, n_cells - cell0);
  stage_rows<NP, STR>(sm, corr + cell0 * NP, ncell);
  const bool active = (int)threadIdx.x < ncell;
  float* row = sm + threadIdx.x * STR;
  const uint32_t rowa = static_cast<uint32_t>(__cvta_generic_to_shared(row));
  auto pk = [](int a, int b) { return a * N - a * (a - 1) / 2 + (b - a); };  // a <= b
  float a[NP];
  static_for<NP>([&](auto ee) {
    constexpr int e = decltype(ee)::value;
    a[e] = active ? row[e] : (Slots<N>::row_of(e) == Slots<N>::col_of(e) ? 1.f : 0.f);
  });
  // Reflector k (acting on indices k+1..N-1) is stored at row[voff(k) ..],
  // its beta at row[NP - 1 - k]; the staged input is already in registers.
  auto voff = [](int k) { return k * (N - 1) - k * (k - 1) / 2; };
  float d[N], e[N];
  static_for<(N > 2 ? N - 2 : 0)>([&](auto kk) {
    constexpr int k = decltype(kk)::value;
    constexpr int m = N - k - 1;
    float v[m], p[m];
    float s2 = 0.f;
    static_for<m>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      v[i] = a[pk(k, k + 1 + i)];
      s2 = fmaf(v[i], v[i], s2);
    });
    const float x0 = v[0];
    const float nx = s2 > 0.f ? s2 * rsqrtf(s2) : 0.f;
    const float alpha = x0 >= 0.f ? -nx : nx;
    v[0] = x0 - alpha;                                   // |v0| = |x0| + |x|
    const float vtv = 2.f * nx * (nx + fabsf(x0));
    const bool refl = vtv > 1e-30f;
    const float beta = refl ? __fdividef(2.f, vtv) : 0.f;
    d[k] = a[pk(k, k)];
    e[k] = refl ? alpha : x0;
    static_for<m>([&](auto ii) { sts(rowa + 4 * (voff(k) + decltype(ii)::value), v[decltype(ii)::value]); });
    sts(rowa + 4 * (NP - 1 - k), beta);
    // p = beta A' v over the trailing block (packed, each entry used twice)
    static_for<m>([&](auto ii) { p[decltype(ii)::value] = 0.f; });
    static_for<m>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      static_for<m - i>([&](auto jj) {
        constexpr int j = i + decltype(jj)::value;
        const float aij = a[pk(k + 1 + i, k + 1 + j)];
        p[i] = fmaf(aij, v[j], p[i]);
        if constexpr (j != i) p[j] = fmaf(aij, v[i], p[j]);
      });
    });
    float vp = 0.f;
    static_for<m>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      p[i] *= beta;
      vp = fmaf(v[i], p[i], vp);
    });
    const float kh = 0.5f * beta * vp;
    static_for<m>([&](auto ii) { p[decltype(ii)::value] = fmaf(-kh, v[decltype(ii)::value], p[decltype(ii)::value]); });
    // A' -= v w^T + w v^T (w in p)
    static_for<m>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      static_for<m - i>([&](auto jj) {
        constexpr int j = i + decltype(jj)::value;
        float& x = a[pk(k + 1 + i, k + 1 + j)];
        x = fmaf(-v[i], p[j], fmaf(-p[i], v[j], x));
      });
    });
  });
  d[N - 2] = a[pk(N - 2, N - 2)];
  d[N - 1] = a[pk(N - 1, N - 1)];
  e[N - 2] = a[pk(N - 2, N - 1)];
  e[N - 1] = 0.f;
  float td[N], te[N];
  static_for<N>([&](auto ii) {
    td[decltype(ii)::value] = d[decltype(ii)::value];
    te[decltype(ii)::value] = e[decltype(ii)::value];
  });

  // Implicit QR on T. |e| <= 1e-6 ||T||_F counts as zero: by Weyl's
  // inequality this moves no eigenvalue by more than 1e-6 sqrt(N) lambda_max.
  float an2 = 0.f;
  static_for<N>([&](auto ii) {
    constexpr int i = decltype(ii)::value;
    an2 = fmaf(d[i], d[i], an2);
    if constexpr (i < N - 1) an2 = fmaf(2.f * e[i], e[i], an2);
  });
  const float thr2 = 1e-12f * an2;
  int steps = 0;
  if constexpr (!kCompact) {
    // one unrolled copy of the QR step per deflation level m: the warp
    // moves to the next level once every lane has deflated this one
    static_for<N - 1>([&](auto mm) {
      constexpr int m = N - 1 - decltype(mm)::value;
      for (int it = 0; it < kMaxQrIter; ++it) {
        const bool need = active && e[m - 1] * e[m - 1] > thr2;
        if (!__any_sync(0xffffffffu, need)) break;
        if (need) {
          int l = 0;  // top of the unreduced block that ends at m
          static_for<m - 1>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            if (e[i] * e[i] <= thr2) l = i + 1;
          });
          qr_step<N>(d, e, l, m, d[m - 1], d[m], e[m - 1]);
          ++steps;
        }
      }
    });
  } else {
    // one copy of the step over the whole length, masked to each lane's
    // unreduced block [l, m]: lanes deflate at their own pace
    for (int it = 0; it < kMaxQrIter * (N - 1); ++it) {
      // one pass from the top: m is one past the last non-negligible e
      // (the bottom of the lowest unreduced block), l one past the last
      // negligible e above it (its top)
      int m = 0, l = 0, last_small = 0;
      float dm1 = 0.f, dm = 0.f, em = 0.f;
      static_for<N - 1>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        if (e[i] * e[i] > thr2) {
          m = i + 1;
          l = last_small;
          dm1 = d[i];
          dm = d[i + 1];
          em = e[i];
        } else {
          last_small = i + 1;
        }
      });
      const bool need = active && m > 0;
      if (!__any_sync(0xffffffffu, need)) break;
      // The lowest unreduced block moves up as eigenvalues deflate; the
      // warp's deepest block bounds the positions a step can touch, so
      // copies of the step over the first third and two thirds of the
      // positions serve the later steps (same arithmetic, fewer masked
      // positions issued).
      const int mw = __reduce_max_sync(0xffffffffu, need ? m : 0);
      if (need) {
        if constexpr (N - 1 >= 6) {
          constexpr int K1 = (N - 1) / 3, K2 = 2 * (N - 1) / 3;
          if (mw <= K1)
            qr_step<N, K1>(d, e, l, m, dm1, dm, em);
          else if (mw <= K2)
            qr_step<N, K2>(d, e, l, m, dm1, dm, em);
          else
            qr_step<N>(d, e, l, m, dm1, dm, em);
        } else {
          qr_step<N>(d, e, l, m, dm1, dm, em);
        }
        ++steps;
      }
    }
  }
  if (step_count) {
    const int wmax = __reduce_max_sync(0xffffffffu, steps);
    const unsigned wsum = __reduce_add_sync(0xffffffffu, (unsigned)steps);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&step_count[0], (unsigned long long)wsum);
      atomicAdd(&step_count[1], (unsigned long long)wmax);
    }
  }
  // odd-even transposition sort, descending
  static_for<N>([&](auto pp) {
    constexpr int pass = decltype(pp)::value;
    static_for<(N - (pass & 1)) / 2>([&](auto kk) {
      constexpr int k = (pass & 1) + 2 * decltype(kk)::value;
      const float hi = fmaxf(d[k], d[k + 1]), lo = fminf(d[k], d[k + 1]);
      d[k] = hi;
      d[k + 1] = lo;
    });
  });
  if (!active) return;
  const int64_t cell = cell0 + threadIdx.x;
  float ss = 0.f;
  static_for<N>([&](auto kk) { ss = fmaf(d[decltype(kk)::value], d[decltype(kk)::value], ss); });
  stat[cell] = ss > 0.f ? d[0] * d[0] / ss : 0.f;
  if (evals) static_for<N>([&](auto kk) { evals[cell * N + decltype(kk)::value] = d[decltype(kk)::value]; });
  if (!q1) return;

  // q1: inverse iteration with sigma I - T = L D L^T (sigma just above
  // lambda_1, so every pivot is positive), then x = Q y.
  const float lambda1 = d[0];
  float delta = fmaxf(4e-5f * fabsf(lambda1), 1e-6f);
  float dinv[N], lo[N];
  bool ok = false;
  for (int attempt = 0; attempt < 4 && !ok; ++attempt, delta *= 16.f) {
    const float sig = lambda1 + delta;
    ok = true;
    float piv = sig - td[0];
    static_for<N>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      if constexpr (i > 0) {
        const float l = -te[i - 1] * dinv[i - 1];
        lo[i] = l;
        piv = fmaf(-l * l, piv, sig - td[i]);
      }
      ok = ok && piv > 0.f;
      dinv[i] = __fdividef(1.f, fmaxf(piv, 1e-30f));
    });
  }
  float y[N];
  static_for<N>([&](auto ii) {
    constexpr int i = decltype(ii)::value;
    y[i] = 1.f + 0.25f * (float)((i * 7) % 5);
  });
  for (int it = 0; it < 3; ++it) {
    static_for<N - 1>([&](auto ii) {
      constexpr int i = decltype(ii)::value + 1;
      y[i] = fmaf(-lo[i], y[i - 1], y[i]);
    });
    static_for<N>([&](auto ii) { y[decltype(ii)::value] *= dinv[decltype(ii)::value]; });
    static_for<N - 1>([&](auto ii) {
      constexpr int i = N - 2 - decltype(ii)::value;
      y[i] = fmaf(-lo[i + 1], y[i + 1], y[i]);
    });
    float nn = 0.f;
    static_for<N>([&](auto ii) { nn = fmaf(y[decltype(ii)::value], y[decltype(ii)::value], nn); });
    const float inv = rsqrtf(fmaxf(nn, 1e-37f));
    static_for<N>([&](auto ii) { y[decltype(ii)::value] *= inv; });
  }
  // x = H_0 H_1 ... H_{N-3} y, the last reflector first
  static_for<(N > 2 ? N - 2 : 0)>([&](auto kk) {
    constexpr int k = N - 3 - decltype(kk)::value;
    constexpr int m = N - k - 1;
    float vk[m];
    float t = 0.f;
    static_for<m>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      vk[i] = lds(rowa + 4 * (voff(k) + i));
      t = fmaf(vk[i], y[k + 1 + i], t);
    });
    t *= lds(rowa + 4 * (NP - 1 - k));
    static_for<m>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      y[k + 1 + i] = fmaf(-t, vk[i], y[k + 1 + i]);
    });
  });
  float best = 0.f, sgn = 1.f;
  static_for<N>([&](auto kk) {
    const float v = y[decltype(kk)::value];
    if (fabsf(v) > best) {
      best = fabsf(v);
      sgn = v < 0.f ? -1.f : 1.f;
    }
  });
  if (!ok) sgn = __int_as_float(0x7fc00000);  // NaN marks a failed factor
  static_for<N>([&](auto kk) { q1[cell * N + decltype(kk)::value] = sgn * y[decltype(kk)::value]; });
}

// ---------------------------------------------------------------------------
// Split tridiagonal route (variant 4): the same arithmetic as the route
// above in two kernels. The one-kernel route holds the whole packed matrix
// in registers during the reduction (255 registers, 8 warps per SM), and the
// implicit QR steps that follow, two thirds of its time on the FAST block
// (0.36 ms reduction, 1.03 ms QR, 0.13 ms q1), ran at that occupancy too.
// Here the reduction kernel writes T (d and e, [2N][cell]) and finds
// lambda_1 of T itself, by Newton's method on det(T - x I) from Gershgorin's
// upper bound: above every eigenvalue the pivots of T - x I are all
// negative, (log det)' = sum_j 1 / (x - lambda_j), and the iterates fall
// monotonically to lambda_1, so sigma = lambda_1 + delta for the inverse
// iteration stays above it. It then computes q1 while the reflectors are in
// its shared memory. A second kernel with a few dozen registers runs QR on
// T for all eigenvalues at several times the occupancy.
constexpr int kNewtonMax = 40;
constexpr int kEigQrThreads = 128;

template <int N>
__global__ void __launch_bounds__(kEigThreads)
eig_tri_a_kernel(const float* __restrict__ corr, int64_t n_cells, float* __restrict__ de,
                 float* __restrict__ q1) {
  constexpr int NP = Slots<N>::NP;
  constexpr int STR = Slots<N>::STR;
  extern __shared__ float sm[];
  const int64_t cell0 = (int64_t)blockIdx.x * kEigThreads;
  const int ncell = (int)min((int64_t)kEigThreads, n_cells - cell0);
  stage_rows<NP, STR>(sm, corr + cell0 * NP, ncell);
  const bool active = (int)threadIdx.x < ncell;
  float* row = sm + threadIdx.x * STR;
  const uint32_t rowa = static_cast<uint32_t>(__cvta_generic_to_shared(row));
  auto pk = [](int a, int b) { return a * N - a * (a - 1) / 2 + (b - a); };  // a <= b
  float a[NP];
  static_for<NP>([&](auto ee) {
    constexpr int e = decltype(ee)::value;
    a[e] = active ? row[e] : (Slots<N>::row_of(e) == Slots<N>::col_of(e) ? 1.f : 0.f);
  });
  // Reflector k (acting on indices k+1..N-1) is stored at row[voff(k) ..],
  // its beta at row[NP - 1 - k]; the staged input is already in registers.
  auto voff = [](int k) { return k * (N - 1) - k * (k - 1) / 2; };
  float d[N], e[N];
  static_for<(N > 2 ? N - 2 : 0)>([&](auto kk) {
    constexpr int k = decltype(kk)::value;
    constexpr int m = N - k - 1;
    float v[m], p[m];
    float s2 = 0.f;
    static_for<m>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      v[i] = a[pk(k, k + 1 + i)];
      s2 = fmaf(v[i], v[i], s2);
    });
    const float x0 = v[0];
    const float nx = s2 > 0.f ? s2 * rsqrtf(s2) : 0.f;
    const float alpha = x0 >= 0.f ? -nx : nx;
    v[0] = x0 - alpha;                                   // |v0| = |x0| + |x|
    const float vtv = 2.f * nx * (nx + fabsf(x0));
    const bool refl = vtv > 1e-30f;
    const float beta = refl ? __fdividef(2.f, vtv) : 0.f;
    d[k] = a[pk(k, k)];
    e[k] = refl ? alpha : x0;
    static_for<m>([&](auto ii) { sts(rowa + 4 * (voff(k) + decltype(ii)::value), v[decltype(ii)::value]); });
    sts(rowa + 4 * (NP - 1 - k), beta);
    // p = beta A' v over the trailing block (packed, each entry used twice)
    static_for<m>([&](auto ii) { p[decltype(ii)::value] = 0.f; });
    static_for<m>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      static_for<m - i>([&](auto jj) {
        constexpr int j = i + decltype(jj)::value;
        const float aij = a[pk(k + 1 + i, k + 1 + j)];
        p[i] = fmaf(aij, v[j], p[i]);
        if constexpr (j != i) p[j] = fmaf(aij, v[i], p[j]);
      });
    });
    float vp = 0.f;
    static_for<m>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      p[i] *= beta;
      vp = fmaf(v[i], p[i], vp);
    });
    const float kh = 0.5f * beta * vp;
    static_for<m>([&](auto ii) { p[decltype(ii)::value] = fmaf(-kh, v[decltype(ii)::value], p[decltype(ii)::value]); });
    // A' -= v w^T + w v^T (w in p)
    static_for<m>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      static_for<m - i>([&](auto jj) {
        constexpr int j = i + decltype(jj)::value;
        float& x = a[pk(k + 1 + i, k + 1 + j)];
        x = fmaf(-v[i], p[j], fmaf(-p[i], v[j], x));
      });
    });
  });
  d[N - 2] = a[pk(N - 2, N - 2)];
  d[N - 1] = a[pk(N - 1, N - 1)];
  e[N - 2] = a[pk(N - 2, N - 1)];
  e[N - 1] = 0.f;
  float td[N], te[N];
  static_for<N>([&](auto ii) {
    td[decltype(ii)::value] = d[decltype(ii)::value];
    te[decltype(ii)::value] = e[decltype(ii)::value];
  });

  if (!active) return;
  const int64_t cell = cell0 + threadIdx.x;
  // T for the QR kernel, d then e, one row of n_cells floats per entry
  static_for<N>([&](auto ii) {
    constexpr int i = decltype(ii)::value;
    de[(int64_t)i * n_cells + cell] = td[i];
    de[(int64_t)(N + i) * n_cells + cell] = te[i];
  });
  if (!q1) return;
  // lambda_1 of T: Newton on det(T - x I) from Gershgorin's upper bound
  float lam = -3.0e38f;
  static_for<N>([&](auto ii) {
    constexpr int i = decltype(ii)::value;
    float g = td[i] + fabsf(te[i]);
    if constexpr (i > 0) g += fabsf(te[i - 1]);
    lam = fmaxf(lam, g);
  });
  for (int it = 0; it < kNewtonMax; ++it) {
    // pivots q_i of T - lam I, their derivatives q_i' in lam, and
    // sum q_i' / q_i = (log det)'
    float q = td[0] - lam, dq = -1.f;
    bool hit = q == 0.f;
    float r = __fdividef(1.f, q);
    float sum = dq * r;
    static_for<N - 1>([&](auto ii) {
      constexpr int i = decltype(ii)::value + 1;
      const float e2 = te[i - 1] * te[i - 1];
      q = (td[i] - lam) - e2 * r;
      dq = fmaf(e2 * dq, r * r, -1.f);
      hit = hit || q == 0.f;
      r = __fdividef(1.f, q);
      sum = fmaf(dq, r, sum);
    });
    if (hit) break;  // lam is an eigenvalue of T, hence lambda_1
    const float step = __fdividef(1.f, sum);
    if (!(step > 0.f)) break;
    lam -= step;
    if (!(step > 1e-7f * fabsf(lam))) break;
  }

  // q1: inverse iteration with sigma I - T = L D L^T (sigma just above
  // lambda_1, so every pivot is positive), then x = Q y.
  const float lambda1 = lam;
  float delta = fmaxf(4e-5f * fabsf(lambda1), 1e-6f);
  float dinv[N], lo[N];
  bool ok = false;
  for (int attempt = 0; attempt < 4 && !ok; ++attempt, delta *= 16.f) {
    const float sig = lambda1 + delta;
    ok = true;
    float piv = sig - td[0];
    static_for<N>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      if constexpr (i > 0) {
        const float l = -te[i - 1] * dinv[i - 1];
        lo[i] = l;
        piv = fmaf(-l * l, piv, sig - td[i]);
      }
      ok = ok && piv > 0.f;
      dinv[i] = __fdividef(1.f, fmaxf(piv, 1e-30f));
    });
  }
  float y[N];
  static_for<N>([&](auto ii) {
    constexpr int i = decltype(ii)::value;
    y[i] = 1.f + 0.25f * (float)((i * 7) % 5);
  });
  for (int it = 0; it < 3; ++it) {
    static_for<N - 1>([&](auto ii) {
      constexpr int i = decltype(ii)::value + 1;
      y[i] = fmaf(-lo[i], y[i - 1], y[i]);
    });
    static_for<N>([&](auto ii) { y[decltype(ii)::value] *= dinv[decltype(ii)::value]; });
    static_for<N - 1>([&](auto ii) {
      constexpr int i = N - 2 - decltype(ii)::value;
      y[i] = fmaf(-lo[i + 1], y[i + 1], y[i]);
    });
    float nn = 0.f;
    static_for<N>([&](auto ii) { nn = fmaf(y[decltype(ii)::value], y[decltype(ii)::value], nn); });
    const float inv = rsqrtf(fmaxf(nn, 1e-37f));
    static_for<N>([&](auto ii) { y[decltype(ii)::value] *= inv; });
  }
  // x = H_0 H_1 ... H_{N-3} y, the last reflector first
  static_for<(N > 2 ? N - 2 : 0)>([&](auto kk) {
    constexpr int k = N - 3 - decltype(kk)::value;
    constexpr int m = N - k - 1;
    float vk[m];
    float t = 0.f;
    static_for<m>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      vk[i] = lds(rowa + 4 * (voff(k) + i));
      t = fmaf(vk[i], y[k + 1 + i], t);
    });
    t *= lds(rowa + 4 * (NP - 1 - k));
    static_for<m>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      y[k + 1 + i] = fmaf(-t, vk[i], y[k + 1 + i]);
    });
  });
  float best = 0.f, sgn = 1.f;
  static_for<N>([&](auto kk) {
    const float v = y[decltype(kk)::value];
    if (fabsf(v) > best) {
      best = fabsf(v);
      sgn = v < 0.f ? -1.f : 1.f;
    }
  });
  if (!ok) sgn = __int_as_float(0x7fc00000);  // NaN marks a failed factor
  static_for<N>([&](auto kk) { q1[cell * N + decltype(kk)::value] = sgn * y[decltype(kk)::value]; });
}


// kRootFree: the root-free step on the squared off-diagonals (e holds e^2)
template <int N, bool kCompact, bool kRootFree = false>
__global__ void __launch_bounds__(kEigQrThreads)
eig_qr_kernel(const float* __restrict__ de, int64_t n_cells, float* __restrict__ evals,
              float* __restrict__ stat, unsigned long long* __restrict__ step_count) {
  const int64_t cell = (int64_t)blockIdx.x * kEigQrThreads + threadIdx.x;
  const bool active = cell < n_cells;
  float d[N], e[N];
  static_for<N>([&](auto ii) {
    constexpr int i = decltype(ii)::value;
    d[i] = active ? de[(int64_t)i * n_cells + cell] : 1.f;
    e[i] = active ? de[(int64_t)(N + i) * n_cells + cell] : 0.f;
    if constexpr (kRootFree) e[i] *= e[i];
  });
  // |e| as compared below: e itself, or its square already
  auto esq = [&](float x) { return kRootFree ? x : x * x; };
  // Implicit QR on T. |e| <= 1e-5 ||T||_F counts as zero: by Weyl's
  // inequality this moves no eigenvalue by more than 1e-5 sqrt(N) lambda_max
  // (4.4e-5 lambda_max for 19 beams, inside the 1e-4 bound), and by about
  // e^2 / gap where the eigenvalues are apart. (This kernel only gives the
  // eigenvalues; q1 comes from the first kernel.)
  float an2 = 0.f;
  static_for<N>([&](auto ii) {
    constexpr int i = decltype(ii)::value;
    an2 = fmaf(d[i], d[i], an2);
    if constexpr (i < N - 1) an2 = fmaf(2.f, esq(e[i]), an2);
  });
  const float thr2 = 1e-10f * an2;
  int steps = 0;
  if constexpr (!kCompact) {
    // one unrolled copy of the QR step per deflation level m: the warp
    // moves to the next level once every lane has deflated this one
    static_for<N - 1>([&](auto mm) {
      constexpr int m = N - 1 - decltype(mm)::value;
      for (int it = 0; it < kMaxQrIter; ++it) {
        const bool need = active && esq(e[m - 1]) > thr2;
        if (!__any_sync(0xffffffffu, need)) break;
        if (need) {
          int l = 0;  // top of the unreduced block that ends at m
          static_for<m - 1>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            if (esq(e[i]) <= thr2) l = i + 1;
          });
          if constexpr (kRootFree)
            qr_step_pwk<N>(d, e, l, m, d[m - 1], d[m], e[m - 1]);
          else
            qr_step<N>(d, e, l, m, d[m - 1], d[m], e[m - 1]);
          ++steps;
        }
      }
    });
  } else {
    // one copy of the step over the whole length, masked to each lane's
    // unreduced block [l, m]: lanes deflate at their own pace
    for (int it = 0; it < kMaxQrIter * (N - 1); ++it) {
      // one pass from the top: m is one past the last non-negligible e
      // (the bottom of the lowest unreduced block), l one past the last
      // negligible e above it (its top)
      int m = 0, l = 0, last_small = 0;
      float dm1 = 0.f, dm = 0.f, em = 0.f;
      static_for<N - 1>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        if (esq(e[i]) > thr2) {
          m = i + 1;
          l = last_small;
          dm1 = d[i];
          dm = d[i + 1];
          em = e[i];
        } else {
          last_small = i + 1;
        }
      });
      const bool need = active && m > 0;
      if (!__any_sync(0xffffffffu, need)) break;
      // The lowest unreduced block moves up as eigenvalues deflate; the
      // warp's deepest block bounds the positions a step can touch, so
      // copies of the step over the first third and two thirds of the
      // positions serve the later steps (same arithmetic, fewer masked
      // positions issued).
      const int mw = __reduce_max_sync(0xffffffffu, need ? m : 0);
      if (need) {
        auto step = [&](auto kc) {
          constexpr int KK = decltype(kc)::value;
          if constexpr (kRootFree)
            qr_step_pwk<N, KK>(d, e, l, m, dm1, dm, em);
          else
            qr_step<N, KK>(d, e, l, m, dm1, dm, em);
        };
        if constexpr (N - 1 >= 6) {
          constexpr int K1 = (N - 1) / 3, K2 = 2 * (N - 1) / 3;
          if (mw <= K1)
            step(std::integral_constant<int, K1>{});
          else if (mw <= K2)
            step(std::integral_constant<int, K2>{});
          else
            step(std::integral_constant<int, N - 1>{});
        } else {
          step(std::integral_constant<int, N - 1>{});
        }
        ++steps;
      }
    }
  }
  if (step_count) {
    const int wmax = __reduce_max_sync(0xffffffffu, steps);
    const unsigned wsum = __reduce_add_sync(0xffffffffu, (unsigned)steps);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&step_count[0], (unsigned long long)wsum);
      atomicAdd(&step_count[1], (unsigned long long)wmax);
    }
  }
  // odd-even transposition sort, descending
  static_for<N>([&](auto pp) {
    constexpr int pass = decltype(pp)::value;
    static_for<(N - (pass & 1)) / 2>([&](auto kk) {
      constexpr int k = (pass & 1) + 2 * decltype(kk)::value;
      const float hi = fmaxf(d[k], d[k + 1]), lo = fminf(d[k], d[k + 1]);
      d[k] = hi;
      d[k + 1] = lo;
    });
  });
  if (!active) return;
  float ss = 0.f;
  static_for<N>([&](auto kk) { ss = fmaf(d[decltype(kk)::value], d[decltype(kk)::value], ss); });
  stat[cell] = ss > 0.f ? d[0] * d[0] / ss : 0.f;
  if (evals) static_for<N>([&](auto kk) { evals[cell * N + decltype(kk)::value] = d[decltype(kk)::value]; });
}

// ---------------------------------------------------------------------------
// Larger N (PAF-like receivers): one warp per matrix, the packed upper
// triangle in shared memory, rotated in place. Round r of the circle
// schedule pairs index M-1 with r and (r+i, r-i) mod (M-1) for i >= 1 (index
// N is a dummy when N is odd). Lanes first compute the rotations of the
// pairs and update the pairs' own 2x2 blocks, then rotate the off-diagonal
// 2x2 blocks (rows by J_i^T, columns by J_j); the warp only syncs between
// the two phases.
constexpr int kWarpEigWarps = 4;

__device__ __forceinline__ int pk_dyn(int a, int b, int N) {
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
  return a * N - a * (a - 1) / 2 + (b - a);
}

__global__ void __launch_bounds__(32 * kWarpEigWarps)
eig_warp_kernel(const float* __restrict__ corr, int64_t n_cells, int N, float* __restrict__ evals,
                float* __restrict__ q1, float* __restrict__ stat,
                unsigned long long* __restrict__ sweep_count) {
  extern __shared__ float wsm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int M = (N & 1) ? N + 1 : N, H = M / 2, NP = N * (N + 1) / 2;
  const int per_warp = NP + 4 * H + 2 * N + 32;
  float* A = wsm + (size_t)w * per_warp;   // packed matrix
  float* cs = A + NP;                      // [H][2] c, s of each pair
  int* pq = reinterpret_cast<int*>(cs + 2 * H);  // [H][2] indices (p = -1: idle pair)
  float* ev = reinterpret_cast<float*>(pq + 2 * H);  // [N] sorted eigenvalues
  float* xv = ev + N;                      // [N] 1 / U_aa of the q1 factor
  const int NBLK = H * (H - 1) / 2;
  for (int64_t cell = (int64_t)blockIdx.x * kWarpEigWarps + w; cell < n_cells;
       cell += (int64_t)gridDim.x * kWarpEigWarps) {
    const float* src = corr + cell * NP;
    const uint32_t abase = static_cast<uint32_t>(__cvta_generic_to_shared(A));
    for (int e = lane; e < NP; e += 32) cp_async4(abase + 4u * e, src + e);
    cp_async_wait_all();
    __syncwarp();
    int sweeps = 0;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
      for (int r = 0; r < M - 1; ++r) {
        // phase 1: rotations and the pairs' own blocks
        for (int i = lane; i < H; i += 32) {
          int p, q;
          if (i == 0) {
            p = r;
            q = M - 1;
          } else {
            p = (r + i) % (M - 1);
            q = (r - i + (M - 1)) % (M - 1);
          }
          if (p > q) {
            const int t = p;
            p = q;
            q = t;
          }
          if (q >= N) {  // paired with the dummy: idle
            pq[2 * i] = -1;
            pq[2 * i + 1] = p;
            cs[2 * i] = 1.f;
            cs[2 * i + 1] = 0.f;
            continue;
          }
          const float app = A[pk_dyn(p, p, N)], aqq = A[pk_dyn(q, q, N)], apq = A[pk_dyn(p, q, N)];
          float c, sn, t;
          rotation(app, aqq, apq, c, sn, t);
          A[pk_dyn(p, p, N)] = fmaf(-t, apq, app);
          A[pk_dyn(q, q, N)] = fmaf(t, apq, aqq);
          A[pk_dyn(p, q, N)] = 0.f;
          pq[2 * i] = p;
          pq[2 * i + 1] = q;
          cs[2 * i] = c;
          cs[2 * i + 1] = sn;
        }
        __syncwarp();
        // phase 2: off-diagonal 2x2 blocks (i < j)
        for (int e = lane; e < NBLK; e += 32) {
          int i = 0, rem = e;
          while (rem >= H - 1 - i) {
            rem -= H - 1 - i;
            ++i;
          }
          const int j = i + 1 + rem;
          const int pi = pq[2 * i], qi = pq[2 * i + 1], pj = pq[2 * j], qj = pq[2 * j + 1];
          const float ci = cs[2 * i], si = cs[2 * i + 1], cj = cs[2 * j], sj = cs[2 * j + 1];
          if (pi < 0 && pj < 0) continue;
          if (pi < 0) {  // row pair idle: its one real index qi, columns rotate
            const int k0 = pk_dyn(qi, pj, N), k1 = pk_dyn(qi, qj, N);
            const float y0 = A[k0], y1 = A[k1];
            A[k0] = cj * y0 - sj * y1;
            A[k1] = fmaf(sj, y0, cj * y1);
          } else if (pj < 0) {  // column pair idle: rows rotate
            const int k0 = pk_dyn(pi, qj, N), k1 = pk_dyn(qi, qj, N);
            const float y0 = A[k0], y1 = A[k1];
            A[k0] = ci * y0 - si * y1;
            A[k1] = fmaf(si, y0, ci * y1);
          } else {
            const int k00 = pk_dyn(pi, pj, N), k01 = pk_dyn(pi, qj, N);
            const int k10 = pk_dyn(qi, pj, N), k11 = pk_dyn(qi, qj, N);
            const float x00 = A[k00], x01 = A[k01], x10 = A[k10], x11 = A[k11];
            const float l00 = ci * x00 - si * x10, l01 = ci * x01 - si * x11;
            const float l10 = fmaf(si, x00, ci * x10), l11 = fmaf(si, x01, ci * x11);
            A[k00] = cj * l00 - sj * l01;
            A[k01] = fmaf(sj, l00, cj * l01);
            A[k10] = cj * l10 - sj * l11;
            A[k11] = fmaf(sj, l10, cj * l11);
          }
        }
        __syncwarp();
      }
      ++sweeps;
      float off = 0.f, dia = 0.f;
      for (int e = lane; e < NP; e += 32) {
        int a = 0, rem = e;
        while (rem >= N - a) {
          rem -= N - a;
          ++a;
        }
        const float v = A[e];
        if (rem == 0) dia = fmaf(v, v, dia);
        else off = fmaf(v, v, off);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        dia += __shfl_xor_sync(0xffffffffu, dia, o);
      }
      if (off <= kTol2 * fmaf(2.f, off, dia)) break;
    }
    if (sweep_count && lane == 0) {
      atomicAdd(&sweep_count[0], (unsigned long long)sweeps);
      atomicAdd(&sweep_count[1], (unsigned long long)sweeps);
    }
    // eigenvalues: rank sort of the diagonal, largest first
    for (int k = lane; k < N; k += 32) {
      const float v = A[pk_dyn(k, k, N)];
      int rank = 0;
      for (int m2 = 0; m2 < N; ++m2) {
        const float u = A[pk_dyn(m2, m2, N)];
        rank += (u > v) || (u == v && m2 < k);
      }
      ev[rank] = v;
    }
    __syncwarp();
    float ss = 0.f;
    for (int k = lane; k < N; k += 32) ss = fmaf(ev[k], ev[k], ss);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const float lam1 = ev[0];
    if (lane == 0) stat[cell] = ss > 0.f ? lam1 * lam1 / ss : 0.f;
    if (evals)
      for (int k = lane; k < N; k += 32) evals[cell * N + k] = ev[k];
    if (q1) {
      // inverse iteration: U^T U = sigma I - r, right-looking Cholesky by the warp
      float delta = fmaxf(4e-5f * fabsf(lam1), 1e-6f);
      bool ok = false;
      for (int attempt = 0; attempt < 4 && !ok; ++attempt, delta *= 16.f) {
        __syncwarp();
        for (int e = lane; e < NP; e += 32) {
          int a = 0, rem = e;
          while (rem >= N - a) {
            rem -= N - a;
            ++a;
          }
          A[e] = (rem == 0 ? lam1 + delta : 0.f) - src[e];
        }
        __syncwarp();
        ok = true;
        for (int a = 0; a < N; ++a) {
          const float piv = A[pk_dyn(a, a, N)];
          ok = ok && piv > 0.f;
          const float inv = rsqrtf(fmaxf(piv, 1e-30f));
          __syncwarp();
          for (int b = a + 1 + lane; b < N; b += 32) A[pk_dyn(a, b, N)] *= inv;
          if (lane == 0) {
            A[pk_dyn(a, a, N)] = piv * inv;
            xv[a] = inv;  // 1 / U_aa
          }
          __syncwarp();
          for (int b = a + 1 + lane; b < N; b += 32) {
            const float uab = A[pk_dyn(a, b, N)];
            for (int c = b; c < N; ++c) A[pk_dyn(b, c, N)] = fmaf(-uab, A[pk_dyn(a, c, N)], A[pk_dyn(b, c, N)]);
          }
          __syncwarp();
        }
      }
      // x held in registers by lane (x[k] for k = lane, lane + 32, ...)
      float xr[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = lane + 32 * u;
        xr[u] = (k < N) ? 1.f + 0.25f * (float)((k * 7) % 5) : 0.f;
      }
      for (int it = 0; it < 3 && ok; ++it) {
        // forward U^T z = x
        for (int a = 0; a < N; ++a) {
          float part = 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int k = lane + 32 * u;
            if (k < a) part = fmaf(A[pk_dyn(k, a, N)], xr[u], part);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
          if ((a & 31) == lane) xr[a >> 5] = (xr[a >> 5] - part) * xv[a];
        }
        // backward U x = z
        for (int a = N - 1; a >= 0; --a) {
          float part = 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int k = lane + 32 * u;
            if (k > a && k < N) part = fmaf(A[pk_dyn(a, k, N)], xr[u], part);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
          if ((a & 31) == lane) xr[a >> 5] = (xr[a >> 5] - part) * xv[a];
        }
        float nn = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) nn = fmaf(xr[u], xr[u], nn);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
        const float inv = rsqrtf(fmaxf(nn, 1e-37f));
#pragma unroll
        for (int u = 0; u < 4; ++u) xr[u] *= inv;
      }
      // sign rule: largest-magnitude element positive (lowest index on ties)
      float best = -1.f;
      int bi = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = lane + 32 * u;
        if (k < N && fabsf(xr[u]) > best) {
          best = fabsf(xr[u]);
          bi = k;
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
      const float vbi = __shfl_sync(0xffffffffu, xr[bi >> 5], bi & 31);
      const float sgn = ok ? (vbi < 0.f ? -1.f : 1.f) : __int_as_float(0x7fc00000);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = lane + 32 * u;
        if (k < N) q1[cell * N + k] = sgn * xr[u];
      }
    }
    __syncwarp();
  }
}

template <int N>
cudaError_t launch_reg(const float* d_corr, int64_t n_cells, float* d_evals, float* d_q1,
                       float* d_stat, unsigned long long* sweep_count, int variant, int sm_count,
                       float* d_de, cudaStream_t stream) {
  constexpr int STR = Slots<N>::STR;
  const size_t smem = (size_t)kEigThreads * STR * sizeof(float);
  const int64_t blocks = (n_cells + kEigThreads - 1) / kEigThreads;
  cudaError_t e;
  if (variant >= 4 && !d_de) variant = 3;  // no T buffer: the one-kernel route
  if (variant >= 4) {
    e = cudaFuncSetAttribute(eig_tri_a_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    if (blocks > 0)
      eig_tri_a_kernel<N><<<(unsigned)blocks, kEigThreads, smem, stream>>>(d_corr, n_cells, d_de,
                                                                             d_q1);
    const int64_t qb = (n_cells + kEigQrThreads - 1) / kEigQrThreads;
    if (qb > 0) {
      if (variant == 5)
        eig_qr_kernel<N, true, true><<<(unsigned)qb, kEigQrThreads, 0, stream>>>(
            d_de, n_cells, d_evals, d_stat, sweep_count);
      else
        eig_qr_kernel<N, true><<<(unsigned)qb, kEigQrThreads, 0, stream>>>(d_de, n_cells, d_evals,
                                                                             d_stat, sweep_count);
    }
    return cudaGetLastError();
  }
  if (variant == 2 || variant == 3) {
    auto kern = variant == 2 ? eig_tri_kernel<N, false> : eig_tri_kernel<N, true>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // Variant 2 unrolls one QR step per deflation level and its code
    // outgrows the instruction cache: it is launched one wave of resident
    // blocks at a time, so the warps of a wave walk the code together and
    // share instruction fetches (in one launch over all cells later blocks
    // drift apart and the kernel becomes bound by instruction-cache misses;
    // measured 6.9 ms against 4.3 ms on 819 200 cells of 19 beams). The
    // compact variant 3 runs as one launch.
    int64_t step = n_cells;
    if (variant == 2) {
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kEigThreads, smem);
      if (e != cudaSuccess) return e;
      step = (int64_t)(per_sm > 0 ? per_sm : 1) * sm_count * kEigThreads;
    }
    for (int64_t c0 = 0; c0 < n_cells; c0 += step) {
      const int64_t nc = (n_cells - c0) < step ? (n_cells - c0) : step;
      const int64_t bl = (nc + kEigThreads - 1) / kEigThreads;
      kern<<<(unsigned)bl, kEigThreads, smem, stream>>>(
          d_corr + c0 * Slots<N>::NP, nc, d_evals ? d_evals + c0 * N : nullptr,
          d_q1 ? d_q1 + c0 * N : nullptr, d_stat + c0, sweep_count);
    }
    return cudaGetLastError();
  }
  if (variant == 1) {
    e = cudaFuncSetAttribute(eig_reg_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    if (blocks > 0)
      eig_reg_kernel<N, true><<<(unsigned)blocks, kEigThreads, smem, stream>>>(
          d_corr, n_cells, d_evals, d_stat, sweep_count);
  } else {
    e = cudaFuncSetAttribute(eig_reg_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    if (blocks > 0)
      eig_reg_kernel<N, false><<<(unsigned)blocks, kEigThreads, smem, stream>>>(
          d_corr, n_cells, d_evals, d_stat, sweep_count);
  }
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

bool eig_needs_tri_workspace(const mraid_plan_s* pl) {
  const int N = pl->p.n_beam;
  const bool reg = N == 2 || N == 3 || N == 4 || N == 13 || N == 19;
  return !reg && pl->eig_variant >= 2;
}

bool eig_q1_needs_evals(int n_beam) { return n_beam >= 2; }

namespace {
cudaError_t launch_eig_solver(const mraid_plan_s* pl, const float* d_corr, int64_t n_cells,
                              float* d_evals, float* d_q1, float* d_stat, cudaStream_t stream) {
  const int N = pl->p.n_beam;
  switch (N) {
    case 2: return launch_reg<2>(d_corr, n_cells, d_evals, d_q1, d_stat, pl->d_sweeps, pl->eig_variant, pl->sm_count, pl->ws.de_cells >= (size_t)n_cells ? pl->ws.de : nullptr, stream);
    case 3: return launch_reg<3>(d_corr, n_cells, d_evals, d_q1, d_stat, pl->d_sweeps, pl->eig_variant, pl->sm_count, pl->ws.de_cells >= (size_t)n_cells ? pl->ws.de : nullptr, stream);
    case 4: return launch_reg<4>(d_corr, n_cells, d_evals, d_q1, d_stat, pl->d_sweeps, pl->eig_variant, pl->sm_count, pl->ws.de_cells >= (size_t)n_cells ? pl->ws.de : nullptr, stream);
    case 13: return launch_reg<13>(d_corr, n_cells, d_evals, d_q1, d_stat, pl->d_sweeps, pl->eig_variant, pl->sm_count, pl->ws.de_cells >= (size_t)n_cells ? pl->ws.de : nullptr, stream);
    case 19: return launch_reg<19>(d_corr, n_cells, d_evals, d_q1, d_stat, pl->d_sweeps, pl->eig_variant, pl->sm_count, pl->ws.de_cells >= (size_t)n_cells ? pl->ws.de : nullptr, stream);
    default: break;
  }
  if (eig_needs_tri_workspace(pl)) {
    if (!pl->ws.tri || pl->ws.tri_cells < (size_t)n_cells) return cudaErrorInvalidValue;
    return launch_eig_large(pl, d_corr, n_cells, d_evals, d_q1, d_stat, pl->ws.tri, stream);
  }
  const int M = (N & 1) ? N + 1 : N, H = M / 2, NP = N * (N + 1) / 2;
  const size_t smem = sizeof(float) * (size_t)kWarpEigWarps * (NP + 4 * H + 2 * N + 32);
  cudaError_t e = cudaFuncSetAttribute(eig_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t want = (n_cells + kWarpEigWarps - 1) / kWarpEigWarps;
  const int64_t cap = (int64_t)pl->sm_count * 32;
  const int64_t blocks = want < cap ? want : cap;
  if (blocks > 0)
    eig_warp_kernel<<<(unsigned)blocks, 32 * kWarpEigWarps, smem, stream>>>(
        d_corr, n_cells, N, d_evals, d_q1, d_stat, pl->d_sweeps);
  return cudaGetLastError();
}
}  // namespace

// The FP32 solver, then the FP64 final step of q1 on the near-degenerate
// cells (q1_refine.cu) whenever q1 is wanted (callers pass d_evals then).
cudaError_t launch_eig(const mraid_plan_s* pl, const float* d_corr, int64_t n_cells, float* d_evals,
                       float* d_q1, float* d_stat, cudaStream_t stream) {
  cudaError_t e = launch_eig_solver(pl, d_corr, n_cells, d_evals, d_q1, d_stat, stream);
  if (e != cudaSuccess || !d_q1) return e;
  if (!d_evals) return cudaErrorInvalidValue;
  return launch_q1_refine(pl, d_corr, n_cells, d_evals, d_q1,
                          pl->d_sweeps ? pl->d_sweeps + 2 : nullptr, stream);
}

cudaError_t launch_eig(const mraid_plan_s* pl, const float* d_corr, int64_t n_cells, float* d_evals,
                       float* d_q1, float* d_stat) {
  return launch_eig(pl, d_corr, n_cells, d_evals, d_q1, d_stat, pl->stream);
}

}  // namespace mraid
