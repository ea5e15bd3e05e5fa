// gram_tc.cu - exact augmented Gram sums of 8-bit multi-beam data on the
// 5th-generation tensor cores (tcgen05), fused with the correlation.
//
// Section 3.2, Eq. 1. For a cell (channel j, sub-integration k) with
// samples x_b(t), the kernel forms G = Y~ Y~^T with Y~ = [x - 128; 1]:
// the centred values x - 128 are exact in f16, every product is an integer
// of magnitude <= 2^14 and every partial sum over <= 1024 samples is an
// integer of magnitude <= 2^24, so the FP32 tensor-core accumulation is
// exact. From the centred sums, cov_ab = n G_ab - G_a G_b is exact in int64
// (it does not depend on the centring) and r_ab = cov_ab / sqrt(var_a var_b)
// is rounded to float once. The raw uint8 sums, when requested, follow from
// S_ab = G_ab + 128 (G_a + G_b) + 128^2 n and S_a = G_a + 128 n.
//
// Data flow per persistent CTA (one per SM), warp-specialised:
//   warp 0    TMA: box {16 channels, 32 samples, N beams} of u8 into a ring
//             as deep as shared memory allows (cp.async.bulk.tensor, mbarrier
//             transaction count), so streaming continues through epilogues;
//   warps 4-7 convert each box to centred f16 operand tiles in the
//             MN-major canonical layout (8 channels x 8 samples per core
//             matrix) into a 2-deep ring. A slot is one beam (slot N is the
//             row of ones) across the 8 channels of a group; the slots are
//             laid out as [g0 0..15][g0 16..N][g1 16..N][g1 0..15];
//   warp 1    one thread issues tcgen05.mma (kind::f16, FP32 accumulate in
//             TMEM): per group D1 = A(slots 0..15) x B(slots 0..N)^T, and
//             for N >= 16 one D2 = A x B^T over the two groups' slots
//             16..N together (the layout puts them side by side), so the
//             extra rows cost one MMA instead of two half-empty ones; the
//             useful entries of D are those with equal channel and group;
//   warps 8-11 read TMEM (tcgen05.ld), keep each row's own-channel entries,
//             and write the packed correlation (and optionally the sums).
// Every wait is bounded (~2 s on the global timer); on expiry the kernel
// records an error word, drains its in-flight copies and MMAs (again
// bounded), frees its TMEM and returns.
//
// gram_tc_f32_kernel (below) runs the same pipeline on float32 samples,
// split into bf16 high and low parts on the way into shared memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "internal.h"
#include "tc_ptx.h"

namespace mraid {
namespace {

constexpr int kBoxCh = 16;             // channels per TMA box (16 bytes)
constexpr int kGroupSlots = 24;        // slots of an 8-channel group at most (N + 1 <= 24)
constexpr int kMaxNU = 16;             // u8 ring depth bound (sized at launch)
constexpr int kMaxNF = 4;              // f16 ring depth bound
constexpr size_t kSmemBudget = 227 * 1024;

// Tile shape of one kernel variant: T samples per stage, NF f16 stages.
template <int T_, int NF_, int U_ = 1>
struct TcCfg {
  static constexpr int kT = T_;
  static constexpr int kNF = NF_;
  static constexpr int kUnroll = U_;  // converter loop unrolling
  static constexpr int kSlotBytes = kT * 16;  // one slot: kT samples x 8 channels x f16
  static_assert(kT % 16 == 0 && NF_ <= kMaxNF, "bad variant");
};
constexpr int kThreads = 384;
constexpr int kConvThreads = 128;
constexpr int kEpiThreads = 128;
constexpr uint32_t kTmemCols = 512;

struct TcArgs {
  int n_beam, n_chan, n_samp_sub, sub0, n_sub;
  int n_pol;   // 2: blocks b and N + b are two polarisations of beam b, summed
  int center;  // subtracted before f16: 128 (one polarisation), 255 (sum of two)
  int piece_stages;  // stages per TMEM accumulation; the epilogue adds the pieces
  int n_u8;  // u8 ring depth (stages), fixed at launch with the shared-memory size
  int R;    // slots per group: N + 1
  int R2;   // slots 16..N per group (0 if N + 1 <= 16)
  int rb;   // slots in B of the first MMAs (R rounded up to even)
  int64_t* sums;
  int64_t* sums8;  // the same sums as [cell / 8][P][cell % 8] (internal layout)
  float* corr;
  unsigned long long* degenerate;
  unsigned* error;
  unsigned long long wait_ns;  // bound of every wait (the plan's wait limit)
  long long withhold;  // fault injection: CTA 0's TMA producer never issues this stage (-1: none)
};

// Keep the 4 entries of a 32-column chunk whose channel equals c (columns
// 8u + c, u = 0..3) with compile-time register indices.
__device__ __forceinline__ void pick4(const uint32_t (&v)[32], int c, float* out) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    uint32_t x = v[8 * u];
#pragma unroll
    for (int k = 1; k < 8; ++k) x = (c == k) ? v[8 * u + k] : x;
    out[u] = __uint_as_float(x);
  }
}

// Slot position in an f16 stage: [g0 0..15][g0 16..R-1][g1 16..R-1][g1 0..15].
__device__ __forceinline__ int slot_pos(int grp, int slot, int R, int R2) {
  return grp == 0 ? slot : (slot < 16 ? R + R2 + slot : R + slot - 16);
}
// Beam slot of column block j of a group's first MMA (B = positions
// 0..R-1 for group 0, R..2R-1 for group 1).
__device__ __forceinline__ int d1_slot(int grp, int j, int R2) {
  return grp == 0 ? j : (j < R2 ? 16 + j : j - R2);
}

struct Smem {
  uint64_t u8_full[kMaxNU], u8_empty[kMaxNU];
  uint64_t f16_full[kMaxNF], f16_empty[kMaxNF];
  uint64_t acc_full, acc_empty, drain;
  int epi_go;  // the epilogue leader's wait outcome
  uint32_t tmem_base;
  int32_t s_sum[2][8][kGroupSlots];   // centred row sums G_a per group/channel/slot
  float s_inv[2][8][kGroupSlots];     // 1/sqrt(var_a), 0 if var_a == 0
};

// Slots of one f16 stage for n_beam beams: both groups (2R positions, one
// more for the even B width when R is odd) and at least the 32 positions
// the extra-slot MMA reads.
__host__ __device__ constexpr int stage_slots(int n_beam) {
  return (2 * (n_beam + 1) + ((n_beam + 1) & 1)) > 32 ? (2 * (n_beam + 1) + ((n_beam + 1) & 1)) : 32;
}
template <class C>
__host__ __device__ constexpr size_t f16_stage_bytes(int n_beam) {
  return (size_t)stage_slots(n_beam) * C::kSlotBytes;
}
// u8 ring depth for n_beam beams (n_pol blocks each): as deep as the
// shared memory allows, so TMA keeps streaming while the MMAs pause for an
// epilogue
template <class C>
__host__ __device__ constexpr int u8_ring_depth(int n_beam, int n_pol = 1) {
  return (int)((kSmemBudget - 1024 - (size_t)C::kNF * f16_stage_bytes<C>(n_beam) - sizeof(Smem)) /
               ((size_t)n_pol * n_beam * C::kT * kBoxCh)) < kMaxNU
             ? (int)((kSmemBudget - 1024 - (size_t)C::kNF * f16_stage_bytes<C>(n_beam) -
                      sizeof(Smem)) /
                     ((size_t)n_pol * n_beam * C::kT * kBoxCh))
             : kMaxNU;
}
// dynamic shared memory for n_beam beams and a ring of n_u8 stages
template <class C>
__host__ __device__ constexpr size_t smem_bytes(int n_beam, int n_u8, int n_pol = 1) {
  return 1024 /* alignment slack */ + (size_t)C::kNF * f16_stage_bytes<C>(n_beam) +
         (size_t)n_u8 * n_pol * n_beam * C::kT * kBoxCh + sizeof(Smem);
}

// kPol 2: the two-polarisation mode (converter adds blocks b and N + b;
// the epilogue adds the TMEM pieces of a sub-integration as integers)
template <int T_, int NF_, int U_, int kPol>
__global__ void __launch_bounds__(kThreads, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, TcArgs g) {
  using C = TcCfg<T_, NF_, U_>;
  constexpr int kT = C::kT, kNF = C::kNF, kSlotBytes = C::kSlotBytes;
  const int kF16StageBytes = (int)f16_stage_bytes<C>(g.n_beam);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kNU = g.n_u8;
  unsigned char* f16 = base;                                   // kNF stages
  unsigned char* u8 = f16 + (size_t)kNF * kF16StageBytes;      // kNU stages
  const int u8_stage_bytes = g.n_pol * g.n_beam * kT * kBoxCh;
  Smem* s = reinterpret_cast<Smem*>(u8 + (size_t)kNU * u8_stage_bytes);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int N = g.n_beam;
  const int chunks = g.n_chan / kBoxCh;
  const int64_t items = (int64_t)g.n_sub * chunks;
  const int stages = g.n_samp_sub / kT;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kNU; ++i) {
      mbar_init(&s->u8_full[i], 1);
      mbar_init(&s->u8_empty[i], kConvThreads);
    }
    for (int i = 0; i < kNF; ++i) {
      mbar_init(&s->f16_full[i], kConvThreads);
      mbar_init(&s->f16_empty[i], 1);
    }
    mbar_init(&s->acc_full, 1);
    mbar_init(&s->acc_empty, kEpiThreads);
    mbar_init(&s->drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // constant slots of every f16 stage: the rows of ones (slot N of each
  // group) and zeros everywhere the converter does not write
  const uint32_t one2 = 0x3c003c00u;  // f16x2 (1.0, 1.0)
  const int p_one0 = slot_pos(0, N, g.R, g.R2), p_one1 = slot_pos(1, N, g.R, g.R2);
  for (int st = 0; st < kNF; ++st) {
    uint32_t* w = reinterpret_cast<uint32_t*>(f16 + (size_t)st * kF16StageBytes);
    for (int i = threadIdx.x; i < kF16StageBytes / 4; i += blockDim.x) {
      const int pos = i / (kSlotBytes / 4);
      w[i] = (pos == p_one0 || pos == p_one1) ? one2 : 0u;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s->tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  fence_after();
  const uint32_t tmem = s->tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA
    if (lane == 0) {
      uint32_t cnt = 0;
      long long withheld = -1;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int k = (int)(it / chunks), ch0 = (int)(it % chunks) * kBoxCh;
        const int64_t t_item = (int64_t)(g.sub0 + k) * g.n_samp_sub;
        for (int st = 0; st < stages && ok; ++st, ++cnt) {
          const int slot = cnt % kNU;
          ok = mbar_wait(&s->u8_empty[slot], ((cnt / kNU) & 1) ^ 1, g.error, g.wait_ns);
          if (!ok) break;
          if (blockIdx.x == 0 && (long long)cnt == g.withhold) {
            // injected fault: this stage is never issued, so the converter's
            // bounded wait for it expires (nothing is in flight for it)
            withheld = cnt;
            continue;
          }
          mbar_expect_tx(&s->u8_full[slot], (uint32_t)u8_stage_bytes);
          tma_load_3d(u8 + (size_t)slot * u8_stage_bytes, &tmap, ch0, (int)(t_item + st * kT), 0,
                      &s->u8_full[slot]);
        }
      }
      // drain: every issued copy has landed before the CTA may exit
      for (uint32_t d = cnt > kNU ? cnt - kNU : 0; d < cnt; ++d)
        if ((long long)d != withheld)
          mbar_drain(&s->u8_full[d % kNU], (d / kNU) & 1, g.error, g.wait_ns);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA
    if (lane == 0) {
      const uint32_t f16_base = smem_u32(f16);
      const uint32_t id1 = idesc_f16(128, 8 * g.rb);
      const uint32_t id2 = idesc_f16(128, g.R2 > 0 ? 16 * g.R2 : 16);
      const uint32_t pa1 = (uint32_t)(g.R + g.R2) * kSlotBytes;  // group 1: A1 and B1
      const uint32_t pb1 = (uint32_t)g.R * kSlotBytes;
      // no-swizzle canonical layout: K-adjacent core matrices 128 B apart,
      // MN-adjacent (next slot) kSlotBytes apart
      const uint32_t lbo = 128, sbo = kSlotBytes;
      uint32_t fcnt = 0, pcnt = 0;  // stages and accumulation pieces issued
      bool ok = true;
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
        for (int st = 0; st < stages && ok; ++st, ++fcnt) {
          const int fs = fcnt % kNF;
          // stage within the TMEM accumulation piece (the whole item for one
          // polarisation)
          int ps = st;
          if constexpr (kPol == 2) ps = st % g.piece_stages;
          const int last = kPol == 2 ? g.piece_stages - 1 : stages - 1;
          ok = mbar_wait(&s->f16_full[fs], (fcnt / kNF) & 1, g.error, g.wait_ns);
          if (!ok) break;
          if (ps == 0 && pcnt > 0) {
            ok = mbar_wait(&s->acc_empty, (pcnt - 1) & 1, g.error, g.wait_ns);
            if (!ok) break;
          }
          fence_after();
          const uint32_t stage_addr = f16_base + (uint32_t)(fs * kF16StageBytes);
          // TMEM: D1 of group 0 at column 0, of group 1 at 192, D2 at 384
#pragma unroll
          for (int ks = 0; ks < kT / 16; ++ks) {
            const uint32_t a = stage_addr + ks * 256;  // 16 samples = two 128-byte core matrices
            const uint32_t acc = (ps > 0 || ks > 0) ? 1u : 0u;
            mma_f16(tmem, smem_desc(a, lbo, sbo), smem_desc(a, lbo, sbo), id1, acc);
            mma_f16(tmem + 192, smem_desc(a + pa1, lbo, sbo), smem_desc(a + pb1, lbo, sbo), id1,
                    acc);
            if (g.R2 > 0)
              mma_f16(tmem + 384, smem_desc(a + 16 * kSlotBytes, lbo, sbo),
                      smem_desc(a + 16 * kSlotBytes, lbo, sbo), id2, acc);
          }
          mma_commit(&s->f16_empty[fs]);  // stage buffer free once these MMAs finish
          if (ps == last) {
            mma_commit(&s->acc_full);
            ++pcnt;
          }
        }
      }
      mma_commit(&s->drain);  // every MMA issued has finished before TMEM is freed
      mbar_drain(&s->drain, 0, g.error, g.wait_ns);
    }
  } else if (warp >= 4 && warp < 8) {
    // ------------------------------------------------------------ convert
    const int ct = threadIdx.x - 4 * 32;
    const uint32_t magic = 0x64646464u;   // f16 bit pattern 0x64xx = 1024 + x
    const uint32_t bias = 0x64806480u;    // f16x2 (1152, 1152)
    const uint32_t bias2 = 0x64ff64ffu;   // f16x2 (1279, 1279): two polarisations
    uint32_t cnt = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
      for (int st = 0; st < stages && ok; ++st, ++cnt) {
        const int us = cnt % kNU, fs = cnt % kNF;
        ok = mbar_wait(&s->u8_full[us], (cnt / kNU) & 1, g.error, g.wait_ns);
        if (ok) ok = mbar_wait(&s->f16_empty[fs], ((cnt / kNF) & 1) ^ 1, g.error, g.wait_ns);
        if (!ok) break;
        const uint4* src = reinterpret_cast<const uint4*>(u8 + (size_t)us * u8_stage_bytes);
        unsigned char* dst = f16 + (size_t)fs * kF16StageBytes;
        if constexpr (kPol == 2) {
          // total power of two polarisations: x = p0 + p1 (0..510) in
          // 16-bit lanes; f16 0x6400 | x = 1024 + x, minus 1279 gives
          // x - 255 exactly (|x - 255| <= 255)
          for (int r = ct; r < N * kT; r += kConvThreads) {
            const uint4 wa = src[r], wb = src[r + N * kT];
            const int b = r / kT, t = r % kT;
            const uint32_t off = (t / 8) * 128 + (t % 8) * 16;
            const uint32_t off0 = (uint32_t)b * kSlotBytes + off;
            const uint32_t off1 = (uint32_t)slot_pos(1, b, g.R, g.R2) * kSlotBytes + off;
            auto two = [&](uint32_t x, uint32_t y, uint32_t sel) {
              const uint32_t v = (__byte_perm(x, 0u, sel) + __byte_perm(y, 0u, sel)) | 0x64006400u;
              uint32_t o;
              asm("sub.f16x2 %0, %1, %2;" : "=r"(o) : "r"(v), "r"(bias2));
              return o;
            };
            const uint4 o0 = make_uint4(two(wa.x, wb.x, 0x4140), two(wa.x, wb.x, 0x4342),
                                        two(wa.y, wb.y, 0x4140), two(wa.y, wb.y, 0x4342));
            const uint4 o1 = make_uint4(two(wa.z, wb.z, 0x4140), two(wa.z, wb.z, 0x4342),
                                        two(wa.w, wb.w, 0x4140), two(wa.w, wb.w, 0x4342));
            *reinterpret_cast<uint4*>(dst + off0) = o0;
            *reinterpret_cast<uint4*>(dst + off1) = o1;
          }
        } else {
#pragma unroll C::kUnroll
        for (int r = ct; r < N * kT; r += kConvThreads) {
          const uint4 w = src[r];  // 16 channels of beam b at sample t
          const int b = r / kT, t = r % kT;
          const uint32_t off = (t / 8) * 128 + (t % 8) * 16;
          const uint32_t off0 = (uint32_t)b * kSlotBytes + off;
          const uint32_t off1 = (uint32_t)slot_pos(1, b, g.R, g.R2) * kSlotBytes + off;
          uint4 o0, o1;
          asm("sub.f16x2 %0, %1, %2;" : "=r"(o0.x) : "r"(__byte_perm(w.x, magic, 0x4140)), "r"(bias));
          asm("sub.f16x2 %0, %1, %2;" : "=r"(o0.y) : "r"(__byte_perm(w.x, magic, 0x4342)), "r"(bias));
          asm("sub.f16x2 %0, %1, %2;" : "=r"(o0.z) : "r"(__byte_perm(w.y, magic, 0x4140)), "r"(bias));
          asm("sub.f16x2 %0, %1, %2;" : "=r"(o0.w) : "r"(__byte_perm(w.y, magic, 0x4342)), "r"(bias));
          asm("sub.f16x2 %0, %1, %2;" : "=r"(o1.x) : "r"(__byte_perm(w.z, magic, 0x4140)), "r"(bias));
          asm("sub.f16x2 %0, %1, %2;" : "=r"(o1.y) : "r"(__byte_perm(w.z, magic, 0x4342)), "r"(bias));
          asm("sub.f16x2 %0, %1, %2;" : "=r"(o1.z) : "r"(__byte_perm(w.w, magic, 0x4140)), "r"(bias));
          asm("sub.f16x2 %0, %1, %2;" : "=r"(o1.w) : "r"(__byte_perm(w.w, magic, 0x4342)), "r"(bias));
          *reinterpret_cast<uint4*>(dst + off0) = o0;
          *reinterpret_cast<uint4*>(dst + off1) = o1;
        }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&s->u8_empty[us]);
        mbar_arrive(&s->f16_full[fs]);
      }
    }
  } else if (warp >= 8) {
    // ------------------------------------------------------------ epilogue
    const int q = warp - 8;              // TMEM lane quarter (warp % 4)
    const int c = lane % 8;              // channel within the group
    const int slot = 4 * q + lane / 8;   // D1 row slot (beam a, 0..15), both groups
    // D2 row of this lane: stage position 16 + 4q + lane/8, which holds
    // slot 16.. of group 0, then slot 16.. of group 1, then nothing useful
    const int p2 = 4 * q + lane / 8;     // position - 16
    const int g2 = p2 < g.R2 ? 0 : (p2 < 2 * g.R2 ? 1 : -1);
    const int slot2 = 16 + (g2 == 1 ? p2 - g.R2 : p2);
    const int64_t n = g.n_samp_sub;
    const int R = g.R, R2 = g.R2;
    uint32_t pcnt = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
      // the rest of the item from the rows D1 `slot` of each group and D2
      // `slot2` (by column block): floats of exact integers (one
      // polarisation) or int32 sums of the pieces (two)
      auto finish = [&](auto& row, auto& row2) {
        // G[a][N] (row sum) and G[a][a] from each row, picked with
        // compile-time register indices and runtime block -> slot maps
        using V = std::remove_reference_t<decltype(row[0][0])>;
        V sumN[2], diag[2], sumN2 = 0, diag2 = 0;
  #pragma unroll
        for (int grp = 0; grp < 2; ++grp) {
          sumN[grp] = diag[grp] = 0;
  #pragma unroll
          for (int jb = 0; jb < kGroupSlots; ++jb) {
            const int b = d1_slot(grp, jb, R2);
            if (jb < R && b == N) sumN[grp] = row[grp][jb];
            if (jb < R && b == slot) diag[grp] = row[grp][jb];
          }
        }
        // D2 columns: blocks 0..R2-1 are group 0 slots 16.., then group 1's
        const int jb2 = g2 == 1 ? R2 : 0;
  #pragma unroll
        for (int jb = 0; jb < 16; ++jb) {
          if (jb - jb2 == N - 16) sumN2 = row2[jb];
          if (jb - jb2 == slot2 - 16) diag2 = row2[jb];
        }

        const int k = (int)(it / chunks), ch0 = (int)(it % chunks) * kBoxCh;
        // row sums and inverse standard deviations, shared through smem
        auto table = [&](int grp, int a, V sum_a, V diag_a) {
          const int64_t sa = (int64_t)sum_a;
          const int64_t var = n * (int64_t)diag_a - sa * sa;
          s->s_sum[grp][c][a] = (int32_t)sa;
          float inv = 0.f;
          if (a < N) {
            if (var > 0) {
              const float vf = (float)var;
              inv = rsqrtf(vf);
              inv = inv * (1.5f - 0.5f * vf * inv * inv);
            } else {
              atomicAdd(g.degenerate, 1ull);
            }
          }
          s->s_inv[grp][c][a] = inv;
        };
  #pragma unroll
        for (int grp = 0; grp < 2; ++grp)
          if (slot < N + 1) table(grp, slot, sumN[grp], diag[grp]);
        if (g2 >= 0 && slot2 < N + 1) table(g2, slot2, sumN2, diag2);
        named_sync(1, kEpiThreads);
        // one packed output row: a, its group, its values by column block and
        // the slot of each block (b < 0: not this group's)
        auto emit = [&](int grp, int a, const V* rv, auto nb_c, auto slot_of) {
          constexpr int NB = decltype(nb_c)::value;
          const int64_t cell = (int64_t)k * g.n_chan + ch0 + grp * 8 + c;
          const int64_t sa = s->s_sum[grp][c][a];
          const float inva = s->s_inv[grp][c][a];
          if (g.corr && a < N) {
            float* dst = g.corr + cell * (int64_t)(N * (N + 1) / 2) + (a * N - a * (a - 1) / 2);
  #pragma unroll
            for (int jb = 0; jb < NB; ++jb) {
              const int b = slot_of(jb);
              if (b < a || b >= N) continue;
              float r;
              if (b == a) {
                r = 1.f;
              } else {
                const int64_t cov = n * (int64_t)rv[jb] - sa * (int64_t)s->s_sum[grp][c][b];
                r = (float)cov * inva * s->s_inv[grp][c][b];
              }
              dst[b - a] = r;
            }
          }
          if (g.sums || g.sums8) {
            const int N1 = N + 1;
            const int64_t P = N1 * (N1 + 1) / 2;
            const int row = a * N1 - a * (a - 1) / 2;
            // public layout: one cell's entries contiguous; interleaved: the
            // 8 channels of a group side by side, so a warp's 8-byte stores
            // fill 64-byte runs
            int64_t* dst = g.sums8 ? g.sums8 + ((cell >> 3) * P + row) * 8 + (cell & 7)
                                   : g.sums + cell * P + row;
            const int step = g.sums8 ? 8 : 1;
  #pragma unroll
            for (int jb = 0; jb < NB; ++jb) {
              const int b = slot_of(jb);
              if (b < a || b > N) continue;
              const int64_t gab = (int64_t)rv[jb];
              int64_t v;
              const int64_t cc = g.center;
              if (a == N) v = n;                                  // (N, N): sample count
              else if (b == N) v = gab + cc * n;                  // S_a
              else v = gab + cc * (sa + (int64_t)s->s_sum[grp][c][b]) + cc * cc * n;
              dst[(b - a) * step] = v;
            }
          }
        };
  #pragma unroll
        for (int grp = 0; grp < 2; ++grp)
          if (slot <= N)
            emit(grp, slot, row[grp], std::integral_constant<int, kGroupSlots>{},
                 [&](int jb) { return jb < R ? d1_slot(grp, jb, R2) : -1; });
        if (g2 >= 0 && slot2 <= N)
          emit(g2, slot2, row2, std::integral_constant<int, 16>{},
               [&](int jb) { return (jb >= jb2 && jb < jb2 + R2) ? 16 + jb - jb2 : -1; });
        named_sync(1, kEpiThreads);  // smem tables reused by the next item
      };
      if constexpr (kPol == 1) {
        ok = epi_wait(&s->acc_full, pcnt & 1, g.error, g.wait_ns, &s->epi_go,
                      threadIdx.x == 256);
        if (!ok) break;
        ++pcnt;
        fence_after();
        float row[2][kGroupSlots];   // D1 row `slot` of each group, by column block
        float row2[16];              // D2 row `slot2`, by column block
#pragma unroll
        for (int grp = 0; grp < 2; ++grp) {
          // chunks of 32 columns (4 blocks x 8 channels), one load in flight
#pragma unroll
          for (int ch = 0; ch < kGroupSlots / 4; ++ch) {
            if (ch * 4 < g.rb) {
              uint32_t v[32];
              tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + grp * 192 + ch * 32, v);
              tmem_wait_ld();
              pick4(v, c, &row[grp][4 * ch]);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u) row[grp][4 * ch + u] = 0.f;
            }
          }
        }
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
          if (2 * R2 > 4 * ch) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 384 + ch * 32, v);
            tmem_wait_ld();
            pick4(v, c, &row2[4 * ch]);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) row2[4 * ch + u] = 0.f;
          }
        }
        fence_before();
        mbar_arrive(&s->acc_empty);  // accumulators may be overwritten now
        finish(row, row2);
      } else {
        // exact integer sums over the accumulation pieces (each piece's
        // sums are integers below 2^24, so exact in FP32; the total fits int32)
        const int pieces = stages / g.piece_stages;
        int32_t row[2][kGroupSlots];
        int32_t row2[16];
#pragma unroll
        for (int grp = 0; grp < 2; ++grp)
#pragma unroll
          for (int jb = 0; jb < kGroupSlots; ++jb) row[grp][jb] = 0;
#pragma unroll
        for (int jb = 0; jb < 16; ++jb) row2[jb] = 0;
        for (int pc = 0; pc < pieces && ok; ++pc, ++pcnt) {
          ok = epi_wait(&s->acc_full, pcnt & 1, g.error, g.wait_ns, &s->epi_go,
                        threadIdx.x == 256);
          if (!ok) break;
          fence_after();
#pragma unroll
          for (int grp = 0; grp < 2; ++grp) {
#pragma unroll
            for (int ch = 0; ch < kGroupSlots / 4; ++ch) {
              if (ch * 4 < g.rb) {
                uint32_t v[32];
                float f4[4];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + grp * 192 + ch * 32, v);
                tmem_wait_ld();
                pick4(v, c, f4);
#pragma unroll
                for (int u = 0; u < 4; ++u) row[grp][4 * ch + u] += __float2int_rn(f4[u]);
              }
            }
          }
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) {
            if (2 * R2 > 4 * ch) {
              uint32_t v[32];
              float f4[4];
              tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 384 + ch * 32, v);
              tmem_wait_ld();
              pick4(v, c, f4);
#pragma unroll
              for (int u = 0; u < 4; ++u) row2[4 * ch + u] += __float2int_rn(f4[u]);
            }
          }
          fence_before();
          mbar_arrive(&s->acc_empty);
        }
        if (!ok) break;
        finish(row, row2);
      }
    }
  }
  __syncthreads();
  if (warp == 2) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

// ---------------------------------------------------------------------------
// The same Gram with the A operand in tensor memory (variants 8 and 9; one
// polarisation, N + 1 <= 20 slots). In the kernel above the tensor core
// reads A (16 beam slots x 8 channels) and B from shared memory: about 96 B
// of operand reads per channel-sample, which with the TMA writes and the
// converter's traffic keeps the SM's shared-memory path ~80 % busy at half
// of HBM. Here the converter writes A straight into TMEM. ldmatrix .trans
// .b8 turns a 16-sample x 16-channel byte tile of one beam into 4
// consecutive samples of channel p and of channel p + 8 per lane (p = lane
// / 4, samples 4 (lane % 4) ..); two beams' registers (slots s, s + 1) fill
// one tcgen05.st 16x256b store, i.e. 16 TMEM lanes (8 channels x 2 slots,
// lane = 8 slot + channel) by 16 K values, which is the K-major A layout of
// kind::f16. The same registers give B in the K-major canonical layout
// (8-byte stores, a warp's 256 contiguous bytes). Only B is read from
// shared memory by the MMA, half the operand bytes. Operands go through
// sub-stages of 16 samples (one K step each): B in shared memory, A in TMEM
// columns after the accumulators (D1 of group 0 at column 0, of group 1 at
// 8 rb, D2 at 16 rb; 24 columns per sub-stage for A of group 0, group 1 and
// D2), as many sub-stages as the 512 columns leave (5 for 19 beams).
constexpr int kMaxNA = 8;  // A/B sub-stages bound
constexpr int kASub = 16;  // samples per A/B sub-stage (one K step)

__host__ __device__ constexpr int tca_g1_col(int rb) { return 8 * rb; }
__host__ __device__ constexpr int tca_d2_col(int rb) { return 16 * rb; }
__host__ __device__ constexpr int tca_a_col(int rb, int R2) { return 16 * rb + 16 * R2; }
__host__ __device__ constexpr int tca_sub_stages(int rb, int R2) {
  return ((int)kTmemCols - tca_a_col(rb, R2)) / 24 < kMaxNA
             ? ((int)kTmemCols - tca_a_col(rb, R2)) / 24
             : kMaxNA;
}
// bytes of one B sub-stage: every slot of both groups, 16 samples x 8 channels x f16
__host__ __device__ constexpr int tca_sub_bytes(int n_beam) { return stage_slots(n_beam) * 256; }

struct SmemA {
  uint64_t u8_full[kMaxNU], u8_empty[kMaxNU];
  uint64_t f16_full[kMaxNA], f16_empty[kMaxNA];
  uint64_t acc_full, acc_empty, drain;
  int epi_go;  // the epilogue leader's wait outcome
  uint32_t tmem_base;
  int32_t s_sum[2][8][kGroupSlots];
  float s_inv[2][8][kGroupSlots];
};
template <int T_>
__host__ __device__ constexpr int tca_u8_depth(int n_beam, int na) {
  return (int)((kSmemBudget - 1024 - (size_t)na * tca_sub_bytes(n_beam) - sizeof(SmemA)) /
               ((size_t)n_beam * T_ * kBoxCh)) < kMaxNU
             ? (int)((kSmemBudget - 1024 - (size_t)na * tca_sub_bytes(n_beam) - sizeof(SmemA)) /
                     ((size_t)n_beam * T_ * kBoxCh))
             : kMaxNU;
}
template <int T_>
__host__ __device__ constexpr size_t tca_smem_bytes(int n_beam, int na, int n_u8) {
  return 1024 + (size_t)na * tca_sub_bytes(n_beam) + (size_t)n_u8 * n_beam * T_ * kBoxCh +
         sizeof(SmemA);
}
__device__ __forceinline__ void mma_f16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b,
                                           uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void tmem_st16x256(uint32_t taddr, uint32_t v0, uint32_t v1, uint32_t v2,
                                              uint32_t v3) {
  asm volatile("tcgen05.st.sync.aligned.16x256b.x1.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(v0), "r"(v1), "r"(v2), "r"(v3)
               : "memory");
}
template <int T_>
__global__ void __launch_bounds__(kThreads, 1)
gram_tc_a_kernel(const __grid_constant__ CUtensorMap tmap, TcArgs g) {
  constexpr int kT = T_, kPol = 1;
  const int kNA = tca_sub_stages(g.rb, g.R2);
  const int kSubBytes = tca_sub_bytes(g.n_beam);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kNU = g.n_u8;
  unsigned char* f16 = base;                                   // kNA B sub-stages
  unsigned char* u8 = f16 + (size_t)kNA * kSubBytes;           // kNU stages
  const int u8_stage_bytes = g.n_beam * kT * kBoxCh;
  SmemA* s = reinterpret_cast<SmemA*>(u8 + (size_t)kNU * u8_stage_bytes);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int N = g.n_beam;
  const int chunks = g.n_chan / kBoxCh;
  const int64_t items = (int64_t)g.n_sub * chunks;
  const int stages = g.n_samp_sub / kT;
  const int g1c = tca_g1_col(g.rb), d2c = tca_d2_col(g.rb), ac = tca_a_col(g.rb, g.R2);

  if (threadIdx.x == 0) {
    for (int i = 0; i < kNU; ++i) {
      mbar_init(&s->u8_full[i], 1);
      mbar_init(&s->u8_empty[i], kConvThreads);
    }
    for (int i = 0; i < kNA; ++i) {
      mbar_init(&s->f16_full[i], kConvThreads);
      mbar_init(&s->f16_empty[i], 1);
    }
    mbar_init(&s->acc_full, 1);
    mbar_init(&s->acc_empty, kEpiThreads);
    mbar_init(&s->drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B sub-stages: the rows of ones (slot N of each group) and zeros where
  // the converter does not write (slots past N)
  const uint32_t one2 = 0x3c003c00u;  // f16x2 (1.0, 1.0)
  const int p_one0 = slot_pos(0, N, g.R, g.R2), p_one1 = slot_pos(1, N, g.R, g.R2);
  for (int st = 0; st < kNA; ++st) {
    uint32_t* w = reinterpret_cast<uint32_t*>(f16 + (size_t)st * kSubBytes);
    for (int i = threadIdx.x; i < kSubBytes / 4; i += blockDim.x) {
      const int pos = i / 64;  // 256 B per slot
      w[i] = (pos == p_one0 || pos == p_one1) ? one2 : 0u;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s->tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  fence_after();
  const uint32_t tmem = s->tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA
    if (lane == 0) {
      uint32_t cnt = 0;
      long long withheld = -1;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int k = (int)(it / chunks), ch0 = (int)(it % chunks) * kBoxCh;
        const int64_t t_item = (int64_t)(g.sub0 + k) * g.n_samp_sub;
        for (int st = 0; st < stages && ok; ++st, ++cnt) {
          const int slot = cnt % kNU;
          ok = mbar_wait(&s->u8_empty[slot], ((cnt / kNU) & 1) ^ 1, g.error, g.wait_ns);
          if (!ok) break;
          if (blockIdx.x == 0 && (long long)cnt == g.withhold) {
            // injected fault: this stage is never issued, so the converter's
            // bounded wait for it expires (nothing is in flight for it)
            withheld = cnt;
            continue;
          }
          mbar_expect_tx(&s->u8_full[slot], (uint32_t)u8_stage_bytes);
          tma_load_3d(u8 + (size_t)slot * u8_stage_bytes, &tmap, ch0, (int)(t_item + st * kT), 0,
                      &s->u8_full[slot]);
        }
      }
      // drain: every issued copy has landed before the CTA may exit
      for (uint32_t d = cnt > kNU ? cnt - kNU : 0; d < cnt; ++d)
        if ((long long)d != withheld)
          mbar_drain(&s->u8_full[d % kNU], (d / kNU) & 1, g.error, g.wait_ns);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA
    if (lane == 0) {
      const uint32_t f16_base = smem_u32(f16);
      const uint32_t id1 = idesc_f16_k(128, 8 * g.rb);
      const uint32_t id2 = idesc_f16_k(128, g.R2 > 0 ? 16 * g.R2 : 16);
      const uint32_t pb1 = (uint32_t)g.R * 256;  // group 1's B: positions R ..
      const uint32_t pb2 = 16u * 256;            // D2's B: positions 16 ..
      // K-major canonical layout, no swizzle: core matrices of 8 rows x 16 B,
      // K-adjacent ones 128 B apart, the next 8 rows (slot) 256 B on
      const uint32_t lbo = 128, sbo = 256;
      const int subs = stages * (kT / kASub);
      uint32_t fcnt = 0, pcnt = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
        for (int st = 0; st < subs && ok; ++st, ++fcnt) {
          const int fs = fcnt % kNA;
          ok = mbar_wait(&s->f16_full[fs], (fcnt / kNA) & 1, g.error, g.wait_ns);
          if (!ok) break;
          if (st == 0 && pcnt > 0) {
            ok = mbar_wait(&s->acc_empty, (pcnt - 1) & 1, g.error, g.wait_ns);
            if (!ok) break;
          }
          fence_after();
          const uint32_t b = f16_base + (uint32_t)(fs * kSubBytes);
          const uint32_t a = tmem + (uint32_t)(ac + 24 * fs);
          const uint32_t acc = st > 0 ? 1u : 0u;
          mma_f16_ta(tmem, a, smem_desc(b, lbo, sbo), id1, acc);
          mma_f16_ta(tmem + g1c, a + 8, smem_desc(b + pb1, lbo, sbo), id1, acc);
          if (g.R2 > 0) mma_f16_ta(tmem + d2c, a + 16, smem_desc(b + pb2, lbo, sbo), id2, acc);
          mma_commit(&s->f16_empty[fs]);  // sub-stage free once these MMAs finish
          if (st == subs - 1) {
            mma_commit(&s->acc_full);
            ++pcnt;
          }
        }
      }
      mma_commit(&s->drain);  // every MMA issued has finished before TMEM is freed
      mbar_drain(&s->drain, 0, g.error, g.wait_ns);
    }
  } else if (warp >= 4 && warp < 8) {
    // ------------------------------------------------------------ convert
    // Warp w4 = warp - 4 writes TMEM lanes 32 w4 .. 32 w4 + 31: the A rows of
    // slots 4 w4 .. 4 w4 + 3 for both groups, and of D2 positions 4 w4 ..
    // 4 w4 + 3; it writes the B rows of the beams it loads.
    const int w4 = warp - 4;
    const int p = lane / 4, q = lane % 4;
    const uint32_t u8_base = smem_u32(u8);
    const uint32_t f16_base_c = smem_u32(f16);
    // this lane's 8 bytes in a slot's 16 samples: K block q / 2, row p
    const uint32_t bq = (uint32_t)((q / 2) * 128 + p * 16 + (q % 2) * 8);
    const int ksub = kT / kASub;
    // The slots this warp converts, fixed for the launch: entries 0..3 are
    // D1 slots 4 w4 + k (both groups), entries 4..7 D2 positions 2u + h for
    // u = 2 w4 + j (j = 0, 1), of group grp. kind 0: a beam (loaded), 1: the
    // row of ones, 2: zeros (or nothing to write). src: the ldmatrix row
    // address of this lane in the slot's u8 tile; b0 / b1: this lane's B
    // bytes in a sub-stage for group 0 / 1 (entries 4..7: of their group).
    int kind[8], grp2[4];
    uint32_t src[8], b0[8], b1[4];
    bool d2_on[2];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      int slot, grp = 0;
      bool on = true;
      if (k < 4) {
        slot = 4 * w4 + k;
      } else {
        const int j = (k - 4) / 2, h = (k - 4) % 2, u = 2 * w4 + j;
        on = u < g.R2;
        if (h == 0) d2_on[j] = on;
        const int i = 2 * u + h;
        grp = i < g.R2 ? 0 : 1;
        slot = 16 + (grp ? i - g.R2 : i);
        grp2[k - 4] = grp;
      }
      kind[k] = !on ? 2 : (slot < N ? 0 : (slot == N ? 1 : 2));
      src[k] = (uint32_t)((slot < N ? slot : 0) * kT * kBoxCh + (lane & 15) * kBoxCh);
      b0[k] = (uint32_t)slot_pos(grp, slot, g.R, g.R2) * 256 + bq;
      if (k < 4) b1[k] = (uint32_t)slot_pos(1, slot, g.R, g.R2) * 256 + bq;
    }
    auto st_b = [&](uint32_t addr, uint32_t x, uint32_t y) {
      asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(x), "r"(y) : "memory");
    };
    uint32_t cnt = 0, fcnt = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
      for (int st = 0; st < stages && ok; ++st, ++cnt) {
        const int us = cnt % kNU;
        ok = mbar_wait(&s->u8_full[us], (cnt / kNU) & 1, g.error, g.wait_ns);
        if (!ok) break;
        const uint32_t u8_stage = u8_base + (uint32_t)us * (uint32_t)u8_stage_bytes;
        for (int ks = 0; ks < ksub && ok; ++ks, ++fcnt) {
          const int fs = fcnt % kNA;
          ok = mbar_wait(&s->f16_empty[fs], ((fcnt / kNA) & 1) ^ 1, g.error, g.wait_ns);
          if (!ok) break;
          fence_after();  // the MMAs that read this sub-stage's A columns have finished
          const uint32_t bsub = f16_base_c + (uint32_t)(fs * kSubBytes);
          const uint32_t acol = tmem + ((uint32_t)(32 * w4) << 16) + (uint32_t)(ac + 24 * fs);
          const uint32_t rows = u8_stage + (uint32_t)(ks * kASub * kBoxCh);
          // every load first (one latency for all), then the conversions,
          // then the B and A stores. Thread (p, q) gets samples 4q..4q+3 of
          // channels p and p + 8: f16x2 registers v[k][0..1] and v[k][2..3].
          uint32_t raw[8][2], v[8][4];
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (kind[k] == 0) ldm_trans_b8(rows + src[k], raw[k][0], raw[k][1]);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            if (kind[k] == 0) {
              u8x4_to_f16(raw[k][0], v[k][0], v[k][1]);
              u8x4_to_f16(raw[k][1], v[k][2], v[k][3]);
            } else {
              const uint32_t c1 = kind[k] == 1 ? one2 : 0u;
              v[k][0] = v[k][1] = v[k][2] = v[k][3] = c1;
            }
          }
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (kind[k] == 0) {
              st_b(bsub + b0[k], v[k][0], v[k][1]);
              st_b(bsub + b1[k], v[k][2], v[k][3]);
            }
#pragma unroll
          for (int k = 4; k < 8; ++k)
            if (kind[k] == 0) {
              const bool g1 = grp2[k - 4] != 0;
              st_b(bsub + b0[k], g1 ? v[k][2] : v[k][0], g1 ? v[k][3] : v[k][1]);
            }
          // D1 A: slots 4 w4 + 2j, + 1 -> lanes 32 w4 + 16 j ..; group 1 eight columns on
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const uint32_t lanes = (uint32_t)(16 * j) << 16;
            const int k = 2 * j;
            tmem_st16x256(acol + lanes, v[k][0], v[k][1], v[k + 1][0], v[k + 1][1]);
            tmem_st16x256(acol + lanes + 8, v[k][2], v[k][3], v[k + 1][2], v[k + 1][3]);
          }
          // D2 A: positions 2u, 2u + 1 -> lanes 16 u .., sixteen columns on
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            if (!d2_on[j]) continue;
            const int k = 4 + 2 * j;
            const bool ga = grp2[2 * j] != 0, gb = grp2[2 * j + 1] != 0;
            tmem_st16x256(acol + ((uint32_t)(16 * j) << 16) + 16, ga ? v[k][2] : v[k][0],
                          ga ? v[k][3] : v[k][1], gb ? v[k + 1][2] : v[k + 1][0],
                          gb ? v[k + 1][3] : v[k + 1][1]);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          fence_before();
          mbar_arrive(&s->f16_full[fs]);
        }
        if (!ok) break;
        mbar_arrive(&s->u8_empty[us]);
      }
    }
  } else if (warp >= 8) {
    // ------------------------------------------------------------ epilogue
    const int q = warp - 8;              // TMEM lane quarter (warp % 4)
    const int c = lane % 8;              // channel within the group
    const int slot = 4 * q + lane / 8;   // D1 row slot (beam a, 0..15), both groups
    // D2 row of this lane: stage position 16 + 4q + lane/8, which holds
    // slot 16.. of group 0, then slot 16.. of group 1, then nothing useful
    const int p2 = 4 * q + lane / 8;     // position - 16
    const int g2 = p2 < g.R2 ? 0 : (p2 < 2 * g.R2 ? 1 : -1);
    const int slot2 = 16 + (g2 == 1 ? p2 - g.R2 : p2);
    const int64_t n = g.n_samp_sub;
    const int R = g.R, R2 = g.R2;
    uint32_t pcnt = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
      // the rest of the item from the rows D1 `slot` of each group and D2
      // `slot2` (by column block): floats of exact integers (one
      // polarisation) or int32 sums of the pieces (two)
      auto finish = [&](auto& row, auto& row2) {
        // G[a][N] (row sum) and G[a][a] from each row, picked with
        // compile-time register indices and runtime block -> slot maps
        using V = std::remove_reference_t<decltype(row[0][0])>;
        V sumN[2], diag[2], sumN2 = 0, diag2 = 0;
  #pragma unroll
        for (int grp = 0; grp < 2; ++grp) {
          sumN[grp] = diag[grp] = 0;
  #pragma unroll
          for (int jb = 0; jb < kGroupSlots; ++jb) {
            const int b = d1_slot(grp, jb, R2);
            if (jb < R && b == N) sumN[grp] = row[grp][jb];
            if (jb < R && b == slot) diag[grp] = row[grp][jb];
          }
        }
        // D2 columns: blocks 0..R2-1 are group 0 slots 16.., then group 1's
        const int jb2 = g2 == 1 ? R2 : 0;
  #pragma unroll
        for (int jb = 0; jb < 16; ++jb) {
          if (jb - jb2 == N - 16) sumN2 = row2[jb];
          if (jb - jb2 == slot2 - 16) diag2 = row2[jb];
        }

        const int k = (int)(it / chunks), ch0 = (int)(it % chunks) * kBoxCh;
        // row sums and inverse standard deviations, shared through smem
        auto table = [&](int grp, int a, V sum_a, V diag_a) {
          const int64_t sa = (int64_t)sum_a;
          const int64_t var = n * (int64_t)diag_a - sa * sa;
          s->s_sum[grp][c][a] = (int32_t)sa;
          float inv = 0.f;
          if (a < N) {
            if (var > 0) {
              const float vf = (float)var;
              inv = rsqrtf(vf);
              inv = inv * (1.5f - 0.5f * vf * inv * inv);
            } else {
              atomicAdd(g.degenerate, 1ull);
            }
          }
          s->s_inv[grp][c][a] = inv;
        };
  #pragma unroll
        for (int grp = 0; grp < 2; ++grp)
          if (slot < N + 1) table(grp, slot, sumN[grp], diag[grp]);
        if (g2 >= 0 && slot2 < N + 1) table(g2, slot2, sumN2, diag2);
        named_sync(1, kEpiThreads);
        // one packed output row: a, its group, its values by column block and
        // the slot of each block (b < 0: not this group's)
        auto emit = [&](int grp, int a, const V* rv, auto nb_c, auto slot_of) {
          constexpr int NB = decltype(nb_c)::value;
          const int64_t cell = (int64_t)k * g.n_chan + ch0 + grp * 8 + c;
          const int64_t sa = s->s_sum[grp][c][a];
          const float inva = s->s_inv[grp][c][a];
          if (g.corr && a < N) {
            float* dst = g.corr + cell * (int64_t)(N * (N + 1) / 2) + (a * N - a * (a - 1) / 2);
  #pragma unroll
            for (int jb = 0; jb < NB; ++jb) {
              const int b = slot_of(jb);
              if (b < a || b >= N) continue;
              float r;
              if (b == a) {
                r = 1.f;
              } else {
                const int64_t cov = n * (int64_t)rv[jb] - sa * (int64_t)s->s_sum[grp][c][b];
                r = (float)cov * inva * s->s_inv[grp][c][b];
              }
              dst[b - a] = r;
            }
          }
          if (g.sums || g.sums8) {
            const int N1 = N + 1;
            const int64_t P = N1 * (N1 + 1) / 2;
            const int row = a * N1 - a * (a - 1) / 2;
            // public layout: one cell's entries contiguous; interleaved: the
            // 8 channels of a group side by side, so a warp's 8-byte stores
            // fill 64-byte runs
            int64_t* dst = g.sums8 ? g.sums8 + ((cell >> 3) * P + row) * 8 + (cell & 7)
                                   : g.sums + cell * P + row;
            const int step = g.sums8 ? 8 : 1;
  #pragma unroll
            for (int jb = 0; jb < NB; ++jb) {
              const int b = slot_of(jb);
              if (b < a || b > N) continue;
              const int64_t gab = (int64_t)rv[jb];
              int64_t v;
              const int64_t cc = g.center;
              if (a == N) v = n;                                  // (N, N): sample count
              else if (b == N) v = gab + cc * n;                  // S_a
              else v = gab + cc * (sa + (int64_t)s->s_sum[grp][c][b]) + cc * cc * n;
              dst[(b - a) * step] = v;
            }
          }
        };
  #pragma unroll
        for (int grp = 0; grp < 2; ++grp)
          if (slot <= N)
            emit(grp, slot, row[grp], std::integral_constant<int, kGroupSlots>{},
                 [&](int jb) { return jb < R ? d1_slot(grp, jb, R2) : -1; });
        if (g2 >= 0 && slot2 <= N)
          emit(g2, slot2, row2, std::integral_constant<int, 16>{},
               [&](int jb) { return (jb >= jb2 && jb < jb2 + R2) ? 16 + jb - jb2 : -1; });
        named_sync(1, kEpiThreads);  // smem tables reused by the next item
      };
      if constexpr (kPol == 1) {
        ok = epi_wait(&s->acc_full, pcnt & 1, g.error, g.wait_ns, &s->epi_go,
                      threadIdx.x == 256);
        if (!ok) break;
        ++pcnt;
        fence_after();
        float row[2][kGroupSlots];   // D1 row `slot` of each group, by column block
        float row2[16];              // D2 row `slot2`, by column block
#pragma unroll
        for (int grp = 0; grp < 2; ++grp) {
          // chunks of 32 columns (4 blocks x 8 channels), one load in flight
#pragma unroll
          for (int ch = 0; ch < kGroupSlots / 4; ++ch) {
            if (ch * 4 < g.rb) {
              uint32_t v[32];
              tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + grp * g1c + ch * 32, v);
              tmem_wait_ld();
              pick4(v, c, &row[grp][4 * ch]);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u) row[grp][4 * ch + u] = 0.f;
            }
          }
        }
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
          if (2 * R2 > 4 * ch) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + d2c + ch * 32, v);
            tmem_wait_ld();
            pick4(v, c, &row2[4 * ch]);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) row2[4 * ch + u] = 0.f;
          }
        }
        fence_before();
        mbar_arrive(&s->acc_empty);  // accumulators may be overwritten now
        finish(row, row2);
      } else {
        // exact integer sums over the accumulation pieces (each piece's
        // sums are integers below 2^24, so exact in FP32; the total fits int32)
        const int pieces = stages / g.piece_stages;
        int32_t row[2][kGroupSlots];
        int32_t row2[16];
#pragma unroll
        for (int grp = 0; grp < 2; ++grp)
#pragma unroll
          for (int jb = 0; jb < kGroupSlots; ++jb) row[grp][jb] = 0;
#pragma unroll
        for (int jb = 0; jb < 16; ++jb) row2[jb] = 0;
        for (int pc = 0; pc < pieces && ok; ++pc, ++pcnt) {
          ok = epi_wait(&s->acc_full, pcnt & 1, g.error, g.wait_ns, &s->epi_go,
                        threadIdx.x == 256);
          if (!ok) break;
          fence_after();
#pragma unroll
          for (int grp = 0; grp < 2; ++grp) {
#pragma unroll
            for (int ch = 0; ch < kGroupSlots / 4; ++ch) {
              if (ch * 4 < g.rb) {
                uint32_t v[32];
                float f4[4];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + grp * g1c + ch * 32, v);
                tmem_wait_ld();
                pick4(v, c, f4);
#pragma unroll
                for (int u = 0; u < 4; ++u) row[grp][4 * ch + u] += __float2int_rn(f4[u]);
              }
            }
          }
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) {
            if (2 * R2 > 4 * ch) {
              uint32_t v[32];
              float f4[4];
              tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + d2c + ch * 32, v);
              tmem_wait_ld();
              pick4(v, c, f4);
#pragma unroll
              for (int u = 0; u < 4; ++u) row2[4 * ch + u] += __float2int_rn(f4[u]);
            }
          }
          fence_before();
          mbar_arrive(&s->acc_empty);
        }
        if (!ok) break;
        finish(row, row2);
      }
    }
  }
  __syncthreads();
  if (warp == 2) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

// ---------------------------------------------------------------------------
// Float32 samples (beamformer output) on the same tensor cores. Each sample,
// shifted by its cell's first sample of the same beam and channel (the
// covariance does not depend on a per-beam shift, and the shift keeps the
// sums near zero mean so that n G_ab - G_a G_b does not cancel), is split
// into bf16 parts hi = RN(x) and lo = RN(x - hi), so x = hi + lo to a
// relative 2^-16. The four products hi hi^T, hi lo^T, lo hi^T and lo lo^T
// accumulate in FP32 in TMEM, which leaves the representation error of the
// split as the only loss beyond FP32 accumulation. Roles, stage layout,
// MMA shapes and the epilogue's walk over TMEM follow the 8-bit kernel; the
// TMA box is 16 channels x 32 samples x N beams of float32, one bf16 stage
// holds a hi tile and a lo tile of the 8-bit kernel's layout, and the
// covariance and variances are formed in FP64 from the FP32 sums. Three
// bf16 stages where the shared memory still leaves two float32 stages
// (up to 21 beams), else two; the converter handles four beams per loop
// trip so that their shared-memory loads overlap.
constexpr int kF32T = 32;              // samples per stage
constexpr int kF32MaxNF = 3;           // bf16 stages (hi + lo tiles each)
constexpr int kF32SlotBytes = kF32T * 16;
constexpr int kF32MaxNU = 8;           // float32 ring depth bound
constexpr int kF32Products = 4;

struct SmemF {
  uint64_t in_full[kF32MaxNU], in_empty[kF32MaxNU];
  uint64_t bf_full[kF32MaxNF], bf_empty[kF32MaxNF];
  uint64_t shift_full[2];
  uint64_t acc_full, acc_empty, drain;
  int epi_go;  // the epilogue leader's wait outcome
  uint32_t tmem_base;
  alignas(16) float shift[2][kGroupSlots][kBoxCh];  // by item parity: [beam][channel]
  float s_sum[2][8][kGroupSlots];                   // row sums G_a of the shifted samples
  float s_inv[2][8][kGroupSlots];                   // 1/sqrt(var_a), 0 if var_a <= 0
};

// one bf16 stage: the hi tile, then the lo tile
__host__ __device__ constexpr size_t bf_stage_bytes(int n_beam) {
  return 2 * (size_t)stage_slots(n_beam) * kF32SlotBytes;
}
__host__ __device__ constexpr size_t f32_in_stage_bytes(int n_beam) {
  return (size_t)n_beam * kF32T * kBoxCh * 4;
}
// float32 ring depth for n_beam beams and nf bf16 stages
__host__ __device__ constexpr int f32_ring_depth(int n_beam, int nf) {
  return (int)((kSmemBudget - 1024 - nf * bf_stage_bytes(n_beam) - sizeof(SmemF)) /
               f32_in_stage_bytes(n_beam)) < kF32MaxNU
             ? (int)((kSmemBudget - 1024 - nf * bf_stage_bytes(n_beam) - sizeof(SmemF)) /
                     f32_in_stage_bytes(n_beam))
             : kF32MaxNU;
}
__host__ __device__ constexpr int f32_stages(int n_beam) {
  return f32_ring_depth(n_beam, 3) >= 2 ? 3 : 2;
}
__host__ __device__ constexpr size_t f32_smem_bytes(int n_beam, int nf, int n_in) {
  return 1024 + nf * bf_stage_bytes(n_beam) + (size_t)n_in * f32_in_stage_bytes(n_beam) +
         sizeof(SmemF);
}
// Instruction descriptor, kind::f16 with bf16 A and B, f32 D, both MN-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 h) {
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <int NF>
__global__ void __launch_bounds__(kThreads, 1)
gram_tc_f32_kernel(const __grid_constant__ CUtensorMap tmap, TcArgs g) {
  const int kBfStageBytes = (int)bf_stage_bytes(g.n_beam);
  const int kTileBytes = kBfStageBytes / 2;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // offset from the shared array itself (not through an integer), so the
  // compiler keeps every derived access in the shared state space
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int kNU = g.n_u8;
  const int in_stage_bytes = (int)f32_in_stage_bytes(g.n_beam);
  unsigned char* bf = base;                                  // NF stages
  unsigned char* in = bf + (size_t)NF * kBfStageBytes;   // kNU stages of float32
  SmemF* s = reinterpret_cast<SmemF*>(in + (size_t)kNU * in_stage_bytes);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int N = g.n_beam;
  const int chunks = g.n_chan / kBoxCh;
  const int64_t items = (int64_t)g.n_sub * chunks;
  const int stages = g.n_samp_sub / kF32T;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kNU; ++i) {
      mbar_init(&s->in_full[i], 1);
      mbar_init(&s->in_empty[i], kConvThreads);
    }
    for (int i = 0; i < NF; ++i) {
      mbar_init(&s->bf_full[i], kConvThreads);
      mbar_init(&s->bf_empty[i], 1);
    }
    mbar_init(&s->shift_full[0], 4);
    mbar_init(&s->shift_full[1], 4);
    mbar_init(&s->acc_full, 1);
    mbar_init(&s->acc_empty, kEpiThreads);
    mbar_init(&s->drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // constant slots: the rows of ones in the hi tile (bf16 1.0), zeros in
  // the lo tile and everywhere the converter does not write
  const uint32_t one2 = 0x3f803f80u;  // bf16x2 (1.0, 1.0)
  const int p_one0 = slot_pos(0, N, g.R, g.R2), p_one1 = slot_pos(1, N, g.R, g.R2);
  for (int st = 0; st < NF; ++st) {
    uint32_t* w = reinterpret_cast<uint32_t*>(bf + (size_t)st * kBfStageBytes);
    for (int i = threadIdx.x; i < kBfStageBytes / 4; i += blockDim.x) {
      const int byte = i * 4;
      const int pos = byte / kF32SlotBytes;  // < stage_slots in the hi tile
      w[i] = (byte < kTileBytes && (pos == p_one0 || pos == p_one1)) ? one2 : 0u;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s->tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  fence_after();
  const uint32_t tmem = s->tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA
    if (lane == 0) {
      uint32_t cnt = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int k = (int)(it / chunks), ch0 = (int)(it % chunks) * kBoxCh;
        const int64_t t_item = (int64_t)(g.sub0 + k) * g.n_samp_sub;
        for (int st = 0; st < stages && ok; ++st, ++cnt) {
          const int slot = cnt % kNU;
          ok = mbar_wait(&s->in_empty[slot], ((cnt / kNU) & 1) ^ 1, g.error, g.wait_ns);
          if (!ok) break;
          mbar_expect_tx(&s->in_full[slot], (uint32_t)in_stage_bytes);
          tma_load_3d(in + (size_t)slot * in_stage_bytes, &tmap, ch0, (int)(t_item + st * kF32T), 0,
                      &s->in_full[slot]);
        }
      }
      for (uint32_t d = cnt > (uint32_t)kNU ? cnt - kNU : 0; d < cnt; ++d)
        mbar_drain(&s->in_full[d % kNU], (d / kNU) & 1, g.error, g.wait_ns);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA
    if (lane == 0) {
      const uint32_t bf_base = smem_u32(bf);
      const uint32_t id1 = idesc_bf16(128, 8 * g.rb);
      const uint32_t id2 = idesc_bf16(128, g.R2 > 0 ? 16 * g.R2 : 16);
      const uint32_t pa1 = (uint32_t)(g.R + g.R2) * kF32SlotBytes;  // group 1: A1 and B1
      const uint32_t pb1 = (uint32_t)g.R * kF32SlotBytes;
      const uint32_t lbo = 128, sbo = kF32SlotBytes;
      uint32_t fcnt = 0, item_iter = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x, ++item_iter) {
        for (int st = 0; st < stages && ok; ++st, ++fcnt) {
          const int fs = fcnt % NF;
          ok = mbar_wait(&s->bf_full[fs], (fcnt / NF) & 1, g.error, g.wait_ns);
          if (!ok) break;
          if (st == 0 && item_iter > 0) {
            ok = mbar_wait(&s->acc_empty, (item_iter - 1) & 1, g.error, g.wait_ns);
            if (!ok) break;
          }
          fence_after();
          const uint32_t hi = bf_base + (uint32_t)(fs * kBfStageBytes);
          const uint32_t lo = hi + (uint32_t)kTileBytes;
#pragma unroll
          for (int ks = 0; ks < kF32T / 16; ++ks) {
            // (A, B) = (hi, hi), (hi, lo), (lo, hi), (lo, lo)
#pragma unroll
            for (int pr = 0; pr < kF32Products; ++pr) {
              const uint32_t ta = ((pr & 2) ? lo : hi) + ks * 256;
              const uint32_t tb = ((pr & 1) ? lo : hi) + ks * 256;
              const uint32_t acc = (st > 0 || ks > 0 || pr > 0) ? 1u : 0u;
              mma_f16(tmem, smem_desc(ta, lbo, sbo), smem_desc(tb, lbo, sbo), id1, acc);
              mma_f16(tmem + 192, smem_desc(ta + pa1, lbo, sbo), smem_desc(tb + pb1, lbo, sbo), id1,
                      acc);
              if (g.R2 > 0)
                mma_f16(tmem + 384, smem_desc(ta + 16 * kF32SlotBytes, lbo, sbo),
                        smem_desc(tb + 16 * kF32SlotBytes, lbo, sbo), id2, acc);
            }
          }
          mma_commit(&s->bf_empty[fs]);
          if (st == stages - 1) mma_commit(&s->acc_full);
        }
      }
      mma_commit(&s->drain);  // every MMA issued has finished before TMEM is freed
      mbar_drain(&s->drain, 0, g.error, g.wait_ns);
    }
  } else if (warp >= 4 && warp < 8) {
    // ------------------------------------------------------------ convert
    // Thread ct converts, for every beam, sample t = ct / 4 of the stage
    // and channels 4q..4q+3, q = ct % 4 (one float4 of the box, so a warp
    // reads 512 contiguous bytes); its 4 values go to 8 bytes of the hi
    // tile and 8 bytes of the lo tile in channel group q / 2.
    const int ct = threadIdx.x - 4 * 32;
    const int t = ct / 4, q = ct % 4, grp = q / 2, half = q % 2;
    const uint32_t t_off = (uint32_t)((t / 8) * 128 + (t % 8) * 16 + half * 8);
    uint32_t cnt = 0, item_iter = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x, ++item_iter) {
      const int par = item_iter & 1;
      const float4* sh = reinterpret_cast<const float4*>(&s->shift[par][0][0]);
      for (int st = 0; st < stages && ok; ++st, ++cnt) {
        const int us = cnt % kNU, fs = cnt % NF;
        ok = mbar_wait(&s->in_full[us], (cnt / kNU) & 1, g.error, g.wait_ns);
        if (ok) ok = mbar_wait(&s->bf_empty[fs], ((cnt / NF) & 1) ^ 1, g.error, g.wait_ns);
        if (!ok) break;
        const float4* src = reinterpret_cast<const float4*>(in + (size_t)us * in_stage_bytes);
        if (st == 0) {
          // the item's shifts are its first samples: the threads holding
          // sample 0 publish them. The table of this parity was last read
          // two items ago, and all converter threads finished that item
          // before the bf16 stage waited on above could be free again.
          if (t == 0) {
            float4* shw = reinterpret_cast<float4*>(&s->shift[par][0][0]);
            for (int b = 0; b < N; ++b) shw[b * 4 + q] = src[b * kF32T * 4 + q];
            mbar_arrive(&s->shift_full[par]);
          }
          ok = mbar_wait(&s->shift_full[par], (item_iter >> 1) & 1, g.error, g.wait_ns);
          if (!ok) break;
        }
        unsigned char* hi = bf + (size_t)fs * kBfStageBytes;
        unsigned char* lo = hi + kTileBytes;
#pragma unroll 4
        for (int b = 0; b < N; ++b) {
          const float4 v = src[b * kF32T * 4 + ct];
          const float4 z = sh[b * 4 + q];
          const float x0 = v.x - z.x, x1 = v.y - z.y, x2 = v.z - z.z, x3 = v.w - z.w;
          const __nv_bfloat162 h01 = __floats2bfloat162_rn(x0, x1);
          const __nv_bfloat162 h23 = __floats2bfloat162_rn(x2, x3);
          const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
          const __nv_bfloat162 l01 = __floats2bfloat162_rn(x0 - f01.x, x1 - f01.y);
          const __nv_bfloat162 l23 = __floats2bfloat162_rn(x2 - f23.x, x3 - f23.y);
          const uint32_t off =
              (uint32_t)(grp == 0 ? b : slot_pos(1, b, g.R, g.R2)) * kF32SlotBytes + t_off;
          *reinterpret_cast<uint2*>(hi + off) = make_uint2(bf16x2_bits(h01), bf16x2_bits(h23));
          *reinterpret_cast<uint2*>(lo + off) = make_uint2(bf16x2_bits(l01), bf16x2_bits(l23));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&s->in_empty[us]);
        mbar_arrive(&s->bf_full[fs]);
      }
    }
  } else if (warp >= 8) {
    // ------------------------------------------------------------ epilogue
    const int qw = warp - 8;
    const int c = lane % 8;
    const int slot = 4 * qw + lane / 8;
    const int p2 = 4 * qw + lane / 8;
    const int g2 = p2 < g.R2 ? 0 : (p2 < 2 * g.R2 ? 1 : -1);
    const int slot2 = 16 + (g2 == 1 ? p2 - g.R2 : p2);
    const double n = (double)g.n_samp_sub;
    const int R = g.R, R2 = g.R2;
    uint32_t item_iter = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x, ++item_iter) {
      ok = epi_wait(&s->acc_full, item_iter & 1, g.error, g.wait_ns, &s->epi_go,
                    threadIdx.x == 256);
      if (!ok) break;
      fence_after();
      float row[2][kGroupSlots];
      float row2[16];
#pragma unroll
      for (int gi = 0; gi < 2; ++gi) {
#pragma unroll
        for (int ch = 0; ch < kGroupSlots / 4; ++ch) {
          if (ch * 4 < g.rb) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * qw) << 16) + gi * 192 + ch * 32, v);
            tmem_wait_ld();
            pick4(v, c, &row[gi][4 * ch]);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) row[gi][4 * ch + u] = 0.f;
          }
        }
      }
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) {
        if (2 * R2 > 4 * ch) {
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(32 * qw) << 16) + 384 + ch * 32, v);
          tmem_wait_ld();
          pick4(v, c, &row2[4 * ch]);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) row2[4 * ch + u] = 0.f;
        }
      }
      fence_before();
      mbar_arrive(&s->acc_empty);
      float sumN[2], diag[2], sumN2 = 0.f, diag2 = 0.f;
#pragma unroll
      for (int gi = 0; gi < 2; ++gi) {
        sumN[gi] = diag[gi] = 0.f;
#pragma unroll
        for (int jb = 0; jb < kGroupSlots; ++jb) {
          const int b = d1_slot(gi, jb, R2);
          if (jb < R && b == N) sumN[gi] = row[gi][jb];
          if (jb < R && b == slot) diag[gi] = row[gi][jb];
        }
      }
      const int jb2 = g2 == 1 ? R2 : 0;
#pragma unroll
      for (int jb = 0; jb < 16; ++jb) {
        if (jb - jb2 == N - 16) sumN2 = row2[jb];
        if (jb - jb2 == slot2 - 16) diag2 = row2[jb];
      }
      const int k = (int)(it / chunks), ch0 = (int)(it % chunks) * kBoxCh;
      auto table = [&](int gi, int a, float sum_a, float diag_a) {
        const double sa = (double)sum_a;
        const double var = n * (double)diag_a - sa * sa;
        s->s_sum[gi][c][a] = sum_a;
        float inv = 0.f;
        if (a < N) {
          if (var > 0.0) inv = (float)(1.0 / sqrt(var));
          else atomicAdd(g.degenerate, 1ull);
        }
        s->s_inv[gi][c][a] = inv;
      };
#pragma unroll
      for (int gi = 0; gi < 2; ++gi)
        if (slot < N + 1) table(gi, slot, sumN[gi], diag[gi]);
      if (g2 >= 0 && slot2 < N + 1) table(g2, slot2, sumN2, diag2);
      named_sync(1, kEpiThreads);
      auto emit = [&](int gi, int a, const float* rv, auto nb_c, auto slot_of) {
        constexpr int NB = decltype(nb_c)::value;
        if (a >= N) return;
        const int64_t cell = (int64_t)k * g.n_chan + ch0 + gi * 8 + c;
        const double sa = (double)s->s_sum[gi][c][a];
        const float inva = s->s_inv[gi][c][a];
        float* dst = g.corr + cell * (int64_t)(N * (N + 1) / 2) + (a * N - a * (a - 1) / 2);
#pragma unroll
        for (int jb = 0; jb < NB; ++jb) {
          const int b = slot_of(jb);
          if (b < a || b >= N) continue;
          float r;
          if (b == a) {
            r = 1.f;
          } else {
            const double cov = n * (double)rv[jb] - sa * (double)s->s_sum[gi][c][b];
            r = (float)cov * inva * s->s_inv[gi][c][b];
          }
          dst[b - a] = r;
        }
      };
#pragma unroll
      for (int gi = 0; gi < 2; ++gi)
        if (slot <= N)
          emit(gi, slot, row[gi], std::integral_constant<int, kGroupSlots>{},
               [&](int jb) { return jb < R ? d1_slot(gi, jb, R2) : -1; });
      if (g2 >= 0 && slot2 <= N)
        emit(g2, slot2, row2, std::integral_constant<int, 16>{},
             [&](int jb) { return (jb >= jb2 && jb < jb2 + R2) ? 16 + jb - jb2 : -1; });
      named_sync(1, kEpiThreads);
    }
  }
  __syncthreads();
  if (warp == 2) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}


}  // namespace

// Tensor-core Gram variants {samples per stage, f16 stages, converter
// unrolling}: 0 = {64, 2, 1}, 1 = {32, 4, 1}, 2 = {32, 2, 1}, 3 = {64, 3, 1},
// 4 = {64, 2, 2}, 5 = {64, 3, 2}, 6 = {64, 4, 1}, 7 = {64, 4, 2}; with A in
// TMEM (gram_tc_a_kernel, up to 19 beams): 8 = 64-sample TMA stages, 9 = 32.
int tc_variant_samples(int v) { return (v == 1 || v == 2 || v == 9) ? 32 : 64; }

// Untuned default: four f16 stages of 64 samples where that still leaves
// an u8 ring of at least three stages (measured fastest for 19 beams),
// else two.
int tc_default_variant(int n_beam) {
  if (n_beam < 2 || n_beam + 1 > kGroupSlots) return 0;
  return u8_ring_depth<TcCfg<64, 4, 1>>(n_beam) >= 3 ? 6 : 0;
}


// u8 ring depth of variant v for n_beam beams of n_pol blocks
static int tc_u8_depth(int v, int n_beam, int n_pol) {
  switch (v) {
    case 1: return u8_ring_depth<TcCfg<32, 4, 1>>(n_beam, n_pol);
    case 2: return u8_ring_depth<TcCfg<32, 2, 1>>(n_beam, n_pol);
    case 3: return u8_ring_depth<TcCfg<64, 3, 1>>(n_beam, n_pol);
    case 4: return u8_ring_depth<TcCfg<64, 2, 2>>(n_beam, n_pol);
    case 5: return u8_ring_depth<TcCfg<64, 3, 2>>(n_beam, n_pol);
    case 6: return u8_ring_depth<TcCfg<64, 4, 1>>(n_beam, n_pol);
    case 7: return u8_ring_depth<TcCfg<64, 4, 2>>(n_beam, n_pol);
    default: return u8_ring_depth<TcCfg<64, 2, 1>>(n_beam, n_pol);
  }
}

// The A-in-TMEM kernel fits where the accumulators leave TMEM room for at
// least two operand sub-stages and shared memory an u8 ring of two stages.
static bool tca_fits(int v, int n_beam) {
  const int R = n_beam + 1, rb = (R + 1) / 2 * 2, R2 = R > 16 ? R - 16 : 0;
  if (n_beam < 2 || R > 20 || tca_sub_stages(rb, R2) < 2) return false;
  const int na = tca_sub_stages(rb, R2);
  return (v == 9 ? tca_u8_depth<32>(n_beam, na) : tca_u8_depth<64>(n_beam, na)) >= 2;
}

// Two polarisations double the u8 stage: they run variant 0 (two f16
// stages), which leaves the u8 ring at least two stages deep. Variants 8
// and 9 where they do not fit the shape run the untuned default.
static int tc_variant_for(const mraid_plan_s* pl, int n_pol) {
  if (n_pol == 2) return 0;
  const int v = pl->tc_variant;
  if (v >= 8 && !tca_fits(v, pl->p.n_beam)) return tc_default_variant(pl->p.n_beam);
  return v;
}

int tc_variant_effective(const mraid_plan_s* pl) { return tc_variant_for(pl, 1); }

bool gram_tc_supported(const mraid_plan_s* pl, const void* d_data, int n_pol) {
  const mraid_params& p = pl->p;
  const int t = tc_variant_samples(tc_variant_for(pl, n_pol));
  return p.bit_depth == 8 && p.n_beam >= 2 && p.n_beam + 1 <= kGroupSlots &&
         (n_pol == 1 || (n_pol == 2 && tc_u8_depth(tc_variant_for(pl, 2), p.n_beam, 2) >= 2)) &&
         p.n_samp_sub % t == 0 && p.n_samp_sub <= 1024 && p.n_chan % kBoxCh == 0 &&
         pl->beam_stride % 16 == 0 && (reinterpret_cast<uintptr_t>(d_data) & 15) == 0 &&
         (int64_t)p.n_sub * p.n_samp_sub <= 2147483647ll /* TMA time coordinate */ &&
         encode_fn() != nullptr;
}

cudaError_t launch_gram_tc(const mraid_plan_s* pl, const uint8_t* d_data, int sub0, int n_sub,
                           int64_t* d_sums, float* d_corr, int64_t* d_sums8, int n_pol) {
  const mraid_params& p = pl->p;
  if (!gram_tc_supported(pl, d_data, n_pol)) return cudaErrorNotSupported;
  const int variant = tc_variant_for(pl, n_pol);
  CUtensorMap map;
  const cuuint64_t n_time = (cuuint64_t)(sub0 + n_sub) * p.n_samp_sub;
  // one box holds every block of the stage: n_pol * N blocks, beam_stride apart
  cuuint64_t dims[3] = {(cuuint64_t)p.n_chan, n_time, (cuuint64_t)n_pol * p.n_beam};
  cuuint64_t strides[2] = {(cuuint64_t)p.n_chan, (cuuint64_t)pl->beam_stride};
  const int t = tc_variant_samples(variant);
  cuuint32_t box[3] = {(cuuint32_t)kBoxCh, (cuuint32_t)t, (cuuint32_t)(n_pol * p.n_beam)};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(d_data),
                           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  TcArgs a;
  a.n_beam = p.n_beam;
  a.n_chan = p.n_chan;
  a.n_samp_sub = p.n_samp_sub;
  a.sub0 = sub0;
  a.n_sub = n_sub;
  a.n_pol = n_pol;
  a.center = n_pol == 2 ? 255 : 128;
  // FP32 sums in TMEM stay exact while they are below 2^24: 1024 samples of
  // products up to 128^2 for one polarisation, 256 samples of products up to
  // 255^2 for the sum of two; a sub-integration of two polarisations is
  // accumulated in pieces (the largest number of stages dividing it within
  // 256 samples) that the epilogue adds as integers
  {
    const int stages = p.n_samp_sub / t;
    int d = stages;
    if (n_pol == 2)
      while (d > 1 && (stages % d != 0 || d * t > 256)) --d;
    a.piece_stages = d;
  }
  const int R = p.n_beam + 1;              // beams + the row of ones
  a.R = R;
  a.R2 = R > 16 ? R - 16 : 0;
  a.rb = (R + 1) / 2 * 2;                  // B of the first MMAs: R slots, even count
  a.sums = d_sums8 ? nullptr : d_sums;
  a.sums8 = d_sums8;
  a.corr = d_corr;
  a.degenerate = pl->d_degenerate;
  a.error = pl->d_error;
  a.wait_ns = pl->wait_ns;
  a.withhold = pl->inject_withhold;
  const int64_t items = (int64_t)n_sub * (p.n_chan / kBoxCh);
  const int grid = (int)(items < pl->sm_count ? items : pl->sm_count);
  cudaError_t e = cudaSuccess;
#define MRAID_TC_LAUNCH_P(T, NF, U, P)                                                             \
  do {                                                                                           \
    using C_ = TcCfg<T, NF, U>;                                                                     \
    const int n_u8 = u8_ring_depth<C_>(p.n_beam, P);                                             \
    a.n_u8 = n_u8;                                                                               \
    const size_t smem = smem_bytes<C_>(p.n_beam, n_u8, P);                                       \
    e = cudaFuncSetAttribute(gram_tc_kernel<T, NF, U, P>,                                        \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);           \
    if (e == cudaSuccess && grid > 0)                                                            \
      gram_tc_kernel<T, NF, U, P><<<grid, kThreads, smem, pl->stream>>>(map, a);                  \
  } while (0)
#define MRAID_TC_LAUNCH(T, NF, U) MRAID_TC_LAUNCH_P(T, NF, U, 1)
#define MRAID_TCA_LAUNCH(T)                                                                       \
  do {                                                                                           \
    const int na_ = tca_sub_stages(a.rb, a.R2);                                                  \
    const int n_u8 = tca_u8_depth<T>(p.n_beam, na_);                                             \
    a.n_u8 = n_u8;                                                                               \
    const size_t smem = tca_smem_bytes<T>(p.n_beam, na_, n_u8);                                  \
    e = cudaFuncSetAttribute(gram_tc_a_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                             (int)smem);                                                        \
    if (e == cudaSuccess && grid > 0)                                                            \
      gram_tc_a_kernel<T><<<grid, kThreads, smem, pl->stream>>>(map, a);                          \
  } while (0)
  if (n_pol == 2) {
    MRAID_TC_LAUNCH_P(64, 2, 1, 2);  // variant 0: two f16 stages leave room for the doubled u8 ring
  } else switch (variant) {
    case 8: MRAID_TCA_LAUNCH(64); break;
    case 9: MRAID_TCA_LAUNCH(32); break;
    case 1: MRAID_TC_LAUNCH(32, 4, 1); break;
    case 2: MRAID_TC_LAUNCH(32, 2, 1); break;
    case 3: MRAID_TC_LAUNCH(64, 3, 1); break;
    case 4: MRAID_TC_LAUNCH(64, 2, 2); break;
    case 5: MRAID_TC_LAUNCH(64, 3, 2); break;
    case 6: MRAID_TC_LAUNCH(64, 4, 1); break;
    case 7: MRAID_TC_LAUNCH(64, 4, 2); break;
    default: MRAID_TC_LAUNCH(64, 2, 1); break;
  }
#undef MRAID_TC_LAUNCH
#undef MRAID_TC_LAUNCH_P
#undef MRAID_TCA_LAUNCH
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

bool gram_tc_f32_supported(const mraid_plan_s* pl, const void* d_data) {
  const mraid_params& p = pl->p;
  return p.bit_depth == 32 && p.n_beam >= 2 && p.n_beam + 1 <= kGroupSlots &&
         p.n_samp_sub % kF32T == 0 && p.n_chan % kBoxCh == 0 && pl->beam_stride % 4 == 0 &&
         (reinterpret_cast<uintptr_t>(d_data) & 15) == 0 && f32_ring_depth(p.n_beam, 2) >= 2 &&
         (int64_t)p.n_sub * p.n_samp_sub <= 2147483647ll && encode_fn() != nullptr;
}

cudaError_t launch_gram_tc_f32(const mraid_plan_s* pl, const float* d_data, int sub0, int n_sub,
                               float* d_corr) {
  const mraid_params& p = pl->p;
  if (!gram_tc_f32_supported(pl, d_data) || !d_corr) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t n_time = (cuuint64_t)(sub0 + n_sub) * p.n_samp_sub;
  cuuint64_t dims[3] = {(cuuint64_t)p.n_chan, n_time, (cuuint64_t)p.n_beam};
  cuuint64_t strides[2] = {(cuuint64_t)p.n_chan * 4, (cuuint64_t)pl->beam_stride * 4};
  cuuint32_t box[3] = {(cuuint32_t)kBoxCh, (cuuint32_t)kF32T, (cuuint32_t)p.n_beam};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(d_data),
                           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  TcArgs a;
  a.n_beam = p.n_beam;
  a.n_chan = p.n_chan;
  a.n_samp_sub = p.n_samp_sub;
  a.sub0 = sub0;
  a.n_sub = n_sub;
  const int R = p.n_beam + 1;
  a.R = R;
  a.R2 = R > 16 ? R - 16 : 0;
  a.rb = (R + 1) / 2 * 2;
  a.n_pol = 1;
  a.center = 0;
  a.piece_stages = 1;
  a.sums = nullptr;
  a.sums8 = nullptr;
  a.corr = d_corr;
  a.degenerate = pl->d_degenerate;
  a.error = pl->d_error;
  a.wait_ns = pl->wait_ns;
  a.withhold = -1;
  const int nf = f32_stages(p.n_beam);
  a.n_u8 = f32_ring_depth(p.n_beam, nf);
  const size_t smem = f32_smem_bytes(p.n_beam, nf, a.n_u8);
  const int64_t items = (int64_t)n_sub * (p.n_chan / kBoxCh);
  const int grid = (int)(items < pl->sm_count ? items : pl->sm_count);
  auto kern = nf == 3 ? gram_tc_f32_kernel<3> : gram_tc_f32_kernel<2>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (grid > 0) kern<<<grid, kThreads, smem, pl->stream>>>(map, a);
  return cudaGetLastError();
}

}  // namespace mraid
