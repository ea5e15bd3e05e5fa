// gram_tcl.cu - exact augmented Gram sums of 8-bit data for 24..127 beams
// on the tensor cores, channels kept apart by rows.
//
// Section 3.2, Eq. 1, for the larger (phased-array-feed) receivers. The
// channel block-diagonal layout of gram_tc.cu holds at most 23 beams (its
// accumulators for 16 channels fill TMEM). Here an operand tile holds G
// channels' beams in 128 rows, R = 128 / G rows each (x - 128 in f16, row
// N of each channel the row of ones, rows past N zero): G = 4 for up to 31
// beams, 2 for up to 63, else 1 with R = np = N + 1 rounded up to 16. One
// MMA (M = 128, K = 16 samples) multiplies the tile by itself (B = its
// first 128 rows, or np for G = 1); the G diagonal R x R blocks of D are
// the channels' Gram matrices, the rest is discarded. Fewer, wider MMAs
// beat one per channel: a tcgen05.mma costs about 90 cycles of issue
// whatever its N. A CTA keeps nc channels' accumulators in TMEM (512
// columns), so a 16-channel TMA box is processed in 16 / nc passes by CTAs
// that run side by side (consecutive work items), the repeated box reads
// coming from L2.
//
// Exactness as in gram_tc.cu: products of centred bytes are integers of
// magnitude <= 2^14 and the FP32 accumulation is exact while a partial sum
// stays within 2^24, i.e. over at most 1024 samples. Longer
// sub-integrations are accumulated in TMEM in pieces of <= 1024 samples,
// which the epilogue adds as int32 (|sum| <= 2^14 n <= 2^30 for n <= 65536)
// into a packed upper-triangle table in shared memory. After the last piece
// the epilogue writes the raw sums S_ab = G_ab + 128 (G_a + G_b) + 128^2 n,
// S_a = G_a + 128 n and n as int64 in the public [cell][P] layout; the
// correlation follows from them (corr_from_sums), as after the CUDA-core
// Gram.
//
// Roles per persistent CTA (one per SM), 16 warps:
//   warp 0    TMA: box {16 channels, 32 samples, N beams} into an u8 ring;
//   warps 2-7 transpose 16 x 16-byte tiles (16 samples of one beam x 16
//             channels, two beams per ldmatrix) and write the pass's
//             channels as centred f16 into the K-major operand tiles;
//   warp 1    one thread issues the MMAs (nc / G per K step) and commits;
//   warps 8-15 drain TMEM after each piece into the shared tables (two
//             warps per TMEM lane quarter, alternate groups), then write
//             the cells' sums, consecutive threads to consecutive entries.
// Every wait is bounded by the plan's limit; on expiry the kernel records
// the error word, drains its copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "tc_ptx.h"

namespace mraid {
namespace {

constexpr int kLT = 32;            // samples per TMA stage
constexpr int kLKs = kLT / 16;     // K steps per stage
constexpr int kLMaxNU = 8;         // u8 ring depth bound
constexpr int kLNF = 2;            // f16 stages
constexpr int kLThreads = 512;
constexpr int kLConvWarps = 6;                 // warps 2..7
constexpr int kLConv = 32 * kLConvWarps;
constexpr int kLRound = 6;                     // pair loads in flight per converter round
// beam pairs per converter warp (64 pairs at most), a whole number of rounds
constexpr int kLMaxPW = ((64 + kLConvWarps - 1) / kLConvWarps + kLRound - 1) / kLRound * kLRound;
constexpr int kLEpiWarps = 8;                  // warps 8..15, two per TMEM lane quarter
constexpr int kLEpi = 32 * kLEpiWarps;
constexpr int kLPiece = 1024;      // samples per exact TMEM accumulation at most
constexpr size_t kLSmemBudget = 227 * 1024;
constexpr uint32_t kLTmemCols = 512;

struct LArgs {
  int n_beam, n_chan, n_samp_sub, sub0, n_sub;
  int G;             // channels per MMA
  int R;             // tile rows per channel (128 / G; np for G = 1)
  int gcols;         // D columns per MMA (128; np for G = 1)
  int nc;            // channels per CTA pass (a multiple of G)
  int passes;        // ceil(16 / nc); the last pass takes the remaining channels
  int piece_stages;  // stages per TMEM accumulation piece
  int n_u8;          // u8 ring depth
  int psum;          // (N + 1)(N + 2) / 2
  uint32_t gstride;    // bytes between group tiles of a K step (G R 32 + 16)
  uint32_t ks_stride;  // bytes between K steps of an f16 stage
  uint32_t f16_stage;  // bytes of an f16 stage
  uint32_t acc_bytes;  // the int32 tables and row sums of nc cells
  int64_t* sums;       // [cell][psum], cells relative to sub0
  unsigned* error;
  unsigned long long wait_ns;
  long long withhold;  // fault injection: CTA 0's TMA producer never issues this stage (-1: none)
};

struct SmemL {
  uint64_t u8_full[kLMaxNU], u8_empty[kLMaxNU];
  uint64_t f16_full[kLNF], f16_empty[kLNF];
  uint64_t acc_full, acc_empty, drain;
  int epi_go;
  uint32_t tmem_base;
};

// Tile shape for n_beam beams: G, R and the D columns of one MMA.
struct LShape {
  int G, R, gcols;
};
__host__ __device__ constexpr LShape l_shape(int n_beam) {
  return n_beam + 1 <= 32   ? LShape{4, 32, 128}
         : n_beam + 1 <= 64 ? LShape{2, 64, 128}
                            : LShape{1, (n_beam + 1 + 15) / 16 * 16, (n_beam + 1 + 15) / 16 * 16};
}
__host__ __device__ constexpr uint32_t l_gstride(LShape sh) {
  return (uint32_t)(sh.G * sh.R) * 32u + 16u;
}
__host__ __device__ constexpr uint32_t l_f16_stage(LShape sh, int nc) {
  return (uint32_t)kLKs * (uint32_t)(nc / sh.G) * l_gstride(sh);
}
// the int32 tables of nc cells (packed upper triangles), then their row
// sums G_a (nc x 128 int32)
__host__ __device__ constexpr uint32_t l_acc_bytes(int n_beam, int nc) {
  return (((uint32_t)nc * (uint32_t)((n_beam + 1) * (n_beam + 2) / 2) * 4u + 15u) & ~15u) +
         (uint32_t)nc * 128u * 4u;
}
// the f16 stages, rounded up so that the u8 ring starts 1024-byte aligned
__host__ __device__ constexpr size_t l_f16_region(uint32_t f16_stage) {
  return ((size_t)kLNF * f16_stage + 1023) & ~(size_t)1023;
}
// channels in pass `pass` of a 16-channel box (the last pass may hold fewer)
__host__ __device__ __forceinline__ int l_pass_channels(int pass, int nc) {
  return 16 - pass * nc < nc ? 16 - pass * nc : nc;
}
// start of row a in the packed upper triangle of an (N+1)^2 matrix
__host__ __device__ __forceinline__ int l_row_off(int a, int n1) { return a * n1 - a * (a - 1) / 2; }

// two 16 x 16-byte tiles transposed: rows of tile 0 from the addresses of
// lanes 0-15, of tile 1 from lanes 16-31; thread t gets bytes 4(t%4)..+3 of
// column t/4 (r0) and t/4 + 8 (r1) of tile 0, the same of tile 1 in r2, r3
__device__ __forceinline__ void ldm_trans_b8_x2(uint32_t addr, uint32_t& r0, uint32_t& r1,
                                                uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m16n16.x2.trans.shared.b8 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
// 8-byte shared store under a predicate
__device__ __forceinline__ void st_shared_v2_if(uint32_t addr, uint32_t x, uint32_t y, uint32_t on) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n @p st.shared.v2.b32 [%0], {%1, %2};\n}\n" ::"r"(
          addr),
      "r"(x), "r"(y), "r"(on));
}
// 16 consecutive TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// kAll16: a pass holds all 16 channels of a box (nc = 16), so a converter
// thread stores both of its channels.
template <bool kAll16>
__global__ void __launch_bounds__(kLThreads, 1)
gram_tcl_kernel(const __grid_constant__ CUtensorMap tmap, LArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // [f16 stages][u8 ring][int32 tables][barriers]; for G = 1 the MMA's A
  // rows past np of the last tile read into the u8 ring (unused rows of D)
  unsigned char* f16 = base;
  unsigned char* u8 = f16 + l_f16_region(g.f16_stage);
  const int N = g.n_beam, N1 = N + 1;
  const uint32_t u8_stage_bytes = (uint32_t)N * kLT * 16u;
  int32_t* acc = reinterpret_cast<int32_t*>(u8 + (size_t)g.n_u8 * u8_stage_bytes);
  SmemL* s = reinterpret_cast<SmemL*>(reinterpret_cast<unsigned char*>(acc) + g.acc_bytes);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int kNU = g.n_u8;
  const int chunks = g.n_chan / 16;
  const int64_t items = (int64_t)g.n_sub * chunks * g.passes;
  const int stages = g.n_samp_sub / kLT;
  const int nc = g.nc, G = g.G, R = g.R;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kNU; ++i) {
      mbar_init(&s->u8_full[i], 1);
      mbar_init(&s->u8_empty[i], kLConv);
    }
    for (int i = 0; i < kLNF; ++i) {
      mbar_init(&s->f16_full[i], kLConv);
      mbar_init(&s->f16_empty[i], 1);
    }
    mbar_init(&s->acc_full, 1);
    mbar_init(&s->acc_empty, kLEpi);
    mbar_init(&s->drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // operand tiles: row N of every channel (ones) and rows N+1..R-1 (zeros)
  // are never rewritten
  {
    const uint32_t words = (uint32_t)kLNF * g.f16_stage / 4u;
    uint32_t* w = reinterpret_cast<uint32_t*>(f16);
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) {
      const uint32_t off = (i * 4u) % g.gstride;  // byte offset within a group tile
      uint32_t v = 0u;
      if (off < (uint32_t)(G * R) * 32u) {
        const uint32_t row = (off / 256u) * 8u + (off % 128u) / 16u;
        if ((int)(row % (uint32_t)R) == N) v = 0x3c003c00u;  // f16x2 (1, 1)
      }
      w[i] = v;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s->tmem_base)),
                 "r"(kLTmemCols));
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
        const int64_t rest = it / g.passes;
        const int k = (int)(rest / chunks), ch0 = (int)(rest % chunks) * 16;
        const int64_t t_item = (int64_t)(g.sub0 + k) * g.n_samp_sub;
        for (int st = 0; st < stages && ok; ++st, ++cnt) {
          const int slot = cnt % kNU;
          ok = mbar_wait(&s->u8_empty[slot], ((cnt / kNU) & 1) ^ 1, g.error, g.wait_ns);
          if (!ok) break;
          if (blockIdx.x == 0 && (long long)cnt == g.withhold) {
            // injected fault: this stage is never issued, so the converters'
            // bounded wait for it expires (nothing is in flight for it)
            withheld = cnt;
            continue;
          }
          mbar_expect_tx(&s->u8_full[slot], u8_stage_bytes);
          tma_load_3d(u8 + (size_t)slot * u8_stage_bytes, &tmap, ch0, (int)(t_item + st * kLT), 0,
                      &s->u8_full[slot]);
        }
      }
      // every issued copy has landed before the CTA may exit
      for (uint32_t d = cnt > (uint32_t)kNU ? cnt - kNU : 0; d < cnt; ++d)
        if ((long long)d != withheld)
          mbar_drain(&s->u8_full[d % kNU], (d / kNU) & 1, g.error, g.wait_ns);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA
    if (lane == 0) {
      const uint32_t f16_base = smem_u32(f16);
      const uint32_t idesc = idesc_f16_k(128, g.gcols);
      // K-major canonical layout, no swizzle: 8-row core matrices of 16 B
      // rows, the two K halves 128 B apart, the next 8 rows 256 B on
      const uint32_t lbo = 128, sbo = 256;
      uint32_t fcnt = 0, pcnt = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int ng = l_pass_channels((int)(it % g.passes), nc) / G;  // this pass's MMAs per K step
        for (int st = 0; st < stages && ok; ++st, ++fcnt) {
          const int fs = fcnt % kLNF;
          const int ps = st % g.piece_stages;
          ok = mbar_wait(&s->f16_full[fs], (fcnt / kLNF) & 1, g.error, g.wait_ns);
          if (!ok) break;
          if (ps == 0 && pcnt > 0) {
            ok = mbar_wait(&s->acc_empty, (pcnt - 1) & 1, g.error, g.wait_ns);
            if (!ok) break;
          }
          fence_after();
          const uint32_t stage = f16_base + (uint32_t)fs * g.f16_stage;
          for (int ks = 0; ks < kLKs; ++ks)
            for (int gi = 0; gi < ng; ++gi) {
              const uint32_t t = stage + (uint32_t)ks * g.ks_stride + (uint32_t)gi * g.gstride;
              const uint64_t d = smem_desc(t, lbo, sbo);
              mma_f16(tmem + (uint32_t)(gi * g.gcols), d, d, idesc, (ps > 0 || ks > 0) ? 1u : 0u);
            }
          mma_commit(&s->f16_empty[fs]);
          if (ps == g.piece_stages - 1) {
            mma_commit(&s->acc_full);
            ++pcnt;
          }
        }
      }
      mma_commit(&s->drain);
      mbar_drain(&s->drain, 0, g.error, g.wait_ns);
    }
  } else if (warp >= 2 && warp < 2 + kLConvWarps) {
    // ------------------------------------------------------------ convert
    // Converter warp cw transposes beam pairs (2pr, 2pr + 1), pr = cw + 6j,
    // with one ldmatrix .x2 per pair and K step: thread (p, q) = (lane / 4,
    // lane % 4) gets samples 4q..4q+3 of channels p and p + 8 of each beam.
    // Channel c0 + ci of the pass goes to group tile ci / G, rows
    // R (ci % G) + b, K offset 4q: for nc <= 8 at most one of the thread's
    // two channels (stored under a predicate), for nc = 16 both. A K step's
    // loads are issued before its stores.
    const int cw = warp - 2;
    const int p = lane / 4, q = lane % 4;
    const int n_pairs = (N + 1) / 2;
    const uint32_t u8_base = smem_u32(u8), f16_base = smem_u32(f16);
    const uint32_t lane_off = (uint32_t)((q / 2) * 128 + (q % 2) * 8);
    // this warp's pairs: row offsets of beam 2pr in a channel's rows, and
    // the lane's beam (2pr + lane / 16; the last pair of an odd N repeats
    // beam 2pr)
    uint32_t rowoff[kLMaxPW], srcoff[kLMaxPW];
#pragma unroll
    for (int j = 0; j < kLMaxPW; ++j) {
      const int pr = cw + kLConvWarps * j;
      const int b = 2 * pr, bl = (b + (lane >> 4) < N) ? b + (lane >> 4) : b;
      rowoff[j] = (uint32_t)((b >> 3) * 256 + (b & 7) * 16);
      srcoff[j] = (uint32_t)(pr < n_pairs ? bl : 0) * (kLT * 16u);
    }
    // byte offset of channel ci's rows in a K step's tiles
    auto chan_off = [&](int ci) {
      return (uint32_t)(ci / G) * g.gstride + (uint32_t)((ci % G) * R) * 32u;
    };
    uint32_t cnt = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
      const int c0 = (int)(it % g.passes) * nc;
      const int ncp = l_pass_channels((int)(it % g.passes), nc);
      const int ci0 = p - c0, ci1 = p + 8 - c0;  // channel p / p + 8 in the pass (valid in [0, ncp))
      const bool use0 = ci0 >= 0 && ci0 < ncp, use1 = ci1 >= 0 && ci1 < ncp;
      // first store: channel p if it is the pass's, else p + 8; second
      // (nc = 16 only): channel p + 8
      const uint32_t ta = chan_off(use0 ? ci0 : (use1 ? ci1 : 0)) + lane_off;
      const uint32_t tb = chan_off(use1 ? ci1 : 0) + lane_off;
      const uint32_t pa = (use0 || use1) ? 1u : 0u, pb = (use0 && use1) ? 1u : 0u;
      for (int st = 0; st < stages && ok; ++st, ++cnt) {
        const int us = cnt % kNU, fs = cnt % kLNF;
        ok = mbar_wait(&s->u8_full[us], (cnt / kNU) & 1, g.error, g.wait_ns);
        if (ok) ok = mbar_wait(&s->f16_empty[fs], ((cnt / kLNF) & 1) ^ 1, g.error, g.wait_ns);
        if (!ok) break;
        const uint32_t src = u8_base + (uint32_t)us * u8_stage_bytes;
        const uint32_t dst = f16_base + (uint32_t)fs * g.f16_stage;
#pragma unroll
        for (int ks = 0; ks < kLKs; ++ks) {
          const uint32_t rows = src + (uint32_t)(ks * 16 + (lane & 15)) * 16u;
          const uint32_t kda = dst + (uint32_t)ks * g.ks_stride + ta;
          const uint32_t kdb = dst + (uint32_t)ks * g.ks_stride + tb;
#pragma unroll
          for (int j0 = 0; j0 < kLMaxPW; j0 += kLRound) {
            if (cw + kLConvWarps * j0 >= n_pairs) break;
            uint32_t r[kLRound][4];
#pragma unroll
            for (int jj = 0; jj < kLRound; ++jj)
              if (cw + kLConvWarps * (j0 + jj) < n_pairs)
                ldm_trans_b8_x2(rows + srcoff[j0 + jj], r[jj][0], r[jj][1], r[jj][2], r[jj][3]);
#pragma unroll
            for (int jj = 0; jj < kLRound; ++jj) {
              const int pr = cw + kLConvWarps * (j0 + jj);
              if (pr >= n_pairs) break;
              const uint32_t odd = (2 * pr + 1 < N) ? 1u : 0u;  // the pair's second beam exists
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const uint32_t ra = use0 ? r[jj][2 * h] : r[jj][2 * h + 1];
                const uint32_t row = rowoff[j0 + jj] + 16u * h;
                uint32_t lo, hi;
                u8x4_to_f16(ra, lo, hi);
                st_shared_v2_if(kda + row, lo, hi, h ? (pa & odd) : pa);
                if (kAll16) {
                  u8x4_to_f16(r[jj][2 * h + 1], lo, hi);
                  st_shared_v2_if(kdb + row, lo, hi, h ? (pb & odd) : pb);
                }
              }
            }
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&s->u8_empty[us]);
        mbar_arrive(&s->f16_full[fs]);
      }
    }
  } else if (warp >= 8) {
    // ------------------------------------------------------------ epilogue
    // Warp (q, h) = (warp % 4, (warp - 8) / 4) reads TMEM lanes 32q..32q+31
    // of the groups gi = h, h + 2, ...: lane l = 32q + lane holds row
    // a = l % R of the group's channel slot l / R (one slot per warp, as
    // R >= 32; for G = 1 lanes past np hold nothing). After the last piece
    // all epilogue threads write the cells' packed sums, consecutive
    // threads to consecutive entries.
    const int q = warp % 4, h = (warp - 8) / 4;
    const int et = threadIdx.x - 8 * 32;  // 0..kLEpi-1
    const int slot = (32 * q) / R;        // this warp's channel slot in a group
    const int a = (32 * q + lane) - slot * R;
    const bool mine = slot < G && a < N1 && (32 * q + lane) / R == slot;
    const int col0 = slot * R;            // the slot's first D column in a group
    const int amin = 32 * q - col0;       // the warp's first row
    const int jb0 = (col0 + amin) / 16;
    const int jb1 = (col0 + N1 + 15) / 16;
    const int psum = g.psum;
    const int n_pieces = stages / g.piece_stages;
    const int64_t n = g.n_samp_sub;
    int32_t* rowsum = acc + ((nc * psum + 3) & ~3);  // [ci][128]: G_a of each cell
    uint32_t pcnt = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
      const int64_t rest = it / g.passes;
      const int k = (int)(rest / chunks), ch0 = (int)(rest % chunks) * 16;
      const int c0 = (int)(it % g.passes) * nc;
      const int ncp = l_pass_channels((int)(it % g.passes), nc);
      for (int pc = 0; pc < n_pieces && ok; ++pc) {
        ok = epi_wait(&s->acc_full, pcnt & 1, g.error, g.wait_ns, &s->epi_go, et == 0, kLEpi);
        if (!ok) break;
        ++pcnt;
        fence_after();
        if (slot < G) {
          for (int gi = h; gi < ncp / G; gi += 2) {
            const int ci = gi * G + slot;
            // this row's entries b >= a: tab[row_off(a) + b - a]
            int32_t* row = acc + ci * psum + (mine ? l_row_off(a, N1) : 0);
            for (int jb = jb0; jb < jb1; ++jb) {
              uint32_t v[16];
              tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(gi * g.gcols + 16 * jb), v);
              tmem_wait_ld();
              if (mine) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  const int b = 16 * jb + i - col0;
                  if (b >= a && b < N1) {
                    const int32_t x = __float2int_rn(__uint_as_float(v[i]));
                    row[b - a] = pc == 0 ? x : row[b - a] + x;
                  }
                }
              }
            }
            if (pc == n_pieces - 1 && mine && a < N) rowsum[ci * 128 + a] = row[N - a];
          }
        }
        // TMEM may take the next piece
        fence_before();
        mbar_arrive(&s->acc_empty);
      }
      if (!ok) break;
      named_sync(1, kLEpi);  // every table and row sum complete
      for (int ci = 0; ci < ncp; ++ci) {
        const int32_t* tab = acc + ci * psum;
        const int32_t* gs = rowsum + ci * 128;
        const int64_t cell = (int64_t)k * g.n_chan + ch0 + c0 + ci;
        int64_t* dst = g.sums + cell * psum;
        // (ra, ra + off) = row and column of packed entry idx, advanced
        // kLEpi at a time
        int ra = 0, off = et;
        while (ra <= N && off >= N1 - ra) {
          off -= N1 - ra;
          ++ra;
        }
        for (int idx = et; idx < psum; idx += kLEpi) {
          const int rb = ra + off;
          int64_t v;
          if (ra == N) {
            v = n;
          } else if (rb == N) {
            v = (int64_t)gs[ra] + 128 * n;
          } else {
            v = (int64_t)tab[idx] + 128 * ((int64_t)gs[ra] + gs[rb]) + 16384 * n;
          }
          dst[idx] = v;
          off += kLEpi;
          while (ra <= N && off >= N1 - ra) {
            off -= N1 - ra;
            ++ra;
          }
        }
      }
      named_sync(1, kLEpi);  // tables reused by the next item
    }
  }
  __syncthreads();
  if (warp == 2) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kLTmemCols));
  }
}

// Channels per pass: the most whose accumulators fit TMEM ((nc / G) x gcols
// <= 512 columns) and whose tables, two f16 stages and an u8 ring of two
// stages fit shared memory: 16 or 8 for the four- and two-channel tiles
// (a divisor of 16 that is a multiple of G), any count for one channel per
// tile (the box's last pass then takes the remaining channels); 0 if none
// fits.
int l_channels(int n_beam, int* n_u8_out) {
  const LShape sh = l_shape(n_beam);
  for (int nc = 16; nc >= sh.G; nc = sh.G > 1 ? nc / 2 : nc - 1) {
    if ((nc / sh.G) * sh.gcols > (int)kLTmemCols) continue;
    const size_t fixed = 1024 + l_f16_region(l_f16_stage(sh, nc)) + l_acc_bytes(n_beam, nc) +
                         sizeof(SmemL);
    const size_t u8_stage = (size_t)n_beam * kLT * 16;
    if (fixed + 2 * u8_stage > kLSmemBudget) continue;
    int n_u8 = (int)((kLSmemBudget - fixed) / u8_stage);
    if (n_u8 > kLMaxNU) n_u8 = kLMaxNU;
    if (n_u8_out) *n_u8_out = n_u8;
    return nc;
  }
  return 0;
}

}  // namespace

bool gram_tcl_supported(const mraid_plan_s* pl, const void* d_data) {
  const mraid_params& p = pl->p;
  return p.bit_depth == 8 && p.n_beam >= 24 && p.n_beam + 1 <= 128 &&
         p.n_samp_sub % kLT == 0 && p.n_samp_sub <= 65536 && p.n_chan % 16 == 0 &&
         pl->beam_stride % 16 == 0 && (reinterpret_cast<uintptr_t>(d_data) & 15) == 0 &&
         (int64_t)p.n_sub * p.n_samp_sub <= 2147483647ll && l_channels(p.n_beam, nullptr) > 0 &&
         encode_fn() != nullptr;
}

cudaError_t launch_gram_tcl(const mraid_plan_s* pl, const uint8_t* d_data, int sub0, int n_sub,
                            int64_t* d_sums) {
  const mraid_params& p = pl->p;
  if (!gram_tcl_supported(pl, d_data) || !d_sums) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t n_time = (cuuint64_t)(sub0 + n_sub) * p.n_samp_sub;
  cuuint64_t dims[3] = {(cuuint64_t)p.n_chan, n_time, (cuuint64_t)p.n_beam};
  cuuint64_t strides[2] = {(cuuint64_t)p.n_chan, (cuuint64_t)pl->beam_stride};
  cuuint32_t box[3] = {16u, (cuuint32_t)kLT, (cuuint32_t)p.n_beam};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(d_data),
                           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const LShape sh = l_shape(p.n_beam);
  LArgs a;
  a.n_beam = p.n_beam;
  a.n_chan = p.n_chan;
  a.n_samp_sub = p.n_samp_sub;
  a.sub0 = sub0;
  a.n_sub = n_sub;
  a.G = sh.G;
  a.R = sh.R;
  a.gcols = sh.gcols;
  a.nc = l_channels(p.n_beam, &a.n_u8);
  a.passes = (16 + a.nc - 1) / a.nc;
  {
    const int stages = p.n_samp_sub / kLT;
    int d = stages;
    while (d > 1 && (stages % d != 0 || d * kLT > kLPiece)) --d;
    a.piece_stages = d;
  }
  a.psum = (p.n_beam + 1) * (p.n_beam + 2) / 2;
  a.gstride = l_gstride(sh);
  a.ks_stride = (uint32_t)(a.nc / sh.G) * a.gstride;
  a.f16_stage = l_f16_stage(sh, a.nc);
  a.acc_bytes = l_acc_bytes(p.n_beam, a.nc);
  a.sums = d_sums;
  a.error = pl->d_error;
  a.wait_ns = pl->wait_ns;
  a.withhold = pl->inject_withhold;
  const size_t smem = 1024 + l_f16_region(a.f16_stage) + (size_t)a.n_u8 * p.n_beam * kLT * 16 +
                      a.acc_bytes + sizeof(SmemL);
  const int64_t items = (int64_t)n_sub * (p.n_chan / 16) * a.passes;
  const int grid = (int)(items < pl->sm_count ? items : pl->sm_count);
  cudaError_t e;
  if (a.nc == 16) {
    e = cudaFuncSetAttribute(gram_tcl_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e == cudaSuccess && grid > 0)
      gram_tcl_kernel<true><<<grid, kLThreads, smem, pl->stream>>>(map, a);
  } else {
    e = cudaFuncSetAttribute(gram_tcl_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e == cudaSuccess && grid > 0)
      gram_tcl_kernel<false><<<grid, kLThreads, smem, pl->stream>>>(map, a);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace mraid
