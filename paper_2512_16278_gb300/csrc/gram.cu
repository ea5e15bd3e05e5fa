// gram.cu - exact augmented Gram sums of 8-bit multi-beam data on CUDA
// cores (dp4a), and the conversion of the sums to the Pearson correlation.
//
// Section 3.2, Eq. 1: per cell (channel j, sub-integration k) the beams'
// cross-correlation. For X the N_beam x N_s samples of a cell and
// X~ = [X; 1], G = X~ X~^T holds every sum the correlation needs:
// S_ab = G[a][b], S_a = G[a][N], N_s = G[N][N]. Integer sums are exact;
// the correlation r_ab = (n S_ab - S_a S_b) / sqrt(var_a var_b) is formed
// from exact int64 numerators and converted to float once.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mraid {
namespace {

constexpr int kGramThreads = 256;
constexpr int kT = 32;          // samples staged per chunk
constexpr int kTW = kT / 4;     // 32-bit words per staged row
// Staged row stride in words: one more than a row, so the rows of the
// 4-row tiles that a warp's lanes read at once fall in different banks
// (a stride of kTW = 8 words put every tile's rows 32 words apart, on the
// same bank).
constexpr int kRS = kTW + 1;

struct GramArgs {
  const uint8_t* data;
  int64_t beam_stride;
  int n_beam, n_chan, n_samp_sub;
  int sub0;
  int R;        // augmented rows rounded up to a multiple of 4
  int cpb;      // channels per block
  int tiles;    // 4x4 row tiles in the upper triangle: T1(T1+1)/2, T1 = R/4
  int ntask;    // cpb * tiles
  int cs;       // staged words per channel: R * kRS + 1 (odd: channels in different banks)
  int psum;     // (N+1)(N+2)/2
  int64_t* sums;
};

__device__ __forceinline__ uint32_t ones_word(int valid) {
  // bytes of value 1 for the first `valid` samples of a 4-sample word
  return valid >= 4 ? 0x01010101u : (valid <= 0 ? 0u : (0x01010101u >> (8 * (4 - valid))));
}

// Stage kT samples x R rows x cpb channels, time-contiguous per (channel,
// row): word xs[c*cs + row*kRS + t/4] holds samples t..t+3 of that row.
template <bool VEC4>
__device__ __forceinline__ void stage_chunk(const GramArgs& g, uint32_t* xs, int sub,
                                            int c0, int t_base) {
  const int nv = min(kT, g.n_samp_sub - t_base);  // valid samples in chunk
  const int64_t t_abs0 = (int64_t)sub * g.n_samp_sub + t_base;
  if (VEC4) {
    const int c4n = g.cpb / 4;
    const int work = g.n_beam * kTW * c4n;
    for (int w = threadIdx.x; w < work; w += blockDim.x) {
      const int c4 = w % c4n;
      const int bt = w / c4n;
      const int t4 = bt % kTW;
      const int b = bt / kTW;
      const int ch = c0 + 4 * c4;
      uint32_t v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int t = 4 * t4 + i;
        v[i] = 0;
        if (t < nv && ch < g.n_chan)
          v[i] = __ldg(reinterpret_cast<const uint32_t*>(
              g.data + b * g.beam_stride + (t_abs0 + t) * g.n_chan + ch));
      }
      // 4x4 byte transpose: out[j] = channel ch+j, samples t..t+3
      const uint32_t lo01 = __byte_perm(v[0], v[1], 0x5140);
      const uint32_t hi01 = __byte_perm(v[0], v[1], 0x7362);
      const uint32_t lo23 = __byte_perm(v[2], v[3], 0x5140);
      const uint32_t hi23 = __byte_perm(v[2], v[3], 0x7362);
      uint32_t* dst = xs + (4 * c4) * g.cs + b * kRS + t4;
      dst[0] = __byte_perm(lo01, lo23, 0x5410);
      dst[g.cs] = __byte_perm(lo01, lo23, 0x7632);
      dst[2 * g.cs] = __byte_perm(hi01, hi23, 0x5410);
      dst[3 * g.cs] = __byte_perm(hi01, hi23, 0x7632);
    }
  } else {
    uint8_t* xb = reinterpret_cast<uint8_t*>(xs);
    const int work = g.n_beam * kT * g.cpb;
    for (int w = threadIdx.x; w < work; w += blockDim.x) {
      const int c = w % g.cpb;
      const int bt = w / g.cpb;
      const int t = bt % kT;
      const int b = bt / kT;
      uint8_t x = 0;
      if (t < nv && c0 + c < g.n_chan)
        x = __ldg(g.data + b * g.beam_stride + (t_abs0 + t) * g.n_chan + c0 + c);
      xb[4 * (c * g.cs + b * kRS + t / 4) + (t & 3)] = x;
    }
  }
  // ones row (index N) and zero padding rows
  const int extra = (g.R - g.n_beam) * kTW * g.cpb;
  for (int w = threadIdx.x; w < extra; w += blockDim.x) {
    const int c = w % g.cpb;
    const int rt = w / g.cpb;
    const int t4 = rt % kTW;
    const int row = g.n_beam + rt / kTW;
    xs[c * g.cs + row * kRS + t4] = (row == g.n_beam) ? ones_word(nv - 4 * t4) : 0u;
  }
}

// kSeg: sub-integrations longer than kGramSegment samples, whose int32
// partial sums must be flushed into int64 totals; shorter ones (every
// receiver here) accumulate in int32 only and keep half the registers.
// Resident blocks per SM asked of the register allocator: three for up to
// three tasks per thread (80 registers; measured 11 % faster at 72 beams than
// the two blocks of the unconstrained 116), two for four.
template <int TPT, bool kSeg>
constexpr int gram_min_blocks() {
  return kSeg ? 1 : (TPT <= 3 ? 3 : 2);
}

template <int TPT, bool VEC4, bool kSeg>
__global__ void __launch_bounds__(kGramThreads, (gram_min_blocks<TPT, kSeg>()))
gram_u8_kernel(GramArgs g) {
  extern __shared__ uint32_t smem[];
  uint32_t* xs = smem;
  uint16_t* tile_ij = reinterpret_cast<uint16_t*>(xs + g.cpb * g.cs);
  const int c0 = blockIdx.x * g.cpb;
  const int sub = g.sub0 + blockIdx.y;
  const int T1 = g.R / 4;
  for (int t = threadIdx.x; t < g.tiles; t += blockDim.x) {
    // t -> (ti, tj), ti <= tj, row-major over the upper triangle
    int ti = 0, rem = t;
    while (rem >= T1 - ti) {
      rem -= T1 - ti;
      ++ti;
    }
    tile_ij[t] = (uint16_t)(ti | ((ti + rem) << 8));
  }

  uint32_t acc[TPT][16];
  unsigned long long tot[kSeg ? TPT : 1][16];
#pragma unroll
  for (int j = 0; j < TPT; ++j)
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[j][e] = 0;
#pragma unroll
  for (int j = 0; j < (kSeg ? TPT : 1); ++j)
#pragma unroll
    for (int e = 0; e < 16; ++e) tot[j][e] = 0;
  __syncthreads();

  int in_segment = 0;
  for (int t_base = 0; t_base < g.n_samp_sub; t_base += kT) {
    __syncthreads();
    stage_chunk<VEC4>(g, xs, sub, c0, t_base);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
      const int task = threadIdx.x + j * kGramThreads;
      if (task < g.ntask) {
        const int c = task % g.cpb;
        const uint16_t tij = tile_ij[task / g.cpb];
        const uint32_t* ra = xs + c * g.cs + 4 * (tij & 0xff) * kRS;
        const uint32_t* rb = xs + c * g.cs + 4 * (tij >> 8) * kRS;
#pragma unroll
        for (int t4 = 0; t4 < kTW; ++t4) {
          uint32_t a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            a[i] = ra[i * kRS + t4];
            b[i] = rb[i * kRS + t4];
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[j][4 * i + k] = __dp4a(a[i], b[k], acc[j][4 * i + k]);
        }
      }
    }
    if constexpr (kSeg) {
      in_segment += kT;
      if (in_segment >= kGramSegment || t_base + kT >= g.n_samp_sub) {
#pragma unroll
        for (int j = 0; j < TPT; ++j)
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            tot[j][e] += acc[j][e];
            acc[j][e] = 0;
          }
        in_segment = 0;
      }
    }
  }

  const int N1 = g.n_beam + 1;
#pragma unroll
  for (int j = 0; j < TPT; ++j) {
    const int task = threadIdx.x + j * kGramThreads;
    if (task >= g.ntask) continue;
    const int c = task % g.cpb;
    if (c0 + c >= g.n_chan) continue;
    const uint16_t tij = tile_ij[task / g.cpb];
    const int64_t cell = (int64_t)blockIdx.y * g.n_chan + c0 + c;  // relative to sub0
    int64_t* out = g.sums + cell * g.psum;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int a = 4 * (tij & 0xff) + i;
        const int b = 4 * (tij >> 8) + k;
        if (a <= b && b < N1)
          out[a * N1 - a * (a - 1) / 2 + (b - a)] =
              kSeg ? (int64_t)tot[kSeg ? j : 0][4 * i + k] : (int64_t)acc[j][4 * i + k];
      }
  }
}

// Pearson correlation from the exact sums: one warp per cell.
__global__ void corr_from_sums_kernel(const int64_t* __restrict__ sums, int64_t n_cells,
                                      int n_beam, int psum, int np, float* __restrict__ corr,
                                      unsigned long long* degenerate, int interleaved) {
  extern __shared__ unsigned char sm_raw[];
  const int warps = blockDim.x / 32;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  int64_t* S = reinterpret_cast<int64_t*>(sm_raw) + (size_t)warp * psum;
  float* inv_sd = reinterpret_cast<float*>(reinterpret_cast<int64_t*>(sm_raw) + (size_t)warps * psum) +
                  (size_t)warp * kMaxBeam;
  const int64_t cell = (int64_t)blockIdx.x * warps + warp;
  if (cell >= n_cells) return;
  const int N1 = n_beam + 1;
  if (interleaved) {  // [cell / 8][P][cell % 8]
    const int64_t* src = sums + (cell >> 3) * psum * 8 + (cell & 7);
    for (int e = lane; e < psum; e += 32) S[e] = src[(int64_t)e * 8];
  } else {
    const int64_t* src = sums + cell * psum;
    for (int e = lane; e < psum; e += 32) S[e] = src[e];
  }
  __syncwarp();
  const int64_t n = S[psum - 1];
  int deg = 0;
  for (int a = lane; a < n_beam; a += 32) {
    const int64_t sa = S[a * N1 - a * (a - 1) / 2 + (n_beam - a)];
    const int64_t var = n * S[a * N1 - a * (a - 1) / 2] - sa * sa;
    float r = 0.f;
    if (var > 0) {
      const float v = (float)var;
      r = rsqrtf(v);
      r = r * (1.5f - 0.5f * v * r * r);  // one Newton step
    } else {
      ++deg;
    }
    inv_sd[a] = r;
  }
  __syncwarp();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) deg += __shfl_xor_sync(0xffffffffu, deg, o);
  if (lane == 0 && deg > 0) atomicAdd(degenerate, (unsigned long long)deg);
  float* dst = corr + cell * np;
  // walk the packed upper triangle: lane handles entries e = lane, lane+32, ...
  int a = 0, rowlen = n_beam, row_start = 0;
  for (int e = lane; e < np; e += 32) {
    while (e >= row_start + rowlen) {
      row_start += rowlen;
      --rowlen;
      ++a;
    }
    const int b = a + (e - row_start);
    float r;
    if (a == b) {
      r = 1.f;
    } else {
      const int64_t sa = S[a * N1 - a * (a - 1) / 2 + (n_beam - a)];
      const int64_t sb = S[b * N1 - b * (b - 1) / 2 + (n_beam - b)];
      const int64_t cov = n * S[a * N1 - a * (a - 1) / 2 + (b - a)] - sa * sb;
      r = (float)cov * inv_sd[a] * inv_sd[b];
    }
    dst[e] = r;
  }
}

}  // namespace

cudaError_t launch_gram_u8(const mraid_plan_s* pl, const uint8_t* d_data, int sub0, int n_sub,
                           int64_t* d_sums) {
  GramArgs g;
  g.data = d_data;
  g.beam_stride = pl->beam_stride;
  g.n_beam = pl->p.n_beam;
  g.n_chan = pl->p.n_chan;
  g.n_samp_sub = pl->p.n_samp_sub;
  g.sub0 = sub0;
  g.R = ((g.n_beam + 1 + 3) / 4) * 4;
  const int T1 = g.R / 4;
  g.tiles = T1 * (T1 + 1) / 2;
  // channels per block: as many as fit 4 tasks per thread, multiple of 4
  int cpb = (4 * kGramThreads) / g.tiles;
  cpb = cpb >= 32 ? 32 : (cpb >= 4 ? (cpb / 4) * 4 : (cpb < 1 ? 1 : cpb));
  if (cpb > g.n_chan) cpb = g.n_chan;
  g.cpb = cpb;
  g.ntask = cpb * g.tiles;
  g.cs = g.R * kRS + 1;
  if ((g.cs & 1) == 0) ++g.cs;
  g.psum = pl->psum;
  g.sums = d_sums;
  const bool vec4 = (cpb % 4 == 0) && (g.n_chan % 4 == 0) && (g.beam_stride % 4 == 0) &&
                    ((reinterpret_cast<uintptr_t>(d_data) & 3) == 0);
  const size_t smem = (size_t)cpb * g.cs * 4 + (size_t)g.tiles * 2 + 16;
  dim3 grid((g.n_chan + cpb - 1) / cpb, n_sub);
  const int tpt = (g.ntask + kGramThreads - 1) / kGramThreads;
  cudaError_t e = cudaSuccess;
#define MRAID_GRAM_LAUNCH(T, V, S)                                                                \
  do {                                                                                            \
    e = cudaFuncSetAttribute(gram_u8_kernel<T, V, S>,                                             \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);             \
    if (e == cudaSuccess) gram_u8_kernel<T, V, S><<<grid, kGramThreads, smem, pl->stream>>>(g);    \
  } while (0)
#define MRAID_GRAM_TPT(T)                                                                         \
  do {                                                                                            \
    if (seg) {                                                                                    \
      if (vec4) MRAID_GRAM_LAUNCH(T, true, true); else MRAID_GRAM_LAUNCH(T, false, true);          \
    } else {                                                                                      \
      if (vec4) MRAID_GRAM_LAUNCH(T, true, false); else MRAID_GRAM_LAUNCH(T, false, false);        \
    }                                                                                             \
  } while (0)
  const bool seg = g.n_samp_sub > kGramSegment;
  if (tpt <= 1) MRAID_GRAM_TPT(1);
  else if (tpt == 2) MRAID_GRAM_TPT(2);
  else if (tpt == 3) MRAID_GRAM_TPT(3);
  else MRAID_GRAM_TPT(4);
#undef MRAID_GRAM_TPT
#undef MRAID_GRAM_LAUNCH
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_corr_from_sums(const mraid_plan_s* pl, const int64_t* d_sums, int64_t n_cells,
                                  float* d_corr, bool interleaved) {
  const int psum = pl->psum;
  int warps = (int)(40960 / ((size_t)psum * 8 + kMaxBeam * 4));
  warps = warps < 1 ? 1 : (warps > 8 ? 8 : warps);
  const size_t smem = (size_t)warps * ((size_t)psum * 8 + kMaxBeam * 4);
  cudaError_t e = cudaFuncSetAttribute(corr_from_sums_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (n_cells + warps - 1) / warps;
  if (blocks > 0)
    corr_from_sums_kernel<<<(unsigned)blocks, warps * 32, smem, pl->stream>>>(
        d_sums, n_cells, pl->p.n_beam, psum, pl->np, d_corr, pl->d_degenerate,
        interleaved ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace mraid

// ---------------------------------------------------------------------------
// Float32 samples (beamformer output): correlation on CUDA cores in FP32.
// Each cell's samples are shifted by the cell's first sample of each beam
// before the sums (the covariance does not depend on a per-beam shift, and
// the shift keeps the sums near zero mean so n S_ab - S_a S_b does not
// cancel); the sums, the covariance and the correlation are FP32.
namespace mraid {
namespace {

constexpr int kF32T = 16;       // samples staged per chunk
constexpr int kF32RS = kF32T + 1;  // staged row stride: a tile's 4 rows in different banks

struct F32Args {
  const float* data;
  int64_t beam_stride;
  int n_beam, n_chan, n_samp_sub, sub0;
  int R, cpb, tiles, ntask, cs;
  int np;
  float* corr;
  unsigned long long* degenerate;
};

__global__ void __launch_bounds__(kGramThreads) gram_f32_kernel(F32Args g) {
  extern __shared__ float fsm[];
  float* xs = fsm;                                 // [cpb][R][kF32RS] (+1 pad per channel)
  float* shift = xs + g.cpb * g.cs;                // [cpb][R]
  float* gram = shift + g.cpb * g.R;               // [cpb][R][R] for the epilogue
  uint16_t* tile_ij = reinterpret_cast<uint16_t*>(gram + g.cpb * g.R * g.R);
  const int c0 = blockIdx.x * g.cpb;
  const int sub = g.sub0 + blockIdx.y;
  const int T1 = g.R / 4;
  for (int t = threadIdx.x; t < g.tiles; t += blockDim.x) {
    int ti = 0, rem = t;
    while (rem >= T1 - ti) {
      rem -= T1 - ti;
      ++ti;
    }
    tile_ij[t] = (uint16_t)(ti | ((ti + rem) << 8));
  }
  const int64_t t_sub0 = (int64_t)sub * g.n_samp_sub;
  // shifts: the cell's first sample per beam (0 for the ones row and padding)
  for (int i = threadIdx.x; i < g.cpb * g.R; i += blockDim.x) {
    const int c = i / g.R, r = i % g.R;
    float v = 0.f;
    if (r < g.n_beam && c0 + c < g.n_chan) v = g.data[r * g.beam_stride + t_sub0 * g.n_chan + c0 + c];
    shift[i] = v;
  }
  float acc[4][16];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[j][e] = 0.f;
  __syncthreads();
  for (int tb = 0; tb < g.n_samp_sub; tb += kF32T) {
    __syncthreads();
    const int nv = min(kF32T, g.n_samp_sub - tb);
    for (int w = threadIdx.x; w < g.R * kF32T * g.cpb; w += blockDim.x) {
      const int c = w % g.cpb;
      const int rt = w / g.cpb;
      const int t = rt % kF32T, r = rt / kF32T;
      float v = 0.f;
      if (t < nv && c0 + c < g.n_chan) {
        if (r < g.n_beam)
          v = g.data[r * g.beam_stride + (t_sub0 + tb + t) * g.n_chan + c0 + c] - shift[c * g.R + r];
        else if (r == g.n_beam)
          v = 1.f;
      }
      xs[c * g.cs + r * kF32RS + t] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int task = threadIdx.x + j * kGramThreads;
      if (task < g.ntask) {
        const int c = task % g.cpb;
        const uint16_t tij = tile_ij[task / g.cpb];
        const float* ra = xs + c * g.cs + 4 * (tij & 0xff) * kF32RS;
        const float* rb = xs + c * g.cs + 4 * (tij >> 8) * kF32RS;
        for (int t = 0; t < kF32T; ++t) {
          float a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            a[i] = ra[i * kF32RS + t];
            b[i] = rb[i * kF32RS + t];
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[j][4 * i + k] = fmaf(a[i], b[k], acc[j][4 * i + k]);
        }
      }
    }
  }
  __syncthreads();
  // Gram tiles to shared memory (both triangles), then the correlation
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int task = threadIdx.x + j * kGramThreads;
    if (task >= g.ntask) continue;
    const int c = task % g.cpb;
    const uint16_t tij = tile_ij[task / g.cpb];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int a = 4 * (tij & 0xff) + i, b = 4 * (tij >> 8) + k;
        gram[(c * g.R + a) * g.R + b] = acc[j][4 * i + k];
        gram[(c * g.R + b) * g.R + a] = acc[j][4 * i + k];
      }
  }
  __syncthreads();
  const int N = g.n_beam;
  for (int e = threadIdx.x; e < g.cpb * g.np; e += blockDim.x) {
    const int c = e / g.np;
    if (c0 + c >= g.n_chan) continue;
    int rem = e - c * g.np, a = 0;
    while (rem >= N - a) {
      rem -= N - a;
      ++a;
    }
    const int b = a + rem;
    const float* G = gram + c * g.R * g.R;
    const float n = G[N * g.R + N];
    const float va = n * G[a * g.R + a] - G[a * g.R + N] * G[a * g.R + N];
    const float vb = n * G[b * g.R + b] - G[b * g.R + N] * G[b * g.R + N];
    float r;
    if (a == b) {
      r = 1.f;
      if (!(va > 0.f)) atomicAdd(g.degenerate, 1ull);
    } else if (!(va > 0.f) || !(vb > 0.f)) {
      r = 0.f;
    } else {
      const float cov = n * G[a * g.R + b] - G[a * g.R + N] * G[b * g.R + N];
      r = cov * rsqrtf(va) * rsqrtf(vb);
    }
    g.corr[((int64_t)blockIdx.y * g.n_chan + c0 + c) * g.np + (e - c * g.np)] = r;
  }
}

}  // namespace

cudaError_t launch_gram_f32(const mraid_plan_s* pl, const float* d_data, int sub0, int n_sub,
                            float* d_corr) {
  F32Args g;
  g.data = d_data;
  g.beam_stride = pl->beam_stride;
  g.n_beam = pl->p.n_beam;
  g.n_chan = pl->p.n_chan;
  g.n_samp_sub = pl->p.n_samp_sub;
  g.sub0 = sub0;
  g.R = ((g.n_beam + 1 + 3) / 4) * 4;
  const int T1 = g.R / 4;
  g.tiles = T1 * (T1 + 1) / 2;
  int cpb = (4 * kGramThreads) / g.tiles;
  cpb = cpb >= 16 ? 16 : (cpb < 1 ? 1 : cpb);
  if (cpb > g.n_chan) cpb = g.n_chan;
  g.cpb = cpb;
  g.ntask = cpb * g.tiles;
  g.cs = g.R * kF32RS + 1;
  if ((g.cs & 1) == 0) ++g.cs;
  g.np = pl->np;
  g.corr = d_corr;
  g.degenerate = pl->d_degenerate;
  const size_t smem = sizeof(float) * ((size_t)cpb * g.cs + (size_t)cpb * g.R + (size_t)cpb * g.R * g.R) +
                      (size_t)g.tiles * 2 + 16;
  cudaError_t e = cudaFuncSetAttribute(gram_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((g.n_chan + cpb - 1) / cpb, n_sub);
  gram_f32_kernel<<<grid, kGramThreads, smem, pl->stream>>>(g);
  return cudaGetLastError();
}

}  // namespace mraid
