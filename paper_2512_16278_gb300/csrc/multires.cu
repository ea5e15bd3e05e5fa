// multires.cu - Gram sums of longer sub-intervals from shorter ones.
//
// Section 4.2 (Table 1, Fig. 7) runs the method at sub-interval lengths
// from 0.05 s to 10 s. The augmented Gram of Eq. 1 over a sub-interval made
// of m consecutive shorter ones is the sum of their Grams: every entry
// (sum x_a x_b, sum x_a, n) is a sum over samples, and int64 addition is
// exact, so the longer timescales cost no further pass over the samples.
// This kernel forms out[k] = sum_{j < m} in[k m + j] for every cell entry:
// a plain streaming reduction, coalesced along the (channel, entry) run of
// one sub-integration, bound by HBM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mraid {
namespace {

constexpr int kAggThreads = 256;

// per_sub: int64 entries of one sub-integration (n_chan * P); n_out_sub:
// output sub-intervals; m: input sub-integrations per output one.
template <int V>
__global__ void __launch_bounds__(kAggThreads)
gram_aggregate_kernel(const int64_t* __restrict__ src, int64_t* __restrict__ dst,
                      int64_t per_sub, int n_out_sub, int m) {
  const int64_t per_vec = per_sub / V;
  const int64_t n_out = per_vec * n_out_sub;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += stride) {
    const int64_t k = o / per_vec, e = o - k * per_vec;
    const int64_t* s = src + (k * m * per_vec + e) * V;
    if (V == 2) {
      longlong2 acc = make_longlong2(0, 0);
      for (int j = 0; j < m; ++j) {
        const longlong2 v = *reinterpret_cast<const longlong2*>(s + (int64_t)j * per_sub);
        acc.x += v.x;
        acc.y += v.y;
      }
      *reinterpret_cast<longlong2*>(dst + o * V) = acc;
    } else {
      int64_t acc = 0;
      for (int j = 0; j < m; ++j) acc += s[(int64_t)j * per_sub];
      dst[o] = acc;
    }
  }
}

}  // namespace

cudaError_t launch_gram_aggregate(const mraid_plan_s* pl, const int64_t* d_src, int64_t* d_dst,
                                  int n_out_sub, int m) {
  const int64_t per_sub = (int64_t)pl->p.n_chan * pl->psum;
  const bool vec2 = per_sub % 2 == 0 && (reinterpret_cast<uintptr_t>(d_src) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(d_dst) & 15) == 0;
  const int64_t n_out = per_sub / (vec2 ? 2 : 1) * n_out_sub;
  if (n_out <= 0) return cudaSuccess;
  int64_t blocks = (n_out + kAggThreads - 1) / kAggThreads;
  const int64_t cap = (int64_t)pl->sm_count * 8;  // 8 resident blocks per SM
  if (blocks > cap) blocks = cap;
  if (vec2)
    gram_aggregate_kernel<2><<<(unsigned)blocks, kAggThreads, 0, pl->stream>>>(d_src, d_dst, per_sub,
                                                                              n_out_sub, m);
  else
    gram_aggregate_kernel<1><<<(unsigned)blocks, kAggThreads, 0, pl->stream>>>(d_src, d_dst, per_sub,
                                                                              n_out_sub, m);
  return cudaGetLastError();
}

}  // namespace mraid

// ---------------------------------------------------------------------------
// Entry points (include/mraid.h)

using namespace mraid;

mraid_status mraid_multires(mraid_plan_t pl, const void* d_data, int32_t n_levels,
                            const int32_t* factors, float* const* d_stats,
                            uint8_t* const* d_flags, mraid_flag_info* infos) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (!d_data || !factors || !d_stats || !d_flags || n_levels < 1 || n_levels > kMaxLevels) {
    set_error("mraid_multires: d_data, factors, d_stats and d_flags are required; n_levels in 1..%d",
              kMaxLevels);
    return MRAID_ERR_INVALID_ARG;
  }
  if (pl->p.bit_depth != 8) {
    set_error("mraid_multires: exact Gram sums exist for 8-bit samples only");
    return MRAID_ERR_UNSUPPORTED;
  }
  const int n_sub = pl->p.n_sub, n_chan = pl->p.n_chan;
  int order[kMaxLevels];
  for (int i = 0; i < n_levels; ++i) {
    const int f = factors[i];
    if (f < 1 || f > n_sub || !d_stats[i] || !d_flags[i]) {
      set_error("mraid_multires: level %d: factor %d outside 1..%d or a NULL output", i, f, n_sub);
      return MRAID_ERR_INVALID_ARG;
    }
    for (int j = 0; j < i; ++j)
      if (factors[j] == f) {
        set_error("mraid_multires: factor %d given twice", f);
        return MRAID_ERR_INVALID_ARG;
      }
    // insertion into ascending factor order
    int k = i;
    while (k > 0 && factors[order[k - 1]] > f) {
      order[k] = order[k - 1];
      --k;
    }
    order[k] = i;
  }
  // sums of the longer levels, one after another in ml_sums
  const int64_t per_sub = (int64_t)n_chan * pl->psum;
  size_t off[kMaxLevels] = {};
  size_t need = 0;
  for (int i = 0; i < n_levels; ++i)
    if (factors[i] > 1) {
      off[i] = need;
      need += (size_t)(n_sub / factors[i]) * (size_t)per_sub;
      need = (need + 1) & ~size_t(1);  // keep every level 16-byte aligned
    }
  st = ensure_workspace(pl, (size_t)pl->n_cells);
  if (st != MRAID_OK) return st;
  cudaError_t e = cudaSuccess;
  if (need > pl->ml_sums_elems) {
    cudaFree(pl->ml_sums);
    pl->ml_sums = nullptr;
    pl->ml_sums_elems = 0;
    e = cudaMalloc(&pl->ml_sums, need * sizeof(int64_t));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "multires sums allocation");
    }
    pl->ml_sums_elems = need;
  }
  if (!pl->d_ml_info) {
    e = cudaMalloc(&pl->d_ml_info, kMaxLevels * sizeof(mraid_flag_info));
    if (e == cudaSuccess) e = cudaMallocHost(&pl->h_ml_info, kMaxLevels * sizeof(mraid_flag_info));
    if (e != cudaSuccess) {
      cudaFree(pl->d_ml_info);
      pl->d_ml_info = nullptr;
      cudaGetLastError();
      return cuda_fail(e, "multires report allocation");
    }
  }
  auto reset_counters = [&]() {
    cudaError_t r = cudaMemsetAsync(pl->d_degenerate, 0, sizeof(unsigned long long), pl->stream);
    if (r == cudaSuccess)
      r = cudaMemsetAsync(pl->d_sweeps, 0, 3 * sizeof(unsigned long long), pl->stream);
    return r;
  };
  e = cudaMemsetAsync(pl->d_ml_info, 0, (size_t)n_levels * sizeof(mraid_flag_info), pl->stream);
  if (e == cudaSuccess) e = reset_counters();
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  // the one pass over the samples: Gram sums of every sub-integration, and
  // the correlation too when the plan's own length is a level; the
  // aggregation adds whole sub-integrations, so it does not depend on the
  // sums' layout, and the correlation kernel reads either
  const bool has1 = factors[order[0]] == 1;
  bool inter = false;
  st = gram_sums_pass(pl, d_data, has1 ? pl->ws.corr : nullptr, &inter);
  if (st != MRAID_OK) return st;
  for (int li = 0; li < n_levels; ++li) {
    const int i = order[li], f = factors[i];
    const int n_f = n_sub / f;
    const int64_t cells = (int64_t)n_f * n_chan;
    if (f > 1) {
      // source: the longest level already formed whose length divides f
      int g = 1;
      const int64_t* src = pl->ws.sums;
      for (int lj = 0; lj < li; ++lj) {
        const int j = order[lj];
        if (factors[j] > g && f % factors[j] == 0) {
          g = factors[j];
          src = pl->ml_sums + off[j];
        }
      }
      int64_t* dst = pl->ml_sums + off[i];
      e = reset_counters();
      if (e == cudaSuccess)
        e = MRAID_PROF(pl, K_AGG, launch_gram_aggregate(pl, src, dst, n_f, f / g));
      if (e == cudaSuccess)
        e = MRAID_PROF(pl, K_CORR, launch_corr_from_sums(pl, dst, cells, pl->ws.corr, inter));
      if (e != cudaSuccess) return cuda_fail(e, "multires sums");
    }
    e = MRAID_PROF(pl, K_EIG, launch_eig(pl, pl->ws.corr, cells, nullptr, nullptr, d_stats[i]));
    if (e != cudaSuccess) return cuda_fail(e, "eig launch");
    e = MRAID_PROF(pl, K_FLAG, launch_flag(pl, d_stats[i], d_flags[i], cells, pl->d_ml_info + i));
    if (e != cudaSuccess) return cuda_fail(e, "flag launch");
    e = cudaMemcpyAsync(&pl->d_ml_info[i].n_degenerate, pl->d_degenerate, sizeof(int64_t),
                        cudaMemcpyDeviceToDevice, pl->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&pl->d_ml_info[i].jacobi_sweeps, pl->d_sweeps, 2 * sizeof(int64_t),
                          cudaMemcpyDeviceToDevice, pl->stream);
    if (e == cudaSuccess)  // the FP64 q1 count (low half of the counter)
      e = cudaMemcpyAsync(&pl->d_ml_info[i].q1_refined, pl->d_sweeps + 2, sizeof(int32_t),
                          cudaMemcpyDeviceToDevice, pl->stream);
    if (e != cudaSuccess) return cuda_fail(e, "counter copy");
  }
  e = cudaMemcpyAsync(pl->h_ml_info, pl->d_ml_info, (size_t)n_levels * sizeof(mraid_flag_info),
                      cudaMemcpyDeviceToHost, pl->stream);
  if (e != cudaSuccess) return cuda_fail(e, "info copy");
  pl->pending_ml = infos;
  pl->pending_ml_n = infos ? n_levels : 0;
  return MRAID_OK;
}
