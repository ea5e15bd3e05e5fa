// pol2.cu - total power of two recorded polarisations (Section 2: the FAST
// data record two; Eq. 1's B is the total power).
//
// With x_a = p0_a + p1_a, sum_t x_a x_b is the sum of the four
// polarisation products sum p0_a p0_b + p0_a p1_b + p1_a p0_b + p1_a p1_b,
// and sum_t x_a = sum p0_a + sum p1_a. So the exact Gram of the total power
// is a fold of the exact Gram of the 2N stacked polarisation blocks (block
// p*N + a = polarisation p of beam a), which the 8-bit Gram kernels form
// as they stand; int64 addition keeps it exact. (Where the tensor-core Gram
// takes the shape it adds the polarisations itself and needs none of this.)
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mraid {
namespace {

// out [cell][P], P = (N+1)(N+2)/2, from in [cell][P2], P2 = (2N+1)(2N+2)/2;
// both packed upper triangles, row-major.
__global__ void pol2_fold_kernel(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                 int64_t n_cells, int N, int P, int P2) {
  const int M2 = 2 * N + 1;
  const int64_t total = n_cells * P;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / P;
    int e = (int)(idx - cell * P);
    int a = 0;
    while (e >= N + 1 - a) {  // row a of the (N+1)-triangle holds N + 1 - a entries
      e -= N + 1 - a;
      ++a;
    }
    const int b = a + e;
    const int64_t* S = in + cell * P2;
    auto at = [&](int i, int j) {  // entry (i, j) of the stacked Gram, any order
      if (i > j) {
        const int t = i;
        i = j;
        j = t;
      }
      return S[i * M2 - i * (i - 1) / 2 + (j - i)];
    };
    int64_t v;
    if (a == N) v = at(2 * N, 2 * N);                          // n
    else if (b == N) v = at(a, 2 * N) + at(a + N, 2 * N);      // sum x_a
    else v = at(a, b) + at(a, b + N) + at(a + N, b) + at(a + N, b + N);
    out[idx] = v;
  }
}

}  // namespace

cudaError_t launch_pol2_fold(const mraid_plan_s* pl, const int64_t* d_stacked, int64_t n_cells,
                             int64_t* d_sums) {
  const int N = pl->p.n_beam;
  const int P = pl->psum, P2 = (2 * N + 1) * (2 * N + 2) / 2;
  const int64_t total = n_cells * P;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)pl->sm_count * 16) blocks = (int64_t)pl->sm_count * 16;
  if (blocks < 1) return cudaSuccess;
  pol2_fold_kernel<<<(unsigned)blocks, 256, 0, pl->stream>>>(d_stacked, d_sums, n_cells, N, P, P2);
  return cudaGetLastError();
}

}  // namespace mraid

namespace mraid {
namespace {
// True when the tensor-core Gram takes a two-polarisation block whole: it
// adds the polarisations in its converter and the pieces of each
// sub-integration in its epilogue, so it writes the total power's sums
// and correlation directly.
bool pol2_on_tensor_cores(const mraid_plan_s* pl, const void* d_data) {
  return !pl->force_dp4a && pl->p.bit_depth == 8 && gram_tc_supported(pl, d_data, 2);
}

// Otherwise: the exact 8-bit Gram of the 2N stacked blocks (a plan view
// with 2N beams), folded into the total power's sums [cell][P] in d_sums.
mraid_status pol2_stacked_sums(mraid_plan_s* pl, const void* d_data, int64_t* d_sums) {
  const int N = pl->p.n_beam;
  const int P2 = (2 * N + 1) * (2 * N + 2) / 2;
  const size_t need = (size_t)pl->n_cells * P2;
  if (need > pl->pol_cells) {  // pol_cells counts int64 elements
    cudaFree(pl->pol_sums);
    pl->pol_sums = nullptr;
    pl->pol_cells = 0;
    cudaError_t e = cudaMalloc(&pl->pol_sums, need * sizeof(int64_t));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "two-polarisation workspace allocation");
    }
    pl->pol_cells = need;
  }
  mraid_plan_s v;
  v.p = pl->p;
  v.p.n_beam = 2 * N;
  v.p.keep = nullptr;
  v.device = pl->device;
  v.sm_count = pl->sm_count;
  v.stream = pl->stream;
  v.n_cells = pl->n_cells;
  v.beam_stride = pl->beam_stride;
  v.np = 2 * N * (2 * N + 1) / 2;
  v.psum = P2;
  v.d_degenerate = pl->d_degenerate;
  v.d_error = pl->d_error;
  v.force_dp4a = pl->force_dp4a;
  v.tc_variant = tc_default_variant(2 * N);
  cudaError_t e = cudaSuccess;
  if (!v.force_dp4a && gram_tc_supported(&v, d_data)) {
    e = MRAID_PROF(pl, K_GRAM_TC,
                   launch_gram_tc(&v, static_cast<const uint8_t*>(d_data), 0, v.p.n_sub,
                                  pl->pol_sums, nullptr));
  } else {
    for (int s = 0; s < v.p.n_sub && e == cudaSuccess; s += kMaxSubPerLaunch) {
      const int ns = (v.p.n_sub - s) < kMaxSubPerLaunch ? (v.p.n_sub - s) : kMaxSubPerLaunch;
      e = MRAID_PROF(pl, K_GRAM,
                     launch_gram_u8(&v, static_cast<const uint8_t*>(d_data), s, ns,
                                    pl->pol_sums + (int64_t)s * v.p.n_chan * P2));
    }
  }
  if (e == cudaSuccess)
    e = MRAID_PROF(pl, K_POL2_FOLD, launch_pol2_fold(pl, pl->pol_sums, pl->n_cells, d_sums));
  return e == cudaSuccess ? MRAID_OK : cuda_fail(e, "two-polarisation Gram");
}

mraid_status check_pol2(const mraid_plan_s* pl) {
  if (pl->p.bit_depth != 8 || 2 * pl->p.n_beam > kMaxBeam) {
    set_error("two polarisations: 8-bit samples and at most %d beams", kMaxBeam / 2);
    return MRAID_ERR_UNSUPPORTED;
  }
  return MRAID_OK;
}

// Sums ([cell][P], may be null) and correlation (may be null) of the
// total power of a two-polarisation block; counts zero-variance beams.
mraid_status pol2_ccm(mraid_plan_s* pl, const void* d_data, int64_t* d_sums, float* d_corr) {
  cudaError_t e = cudaMemsetAsync(pl->d_degenerate, 0, sizeof(unsigned long long), pl->stream);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  if (pol2_on_tensor_cores(pl, d_data)) {
    e = MRAID_PROF(pl, K_GRAM_TC,
                   launch_gram_tc(pl, static_cast<const uint8_t*>(d_data), 0, pl->p.n_sub, d_sums,
                                  d_corr, nullptr, 2));
    return e == cudaSuccess ? MRAID_OK : cuda_fail(e, "gram_tc launch");
  }
  int64_t* sums = d_sums;
  if (!sums) {
    mraid_status st = ensure_workspace(pl, (size_t)pl->n_cells);
    if (st != MRAID_OK) return st;
    sums = pl->ws.sums;
  }
  mraid_status st = pol2_stacked_sums(pl, d_data, sums);
  if (st != MRAID_OK) return st;
  if (d_corr) {
    // the stacked Gram's own counts are of the 2N blocks: count again
    e = cudaMemsetAsync(pl->d_degenerate, 0, sizeof(unsigned long long), pl->stream);
    if (e == cudaSuccess)
      e = MRAID_PROF(pl, K_CORR, launch_corr_from_sums(pl, sums, pl->n_cells, d_corr));
    if (e != cudaSuccess) return cuda_fail(e, "corr launch");
  }
  return MRAID_OK;
}
}  // namespace
}  // namespace mraid

// ---------------------------------------------------------------------------
// Entry points (include/mraid.h)

using namespace mraid;

mraid_status mraid_ccm_pol2(mraid_plan_t pl, const void* d_data, int64_t* d_sums,
                            float* d_corr) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (!d_data || (!d_sums && !d_corr)) {
    set_error("mraid_ccm_pol2: d_data and one of d_sums, d_corr are required");
    return MRAID_ERR_INVALID_ARG;
  }
  st = check_pol2(pl);
  if (st != MRAID_OK) return st;
  return pol2_ccm(pl, d_data, d_sums, d_corr);
}

mraid_status mraid_run_pol2(mraid_plan_t pl, const void* d_data, float* d_evals, float* d_q1,
                            float* d_stat, uint8_t* d_flags, mraid_flag_info* info) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (!d_data || !d_stat || !d_flags) {
    set_error("mraid_run_pol2: d_data, d_stat and d_flags are required");
    return MRAID_ERR_INVALID_ARG;
  }
  st = check_pol2(pl);
  if (st != MRAID_OK) return st;
  st = ensure_workspace(pl, (size_t)pl->n_cells);
  if (st != MRAID_OK) return st;
  if (d_q1) {
    st = evals_for_q1(pl, (size_t)pl->n_cells, &d_evals);
    if (st != MRAID_OK) return st;
  }
  cudaError_t e = cudaMemsetAsync(pl->d_sweeps, 0, 3 * sizeof(unsigned long long), pl->stream);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  st = pol2_ccm(pl, d_data, nullptr, pl->ws.corr);
  if (st != MRAID_OK) return st;
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
