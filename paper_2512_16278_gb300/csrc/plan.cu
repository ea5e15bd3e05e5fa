// plan.cu - the C ABI (include/mraid.h): validation, plans, launches of the
// per-stage kernels and the host-buffer path.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "internal.h"

namespace mraid {

static thread_local char g_err[512];

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

mraid_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return MRAID_ERR_OOM;
  return MRAID_ERR_CUDA;
}

const char* kernel_name(int id) {
  switch (id) {
    case K_GRAM: return "gram_u8";
    case K_CORR: return "corr_from_sums";
    case K_EIG: return "eig";
    case K_FLAG: return "flag_clip";
    case K_GRAM_TC: return "gram_tc";
    case K_GRAM_F32: return "gram_f32";
    case K_GRAM_TC_F32: return "gram_tc_f32";
    case K_AGG: return "gram_aggregate";
    case K_BP_INPUT: return "bandpass_input";
    case K_ARPLS: return "arpls";
    case K_CCM_BP: return "ccm_bandpass";
    case K_POL2_FOLD: return "pol2_fold";
    case K_GRAM_TCL: return "gram_tcl";
  }
  return "unknown";
}

static cudaEvent_t take_event(mraid_plan_s* pl) {
  if (!pl->prof.pool.empty()) {
    cudaEvent_t e = pl->prof.pool.back();
    pl->prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void prof_begin(mraid_plan_s* pl, int id, cudaEvent_t* start, cudaStream_t stream) {
  (void)id;
  *start = nullptr;
  if (!pl->prof.on) return;
  *start = take_event(pl);
  if (*start) cudaEventRecord(*start, stream);
}

void prof_end(mraid_plan_s* pl, int id, cudaEvent_t start, cudaStream_t stream) {
  if (!pl->prof.on || !start) return;
  cudaEvent_t stop = take_event(pl);
  if (!stop) return;
  cudaEventRecord(stop, stream);
  pl->prof.pending.push_back({id, start, stop});
}

// Fold recorded event pairs into the totals (the stream has been synced).
static void prof_fold(mraid_plan_s* pl) {
  for (auto& r : pl->prof.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
      pl->prof.total_ms[r.id] += ms;
      pl->prof.launches[r.id] += 1;
    }
    pl->prof.pool.push_back(r.start);
    pl->prof.pool.push_back(r.stop);
  }
  pl->prof.pending.clear();
}


// Plan helpers shared with the entry points of the other files (internal.h).

// Workspace of the tridiagonal eigensolver, for beam counts it serves.
mraid_status ensure_tri_workspace(mraid_plan_s* pl, size_t cells) {
  const int N = pl->p.n_beam;
  const bool reg = N == 2 || N == 3 || N == 4 || N == 13 || N == 19;
  if (reg) {  // T of the split tridiagonal route: 2N floats per cell
    if (pl->ws.de_cells >= cells) return MRAID_OK;
    cudaFree(pl->ws.de);
    pl->ws.de = nullptr;
    pl->ws.de_cells = 0;
    cudaError_t e = cudaMalloc(&pl->ws.de, cells * 2 * (size_t)N * sizeof(float));
    if (e != cudaSuccess) {
      pl->ws.de = nullptr;
      cudaGetLastError();
      return cuda_fail(e, "eigensolver workspace");
    }
    pl->ws.de_cells = cells;
    return MRAID_OK;
  }
  if (pl->ws.tri_cells >= cells) return MRAID_OK;
  cudaFree(pl->ws.tri);
  pl->ws.tri = nullptr;
  pl->ws.tri_cells = 0;
  cudaError_t e = cudaMalloc(&pl->ws.tri, cells * tri_workspace_floats(N) * sizeof(float));
  if (e != cudaSuccess) {
    pl->ws.tri = nullptr;
    cudaGetLastError();
    return cuda_fail(e, "eigensolver workspace");
  }
  pl->ws.tri_cells = cells;
  return MRAID_OK;
}

mraid_status ensure_workspace(mraid_plan_s* pl, size_t cells) {
  mraid_status st = ensure_tri_workspace(pl, cells);
  if (st != MRAID_OK) return st;
  if (pl->ws.cells >= cells) return MRAID_OK;
  if (pl->inject_alloc) {  // MRAID_FAULT_ALLOC: this allocation fails
    pl->inject_alloc = false;
    set_error("workspace allocation: out of memory (injected fault)");
    return MRAID_ERR_OOM;
  }
  cudaFree(pl->ws.sums);
  cudaFree(pl->ws.corr);
  pl->ws.sums = nullptr;
  pl->ws.corr = nullptr;
  pl->ws.cells = 0;
  cudaError_t e = cudaMalloc(&pl->ws.sums, cells * (size_t)pl->psum * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&pl->ws.corr, cells * (size_t)pl->np * sizeof(float));
  if (e != cudaSuccess) {
    cudaFree(pl->ws.sums);
    pl->ws.sums = nullptr;
    pl->ws.corr = nullptr;
    cudaGetLastError();
    return cuda_fail(e, "workspace allocation");
  }
  pl->ws.cells = cells;
  return MRAID_OK;
}

// buffers of a q1 request: the cell list of the FP64 step, and an
// eigenvalue buffer when the caller wants q1 but not evals
mraid_status evals_for_q1(mraid_plan_s* pl, size_t cells, float** evals) {
  if (pl->ws.q1_list_cells < cells || !pl->ws.q1_list_n) {
    cudaFree(pl->ws.q1_list);
    pl->ws.q1_list = nullptr;
    pl->ws.q1_list_cells = 0;
    cudaError_t e = cudaMalloc(&pl->ws.q1_list, cells * sizeof(uint32_t));
    if (e == cudaSuccess && !pl->ws.q1_list_n) e = cudaMalloc(&pl->ws.q1_list_n, sizeof(unsigned));
    if (e != cudaSuccess) {
      cudaFree(pl->ws.q1_list);
      pl->ws.q1_list = nullptr;
      cudaGetLastError();
      return cuda_fail(e, "q1 list");
    }
    pl->ws.q1_list_cells = cells;
  }
  if (*evals || !eig_q1_needs_evals(pl->p.n_beam)) return MRAID_OK;
  if (pl->ws.evals_cells < cells) {
    cudaFree(pl->ws.evals);
    pl->ws.evals = nullptr;
    pl->ws.evals_cells = 0;
    cudaError_t e = cudaMalloc(&pl->ws.evals, cells * (size_t)pl->p.n_beam * sizeof(float));
    if (e != cudaSuccess) {
      pl->ws.evals = nullptr;
      cudaGetLastError();
      return cuda_fail(e, "eigenvalue workspace");
    }
    pl->ws.evals_cells = cells;
  }
  *evals = pl->ws.evals;
  return MRAID_OK;
}

mraid_status check_plan(mraid_plan_t pl) {
  if (!pl) {
    set_error("plan is NULL");
    return MRAID_ERR_INVALID_ARG;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != pl->device) {
    e = cudaSetDevice(pl->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  }
  return MRAID_OK;
}

// Gram sums + correlation of sub-integrations [sub0, sub0+n_sub) of d_data;
// d_sums / d_corr are indexed by cell relative to sub0.
mraid_status ccm_range(mraid_plan_s* pl, const void* d_data, int sub0, int n_sub, int64_t* d_sums,
                       float* d_corr) {
  const int64_t cells = (int64_t)n_sub * pl->p.n_chan;
  if (pl->p.bit_depth == 32) {
    if (d_sums) {
      set_error("exact sums exist for 8-bit data only");
      return MRAID_ERR_INVALID_ARG;
    }
    if (!d_corr) return MRAID_OK;
    if (!pl->force_dp4a && gram_tc_f32_supported(pl, d_data)) {
      cudaError_t e = MRAID_PROF(pl, K_GRAM_TC_F32,
                                 launch_gram_tc_f32(pl, static_cast<const float*>(d_data), sub0,
                                                    n_sub, d_corr));
      return e == cudaSuccess ? MRAID_OK : cuda_fail(e, "gram_tc_f32 launch");
    }
    for (int s = 0; s < n_sub; s += kMaxSubPerLaunch) {
      const int ns = (n_sub - s) < kMaxSubPerLaunch ? (n_sub - s) : kMaxSubPerLaunch;
      cudaError_t e = MRAID_PROF(pl, K_GRAM_F32,
                                 launch_gram_f32(pl, static_cast<const float*>(d_data), sub0 + s, ns,
                                                 d_corr + (int64_t)s * pl->p.n_chan * pl->np));
      if (e != cudaSuccess) return cuda_fail(e, "gram_f32 launch");
    }
    return MRAID_OK;
  }
  if (!pl->force_dp4a && gram_tc_supported(pl, d_data)) {
    cudaError_t e = MRAID_PROF(pl, K_GRAM_TC,
                               launch_gram_tc(pl, static_cast<const uint8_t*>(d_data), sub0, n_sub,
                                              d_sums, d_corr));
    return e == cudaSuccess ? MRAID_OK : cuda_fail(e, "gram_tc launch");
  }
  int64_t* sums = d_sums;
  if (!sums) {
    mraid_status st = ensure_workspace(pl, (size_t)cells);
    if (st != MRAID_OK) return st;
    sums = pl->ws.sums;
  }
  if (!pl->force_dp4a && gram_tcl_supported(pl, d_data)) {
    cudaError_t e = MRAID_PROF(pl, K_GRAM_TCL,
                               launch_gram_tcl(pl, static_cast<const uint8_t*>(d_data), sub0, n_sub,
                                               sums));
    if (e != cudaSuccess) return cuda_fail(e, "gram_tcl launch");
  } else {
    for (int s = 0; s < n_sub; s += kMaxSubPerLaunch) {
      const int ns = (n_sub - s) < kMaxSubPerLaunch ? (n_sub - s) : kMaxSubPerLaunch;
      cudaError_t e = MRAID_PROF(pl, K_GRAM,
                                 launch_gram_u8(pl, static_cast<const uint8_t*>(d_data), sub0 + s,
                                                ns, sums + (int64_t)s * pl->p.n_chan * pl->psum));
      if (e != cudaSuccess) return cuda_fail(e, "gram launch");
    }
  }
  if (d_corr) {
    cudaError_t e = MRAID_PROF(pl, K_CORR, launch_corr_from_sums(pl, sums, cells, d_corr));
    if (e != cudaSuccess) return cuda_fail(e, "corr launch");
  }
  return MRAID_OK;
}

mraid_status enqueue_info_copy(mraid_plan_s* pl, mraid_flag_info* info) {
  cudaError_t e = cudaMemcpyAsync(pl->h_info, pl->d_info, sizeof(mraid_flag_info),
                                  cudaMemcpyDeviceToHost, pl->stream);
  if (e != cudaSuccess) return cuda_fail(e, "info copy");
  pl->pending_info = info;
  return MRAID_OK;
}

// One pass over 8-bit samples for the paths that need the Gram sums: the
// int64 sums of every sub-integration into ws.sums (and the correlation
// into d_corr when it is not null). The tensor-core kernel writes the sums
// interleaved by 8 channels ([cell / 8][P][cell % 8], 64-byte store runs;
// *interleaved = true); otherwise they are [cell][P].
mraid_status gram_sums_pass(mraid_plan_s* pl, const void* d_data, float* d_corr,
                            bool* interleaved) {
  *interleaved = !pl->force_dp4a && gram_tc_supported(pl, d_data);
  if (*interleaved) {
    cudaError_t e = MRAID_PROF(pl, K_GRAM_TC,
                               launch_gram_tc(pl, static_cast<const uint8_t*>(d_data), 0,
                                              pl->p.n_sub, nullptr, d_corr, pl->ws.sums));
    return e == cudaSuccess ? MRAID_OK : cuda_fail(e, "gram_tc launch");
  }
  return ccm_range(pl, d_data, 0, pl->p.n_sub, pl->ws.sums, d_corr);
}

mraid_status plan_prepare(mraid_plan_s* pl) {
  mraid_status st = ensure_workspace(pl, (size_t)pl->n_cells);
  if (st != MRAID_OK) return st;
  float* ev = nullptr;
  return evals_for_q1(pl, (size_t)pl->n_cells, &ev);
}

void plan_deliver_info(mraid_plan_s* pl) {
  if (pl->pending_info) {
    *pl->pending_info = *pl->h_info;
    pl->pending_info = nullptr;
  }
}

}  // namespace mraid

namespace mraid {
namespace {
// Mean time of `reps` runs of fn on the plan's stream (after one warm-up).
template <class F>
mraid_status time_runs(mraid_plan_s* pl, int reps, cudaEvent_t e0, cudaEvent_t e1, F fn,
                       float* ms) {
  mraid_status st = fn();
  if (st != MRAID_OK) return st;
  cudaError_t e = cudaEventRecord(e0, pl->stream);
  for (int r = 0; r < reps && st == MRAID_OK && e == cudaSuccess; ++r) st = fn();
  if (st != MRAID_OK) return st;
  if (e == cudaSuccess) e = cudaEventRecord(e1, pl->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e != cudaSuccess) return cuda_fail(e, "mraid_autotune");
  *ms /= reps;
  return MRAID_OK;
}
}  // namespace
}  // namespace mraid

using namespace mraid;

extern "C" {

int32_t mraid_abi_version(void) { return MRAID_ABI_VERSION; }

const char* mraid_last_error(void) { return g_err; }

const char* mraid_status_string(mraid_status s) {
  switch (s) {
    case MRAID_OK: return "ok";
    case MRAID_ERR_INVALID_ARG: return "invalid argument";
    case MRAID_ERR_UNSUPPORTED: return "unsupported";
    case MRAID_ERR_OOM: return "out of memory";
    case MRAID_ERR_CUDA: return "CUDA error";
    case MRAID_ERR_TIMEOUT: return "device wait timed out";
    case MRAID_ERR_NOT_READY: return "not ready";
  }
  return "unknown status";
}

void mraid_default_params(mraid_params* p, int32_t n_beam, int32_t n_chan, int32_t n_samp_sub,
                          int32_t n_sub) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->n_beam = n_beam;
  p->n_chan = n_chan;
  p->n_samp_sub = n_samp_sub;
  p->n_sub = n_sub;
  p->bit_depth = 8;
  p->beam_stride = 0;
  p->eig_k = 3.0;
  p->vec_t = 1.0;
  p->max_clip_iter = 64;
  p->keep = nullptr;
}

mraid_status mraid_validate(const mraid_params* p) {
  g_err[0] = 0;
  if (!p) {
    set_error("params is NULL");
    return MRAID_ERR_INVALID_ARG;
  }
  if (p->n_beam < 2) {
    set_error("n_beam %d < 2", p->n_beam);
    return MRAID_ERR_INVALID_ARG;
  }
  if (p->n_beam > kMaxBeam) {
    set_error("n_beam %d > %d", p->n_beam, kMaxBeam);
    return MRAID_ERR_UNSUPPORTED;
  }
  if (p->n_chan < 1 || p->n_sub < 1) {
    set_error("n_chan %d and n_sub %d must be >= 1", p->n_chan, p->n_sub);
    return MRAID_ERR_INVALID_ARG;
  }
  if (p->n_samp_sub < 2 || p->n_samp_sub > kMaxSampSub) {
    set_error("n_samp_sub %d outside [2, %d]", p->n_samp_sub, kMaxSampSub);
    return MRAID_ERR_INVALID_ARG;
  }
  if (p->bit_depth != 8 && p->bit_depth != 32) {
    set_error("bit_depth %d: 8-bit and float32 samples are built", p->bit_depth);
    return MRAID_ERR_UNSUPPORTED;
  }
  if ((int64_t)p->n_sub * p->n_chan > 2147483647ll) {  // before any product with it
    set_error("n_sub * n_chan exceeds 2^31 - 1 cells");
    return MRAID_ERR_INVALID_ARG;
  }
  // at most 2^31 cells of 2^20 samples: no overflow
  const int64_t dense = (int64_t)p->n_sub * p->n_samp_sub * p->n_chan;
  if (p->beam_stride != 0 && p->beam_stride < dense) {
    set_error("beam_stride %lld smaller than one beam's block (%lld)", (long long)p->beam_stride,
              (long long)dense);
    return MRAID_ERR_INVALID_ARG;
  }
  if (!(p->eig_k > 0.0) || !(p->vec_t >= 0.0) || p->eig_k > 1e6) {
    set_error("eig_k must be > 0 and vec_t >= 0");
    return MRAID_ERR_INVALID_ARG;
  }
  if (p->max_clip_iter < 1 || p->max_clip_iter > kMaxClipIter) {
    set_error("max_clip_iter %d outside [1, %d]", p->max_clip_iter, kMaxClipIter);
    return MRAID_ERR_INVALID_ARG;
  }
  if (p->reserved != 0) {
    set_error("reserved field must be 0");
    return MRAID_ERR_INVALID_ARG;
  }
  return MRAID_OK;
}

mraid_status mraid_plan(const mraid_params* p, void* stream, mraid_plan_t* out) {
  if (!out) {
    set_error("out is NULL");
    return MRAID_ERR_INVALID_ARG;
  }
  *out = nullptr;
  mraid_status st = mraid_validate(p);
  if (st != MRAID_OK) return st;
  mraid_plan_s* pl = new (std::nothrow) mraid_plan_s();
  if (!pl) {
    set_error("host allocation failed");
    return MRAID_ERR_OOM;
  }
  pl->p = *p;
  pl->p.keep = nullptr;
  pl->tc_variant = tc_default_variant(p->n_beam);
  pl->stream = static_cast<cudaStream_t>(stream);
  pl->n_cells = (int64_t)p->n_sub * p->n_chan;
  pl->beam_stride = p->beam_stride ? p->beam_stride : (int64_t)p->n_sub * p->n_samp_sub * p->n_chan;
  pl->np = p->n_beam * (p->n_beam + 1) / 2;
  pl->psum = (p->n_beam + 1) * (p->n_beam + 2) / 2;
  cudaError_t e = cudaGetDevice(&pl->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&pl->sm_count, cudaDevAttrMultiProcessorCount, pl->device);
  if (e == cudaSuccess) {
    pl->flag_blocks = flag_grid_blocks(pl->device, pl->sm_count);
    if (pl->flag_blocks < 1) e = cudaErrorLaunchOutOfResources;
  }
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_partials, sizeof(double) * 6 * (size_t)pl->flag_blocks);
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_info, sizeof(mraid_flag_info));
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_degenerate, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_error, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_sweeps, 3 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_sweeps, 0, 3 * sizeof(unsigned long long), pl->stream);
  if (e == cudaSuccess) e = cudaMallocHost(&pl->h_info, sizeof(mraid_flag_info));
  if (e == cudaSuccess && p->keep) {
    e = cudaMalloc(&pl->d_keep, (size_t)p->n_chan);
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_keep, p->keep, (size_t)p->n_chan, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_degenerate, 0, sizeof(unsigned long long), pl->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_error, 0, sizeof(unsigned), pl->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_info, 0, sizeof(mraid_flag_info), pl->stream);
  if (e != cudaSuccess) {
    st = cuda_fail(e, "mraid_plan");
    mraid_destroy(pl);
    return st;
  }
  *out = pl;
  return MRAID_OK;
}

mraid_status mraid_ccm(mraid_plan_t pl, const void* d_data, int64_t* d_sums, float* d_corr) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (!d_data || (!d_sums && !d_corr)) {
    set_error("mraid_ccm: d_data and one of d_sums / d_corr are required");
    return MRAID_ERR_INVALID_ARG;
  }
  if (d_sums && pl->p.bit_depth != 8) {
    set_error("mraid_ccm: exact sums exist for 8-bit data only");
    return MRAID_ERR_INVALID_ARG;
  }
  return ccm_range(pl, d_data, 0, pl->p.n_sub, d_sums, d_corr);
}

mraid_status mraid_eig(mraid_plan_t pl, const float* d_corr, float* d_evals, float* d_q1,
                       float* d_stat) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (!d_corr || !d_stat) {
    set_error("mraid_eig: d_corr and d_stat are required");
    return MRAID_ERR_INVALID_ARG;
  }
  if (d_q1) {
    st = evals_for_q1(pl, (size_t)pl->n_cells, &d_evals);
    if (st != MRAID_OK) return st;
  }
  st = ensure_tri_workspace(pl, (size_t)pl->n_cells);
  if (st != MRAID_OK) return st;
  cudaError_t e = MRAID_PROF(pl, K_EIG, launch_eig(pl, d_corr, pl->n_cells, d_evals, d_q1, d_stat));
  return e == cudaSuccess ? MRAID_OK : cuda_fail(e, "eig launch");
}

mraid_status mraid_flag(mraid_plan_t pl, const float* d_stat, uint8_t* d_flags,
                        mraid_flag_info* info) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (!d_stat || !d_flags) {
    set_error("mraid_flag: d_stat and d_flags are required");
    return MRAID_ERR_INVALID_ARG;
  }
  cudaError_t e = MRAID_PROF(pl, K_FLAG, launch_flag(pl, d_stat, d_flags));
  if (e != cudaSuccess) return cuda_fail(e, "flag launch");
  return enqueue_info_copy(pl, info);
}

mraid_status mraid_refine(mraid_plan_t pl, const float* d_q1, const uint8_t* d_flags,
                          uint32_t* d_beam_bits, double* d_mu_sigma) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (!d_q1 || !d_flags || !d_beam_bits) {
    set_error("mraid_refine: d_q1, d_flags and d_beam_bits are required");
    return MRAID_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaSuccess;
  if (!pl->d_refine_part) {
    e = cudaMalloc(&pl->d_refine_part, sizeof(double) * 3 * (size_t)kRefBlocks * kMaxBeam);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_refine_thresh, sizeof(float) * kMaxBeam);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_refine_ms, sizeof(double) * 2 * kMaxBeam);
    if (e != cudaSuccess) return cuda_fail(e, "refine buffers");
  }
  e = launch_refine(pl, d_q1, d_flags, d_beam_bits, d_mu_sigma ? d_mu_sigma : pl->d_refine_ms);
  return e == cudaSuccess ? MRAID_OK : cuda_fail(e, "refine launch");
}

mraid_status mraid_run(mraid_plan_t pl, const void* d_data, float* d_evals, float* d_q1,
                       float* d_stat, uint8_t* d_flags, mraid_flag_info* info) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (!d_data || !d_stat || !d_flags) {
    set_error("mraid_run: d_data, d_stat and d_flags are required");
    return MRAID_ERR_INVALID_ARG;
  }
  st = ensure_workspace(pl, (size_t)pl->n_cells);
  if (st != MRAID_OK) return st;
  cudaError_t e = cudaMemsetAsync(pl->d_degenerate, 0, sizeof(unsigned long long), pl->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(pl->d_sweeps, 0, 3 * sizeof(unsigned long long), pl->stream);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  if (d_q1) {
    st = evals_for_q1(pl, (size_t)pl->n_cells, &d_evals);
    if (st != MRAID_OK) return st;
  }
  st = ccm_range(pl, d_data, 0, pl->p.n_sub, nullptr, pl->ws.corr);
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


mraid_status mraid_run_host(mraid_plan_t pl, const void* h_data, float* h_stat, uint8_t* h_flags,
                            mraid_flag_info* info) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (!h_data || !h_flags) {
    set_error("mraid_run_host: h_data and h_flags are required");
    return MRAID_ERR_INVALID_ARG;
  }
  const size_t esz = pl->p.bit_depth == 8 ? 1 : 4;
  const int64_t sub_bytes = (int64_t)pl->p.n_samp_sub * pl->p.n_chan * (int64_t)esz;  // per beam
  cudaError_t e = cudaSuccess;
  if (!pl->copy_stream) {
    // chunk: ~1 GiB of samples across all beams, whole sub-integrations,
    // and at least four chunks where the block allows (so copies overlap
    // compute). One 2D copy per chunk moves every beam's rows: measured on
    // GB300 the host-to-device rate (~210 GB/s) is the same from 12 MB
    // copies to one block-sized copy, but one copy call per beam and chunk
    // (19 x 67 calls for the FAST block at 256 MiB chunks) left the host
    // enqueueing at ~0.6 ms per chunk and the step 30-200 % above the copy
    // time.
    int64_t per_sub = sub_bytes * pl->p.n_beam;
    int chunk = (int)((1ll << 30) / (per_sub > 0 ? per_sub : 1));
    const int quarter = (pl->p.n_sub + 3) / 4;
    chunk = chunk > quarter ? quarter : chunk;
    chunk = chunk < 1 ? 1 : (chunk > pl->p.n_sub ? pl->p.n_sub : chunk);
    pl->chunk_subs = chunk;
    pl->chunk_bytes = (size_t)per_sub * chunk;
    e = cudaStreamCreateWithFlags(&pl->copy_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = cudaMalloc(&pl->d_chunk[i], pl->chunk_bytes);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ev_copied[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ev_consumed[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_stat_full, sizeof(float) * (size_t)pl->n_cells);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_flags_full, (size_t)pl->n_cells);
    if (e != cudaSuccess) return cuda_fail(e, "host-path buffers");
  }
  const int chunk = pl->chunk_subs;
  st = ensure_workspace(pl, (size_t)chunk * pl->p.n_chan);
  if (st != MRAID_OK) return st;
  e = cudaMemsetAsync(pl->d_degenerate, 0, sizeof(unsigned long long), pl->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(pl->d_sweeps, 0, 3 * sizeof(unsigned long long), pl->stream);
  // The chunk buffer holds [beam][chunk subs * n_samp_sub][chan]; the kernels
  // see it as a block of `chunk` sub-integrations with beam stride
  // chunk * n_samp_sub * n_chan.
  const int64_t saved_stride = pl->beam_stride;
  const int32_t saved_nsub = pl->p.n_sub;
  const int64_t saved_cells = pl->n_cells;
  int k = 0;
  for (int s0 = 0; s0 < saved_nsub && e == cudaSuccess; s0 += chunk, ++k) {
    const int ns = (saved_nsub - s0) < chunk ? (saved_nsub - s0) : chunk;
    const int slot = k & 1;
    e = cudaStreamWaitEvent(pl->copy_stream, pl->ev_consumed[slot], 0);
    if (e == cudaSuccess)  // rows: beams; one row holds ns sub-integrations of a beam
      e = cudaMemcpy2DAsync(pl->d_chunk[slot], (size_t)chunk * sub_bytes,
                            static_cast<const char*>(h_data) + (size_t)s0 * sub_bytes,
                            (size_t)saved_stride * esz, (size_t)ns * sub_bytes,
                            (size_t)pl->p.n_beam, cudaMemcpyHostToDevice, pl->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(pl->ev_copied[slot], pl->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(pl->stream, pl->ev_copied[slot], 0);
    if (e != cudaSuccess) break;
    pl->beam_stride = (int64_t)chunk * pl->p.n_samp_sub * pl->p.n_chan;
    pl->p.n_sub = ns;
    pl->n_cells = (int64_t)ns * pl->p.n_chan;
    st = ccm_range(pl, pl->d_chunk[slot], 0, ns, nullptr, pl->ws.corr);
    if (st == MRAID_OK) {
      e = MRAID_PROF(pl, K_EIG, launch_eig(pl, pl->ws.corr, pl->n_cells, nullptr, nullptr,
                                           pl->d_stat_full + (int64_t)s0 * pl->p.n_chan));
    }
    pl->beam_stride = saved_stride;
    pl->p.n_sub = saved_nsub;
    pl->n_cells = saved_cells;
    if (st != MRAID_OK) return st;
    if (e == cudaSuccess) e = cudaEventRecord(pl->ev_consumed[slot], pl->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "mraid_run_host");
  e = MRAID_PROF(pl, K_FLAG, launch_flag(pl, pl->d_stat_full, pl->d_flags_full));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&pl->d_info->n_degenerate, pl->d_degenerate, sizeof(int64_t),
                        cudaMemcpyDeviceToDevice, pl->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&pl->d_info->jacobi_sweeps, pl->d_sweeps, 2 * sizeof(int64_t),
                        cudaMemcpyDeviceToDevice, pl->stream);
  if (e == cudaSuccess)  // the FP64 q1 count (low half of the counter)
    e = cudaMemcpyAsync(&pl->d_info->q1_refined, pl->d_sweeps + 2, sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, pl->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_flags, pl->d_flags_full, (size_t)pl->n_cells, cudaMemcpyDeviceToHost, pl->stream);
  if (e == cudaSuccess && h_stat)
    e = cudaMemcpyAsync(h_stat, pl->d_stat_full, sizeof(float) * (size_t)pl->n_cells,
                        cudaMemcpyDeviceToHost, pl->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mraid_run_host");
  return enqueue_info_copy(pl, info);
}

mraid_status mraid_sync(mraid_plan_t pl) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  cudaError_t e = cudaStreamSynchronize(pl->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mraid_sync");
  pl->inject_withhold = -1;
  pl->inject_alloc = false;
  prof_fold(pl);
  unsigned dev_err = 0;
  e = cudaMemcpy(&dev_err, pl->d_error, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "mraid_sync");
  if (dev_err) {
    pl->h_info->timed_out = 1;
    cudaMemset(pl->d_error, 0, sizeof(unsigned));
  }
  if (pl->pending_info) {
    *pl->pending_info = *pl->h_info;
    pl->pending_info = nullptr;
  }
  if (pl->pending_ml) {
    for (int i = 0; i < pl->pending_ml_n; ++i) {
      pl->pending_ml[i] = pl->h_ml_info[i];
      if (pl->h_info->timed_out) pl->pending_ml[i].timed_out = 1;
    }
    pl->pending_ml = nullptr;
    pl->pending_ml_n = 0;
  }
  if (pl->h_info->timed_out) {
    pl->h_info->timed_out = 0;
    set_error("a bounded device wait expired");
    return MRAID_ERR_TIMEOUT;
  }
  return MRAID_OK;
}

mraid_status mraid_query(mraid_plan_t pl) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  cudaError_t e = cudaStreamQuery(pl->stream);
  if (e == cudaErrorNotReady) return MRAID_ERR_NOT_READY;
  if (e != cudaSuccess) return cuda_fail(e, "mraid_query");
  return mraid_sync(pl);
}

mraid_status mraid_set_variant(mraid_plan_t pl, int32_t variant) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (variant < -1 || variant >= kTcVariants) {
    set_error("mraid_set_variant: variant %d outside [-1, %d)", variant, kTcVariants);
    return MRAID_ERR_INVALID_ARG;
  }
  pl->force_dp4a = variant < 0;
  pl->tc_variant = variant < 0 ? 0 : variant;
  return MRAID_OK;
}

mraid_status mraid_set_wait_limit(mraid_plan_t pl, int64_t ns) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (ns < 1000000ll || ns > 60000000000ll) {
    set_error("mraid_set_wait_limit: %lld ns outside [1e6, 6e10]", (long long)ns);
    return MRAID_ERR_INVALID_ARG;
  }
  pl->wait_ns = (unsigned long long)ns;
  return MRAID_OK;
}

mraid_status mraid_inject_fault(mraid_plan_t pl, int32_t kind, int64_t arg) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  switch (kind) {
    case MRAID_FAULT_NONE:
      pl->inject_withhold = -1;
      pl->inject_alloc = false;
      return MRAID_OK;
    case MRAID_FAULT_WITHHOLD_STAGE:
      if (arg < 0) {
        set_error("mraid_inject_fault: stage %lld < 0", (long long)arg);
        return MRAID_ERR_INVALID_ARG;
      }
      pl->inject_withhold = arg;
      return MRAID_OK;
    case MRAID_FAULT_ALLOC:
      pl->inject_alloc = true;
      return MRAID_OK;
    default:
      set_error("mraid_inject_fault: unknown kind %d", kind);
      return MRAID_ERR_INVALID_ARG;
  }
}

mraid_status mraid_set_eig_variant(mraid_plan_t pl, int32_t variant) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (variant < 0 || variant >= kEigVariants) {
    set_error("mraid_set_eig_variant: variant %d outside [0, %d)", variant, kEigVariants);
    return MRAID_ERR_INVALID_ARG;
  }
  pl->eig_variant = variant;
  return MRAID_OK;
}


mraid_status mraid_autotune(mraid_plan_t pl, const void* d_data, int32_t reps, int32_t* gram_choice,
                            int32_t* eig_choice, char* report, int32_t report_len) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (!d_data || !gram_choice || !eig_choice || reps < 1 || reps > 1000 ||
      (report && report_len < 1)) {
    set_error("mraid_autotune: bad arguments");
    return MRAID_ERR_INVALID_ARG;
  }
  st = ensure_workspace(pl, (size_t)pl->n_cells);
  if (st != MRAID_OK) return st;
  float* stat = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMalloc(&stat, sizeof(float) * (size_t)pl->n_cells);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cuda_fail(e, "mraid_autotune");
  }
  int used = 0;
  if (report) report[0] = 0;
  auto note = [&](char tag, int v, float ms) {
    if (report && used < report_len - 1)
      used += snprintf(report + used, (size_t)(report_len - used), "%c%d:%.4f;", tag, v, ms);
  };
  // Gram stage
  const bool save_dp4a = pl->force_dp4a;
  const int save_v = pl->tc_variant;
  float best = 1e30f;
  int best_g = -2;
  for (int v = -1; v < kTcVariants && st == MRAID_OK; ++v) {
    pl->force_dp4a = v < 0;
    pl->tc_variant = v < 0 ? 0 : v;
    // float32 samples, and 24..127 beams, have one tensor-core kernel each,
    // timed as variant 0
    if (v >= 0 && (pl->p.bit_depth == 32 ? (v > 0 || !gram_tc_f32_supported(pl, d_data))
                   : gram_tcl_supported(pl, d_data) ? v > 0
                                                    : (!gram_tc_supported(pl, d_data) ||
                                                       tc_variant_effective(pl) != v)))
      continue;
    float ms = 0.f;
    st = time_runs(pl, reps, e0, e1,
                   [&] { return ccm_range(pl, d_data, 0, pl->p.n_sub, nullptr, pl->ws.corr); }, &ms);
    if (st != MRAID_OK) break;
    note('g', v, ms);
    if (ms < best) {
      best = ms;
      best_g = v;
    }
  }
  if (st == MRAID_OK && best_g >= -1) {
    pl->force_dp4a = best_g < 0;
    pl->tc_variant = best_g < 0 ? 0 : best_g;
  } else {
    pl->force_dp4a = save_dp4a;
    pl->tc_variant = save_v;
  }
  // Jacobi stage on the correlations just computed
  int best_e = pl->eig_variant;
  if (st == MRAID_OK) {
    best = 1e30f;
    for (int v = 0; v < kEigVariants && st == MRAID_OK; ++v) {
      pl->eig_variant = v;
      float ms = 0.f;
      st = time_runs(pl, reps, e0, e1,
                     [&]() -> mraid_status {
                       cudaError_t le = launch_eig(pl, pl->ws.corr, pl->n_cells, nullptr, nullptr, stat);
                       return le == cudaSuccess ? MRAID_OK : cuda_fail(le, "eig launch");
                     },
                     &ms);
      if (st != MRAID_OK) break;
      note('e', v, ms);
      if (ms < best) {
        best = ms;
        best_e = v;
      }
    }
    pl->eig_variant = best_e;
  }
  cudaStreamSynchronize(pl->stream);
  cudaFree(stat);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MRAID_OK) return st;
  if (best_g < -1) return MRAID_ERR_UNSUPPORTED;
  *gram_choice = best_g;
  *eig_choice = best_e;
  return MRAID_OK;
}

mraid_status mraid_profile_enable(mraid_plan_t pl, int32_t enable) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  pl->prof.on = enable != 0;
  return MRAID_OK;
}

mraid_status mraid_profile_read(mraid_plan_t pl, mraid_kernel_time* out, int32_t max, int32_t* n) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  if (!n || (max > 0 && !out) || max < 0) {
    set_error("mraid_profile_read: bad arguments");
    return MRAID_ERR_INVALID_ARG;
  }
  int32_t k = 0;
  for (int id = 0; id < K_COUNT; ++id) {
    if (pl->prof.launches[id] == 0) continue;
    if (k < max) {
      memset(&out[k], 0, sizeof(out[k]));
      strncpy(out[k].name, kernel_name(id), sizeof(out[k].name) - 1);
      out[k].launches = pl->prof.launches[id];
      out[k].total_ms = pl->prof.total_ms[id];
    }
    ++k;
  }
  *n = k;
  return MRAID_OK;
}

mraid_status mraid_profile_reset(mraid_plan_t pl) {
  mraid_status st = check_plan(pl);
  if (st != MRAID_OK) return st;
  for (int id = 0; id < K_COUNT; ++id) {
    pl->prof.launches[id] = 0;
    pl->prof.total_ms[id] = 0.0;
  }
  return MRAID_OK;
}

void mraid_destroy(mraid_plan_t pl) {
  if (!pl) return;
  int dev = -1;
  if (cudaGetDevice(&dev) == cudaSuccess && dev != pl->device) cudaSetDevice(pl->device);
  if (pl->stream || pl->d_info) cudaStreamSynchronize(pl->stream);
  if (pl->copy_stream) {
    cudaStreamSynchronize(pl->copy_stream);
    cudaStreamDestroy(pl->copy_stream);
  }
  for (int i = 0; i < 2; ++i) {
    cudaFree(pl->d_chunk[i]);
    if (pl->ev_copied[i]) cudaEventDestroy(pl->ev_copied[i]);
    if (pl->ev_consumed[i]) cudaEventDestroy(pl->ev_consumed[i]);
  }
  prof_fold(pl);
  for (cudaEvent_t ev : pl->prof.pool) cudaEventDestroy(ev);

  cudaFree(pl->d_stat_full);
  cudaFree(pl->d_flags_full);
  cudaFree(pl->ws.sums);
  cudaFree(pl->ws.corr);
  cudaFree(pl->ws.evals);
  cudaFree(pl->ws.tri);
  cudaFree(pl->ws.de);
  cudaFree(pl->ws.q1_list);
  cudaFree(pl->ws.q1_list_n);
  cudaFree(pl->pol_sums);
  cudaFree(pl->bp_y);
  cudaFree(pl->bp_z);
  cudaFree(pl->bp_iters);
  cudaFree(pl->ar_work);
  cudaFree(pl->ml_sums);
  cudaFree(pl->d_ml_info);
  if (pl->h_ml_info) cudaFreeHost(pl->h_ml_info);
  cudaFree(pl->d_refine_part);
  cudaFree(pl->d_refine_thresh);
  cudaFree(pl->d_refine_ms);
  cudaFree(pl->d_keep);
  cudaFree(pl->d_partials);
  cudaFree(pl->d_info);
  cudaFree(pl->d_degenerate);
  cudaFree(pl->d_error);
  cudaFree(pl->d_sweeps);
  if (pl->h_info) cudaFreeHost(pl->h_info);
  if (dev >= 0 && dev != pl->device) cudaSetDevice(dev);
  delete pl;
}

}  // extern "C"
