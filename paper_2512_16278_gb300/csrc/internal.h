// internal.h - plan state and kernel launchers shared by the library's
// translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "mraid.h"

namespace mraid {

constexpr int kMaxBeam = 128;
constexpr int kRefBlocks = 4096;  // eigenvector refinement: partial-sum blocks
constexpr int kMaxSampSub = 1 << 20;
constexpr int kMaxClipIter = 1000;
constexpr int kMaxLevels = 16;  // timescales in one mraid_multires call
// Samples per int32 accumulation segment: 32768 * 255^2 < 2^32 (unsigned).
constexpr int kGramSegment = 32768;

struct FlagDev {  // device image of mraid_flag_info
  mraid_flag_info info;
};

enum KernelId {
  K_GRAM = 0, K_CORR, K_EIG, K_FLAG, K_GRAM_TC, K_GRAM_F32, K_GRAM_TC_F32, K_AGG,
  K_BP_INPUT, K_ARPLS, K_CCM_BP, K_POL2_FOLD, K_GRAM_TCL, K_COUNT
};
const char* kernel_name(int id);

struct Profiler {
  bool on = false;
  struct Rec {
    int id;
    cudaEvent_t start, stop;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  int64_t launches[K_COUNT] = {};
  double total_ms[K_COUNT] = {};
};

struct Workspace {
  int64_t* sums = nullptr;  // [cell][P] (staged Gram for mraid_run)
  float* corr = nullptr;    // [cell][NP]
  size_t cells = 0;
  float* evals = nullptr;   // [cell][N] when q1 is wanted without eigenvalues
  size_t evals_cells = 0;
  float* tri = nullptr;     // [cell][tri_workspace_floats(N)]: larger-N eigensolver
  size_t tri_cells = 0;
  float* de = nullptr;      // [2N][cell]: T of the split tridiagonal route (eig variant 4)
  size_t de_cells = 0;
  uint32_t* q1_list = nullptr;   // [cell]: cells whose q1 takes the FP64 step
  size_t q1_list_cells = 0;
  unsigned* q1_list_n = nullptr;  // entries in q1_list
};

}  // namespace mraid

struct mraid_plan_s {
  mraid_params p{};
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  int64_t n_cells = 0;
  int64_t beam_stride = 0;
  int np = 0;    // N(N+1)/2
  int psum = 0;  // (N+1)(N+2)/2
  uint8_t* d_keep = nullptr;          // [n_chan]
  double* d_partials = nullptr;       // flag partial sums [2][blocks][3]
  int flag_blocks = 0;
  mraid_flag_info* d_info = nullptr;  // device flag info
  unsigned long long* d_degenerate = nullptr;
  unsigned* d_error = nullptr;        // device error word (bounded waits)
  unsigned long long* d_sweeps = nullptr;  // Jacobi sweeps: [0] per cell, [1] per warp;
                                           // [2] cells whose q1 took the FP64 step
  mraid_flag_info* h_info = nullptr;  // pinned staging
  mraid_flag_info* pending_info = nullptr;  // user pointer to fill at sync
  mraid::Workspace ws;
  // host-buffer path (mraid_run_host)
  uint8_t* d_chunk[2] = {nullptr, nullptr};
  size_t chunk_bytes = 0;
  int chunk_subs = 0;
  float* d_stat_full = nullptr;
  uint8_t* d_flags_full = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_consumed[2] = {nullptr, nullptr};
  mraid::Profiler prof;
  bool force_dp4a = false;  // use the CUDA-core Gram even where tcgen05 fits
  int tc_variant = 0;       // tensor-core Gram variant (tc_default_variant, or autotuned)
  unsigned long long wait_ns = 2000000000ull;  // bound of every device wait
  long long inject_withhold = -1;  // MRAID_FAULT_WITHHOLD_STAGE: stage to skip, or -1
  bool inject_alloc = false;       // MRAID_FAULT_ALLOC armed
  int eig_variant = 4;      // register kernels: 0 = Jacobi, looped rounds; 1 = Jacobi,
                            // unrolled sweep; 2 = Householder + implicit QR, one
                            // step copy per level; 3 = the same, one masked copy;
                            // 4 = the same split over two kernels (reduction and
                            // q1 / QR), the default
  double* d_refine_part = nullptr;   // eigenvector refinement: [block][N][3]
  float* d_refine_thresh = nullptr;  // [N]
  double* d_refine_ms = nullptr;     // [N][2] when the caller passes none
  // several timescales (mraid_multires): Gram sums of the longer levels,
  // per-level flag reports on the device and pinned staging
  int64_t* ml_sums = nullptr;
  size_t ml_sums_elems = 0;
  mraid_flag_info* d_ml_info = nullptr;  // [kMaxLevels]
  mraid_flag_info* h_ml_info = nullptr;  // [kMaxLevels], pinned
  mraid_flag_info* pending_ml = nullptr;
  int pending_ml_n = 0;
  // bandpass path (mraid_run_bandpass, mraid_arpls): time-aggregated
  // spectra and baselines [interval][beam][chan] (FP64), solves per
  // spectrum, and the ArPLS arrays when they do not fit in shared memory
  double* bp_y = nullptr;
  double* bp_z = nullptr;
  size_t bp_elems = 0;
  int32_t* bp_iters = nullptr;
  size_t bp_sys = 0;
  double* ar_work = nullptr;
  size_t ar_work_elems = 0;
  // two polarisations: Gram sums of the 2N stacked blocks where the tensor
  // cores do not take the block; pol_cells counts its int64 elements
  int64_t* pol_sums = nullptr;
  size_t pol_cells = 0;
};

namespace mraid {

void set_error(const char* fmt, ...);
// plan.cu helpers shared by the entry points of the other files
constexpr int kMaxSubPerLaunch = 32768;  // sub-integrations per Gram launch (grid.y bound)
mraid_status check_plan(mraid_plan_t pl);
mraid_status ensure_tri_workspace(mraid_plan_s* pl, size_t cells);
// the plan's sums and correlation buffers (and the eigensolver's) for `cells`
mraid_status ensure_workspace(mraid_plan_s* pl, size_t cells);
// buffers of a q1 request: the FP64 step's cell list, and eigenvalues when
// the caller wants q1 but not evals (the q1 passes read lambda_1, lambda_2)
mraid_status evals_for_q1(mraid_plan_s* pl, size_t cells, float** evals);
// Gram sums + correlation of sub-integrations [sub0, sub0 + n_sub) of d_data
// (either output may be null; cells relative to sub0)
mraid_status ccm_range(mraid_plan_s* pl, const void* d_data, int sub0, int n_sub,
                       int64_t* d_sums, float* d_corr);
// copy the device masking report to the caller's struct at the next sync
mraid_status enqueue_info_copy(mraid_plan_s* pl, mraid_flag_info* info);
// one pass over 8-bit samples: the Gram sums of every sub-integration into
// ws.sums (interleaved by 8 channels when the tensor cores form them), and
// the correlation into d_corr when it is not null
mraid_status gram_sums_pass(mraid_plan_s* pl, const void* d_data, float* d_corr,
                            bool* interleaved);
// Allocate every work buffer mraid_run can need (so later calls allocate
// nothing, e.g. inside a stream capture).
mraid_status plan_prepare(mraid_plan_s* pl);
// Copy the staged mraid_flag_info to the caller's struct (stream synced).
void plan_deliver_info(mraid_plan_s* pl);
// Bracket a kernel launch with profiling events (no-ops unless enabled).
void prof_begin(mraid_plan_s* pl, int id, cudaEvent_t* start, cudaStream_t stream);
void prof_end(mraid_plan_s* pl, int id, cudaEvent_t start, cudaStream_t stream);
// run expr (a launch returning cudaError_t) between profiling events
#define MRAID_PROF_ON(pl, id, stream, expr)   \
  ([&]() {                                    \
    cudaEvent_t s_;                           \
    mraid::prof_begin((pl), (id), &s_, (stream)); \
    cudaError_t e_ = (expr);                  \
    mraid::prof_end((pl), (id), s_, (stream));    \
    return e_;                                \
  }())
#define MRAID_PROF(pl, id, expr) MRAID_PROF_ON(pl, id, (pl)->stream, expr)
mraid_status cuda_fail(cudaError_t e, const char* what);

// gram.cu
// sums of sub-integrations [sub0, sub0 + n_sub) of d_data; d_sums is indexed
// by cell relative to sub0 (cell = (sub - sub0) * n_chan + chan).
cudaError_t launch_gram_u8(const mraid_plan_s* pl, const uint8_t* d_data,
                           int sub0, int n_sub, int64_t* d_sums);
// float32 samples: correlation on CUDA cores (d_corr relative to sub0)
cudaError_t launch_gram_f32(const mraid_plan_s* pl, const float* d_data, int sub0, int n_sub,
                            float* d_corr);
// tensor-core Gram fused with the correlation (gram_tc.cu); either output
// may be null. cudaErrorNotSupported when the shape or layout does not fit.
// n_pol 2: blocks b and N + b are two polarisations of beam b, summed in
// the converter; the sums and the correlation are of the total power (exact:
// TMEM accumulates pieces of at most 256 samples, the epilogue adds them)
bool gram_tc_supported(const mraid_plan_s* pl, const void* d_data, int n_pol = 1);
int tc_variant_samples(int v);
int tc_default_variant(int n_beam);
constexpr int kTcVariants = 10;
// the tensor-core variant a plan's launch runs (variants 8 and 9 fall back
// to the default where their A-in-TMEM kernel does not fit the shape)
int tc_variant_effective(const mraid_plan_s* pl);
constexpr int kEigVariants = 6;  // register eigensolvers (see eig_variant)
// d_sums8 (instead of d_sums): the sums in the interleaved layout
// [cell / 8][P][cell % 8], which the kernel writes in 64-byte runs
cudaError_t launch_gram_tc(const mraid_plan_s* pl, const uint8_t* d_data, int sub0, int n_sub,
                           int64_t* d_sums, float* d_corr, int64_t* d_sums8 = nullptr,
                           int n_pol = 1);
// float32 samples on the tensor cores (split-bf16 products, gram_tc.cu):
// correlation only, d_corr relative to sub0
// Tensor-core Gram for 24..127 beams, one channel per MMA (gram_tcl.cu):
// int64 sums [cell][P] of sub-integrations [sub0, sub0 + n_sub), cells
// relative to sub0.
bool gram_tcl_supported(const mraid_plan_s* pl, const void* d_data);
cudaError_t launch_gram_tcl(const mraid_plan_s* pl, const uint8_t* d_data, int sub0, int n_sub,
                            int64_t* d_sums);
bool gram_tc_f32_supported(const mraid_plan_s* pl, const void* d_data);
cudaError_t launch_gram_tc_f32(const mraid_plan_s* pl, const float* d_data, int sub0, int n_sub,
                               float* d_corr);
// interleaved: d_sums in the [cell / 8][P][cell % 8] layout
cudaError_t launch_corr_from_sums(const mraid_plan_s* pl, const int64_t* d_sums,
                                  int64_t n_cells, float* d_corr, bool interleaved = false);
// eig.cu
cudaError_t launch_eig(const mraid_plan_s* pl, const float* d_corr, int64_t n_cells,
                       float* d_evals, float* d_q1, float* d_stat);
// the same on another stream of the plan's device
cudaError_t launch_eig(const mraid_plan_s* pl, const float* d_corr, int64_t n_cells,
                       float* d_evals, float* d_q1, float* d_stat, cudaStream_t stream);
bool eig_supported(int n_beam);
// q1_refine.cu: FP64 inverse iteration for q1 on cells whose relative gap
// (lambda_1 - lambda_2) / lambda_1 lies in [1e-6, q1_refine_gap_hi(pl));
// d_count (or null) counts the refined cells
float q1_refine_gap_hi(const mraid_plan_s* pl);
cudaError_t launch_q1_refine(const mraid_plan_s* pl, const float* d_corr, int64_t n_cells,
                             const float* d_evals, float* d_q1, unsigned long long* d_count,
                             cudaStream_t stream);
// eig_large.cu: tridiagonal eigensolver for beam counts without a
// one-thread kernel; d_work holds tri_workspace_floats(N) floats per cell
size_t tri_workspace_floats(int n_beam);
cudaError_t launch_eig_large(const mraid_plan_s* pl, const float* d_corr, int64_t n_cells,
                             float* d_evals, float* d_q1, float* d_stat, float* d_work,
                             cudaStream_t stream);
// true if the plan's eigensolver needs the tridiagonal workspace
bool eig_needs_tri_workspace(const mraid_plan_s* pl);
// true if a q1 request needs d_evals (the q1 pass reads lambda_1 from it;
// the FP64 step of q1 reads lambda_1 and lambda_2 for every beam count)
bool eig_q1_needs_evals(int n_beam);
// refine.cu
cudaError_t launch_refine(mraid_plan_s* pl, const float* d_q1, const uint8_t* d_flags,
                          uint32_t* d_bits, double* d_mu_sigma);
// flag.cu: over the plan's cells into its device report, or over n_cells
// cells into d_info when those are given
cudaError_t launch_flag(mraid_plan_s* pl, const float* d_stat, uint8_t* d_flags,
                        int64_t n_cells = -1, mraid_flag_info* d_info = nullptr);
// bandpass.cu: ArPLS baselines of n_sys spectra of n points ([sys][n]
// FP64; d_zf an optional float copy, d_iters solves per spectrum or -1);
// d_work holds arpls_work_doubles(n, n_sys) doubles when that is nonzero
size_t arpls_work_doubles(int n, int n_sys);
cudaError_t launch_arpls(const mraid_plan_s* pl, const double* d_y, int n_sys, int n, double lam,
                         double ratio, int itermax, double* d_z, float* d_zf, int32_t* d_iters,
                         double* d_work);
// time-aggregated spectra [interval][beam][chan] from the Gram sums
cudaError_t launch_bandpass_input(const mraid_plan_s* pl, const int64_t* d_sums, bool interleaved,
                                  int interval, double* d_y);
// per cell C_ab = cov_ab / n^2 + (mu_a - z_a)(mu_b - z_b), packed, all cells
cudaError_t launch_ccm_bandpass(const mraid_plan_s* pl, const int64_t* d_sums, bool interleaved,
                                int interval, const double* d_z, float* d_ccm);
// pol2.cu: total-power sums [cell][P] from the stacked 2N-block sums
cudaError_t launch_pol2_fold(const mraid_plan_s* pl, const int64_t* d_stacked, int64_t n_cells,
                             int64_t* d_sums);
// multires.cu: d_dst[k] = sum_{j < m} d_src[k m + j] over the int64 Gram
// sums of n_out_sub sub-intervals (n_chan cells each)
cudaError_t launch_gram_aggregate(const mraid_plan_s* pl, const int64_t* d_src, int64_t* d_dst,
                                  int n_out_sub, int m);
int flag_grid_blocks(int device, int sm_count);

}  // namespace mraid
