/* mraid.h - C ABI of the GB300 eigenvalue RFI flagger.
 *
 * Method: mRAID (arXiv 2512.16278). For every cell (channel j,
 * sub-integration k) of multi-beam search-mode data:
 *   1. the N_beam x N_beam cross-correlation matrix of the beams' total
 *      power (Section 3.2, Eq. 1), read as the Pearson correlation of the
 *      N_s = T_k / t_s samples: r_ab = cov_ab / sqrt(cov_aa cov_bb);
 *   2. its eigendecomposition (Section 3.3, Eq. 2), eigenvalues ordered
 *      largest first, and the normalised dominant eigenvalue
 *      s = lambda_1^2 / sum_i lambda_i^2 (Section 3.3);
 *   3. iterative masking: a Gaussian (mean, sigma) fit to s over the cells
 *      not yet masked, mask s > mean + k sigma, repeat until the mask is
 *      stable (Section 3.3 masking paragraph; k = 3 in Section 4.5), never
 *      masking preserved channels (Section 4.3).
 *
 * Conventions for every call below:
 *   - Data layout: samples [beam][time][chan], channel fastest (as recorded),
 *     beam b starting beam_stride elements after beam b-1. 8-bit unsigned
 *     (bit_depth 8) or float32 (bit_depth 32) samples.
 *   - Cell index = sub * n_chan + chan. All per-cell outputs are dense in
 *     that order.
 *   - Pointers named d_* are device pointers allocated and owned by the
 *     caller; h_* are host pointers owned by the caller (pinned memory makes
 *     host transfers asynchronous and faster, pageable memory also works).
 *   - All device work is enqueued on the plan's stream and is asynchronous;
 *     outputs are valid after mraid_sync (or any later work on that stream).
 *   - Argument errors are reported synchronously and enqueue nothing. Device
 *     errors and expired bounded waits surface at the next call or at
 *     mraid_sync. There is no CPU fallback: without a usable CUDA device
 *     mraid_plan fails with MRAID_ERR_CUDA.
 */
#ifndef MRAID_H
#define MRAID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* 1: the plain, batched and served paths; 2: adds mraid_multires, the
 * bandpass entry points (mraid_bandpass_params) and the two-polarisation
 * entry points. Existing structures and calls are unchanged. */
#define MRAID_ABI_VERSION 2

typedef enum {
  MRAID_OK = 0,
  MRAID_ERR_INVALID_ARG = 1, /* NULL pointer, size out of range, bad layout */
  MRAID_ERR_UNSUPPORTED = 2, /* valid but not built: bit depth, N_beam > 128 */
  MRAID_ERR_OOM = 3,         /* device or pinned host allocation failed */
  MRAID_ERR_CUDA = 4,        /* a CUDA call failed (message: mraid_last_error) */
  MRAID_ERR_TIMEOUT = 5,     /* a bounded device wait expired */
  MRAID_ERR_NOT_READY = 6    /* mraid_query: work still in flight */
} mraid_status;

/* Problem statement (Section 3.2 and Section 4.5). */
typedef struct {
  int32_t n_beam;        /* N_beam, 2..128 (Eq. 1) */
  int32_t n_chan;        /* frequency channels, >= 1 */
  int32_t n_samp_sub;    /* N_s = T_k / t_s, samples per sub-integration, 2..2^20 */
  int32_t n_sub;         /* sub-integrations in one block, >= 1 */
  int32_t bit_depth;     /* 8: uint8 samples; 32: float32 samples */
  int64_t beam_stride;   /* elements between beams; 0 = dense (n_sub*n_samp_sub*n_chan) */
  double eig_k;          /* eigenvalue threshold multiple k (Section 4.5), > 0; 3 */
  double vec_t;          /* eigenvector threshold multiple (Section 4.5), >= 0; 1 */
  int32_t max_clip_iter; /* bound on masking iterations, 1..1000; 64 */
  int32_t reserved;      /* must be 0 */
  const uint8_t* keep;   /* host, n_chan bytes, nonzero = preserved channel
                            (Section 4.3); NULL = none. Copied by mraid_plan. */
} mraid_params;

/* Result of the masking step (Section 3.3). */
typedef struct {
  double mu;             /* mean of s over the final unmasked, unpreserved cells */
  double sigma;          /* population standard deviation of that set */
  double thresh;         /* mu + k * sigma: the converged dynamic threshold */
  int32_t iterations;    /* Gaussian fits made */
  int32_t converged;     /* 1 if the mask stopped changing within max_clip_iter */
  int64_t n_flagged;     /* cells masked */
  int64_t n_used;        /* cells in the final fit */
  int64_t n_near;        /* unpreserved cells with |s - thresh| <= 2e-4 * s */
  int64_t n_degenerate;  /* (beam, cell) pairs with zero variance (mraid_run) */
  int64_t jacobi_sweeps; /* eigensolver iterations summed over cells (mraid_run; 0 if not
                            counted): Jacobi sweeps, or implicit QR steps for the
                            tridiagonal variant */
  int64_t jacobi_warp_sweeps; /* the same, as executed: each 32-cell warp counts its slowest
                                 cell (mraid_run) */
  int32_t timed_out;     /* 1 if a bounded device wait expired */
  int32_t q1_refined;    /* cells whose q1 took the FP64 final step: relative gap
                            (lambda_1 - lambda_2) / lambda_1 in [1e-6, 2e-3), or
                            [1e-6, 1e-2) behind the one-thread Jacobi variants
                            (mraid_set_eig_variant 0 and 1, N = 2, 3, 4, 13, 19) */
} mraid_flag_info;

typedef struct mraid_plan_s* mraid_plan_t;

/* Fill p with the paper's defaults (eig_k 3, vec_t 1, max_clip_iter 64,
 * bit_depth 8, dense layout) for the given sizes. Host only. */
void mraid_default_params(mraid_params* p, int32_t n_beam, int32_t n_chan,
                          int32_t n_samp_sub, int32_t n_sub);

/* Check p without touching the GPU. MRAID_OK, MRAID_ERR_INVALID_ARG or
 * MRAID_ERR_UNSUPPORTED. */
mraid_status mraid_validate(const mraid_params* p);

/* Validate p, bind the plan to the current CUDA device and to stream
 * (a cudaStream_t; NULL = the legacy default stream), allocate the plan's
 * small device state and copy keep[]. Large work buffers are allocated on
 * first use and kept until mraid_destroy. *out receives the plan. */
mraid_status mraid_plan(const mraid_params* p, void* stream, mraid_plan_t* out);

/* Section 3.2, Eq. 1: per cell, the exact augmented Gram sums and/or the
 * Pearson correlation.
 *   d_data: samples, layout above (bit_depth 8 only for d_sums).
 *   d_sums: int64 [cell][P], P = (N+1)(N+2)/2, the upper triangle (a <= b,
 *           row-major) of G = X~ X~^T with X~ = [X; 1]: G[a][b] = sum x_a x_b,
 *           G[a][N] = sum x_a, G[N][N] = N_s. Exact. May be NULL.
 *   d_corr: float32 [cell][N(N+1)/2], upper triangle (a <= b, row-major) of r,
 *           r_aa = 1; a zero-variance beam has r_ab = 0 (a != b). May be NULL.
 * At least one of d_sums, d_corr must be non-NULL. */
mraid_status mraid_ccm(mraid_plan_t plan, const void* d_data, int64_t* d_sums,
                       float* d_corr);

/* mraid_ccm without any allocation (the paper has no counterpart; this is
 * an interface for callers). Some callers cannot call cudaMalloc: pipelines
 * that reserved the whole device for their own memory pool before loading
 * this library, and real-time loops that must not make a call that can
 * synchronise the device and stall their other streams. This entry point
 * needs no plan and allocates nothing: its int64 Gram sums and zero-variance
 * counter live in one fixed 8 MiB __device__ array inside the library, which
 * every GPU that loads the library holds until the process exits.
 *   p:        as for mraid_plan (bit_depth 8; keep is ignored).
 *   d_data:   samples of the whole block, layout above.
 *   sub0, n_sub: the sub-integrations [sub0, sub0 + n_sub) to process.
 *   d_corr:   float32 [n_sub * n_chan][N(N+1)/2], cells relative to sub0,
 *             the same values mraid_ccm writes for those cells.
 *   stream:   cudaStream_t (NULL = legacy default stream).
 * Limit: n_sub * n_chan * 8 * (N+1)(N+2)/2 + 256 bytes must fit the 8 MiB
 * array (4993 cells for 19 beams); larger requests return
 * MRAID_ERR_INVALID_ARG with a message, so split the block over calls.
 * The first call on a device looks up the array's device address with
 * that device current (cudaGetSymbolAddress); make that first call before
 * any stream capture. The address is kept for the life of the process, so
 * calls after the device's context is destroyed and recreated (e.g. after
 * cudaDeviceReset) are not supported. Every call reuses the same array: calls that can
 * overlap on the GPU (different streams, or different host threads on one
 * device) race and corrupt each other's sums, so serialise them, e.g. on
 * one stream. */
mraid_status mraid_ccm_noalloc(const mraid_params* p, const void* d_data, int32_t sub0,
                               int32_t n_sub, float* d_corr, void* stream);

/* Section 3.3, Eq. 2: eigenvalues of every cell's correlation (parallel
 * cyclic Jacobi in FP32), its dominant eigenvector and statistic.
 *   d_corr:  float32 [cell][N(N+1)/2] as written by mraid_ccm.
 *   d_evals: float32 [cell][N], largest first. May be NULL.
 *   d_q1:    float32 [cell][N], unit eigenvector of evals[0] with its
 *            largest-magnitude element positive. May be NULL.
 *   d_stat:  float32 [cell], s = lambda_1^2 / sum lambda_i^2. Required. */
mraid_status mraid_eig(mraid_plan_t plan, const float* d_corr, float* d_evals,
                       float* d_q1, float* d_stat);

/* Section 3.3 masking: iterative Gaussian-fit threshold on d_stat.
 *   d_stat:  float32 [cell].
 *   d_flags: uint8 [cell], 1 = RFI. Required.
 *   info:    host struct, filled by the next mraid_sync; may be NULL. */
mraid_status mraid_flag(mraid_plan_t plan, const float* d_stat, uint8_t* d_flags,
                        mraid_flag_info* info);

/* Eigenvector refinement (Section 3.3 last paragraph; threshold multiple
 * vec_t, Section 4.5): which beams each RFI cell affects. For every beam b,
 * a Gaussian fit (mean, population sigma) to |q1_b| over the cells that
 * d_flags leaves unflagged (and not preserved); a flagged cell gets bit b
 * when |q1_b| > mu_b + vec_t sigma_b.
 *   d_q1:        float32 [cell][N] from mraid_eig / mraid_run.
 *   d_flags:     uint8 [cell] from mraid_flag / mraid_run.
 *   d_beam_bits: uint32 [cell][ceil(N/32)], bit b % 32 of word b / 32.
 *   d_mu_sigma:  float64 [N][2] (mu_b, sigma_b), device; may be NULL. */
mraid_status mraid_refine(mraid_plan_t plan, const float* d_q1, const uint8_t* d_flags,
                          uint32_t* d_beam_bits, double* d_mu_sigma);

/* The whole path (Eq. 1, Eq. 2, masking) on one block already in device
 * memory. d_evals and d_q1 may be NULL; d_stat and d_flags are required;
 * info as in mraid_flag. */
mraid_status mraid_run(mraid_plan_t plan, const void* d_data, float* d_evals,
                       float* d_q1, float* d_stat, uint8_t* d_flags,
                       mraid_flag_info* info);

/* The whole path on one block in HOST memory (layout and beam stride as in
 * the plan): copies h_data to the device in pieces overlapped with the
 * computation, then copies the statistic and the flags back. h_stat (float32 [cell]) may be NULL; h_flags (uint8 [cell]) is
 * required. Outputs are valid after mraid_sync. */
mraid_status mraid_run_host(mraid_plan_t plan, const void* h_data, float* h_stat,
                            uint8_t* h_flags, mraid_flag_info* info);

/* Several timescales in one pass (Section 4.2, Table 1 and Fig. 7 run the
 * method at sub-interval lengths from 0.05 s to 10 s). Level i uses
 * sub-intervals of factors[i] consecutive sub-integrations of the plan
 * (factors[i] * n_samp_sub samples each): the whole path (Eq. 1, Eq. 2,
 * masking with its own Gaussian fit over that level's cells) as mraid_run
 * would give for a plan with n_samp_sub * factors[i] samples per
 * sub-integration over the first (n_sub / factors[i]) * factors[i]
 * sub-integrations (integer division: trailing sub-integrations that do
 * not fill a sub-interval are left out of that level). The samples are read
 * once: the Gram sums of the plan's sub-integrations are formed, and each
 * longer sub-interval's sums are the exact int64 sum of shorter ones.
 *   d_data:    8-bit samples (bit_depth 8), layout as for mraid_run.
 *   n_levels:  1..16.
 *   factors:   host, n_levels distinct values in 1..n_sub, any order.
 *   d_stats:   host array of n_levels device pointers, float32
 *              [(n_sub / factors[i]) * n_chan], cell = sub-interval * n_chan
 *              + chan. Required.
 *   d_flags:   host array of n_levels device pointers, uint8, same cells.
 *              Required.
 *   infos:     host, n_levels entries filled at mraid_sync (may be NULL);
 *              n_degenerate and jacobi_sweeps count that level's cells.
 * Work buffers (the Gram sums of every level) are allocated on first use
 * and kept by the plan. */
mraid_status mraid_multires(mraid_plan_t plan, const void* d_data, int32_t n_levels,
                            const int32_t* factors, float* const* d_stats,
                            uint8_t* const* d_flags, mraid_flag_info* infos);

/* Two recorded polarisations (Section 2): d_data holds 2N blocks of 8-bit
 * samples, polarisation-major: block p*N + a is polarisation p of beam a,
 * [time][chan], blocks the plan's beam_stride apart. Eq. 1 is taken of the
 * total power x_a = p0_a + p1_a (0..510). d_sums, d_corr and the rest as
 * in mraid_ccm and mraid_run; the sums are those of x, exact. The plan
 * describes the N beams (n_beam <= 64, bit_depth 8). Where the tensor-core
 * Gram takes the shape (N <= 23, channels a multiple of 16, samples per
 * sub-integration a multiple of 64 up to 1024, 16-byte aligned) it adds the
 * polarisations as it reads them and needs no work buffer; otherwise the
 * Gram of the 2N stacked blocks is formed and folded, in a work buffer of
 * (2N+1)(2N+2)/2 int64 per cell allocated on first use. */
mraid_status mraid_ccm_pol2(mraid_plan_t plan, const void* d_data, int64_t* d_sums,
                            float* d_corr);
mraid_status mraid_run_pol2(mraid_plan_t plan, const void* d_data, float* d_evals,
                            float* d_q1, float* d_stat, uint8_t* d_flags,
                            mraid_flag_info* info);

/* Bandpass normalisation (Section 3.1) with ArPLS, the asymmetrically
 * reweighted penalized least squares of Baek, Park, Ahn and Ahn (2015) that
 * the paper uses; Section 4.5 names its three parameters without values. */
typedef struct {
  double lam;        /* weight of the second-difference penalty (smoothness), > 0 */
  double ratio;      /* stop when |w_new - w| / |w| < ratio (Euclidean norms), > 0 */
  int32_t itermax;   /* bound on weighted solves, 1..1000 */
  int32_t interval;  /* sub-integrations per bandpass fit interval, >= 1 (the last
                        interval of a block may be shorter; one at least as long
                        as the block makes the block one interval) */
} mraid_bandpass_params;

/* lam 1e5, ratio 1e-3, itermax 50, interval 20 (about 1 s of 1024-sample
 * sub-integrations at 49.152 us, Section 3.1's example). Host only. */
void mraid_default_bandpass_params(mraid_bandpass_params* bp);

/* ArPLS baselines of n_sys spectra on the plan's device and stream: start
 * with unit weights w; repeat: solve (W + lam D^T D) z = W y (D: second
 * differences over the n points; FP64, banded LDL^T); d = y - z; m, s =
 * mean and population standard deviation of the negative d_i; new weights
 * 1 / (1 + exp(2 (d_i - (2 s - m)) / s)); stop when the weights moved by
 * less than ratio, when no d_i is negative or s is 0, or after itermax
 * solves (bp->interval is not used here).
 *   d_y:     float64 [n_sys][n], device, 3 <= n <= 2^20.
 *   d_z:     float64 [n_sys][n], device: the last solve.
 *   d_iters: int32 [n_sys] or NULL: solves made, -1 if a pivot of the
 *            system was not positive (z is then not valid). */
mraid_status mraid_arpls(mraid_plan_t plan, const double* d_y, int32_t n_sys, int32_t n,
                         const mraid_bandpass_params* bp, double* d_z, int32_t* d_iters);

/* The whole path under the bandpass-centred reading of Eq. 1: per fit
 * interval and beam, the time-aggregated spectrum (the mean of each channel
 * over the interval's samples, exact from the Gram sums) and its ArPLS
 * baseline z; per cell C_ab = (1/N_s) sum_t (x_a - z_a)(x_b - z_b), the
 * beams' power with the bandpass subtracted "uniformly across all time
 * samples" (Section 3.1) and no further centring or normalisation; then
 * Eq. 2 and the masking as in mraid_run. 8-bit samples, 3 to 2^20 channels.
 *   d_bandpass: float32 [ceil(n_sub / interval)][N][n_chan] or NULL: z.
 *   d_evals, d_q1: as in mraid_run (may be NULL); d_stat, d_flags required.
 *   info: as in mraid_run (n_degenerate is 0: nothing is normalised). */
mraid_status mraid_run_bandpass(mraid_plan_t plan, const void* d_data,
                                const mraid_bandpass_params* bp, float* d_bandpass,
                                float* d_evals, float* d_q1, float* d_stat, uint8_t* d_flags,
                                mraid_flag_info* info);

/* Autotuner (the paper has no counterpart; it picks among this library's
 * kernel variants). Times, `reps` runs each on d_data, every Gram variant
 * that fits the plan's shape (ten tensor-core variants: samples per stage,
 * f16 stages and converter unrolling with both operands in shared memory;
 * 64 or 32 samples per stage with A in tensor memory, up to 19 beams; and the
 * CUDA-core Gram) and the register
 * eigensolvers (Jacobi rounds in a loop; the Jacobi sweep unrolled;
 * Householder tridiagonalisation + implicit QR in two code layouts), and
 * keeps the fastest of each for this plan. *gram_choice: -1 = CUDA-core,
 * 0..9 tensor-core variants; *eig_choice: 0..5. report (may be NULL) receives "g<id>:ms;e<id>:ms;...".
 * Synchronous. */
mraid_status mraid_autotune(mraid_plan_t plan, const void* d_data, int32_t reps,
                            int32_t* gram_choice, int32_t* eig_choice, char* report,
                            int32_t report_len);

/* Select variants by id (e.g. from a tuning cache). Gram: -1 = CUDA-core,
 * 0..9 tensor-core variants for up to 23 beams (ignored where the shape does
 * not fit); for 24..127 beams any id >= 0 selects the one-channel-per-MMA
 * tensor-core Gram (exact in pieces of <= 1024 samples).
 * Eigensolver (beam counts with a one-thread-per-matrix kernel: 2, 3, 4, 13,
 * 19; other counts always use the warp-per-matrix Jacobi): 0 = Jacobi,
 * looped rounds; 1 = Jacobi, unrolled sweep; 2 = Householder reduction to
 * tridiagonal form, implicit QR with the Wilkinson shift (one unrolled step
 * per deflation level), q1 by inverse iteration on the tridiagonal matrix;
 * 3 = the same with one masked QR step for all levels (smaller code);
 * 4 = the same arithmetic split over two kernels: the reduction, lambda_1
 * (Newton's method on det(T - x I)) and q1 in one, QR on T for all
 * eigenvalues in a second with few registers (the default); 5 = variant 4
 * with the root-free (Pal-Walker-Kahan) QR step on the squared
 * off-diagonals in the second kernel. All give the same outputs to the
 * stated tolerances. */
mraid_status mraid_set_variant(mraid_plan_t plan, int32_t variant);
mraid_status mraid_set_eig_variant(mraid_plan_t plan, int32_t variant);

/* Failure detection (no counterpart in the paper). Every wait inside the
 * tensor-core kernels is bounded: when one runs out the kernel records an
 * error, waits (with the same bound) for its own bulk copies and MMAs in
 * flight, frees its tensor memory and returns, so the context stays
 * usable; mraid_sync then returns MRAID_ERR_TIMEOUT (and the info's
 * timed_out is 1). Outputs of that call are not valid; later calls are.
 *   ns: the bound of each wait in nanoseconds, 1e6 .. 6e10 (default 2e9). */
mraid_status mraid_set_wait_limit(mraid_plan_t plan, int64_t ns);

/* Fault injection for tests of the failure paths, on the host's side of
 * the launch (no counterpart in the paper; nothing faults the device):
 *   MRAID_FAULT_NONE:           clear.
 *   MRAID_FAULT_WITHHOLD_STAGE: in the plan's next tensor-core Gram launch
 *     (8-bit samples, any beam count), the first CTA's bulk-copy producer skips its stage
 *     number arg (counted from 0 over that CTA's stages): the copy is never
 *     issued, so the consumer's bounded wait for it expires and mraid_sync
 *     returns MRAID_ERR_TIMEOUT.
 *   MRAID_FAULT_ALLOC:          the plan's next work-buffer allocation
 *     fails as out of memory: the call returns MRAID_ERR_OOM (arg unused).
 * An injection is cleared by the next mraid_sync (MRAID_FAULT_ALLOC also by
 * the failure it causes). */
#define MRAID_FAULT_NONE 0
#define MRAID_FAULT_WITHHOLD_STAGE 1
#define MRAID_FAULT_ALLOC 2
mraid_status mraid_inject_fault(mraid_plan_t plan, int32_t kind, int64_t arg);

/* ------------------------------------------------------------------------
 * Batched form: blocks of uneven receiver shapes (different N_beam, N_s,
 * channel counts; e.g. 13-, 19-, 36- and 72-beam systems, Section 5) in one
 * pass. Cells are independent (Section 3.3); the masking statistics stay per
 * unit (each unit is its own observation). The pass is captured into a CUDA
 * graph on the batch's stream, with the units either as concurrent branches
 * or chained one after another: the first mraid_batch_run times both
 * packings on the caller's buffers (so that call waits for the GPU) and
 * keeps the faster. A later call with different buffers rebinds them
 * through a graph update instead of a new instantiation.
 */
typedef struct mraid_batch_s* mraid_batch_t;

typedef struct {
  const void* d_data;  /* the unit's samples, layout as for mraid_run */
  float* d_evals;      /* float32 [cell][N] or NULL */
  float* d_q1;         /* float32 [cell][N] or NULL */
  float* d_stat;       /* float32 [cell], required */
  uint8_t* d_flags;    /* uint8 [cell], required */
} mraid_unit_io;

/* One plan per unit (params[i], validated as for mraid_plan), all work
 * buffers allocated here. stream: cudaStream_t of the batch. */
mraid_status mraid_batch_plan(const mraid_params* params, int32_t n_units, void* stream,
                              mraid_batch_t* out);

/* Run every unit: io[n_units] buffers, infos[n_units] host structs filled at
 * mraid_batch_sync (may be NULL). */
mraid_status mraid_batch_run(mraid_batch_t batch, const mraid_unit_io* io,
                             mraid_flag_info* infos);

/* Wait for the batch's stream and deliver the per-unit infos. */
mraid_status mraid_batch_sync(mraid_batch_t batch);

/* Number of graph instantiations and graph updates made so far (a replay
 * with new buffers is an update, not an instantiation). */
mraid_status mraid_batch_graph_stats(mraid_batch_t batch, int32_t* instantiations,
                                     int32_t* updates);

/* The packing the first run chose (*packing: 0 = concurrent branches,
 * 1 = chained; -1 before the first run) and the measured pass time of each
 * in milliseconds (-1 if not measured). The times may be NULL. */
mraid_status mraid_batch_packing(mraid_batch_t batch, int32_t* packing, float* ms_concurrent,
                                 float* ms_chained);

void mraid_batch_destroy(mraid_batch_t batch);

/* ------------------------------------------------------------------------
 * Served form: continuous batching of blocks from several concurrent
 * observations (streams) as they arrive. Each observation has its own
 * receiver shape; its blocks need not hold whole sub-integrations: the
 * samples left over at the end of a block are kept on the device and
 * prepended to the next block of that stream, so every cell still spans
 * N_s consecutive samples (Section 3.2). A server thread admits submitted
 * blocks while device slots and the HBM budget allow, copies them in on
 * their stream, runs the path (masking statistics per block, Section 3.3)
 * and copies the flags out; blocks of different streams overlap on the GPU.
 * Per-stream state (carry, last flag mask, counters) stays on the device.
 */
typedef struct mraid_server_s* mraid_server_t;

typedef struct {
  mraid_params params;      /* shape of the stream; n_sub is ignored */
  int32_t block_samples;    /* samples per beam and channel in every block */
  int32_t reserved;
} mraid_stream_desc;

typedef struct {
  int32_t stream;           /* observation index */
  int32_t n_sub;            /* whole sub-integrations processed for this block */
  int64_t seq;              /* the caller's sequence number from mraid_serve_submit */
  int64_t n_cells, n_flagged;
  double mu, sigma, thresh; /* masking result of this block */
  double latency_ms;        /* submit -> flags in host memory, host clock */
  double device_ms;         /* copy-in start -> flags copied out, device events */
  int32_t status;           /* mraid_status of this block */
  int32_t reserved;
} mraid_block_result;

/* Open a server for n_streams observations. hbm_budget: device bytes the
 * server may hold (0 = 80 % of the free memory at open); max_inflight: blocks
 * admitted to the GPU at once across streams (>= 1). Buffers of a stream are
 * allocated when its first block is admitted and only if they fit the
 * budget; blocks wait in the queue until they do. */
mraid_status mraid_serve_open(const mraid_stream_desc* streams, int32_t n_streams,
                              int64_t hbm_budget, int32_t max_inflight, mraid_server_t* out);

/* Queue one block of stream `stream`: h_block is uint8 [beam][block_samples]
 * [chan] in host memory (pinned for asynchronous copies) and must stay
 * untouched until its result is polled; h_flags receives uint8 flags of the
 * block's whole sub-integrations ([n_sub][chan], at most
 * ceil((block_samples + N_s) / N_s) * n_chan bytes). Non-blocking. */
mraid_status mraid_serve_submit(mraid_server_t srv, int32_t stream, const void* h_block,
                                uint8_t* h_flags, int64_t seq);

/* Copy up to max finished blocks into out (FIFO order of completion);
 * *n receives the count. Non-blocking. */
mraid_status mraid_serve_poll(mraid_server_t srv, mraid_block_result* out, int32_t max,
                              int32_t* n);

/* Wait until every submitted block has finished (bounded by timeout_ms;
 * MRAID_ERR_TIMEOUT when it expires). */
mraid_status mraid_serve_drain(mraid_server_t srv, int32_t timeout_ms);

/* Stop the server thread and free everything (finishes admitted blocks). */
void mraid_serve_close(mraid_server_t srv);

/* Wait for the plan's stream, then deliver pending mraid_flag_info. Returns
 * the first device error seen (MRAID_ERR_TIMEOUT, MRAID_ERR_CUDA) or OK. */
mraid_status mraid_sync(mraid_plan_t plan);

/* Non-blocking: MRAID_OK if the plan's stream is idle (info delivered),
 * MRAID_ERR_NOT_READY if work is in flight, or an error. */
mraid_status mraid_query(mraid_plan_t plan);

/* Free everything the plan owns (waits for its stream first). NULL is a
 * no-op. */
void mraid_destroy(mraid_plan_t plan);

/* Per-kernel timing. While enabled, the plan brackets every kernel it
 * launches with a pair of CUDA events on its stream; mraid_sync folds the
 * elapsed times into per-kernel totals. mraid_profile_read copies up to max
 * records (name, launches, total milliseconds) into out and sets *n to the
 * number of kernels seen; mraid_profile_reset clears the totals. */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
} mraid_kernel_time;

mraid_status mraid_profile_enable(mraid_plan_t plan, int32_t enable);
mraid_status mraid_profile_read(mraid_plan_t plan, mraid_kernel_time* out, int32_t max,
                                int32_t* n);
mraid_status mraid_profile_reset(mraid_plan_t plan);

/* Static strings. mraid_last_error describes the last failure in this
 * thread (empty if none). */
const char* mraid_status_string(mraid_status s);
const char* mraid_last_error(void);
int32_t mraid_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MRAID_H */
