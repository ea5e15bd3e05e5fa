/* mraid_oracle.h - plain, slow CPU oracle of the eigenvalue RFI flagger.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the
 * benchmark's CPU baseline leg and reference arm (which time it) may call
 * this code; the library's product path never does. It shares no source
 * with the CUDA path.
 *
 * Method (mRAID, arXiv 2512.16278):
 *   Section 3.2, Eq. 1: per (channel j, sub-integration k) the N_beam x N_beam
 *     cross-correlation matrix of the beams' total power; read here as the
 *     Pearson correlation (mean-subtracted, unit diagonal) of the N_s samples.
 *   Section 3.3, Eq. 2: eigendecomposition C = Q Lambda Q^-1; eigenvalues
 *     ordered largest first, normalised as lambda_i^2 / sum_j lambda_j^2.
 *   Section 3.3 (masking paragraph) and Section 4.5: iterative Gaussian fit
 *     to the dominant normalised eigenvalue over all cells; cells above
 *     mean + k * sigma (k = 3) are masked; repeat until the mask is stable.
 *   Section 4.3: user-preserved frequency ranges are never masked.
 * Everything is FP64 except the Gram sums, which are exact int64.
 */
#ifndef MRAID_ORACLE_H
#define MRAID_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double mu;          /* mean of the statistic over the last unmasked set */
  double sigma;       /* population standard deviation of that set */
  double thresh;      /* mu + k * sigma */
  int32_t iterations; /* statistic evaluations made */
  int32_t converged;  /* 1 if the mask stopped changing */
  int64_t n_flagged;
  int64_t n_used;     /* cells in the last unmasked, non-preserved set */
} orc_flag_info;

/* Exact augmented Gram of one cell (Eq. 1 before normalisation). G is the
 * full (N+1)x(N+1) row-major matrix of X~ X~^T with X~ = [X; 1]:
 * G[a][b] = sum_t x_a(t) x_b(t), G[a][N] = sum_t x_a(t), G[N][N] = N_s.
 * data is uint8 [beam][time][chan], beam b at data + b*beam_stride, time
 * stride n_chan. Returns 0, or -1 on bad arguments. */
int orc_cell_gram_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                     int32_t n_chan, int32_t n_samp_sub, int32_t sub,
                     int32_t chan, int64_t* G);

/* Two polarisations (Section 2: the FAST data record two; the total power
 * B of Eq. 1 is their sum): polarisation p of beam a is block p*N + a of
 * data (blocks beam_stride apart), x_a(t) = p0_a(t) + p1_a(t) in 0..510.
 * Exact augmented Gram of x, as orc_cell_gram_u8. */
int orc_cell_gram_pol2_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                          int32_t n_chan, int32_t n_samp_sub, int32_t sub, int32_t chan,
                          int64_t* G);

/* Same for float32 samples: G is not exact here, so the oracle forms the
 * mean-subtracted covariance directly in FP64 (cov[a][b], N x N). */
int orc_cell_cov_f32(const float* data, int32_t n_beam, int64_t beam_stride,
                     int32_t n_chan, int32_t n_samp_sub, int32_t sub,
                     int32_t chan, double* cov);

/* Pearson correlation r (N x N) from the augmented Gram:
 * r_ab = (n S_ab - S_a S_b) / sqrt((n S_aa - S_a^2)(n S_bb - S_b^2)),
 * numerators exact in int64. A beam of zero variance gets r_aa = 1 and
 * r_ab = 0. Returns the number of zero-variance beams. */
int orc_corr_from_gram(const int64_t* G, int32_t n_beam, double* r);

/* Correlation from an FP64 covariance (same zero-variance rule). */
int orc_corr_from_cov(const double* cov, int32_t n_beam, double* r);

/* Cyclic (row-by-row) two-sided Jacobi in FP64 on a symmetric n x n matrix.
 * evals: n eigenvalues, largest first. q1: the unit eigenvector of evals[0],
 * sign chosen so its largest-magnitude element is positive (lowest index on
 * ties); may be NULL. sweeps: sweeps used; may be NULL. Stops when the
 * off-diagonal Frobenius norm is <= 1e-14 of the matrix norm, or after 100
 * sweeps. Returns 0, or -1 on bad arguments / no convergence. */
int orc_jacobi(const double* a, int32_t n, double* evals, double* q1,
               int32_t* sweeps);

/* Normalised dominant eigenvalue s = lambda_1^2 / sum_i lambda_i^2. */
double orc_stat(const double* evals, int32_t n);

/* Whole path for one cell: Gram, correlation, eigenvalues, q1, statistic.
 * Any output pointer may be NULL. Returns zero-variance beam count or -1. */
int orc_cell_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                int32_t n_chan, int32_t n_samp_sub, int32_t sub, int32_t chan,
                int64_t* G, double* r, double* evals, double* q1, double* stat);

/* All cells (cell index = sub * n_chan + chan) with n_threads host threads.
 * evals [cell][N], q1 [cell][N] may be NULL; stat [cell] required.
 * Returns 0 or -1. */
int orc_block_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                 int32_t n_chan, int32_t n_samp_sub, int32_t n_sub,
                 int32_t n_threads, double* evals, double* q1, double* stat);

/* Same for a list of cells (sub[i], chan[i]); outputs indexed by i. */
int orc_cells_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                 int32_t n_chan, int32_t n_samp_sub, int64_t n_list,
                 const int32_t* subs, const int32_t* chans, int32_t n_threads,
                 int64_t* G, double* evals, double* q1, double* stat);

/* orc_cells_u8 on the total power of a two-polarisation block. */
int orc_cells_pol2_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                      int32_t n_chan, int32_t n_samp_sub, int64_t n_list,
                      const int32_t* subs, const int32_t* chans, int32_t n_threads,
                      int64_t* G, double* evals, double* q1, double* stat);

/* Iterative clipping of the statistic (cells [sub][chan], n_cells a multiple
 * of n_chan). keep: n_chan bytes, nonzero = preserved channel (never flagged,
 * not in the statistics); may be NULL. Starting from an empty mask: mean and
 * population sigma of the statistic over unmasked, unpreserved cells,
 * threshold mu + k_sigma*sigma, add every unpreserved cell with s > threshold
 * to the mask; stop when nothing was added or after max_iter evaluations.
 * flags: n_cells bytes, 1 = RFI. Returns 0 or -1. */
int orc_flag(const double* stat, int64_t n_cells, int32_t n_chan,
             const uint8_t* keep, double k_sigma, int32_t max_iter,
             uint8_t* flags, orc_flag_info* info);

/* Eigenvector refinement (Section 3.3 last paragraph, Section 4.5
 * eigenvector threshold, t = 1): for every beam b a Gaussian fit (mean,
 * population sigma) to |q1_b| over the cells NOT flagged by the eigenvalue
 * mask and not preserved; a flagged cell marks beam b as affected when
 * |q1_b| > mu_b + t sigma_b. q1 [cell][N]; flags [cell]; keep [n_chan] or
 * NULL; bits [cell][ceil(N/32)] (bit b of word b/32); mu_sigma [N][2] or
 * NULL. Returns 0 or -1. */
int orc_beam_flags(const double* q1, const uint8_t* flags, int64_t n_cells, int32_t n_chan,
                   const uint8_t* keep, int32_t n_beam, double t, uint32_t* bits,
                   double* mu_sigma);

/* ------------------------------------------------------------------------
 * Section 3.1 bandpass and the bandpass-centred reading of Eq. 1.
 *
 * The bandpass of one beam over a fit interval is the time-aggregated
 * spectrum (the mean of each channel over the interval's samples); its
 * baseline z is fitted over channels with ArPLS (asymmetrically reweighted
 * penalized least squares, Baek, Park, Ahn and Ahn 2015, the method Section
 * 3.1 names; parameters lam, ratio, itermax as in Section 4.5's list) and
 * subtracted from every sample of the channel. Under the bandpass-centred
 * reading the CCM is C_ab = (1/N_s) sum_t (x_a(t) - z_a)(x_b(t) - z_b)
 * with no further centring or normalisation. */

/* One weighted Whittaker solve: z minimising sum_i w_i (y_i - z_i)^2 +
 * lam sum_k (z_k - 2 z_{k+1} + z_{k+2})^2, i.e. (W + lam D^T D) z = W y,
 * D the (n-2) x n second-difference matrix. The pentadiagonal symmetric
 * system is factored as L D L^T (unit lower-banded L) and solved by forward
 * and back substitution, FP64. n >= 3. Returns 0, or -1 on bad arguments or
 * a non-positive pivot. */
int orc_whittaker(const double* y, const double* w, int32_t n, double lam, double* z);

/* ArPLS baseline of y (n points): unit weights; then repeatedly z =
 * orc_whittaker(y, w); d = y - z; m and s = mean and population standard
 * deviation of the negative d_i; new weights 1 / (1 + exp(2 (d_i - (2 s - m))
 * / s)); stop when |w_new - w| / |w| < ratio (Euclidean norms), when no d_i
 * is negative or s == 0, or after itermax solves; z is the last solve.
 * Returns the number of solves (>= 1), or -1. */
int orc_arpls(const double* y, int32_t n, double lam, double ratio, int32_t itermax,
              double* z);

/* Time-aggregated spectrum of beam `beam` over sub-integrations
 * [sub0, sub0 + n_subs): y[j] = mean of x(t, j) over those samples. */
int orc_bandpass_input_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                          int32_t n_chan, int32_t n_samp_sub, int32_t sub0, int32_t n_subs,
                          int32_t beam, double* y);

/* C (N x N, FP64) of one cell under the bandpass-centred reading; zc[a] is
 * beam a's fitted bandpass at this cell's channel. */
int orc_cell_ccm_bandpass_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                             int32_t n_chan, int32_t n_samp_sub, int32_t sub, int32_t chan,
                             const double* zc, double* C);

/* Whole block under the bandpass-centred reading: fit intervals of
 * `interval` sub-integrations (the last one may be shorter), per interval
 * and beam the ArPLS baseline of the time-aggregated spectrum (z out:
 * [interval][beam][chan], may be NULL; iters out: [interval][beam], may be
 * NULL), then per cell C, its eigenvalues (FP64 Jacobi) and the statistic.
 * evals [cell][N] may be NULL; stat [cell] required. Returns 0 or -1. */
int orc_block_bandpass_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                          int32_t n_chan, int32_t n_samp_sub, int32_t n_sub, int32_t interval,
                          double lam, double ratio, int32_t itermax, int32_t n_threads,
                          double* z, int32_t* iters, double* evals, double* stat);

#ifdef __cplusplus
}
#endif
#endif
