/* mraid_oracle.c - plain CPU oracle (TEST INFRASTRUCTURE ONLY; see header).
 *
 * Written for a reader checking it against the paper: no blocking, no
 * fusion, FP64 everywhere except the exact int64 sums.
 */
#include "mraid_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Eq. 1 */

int orc_cell_gram_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                     int32_t n_chan, int32_t n_samp_sub, int32_t sub,
                     int32_t chan, int64_t* G) {
  if (!data || !G || n_beam < 1 || n_chan < 1 || n_samp_sub < 1 || sub < 0 ||
      chan < 0 || chan >= n_chan)
    return -1;
  const int32_t N = n_beam, M = n_beam + 1;
  const int64_t t0 = (int64_t)sub * n_samp_sub;
  for (int32_t a = 0; a < M; ++a)
    for (int32_t b = 0; b < M; ++b) {
      int64_t s = 0;
      for (int32_t t = 0; t < n_samp_sub; ++t) {
        int64_t xa = (a < N) ? data[a * beam_stride + (t0 + t) * n_chan + chan] : 1;
        int64_t xb = (b < N) ? data[b * beam_stride + (t0 + t) * n_chan + chan] : 1;
        s += xa * xb;
      }
      G[a * M + b] = s;
    }
  return 0;
}

int orc_cell_gram_pol2_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                          int32_t n_chan, int32_t n_samp_sub, int32_t sub, int32_t chan,
                          int64_t* G) {
  if (!data || !G || n_beam < 1 || n_chan < 1 || n_samp_sub < 1 || sub < 0 ||
      chan < 0 || chan >= n_chan)
    return -1;
  const int32_t N = n_beam, M = n_beam + 1;
  const int64_t t0 = (int64_t)sub * n_samp_sub;
  for (int32_t a = 0; a < M; ++a)
    for (int32_t b = 0; b < M; ++b) {
      int64_t s = 0;
      for (int32_t t = 0; t < n_samp_sub; ++t) {
        const int64_t o = (t0 + t) * n_chan + chan;
        /* total power: polarisation 0 (block a) plus polarisation 1 (block N + a) */
        int64_t xa = (a < N) ? (int64_t)data[a * beam_stride + o] + data[(N + a) * beam_stride + o] : 1;
        int64_t xb = (b < N) ? (int64_t)data[b * beam_stride + o] + data[(N + b) * beam_stride + o] : 1;
        s += xa * xb;
      }
      G[a * M + b] = s;
    }
  return 0;
}

int orc_cell_cov_f32(const float* data, int32_t n_beam, int64_t beam_stride,
                     int32_t n_chan, int32_t n_samp_sub, int32_t sub,
                     int32_t chan, double* cov) {
  if (!data || !cov || n_beam < 1 || n_chan < 1 || n_samp_sub < 1 || sub < 0 ||
      chan < 0 || chan >= n_chan)
    return -1;
  const int32_t N = n_beam;
  const int64_t t0 = (int64_t)sub * n_samp_sub;
  double* mean = (double*)calloc((size_t)N, sizeof(double));
  if (!mean) return -1;
  for (int32_t a = 0; a < N; ++a) {
    double s = 0.0;
    for (int32_t t = 0; t < n_samp_sub; ++t)
      s += (double)data[a * beam_stride + (t0 + t) * n_chan + chan];
    mean[a] = s / n_samp_sub;
  }
  for (int32_t a = 0; a < N; ++a)
    for (int32_t b = 0; b < N; ++b) {
      double s = 0.0;
      for (int32_t t = 0; t < n_samp_sub; ++t) {
        double xa = (double)data[a * beam_stride + (t0 + t) * n_chan + chan] - mean[a];
        double xb = (double)data[b * beam_stride + (t0 + t) * n_chan + chan] - mean[b];
        s += xa * xb;
      }
      cov[a * N + b] = s / n_samp_sub;
    }
  free(mean);
  return 0;
}

int orc_corr_from_gram(const int64_t* G, int32_t n_beam, double* r) {
  if (!G || !r || n_beam < 1) return -1;
  const int32_t N = n_beam, M = n_beam + 1;
  const int64_t n = G[N * M + N];
  int degenerate = 0;
  int64_t* cov = (int64_t*)malloc(sizeof(int64_t) * (size_t)N * (size_t)N);
  if (!cov) return -1;
  for (int32_t a = 0; a < N; ++a)
    for (int32_t b = 0; b < N; ++b)
      cov[a * N + b] = n * G[a * M + b] - G[a * M + N] * G[b * M + N];
  for (int32_t a = 0; a < N; ++a)
    if (cov[a * N + a] == 0) ++degenerate;
  for (int32_t a = 0; a < N; ++a)
    for (int32_t b = 0; b < N; ++b) {
      if (a == b) {
        r[a * N + b] = 1.0;
      } else if (cov[a * N + a] == 0 || cov[b * N + b] == 0) {
        r[a * N + b] = 0.0;
      } else {
        r[a * N + b] = (double)cov[a * N + b] /
                       (sqrt((double)cov[a * N + a]) * sqrt((double)cov[b * N + b]));
      }
    }
  free(cov);
  return degenerate;
}

int orc_corr_from_cov(const double* cov, int32_t n_beam, double* r) {
  if (!cov || !r || n_beam < 1) return -1;
  const int32_t N = n_beam;
  int degenerate = 0;
  for (int32_t a = 0; a < N; ++a)
    if (cov[a * N + a] == 0.0) ++degenerate;
  for (int32_t a = 0; a < N; ++a)
    for (int32_t b = 0; b < N; ++b) {
      if (a == b)
        r[a * N + b] = 1.0;
      else if (cov[a * N + a] == 0.0 || cov[b * N + b] == 0.0)
        r[a * N + b] = 0.0;
      else
        r[a * N + b] = cov[a * N + b] / (sqrt(cov[a * N + a]) * sqrt(cov[b * N + b]));
    }
  return degenerate;
}

/* ---------------------------------------------------------------- Eq. 2 */

static double off_norm(const double* A, int32_t n) {
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j)
      if (i != j) s += A[i * n + j] * A[i * n + j];
  return sqrt(s);
}

static double fro_norm(const double* A, int32_t n) {
  double s = 0.0;
  for (int32_t i = 0; i < n * n; ++i) s += A[i] * A[i];
  return sqrt(s);
}

int orc_jacobi(const double* a_in, int32_t n, double* evals, double* q1,
               int32_t* sweeps) {
  if (!a_in || !evals || n < 1) return -1;
  double* A = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  if (!A || !V) {
    free(A);
    free(V);
    return -1;
  }
  memcpy(A, a_in, sizeof(double) * (size_t)n * (size_t)n);
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;

  const double norm = fro_norm(A, n);
  int32_t sweep = 0;
  int converged = (n == 1) || off_norm(A, n) <= 1e-14 * norm;
  while (!converged && sweep < 100) {
    for (int32_t p = 0; p < n - 1; ++p)
      for (int32_t q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (apq == 0.0) continue;
        /* rotation that zeroes A[p][q] (Golub & Van Loan, symmetric Schur) */
        const double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                      : -1.0 / (-tau + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double s = t * c;
        /* A <- A J: columns p and q */
        for (int32_t k = 0; k < n; ++k) {
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        /* A <- J^T A: rows p and q */
        for (int32_t k = 0; k < n; ++k) {
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        /* V <- V J */
        for (int32_t k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
    ++sweep;
    converged = off_norm(A, n) <= 1e-14 * norm;
  }

  /* eigenvalues largest first (selection of the remaining maximum) */
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  uint8_t* used = (uint8_t*)calloc((size_t)n, 1);
  if (!order || !used) {
    free(A);
    free(V);
    free(order);
    free(used);
    return -1;
  }
  for (int32_t i = 0; i < n; ++i) {
    int32_t best = -1;
    for (int32_t j = 0; j < n; ++j)
      if (!used[j] && (best < 0 || A[j * n + j] > A[best * n + best])) best = j;
    used[best] = 1;
    order[i] = best;
    evals[i] = A[best * n + best];
  }
  if (q1) {
    const int32_t col = order[0];
    double nrm = 0.0;
    for (int32_t k = 0; k < n; ++k) nrm += V[k * n + col] * V[k * n + col];
    nrm = sqrt(nrm);
    int32_t imax = 0;
    for (int32_t k = 1; k < n; ++k)
      if (fabs(V[k * n + col]) > fabs(V[imax * n + col])) imax = k;
    const double sign = (V[imax * n + col] < 0.0) ? -1.0 : 1.0;
    for (int32_t k = 0; k < n; ++k) q1[k] = sign * V[k * n + col] / nrm;
  }
  if (sweeps) *sweeps = sweep;
  free(A);
  free(V);
  free(order);
  free(used);
  return converged ? 0 : -1;
}

double orc_stat(const double* evals, int32_t n) {
  double ss = 0.0;
  for (int32_t i = 0; i < n; ++i) ss += evals[i] * evals[i];
  return ss > 0.0 ? evals[0] * evals[0] / ss : 0.0;
}

/* ------------------------------------------------------------- per cell */

int orc_cell_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                int32_t n_chan, int32_t n_samp_sub, int32_t sub, int32_t chan,
                int64_t* G, double* r, double* evals, double* q1, double* stat) {
  const int32_t N = n_beam, M = n_beam + 1;
  int64_t* g = (int64_t*)malloc(sizeof(int64_t) * (size_t)M * (size_t)M);
  double* rr = (double*)malloc(sizeof(double) * (size_t)N * (size_t)N);
  double* ev = (double*)malloc(sizeof(double) * (size_t)N);
  int rc = -1;
  if (g && rr && ev &&
      orc_cell_gram_u8(data, n_beam, beam_stride, n_chan, n_samp_sub, sub, chan, g) == 0) {
    int deg = orc_corr_from_gram(g, N, rr);
    if (deg >= 0 && orc_jacobi(rr, N, ev, q1, NULL) == 0) {
      if (G) memcpy(G, g, sizeof(int64_t) * (size_t)M * (size_t)M);
      if (r) memcpy(r, rr, sizeof(double) * (size_t)N * (size_t)N);
      if (evals) memcpy(evals, ev, sizeof(double) * (size_t)N);
      if (stat) *stat = orc_stat(ev, N);
      rc = deg;
    }
  }
  free(g);
  free(rr);
  free(ev);
  return rc;
}

/* the path of orc_cell_u8 on the total power of two polarisations */
static int cell_pol2_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                        int32_t n_chan, int32_t n_samp_sub, int32_t sub, int32_t chan,
                        int64_t* G, double* evals, double* q1, double* stat) {
  const int32_t N = n_beam, M = n_beam + 1;
  int64_t* g = (int64_t*)malloc(sizeof(int64_t) * (size_t)M * (size_t)M);
  double* rr = (double*)malloc(sizeof(double) * (size_t)N * (size_t)N);
  double* ev = (double*)malloc(sizeof(double) * (size_t)N);
  int rc = -1;
  if (g && rr && ev &&
      orc_cell_gram_pol2_u8(data, n_beam, beam_stride, n_chan, n_samp_sub, sub, chan, g) == 0) {
    int deg = orc_corr_from_gram(g, N, rr);
    if (deg >= 0 && orc_jacobi(rr, N, ev, q1, NULL) == 0) {
      if (G) memcpy(G, g, sizeof(int64_t) * (size_t)M * (size_t)M);
      if (evals) memcpy(evals, ev, sizeof(double) * (size_t)N);
      if (stat) *stat = orc_stat(ev, N);
      rc = deg;
    }
  }
  free(g);
  free(rr);
  free(ev);
  return rc;
}

typedef struct {
  const uint8_t* data;
  int32_t n_beam, n_chan, n_samp_sub;
  int64_t beam_stride;
  const int32_t* subs;
  const int32_t* chans;
  int64_t i0, i1;
  int64_t* G;
  double *evals, *q1, *stat;
  int rc;
  int pol2;  /* 1: total power of two polarisations */
} cells_job;

static void* cells_worker(void* arg) {
  cells_job* j = (cells_job*)arg;
  const int32_t N = j->n_beam, M = N + 1;
  j->rc = 0;
  for (int64_t i = j->i0; i < j->i1; ++i) {
    int32_t sub = j->subs ? j->subs[i] : (int32_t)(i / j->n_chan);
    int32_t chan = j->chans ? j->chans[i] : (int32_t)(i % j->n_chan);
    int64_t* Gi = j->G ? j->G + i * M * M : NULL;
    double* evi = j->evals ? j->evals + i * N : NULL;
    double* q1i = j->q1 ? j->q1 + i * N : NULL;
    const int rc = j->pol2 ? cell_pol2_u8(j->data, N, j->beam_stride, j->n_chan, j->n_samp_sub,
                                          sub, chan, Gi, evi, q1i, &j->stat[i])
                           : orc_cell_u8(j->data, N, j->beam_stride, j->n_chan, j->n_samp_sub,
                                         sub, chan, Gi, NULL, evi, q1i, &j->stat[i]);
    if (rc < 0) j->rc = -1;
  }
  return NULL;
}

static int run_cells(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                     int32_t n_chan, int32_t n_samp_sub, int64_t n_list,
                     const int32_t* subs, const int32_t* chans, int32_t n_threads,
                     int64_t* G, double* evals, double* q1, double* stat, int pol2) {
  if (!data || !stat || n_list < 0) return -1;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 512) n_threads = 512;
  if (n_list < n_threads) n_threads = n_list > 0 ? (int32_t)n_list : 1;
  pthread_t th[512];
  cells_job jobs[512];
  int created[512];
  for (int32_t i = 0; i < n_threads; ++i) {
    cells_job j = {data, n_beam, n_chan, n_samp_sub, beam_stride, subs, chans,
                   n_list * i / n_threads, n_list * (i + 1) / n_threads, G,
                   evals, q1, stat, -1, pol2};
    jobs[i] = j;
    created[i] = i > 0 && pthread_create(&th[i], NULL, cells_worker, &jobs[i]) == 0;
  }
  for (int32_t i = 0; i < n_threads; ++i)
    if (!created[i]) cells_worker(&jobs[i]);
  int rc = 0;
  for (int32_t i = 0; i < n_threads; ++i) {
    if (created[i]) pthread_join(th[i], NULL);
    rc |= jobs[i].rc;
  }
  return rc;
}

int orc_block_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                 int32_t n_chan, int32_t n_samp_sub, int32_t n_sub,
                 int32_t n_threads, double* evals, double* q1, double* stat) {
  return run_cells(data, n_beam, beam_stride, n_chan, n_samp_sub,
                   (int64_t)n_sub * n_chan, NULL, NULL, n_threads, NULL, evals,
                   q1, stat, 0);
}

int orc_cells_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                 int32_t n_chan, int32_t n_samp_sub, int64_t n_list,
                 const int32_t* subs, const int32_t* chans, int32_t n_threads,
                 int64_t* G, double* evals, double* q1, double* stat) {
  if (!subs || !chans) return -1;
  return run_cells(data, n_beam, beam_stride, n_chan, n_samp_sub, n_list, subs,
                   chans, n_threads, G, evals, q1, stat, 0);
}

int orc_cells_pol2_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                      int32_t n_chan, int32_t n_samp_sub, int64_t n_list,
                      const int32_t* subs, const int32_t* chans, int32_t n_threads,
                      int64_t* G, double* evals, double* q1, double* stat) {
  if (!subs || !chans) return -1;
  return run_cells(data, n_beam, beam_stride, n_chan, n_samp_sub, n_list, subs,
                   chans, n_threads, G, evals, q1, stat, 1);
}

/* ------------------------------------------------- iterative RFI masking */

static double pairwise_sum(const double* x, int64_t n) {
  if (n <= 8) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += x[i];
    return s;
  }
  const int64_t h = n / 2;
  return pairwise_sum(x, h) + pairwise_sum(x + h, n - h);
}

int orc_flag(const double* stat, int64_t n_cells, int32_t n_chan,
             const uint8_t* keep, double k_sigma, int32_t max_iter,
             uint8_t* flags, orc_flag_info* info) {
  if (!stat || !flags || n_chan < 1 || n_cells < 0 || n_cells % n_chan != 0 ||
      max_iter < 1)
    return -1;
  double* vals = (double*)malloc(sizeof(double) * (size_t)(n_cells > 0 ? n_cells : 1));
  if (!vals) return -1;
  memset(flags, 0, (size_t)n_cells);
  double mu = 0.0, sigma = 0.0, thresh = 0.0;
  int64_t used = 0;
  int32_t it = 0;
  int converged = 0;
  while (it < max_iter) {
    /* Gaussian fit (mean, population sigma) of the unmasked distribution */
    used = 0;
    for (int64_t i = 0; i < n_cells; ++i)
      if (!flags[i] && !(keep && keep[i % n_chan])) vals[used++] = stat[i];
    ++it;
    if (used == 0) {
      mu = sigma = 0.0;
      thresh = INFINITY;
      converged = 1;
      break;
    }
    mu = pairwise_sum(vals, used) / (double)used;
    for (int64_t i = 0; i < used; ++i) vals[i] = (vals[i] - mu) * (vals[i] - mu);
    sigma = sqrt(pairwise_sum(vals, used) / (double)used);
    thresh = mu + k_sigma * sigma;
    /* mask every unpreserved cell above the dynamic threshold */
    int64_t added = 0;
    for (int64_t i = 0; i < n_cells; ++i)
      if (!flags[i] && !(keep && keep[i % n_chan]) && stat[i] > thresh) {
        flags[i] = 1;
        ++added;
      }
    if (added == 0) {
      converged = 1;
      break;
    }
  }
  if (info) {
    int64_t nf = 0;
    for (int64_t i = 0; i < n_cells; ++i) nf += flags[i];
    info->mu = mu;
    info->sigma = sigma;
    info->thresh = thresh;
    info->iterations = it;
    info->converged = converged;
    info->n_flagged = nf;
    info->n_used = used;
  }
  free(vals);
  return 0;
}

/* --------------------------------------- eigenvector refinement (Sec. 3.3) */

int orc_beam_flags(const double* q1, const uint8_t* flags, int64_t n_cells, int32_t n_chan,
                   const uint8_t* keep, int32_t n_beam, double t, uint32_t* bits,
                   double* mu_sigma) {
  if (!q1 || !flags || !bits || n_cells < 0 || n_chan < 1 || n_beam < 1 || !(t >= 0.0))
    return -1;
  const int32_t W = (n_beam + 31) / 32;
  double* vals = (double*)malloc(sizeof(double) * (size_t)(n_cells > 0 ? n_cells : 1));
  double* mu = (double*)calloc((size_t)n_beam, sizeof(double));
  double* sg = (double*)calloc((size_t)n_beam, sizeof(double));
  if (!vals || !mu || !sg) {
    free(vals);
    free(mu);
    free(sg);
    return -1;
  }
  for (int32_t b = 0; b < n_beam; ++b) {
    /* Gaussian fit to the beam's eigenvector elements of non-RFI cells */
    int64_t m = 0;
    for (int64_t i = 0; i < n_cells; ++i)
      if (!flags[i] && !(keep && keep[i % n_chan])) vals[m++] = fabs(q1[i * n_beam + b]);
    if (m > 0) {
      mu[b] = pairwise_sum(vals, m) / (double)m;
      for (int64_t i = 0; i < m; ++i) vals[i] = (vals[i] - mu[b]) * (vals[i] - mu[b]);
      sg[b] = sqrt(pairwise_sum(vals, m) / (double)m);
    }
  }
  for (int64_t i = 0; i < n_cells; ++i) {
    for (int32_t w = 0; w < W; ++w) bits[i * W + w] = 0u;
    if (!flags[i]) continue;
    for (int32_t b = 0; b < n_beam; ++b)
      if (fabs(q1[i * n_beam + b]) > mu[b] + t * sg[b]) bits[i * W + b / 32] |= 1u << (b % 32);
  }
  if (mu_sigma)
    for (int32_t b = 0; b < n_beam; ++b) {
      mu_sigma[2 * b] = mu[b];
      mu_sigma[2 * b + 1] = sg[b];
    }
  free(vals);
  free(mu);
  free(sg);
  return 0;
}

/* ------------------------------------- Section 3.1: bandpass with ArPLS */

int orc_whittaker(const double* y, const double* w, int32_t n, double lam, double* z) {
  if (!y || !w || !z || n < 3 || !(lam >= 0.0)) return -1;
  /* A = W + lam D^T D as three bands: A[i][i], A[i][i+1], A[i][i+2].
   * D^T D is accumulated row by row of D (coefficients 1, -2, 1). */
  double* a0 = calloc((size_t)n, sizeof(double));
  double* a1 = calloc((size_t)n, sizeof(double));
  double* a2 = calloc((size_t)n, sizeof(double));
  double* l1 = calloc((size_t)n, sizeof(double));
  double* l2 = calloc((size_t)n, sizeof(double));
  double* dg = calloc((size_t)n, sizeof(double));
  double* u = calloc((size_t)n, sizeof(double));
  int rc = 0;
  if (!a0 || !a1 || !a2 || !l1 || !l2 || !dg || !u) {
    rc = -1;
    goto done;
  }
  {
    const double c[3] = {1.0, -2.0, 1.0};
    for (int32_t k = 0; k + 2 < n; ++k)
      for (int p = 0; p < 3; ++p)
        for (int q = p; q < 3; ++q) {
          const double v = lam * c[p] * c[q];
          if (q == p) a0[k + p] += v;
          else if (q == p + 1) a1[k + p] += v;
          else a2[k + p] += v;
        }
    for (int32_t i = 0; i < n; ++i) a0[i] += w[i];
    /* A = L diag(dg) L^T, L unit lower with L[i][i-1] = l1[i], L[i][i-2] = l2[i] */
    for (int32_t i = 0; i < n; ++i) {
      l2[i] = (i >= 2) ? a2[i - 2] / dg[i - 2] : 0.0;
      l1[i] = (i >= 1) ? (a1[i - 1] - ((i >= 2) ? l2[i] * dg[i - 2] * l1[i - 1] : 0.0)) / dg[i - 1]
                       : 0.0;
      dg[i] = a0[i] - ((i >= 1) ? l1[i] * l1[i] * dg[i - 1] : 0.0) -
              ((i >= 2) ? l2[i] * l2[i] * dg[i - 2] : 0.0);
      if (!(dg[i] > 0.0)) {
        rc = -1;
        goto done;
      }
    }
    /* L u = W y; then L^T z = u / dg */
    for (int32_t i = 0; i < n; ++i)
      u[i] = w[i] * y[i] - ((i >= 1) ? l1[i] * u[i - 1] : 0.0) -
             ((i >= 2) ? l2[i] * u[i - 2] : 0.0);
    for (int32_t i = n - 1; i >= 0; --i)
      z[i] = u[i] / dg[i] - ((i + 1 < n) ? l1[i + 1] * z[i + 1] : 0.0) -
             ((i + 2 < n) ? l2[i + 2] * z[i + 2] : 0.0);
  }
done:
  free(a0);
  free(a1);
  free(a2);
  free(l1);
  free(l2);
  free(dg);
  free(u);
  return rc;
}

int orc_arpls(const double* y, int32_t n, double lam, double ratio, int32_t itermax,
              double* z) {
  if (!y || !z || n < 3 || itermax < 1) return -1;
  double* w = malloc(sizeof(double) * (size_t)n);
  double* wt = malloc(sizeof(double) * (size_t)n);
  if (!w || !wt) {
    free(w);
    free(wt);
    return -1;
  }
  for (int32_t i = 0; i < n; ++i) w[i] = 1.0;
  int32_t solves = 0;
  int rc = 0;
  while (solves < itermax) {
    if (orc_whittaker(y, w, n, lam, z) < 0) {
      rc = -1;
      break;
    }
    ++solves;
    /* statistics of the negative residuals */
    double sum = 0.0, sum2 = 0.0;
    int64_t cnt = 0;
    for (int32_t i = 0; i < n; ++i) {
      const double d = y[i] - z[i];
      if (d < 0.0) {
        sum += d;
        ++cnt;
      }
    }
    if (cnt == 0) break;
    const double m = sum / (double)cnt;
    for (int32_t i = 0; i < n; ++i) {
      const double d = y[i] - z[i];
      if (d < 0.0) sum2 += (d - m) * (d - m);
    }
    const double s = sqrt(sum2 / (double)cnt);
    if (!(s > 0.0)) break;
    double dw2 = 0.0, w2 = 0.0;
    for (int32_t i = 0; i < n; ++i) {
      const double d = y[i] - z[i];
      wt[i] = 1.0 / (1.0 + exp(2.0 * (d - (2.0 * s - m)) / s));
      dw2 += (w[i] - wt[i]) * (w[i] - wt[i]);
      w2 += w[i] * w[i];
    }
    if (sqrt(dw2) / sqrt(w2) < ratio) break;
    for (int32_t i = 0; i < n; ++i) w[i] = wt[i];
  }
  free(w);
  free(wt);
  return rc < 0 ? -1 : solves;
}

int orc_bandpass_input_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                          int32_t n_chan, int32_t n_samp_sub, int32_t sub0, int32_t n_subs,
                          int32_t beam, double* y) {
  if (!data || !y || beam < 0 || beam >= n_beam || n_subs < 1 || sub0 < 0) return -1;
  const int64_t t0 = (int64_t)sub0 * n_samp_sub, nt = (int64_t)n_subs * n_samp_sub;
  for (int32_t j = 0; j < n_chan; ++j) {
    int64_t s = 0;
    for (int64_t t = 0; t < nt; ++t) s += data[beam * beam_stride + (t0 + t) * n_chan + j];
    y[j] = (double)s / (double)nt;
  }
  return 0;
}

int orc_cell_ccm_bandpass_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                             int32_t n_chan, int32_t n_samp_sub, int32_t sub, int32_t chan,
                             const double* zc, double* C) {
  if (!data || !zc || !C || n_beam < 1 || chan < 0 || chan >= n_chan || sub < 0) return -1;
  const int64_t t0 = (int64_t)sub * n_samp_sub;
  for (int32_t a = 0; a < n_beam; ++a)
    for (int32_t b = 0; b < n_beam; ++b) {
      double s = 0.0;
      for (int32_t t = 0; t < n_samp_sub; ++t) {
        const double xa = data[a * beam_stride + (t0 + t) * n_chan + chan] - zc[a];
        const double xb = data[b * beam_stride + (t0 + t) * n_chan + chan] - zc[b];
        s += xa * xb;
      }
      C[a * n_beam + b] = s / (double)n_samp_sub;
    }
  return 0;
}

typedef struct {
  const uint8_t* data;
  int32_t n_beam, n_chan, n_samp_sub, interval;
  int64_t beam_stride;
  const double* z;
  int64_t i0, i1;
  double *evals, *stat;
  int rc;
} bp_job;

static void* bp_worker(void* arg) {
  bp_job* j = (bp_job*)arg;
  const int32_t N = j->n_beam;
  double* zc = malloc(sizeof(double) * (size_t)N);
  double* C = malloc(sizeof(double) * (size_t)N * N);
  double* ev = malloc(sizeof(double) * (size_t)N);
  j->rc = (zc && C && ev) ? 0 : -1;
  for (int64_t i = j->i0; i < j->i1 && j->rc == 0; ++i) {
    const int32_t sub = (int32_t)(i / j->n_chan), chan = (int32_t)(i % j->n_chan);
    const int32_t I = sub / j->interval;
    for (int32_t a = 0; a < N; ++a) zc[a] = j->z[((int64_t)I * N + a) * j->n_chan + chan];
    if (orc_cell_ccm_bandpass_u8(j->data, N, j->beam_stride, j->n_chan, j->n_samp_sub, sub,
                                 chan, zc, C) < 0 ||
        orc_jacobi(C, N, ev, NULL, NULL) < 0) {
      j->rc = -1;
      break;
    }
    if (j->evals)
      for (int32_t a = 0; a < N; ++a) j->evals[i * N + a] = ev[a];
    j->stat[i] = orc_stat(ev, N);
  }
  free(zc);
  free(C);
  free(ev);
  return NULL;
}

int orc_block_bandpass_u8(const uint8_t* data, int32_t n_beam, int64_t beam_stride,
                          int32_t n_chan, int32_t n_samp_sub, int32_t n_sub, int32_t interval,
                          double lam, double ratio, int32_t itermax, int32_t n_threads,
                          double* z, int32_t* iters, double* evals, double* stat) {
  if (!data || !stat || n_beam < 1 || n_chan < 3 || n_sub < 1 || interval < 1) return -1;
  const int32_t n_int = (n_sub + interval - 1) / interval;
  double* zz = z ? z : malloc(sizeof(double) * (size_t)n_int * n_beam * n_chan);
  double* y = malloc(sizeof(double) * (size_t)n_chan);
  int rc = (zz && y) ? 0 : -1;
  for (int32_t I = 0; I < n_int && rc == 0; ++I) {
    const int32_t s0 = I * interval;
    const int32_t ns = (n_sub - s0) < interval ? (n_sub - s0) : interval;
    for (int32_t a = 0; a < n_beam && rc == 0; ++a) {
      double* za = zz + ((int64_t)I * n_beam + a) * n_chan;
      if (orc_bandpass_input_u8(data, n_beam, beam_stride, n_chan, n_samp_sub, s0, ns, a, y) < 0)
        rc = -1;
      const int it = rc == 0 ? orc_arpls(y, n_chan, lam, ratio, itermax, za) : -1;
      if (it < 0) rc = -1;
      if (iters && rc == 0) iters[(int64_t)I * n_beam + a] = it;
    }
  }
  if (rc == 0) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 512) n_threads = 512;
    const int64_t n_cells = (int64_t)n_sub * n_chan;
    pthread_t th[512];
    bp_job jobs[512];
    int created[512];
    for (int32_t i = 0; i < n_threads; ++i) {
      bp_job j = {data, n_beam, n_chan, n_samp_sub, interval, beam_stride, zz,
                  n_cells * i / n_threads, n_cells * (i + 1) / n_threads, evals, stat, -1};
      jobs[i] = j;
      created[i] = i > 0 && pthread_create(&th[i], NULL, bp_worker, &jobs[i]) == 0;
    }
    for (int32_t i = 0; i < n_threads; ++i)
      if (!created[i]) bp_worker(&jobs[i]);
    for (int32_t i = 0; i < n_threads; ++i) {
      if (created[i]) pthread_join(th[i], NULL);
      rc |= jobs[i].rc;
    }
  }
  if (!z) free(zz);
  free(y);
  return rc;
}
