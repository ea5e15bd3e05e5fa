/* synth.c - seeded synthetic multi-beam filterbank generator (see synth.h).
 *
 * Integer-only so the bytes do not depend on the host's floating point,
 * libm or compiler contraction. Constants:
 *   GOLDEN   = 0x9e3779b97f4a7c15, the SplitMix64 increment;
 *   IH_SD_K  = round(2^32 / sqrt(8 * (256^2 - 1) / 12)) = 20547966: one over
 *              the standard deviation of a sum of eight uniform bytes, Q32;
 *   SIN16[i] = round(65536 * sin(2*pi*i/16)).
 */
#include "synth.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9e3779b97f4a7c15ULL
#define IH_MEAN 1020
#define IH_SD_K 20547966LL
#define SPIKE_LEN 16

enum { TAG_NOISE = 1, TAG_BANDPASS, TAG_NB_CHAN, TAG_NB_PHASE, TAG_NB_GAIN,
       TAG_BB_SUB, TAG_BB_OFF, TAG_BB_GAIN, TAG_SP_BEAM, TAG_SP_CHAN,
       TAG_SP_SUB, TAG_SP_OFF };

static const int32_t SIN16[16] = {0,      25080,  46341,  60547,  65536,  60547,
                                  46341,  25080,  0,      -25080, -46341, -60547,
                                  -65536, -60547, -46341, -25080};

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* Counter-based draw: the i-th SplitMix64 output of the stream keyed by
 * (seed, tag). */
static inline uint64_t draw(uint64_t seed, uint64_t tag, uint64_t i) {
  uint64_t key = mix64(seed ^ (tag * 0xd1b54a32d192ed03ULL));
  return mix64(key + (i + 1) * GOLDEN);
}

/* floor(v / 65536) for signed v, independent of the sign convention of >>. */
static inline int64_t floor_q16(int64_t v) {
  return v >= 0 ? (v >> 16) : -((-v + 65535) >> 16);
}

/* Per-beam event gain U(0.5, 1.5) in Q16. */
static inline int64_t event_gain_q16(uint64_t seed, uint64_t tag, uint64_t ev,
                                     int32_t n_beam, int32_t beam) {
  return 32768 + (int64_t)(draw(seed, tag, ev * (uint64_t)n_beam + beam) >> 48);
}

typedef struct {
  synth_cfg c;
  int64_t n_time;
  synth_narrow* nb;
  synth_burst* bb;
  synth_spike* sp;
  int32_t* nb_of_chan; /* narrowband event index per channel, or -1 */
  int32_t* sp_order;   /* spikes sorted by (beam, absolute start) */
} ctx_t;

static int cfg_ok(const synth_cfg* c) {
  if (c->n_beam < 1 || c->n_chan < 1 || c->n_samp_sub < 1 || c->n_sub < 1)
    return 0;
  if (c->n_narrow < 0 || c->n_narrow > c->n_chan) return 0;
  if (c->n_burst < 0 || (c->n_burst > 0 && c->n_sub < 2)) return 0;
  if (c->n_burst > c->n_sub - 1 && c->n_burst > 0) return 0;
  if (c->n_spike < 0) return 0;
  if (c->n_spike > 0 && c->n_narrow >= c->n_chan) return 0;
  return 1;
}

static int spike_cmp_ctx_beam(const synth_spike* a, const synth_spike* b,
                              int32_t n_s) {
  if (a->beam != b->beam) return a->beam < b->beam ? -1 : 1;
  int64_t ta = (int64_t)a->sub * n_s + a->off, tb = (int64_t)b->sub * n_s + b->off;
  if (ta != tb) return ta < tb ? -1 : 1;
  return 0;
}

static int build_events(const synth_cfg* c, synth_narrow* nb, synth_burst* bb,
                        synth_spike* sp, int32_t* nb_of_chan) {
  const uint64_t s = c->seed;
  for (int32_t ch = 0; ch < c->n_chan; ++ch) nb_of_chan[ch] = -1;
  for (int32_t i = 0; i < c->n_narrow; ++i) {
    int32_t ch = (int32_t)(draw(s, TAG_NB_CHAN, i) % (uint64_t)c->n_chan);
    while (nb_of_chan[ch] >= 0) ch = (ch + 1) % c->n_chan;
    nb_of_chan[ch] = i;
    nb[i].chan = ch;
    nb[i].phase = (int32_t)(draw(s, TAG_NB_PHASE, i) >> 60);
  }
  /* Broadband bursts: distinct start sub-integrations k in [0, n_sub-2]. */
  uint8_t* sub_used = (uint8_t*)calloc((size_t)c->n_sub, 1);
  if (!sub_used) return -1;
  for (int32_t i = 0; i < c->n_burst; ++i) {
    int32_t k = (int32_t)(draw(s, TAG_BB_SUB, i) % (uint64_t)(c->n_sub - 1));
    while (sub_used[k]) k = (k + 1) % (c->n_sub - 1);
    sub_used[k] = 1;
    int32_t quarter = c->n_samp_sub / 4;
    int32_t half = c->n_samp_sub / 2 > 0 ? c->n_samp_sub / 2 : 1;
    int32_t off = quarter + (int32_t)(draw(s, TAG_BB_OFF, i) % (uint64_t)half);
    bb[i].sub = k;
    bb[i].t0 = (int64_t)k * c->n_samp_sub + off;
  }
  /* Spikes avoid narrowband channels and burst sub-integrations, so a spike
   * cell carries no other RFI. */
  for (int32_t i = 0; i < c->n_spike; ++i) {
    int32_t beam = (int32_t)(draw(s, TAG_SP_BEAM, i) % (uint64_t)c->n_beam);
    int32_t ch = (int32_t)(draw(s, TAG_SP_CHAN, i) % (uint64_t)c->n_chan);
    while (nb_of_chan[ch] >= 0) ch = (ch + 1) % c->n_chan;
    int32_t k = (int32_t)(draw(s, TAG_SP_SUB, i) % (uint64_t)c->n_sub);
    for (int32_t tries = 0; tries < c->n_sub; ++tries) {
      int hit = sub_used[k] || (k > 0 && sub_used[k - 1]);
      if (!hit) break;
      k = (k + 1) % c->n_sub;
    }
    int32_t len = c->n_samp_sub < SPIKE_LEN ? c->n_samp_sub : SPIKE_LEN;
    int32_t off = (int32_t)(draw(s, TAG_SP_OFF, i) % (uint64_t)(c->n_samp_sub - len + 1));
    sp[i].beam = beam;
    sp[i].chan = ch;
    sp[i].sub = k;
    sp[i].off = off;
  }
  free(sub_used);
  return 0;
}

static void ctx_free(ctx_t* x) {
  free(x->nb);
  free(x->bb);
  free(x->sp);
  free(x->nb_of_chan);
  free(x->sp_order);
}

static int ctx_init(ctx_t* x, const synth_cfg* c) {
  memset(x, 0, sizeof(*x));
  if (!cfg_ok(c)) return -1;
  x->c = *c;
  x->n_time = (int64_t)c->n_sub * c->n_samp_sub;
  x->nb = (synth_narrow*)calloc((size_t)c->n_narrow + 1, sizeof(synth_narrow));
  x->bb = (synth_burst*)calloc((size_t)c->n_burst + 1, sizeof(synth_burst));
  x->sp = (synth_spike*)calloc((size_t)c->n_spike + 1, sizeof(synth_spike));
  x->nb_of_chan = (int32_t*)calloc((size_t)c->n_chan, sizeof(int32_t));
  x->sp_order = (int32_t*)calloc((size_t)c->n_spike + 1, sizeof(int32_t));
  if (!x->nb || !x->bb || !x->sp || !x->nb_of_chan || !x->sp_order ||
      build_events(c, x->nb, x->bb, x->sp, x->nb_of_chan) != 0) {
    ctx_free(x);
    return -1;
  }
  /* insertion sort of spike indices by (beam, start); lists are small */
  for (int32_t i = 0; i < c->n_spike; ++i) {
    int32_t j = i;
    while (j > 0 && spike_cmp_ctx_beam(&x->sp[x->sp_order[j - 1]], &x->sp[i],
                                       c->n_samp_sub) > 0) {
      x->sp_order[j] = x->sp_order[j - 1];
      --j;
    }
    x->sp_order[j] = i;
  }
  return 0;
}

static inline int64_t bandpass_q16(const synth_cfg* c, int32_t b, int32_t ch) {
  if (!c->bandpass) return 65536;
  uint64_t h = draw(c->seed, TAG_BANDPASS, (uint64_t)b * c->n_chan + ch);
  return 45875 + (int64_t)(((h >> 40) * 39322ULL) >> 24);
}

/* Noise scale of every channel of beam b: Q16 DN per unit of the centred
 * Irwin-Hall sum. */
static void beam_scales(const ctx_t* x, int32_t b, int64_t* scale) {
  for (int32_t ch = 0; ch < x->c.n_chan; ++ch)
    scale[ch] = ((int64_t)x->c.sigma_dn * bandpass_q16(&x->c, b, ch) * IH_SD_K) >> 32;
}

/* Generate one (beam, time) row of n_chan bytes; v is scratch of n_chan and
 * scale the beam's noise scales (beam_scales). */
static void gen_row(const ctx_t* x, int32_t b, int64_t t, uint8_t* out,
                    int64_t* v, const int64_t* scale) {
  const synth_cfg* c = &x->c;
  const int64_t n_chan = c->n_chan;
  const uint64_t key = mix64(c->seed ^ ((uint64_t)TAG_NOISE * 0xd1b54a32d192ed03ULL));
  const uint64_t base = ((uint64_t)b * (uint64_t)x->n_time + (uint64_t)t) * (uint64_t)n_chan;
  const int64_t mean_q16 = (int64_t)c->mean_dn << 16;
  for (int64_t ch = 0; ch < n_chan; ++ch) {
    uint64_t h = mix64(key + (base + (uint64_t)ch + 1) * GOLDEN);
    uint64_t s1 = (h & 0x00ff00ff00ff00ffULL) + ((h >> 8) & 0x00ff00ff00ff00ffULL);
    uint64_t s2 = (s1 & 0x0000ffff0000ffffULL) + ((s1 >> 16) & 0x0000ffff0000ffffULL);
    int64_t z = (int64_t)((s2 & 0xffffffffULL) + (s2 >> 32)) - IH_MEAN;
    v[ch] = mean_q16 + z * scale[ch];
  }
  /* broadband boxcars, all channels */
  for (int32_t i = 0; i < c->n_burst; ++i) {
    if (t >= x->bb[i].t0 && t < x->bb[i].t0 + c->n_samp_sub) {
      int64_t a = (int64_t)c->burst_amp_dn *
                  event_gain_q16(c->seed, TAG_BB_GAIN, (uint64_t)i, c->n_beam, b);
      for (int64_t ch = 0; ch < n_chan; ++ch) v[ch] += a;
    }
  }
  /* narrowband sines */
  for (int32_t i = 0; i < c->n_narrow; ++i) {
    int64_t a = (int64_t)c->narrow_amp_dn *
                event_gain_q16(c->seed, TAG_NB_GAIN, (uint64_t)i, c->n_beam, b);
    v[x->nb[i].chan] += floor_q16(a * SIN16[(t + x->nb[i].phase) & 15]);
  }
  /* single-beam spikes: binary search the first spike of this beam that could
   * cover t (spikes of one beam sorted by start) */
  if (c->n_spike > 0) {
    int32_t lo = 0, hi = c->n_spike;
    while (lo < hi) {
      int32_t mid = (lo + hi) / 2;
      const synth_spike* s = &x->sp[x->sp_order[mid]];
      int64_t ts = (int64_t)s->sub * c->n_samp_sub + s->off;
      if (s->beam < b || (s->beam == b && ts + SPIKE_LEN <= t)) lo = mid + 1;
      else hi = mid;
    }
    for (int32_t j = lo; j < c->n_spike; ++j) {
      const synth_spike* s = &x->sp[x->sp_order[j]];
      if (s->beam != b) break;
      int64_t ts = (int64_t)s->sub * c->n_samp_sub + s->off;
      int32_t len = c->n_samp_sub < SPIKE_LEN ? c->n_samp_sub : SPIKE_LEN;
      if (ts > t) break;
      if (t < ts + len) v[s->chan] += (int64_t)c->spike_amp_dn << 16;
    }
  }
  for (int64_t ch = 0; ch < n_chan; ++ch) {
    int64_t r = floor_q16(v[ch] + 32768);
    out[ch] = (uint8_t)(r < 0 ? 0 : (r > 255 ? 255 : r));
  }
}

typedef struct {
  const ctx_t* x;
  uint8_t* out;
  int64_t row0, row1;
  int rc;
} job_t;

static void* worker(void* arg) {
  job_t* j = (job_t*)arg;
  const ctx_t* x = j->x;
  int64_t* v = (int64_t*)malloc(sizeof(int64_t) * (size_t)x->c.n_chan);
  int64_t* scale = (int64_t*)malloc(sizeof(int64_t) * (size_t)x->c.n_chan);
  if (!v || !scale) {
    free(v);
    free(scale);
    j->rc = -1;
    return NULL;
  }
  int32_t cur_b = -1;
  for (int64_t r = j->row0; r < j->row1; ++r) {
    int32_t b = (int32_t)(r / x->n_time);
    int64_t t = r % x->n_time;
    if (b != cur_b) {
      beam_scales(x, b, scale);
      cur_b = b;
    }
    gen_row(x, b, t, j->out + r * (int64_t)x->c.n_chan, v, scale);
  }
  free(v);
  free(scale);
  j->rc = 0;
  return NULL;
}

int synth_generate(const synth_cfg* cfg, uint8_t* out, int n_threads) {
  ctx_t x;
  if (!out || ctx_init(&x, cfg) != 0) return -1;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  const int64_t rows = (int64_t)cfg->n_beam * x.n_time;
  if (rows < n_threads) n_threads = (int)(rows > 0 ? rows : 1);
  pthread_t th[256];
  job_t jobs[256];
  int created[256];
  int rc = 0;
  for (int i = 0; i < n_threads; ++i) {
    jobs[i].x = &x;
    jobs[i].out = out;
    jobs[i].row0 = rows * i / n_threads;
    jobs[i].row1 = rows * (i + 1) / n_threads;
    jobs[i].rc = -1;
    created[i] = i > 0 && pthread_create(&th[i], NULL, worker, &jobs[i]) == 0;
  }
  for (int i = 0; i < n_threads; ++i)
    if (!created[i]) worker(&jobs[i]);
  for (int i = 1; i < n_threads; ++i)
    if (created[i]) pthread_join(th[i], NULL);
  for (int i = 0; i < n_threads; ++i) rc |= jobs[i].rc;
  ctx_free(&x);
  return rc == 0 ? 0 : -1;
}

int synth_events(const synth_cfg* cfg, synth_narrow* nb, synth_burst* bb,
                 synth_spike* sp) {
  ctx_t x;
  if (ctx_init(&x, cfg) != 0) return -1;
  if (nb) memcpy(nb, x.nb, sizeof(synth_narrow) * (size_t)cfg->n_narrow);
  if (bb) memcpy(bb, x.bb, sizeof(synth_burst) * (size_t)cfg->n_burst);
  if (sp) memcpy(sp, x.sp, sizeof(synth_spike) * (size_t)cfg->n_spike);
  ctx_free(&x);
  return 0;
}

uint8_t synth_sample(const synth_cfg* cfg, int32_t beam, int64_t t, int32_t chan) {
  ctx_t x;
  if (ctx_init(&x, cfg) != 0) return 0;
  int64_t* v = (int64_t*)malloc(sizeof(int64_t) * (size_t)cfg->n_chan);
  int64_t* scale = (int64_t*)malloc(sizeof(int64_t) * (size_t)cfg->n_chan);
  uint8_t* row = (uint8_t*)malloc((size_t)cfg->n_chan);
  uint8_t r = 0;
  if (v && row && scale && beam >= 0 && beam < cfg->n_beam && t >= 0 &&
      t < x.n_time && chan >= 0 && chan < cfg->n_chan) {
    beam_scales(&x, beam, scale);
    gen_row(&x, beam, t, row, v, scale);
    r = row[chan];
  }
  free(v);
  free(scale);
  free(row);
  ctx_free(&x);
  return r;
}
