/* synth.h - seeded synthetic multi-beam filterbank generator.
 *
 * Produces 8-bit total-power samples laid out [beam][time][chan] (channel
 * fastest, the order a search-mode filterbank records them; the paper's data,
 * Section 2: 8-bit samples, 4096 channels, 1024 samples per sub-integration).
 * The generator holds none of the RFI method's arithmetic: it only draws
 * noise and injects RFI. Every value is computed with integer arithmetic
 * from a counter-based hash, so the bytes are identical on every host
 * (x86-64 and aarch64) and for every thread count.
 *
 * Noise: Irwin-Hall sum of the eight bytes of one SplitMix64 output
 * (Steele, Lea & Flood 2014), centred and scaled to sigma_dn DN, times an
 * optional per-(beam, channel) bandpass gain U(0.7, 1.3).
 * RFI common to all beams, each event with per-beam gains U(0.5, 1.5):
 *   - narrowband: a sine of period 16 samples in n_narrow channels, all times;
 *   - broadband: a boxcar n_samp_sub long in every channel, starting at a
 *     drawn offset inside a sub-integration, so it spans two sub-integrations;
 * and the single-beam control: a 16-sample spike in one beam of one cell.
 * x = clip(round_half_up(mean + noise + rfi), 0, 255).
 */
#ifndef MRAID_SYNTH_H
#define MRAID_SYNTH_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n_beam;
  int32_t n_chan;
  int32_t n_samp_sub;     /* samples per sub-integration */
  int32_t n_sub;          /* sub-integrations in the block */
  uint64_t seed;
  int32_t mean_dn;        /* noise mean, DN (128) */
  int32_t sigma_dn;       /* noise standard deviation, DN (20) */
  int32_t bandpass;       /* 1: per-(beam,chan) gain U(0.7,1.3); 0: gain 1 */
  int32_t n_narrow;       /* beam-common narrowband channels */
  int32_t narrow_amp_dn;  /* sine amplitude, DN (15) */
  int32_t n_burst;        /* beam-common broadband boxcars */
  int32_t burst_amp_dn;   /* DN (40) */
  int32_t n_spike;        /* single-beam spikes (controls) */
  int32_t spike_amp_dn;   /* DN (80) */
} synth_cfg;

/* Event lists, so tests can tell which cells carry which RFI. */
typedef struct {
  int32_t chan;   /* narrowband channel */
  int32_t phase;  /* 0..15 */
} synth_narrow;
typedef struct {
  int64_t t0;     /* first sample (absolute time index) */
  int32_t sub;    /* sub-integration containing t0; the boxcar ends in sub+1 */
} synth_burst;
typedef struct {
  int32_t beam, chan, sub;
  int32_t off;    /* first sample inside the sub-integration */
} synth_spike;

/* Fill out[] (n_beam * n_sub*n_samp_sub * n_chan bytes, [beam][time][chan])
 * using n_threads host threads (<=0: one). Returns 0, or -1 on bad sizes. */
int synth_generate(const synth_cfg* cfg, uint8_t* out, int n_threads);

/* Event lists (caller-allocated arrays of n_narrow / n_burst / n_spike). */
int synth_events(const synth_cfg* cfg, synth_narrow* nb, synth_burst* bb,
                 synth_spike* sp);

/* One sample, for spot checks: identical to out[] of synth_generate. */
uint8_t synth_sample(const synth_cfg* cfg, int32_t beam, int64_t t, int32_t chan);

#ifdef __cplusplus
}
#endif
#endif
