/*
 * sp_synth.h — seeded synthetic inputs for the Spatial Pooler (SP).
 *
 * The paper measures on a rendered "shapes" video dataset (Section 4.2,
 * Table 1: 960x540 renders reduced to 240x134, binarised by an adaptive
 * threshold, Section 3 "Adaptive Video Encoder").  That dataset is not
 * available, so every input of this library's tests and benchmarks is drawn
 * here from a seed instead: the SP's initial state (potential pools and
 * permanences, Section 1.1 "connected synapses" of Alg. 1, initial perm of
 * Table 2) and binary frames with the density and blob structure of
 * thresholded video.
 *
 * This module holds none of the SP's own arithmetic (overlap, inhibition,
 * learning).  It is the only code that both the CUDA library and the CPU
 * oracle depend on.  It is plain C99, deterministic on every host (no FMA
 * contraction: compile with -ffp-contract=off), and allocates nothing: every
 * output buffer is owned by the caller.
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), restated from its
 * published definition.
 *
 * Bit packing used everywhere in this library: input bit i lives in 32-bit
 * word i >> 5 at bit position i & 31 (LSB first); a W x H frame is flattened
 * row-major, i = y * W + x.
 *
 * Return codes: 0 on success, -1 when an argument is invalid (null pointer,
 * zero size, S larger than the candidate set, ...).  Nothing is written on
 * error.
 */
#ifndef SP_SYNTH_H
#define SP_SYNTH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(SP_SYNTH_BUILD)
#define SYNTH_API __attribute__((visibility("default")))
#else
#define SYNTH_API
#endif

/* Purposes for synth_derive_seed: sub-streams of one base seed. */
enum {
  SYNTH_PURPOSE_POOL = 1,   /* potential pools */
  SYNTH_PURPOSE_PERM = 2,   /* initial permanences */
  SYNTH_PURPOSE_FRAME = 3,  /* input frames (index = frame number) */
  SYNTH_PURPOSE_INSTANCE = 4, /* per-instance / per-stream base seeds */
  SYNTH_PURPOSE_SHAPE = 5   /* random sizes of batched instances */
};

/* One SplitMix64 step: advances *state and returns the next 64-bit output. */
SYNTH_API uint64_t synth_splitmix64(uint64_t* state);

/* Sub-seed for (base, purpose, index): two SplitMix64 mixes, stable across
 * hosts.  Used to give every frame / instance / stream its own stream. */
SYNTH_API uint64_t synth_derive_seed(uint64_t base, uint64_t purpose, uint64_t index);

/* Uniform potential pools: for each of C columns, S distinct input indices
 * drawn without replacement from [0, n_in) by a partial Fisher-Yates shuffle
 * (j = i + r mod (n - i)), then sorted ascending.  out_idx is [C][S].
 * scratch must hold n_in uint32 values. */
SYNTH_API int synth_pool_uniform(uint64_t seed, uint32_t C, uint32_t S, uint32_t n_in,
                                 uint32_t* out_idx, uint32_t* scratch);

/* Windowed potential pools (receptive fields): the columns lie on a
 * gw x gh grid (column c = j*gw + i); column (i, j) has its centre at
 * cx = floor((i + 1/2) W / gw), cy = floor((j + 1/2) H / gh); its window is
 * [cx - rf_w/2, cx - rf_w/2 + rf_w) x [cy - rf_h/2, ...), shifted inward to
 * lie inside the W x H frame, so every column has rf_w * rf_h candidates.
 * S of them are drawn as in synth_pool_uniform and sorted ascending.
 * out_idx is [C][S] with C = gw * gh; scratch holds rf_w * rf_h values. */
SYNTH_API int synth_pool_window(uint64_t seed, uint32_t gw, uint32_t gh, uint32_t W,
                                uint32_t H, uint32_t rf_w, uint32_t rf_h, uint32_t S,
                                uint32_t* out_idx, uint32_t* scratch);

/* Dense pools: every column's pool is the whole input, idx[c][s] = s. */
SYNTH_API int synth_pool_dense(uint32_t C, uint32_t n_in, uint32_t* out_idx);

/* Permanences uniform in [lo, hi): u = (r >> 40) * 2^-24 (exact in fp32),
 * perm = fl(lo + fl((hi - lo) * u)), each step one fp32 round-to-nearest op.
 * If lo == hi every permanence is lo (Table 2's single initial value). */
SYNTH_API int synth_perm_uniform(uint64_t seed, uint64_t n, float lo, float hi,
                                 float* out_perm);

/* Bernoulli(p) frame of n bits, one byte (0/1) per bit: bit = u < p with
 * u = (r >> 11) * 2^-53. */
SYNTH_API int synth_frame_bernoulli(uint64_t seed, uint64_t n, double p, uint8_t* out_bits);

/* Blobbed binary frame of W x H pixels, one byte (0/1) per pixel:
 *   1. p ~ U[p_lo, p_hi] (p = p_lo + (p_hi - p_lo) u, double);
 *   2. Bernoulli(p) noise n(x, y);
 *   3. v = sum of n over the 7x7 box around (x, y), clipped at the borders;
 *   4. pixel = (v * 255 + 24) / 49 (uint8, integer division);
 *   5. bit = pixel > t, t the smallest integer in [0, 255] for which the
 *      number of pixels > t is <= p * W * H (a 256-bin histogram).
 * scratch must hold 2 * W * H bytes.  *out_p (nullable) receives p. */
SYNTH_API int synth_frame_blobbed(uint64_t seed, uint32_t W, uint32_t H, double p_lo,
                                  double p_hi, uint8_t* out_bits, uint8_t* scratch,
                                  double* out_p);

/* Colour video-like frame of W x H pixels, 3 bytes (R, G, B) per pixel,
 * row-major: blobs under an illumination ramp, for the frame encoder.
 *   1. p = 0.05 + 0.15 u; per-channel gains g_c = 96 + (r mod 160); a ramp
 *      direction from the low 2 bits of one draw;
 *   2. field = (v * 255 + 24) / 49 with v the 7x7 box sum (clipped at the
 *      borders) of Bernoulli(p) noise, as in synth_frame_blobbed;
 *   3. light = 64 + 191 (x' + y') / (W + H - 2), x'/y' mirrored by the
 *      direction bits;
 *   4. channel c = (min(255, (field g_c + 32) / 64) * light + 127) / 255.
 * scratch must hold 2 * W * H bytes. */
SYNTH_API int synth_frame_rgb(uint64_t seed, uint32_t W, uint32_t H, uint8_t* out_rgb,
                              uint8_t* scratch);

/* Pack n one-byte bits (nonzero = 1) into ceil(n/32) LSB-first words; the
 * unused high bits of the last word are zero. */
SYNTH_API int synth_pack_bits(const uint8_t* bits, uint64_t n, uint32_t* out_words);

#ifdef __cplusplus
}
#endif

#endif /* SP_SYNTH_H */
