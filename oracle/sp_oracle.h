/*
 * sp_oracle.h — plain, slow CPU oracle of the Spatial Pooler (SP) hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the reference the CUDA library is
 * checked against.  Only the tests, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load it; the library never does.  It shares no
 * code with the CUDA path: it takes the SP state (pools, permanences, boosts)
 * and the input frames as plain arrays, one byte per input bit, and does
 * every step literally, column by column and synapse by synapse.
 *
 * What it computes (Wielgosz & Pietron, "OpenCL-accelerated object
 * classification in video streams using Spatial Pooler of HTM"):
 *   - Overlap, Alg. 1 (Section 1.1): per column, the number of connected
 *     potential synapses whose input bit is 1; zero if below min_overlap,
 *     else multiplied by the column's boost.
 *   - Inhibition, Alg. 2 (Section 1.1, and the "winners_set_size comparison"
 *     of Section 3 "Hardware architecture"): a column is active iff its
 *     overlap is nonzero and it ranks among the winners_set_size highest in
 *     its neighbourhood (the whole SP, or a clipped square window on the
 *     column grid), ties going to the lower column index.
 *   - Learning (Section 1.1: the update the paper keeps on the CPU; inc/dec
 *     of Table 2): every potential synapse of an active column moves up by
 *     perm_inc when its input bit is 1 and down by perm_dec when it is 0,
 *     clamped to [0, 1].
 *   - Duty cycles (optional, Section 1.1 defers boosting to the Numenta
 *     rules and gives no formula): an exponential moving average of each
 *     column's activity, d <- d + (a - d) / period.
 *
 * Readings where the paper is silent or ambiguous:
 *   - "connected" means perm >= connect_threshold, compared in fp32;
 *   - a count equal to min_overlap survives (Alg. 1 zeroes only "<");
 *   - Alg. 2's max(..., 1) floor is read as "winners have overlap > 0";
 *   - Alg. 2's strict ">" against the n-th largest value is read as a rank
 *     count: the top winners_set_size under (overlap desc, index asc);
 *   - learning updates all potential synapses of the winners, with this
 *     frame's input, after inhibition; clamps are fminf(1, .)/fmaxf(0, .);
 *   - fp32 round-to-nearest for every arithmetic step, no FMA contraction
 *     (build with -ffp-contract=off).
 *
 * Every function returns 0 on success and -1 on an invalid argument (null
 * pointer, out-of-range index, zero size), writing nothing in that case.
 * Caller owns every buffer.
 */
#ifndef SP_ORACLE_H
#define SP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Parameters of one SP (all plain values). */
typedef struct {
  uint32_t C;             /* columns */
  uint32_t S;             /* potential synapses per column */
  uint64_t n_in;          /* input bits */
  float connect_threshold;
  float perm_inc, perm_dec;
  uint32_t min_overlap;
  uint32_t winners_set_size;
  uint32_t inhibition;    /* 0 global, 1 local window on the column grid,
                             2 the paper-literal reading of Alg. 2 (global) */
  uint32_t col_grid_w, col_grid_h; /* C = w * h when inhibition == 1 */
  uint32_t local_radius;  /* window (2r+1) x (2r+1), clipped at the edges */
} orc_params;

/* Alg. 1.  raw[c] = number of s with perm[c][s] >= thr and x[idx[c][s]] == 1;
 * ov[c] = raw < min_overlap ? 0 : (float)raw * boost[c].  idx, perm are
 * [C][S]; x has n_in bytes (nonzero = 1). raw may be NULL. */
int orc_overlap(uint32_t C, uint32_t S, const uint32_t* idx, const float* perm,
                const float* boost, uint64_t n_in, const uint8_t* x, float thr,
                uint32_t min_overlap, int32_t* raw, float* ov);

/* Alg. 2, global neighbourhood: active[c] = 1 for the (at most) k columns with
 * the highest overlap under (ov desc, c asc), among those with ov > 0.
 * Sort-based.  ov must be finite and >= 0. */
int orc_inhibit_global(uint32_t C, const float* ov, uint32_t k, uint8_t* active);

/* Alg. 2, local neighbourhood: column c = j*gw + i is active iff ov[c] > 0 and
 * fewer than k columns d of the window |i'-i| <= r, |j'-j| <= r (clipped)
 * beat it, where d beats c iff ov[d] > ov[c] or (ov[d] == ov[c] and d < c). */
int orc_inhibit_local(uint32_t gw, uint32_t gh, const float* ov, uint32_t k, uint32_t r,
                      uint8_t* active);

/* Paper-literal reading of Alg. 2 (global neighbourhood), for comparison
 * only: active iff ov[c] > max(v, 1), v the k-th largest overlap among the
 * other C - 1 columns (0 when there are fewer than k).  Boundary ties lose. */
int orc_inhibit_paper_literal(uint32_t C, const float* ov, uint32_t k, uint8_t* active);

/* Learning on the active columns, in place on perm [C][S]. */
int orc_learn(uint32_t C, uint32_t S, const uint32_t* idx, float* perm, uint64_t n_in,
              const uint8_t* x, const uint8_t* active, float inc, float dec);

/* One frame: overlap, inhibition, then learning when learn != 0.
 * raw and ov (nullable) receive the frame's overlaps; active receives C bytes. */
int orc_step(const orc_params* p, const uint32_t* idx, float* perm, const float* boost,
             const uint8_t* x, int learn, int32_t* raw, float* ov, uint8_t* active);

/* n_frames frames in sequence; frames is [n_frames][n_in] bytes; active_out
 * (nullable) is [n_frames][C] bytes; ov_out (nullable) is [n_frames][C]. */
int orc_run(const orc_params* p, const uint32_t* idx, float* perm, const float* boost,
            const uint8_t* frames, uint32_t n_frames, int learn, uint8_t* active_out,
            float* ov_out);

/* Duty-cycle update: d[c] = fl(d[c] + fl(fl(a[c] - d[c]) / period)), a[c] in {0, 1}
 * the column's activity this frame (fp32, each step rounded). */
int orc_duty_update(uint32_t C, float* duty, const uint8_t* active, float period);

/* Frame encoder (Section 2, and "Adaptive Video Encoder" in Section 3.1):
 * a colour frame becomes a binary image in three steps.
 *   1. Reduction by an integer factor f (optional, f = 1 keeps the size):
 *      the output is floor(W/f) x floor(H/f); each channel of an output pixel
 *      is the mean of its f x f source block, rounded half up:
 *      (sum + f*f/2) / (f*f).
 *   2. Grayscale: g = (77 R + 150 G + 29 B + 128) >> 8 (8-bit fixed-point
 *      luma weights summing to 256); a one-channel source is its own gray.
 *   3. Adaptive Gaussian threshold over a B x B window (B odd, 3..13): the
 *      Gaussian weights are the binomial coefficients w_i = C(B-1, i), the
 *      window weight of (dx, dy) is w_dx w_dy, coordinates outside the image
 *      take the nearest edge pixel; the local mean is
 *      m = (sum + 2^(2B-3)) >> (2B-2) (the weighted sum divided by the total
 *      weight 4^(B-1), rounded half up), and the bit is g > m - offset.
 * src is [H][W][channels] bytes (channels 1 or 3, R, G, B order); out_bits
 * receives floor(H/f) * floor(W/f) bytes (0/1), row-major.  Every step is
 * integer arithmetic, so the result is exact. */
int orc_encode(const uint8_t* src, uint32_t W, uint32_t H, uint32_t channels, uint32_t reduce,
               uint32_t block, int32_t offset, uint8_t* out_bits);

#ifdef __cplusplus
}
#endif

#endif /* SP_ORACLE_H */
