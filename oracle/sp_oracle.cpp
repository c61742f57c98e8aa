// Plain CPU oracle of the Spatial Pooler hot path.  TEST INFRASTRUCTURE ONLY:
// loaded by the tests, __graft_entry__.smoke() and bench.py's CPU baseline
// leg, never by the library.  Definitions and readings: sp_oracle.h.
//
// Every loop below walks the paper's objects in the paper's order: columns,
// then each column's synapses (Alg. 1); columns, then each column's
// competitors (Alg. 2).  No blocking, no bit tricks, no reuse of anything
// from the CUDA library.  Build with -O2 -ffp-contract=off.
#include "sp_oracle.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

// The total order used by inhibition: a beats b iff it has a higher overlap,
// or the same overlap and a lower column index.
bool beats(float ov_a, uint32_t a, float ov_b, uint32_t b) {
  if (ov_a != ov_b) return ov_a > ov_b;
  return a < b;
}

bool valid_overlaps(uint32_t C, const float* ov) {
  for (uint32_t c = 0; c < C; ++c)
    if (!(ov[c] >= 0.0f) || std::isinf(ov[c])) return false;
  return true;
}

}  // namespace

extern "C" {

// Alg. 1 (Section 1.1), with the boost applied inside the overlap as the
// paper's overlap unit does (Section 3, "Hardware architecture").
int orc_overlap(uint32_t C, uint32_t S, const uint32_t* idx, const float* perm,
                const float* boost, uint64_t n_in, const uint8_t* x, float thr,
                uint32_t min_overlap, int32_t* raw, float* ov) {
  if (!idx || !perm || !boost || !x || !ov || C == 0 || S == 0 || n_in == 0) return -1;
  for (uint64_t i = 0; i < (uint64_t)C * S; ++i)
    if (idx[i] >= n_in) return -1;
  for (uint32_t c = 0; c < C; ++c) {
    int32_t overlap = 0;
    for (uint32_t s = 0; s < S; ++s) {
      const uint64_t e = (uint64_t)c * S + s;
      const bool connected = perm[e] >= thr;
      const bool input_active = x[idx[e]] != 0;
      if (connected && input_active) overlap += 1;
    }
    if (raw) raw[c] = overlap;
    if ((uint32_t)overlap < min_overlap)
      ov[c] = 0.0f;
    else
      ov[c] = (float)overlap * boost[c];
  }
  return 0;
}

// Alg. 2 over the whole SP: sort every candidate with a nonzero overlap by the
// total order and keep the first k.
int orc_inhibit_global(uint32_t C, const float* ov, uint32_t k, uint8_t* active) {
  if (!ov || !active || C == 0 || !valid_overlaps(C, ov)) return -1;
  std::vector<uint32_t> cand;
  for (uint32_t c = 0; c < C; ++c)
    if (ov[c] > 0.0f) cand.push_back(c);
  std::sort(cand.begin(), cand.end(),
            [&](uint32_t a, uint32_t b) { return beats(ov[a], a, ov[b], b); });
  for (uint32_t c = 0; c < C; ++c) active[c] = 0;
  for (size_t r = 0; r < cand.size() && r < k; ++r) active[cand[r]] = 1;
  return 0;
}

// Alg. 2 with a square neighbourhood of radius r on the column grid: count the
// neighbours that beat the column; it wins when fewer than k do.
int orc_inhibit_local(uint32_t gw, uint32_t gh, const float* ov, uint32_t k, uint32_t r,
                      uint8_t* active) {
  if (!ov || !active || gw == 0 || gh == 0) return -1;
  const uint32_t C = gw * gh;
  if (!valid_overlaps(C, ov)) return -1;
  for (uint32_t j = 0; j < gh; ++j) {
    for (uint32_t i = 0; i < gw; ++i) {
      const uint32_t c = j * gw + i;
      active[c] = 0;
      if (!(ov[c] > 0.0f)) continue;
      const uint32_t j0 = j >= r ? j - r : 0, j1 = std::min(gh - 1, j + r);
      const uint32_t i0 = i >= r ? i - r : 0, i1 = std::min(gw - 1, i + r);
      uint32_t beaten_by = 0;
      for (uint32_t jj = j0; jj <= j1; ++jj)
        for (uint32_t ii = i0; ii <= i1; ++ii) {
          const uint32_t d = jj * gw + ii;
          if (d != c && beats(ov[d], d, ov[c], c)) ++beaten_by;
        }
      if (beaten_by < k) active[c] = 1;
    }
  }
  return 0;
}

// Alg. 2 taken word for word, over the whole SP: n_max_overlap(col, n) is read
// as the n-th largest overlap among the other columns (0 when there are fewer
// than n), and a column is active iff its overlap strictly exceeds the larger
// of that value and 1.  Ties at the boundary therefore all lose.
int orc_inhibit_paper_literal(uint32_t C, const float* ov, uint32_t k, uint8_t* active) {
  if (!ov || !active || C == 0 || !valid_overlaps(C, ov)) return -1;
  for (uint32_t c = 0; c < C; ++c) {
    std::vector<float> others;
    for (uint32_t d = 0; d < C; ++d)
      if (d != c) others.push_back(ov[d]);
    std::sort(others.begin(), others.end(), [](float a, float b) { return a > b; });
    const float nth = (k >= 1 && k <= others.size()) ? others[k - 1] : 0.0f;
    const float max_column = std::max(nth, 1.0f);
    active[c] = ov[c] > max_column ? 1 : 0;
  }
  return 0;
}

// Learning (Section 1.1; increments of Table 2).
int orc_learn(uint32_t C, uint32_t S, const uint32_t* idx, float* perm, uint64_t n_in,
              const uint8_t* x, const uint8_t* active, float inc, float dec) {
  if (!idx || !perm || !x || !active || C == 0 || S == 0) return -1;
  for (uint64_t i = 0; i < (uint64_t)C * S; ++i)
    if (idx[i] >= n_in) return -1;
  for (uint32_t c = 0; c < C; ++c) {
    if (!active[c]) continue;
    for (uint32_t s = 0; s < S; ++s) {
      const uint64_t e = (uint64_t)c * S + s;
      if (x[idx[e]]) {
        const float up = perm[e] + inc;
        perm[e] = std::fmin(1.0f, up);
      } else {
        const float down = perm[e] - dec;
        perm[e] = std::fmax(0.0f, down);
      }
    }
  }
  return 0;
}

int orc_step(const orc_params* p, const uint32_t* idx, float* perm, const float* boost,
             const uint8_t* x, int learn, int32_t* raw, float* ov, uint8_t* active) {
  if (!p || !active) return -1;
  std::vector<float> ov_local(p->C);
  float* o = ov ? ov : ov_local.data();
  if (orc_overlap(p->C, p->S, idx, perm, boost, p->n_in, x, p->connect_threshold,
                  p->min_overlap, raw, o) != 0)
    return -1;
  int rc;
  if (p->inhibition == 0) {
    rc = orc_inhibit_global(p->C, o, p->winners_set_size, active);
  } else if (p->inhibition == 2) {
    rc = orc_inhibit_paper_literal(p->C, o, p->winners_set_size, active);
  } else {
    if ((uint64_t)p->col_grid_w * p->col_grid_h != p->C) return -1;
    rc = orc_inhibit_local(p->col_grid_w, p->col_grid_h, o, p->winners_set_size,
                           p->local_radius, active);
  }
  if (rc != 0) return rc;
  if (learn) return orc_learn(p->C, p->S, idx, perm, p->n_in, x, active, p->perm_inc,
                              p->perm_dec);
  return 0;
}

int orc_run(const orc_params* p, const uint32_t* idx, float* perm, const float* boost,
            const uint8_t* frames, uint32_t n_frames, int learn, uint8_t* active_out,
            float* ov_out) {
  if (!p || !frames) return -1;
  std::vector<uint8_t> act(p->C);
  for (uint32_t f = 0; f < n_frames; ++f) {
    const uint8_t* x = frames + (uint64_t)f * p->n_in;
    float* ov = ov_out ? ov_out + (uint64_t)f * p->C : nullptr;
    uint8_t* a = active_out ? active_out + (uint64_t)f * p->C : act.data();
    if (orc_step(p, idx, perm, boost, x, learn, nullptr, ov, a) != 0) return -1;
  }
  return 0;
}

int orc_duty_update(uint32_t C, float* duty, const uint8_t* active, float period) {
  if (!duty || !active || C == 0 || !(period > 0.0f)) return -1;
  for (uint32_t c = 0; c < C; ++c) {
    const float a = active[c] ? 1.0f : 0.0f;
    const float diff = a - duty[c];
    const float step = diff / period;
    duty[c] = duty[c] + step;
  }
  return 0;
}

int orc_encode(const uint8_t* src, uint32_t W, uint32_t H, uint32_t channels, uint32_t reduce,
               uint32_t block, int32_t offset, uint8_t* out_bits) {
  if (!src || !out_bits || W == 0 || H == 0) return -1;
  if (channels != 1 && channels != 3) return -1;
  if (reduce == 0 || block < 3 || block > 13 || block % 2 == 0) return -1;
  const uint32_t Wr = W / reduce, Hr = H / reduce;
  if (Wr == 0 || Hr == 0) return -1;
  // 1 + 2. reduction of each channel, then the luma of the reduced pixel
  std::vector<int64_t> gray((size_t)Wr * Hr);
  const uint64_t area = (uint64_t)reduce * reduce;
  for (uint32_t y = 0; y < Hr; ++y) {
    for (uint32_t x = 0; x < Wr; ++x) {
      uint64_t sum[3] = {0, 0, 0};
      for (uint32_t dy = 0; dy < reduce; ++dy)
        for (uint32_t dx = 0; dx < reduce; ++dx) {
          const uint64_t sx = (uint64_t)x * reduce + dx, sy = (uint64_t)y * reduce + dy;
          const uint8_t* px = src + (sy * W + sx) * channels;
          for (uint32_t c = 0; c < channels; ++c) sum[c] += px[c];
        }
      uint64_t mean[3];
      for (uint32_t c = 0; c < channels; ++c) mean[c] = (sum[c] + area / 2) / area;
      gray[(size_t)y * Wr + x] =
          channels == 1 ? (int64_t)mean[0]
                        : (int64_t)((77 * mean[0] + 150 * mean[1] + 29 * mean[2] + 128) >> 8);
    }
  }
  // 3. binomial weights: row B-1 of Pascal's triangle, built by additions
  std::vector<int64_t> w(1, 1);
  for (uint32_t n = 1; n < block; ++n) {
    std::vector<int64_t> next(n + 1);
    for (uint32_t i = 0; i <= n; ++i)
      next[i] = (i > 0 ? w[i - 1] : 0) + (i < n ? w[i] : 0);
    w = next;
  }
  const int64_t half = (int64_t)(block / 2);
  const uint32_t shift = 2 * (block - 1);
  for (uint32_t y = 0; y < Hr; ++y) {
    for (uint32_t x = 0; x < Wr; ++x) {
      int64_t acc = 0;
      for (int64_t dy = -half; dy <= half; ++dy) {
        int64_t yy = (int64_t)y + dy;
        yy = yy < 0 ? 0 : (yy >= (int64_t)Hr ? (int64_t)Hr - 1 : yy);
        for (int64_t dx = -half; dx <= half; ++dx) {
          int64_t xx = (int64_t)x + dx;
          xx = xx < 0 ? 0 : (xx >= (int64_t)Wr ? (int64_t)Wr - 1 : xx);
          acc += w[(size_t)(dy + half)] * w[(size_t)(dx + half)] * gray[(size_t)yy * Wr + xx];
        }
      }
      const int64_t mean = (acc + ((int64_t)1 << (shift - 1))) >> shift;
      out_bits[(size_t)y * Wr + x] = (uint8_t)(gray[(size_t)y * Wr + x] > mean - offset);
    }
  }
  return 0;
}

}  // extern "C"
