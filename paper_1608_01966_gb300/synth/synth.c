/*
 * Seeded synthetic SP inputs: pools, permanences and binary frames.
 * Declarations and the exact recipes are in include/sp_synth.h.
 *
 * No SP arithmetic lives here.  Build with -ffp-contract=off so that the fp32
 * permanence draw and the double Bernoulli draws round identically on every
 * host (GCC contracts a*b+c to FMA by default on aarch64).
 */
#ifndef SP_SYNTH_HIDDEN /* linked privately into the CUDA library */
#define SP_SYNTH_BUILD 1
#endif
#include "../../include/sp_synth.h"

#include <string.h>

uint64_t synth_splitmix64(uint64_t* state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t synth_derive_seed(uint64_t base, uint64_t purpose, uint64_t index) {
  uint64_t s = base ^ (0xD1B54A32D192ED03ULL * (purpose + 1));
  uint64_t a = synth_splitmix64(&s);
  s = a ^ (0x8CB92BA72F3D8DD7ULL * (index + 1));
  return synth_splitmix64(&s);
}

static void sort_u32(uint32_t* a, uint32_t n) {
  /* insertion sort: pools are at most a few thousand entries */
  for (uint32_t i = 1; i < n; ++i) {
    uint32_t v = a[i];
    uint32_t j = i;
    while (j > 0 && a[j - 1] > v) {
      a[j] = a[j - 1];
      --j;
    }
    a[j] = v;
  }
}

/* Draw S distinct entries of cand[0..n) in place (partial Fisher-Yates) and
 * write them sorted to out. */
static void draw_sorted(uint64_t* st, uint32_t* cand, uint32_t n, uint32_t S, uint32_t* out) {
  for (uint32_t i = 0; i < S; ++i) {
    uint64_t r = synth_splitmix64(st);
    uint32_t j = i + (uint32_t)(r % (uint64_t)(n - i));
    uint32_t t = cand[i];
    cand[i] = cand[j];
    cand[j] = t;
    out[i] = cand[i];
  }
  sort_u32(out, S);
}

int synth_pool_uniform(uint64_t seed, uint32_t C, uint32_t S, uint32_t n_in, uint32_t* out_idx,
                       uint32_t* scratch) {
  if (!out_idx || !scratch || C == 0 || S == 0 || n_in == 0 || S > n_in) return -1;
  uint64_t st = seed;
  for (uint32_t c = 0; c < C; ++c) {
    for (uint32_t i = 0; i < n_in; ++i) scratch[i] = i;
    draw_sorted(&st, scratch, n_in, S, out_idx + (uint64_t)c * S);
  }
  return 0;
}

static uint32_t window_origin(uint32_t centre, uint32_t rf, uint32_t extent) {
  int64_t o = (int64_t)centre - (int64_t)(rf / 2);
  if (o + (int64_t)rf > (int64_t)extent) o = (int64_t)extent - (int64_t)rf;
  if (o < 0) o = 0;
  return (uint32_t)o;
}

int synth_pool_window(uint64_t seed, uint32_t gw, uint32_t gh, uint32_t W, uint32_t H,
                      uint32_t rf_w, uint32_t rf_h, uint32_t S, uint32_t* out_idx,
                      uint32_t* scratch) {
  if (!out_idx || !scratch || gw == 0 || gh == 0 || W == 0 || H == 0) return -1;
  if (rf_w == 0 || rf_h == 0 || rf_w > W || rf_h > H) return -1;
  uint32_t n = rf_w * rf_h;
  if (S == 0 || S > n) return -1;
  uint64_t st = seed;
  for (uint32_t j = 0; j < gh; ++j) {
    uint32_t cy = (uint32_t)(((2ULL * j + 1) * H) / (2ULL * gh));
    uint32_t y0 = window_origin(cy, rf_h, H);
    for (uint32_t i = 0; i < gw; ++i) {
      uint32_t cx = (uint32_t)(((2ULL * i + 1) * W) / (2ULL * gw));
      uint32_t x0 = window_origin(cx, rf_w, W);
      uint32_t t = 0;
      for (uint32_t y = 0; y < rf_h; ++y)
        for (uint32_t x = 0; x < rf_w; ++x) scratch[t++] = (y0 + y) * W + (x0 + x);
      uint64_t c = (uint64_t)j * gw + i;
      draw_sorted(&st, scratch, n, S, out_idx + c * S);
    }
  }
  return 0;
}

int synth_pool_dense(uint32_t C, uint32_t n_in, uint32_t* out_idx) {
  if (!out_idx || C == 0 || n_in == 0) return -1;
  for (uint64_t c = 0; c < C; ++c)
    for (uint32_t s = 0; s < n_in; ++s) out_idx[c * n_in + s] = s;
  return 0;
}

int synth_perm_uniform(uint64_t seed, uint64_t n, float lo, float hi, float* out_perm) {
  if (!out_perm || n == 0 || !(lo <= hi)) return -1;
  uint64_t st = seed;
  const float span = hi - lo;
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t r = synth_splitmix64(&st);
    float u = (float)(uint32_t)(r >> 40) * (1.0f / 16777216.0f);
    float t = span * u;
    out_perm[i] = lo + t;
  }
  return 0;
}

int synth_frame_bernoulli(uint64_t seed, uint64_t n, double p, uint8_t* out_bits) {
  if (!out_bits || n == 0 || !(p >= 0.0 && p <= 1.0)) return -1;
  uint64_t st = seed;
  for (uint64_t i = 0; i < n; ++i) {
    double u = (double)(synth_splitmix64(&st) >> 11) * (1.0 / 9007199254740992.0);
    out_bits[i] = (uint8_t)(u < p);
  }
  return 0;
}

int synth_frame_blobbed(uint64_t seed, uint32_t W, uint32_t H, double p_lo, double p_hi,
                        uint8_t* out_bits, uint8_t* scratch, double* out_p) {
  if (!out_bits || !scratch || W == 0 || H == 0) return -1;
  if (!(p_lo >= 0.0 && p_lo <= p_hi && p_hi <= 1.0)) return -1;
  const uint64_t N = (uint64_t)W * H;
  uint64_t st = seed;
  double u0 = (double)(synth_splitmix64(&st) >> 11) * (1.0 / 9007199254740992.0);
  double span = p_hi - p_lo;
  double prod = span * u0;
  double p = p_lo + prod;
  uint8_t* noise = scratch;
  uint8_t* hsum = scratch + N; /* horizontal 7-wide sums, <= 7 */
  uint8_t* pix = out_bits;     /* pixel values, thresholded in place below */
  for (uint64_t i = 0; i < N; ++i) {
    double u = (double)(synth_splitmix64(&st) >> 11) * (1.0 / 9007199254740992.0);
    noise[i] = (uint8_t)(u < p);
  }
  for (uint32_t y = 0; y < H; ++y) {
    const uint8_t* row = noise + (uint64_t)y * W;
    for (uint32_t x = 0; x < W; ++x) {
      uint32_t xa = x >= 3 ? x - 3 : 0;
      uint32_t xb = x + 3 < W ? x + 3 : W - 1;
      uint32_t v = 0;
      for (uint32_t xx = xa; xx <= xb; ++xx) v += row[xx];
      hsum[(uint64_t)y * W + x] = (uint8_t)v;
    }
  }
  uint64_t hist[256];
  memset(hist, 0, sizeof(hist));
  for (uint32_t y = 0; y < H; ++y) {
    uint32_t ya = y >= 3 ? y - 3 : 0;
    uint32_t yb = y + 3 < H ? y + 3 : H - 1;
    for (uint32_t x = 0; x < W; ++x) {
      uint32_t v = 0;
      for (uint32_t yy = ya; yy <= yb; ++yy) v += hsum[(uint64_t)yy * W + x];
      uint8_t q = (uint8_t)((v * 255u + 24u) / 49u);
      pix[(uint64_t)y * W + x] = q;
      hist[q]++;
    }
  }
  /* smallest t with #(pixel > t) <= p * N */
  double budget = p * (double)N;
  uint64_t above = N; /* #(pixel > t) for t = -1 */
  uint32_t t = 255;
  for (uint32_t cand = 0; cand < 256; ++cand) {
    above -= hist[cand];
    if ((double)above <= budget) {
      t = cand;
      break;
    }
  }
  for (uint64_t i = 0; i < N; ++i) out_bits[i] = (uint8_t)(pix[i] > t);
  if (out_p) *out_p = p;
  return 0;
}

int synth_frame_rgb(uint64_t seed, uint32_t W, uint32_t H, uint8_t* out_rgb, uint8_t* scratch) {
  if (!out_rgb || !scratch || W == 0 || H == 0) return -1;
  const uint64_t N = (uint64_t)W * H;
  uint64_t st = seed;
  double u0 = (double)(synth_splitmix64(&st) >> 11) * (1.0 / 9007199254740992.0);
  double p = 0.05 + 0.15 * u0;
  uint32_t gain[3];
  for (int c = 0; c < 3; ++c) gain[c] = 96u + (uint32_t)(synth_splitmix64(&st) % 160u);
  const uint32_t dir = (uint32_t)(synth_splitmix64(&st) & 3u);
  uint8_t* noise = scratch;
  uint8_t* hsum = scratch + N;
  for (uint64_t i = 0; i < N; ++i) {
    double u = (double)(synth_splitmix64(&st) >> 11) * (1.0 / 9007199254740992.0);
    noise[i] = (uint8_t)(u < p);
  }
  for (uint32_t y = 0; y < H; ++y) {
    const uint8_t* row = noise + (uint64_t)y * W;
    for (uint32_t x = 0; x < W; ++x) {
      uint32_t xa = x >= 3 ? x - 3 : 0;
      uint32_t xb = x + 3 < W ? x + 3 : W - 1;
      uint32_t v = 0;
      for (uint32_t xx = xa; xx <= xb; ++xx) v += row[xx];
      hsum[(uint64_t)y * W + x] = (uint8_t)v;
    }
  }
  const uint32_t span = W + H > 2u ? W + H - 2u : 1u;
  for (uint32_t y = 0; y < H; ++y) {
    uint32_t ya = y >= 3 ? y - 3 : 0;
    uint32_t yb = y + 3 < H ? y + 3 : H - 1;
    for (uint32_t x = 0; x < W; ++x) {
      uint32_t v = 0;
      for (uint32_t yy = ya; yy <= yb; ++yy) v += hsum[(uint64_t)yy * W + x];
      const uint32_t field = (v * 255u + 24u) / 49u;
      const uint32_t xs = (dir & 1u) ? W - 1u - x : x;
      const uint32_t ys = (dir & 2u) ? H - 1u - y : y;
      const uint32_t light = 64u + (191u * (xs + ys)) / span;
      uint8_t* px = out_rgb + ((uint64_t)y * W + x) * 3u;
      for (int c = 0; c < 3; ++c) {
        uint32_t lit = (field * gain[c] + 32u) / 64u;
        if (lit > 255u) lit = 255u;
        px[c] = (uint8_t)((lit * light + 127u) / 255u);
      }
    }
  }
  return 0;
}

int synth_pack_bits(const uint8_t* bits, uint64_t n, uint32_t* out_words) {
  if (!bits || !out_words || n == 0) return -1;
  uint64_t nw = (n + 31) / 32;
  for (uint64_t w = 0; w < nw; ++w) out_words[w] = 0;
  for (uint64_t i = 0; i < n; ++i)
    if (bits[i]) out_words[i >> 5] |= 1u << (i & 31);
  return 0;
}
