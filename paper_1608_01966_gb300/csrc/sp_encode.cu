// Frame encoder on the GPU (Section 2 and "Adaptive Video Encoder" in
// Section 3.1): colour frames -> reduction -> gray -> adaptive Gaussian
// threshold -> packed input bits, in one kernel, plus the sp_encoder_* ABI.
//
// One CTA encodes a band of output rows of one frame.  It owns the output
// words whose first pixel lies in the band; the last of them may run into
// the next rows, so the CTA also computes those.  Three phases, all in
// shared memory and all integer arithmetic:
//   A. gray image of the band's rows plus a halo of (block-1)/2 rows above
//      and below (rows outside the image replicate the edge rows), each
//      pixel the luma of its reduced (block-mean) colour;
//   B. vertical binomial sums V of the band's rows, computed for
//      (block-1)/2 extra columns on each side that replicate the edge
//      columns, so phase C needs no clamping;
//   C. one warp per output word: each lane applies the horizontal binomial
//      sum to V at its pixel, rounds the local mean, compares, and the warp
//      ballot is the word; when rows are a whole number of words, a lane
//      takes four adjacent pixels from vector loads of V and eight lanes
//      OR their nibbles into a word.
// The binomial weights C(block-1, i) are compile-time constants of the
// kernel instance (block 3..13).
#include "sp_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>

namespace sp {
extern std::atomic<uint64_t> g_launches;
}

using namespace sp::rt;

namespace {

constexpr int kEncThreads = 512;
constexpr uint32_t kEncChunkFrames = 32;          // frames per encode + SP step
constexpr uint32_t kEncSmemTarget = 100u << 10;   // two CTAs per SM
constexpr uint32_t kEncSmemMax = 200u << 10;
constexpr uint64_t kEncStageBytes = 64ull << 20;  // host path: raw bytes per chunk

__host__ __device__ constexpr uint32_t binom(uint32_t n, uint32_t k) {
  uint64_t r = 1;
  for (uint32_t i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return (uint32_t)r;
}

struct EncodeArgs {
  const uint8_t* src;
  uint64_t src_stride;  // bytes between frames
  uint32_t W, ch, f;    // source width, channels, reduction factor
  uint32_t Wr, Hr;      // output size
  int32_t offset;
  uint32_t* out;
  uint64_t out_stride;  // words between encoded frames
  uint32_t n_words;
  uint32_t band_rows;   // output rows per CTA
  uint32_t g_pitch;     // bytes per gray row in shared memory
  uint32_t g_bytes;     // bytes of the gray area (16-byte multiple)
  uint32_t v_pitch;     // words per V row: >= Wr + block + 2, a multiple of 4
  uint32_t vec4;        // f == 1 and 4-byte aligned rows: four pixels per load
  uint32_t vecf;        // f % 4 == 0 and 4-byte aligned rows: whole words per block row
};

__device__ __forceinline__ uint32_t reduced_gray(const EncodeArgs& a, const uint8_t* fs,
                                                 uint32_t gy, uint32_t x) {
  if (a.f == 1u) {
    const uint8_t* px = fs + ((uint64_t)gy * a.W + x) * a.ch;
    if (a.ch == 1u) return __ldg(px);
    return (77u * __ldg(px) + 150u * __ldg(px + 1) + 29u * __ldg(px + 2) + 128u) >> 8;
  }
  uint32_t s0 = 0, s1 = 0, s2 = 0;
  for (uint32_t dy = 0; dy < a.f; ++dy) {
    const uint8_t* row = fs + ((uint64_t)(gy * a.f + dy) * a.W + (uint64_t)x * a.f) * a.ch;
    for (uint32_t dx = 0; dx < a.f; ++dx) {
      const uint8_t* px = row + dx * a.ch;
      s0 += __ldg(px);
      if (a.ch == 3u) {
        s1 += __ldg(px + 1);
        s2 += __ldg(px + 2);
      }
    }
  }
  const uint32_t area = a.f * a.f, half = area / 2u;
  const uint32_t r = (s0 + half) / area;
  if (a.ch == 1u) return r;
  const uint32_t g = (s1 + half) / area, b = (s2 + half) / area;
  return (77u * r + 150u * g + 29u * b + 128u) >> 8;
}

// reduced_gray for f % 4 == 0 from aligned words: a block row of f pixels is
// 3f/4 words (RGB, repeating every three words) or f/4 words (gray), whose
// channel bytes are summed with byte dot products.
__device__ __forceinline__ uint32_t reduced_gray_words(const EncodeArgs& a, const uint8_t* fs,
                                                       uint32_t gy, uint32_t x) {
  const uint32_t* base = reinterpret_cast<const uint32_t*>(fs);
  const uint32_t wpr = a.W * a.ch / 4u;  // words per source row
  const uint32_t nw = a.f * a.ch / 4u;   // words per block row
  uint32_t s0 = 0, s1 = 0, s2 = 0;
  for (uint32_t dy = 0; dy < a.f; ++dy) {
    const uint32_t* w = base + (uint64_t)(gy * a.f + dy) * wpr + (uint64_t)x * nw;
    if (a.ch == 1u) {
      for (uint32_t m = 0; m < nw; ++m) s0 = __dp4a(__ldg(w + m), 0x01010101u, s0);
    } else {
      for (uint32_t m = 0; m < nw; m += 3) {
        const uint32_t w0 = __ldg(w + m), w1 = __ldg(w + m + 1), w2 = __ldg(w + m + 2);
        s0 = __dp4a(w0, 0x01000001u, __dp4a(w1, 0x00010000u, __dp4a(w2, 0x00000100u, s0)));
        s1 = __dp4a(w0, 0x00000100u, __dp4a(w1, 0x01000001u, __dp4a(w2, 0x00010000u, s1)));
        s2 = __dp4a(w0, 0x00010000u, __dp4a(w1, 0x00000100u, __dp4a(w2, 0x01000001u, s2)));
      }
    }
  }
  const uint32_t area = a.f * a.f, half = area / 2u;
  const uint32_t r = (s0 + half) / area;
  if (a.ch == 1u) return r;
  const uint32_t g = (s1 + half) / area, b = (s2 + half) / area;
  return (77u * r + 150u * g + 29u * b + 128u) >> 8;
}

// Luma of four RGB pixels held in three little-endian words
// (R0 G0 B0 R1 | G1 B1 R2 G2 | B2 R3 G3 B3), packed as four bytes.
__device__ __forceinline__ uint32_t luma4(uint32_t w0, uint32_t w1, uint32_t w2) {
  constexpr uint32_t kW = 77u | (150u << 8) | (29u << 16);  // byte 3 weighs 0
  const uint32_t g0 = __dp4a(w0, kW, 128u) >> 8;
  const uint32_t g1 = __dp4a(__byte_perm(w0, w1, 0x0543), kW, 128u) >> 8;
  const uint32_t g2 = __dp4a(__byte_perm(w1, w2, 0x0432), kW, 128u) >> 8;
  const uint32_t g3 = __dp4a(w2 >> 8, kW, 128u) >> 8;
  return g0 | (g1 << 8) | (g2 << 16) | (g3 << 24);
}

// Binomial-weighted sum of B values v[0..B-1]: the weights are symmetric,
// so pairs are added first and multiplied once (half the multiplies).
template <int B, typename F>
__device__ __forceinline__ uint32_t binomial_sum(F v) {
  constexpr int kHalf = (B - 1) / 2;
  uint32_t s = binom(B - 1, kHalf) * v(kHalf);
#pragma unroll
  for (int j = 0; j < kHalf; ++j) s += binom(B - 1, j) * (v(j) + v(B - 1 - j));
  return s;
}

// Advance a flat position (r, x) over rows of width w by `step` = sr rows + sx.
__device__ __forceinline__ void advance(uint32_t& r, uint32_t& x, uint32_t sr, uint32_t sx,
                                        uint32_t w) {
  r += sr;
  x += sx;
  if (x >= w) {
    x -= w;
    ++r;
  }
}

template <int B>
__global__ void __launch_bounds__(kEncThreads, 2) sp_encode_kernel(const EncodeArgs a) {
  constexpr uint32_t kHalf = (B - 1) / 2;
  constexpr uint32_t kShift = 2 * (B - 1);
  constexpr uint32_t kRowsPerItem = 4;  // phase B: rows of V per work item
  extern __shared__ __align__(16) uint8_t enc_smem[];
  const uint32_t frame = blockIdx.y;
  const uint32_t y0 = blockIdx.x * a.band_rows;
  if (y0 >= a.Hr) return;
  const uint32_t y1 = min(a.Hr, y0 + a.band_rows);
  const uint32_t n_px = a.Wr * a.Hr;
  const uint32_t w_lo = (uint32_t)(((uint64_t)y0 * a.Wr + 31u) >> 5);
  const uint32_t w_hi = min(a.n_words, (uint32_t)(((uint64_t)y1 * a.Wr + 31u) >> 5));
  if (w_lo >= w_hi) return;  // the band's words start in an earlier band
  const uint32_t p_last = min(w_hi * 32u, n_px) - 1u;
  const uint32_t nV = p_last / a.Wr - y0 + 1u;  // rows of V this CTA needs
  const uint32_t nG = nV + 2u * kHalf;
  uint8_t* G = enc_smem;
  uint32_t* V = reinterpret_cast<uint32_t*>(enc_smem + a.g_bytes);
  const uint8_t* fs = a.src + (uint64_t)frame * a.src_stride;
  const uint32_t tid = threadIdx.x;

  // A. gray rows y0 - half .. y0 + nV - 1 + half, edge rows replicated.
  // Items are taken kUnroll at a time with all their loads issued first, so
  // each thread keeps several source words in flight.
  constexpr int kUnroll = 4;
  auto clamp_row = [&](uint32_t r) {
    int gy = (int)y0 - (int)kHalf + (int)r;
    return (uint32_t)(gy < 0 ? 0 : (gy >= (int)a.Hr ? (int)a.Hr - 1 : gy));
  };
  const uint32_t* fw = reinterpret_cast<const uint32_t*>(fs);
  if (a.vec4) {
    // four pixels per item from aligned words (f == 1, W % 4 == 0)
    const uint32_t q = a.Wr >> 2;
    uint32_t r = tid / q, k = tid - r * q;
    const uint32_t sr = kEncThreads / q, sk = kEncThreads - sr * q;
    while (r < nG) {
      uint32_t ru[kUnroll], ku[kUnroll], w0[kUnroll], w1[kUnroll], w2[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        ru[u] = r;
        ku[u] = k;
        advance(r, k, sr, sk, q);
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        w0[u] = w1[u] = w2[u] = 0u;
        if (ru[u] < nG) {
          const uint32_t gy = clamp_row(ru[u]);
          if (a.ch == 3u) {
            const uint32_t* w = fw + (uint64_t)gy * q * 3u + 3u * ku[u];
            w0[u] = __ldg(w);
            w1[u] = __ldg(w + 1);
            w2[u] = __ldg(w + 2);
          } else {
            w0[u] = __ldg(fw + (uint64_t)gy * q + ku[u]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (ru[u] < nG)
          *reinterpret_cast<uint32_t*>(G + ru[u] * a.g_pitch + 4u * ku[u]) =
              a.ch == 3u ? luma4(w0[u], w1[u], w2[u]) : w0[u];
    }
  } else if (a.vecf && a.f == 4u) {
    // 4 x 4 blocks from aligned words: 3 words (RGB) or 1 word (gray) per block row
    const uint32_t wpr = a.W * a.ch / 4u;
    uint32_t r = tid / a.Wr, x = tid - r * a.Wr;
    const uint32_t sr = kEncThreads / a.Wr, sx = kEncThreads - sr * a.Wr;
    constexpr int kU = kUnroll / 2;
    while (r < nG) {
      uint32_t ru[kU], xu[kU], w[kU][12];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        ru[u] = r;
        xu[u] = x;
        advance(r, x, sr, sx, a.Wr);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
#pragma unroll
        for (int m = 0; m < 12; ++m) w[u][m] = 0u;
        if (ru[u] < nG) {
          const uint32_t gy = clamp_row(ru[u]);
          const uint32_t nw = a.ch;  // words per block row: 4 * ch / 4
#pragma unroll
          for (int dy = 0; dy < 4; ++dy) {
            const uint32_t* row = fw + (uint64_t)(gy * 4u + dy) * wpr + (uint64_t)xu[u] * nw;
            w[u][3 * dy] = __ldg(row);
            if (a.ch == 3u) {
              w[u][3 * dy + 1] = __ldg(row + 1);
              w[u][3 * dy + 2] = __ldg(row + 2);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        if (ru[u] >= nG) continue;
        uint32_t gray;
        if (a.ch == 3u) {
          uint32_t s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
          for (int dy = 0; dy < 4; ++dy) {
            const uint32_t q0 = w[u][3 * dy], q1 = w[u][3 * dy + 1], q2 = w[u][3 * dy + 2];
            s0 = __dp4a(q0, 0x01000001u, __dp4a(q1, 0x00010000u, __dp4a(q2, 0x00000100u, s0)));
            s1 = __dp4a(q0, 0x00000100u, __dp4a(q1, 0x01000001u, __dp4a(q2, 0x00010000u, s1)));
            s2 = __dp4a(q0, 0x00010000u, __dp4a(q1, 0x00000100u, __dp4a(q2, 0x01000001u, s2)));
          }
          gray = (77u * ((s0 + 8u) >> 4) + 150u * ((s1 + 8u) >> 4) + 29u * ((s2 + 8u) >> 4) +
                  128u) >> 8;
        } else {
          uint32_t s0 = 0;
#pragma unroll
          for (int dy = 0; dy < 4; ++dy) s0 = __dp4a(w[u][3 * dy], 0x01010101u, s0);
          gray = (s0 + 8u) >> 4;
        }
        G[ru[u] * a.g_pitch + xu[u]] = (uint8_t)gray;
      }
    }
  } else {
    uint32_t r = tid / a.Wr, x = tid - r * a.Wr;
    const uint32_t sr = kEncThreads / a.Wr, sx = kEncThreads - sr * a.Wr;
    for (; r < nG; advance(r, x, sr, sx, a.Wr)) {
      const uint32_t gy = clamp_row(r);
      G[r * a.g_pitch + x] = (uint8_t)(a.vecf ? reduced_gray_words(a, fs, gy, x)
                                               : reduced_gray(a, fs, gy, x));
    }
  }
  __syncthreads();
  // B. vertical sums over B gray rows, for columns -half .. Wr - 1 + half;
  // an item is kRowsPerItem consecutive rows of one column
  {
    const uint32_t vw = a.v_pitch;
    const uint32_t groups = (nV + kRowsPerItem - 1) / kRowsPerItem;
    uint32_t rg = tid / vw, c = tid - rg * vw;
    const uint32_t sr = kEncThreads / vw, sc = kEncThreads - sr * vw;
    for (; rg < groups; advance(rg, c, sr, sc, vw)) {
      int x = (int)c - (int)kHalf;
      x = x < 0 ? 0 : (x >= (int)a.Wr ? (int)a.Wr - 1 : x);
      const uint32_t r0 = rg * kRowsPerItem;
      const uint8_t* col = G + r0 * a.g_pitch + x;
      uint32_t g[kRowsPerItem + B - 1];
#pragma unroll
      for (uint32_t j = 0; j < kRowsPerItem + B - 1; ++j)
        g[j] = r0 + j < nG ? (uint32_t)col[j * a.g_pitch] : 0u;
#pragma unroll
      for (uint32_t t = 0; t < kRowsPerItem; ++t) {
        const uint32_t s = binomial_sum<B>([&](int j) { return g[t + j]; });
        if (r0 + t < nV) V[(r0 + t) * vw + c] = s;
      }
    }
  }
  __syncthreads();
  const uint32_t lane = tid & 31u, warp = tid >> 5;
  constexpr uint32_t kWarps = kEncThreads / 32;
  uint32_t* out = a.out + (uint64_t)frame * a.out_stride;
  if (a.Wr % 32u == 0u) {
    // C'. words are whole row segments: a lane takes four adjacent pixels
    // (vector loads of V), eight lanes make one word
    constexpr uint32_t kVec = (B + 3 + 3) / 4;  // 16-byte loads covering B + 3 columns
    const uint32_t q_row = a.Wr >> 2;
    const uint32_t n_items = (y1 - y0) * q_row;  // a multiple of 8
    uint32_t i = tid;
    uint32_t r = i / q_row, q = i - r * q_row;
    const uint32_t sr = kEncThreads / q_row, sq = kEncThreads - sr * q_row;
    const uint32_t n_round = (n_items + 31u) & ~31u;
    for (; i < n_round; i += kEncThreads, advance(r, q, sr, sq, q_row)) {
      uint32_t m = 0;
      if (i < n_items) {
        const uint4* vr = reinterpret_cast<const uint4*>(V + r * a.v_pitch + 4u * q);
        uint32_t v[4 * kVec];
#pragma unroll
        for (uint32_t k = 0; k < kVec; ++k) {
          const uint4 t = vr[k];
          v[4 * k] = t.x;
          v[4 * k + 1] = t.y;
          v[4 * k + 2] = t.z;
          v[4 * k + 3] = t.w;
        }
        const uint32_t g4 = *reinterpret_cast<const uint32_t*>(G + (r + kHalf) * a.g_pitch + 4u * q);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t s = binomial_sum<B>([&](int j) { return v[t + j]; });
          const uint32_t mean = (s + (1u << (kShift - 1))) >> kShift;
          const int g = (int)((g4 >> (8 * t)) & 255u);
          m |= (g + a.offset > (int)mean ? 1u : 0u) << t;
        }
      }
      uint32_t word = m << (4u * (lane & 7u));
      word |= __shfl_xor_sync(0xffffffffu, word, 1);
      word |= __shfl_xor_sync(0xffffffffu, word, 2);
      word |= __shfl_xor_sync(0xffffffffu, word, 4);
      if ((lane & 7u) == 0u && i < n_items) out[w_lo + i / 8u] = word;
    }
    return;
  }
  // C. one warp per owned word; (y, x) of each lane's pixel kept incrementally
  uint32_t w = w_lo + warp;
  uint32_t p = w * 32u + lane;
  uint32_t y = p / a.Wr, x = p - y * a.Wr;
  const uint32_t sy = (kWarps * 32u) / a.Wr, sx = kWarps * 32u - sy * a.Wr;
  for (; w < w_hi; w += kWarps, p += kWarps * 32u, advance(y, x, sy, sx, a.Wr)) {
    bool bit = false;
    if (p < n_px) {
      const uint32_t r = y - y0;
      const uint32_t* vr = V + r * a.v_pitch + x;  // vr[i] is column x + i - half
      const uint32_t s = binomial_sum<B>([&](int i) { return vr[i]; });
      const uint32_t mean = (s + (1u << (kShift - 1))) >> kShift;
      const int g = (int)G[(r + kHalf) * a.g_pitch + x];
      bit = g + a.offset > (int)mean;
    }
    const uint32_t m = __ballot_sync(0xffffffffu, bit);
    if (lane == 0) out[w] = m;
  }
}

struct EncPlan {
  uint32_t Wr = 0, Hr = 0, n_words = 0;
  uint64_t src_bytes = 0;
  uint32_t band_rows = 0, g_pitch = 0, g_bytes = 0, v_pitch = 0, smem = 0;
};

uint32_t plan_smem(const sp_encoder_config& c, uint32_t Wr, uint32_t th, uint32_t* g_pitch,
                   uint32_t* g_bytes, uint32_t* v_pitch) {
  const uint32_t half = (c.block - 1) / 2;
  const uint32_t v_rows = th + 1u + 30u / Wr;  // owned words reach at most 31 pixels past
  const uint32_t g_rows = v_rows + 2u * half;
  *g_pitch = (Wr + 3u) & ~3u;
  *g_bytes = (g_rows * *g_pitch + 15u) & ~15u;
  *v_pitch = (Wr + c.block + 2u + 3u) & ~3u;  // 16-byte rows; the vector loads of
                                             // four pixels read up to Wr + block + 1
  return *g_bytes + v_rows * *v_pitch * 4u;
}

sp_status validate_encoder(const sp_encoder_config* c, EncPlan* p) {
  if (!c) return fail(SP_EINVAL, "NULL encoder config");
  if (c->src_w == 0 || c->src_h == 0 || c->src_w > 65535u || c->src_h > 65535u)
    return fail(SP_EINVAL, "source size %ux%u outside 1..65535", c->src_w, c->src_h);
  if (c->channels != 1 && c->channels != 3)
    return fail(SP_EINVAL, "channels %u (1 or 3)", c->channels);
  if (c->reduce < 1 || c->reduce > 8) return fail(SP_EINVAL, "reduce %u outside 1..8", c->reduce);
  if (c->block < 3 || c->block > 13 || c->block % 2 == 0)
    return fail(SP_EINVAL, "block %u (odd, 3..13)", c->block);
  if (c->reserved[0] || c->reserved[1]) return fail(SP_EINVAL, "reserved fields must be zero");
  const uint32_t Wr = c->src_w / c->reduce, Hr = c->src_h / c->reduce;
  if (Wr == 0 || Hr == 0) return fail(SP_EINVAL, "reduction leaves an empty frame");
  if ((uint64_t)Wr * Hr >= (1ull << 31)) return fail(SP_EINVAL, "output frame too large");
  p->Wr = Wr;
  p->Hr = Hr;
  p->n_words = (uint32_t)(((uint64_t)Wr * Hr + 31u) / 32u);
  p->src_bytes = (uint64_t)c->src_w * c->src_h * c->channels;
  uint32_t th = 32;
  for (; th > 1; th /= 2)
    if (plan_smem(*c, Wr, th, &p->g_pitch, &p->g_bytes, &p->v_pitch) <= kEncSmemTarget) break;
  p->smem = plan_smem(*c, Wr, th, &p->g_pitch, &p->g_bytes, &p->v_pitch);
  if (p->smem > kEncSmemMax) return fail(SP_EINVAL, "output width %u too large", Wr);
  p->band_rows = std::min(th, Hr);
  return SP_OK;
}

// Allow every kernel instance the planned shared memory on the current device.
cudaError_t encode_kernels_init() {
  cudaError_t e = cudaSuccess;
  const int bytes = (int)kEncSmemMax;
  auto set = [&](const void* k) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  set((const void*)sp_encode_kernel<3>);
  set((const void*)sp_encode_kernel<5>);
  set((const void*)sp_encode_kernel<7>);
  set((const void*)sp_encode_kernel<9>);
  set((const void*)sp_encode_kernel<11>);
  set((const void*)sp_encode_kernel<13>);
  return e;
}

template <int B>
cudaError_t launch_encode_b(const EncodeArgs& a, uint32_t bands, uint32_t n, uint32_t smem,
                            cudaStream_t st) {
  sp_encode_kernel<B><<<dim3(bands, n), kEncThreads, smem, st>>>(a);
  sp::g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace

struct sp_encoder {
  sp_encoder_config cfg{};
  EncPlan plan;
  int device = 0;
  uint32_t timeout_ms = 10000;
  cudaStream_t stream = nullptr, s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_h2d[kSlots] = {}, ev_comp[kSlots] = {}, ev_d2h[kSlots] = {}, ev_tail = nullptr;
  uint32_t* d_bits = nullptr;  // kEncChunkFrames encoded frames
  uint8_t* d_raw = nullptr;    // host path: [kSlots][chunk][src_bytes]
  uint32_t raw_chunk = 0;
  uint32_t* d_masks = nullptr;  // host path: [kSlots][kEncChunkFrames][mask_words]
  uint32_t mask_words = 0;
};

namespace {

void free_encoder(sp_encoder* e) {
  if (!e) return;
  DeviceGuard g(e->device);
  if (e->stream) cudaStreamSynchronize(e->stream);
  if (e->s_in) cudaStreamSynchronize(e->s_in);
  if (e->s_out) cudaStreamSynchronize(e->s_out);
  for (int i = 0; i < kSlots; ++i) {
    if (e->ev_h2d[i]) cudaEventDestroy(e->ev_h2d[i]);
    if (e->ev_comp[i]) cudaEventDestroy(e->ev_comp[i]);
    if (e->ev_d2h[i]) cudaEventDestroy(e->ev_d2h[i]);
  }
  if (e->ev_tail) cudaEventDestroy(e->ev_tail);
  if (e->d_bits) cudaFree(e->d_bits);
  if (e->d_raw) cudaFree(e->d_raw);
  if (e->d_masks) cudaFree(e->d_masks);
  if (e->stream) cudaStreamDestroy(e->stream);
  if (e->s_in) cudaStreamDestroy(e->s_in);
  if (e->s_out) cudaStreamDestroy(e->s_out);
  delete e;
}

sp_status enqueue_encode(sp_encoder* e, const uint8_t* d_src, uint32_t n, uint64_t src_stride,
                         uint32_t* d_bits, uint64_t bits_stride, cudaStream_t st) {
  const EncPlan& p = e->plan;
  EncodeArgs a{};
  a.W = e->cfg.src_w;
  a.ch = e->cfg.channels;
  a.f = e->cfg.reduce;
  a.Wr = p.Wr;
  a.Hr = p.Hr;
  a.offset = e->cfg.offset;
  a.n_words = p.n_words;
  a.band_rows = p.band_rows;
  a.g_pitch = p.g_pitch;
  a.g_bytes = p.g_bytes;
  a.v_pitch = p.v_pitch;
  a.src_stride = src_stride;
  a.out_stride = bits_stride;
  a.vec4 = (e->cfg.reduce == 1 && e->cfg.src_w % 4 == 0 && src_stride % 4 == 0 &&
            reinterpret_cast<uintptr_t>(d_src) % 4 == 0) ? 1u : 0u;
  a.vecf = (e->cfg.reduce % 4 == 0 && e->cfg.src_w % 4 == 0 && src_stride % 4 == 0 &&
            reinterpret_cast<uintptr_t>(d_src) % 4 == 0) ? 1u : 0u;
  const uint32_t bands = (p.Hr + p.band_rows - 1) / p.band_rows;
  for (uint32_t f0 = 0; f0 < n; f0 += 65535u) {
    const uint32_t nf = std::min(n - f0, 65535u);
    a.src = d_src + (uint64_t)f0 * src_stride;
    a.out = d_bits + (uint64_t)f0 * bits_stride;
    cudaError_t err;
    switch (e->cfg.block) {
      case 3: err = launch_encode_b<3>(a, bands, nf, p.smem, st); break;
      case 5: err = launch_encode_b<5>(a, bands, nf, p.smem, st); break;
      case 7: err = launch_encode_b<7>(a, bands, nf, p.smem, st); break;
      case 9: err = launch_encode_b<9>(a, bands, nf, p.smem, st); break;
      case 11: err = launch_encode_b<11>(a, bands, nf, p.smem, st); break;
      default: err = launch_encode_b<13>(a, bands, nf, p.smem, st); break;
    }
    SP_CUDA(err);
  }
  return SP_OK;
}

cudaStream_t pick_stream(sp_encoder* e, void* stream) {
  return stream ? static_cast<cudaStream_t>(stream) : e->stream;
}

sp_status check_handle(sp_encoder* e, sp_handle* h, uint32_t* mask_words) {
  sp_info info{};
  const sp_status s = sp_get_info(h, &info);
  if (s != SP_OK) return s;
  if (info.input_bits != (uint64_t)e->plan.Wr * e->plan.Hr)
    return fail(SP_EINVAL, "the SP takes %llu input bits, the encoder makes %ux%u",
                (unsigned long long)info.input_bits, e->plan.Wr, e->plan.Hr);
  if (info.device != e->device) return fail(SP_EINVAL, "encoder and SP on different devices");
  *mask_words = info.mask_words;
  return SP_OK;
}

sp_status ensure_bits(sp_encoder* e) {
  if (!e->d_bits)
    SP_CUDA(device_malloc((void**)&e->d_bits, (size_t)kEncChunkFrames * e->plan.n_words * 4));
  return SP_OK;
}

}  // namespace

SP_API sp_status sp_encoder_config_init(sp_encoder_config* cfg) {
  if (!cfg) return fail(SP_EINVAL, "NULL argument");
  *cfg = sp_encoder_config{};
  cfg->src_w = 960;
  cfg->src_h = 540;
  cfg->channels = 3;
  cfg->reduce = 1;
  cfg->block = 11;
  cfg->offset = 2;
  return SP_OK;
}

SP_API sp_status sp_encoder_create(const sp_encoder_config* cfg, sp_encoder** out) {
  if (!out) return fail(SP_EINVAL, "NULL argument");
  *out = nullptr;
  EncPlan plan;
  sp_status s = validate_encoder(cfg, &plan);
  if (s != SP_OK) return s;
  sp_encoder* e = new sp_encoder();
  e->cfg = *cfg;
  e->plan = plan;
  e->timeout_ms = default_timeout_ms();
  cudaError_t err = cudaGetDevice(&e->device);
  if (err == cudaSuccess) err = encode_kernels_init();
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
  if (err != cudaSuccess) {
    free_encoder(e);
    return fail(SP_ECUDA, "encoder set-up: %s", cudaGetErrorString(err));
  }
  *out = e;
  return SP_OK;
}

SP_API void sp_encoder_destroy(sp_encoder* e) { free_encoder(e); }

SP_API sp_status sp_encoder_get_info(const sp_encoder* e, sp_encoder_info* out) {
  if (!e || !out) return fail(SP_EINVAL, "NULL argument");
  out->out_w = e->plan.Wr;
  out->out_h = e->plan.Hr;
  out->out_bits = (uint64_t)e->plan.Wr * e->plan.Hr;
  out->out_words = e->plan.n_words;
  out->src_bytes = e->plan.src_bytes;
  return SP_OK;
}

SP_API sp_status sp_encode_device(sp_encoder* e, const uint8_t* d_src, uint32_t n_frames,
                                  uint64_t src_stride, uint32_t* d_bits, uint64_t bits_stride,
                                  void* stream) {
  if (!e || ((!d_src || !d_bits) && n_frames)) return fail(SP_EINVAL, "NULL argument");
  if (n_frames == 0) return SP_OK;
  if (src_stride < e->plan.src_bytes) return fail(SP_EINVAL, "source stride below the frame size");
  if (bits_stride < e->plan.n_words) return fail(SP_EINVAL, "bit stride below %u words", e->plan.n_words);
  if (reinterpret_cast<uintptr_t>(d_bits) % 4u) return fail(SP_EINVAL, "d_bits not 4-byte aligned");
  DeviceGuard g(e->device);
  return enqueue_encode(e, d_src, n_frames, src_stride, d_bits, bits_stride, pick_stream(e, stream));
}

SP_API sp_status sp_encode_compute_device(sp_encoder* e, sp_handle* h, const uint8_t* d_src,
                                          uint32_t n_frames, uint64_t src_stride, int learn,
                                          uint32_t* d_active_masks, void* stream) {
  if (!e || !h || (!d_src && n_frames)) return fail(SP_EINVAL, "NULL argument");
  if (n_frames == 0) return SP_OK;
  if (src_stride < e->plan.src_bytes) return fail(SP_EINVAL, "source stride below the frame size");
  if (reinterpret_cast<uintptr_t>(d_active_masks) % 4u)
    return fail(SP_EINVAL, "d_active_masks not 4-byte aligned");
  uint32_t mw = 0;
  sp_status s = check_handle(e, h, &mw);
  if (s != SP_OK) return s;
  DeviceGuard g(e->device);
  s = ensure_bits(e);
  if (s != SP_OK) return s;
  cudaStream_t st = pick_stream(e, stream);
  for (uint32_t f0 = 0; f0 < n_frames; f0 += kEncChunkFrames) {
    const uint32_t nf = std::min(n_frames - f0, kEncChunkFrames);
    s = enqueue_encode(e, d_src + (uint64_t)f0 * src_stride, nf, src_stride, e->d_bits,
                       e->plan.n_words, st);
    if (s != SP_OK) return s;
    s = sp_compute_frames_device(h, e->d_bits, nf, e->plan.n_words, learn,
                                 d_active_masks ? d_active_masks + (uint64_t)f0 * mw : nullptr, st);
    if (s != SP_OK) return s;
  }
  return SP_OK;
}

SP_API sp_status sp_encode_compute(sp_encoder* e, sp_handle* h, const uint8_t* h_src,
                                   uint32_t n_frames, int learn, uint32_t* h_active_masks) {
  if (!e || !h || (!h_src && n_frames)) return fail(SP_EINVAL, "NULL argument");
  if (n_frames == 0) return SP_OK;
  uint32_t mw = 0;
  sp_status s = check_handle(e, h, &mw);
  if (s != SP_OK) return s;
  DeviceGuard g(e->device);
  s = ensure_bits(e);
  if (s != SP_OK) return s;
  const uint64_t fb = e->plan.src_bytes;
  if (!e->d_raw) {
    e->raw_chunk = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(kEncChunkFrames, kEncStageBytes / fb));
    SP_CUDA(device_malloc((void**)&e->d_raw, (size_t)kSlots * e->raw_chunk * fb));
    SP_CUDA(cudaStreamCreateWithFlags(&e->s_in, cudaStreamNonBlocking));
    SP_CUDA(cudaStreamCreateWithFlags(&e->s_out, cudaStreamNonBlocking));
    SP_CUDA(cudaEventCreateWithFlags(&e->ev_tail, cudaEventDisableTiming));
    for (int i = 0; i < kSlots; ++i) {
      SP_CUDA(cudaEventCreateWithFlags(&e->ev_h2d[i], cudaEventDisableTiming));
      SP_CUDA(cudaEventCreateWithFlags(&e->ev_comp[i], cudaEventDisableTiming));
      SP_CUDA(cudaEventCreateWithFlags(&e->ev_d2h[i], cudaEventDisableTiming));
      SP_CUDA(cudaEventRecord(e->ev_comp[i], e->stream));
      SP_CUDA(cudaEventRecord(e->ev_d2h[i], e->stream));
    }
  }
  if (h_active_masks && mw > e->mask_words) {
    if (e->d_masks) {
      SP_CUDA(cudaStreamSynchronize(e->s_out));
      cudaFree(e->d_masks);
      e->d_masks = nullptr;
    }
    SP_CUDA(device_malloc((void**)&e->d_masks, (size_t)kSlots * e->raw_chunk * mw * 4));
    e->mask_words = mw;
  }
  const uint32_t chunk = e->raw_chunk;
  for (uint32_t f0 = 0, ci = 0; f0 < n_frames; f0 += chunk, ++ci) {
    const int slot = (int)(ci % kSlots);
    const uint32_t nf = std::min(n_frames - f0, chunk);
    uint8_t* raw = e->d_raw + (size_t)slot * chunk * fb;
    uint32_t* masks = h_active_masks ? e->d_masks + (size_t)slot * chunk * mw : nullptr;
    // copy in once the work that read this slot two chunks ago is done
    SP_CUDA(cudaStreamWaitEvent(e->s_in, e->ev_comp[slot], 0));
    SP_CUDA(cudaMemcpyAsync(raw, h_src + (uint64_t)f0 * fb, (size_t)nf * fb,
                            cudaMemcpyHostToDevice, e->s_in));
    SP_CUDA(cudaEventRecord(e->ev_h2d[slot], e->s_in));
    SP_CUDA(cudaStreamWaitEvent(e->stream, e->ev_h2d[slot], 0));
    SP_CUDA(cudaStreamWaitEvent(e->stream, e->ev_d2h[slot], 0));
    s = sp_encode_compute_device(e, h, raw, nf, fb, learn, masks, e->stream);
    if (s != SP_OK) return s;
    SP_CUDA(cudaEventRecord(e->ev_comp[slot], e->stream));
    if (h_active_masks) {
      SP_CUDA(cudaStreamWaitEvent(e->s_out, e->ev_comp[slot], 0));
      SP_CUDA(cudaMemcpyAsync(h_active_masks + (uint64_t)f0 * mw, masks, (size_t)nf * mw * 4,
                              cudaMemcpyDeviceToHost, e->s_out));
      SP_CUDA(cudaEventRecord(e->ev_d2h[slot], e->s_out));
    }
  }
  // the SP's stream (now the encoder's) waits for the last copy out, so the
  // handle's bounded wait covers everything
  SP_CUDA(cudaEventRecord(e->ev_tail, e->s_out));
  SP_CUDA(cudaStreamWaitEvent(e->stream, e->ev_tail, 0));
  return sp_sync(h);
}
