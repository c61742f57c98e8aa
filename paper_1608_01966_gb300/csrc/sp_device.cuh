// Device helpers shared by the Spatial Pooler kernels: the per-synapse steps
// of Alg. 1 and the learning rule, block-wide scans, and the pieces of
// Alg. 2 (threshold select over overlaps, ordered winner output).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sp {
namespace dev {

constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t input_bit(const uint32_t* __restrict__ x, uint32_t i) {
  return (__ldg(x + (i >> 5)) >> (i & 31u)) & 1u;
}

// Section 1.1 learning of one synapse: one fp32 round-to-nearest add or
// subtract, then the clamp to [0, 1].
__device__ __forceinline__ float learn_one(float p, uint32_t bit, float inc, float dec) {
  return bit ? fminf(1.0f, __fadd_rn(p, inc)) : fmaxf(0.0f, __fsub_rn(p, dec));
}

// Alg. 1 tail: zero below min_overlap, else one fp32 multiply by the boost.
__device__ __forceinline__ float boosted(uint32_t raw, uint32_t min_overlap, float boost) {
  return raw < min_overlap ? 0.0f : __fmul_rn(__uint2float_rn(raw), boost);
}

// Exclusive block-wide prefix sums of two per-thread counters, plus totals.
// Every thread of the block must call it.  sh holds 2 * NW words.
template <int NW>
__device__ __forceinline__ void block_scan2(uint32_t va, uint32_t vb, uint32_t& ex_a,
                                            uint32_t& ex_b, uint32_t& tot_a, uint32_t& tot_b,
                                            uint32_t* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t ia = va, ib = vb;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t ta = __shfl_up_sync(kFull, ia, o);
    const uint32_t tb = __shfl_up_sync(kFull, ib, o);
    if (lane >= o) {
      ia += ta;
      ib += tb;
    }
  }
  if (lane == 31) {
    sh[warp] = ia;
    sh[NW + warp] = ib;
  }
  __syncthreads();
  uint32_t wa = 0, wb = 0, sa = 0, sb = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint32_t xa = sh[w], xb = sh[NW + w];
    if (w < warp) {
      wa += xa;
      wb += xb;
    }
    sa += xa;
    sb += xb;
  }
  ex_a = wa + ia - va;
  ex_b = wb + ib - vb;
  tot_a = sa;
  tot_b = sb;
  __syncthreads();
}

// hist[bin] += 1 for every lane with `active`, one shared-memory atomic per
// distinct bin in the warp.  All 32 lanes must call it.
__device__ __forceinline__ void warp_hist_add(uint32_t* hist, uint32_t bin, bool active) {
  const uint32_t key = active ? bin : 0xffffffffu;
  const uint32_t peers = __match_any_sync(kFull, key);
  const int lane = threadIdx.x & 31;
  if (active && lane == __ffs(peers) - 1) atomicAdd(hist + bin, (uint32_t)__popc(peers));
}

// Threshold of global inhibition over C overlaps (fp32 bit patterns in sv,
// all >= 0): the winners are every v > T plus the first `need` columns (by
// index) with v == T.  nz_tot = number of nonzero overlaps.  Three ways to
// find the k-th largest value, all exact:
//   ghist != nullptr : a histogram of the raw counts (unit boosts, so the
//                      overlap is the count) already built in global memory,
//                      bins 0..unit_S;
//   unit_S != 0      : the same histogram built here from sv (unit boosts);
//   otherwise        : radix select over the 32-bit patterns, 8 bits a pass.
// shist must hold max(256, unit_S + 1) words; sh 2 * NW words; s2 2 words.
// Every thread of the block must call it.
template <int NTHREADS>
__device__ void select_threshold(const uint32_t* sv, uint32_t C, uint32_t k, uint32_t nz_tot,
                                 const uint32_t* ghist, uint32_t unit_S, uint32_t* shist,
                                 uint32_t* sh, uint32_t* s2, uint32_t& T, uint32_t& need) {
  constexpr int NW = NTHREADS / 32;
  const uint32_t t = threadIdx.x;
  if (k == 0u) {
    T = 0xffffffffu;  // no overlap exceeds it (finite patterns are < 0x7f800000)
    need = 0u;
    return;
  }
  if (nz_tot <= k) {
    T = 0u;  // every nonzero column wins
    need = 0u;
    return;
  }
  if (ghist || unit_S) {
    const uint32_t nb = unit_S;  // bins 1..S hold the counts
    if (!ghist) {
      for (uint32_t b = t; b <= nb; b += NTHREADS) shist[b] = 0u;
      __syncthreads();
      const uint32_t rounds = (C + NTHREADS - 1) / NTHREADS;
      for (uint32_t r = 0; r < rounds; ++r) {
        const uint32_t i = r * NTHREADS + t;
        const uint32_t v = i < C ? sv[i] : 0u;
        // unit boosts: the overlap is an exact small integer
        warp_hist_add(shist, (uint32_t)__uint_as_float(v), v != 0u);
      }
      __syncthreads();
    }
    const uint32_t* H = ghist ? ghist : shist;
    // thread t owns bins top = nb - t*pb down to top - cnt + 1 (descending)
    const uint32_t pb = (nb + NTHREADS - 1) / NTHREADS;
    const uint32_t top = nb >= t * pb ? nb - t * pb : 0u;
    const uint32_t cnt_bins = top == 0u ? 0u : min(pb, top);
    uint32_t mine = 0;
    for (uint32_t b = 0; b < cnt_bins; ++b) mine += ghist ? __ldcg(H + (top - b)) : H[top - b];
    uint32_t above, e1, tot, z;
    block_scan2<NW>(mine, 0u, above, e1, tot, z, sh);
    if (above < k && above + mine >= k) {
      uint32_t acc = above;
      for (uint32_t b = 0; b < cnt_bins; ++b) {
        const uint32_t hb = ghist ? __ldcg(H + (top - b)) : H[top - b];
        if (acc + hb >= k) {
          s2[0] = top - b;  // the k-th largest count
          s2[1] = acc;      // columns strictly above it
          break;
        }
        acc += hb;
      }
    }
    __syncthreads();
    T = __float_as_uint(__uint2float_rn(s2[0]));
    need = k - s2[1];
    __syncthreads();
    return;
  }
  // radix select, most significant byte first
  uint32_t prefix = 0u, pmask = 0u, kk = k;
  const uint32_t rounds = (C + NTHREADS - 1) / NTHREADS;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (uint32_t i = t; i < 256u; i += NTHREADS) shist[i] = 0u;
    __syncthreads();
    for (uint32_t r = 0; r < rounds; ++r) {
      const uint32_t i = r * NTHREADS + t;
      const uint32_t v = i < C ? sv[i] : 0u;
      warp_hist_add(shist, (v >> shift) & 255u, v != 0u && (v & pmask) == prefix);
    }
    __syncthreads();
    if (t < 32u) {
      // lane L scans digits 255-8L .. 248-8L (descending)
      uint32_t loc[8], sum = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        loc[j] = shist[255u - 8u * t - j];
        sum += loc[j];
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if ((int)t >= o) incl += y;
      }
      uint32_t above = incl - sum;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (above < kk && above + loc[j] >= kk) {
          s2[0] = 255u - 8u * t - j;
          s2[1] = above;
        }
        above += loc[j];
      }
    }
    __syncthreads();
    prefix |= s2[0] << shift;
    pmask |= 0xffu << shift;
    kk -= s2[1];
    __syncthreads();
  }
  T = prefix;  // the k-th largest overlap (bit pattern)
  need = kk;   // how many columns equal to T still win
}

// The k-th largest of the C overlap patterns in sv, repeats and zeros
// included (0 when k is 0 or larger than C): radix select over all values.
// shist holds 256 words; sh 2 * NW; s2 2.  Every thread must call it.
template <int NTHREADS>
__device__ uint32_t kth_largest(const uint32_t* sv, uint32_t C, uint32_t k, uint32_t* shist,
                                uint32_t* s2) {
  const uint32_t t = threadIdx.x;
  if (k == 0u || k > C) return 0u;
  uint32_t prefix = 0u, pmask = 0u, kk = k;
  const uint32_t rounds = (C + NTHREADS - 1) / NTHREADS;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (uint32_t i = t; i < 256u; i += NTHREADS) shist[i] = 0u;
    __syncthreads();
    for (uint32_t r = 0; r < rounds; ++r) {
      const uint32_t i = r * NTHREADS + t;
      const uint32_t v = i < C ? sv[i] : 0u;
      warp_hist_add(shist, (v >> shift) & 255u, i < C && (v & pmask) == prefix);
    }
    __syncthreads();
    if (t < 32u) {
      uint32_t loc[8], sum = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        loc[j] = shist[255u - 8u * t - j];
        sum += loc[j];
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if ((int)t >= o) incl += y;
      }
      uint32_t above = incl - sum;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (above < kk && above + loc[j] >= kk) {
          s2[0] = 255u - 8u * t - j;
          s2[1] = above;
        }
        above += loc[j];
      }
    }
    __syncthreads();
    prefix |= s2[0] << shift;
    pmask |= 0xffu << shift;
    kk -= s2[1];
    __syncthreads();
  }
  return prefix;
}

// Alg. 2 taken word for word (the paper-literal variant, for comparison):
// column c is active iff ov > max(n-th largest overlap of the other columns,
// 1), n = k.  With w_j the j-th largest of all overlaps, the n-th largest of
// the others is w_{k+1} when ov >= w_k and w_k otherwise (0 when fewer than
// k others exist), so c is active iff ov > 1 and, when k < C, ov >= w_k and
// ov > w_{k+1}.  Sets smask bits; writes the ascending list if list is set.
template <int NTHREADS>
__device__ uint32_t mark_paper_literal(const uint32_t* sv, uint32_t C, uint32_t k,
                                       uint32_t* smask, uint32_t* list, uint32_t* shist,
                                       uint32_t* sh, uint32_t* s2) {
  constexpr int NW = NTHREADS / 32;
  const uint32_t wk = kth_largest<NTHREADS>(sv, C, k, shist, s2);
  const uint32_t wk1 = kth_largest<NTHREADS>(sv, C, k + 1u, shist, s2);
  const uint32_t one = __float_as_uint(1.0f);
  const uint32_t t = threadIdx.x;
  const uint32_t per = (C + NTHREADS - 1) / NTHREADS;
  const uint32_t lo = min(C, t * per), hi = min(C, lo + per);
  uint32_t wins = 0;
  for (uint32_t i = lo; i < hi; ++i) {
    const uint32_t v = sv[i];
    // k = 0 or k >= C: no n-th largest among the others, the floor 1 decides
    const bool w = v > one && ((k == 0u || k >= C) || (v >= wk && v > wk1));
    if (w) {
      ++wins;
      atomicOr(smask + (i >> 5), 1u << (i & 31u));
    }
  }
  uint32_t ex, e1, tot, z;
  block_scan2<NW>(wins, 0u, ex, e1, tot, z, sh);
  if (list) {
    uint32_t pos = ex;
    for (uint32_t i = lo; i < hi; ++i)
      if ((smask[i >> 5] >> (i & 31u)) & 1u) list[pos++] = i;
  }
  return tot;
}

// Winner flags of global inhibition for all C columns, given (T, need):
// sets bits of smask (zeroed by the caller) and, if list != nullptr, writes
// the ascending winner list there.  Returns the number of winners.
template <int NTHREADS>
__device__ uint32_t mark_global(const uint32_t* sv, uint32_t C, uint32_t T, uint32_t need,
                                uint32_t* smask, uint32_t* list, uint32_t* sh) {
  constexpr int NW = NTHREADS / 32;
  const uint32_t t = threadIdx.x;
  const uint32_t per = (C + NTHREADS - 1) / NTHREADS;  // contiguous chunks keep index order
  const uint32_t lo = min(C, t * per), hi = min(C, lo + per);
  uint32_t gt = 0, eq = 0;
  for (uint32_t i = lo; i < hi; ++i) {
    const uint32_t v = sv[i];
    gt += v > T;
    eq += (need != 0u) & (v == T);
  }
  uint32_t gt_ex, eq_ex, gt_tot, eq_tot;
  block_scan2<NW>(gt, eq, gt_ex, eq_ex, gt_tot, eq_tot, sh);
  uint32_t pos = gt_ex + min(eq_ex, need);
  uint32_t e = eq_ex;
  for (uint32_t i = lo; i < hi; ++i) {
    const uint32_t v = sv[i];
    bool w = v > T;
    if (!w && need != 0u && v == T) {
      w = e < need;
      ++e;
    }
    if (w) {
      if (list) list[pos] = i;
      ++pos;
      atomicOr(smask + (i >> 5), 1u << (i & 31u));
    }
  }
  return gt_tot + min(eq_tot, need);
}

// Does column c win its clipped (2r+1)^2 neighbourhood?  sv holds the fp32
// bit patterns of all overlaps (>= 0, so integer order = value order).
__device__ __forceinline__ bool local_winner(const uint32_t* sv, uint32_t c, uint32_t gw,
                                             uint32_t gh, uint32_t r, uint32_t k) {
  const uint32_t vc = sv[c];
  if (vc == 0u || k == 0u) return false;
  const uint32_t i = c % gw, j = c / gw;
  const uint32_t i0 = i >= r ? i - r : 0u, i1 = min(gw - 1u, i + r);
  const uint32_t j0 = j >= r ? j - r : 0u, j1 = min(gh - 1u, j + r);
  uint32_t beaten_by = 0;
  for (uint32_t jj = j0; jj <= j1; ++jj) {
    const uint32_t row = jj * gw;
    for (uint32_t ii = i0; ii <= i1; ++ii) {
      const uint32_t d = row + ii;
      const uint32_t vd = sv[d];
      beaten_by += (vd > vc) | ((vd == vc) & (d < c));
    }
    if (beaten_by >= k) return false;
  }
  return beaten_by < k;
}

// Winner flags of local inhibition for columns [c_lo, c_hi) (sv must hold
// every overlap those windows reach): sets smask bits; writes the ascending
// list of these winners to list (if not nullptr).  Returns their number.
template <int NTHREADS>
__device__ uint32_t mark_local(const uint32_t* sv, uint32_t c_lo, uint32_t c_hi, uint32_t gw,
                               uint32_t gh, uint32_t r, uint32_t k, uint32_t* smask,
                               uint32_t* list, uint32_t* sh) {
  constexpr int NW = NTHREADS / 32;
  const uint32_t t = threadIdx.x;
  const uint32_t n = c_hi - c_lo;
  const uint32_t per = (n + NTHREADS - 1) / NTHREADS;
  const uint32_t lo = c_lo + min(n, t * per), hi = c_lo + min(n, (t + 1) * per);
  uint32_t wins = 0;
  for (uint32_t c = lo; c < hi; ++c) {
    if (local_winner(sv, c, gw, gh, r, k)) {
      ++wins;
      atomicOr(smask + (c >> 5), 1u << (c & 31u));
    }
  }
  uint32_t ex, e1, tot, z;
  block_scan2<NW>(wins, 0u, ex, e1, tot, z, sh);  // also orders the smask atomics
  if (list) {
    uint32_t pos = ex;
    for (uint32_t c = lo; c < hi; ++c)
      if ((smask[c >> 5] >> (c & 31u)) & 1u) list[pos++] = c;
  }
  return tot;
}

}  // namespace dev
}  // namespace sp
