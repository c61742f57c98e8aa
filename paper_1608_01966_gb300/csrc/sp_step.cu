// Fused per-frame Spatial Pooler kernel for sm_103a.
//
//   phase 1 (all CTAs)  Alg. 1 overlap, one warp per column: 128-bit loads of
//                       the column's input indices and permanences, one bit
//                       gather per synapse from the packed frame (L1-resident),
//                       warp popcount-style reduction; min_overlap and the
//                       boost multiply in the epilogue.  A column that won the
//                       previous frame first applies that frame's learning
//                       (Section 1.1) on the same pass, so learning costs no
//                       extra read of the state.
//   phase 2 (last CTA)  Alg. 2 over all C overlaps held in shared memory:
//                       global = find the k-th largest overlap, then ties at
//                       that value go to the lowest indices through one
//                       block scan.  With unit boosts the overlap is the raw
//                       count itself, so phase 1 builds a histogram of the
//                       surviving counts (global atomics) and the k-th value
//                       is read off it in one scan; otherwise a radix select
//                       runs four 8-bit passes over the fp32 bit patterns
//                       (which order like the values, overlaps being >= 0).
//                       Local = rank count over the clipped (2r+1)^2 window.
//                       Output: ascending winner list and winner bitmask.
//
// The CTA that runs phase 2 is the last one to take a ticket from a counter,
// so no CTA ever waits for another (no grid barrier, nothing to hang).
//
// Exactness: counts are integers; the boost multiply and the learning
// add/subtract are explicit round-to-nearest intrinsics (and the file is
// built with -fmad=false); comparisons are exact.
#include "sp_kernels.cuh"

#include <atomic>

#include "../../include/sp.h"

namespace sp {

std::atomic<uint64_t> g_launches{0};

namespace {

constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t input_bit(const uint32_t* __restrict__ x, uint32_t i) {
  return (__ldg(x + (i >> 5)) >> (i & 31u)) & 1u;
}

// Section 1.1 learning of one synapse: one fp32 round-to-nearest add or
// subtract, then the clamp to [0, 1].
__device__ __forceinline__ float learn_one(float p, uint32_t bit, float inc, float dec) {
  return bit ? fminf(1.0f, __fadd_rn(p, inc)) : fmaxf(0.0f, __fsub_rn(p, dec));
}

__device__ __forceinline__ uint32_t connected_active(float p, float thr, const uint32_t* x,
                                                     uint32_t i) {
  return (p >= thr) ? input_bit(x, i) : 0u;
}

// Raw overlap of column c (Alg. 1), computed by one warp.  When learn_now,
// the previous frame's learning is applied first and written back.
template <int VEC>
__device__ __forceinline__ uint32_t column_overlap(const StepArgs& a, uint32_t c, bool learn_now,
                                                   int lane) {
  const uint64_t base = (uint64_t)c * a.S;
  uint32_t cnt = 0;
  if (VEC == 4) {
    const uint4* id4 = reinterpret_cast<const uint4*>(a.idx + base);
    float4* p4 = reinterpret_cast<float4*>(a.perm + base);
    const uint32_t n4 = a.S >> 2;
    for (uint32_t j = lane; j < n4; j += 32) {
      const uint4 id = __ldg(id4 + j);
      float4 p = p4[j];
      if (learn_now) {
        p.x = learn_one(p.x, input_bit(a.x_prev, id.x), a.inc, a.dec);
        p.y = learn_one(p.y, input_bit(a.x_prev, id.y), a.inc, a.dec);
        p.z = learn_one(p.z, input_bit(a.x_prev, id.z), a.inc, a.dec);
        p.w = learn_one(p.w, input_bit(a.x_prev, id.w), a.inc, a.dec);
        p4[j] = p;
      }
      cnt += connected_active(p.x, a.thr, a.x, id.x);
      cnt += connected_active(p.y, a.thr, a.x, id.y);
      cnt += connected_active(p.z, a.thr, a.x, id.z);
      cnt += connected_active(p.w, a.thr, a.x, id.w);
    }
  } else {
    for (uint32_t s = lane; s < a.S; s += 32) {
      const uint32_t id = __ldg(a.idx + base + s);
      float p = a.perm[base + s];
      if (learn_now) {
        p = learn_one(p, input_bit(a.x_prev, id), a.inc, a.dec);
        a.perm[base + s] = p;
      }
      cnt += connected_active(p, a.thr, a.x, id);
    }
  }
  return __reduce_add_sync(kFull, cnt);
}

// Exclusive block-wide prefix sums of two per-thread counters, plus totals.
__device__ __forceinline__ void block_scan2(uint32_t va, uint32_t vb, uint32_t& ex_a,
                                            uint32_t& ex_b, uint32_t& tot_a, uint32_t& tot_b,
                                            uint32_t* sh /* 2 * kStepWarps */) {
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
    sh[kStepWarps + warp] = ib;
  }
  __syncthreads();
  uint32_t wa = 0, wb = 0, sa = 0, sb = 0;
#pragma unroll
  for (int w = 0; w < kStepWarps; ++w) {
    const uint32_t xa = sh[w], xb = sh[kStepWarps + w];
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

// Alg. 2 over all overlaps, run by the last CTA.
__device__ void last_cta_inhibit(const StepArgs& a, uint32_t* sv, uint32_t* smask) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t sh[2 * kStepWarps];
  __shared__ uint32_t s_digit, s_above;
  const uint32_t C = a.C;
  const uint32_t t = threadIdx.x;
  for (uint32_t i = t; i < C; i += kStepThreads) sv[i] = __float_as_uint(__ldcg(a.ov + i));
  for (uint32_t i = t; i < a.mask_words; i += kStepThreads) smask[i] = 0u;
  __syncthreads();
  // each thread owns a contiguous chunk of columns, so chunk order = index order
  const uint32_t per = (C + kStepThreads - 1) / kStepThreads;
  const uint32_t lo = min(C, t * per), hi = min(C, lo + per);
  uint32_t total;

  if (a.inhibition == 0u) {
    uint32_t nz = 0;
    for (uint32_t i = lo; i < hi; ++i) nz += sv[i] != 0u;
    uint32_t e0, e1, nz_tot, z;
    block_scan2(nz, 0u, e0, e1, nz_tot, z, sh);
    // winners: every v > T, then the first `need` columns with v == T
    uint32_t T, need;
    if (a.k == 0u) {
      T = 0xffffffffu;
      need = 0u;
    } else if (nz_tot <= a.k) {
      T = 0u;
      need = 0u;
    } else if (a.hist) {
      // counts are the overlaps: walk the histogram from the top.  Thread t
      // owns bins S - t*pb ... down to S - (t+1)*pb + 1 (descending).
      const uint32_t nb = a.S;  // bins 1..S
      const uint32_t pb = (nb + kStepThreads - 1) / kStepThreads;
      const uint32_t top = nb >= t * pb ? nb - t * pb : 0u;  // first bin of this thread
      const uint32_t cnt_bins = top == 0u ? 0u : min(pb, top);
      uint32_t mine = 0;
      for (uint32_t b = 0; b < cnt_bins; ++b) mine += __ldcg(a.hist + (top - b));
      uint32_t above, e1, tot, z;
      block_scan2(mine, 0u, above, e1, tot, z, sh);
      if (above < a.k && above + mine >= a.k) {
        uint32_t acc = above;
        for (uint32_t b = 0; b < cnt_bins; ++b) {
          const uint32_t hb = __ldcg(a.hist + (top - b));
          if (acc + hb >= a.k) {
            s_digit = top - b;  // the k-th largest count
            s_above = acc;
            break;
          }
          acc += hb;
        }
      }
      __syncthreads();
      T = __float_as_uint(__uint2float_rn(s_digit));
      need = a.k - s_above;
    } else {
      uint32_t prefix = 0u, pmask = 0u, kk = a.k;
      for (int shift = 24; shift >= 0; shift -= 8) {
        for (uint32_t i = t; i < 256u; i += kStepThreads) hist[i] = 0u;
        __syncthreads();
        for (uint32_t i = lo; i < hi; ++i) {
          const uint32_t v = sv[i];
          if (v != 0u && (v & pmask) == prefix) atomicAdd(&hist[(v >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (t < 32u) {
          // lane L scans bins 255-8L .. 248-8L (descending digit order)
          uint32_t loc[8], sum = 0;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            loc[j] = hist[255u - 8u * t - j];
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
              s_digit = 255u - 8u * t - j;
              s_above = above;
            }
            above += loc[j];
          }
        }
        __syncthreads();
        prefix |= s_digit << shift;
        pmask |= 0xffu << shift;
        kk -= s_above;
        __syncthreads();
      }
      T = prefix;  // the k-th largest overlap (bit pattern)
      need = kk;   // how many columns equal to T still win
    }
    uint32_t gt = 0, eq = 0;
    for (uint32_t i = lo; i < hi; ++i) {
      const uint32_t v = sv[i];
      gt += v > T;
      eq += (need != 0u) & (v == T);
    }
    uint32_t gt_ex, eq_ex, gt_tot, eq_tot;
    block_scan2(gt, eq, gt_ex, eq_ex, gt_tot, eq_tot, sh);
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
        a.result[1u + pos++] = i;
        atomicOr(&smask[i >> 5], 1u << (i & 31u));
      }
    }
    total = gt_tot + min(eq_tot, need);
  } else {
    uint32_t wins = 0;
    for (uint32_t c = lo; c < hi; ++c) {
      if (local_winner(sv, c, a.gw, a.gh, a.radius, a.k)) {
        ++wins;
        atomicOr(&smask[c >> 5], 1u << (c & 31u));
      }
    }
    uint32_t ex, e1, tot, z;
    block_scan2(wins, 0u, ex, e1, tot, z, sh);  // also orders the smask atomics
    uint32_t pos = ex;
    for (uint32_t c = lo; c < hi; ++c)
      if ((smask[c >> 5] >> (c & 31u)) & 1u) a.result[1u + pos++] = c;
    total = tot;
  }
  __syncthreads();
  if (t == 0u) a.result[0] = total;
  if (a.hist)
    for (uint32_t b = t; b <= a.S; b += kStepThreads) a.hist[b] = 0u;
  for (uint32_t i = t; i < a.mask_words; i += kStepThreads) {
    const uint32_t m = smask[i];
    a.mask_out[i] = m;
    if (a.mask_copy) a.mask_copy[i] = m;
  }
}

template <int VEC>
__global__ void __launch_bounds__(kStepThreads) sp_step_kernel(const StepArgs a) {
  extern __shared__ uint32_t dyn_smem[];
  __shared__ uint32_t s_ticket;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (a.x_save) {
    for (uint32_t i = blockIdx.x * kStepThreads + threadIdx.x; i < a.n_words;
         i += gridDim.x * kStepThreads)
      a.x_save[i] = __ldg(a.x + i);
  }
  for (uint32_t c = blockIdx.x * kStepWarps + warp; c < a.C; c += gridDim.x * kStepWarps) {
    const bool learn_now = a.mask_prev && ((__ldg(a.mask_prev + (c >> 5)) >> (c & 31u)) & 1u);
    const uint32_t raw = column_overlap<VEC>(a, c, learn_now, lane);
    if (lane == 0) {
      const bool keep = raw >= a.min_overlap;
      a.ov[c] = keep ? __fmul_rn(__uint2float_rn(raw), __ldg(a.boost + c)) : 0.0f;
      if (a.hist && keep && raw != 0u) atomicAdd(a.hist + raw, 1u);  // unit boost: ov == raw
    }
  }
  // publish this CTA's overlaps, then take a ticket; the last CTA inhibits
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(a.counter, 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1u) return;
  __threadfence();
  last_cta_inhibit(a, dyn_smem, dyn_smem + a.C);
  if (threadIdx.x == 0) atomicExch(a.counter, 0u);
}

__global__ void __launch_bounds__(kStepThreads) sp_learn_kernel(const LearnArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint32_t c = blockIdx.x * kStepWarps + warp; c < a.C; c += gridDim.x * kStepWarps) {
    if (!((__ldg(a.mask + (c >> 5)) >> (c & 31u)) & 1u)) continue;
    const uint64_t base = (uint64_t)c * a.S;
    for (uint32_t s = lane; s < a.S; s += 32) {
      const uint32_t id = __ldg(a.idx + base + s);
      a.perm[base + s] = learn_one(a.perm[base + s], input_bit(a.x, id), a.inc, a.dec);
    }
  }
}

}  // namespace

size_t step_smem_bytes(uint32_t C) { return ((size_t)C + (C + 31u) / 32u) * sizeof(uint32_t); }

int step_grid(uint32_t C) { return (int)((C + kStepWarps - 1) / kStepWarps); }

cudaError_t kernels_init() {
  const int bytes = (int)step_smem_bytes(SP_MAX_COLUMNS);
  cudaError_t e = cudaFuncSetAttribute(sp_step_kernel<4>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sp_step_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

cudaError_t launch_step(const StepArgs& a, int grid, cudaStream_t stream) {
  const size_t smem = step_smem_bytes(a.C);
  if (a.S % 4u == 0u)
    sp_step_kernel<4><<<grid, kStepThreads, smem, stream>>>(a);
  else
    sp_step_kernel<1><<<grid, kStepThreads, smem, stream>>>(a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_learn(const LearnArgs& a, cudaStream_t stream) {
  const int grid = step_grid(a.C);
  sp_learn_kernel<<<grid, kStepThreads, 0, stream>>>(a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace sp
