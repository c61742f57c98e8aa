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

#include "sp_device.cuh"

#include "../../include/sp.h"

namespace sp {

std::atomic<uint64_t> g_launches{0};

namespace {

using dev::input_bit;
using dev::kFull;
using dev::learn_one;

__device__ __forceinline__ uint32_t connected_active(float p, float thr, const uint32_t* x,
                                                     uint32_t i) {
  return (p >= thr) ? input_bit(x, i) : 0u;
}

template <bool STREAM, typename T>
__device__ __forceinline__ T ld_state(const T* p) {
  // streamed state (batches, far larger than L2) is read once per launch
  if (STREAM) return __ldcs(p);
  return *p;
}

__device__ __forceinline__ uint32_t count4(const float4& p, const uint4& id, float thr,
                                           const uint32_t* x) {
  return connected_active(p.x, thr, x, id.x) + connected_active(p.y, thr, x, id.y) +
         connected_active(p.z, thr, x, id.z) + connected_active(p.w, thr, x, id.w);
}

__device__ __forceinline__ void learn4(float4& p, const uint4& id, const StepArgs& a) {
  p.x = learn_one(p.x, input_bit(a.x_prev, id.x), a.inc, a.dec);
  p.y = learn_one(p.y, input_bit(a.x_prev, id.y), a.inc, a.dec);
  p.z = learn_one(p.z, input_bit(a.x_prev, id.z), a.inc, a.dec);
  p.w = learn_one(p.w, input_bit(a.x_prev, id.w), a.inc, a.dec);
}

// Raw overlap of column c (Alg. 1), computed by one warp.  When learn_now,
// the previous frame's learning is applied first and written back.  With
// VEC = 4 every lane loads two 16-byte vectors of indices and permanences
// before its first bit gather, so all of a column's state is in flight at once.
template <int VEC, bool STREAM>
__device__ __forceinline__ uint32_t column_overlap(const StepArgs& a, uint32_t c, bool learn_now,
                                                   int lane) {
  const uint64_t base = (uint64_t)c * a.S;
  uint32_t cnt = 0;
  if (VEC == 4) {
    const uint4* id4 = reinterpret_cast<const uint4*>(a.idx + base);
    float4* p4 = reinterpret_cast<float4*>(a.perm + base);
    const uint32_t n4 = a.S >> 2;
    for (uint32_t j0 = 0; j0 < n4; j0 += 64) {
      const uint32_t ja = j0 + lane, jb = j0 + 32 + lane;
      const bool va = ja < n4, vb = jb < n4;
      const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
      const float4 f4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const uint4 ida = va ? ld_state<STREAM>(id4 + ja) : z4;
      const uint4 idb = vb ? ld_state<STREAM>(id4 + jb) : z4;
      float4 pa = va ? ld_state<STREAM>(p4 + ja) : f4;
      float4 pb = vb ? ld_state<STREAM>(p4 + jb) : f4;
      if (learn_now) {
        if (va) {
          learn4(pa, ida, a);
          p4[ja] = pa;
        }
        if (vb) {
          learn4(pb, idb, a);
          p4[jb] = pb;
        }
      }
      if (va) cnt += count4(pa, ida, a.thr, a.x);
      if (vb) cnt += count4(pb, idb, a.thr, a.x);
    }
  } else {
    for (uint32_t s = lane; s < a.S; s += 32) {
      const uint32_t id = ld_state<STREAM>(a.idx + base + s);
      float p = ld_state<STREAM>(a.perm + base + s);
      if (learn_now) {
        p = learn_one(p, input_bit(a.x_prev, id), a.inc, a.dec);
        a.perm[base + s] = p;
      }
      cnt += connected_active(p, a.thr, a.x, id);
    }
  }
  return __reduce_add_sync(kFull, cnt);
}

// Alg. 2 over all overlaps, run by the last CTA.
__device__ void last_cta_inhibit(const StepArgs& a, uint32_t* sv, uint32_t* smask) {
  __shared__ uint32_t shist[256];
  __shared__ uint32_t sh[2 * kStepWarps];
  __shared__ uint32_t s2[2];
  const uint32_t C = a.C;
  const uint32_t t = threadIdx.x;
  uint32_t nz = 0;
  for (uint32_t i = t; i < C; i += kStepThreads) {
    const uint32_t v = __float_as_uint(__ldcg(a.ov + i));
    sv[i] = v;
    nz += v != 0u;
  }
  for (uint32_t i = t; i < a.mask_words; i += kStepThreads) smask[i] = 0u;
  uint32_t total;
  if (a.inhibition == 0u) {
    uint32_t e0, e1, nz_tot, z;
    dev::block_scan2<kStepWarps>(nz, 0u, e0, e1, nz_tot, z, sh);  // also publishes sv
    uint32_t T, need;
    dev::select_threshold<kStepThreads>(sv, C, a.k, nz_tot, a.hist, a.hist ? a.S : 0u, shist,
                                        sh, s2, T, need);
    total = dev::mark_global<kStepThreads>(sv, C, T, need, smask, a.result + 1, sh);
  } else if (a.inhibition == 1u) {
    __syncthreads();
    total = dev::mark_local<kStepThreads>(sv, 0u, C, a.gw, a.gh, a.radius, a.k, smask,
                                          a.result + 1, sh);
  } else {
    __syncthreads();
    total = dev::mark_paper_literal<kStepThreads>(sv, C, a.k, smask, a.result + 1, shist, sh,
                                                  s2);
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
  if (a.duty) {
    // duty cycle d <- d + (a - d) / period, each step one fp32 RN op
    for (uint32_t i = t; i < C; i += kStepThreads) {
      const float act = ((smask[i >> 5] >> (i & 31u)) & 1u) ? 1.0f : 0.0f;
      const float d = a.duty[i];
      a.duty[i] = __fadd_rn(d, __fdiv_rn(__fsub_rn(act, d), a.duty_period));
    }
  }
  if (a.result_copy) {
    __syncthreads();  // the list written above is visible to the whole CTA
    for (uint32_t i = t; i <= total; i += kStepThreads)
      a.result_copy[i] = i == 0u ? total : __ldcg(a.result + i);
  }
}

// One frame of one SP, run by nb CTAs of which this is number bid.
template <int VEC, bool STREAM>
__device__ __forceinline__ void step_body(const StepArgs& a, uint32_t bid, uint32_t nb,
                                          uint32_t* dyn_smem) {
  __shared__ uint32_t s_ticket;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (a.x_save) {
    for (uint32_t i = bid * kStepThreads + threadIdx.x; i < a.n_words; i += nb * kStepThreads)
      a.x_save[i] = __ldg(a.x + i);
  }
  bool wrote = false;
  for (uint32_t c = bid * kStepWarps + warp; c < a.C; c += nb * kStepWarps) {
    const bool learn_now = a.mask_prev && ((__ldg(a.mask_prev + (c >> 5)) >> (c & 31u)) & 1u);
    const uint32_t raw = column_overlap<VEC, STREAM>(a, c, learn_now, lane);
    if (lane == 0) {
      a.ov[c] = dev::boosted(raw, a.min_overlap, __ldg(a.boost + c));
      // unit boosts: the overlap is the count, histogrammed for the select
      if (a.hist && raw >= a.min_overlap && raw != 0u) atomicAdd(a.hist + raw, 1u);
      wrote = true;
    }
  }
  // publish this CTA's overlaps (only their writers need the fence; the
  // other stores are read by the next launch), then take a ticket: the last
  // CTA runs the inhibition
  if (wrote) __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(a.counter, 1u);
  __syncthreads();
  if (s_ticket != nb - 1u) return;
  __threadfence();
  last_cta_inhibit(a, dyn_smem, dyn_smem + a.C);
  if (threadIdx.x == 0) atomicExch(a.counter, 0u);
}

template <int VEC>
__global__ void __launch_bounds__(kStepThreads) sp_step_kernel(const StepArgs a) {
  extern __shared__ uint32_t dyn_smem[];
  step_body<VEC, false>(a, blockIdx.x, gridDim.x, dyn_smem);
}

// Resident CTAs per SM the batch kernel is compiled for (register budget).
#ifndef SP_BATCH_MIN_BLOCKS
#define SP_BATCH_MIN_BLOCKS 16
#endif

// One frame for every SP of a batch: CTA b works on SP cta_inst[b].
__global__ void __launch_bounds__(kStepThreads, SP_BATCH_MIN_BLOCKS) sp_batch_step_kernel(const BatchArgs ba) {
  extern __shared__ uint32_t dyn_smem[];
  const uint32_t inst = __ldg(ba.cta_inst + blockIdx.x);
  const BatchDesc& d = ba.desc[inst];
  StepArgs a;
  a.idx = d.idx;
  a.perm = d.perm;
  a.boost = d.boost;
  a.ov = d.ov;
  uint32_t cur, pending, learn, save, cta_first;
  a.result_copy = nullptr;
  if (ba.tick) {
    const TickMember& tm = ba.tick[inst];
    a.x = tm.x;
    cur = tm.flags & kTickCur;
    pending = tm.flags & kTickPending;
    learn = tm.flags & kTickLearn;
    save = tm.flags & kTickSave;
    cta_first = tm.cta_first;
    a.x_prev = pending ? (cur ? d.xsave0 : d.xsave1) : nullptr;
    a.result_copy = ba.results_out ? ba.results_out + tm.out_off : nullptr;
  } else {
    a.x = ba.frames + d.frame_off;
    cur = ba.cur;
    pending = ba.pending;
    learn = ba.learn;
    save = ba.save;
    cta_first = d.cta_first;
    a.x_prev = !pending ? nullptr
               : (ba.prev_frames ? ba.prev_frames + d.frame_off : (cur ? d.xsave0 : d.xsave1));
  }
  a.mask_prev = pending ? (cur ? d.mask0 : d.mask1) : nullptr;
  a.x_save = (learn && save) ? (cur ? d.xsave1 : d.xsave0) : nullptr;
  a.mask_out = cur ? d.mask1 : d.mask0;
  a.mask_copy = (ba.masks_out && !ba.tick) ? ba.masks_out + d.mask_off : nullptr;
  a.result = d.result;
  a.counter = d.counter;
  a.hist = d.hist;
  a.duty = d.duty;
  a.duty_period = d.duty_period;
  a.C = d.C;
  a.S = d.S;
  a.n_words = d.n_words;
  a.mask_words = d.mask_words;
  a.thr = d.thr;
  a.inc = d.inc;
  a.dec = d.dec;
  a.min_overlap = d.min_overlap;
  a.k = d.k;
  a.inhibition = d.inhibition;
  a.gw = d.gw;
  a.gh = d.gh;
  a.radius = d.radius;
  const uint32_t bid = blockIdx.x - cta_first;
  if ((a.S & 3u) == 0u)
    step_body<4, true>(a, bid, d.n_ctas, dyn_smem);
  else
    step_body<1, true>(a, bid, d.n_ctas, dyn_smem);
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
  e = cudaFuncSetAttribute(sp_batch_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sp_step_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

cudaError_t launch_batch_step(const BatchArgs& a, uint32_t n_ctas, uint32_t max_C,
                              cudaStream_t stream) {
  sp_batch_step_kernel<<<n_ctas, kStepThreads, step_smem_bytes(max_C), stream>>>(a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
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
