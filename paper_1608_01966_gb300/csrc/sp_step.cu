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

#include <algorithm>
#include <atomic>
#include <cstdlib>

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

// count4 against input words staged in shared memory: xs[w - xlo] holds
// input word w for every word the column's pool indexes.
__device__ __forceinline__ uint32_t staged_bit(float p, float thr, const uint32_t* xs,
                                               uint32_t xlo, uint32_t i) {
  return (p >= thr) ? (xs[(i >> 5) - xlo] >> (i & 31u)) & 1u : 0u;
}
__device__ __forceinline__ uint32_t count4_staged(const float4& p, const uint4& id, float thr,
                                                  const uint32_t* xs, uint32_t xlo) {
  return staged_bit(p.x, thr, xs, xlo, id.x) + staged_bit(p.y, thr, xs, xlo, id.y) +
         staged_bit(p.z, thr, xs, xlo, id.z) + staged_bit(p.w, thr, xs, xlo, id.w);
}

__device__ __forceinline__ void learn4(float4& p, const uint4& id, const StepArgs& a) {
  p.x = learn_one(p.x, input_bit(a.x_prev, id.x), a.inc, a.dec);
  p.y = learn_one(p.y, input_bit(a.x_prev, id.y), a.inc, a.dec);
  p.z = learn_one(p.z, input_bit(a.x_prev, id.z), a.inc, a.dec);
  p.w = learn_one(p.w, input_bit(a.x_prev, id.w), a.inc, a.dec);
}

// ---- compact form: 16-bit pool offsets and connected bits -------------------
//
// A lane holds 8 synapses of a column: one 16-byte vector of offsets and one
// byte of connected bits, so a warp keeps kCompactCols columns in flight with
// a few registers each.  A column that learns reads and writes its fp32
// permanences and rewrites its connected bits; the others never touch
// permanences.

#ifndef SP_COMPACT_COLS
#define SP_COMPACT_COLS 4
#endif
constexpr int kCompactCols = SP_COMPACT_COLS;

// Rows are padded to cS = S rounded up to a multiple of 32 synapses (the
// padding: offset 0, never connected).  Lane l of a column holds synapses l,
// l + L, ..., l + 7L (L = cS / 8 lanes in use): the 8 offsets at positions
// 8l .. 8l + 7 and connected bits in byte l, so the k-th gather of all lanes
// reads 32 neighbouring synapses of the sorted pool.

__device__ __forceinline__ uint32_t off16(const uint4& o, int k) {
  const uint32_t w = k < 2 ? o.x : (k < 4 ? o.y : (k < 6 ? o.z : o.w));
  return (k & 1) ? (w >> 16) : (w & 0xffffu);
}

// Apply the pending learning to column c (the lane's 8 synapses, as laid out
// above; rows without padding, S a multiple of 32) and return the lane's new
// byte of connected bits; writes perm and conn.
// Rare (winners of the previous frame only), so kept out of line with its
// own loads to leave the common path's registers alone.
__device__ __noinline__ uint32_t compact_learn(float* perm, const uint16_t* cidx,
                                               const uint32_t* cbase, uint32_t* conn,
                                               const uint32_t* x_prev, uint32_t c, uint32_t S,
                                               float thr, float inc, float dec) {
  const int lane = threadIdx.x & 31;
  const bool act = lane < (int)(S >> 3);
  uint32_t nb = 0;
  if (act) {
    const uint4 o = reinterpret_cast<const uint4*>(cidx + (uint64_t)c * S)[lane];
    const uint32_t base = cbase[c];
    float* prow = perm + (uint64_t)c * S + lane;
    const uint32_t L = S >> 3;
    float q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = prow[k * L];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      q[k] = learn_one(q[k], input_bit(x_prev, base + off16(o, k)), inc, dec);
      nb |= (q[k] >= thr ? 1u : 0u) << k;
      prow[k * L] = q[k];
    }
  }
  uint32_t word = nb << (8u * (lane & 3));
  word |= __shfl_xor_sync(kFull, word, 1);
  word |= __shfl_xor_sync(kFull, word, 2);
  if (act && (lane & 3) == 0) conn[(uint64_t)c * (S >> 5) + (lane >> 2)] = word;
  return nb;
}

// Pending learning of a member whose compact rows are padded (S not a
// multiple of 32), for the previous frame's winners among columns [lo, hi):
// one warp per learner updates the permanences from the full form, then
// rewrites the column's connected bits (synapse s: byte s % L, bit s / L,
// L = cS / 8).  Run before the count, which then reads the new bits.
__device__ void compact_learn_padded(const StepArgs& a, uint32_t lo, uint32_t hi) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t cS = (a.S + 31u) & ~31u, L = cS >> 3;
  uint32_t q = 0;
  for (uint32_t base = lo; base < hi; base += 32u) {
    const uint32_t c = base + (uint32_t)lane;
    uint32_t m = __ballot_sync(kFull, c < hi && ((__ldcg(a.mask_prev + (c >> 5)) >> (c & 31u)) & 1u));
    for (; m; m &= m - 1u, ++q) {
      if ((q % kStepWarps) != (uint32_t)warp) continue;
      const uint32_t cl = base + (uint32_t)(__ffs(m) - 1);
      const uint64_t row = (uint64_t)cl * a.S;
      for (uint32_t s = lane; s < a.S; s += 32)
        a.perm[row + s] = learn_one(a.perm[row + s], input_bit(a.x_prev, __ldg(a.idx + row + s)),
                                    a.inc, a.dec);
      __syncwarp();
      uint8_t* cb8 = reinterpret_cast<uint8_t*>(a.conn + (uint64_t)cl * (cS >> 5));
      for (uint32_t l = lane; l < L; l += 32) {
        uint32_t byte = 0;
        for (uint32_t k = 0; k < 8u; ++k) {
          const uint32_t s = l + k * L;
          byte |= (s < a.S && a.perm[row + s] >= a.thr ? 1u : 0u) << k;
        }
        cb8[l] = (uint8_t)byte;
      }
    }
  }
}

__device__ __forceinline__ uint32_t compact_count(const uint32_t* x, uint32_t base, const uint4& o,
                                                  uint32_t cb) {
  uint32_t n = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if ((cb >> k) & 1u) n += input_bit(x, base + off16(o, k));
  return n;
}

// Raw overlap of column c (Alg. 1), computed by one warp.  When learn_now,
// the previous frame's learning is applied first and written back.  With
// VEC = 4 every lane loads two 16-byte vectors of indices and permanences
// before its first bit gather, so all of a column's state is in flight at once.
template <int VEC, bool STREAM, bool SX = false>
__device__ __forceinline__ uint32_t column_overlap(const StepArgs& a, uint32_t c, bool learn_now,
                                                   int lane, const uint32_t* xs = nullptr,
                                                   uint32_t xlo = 0u) {
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
      if (SX) {
        if (va) cnt += count4_staged(pa, ida, a.thr, xs, xlo);
        if (vb) cnt += count4_staged(pb, idb, a.thr, xs, xlo);
      } else {
        if (va) cnt += count4(pa, ida, a.thr, a.x);
        if (vb) cnt += count4(pb, idb, a.thr, a.x);
      }
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
  if (a.learn_next) {
    // the SP's next frame learns these winners first thing: ask L2 for their
    // pool indices and permanences now
    const uint32_t lines = (a.S * 4u + 127u) / 128u;
    for (uint32_t i = t; i < C; i += kStepThreads)
      if ((smask[i >> 5] >> (i & 31u)) & 1u)
        for (uint32_t l = 0; l < lines; ++l) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(a.idx + (uint64_t)i * a.S + 32u * l));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(a.perm + (uint64_t)i * a.S + 32u * l));
        }
  }
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

// Columns of one SP given to CTA bid of nb: a contiguous range of
// ceil(C / nb) columns (neighbouring receptive fields share cached input
// words, and a window-form CTA's boxes share one band of frame rows).

#ifndef SP_STAGE_RING
#define SP_STAGE_RING 3
#endif
constexpr uint32_t kRing = SP_STAGE_RING;               // column slots per warp
constexpr unsigned long long kStageWaitNs = 1000000000ull;  // give up after 1 s

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Copy one contiguous block of global memory into shared memory with the
// bulk-copy engine, completing on mbar (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(mbar))
      : "memory");
}

// Wait for phase `parity` of mbar to complete; false after kStageWaitNs.
__device__ __forceinline__ bool stage_wait(uint64_t* mbar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (uint32_t i = 0;; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 255u) == 0u) {
      const unsigned long long t = global_ns();
      if (i == 0) t0 = t;
      else if (t - t0 > kStageWaitNs) return false;
    }
  }
}

// Bytes of one warp's ring of column slots (pool row + permanence row each).
__host__ __device__ __forceinline__ uint32_t stage_ring_bytes(uint32_t S) {
  return kRing * 2u * S * 4u;
}

// Alg. 1's tail for column c with raw count `raw` (one lane): the boosted
// overlap to the SP's overlaps (and the caller's record), and, with unit
// boosts, the count into the histogram the last CTA selects from.
__device__ __forceinline__ void publish_overlap(const StepArgs& a, uint32_t c, uint32_t raw) {
  // a histogram is kept only when every boost is exactly 1, and then the
  // product is the count itself: no load stalls the warp here
  const float v = dev::boosted(raw, a.min_overlap, a.hist ? 1.0f : __ldg(a.boost + c));
  a.ov[c] = v;
  if (a.ov_copy) a.ov_copy[c] = v;
  if (a.hist && raw >= a.min_overlap && raw != 0u) atomicAdd(a.hist + raw, 1u);
}

// ---- window form: a 64 x 64 bitmap of connected synapses per column ---------
//
// Pools drawn from a receptive-field window fit a 64 x 64 box of the frame.
// A column then needs only the box origin and a 512-byte bitmap of its
// connected synapses inside the box.  A CTA's columns are consecutive, so
// their boxes cover a band of consecutive frame rows: the band is copied to
// shared memory once per item (one bulk copy).  Every warp then counts its
// columns kWinCols at a time, their bitmaps loaded into registers (16 bytes
// per lane and column, one coalesced request per column) -- with
// SP_WIN_PIPE the next group's loads are issued before the current group is
// counted.  Lane l of a column's warp counts rows l and l + 32 of its box: a
// funnel shift aligns each 64-pixel row segment of the band to the box, an
// AND with the bitmap row and a population count give the row's share of
// Alg. 1's count.  No gather leaves shared memory.
//
// Learning (the previous frame's winners, rare) runs first, CTA-wide: all
// synapses of up to kWinLearn columns at once, a pass's indices and
// permanences loaded before its first input bit is gathered.  The
// permanences (the full form stays authoritative) and the new bitmaps go to
// global memory; the first kWinLearn learners' bitmaps also stay in shared
// memory, where the count reads them (the first group's loads are issued
// before the update), and any further learner's is read back from global
// memory.

#ifndef SP_WINDOW_COLS
#define SP_WINDOW_COLS 4
#endif
#ifndef SP_WIN_PIPE
#define SP_WIN_PIPE 0
#endif
constexpr int kWinCols = SP_WINDOW_COLS;  // columns per warp in flight
constexpr uint32_t kWinLearn = 8;         // learners kept in shared memory
constexpr uint32_t kWinWords = 128;       // bitmap words per column
constexpr uint32_t kWinMaxCols = 256;     // columns of one CTA (4 warps x 64)
#ifndef SP_WIN_LEARN_UNROLL
#define SP_WIN_LEARN_UNROLL 4
#endif
constexpr int kWinLearnUnroll = SP_WIN_LEARN_UNROLL;  // synapses per thread and pass

__device__ __forceinline__ uint32_t window_row(const uint32_t* p, uint32_t sh, uint32_t lo,
                                               uint32_t hi) {
  const uint32_t a0 = p[0], a1 = p[1], a2 = p[2];
  return __popc(__funnelshift_r(a0, a1, sh) & lo) + __popc(__funnelshift_r(a1, a2, sh) & hi);
}

// This lane's share of the raw overlap of a column with bitmap rows bm,
// against the staged band: `at` = (o << 5) | (ox & 31) with o the band word
// holding the box's top-left pixel; lane_off = lane * wpr, row32 = 32 * wpr.
__device__ __forceinline__ uint32_t window_count(const uint32_t* band, const uint4& bm,
                                                 uint32_t at, uint32_t lane_off,
                                                 uint32_t row32) {
  const uint32_t* p = band + (at >> 5) + lane_off;
  return window_row(p, at & 31u, bm.x, bm.y) + window_row(p + row32, at & 31u, bm.z, bm.w);
}

__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
}

// A barrier initialized for one item is invalidated at its end, so that the
// next item of a persistent CTA may initialize the same memory again.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// The window form's pass of one CTA over its columns [lo, hi), whose boxes
// lie in frame rows [y0, y0 + nr) (see above).  If the band's copy does not
// complete in time the error word is set, the copy is waited for (bounded)
// and the columns publish 0.
template <bool STREAM, int COLS = kWinCols>
__device__ __forceinline__ void window_item(const StepArgs& a, uint32_t lo, uint32_t hi,
                                            uint32_t y0, uint32_t nr, uint32_t* dyn_smem,
                                            uint32_t* err) {
  __shared__ uint32_t s_org[kWinMaxCols];
  __shared__ uint8_t s_lmap[kWinMaxCols];  // 0, or 1 + the learner's scratch slot, or 255
  __shared__ uint32_t s_lcol[kWinMaxCols];
  __shared__ uint32_t s_nl;
  __shared__ __align__(8) uint64_t s_bar_band;
  const uint32_t t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const uint32_t n = hi > lo ? hi - lo : 0u;
  const uint32_t wpr = a.wpr;
  // the band: whole frame rows (bit x of row y is bit y * W + x of the
  // frame), 64 rows past the lowest box origin, so every row of every box is
  // in it; rows past the frame's last are zero
  const uint32_t H = a.n_words / wpr;
  const uint32_t w_lo = y0 * wpr, w_hi = min(y0 + nr, H) * wpr, w_end = (y0 + nr) * wpr;
  const bool bulk = (reinterpret_cast<uintptr_t>(a.x) & 15u) == 0u && (a.n_words & 3u) == 0u;
  const uint32_t base = bulk ? (w_lo & ~3u) : w_lo;
  const uint32_t copy_hi = bulk ? ((w_hi + 3u) & ~3u) : w_hi;  // <= n_words
  const uint32_t band_words = (max(copy_hi, w_end) - base + 4u + 3u) & ~3u;
  uint32_t* band = dyn_smem;
  uint32_t* scr = dyn_smem + band_words;
  const uint32_t c0 = lo + (uint32_t)warp;  // this warp's columns: c0, c0 + 4, ...

  if (t == 0) {
    mbar_init1(&s_bar_band);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_nl = 0u;
  }
  for (uint32_t i = t; i < n; i += kStepThreads) s_lmap[i] = 0u;
  __syncthreads();
  // the band (one bulk copy; it reads frames other work wrote with ordinary
  // stores, hence the proxy fence) and the box origins
  if (t == 0 && bulk && n) {
    asm volatile("fence.proxy.async.global;\n" ::: "memory");
    mbar_expect(&s_bar_band, (copy_hi - base) * 4u);
    bulk_g2s(band, a.x + base, (copy_hi - base) * 4u, &s_bar_band);
  }
  for (uint32_t w = copy_hi - base + t; w < band_words; w += kStepThreads) band[w] = 0u;
  if (!bulk)
    for (uint32_t w = w_lo + t; w < w_hi; w += kStepThreads)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(band + (w - base))),
                   "l"(a.x + w)
                   : "memory");
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  // each column's box as a band position: (word of its top-left pixel
  // relative to the band) << 5 | its bit in that word
  for (uint32_t i = t; i < n; i += kStepThreads) {
    const uint32_t org = __ldg(a.worg + lo + i), ox = org & 0xffffu;
    s_org[i] = (((org >> 16) * wpr + (ox >> 5) - base) << 5) | (ox & 31u);
  }
  uint4 bm[COLS];
  auto load_group = [&](uint32_t c, uint4(&b)[COLS]) {
#pragma unroll
    for (int j = 0; j < COLS; ++j) {
      const uint32_t cj = c + j * kStepWarps;
      b[j] = cj < hi ? ld_state<STREAM>(reinterpret_cast<const uint4*>(a.wbits + (uint64_t)cj * kWinWords) + lane)
                     : make_uint4(0u, 0u, 0u, 0u);
    }
  };
  // ---- learning of the previous frame's winners ----------------------------
  if (!a.mask_prev) {
    load_group(c0, bm);  // in flight during the band copy
  } else {
    // the first group's bitmaps are asked of L2 during the band copy and the
    // learning (four 128-byte lines a column)
#pragma unroll
    for (int j = 0; j < COLS; ++j) {
      const uint32_t cj = c0 + j * kStepWarps;
      if (cj < hi && lane < 4)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.wbits + (uint64_t)cj * kWinWords + lane * 32u));
    }
    for (uint32_t i = t; i < n; i += kStepThreads) {
      const uint32_t c = lo + i;
      if ((__ldcg(a.mask_prev + (c >> 5)) >> (c & 31u)) & 1u) {
        const uint32_t j = atomicAdd(&s_nl, 1u);
        s_lcol[j] = c;
        s_lmap[i] = j < kWinLearn ? (uint8_t)(j + 1u) : (uint8_t)255u;
      }
    }
    __syncthreads();
    const uint32_t nl = s_nl;
    // rounds of kWinLearn learners through the scratch, the first round last
    // so that its bitmaps remain there for the count
    const uint32_t rounds = (nl + kWinLearn - 1u) / kWinLearn;
    for (uint32_t rr = rounds; rr-- > 0u;) {
      const uint32_t j0 = rr * kWinLearn, m = min(kWinLearn, nl - j0);
      for (uint32_t i = t; i < m * kWinWords; i += kStepThreads) scr[i] = 0u;
      __syncthreads();
      const uint32_t total = m * a.S;
      // element e = j * S + s: synapse s of learner j0 + j; a thread's
      // elements advance by kStepThreads, so (j, s) is stepped, not divided
      uint32_t ej = t / a.S, es = t - ej * a.S;
      const uint32_t dj = kStepThreads / a.S, ds = kStepThreads - dj * a.S;
      auto step = [&]() {
        ej += dj;
        es += ds;
        if (es >= a.S) {
          es -= a.S;
          ++ej;
        }
      };
      const float inv_w = 1.0f / (float)a.win_w;
      for (uint32_t e0 = 0; e0 < total; e0 += kStepThreads * kWinLearnUnroll) {
        uint32_t id[kWinLearnUnroll], at[kWinLearnUnroll], jj[kWinLearnUnroll], bits = 0u;
        float p[kWinLearnUnroll];
#pragma unroll
        for (int k = 0; k < kWinLearnUnroll; ++k) {
          const bool v = ej < m;
          // C * S < 2^31 (configuration limit): a 32-bit element index
          jj[k] = ej;
          at[k] = v ? s_lcol[j0 + ej] * a.S + es : 0u;
          id[k] = v ? __ldg(a.idx + at[k]) : 0u;
          p[k] = v ? __ldcg(a.perm + at[k]) : 0.0f;
          step();
        }
#pragma unroll
        for (int k = 0; k < kWinLearnUnroll; ++k)
          bits |= (jj[k] < m ? input_bit(a.x_prev, id[k]) : 0u) << k;
#pragma unroll
        for (int k = 0; k < kWinLearnUnroll; ++k) {
          if (jj[k] < m) {
            const float q = learn_one(p[k], (bits >> k) & 1u, a.inc, a.dec);
            a.perm[at[k]] = q;
            if (q >= a.thr) {
              const uint32_t org = __ldg(a.worg + s_lcol[j0 + jj[k]]);
              // the pixel's row inside its box: (id - oy * W) / W < 64,
              // from a float estimate corrected to the exact quotient
              const uint32_t d = id[k] - (org >> 16) * a.win_w;
              uint32_t r = __float2uint_rz(__uint2float_rz(d) * inv_w);
              r = r * a.win_w > d ? r - 1u : ((r + 1u) * a.win_w <= d ? r + 1u : r);
              const uint32_t jx = d - r * a.win_w - (org & 0xffffu);
              atomicOr(scr + jj[k] * kWinWords + 2u * r + (jx >> 5), 1u << (jx & 31u));
            }
          }
        }
      }
      __syncthreads();
      // the new bitmaps to global memory, in the lane layout of the form
      for (uint32_t q = t; q < m * 32u; q += kStepThreads) {
        const uint32_t j = q >> 5, l = q & 31u;
        const uint32_t* b = scr + j * kWinWords;
        reinterpret_cast<uint4*>(a.wbits + (uint64_t)s_lcol[j0 + j] * kWinWords)[l] =
            make_uint4(b[2 * l], b[2 * l + 1], b[2 * l + 64], b[2 * l + 65]);
      }
      if (rr != 0u) __syncthreads();  // the scratch is reused by the next round
    }
    load_group(c0, bm);
  }

  // ---- band and origins in place ---------------------------------------------
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  bool ok = true;
  if (bulk && n) ok = stage_wait(&s_bar_band, 0u);
  if (!ok) {
    if (t == 0 && err) atomicExch(err, 1u);
    stage_wait(&s_bar_band, 0u);  // the copy, if still in flight (bounded)
  }
  __syncthreads();

  // ---- the count: this warp's columns, COLS at a time --------------------
  const uint32_t lane_off = (uint32_t)lane * wpr, row32 = 32u * wpr;
  const bool learners = a.mask_prev && s_nl != 0u;  // s_nl is stable after the barrier
  for (uint32_t c = c0; c < hi; c += COLS * kStepWarps) {
#if SP_WIN_PIPE
    uint4 nx[COLS];
    load_group(c + COLS * kStepWarps, nx);
#endif
    uint32_t cnt[COLS];
#pragma unroll
    for (int j = 0; j < COLS; ++j) {
      const uint32_t cj = c + j * kStepWarps;
      const uint32_t li = (learners && cj < hi) ? s_lmap[cj - lo] : 0u;
      uint4 b = bm[j];
      if (li != 0u) {  // a learner: its bitmap as rewritten above
        if (li != 255u) {
          const uint32_t* s = scr + (li - 1u) * kWinWords;
          b = make_uint4(s[2 * lane], s[2 * lane + 1], s[2 * lane + 64], s[2 * lane + 65]);
        } else {
          b = __ldcg(reinterpret_cast<const uint4*>(a.wbits + (uint64_t)cj * kWinWords) + lane);
        }
      }
      cnt[j] = (ok && cj < hi) ? window_count(band, b, s_org[cj - lo], lane_off, row32) : 0u;
    }
    // lane j publishes the group's column j
    uint32_t mine = 0u;
#pragma unroll
    for (int j = 0; j < COLS; ++j) {
      const uint32_t r = __reduce_add_sync(kFull, cnt[j]);
      mine = lane == j ? r : mine;
    }
    if (lane < COLS && c + (uint32_t)lane * kStepWarps < hi)
      publish_overlap(a, c + (uint32_t)lane * kStepWarps, mine);
#if SP_WIN_PIPE
#pragma unroll
    for (int j = 0; j < COLS; ++j) bm[j] = nx[j];
#else
    load_group(c + COLS * kStepWarps, bm);
#endif
  }
  __syncthreads();  // the band becomes the last CTA's working memory
  if (t == 0) mbar_inval(&s_bar_band);
}

// One frame of one SP, run by nb CTAs of which this is number bid.  With
// STAGE, a CTA whose columns' state fits in stage_cap bytes of dynamic
// shared memory stages it there by bulk copy first.
template <int VEC, bool STREAM, bool STAGE = false, int COLS = kCompactCols>
__device__ __forceinline__ void step_body(const StepArgs& a, uint32_t bid, uint32_t nb,
                                          uint32_t* dyn_smem, uint32_t stage_cap = 0u,
                                          uint32_t* err = nullptr, uint32_t xspan_cap = 0u,
                                          uint32_t* done = nullptr, uint32_t done_value = 0u) {
  __shared__ uint32_t s_ticket;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (a.x_save) {
    for (uint32_t i = bid * kStepThreads + threadIdx.x; i < a.n_words; i += nb * kStepThreads)
      a.x_save[i] = __ldg(a.x + i);
  }
  const uint32_t per = (a.C + nb - 1u) / nb;
  const uint32_t c_lo = min(a.C, bid * per);
  const uint32_t c_first = c_lo + warp, c_end = min(a.C, (bid + 1u) * per);
  const uint32_t c_step = kStepWarps;
  auto publish = [&](uint32_t c, uint32_t raw) { publish_overlap(a, c, raw); };
  auto learning = [&](uint32_t c) {
    return a.mask_prev && ((__ldcg(a.mask_prev + (c >> 5)) >> (c & 31u)) & 1u);
  };
  if (STAGE && a.worg) {
    window_item<STREAM, COLS>(a, c_lo, c_end, __ldg(a.wband + 2u * bid),
                        __ldg(a.wband + 2u * bid + 1u), dyn_smem, err);
  } else if (STAGE && a.cidx) {
    // compact form: COLS columns per warp in flight; the input words
    // the CTA's pools index are first copied to shared memory when they fit
    // (the copy overlaps the first group's loads), so the bit gathers read
    // shared memory instead of making one L1 lookup per lane
    const uint32_t cS = (a.S + 31u) & ~31u;  // rows padded to 32 synapses
    const bool padded = cS != a.S;
    if (padded && a.mask_prev) {
      compact_learn_padded(a, c_lo, c_end);
      __syncthreads();  // the new bits and permanences before the count reads them
    }
    const bool act = lane < (int)(cS >> 3);
    const uint32_t cw = cS >> 5;
    uint32_t xlo = 0u, xhi = 0u;
    if (a.xspan) {
      xlo = __ldg(a.xspan + 2u * bid);
      xhi = __ldg(a.xspan + 2u * bid + 1u);
    }
    const bool sx = xhi > xlo && (xhi - xlo) * 4u <= xspan_cap;
    uint32_t* xs = dyn_smem;
    if (sx) {
      for (uint32_t w = threadIdx.x; w < xhi - xlo; w += kStepThreads)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(xs + w)),
                     "l"(a.x + xlo + w)
                     : "memory");
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    uint4 o[COLS];
    uint32_t cb[COLS], base[COLS];
    auto load_into = [&](uint32_t c0, uint4(&oo)[COLS], uint32_t(&cc)[COLS],
                         uint32_t(&bb)[COLS]) {
#pragma unroll
      for (int j = 0; j < COLS; ++j) {
        const uint32_t c = c0 + j * c_step;
        const bool ok = c < c_end;
        oo[j] = (ok && act)
                    ? ld_state<STREAM>(reinterpret_cast<const uint4*>(a.cidx + (uint64_t)c * cS) + lane)
                    : make_uint4(0u, 0u, 0u, 0u);
        cc[j] = (ok && act)
                    ? (ld_state<STREAM>(a.conn + (uint64_t)c * cw + (lane >> 2)) >> (8u * (lane & 3))) & 255u
                    : 0u;
        bb[j] = ok ? __ldg(a.cbase + c) : 0u;
      }
    };
    auto load_group = [&](uint32_t c0) { load_into(c0, o, cb, base); };
    auto run_group = [&](uint32_t c0, auto count) {
#pragma unroll
      for (int j = 0; j < COLS; ++j) {
        const uint32_t c = c0 + j * c_step;
        if (!padded && c < c_end && learning(c))
          cb[j] = compact_learn(a.perm, a.cidx, a.cbase, a.conn, a.x_prev, c, a.S, a.thr, a.inc,
                                a.dec);
      }
      uint32_t cnt[COLS];
#pragma unroll
      for (int j = 0; j < COLS; ++j) cnt[j] = count(base[j], o[j], cb[j]);
#pragma unroll
      for (int j = 0; j < COLS; ++j) {
        const uint32_t c = c0 + j * c_step;
        const uint32_t r = __reduce_add_sync(kFull, cnt[j]);
        if (c < c_end && lane == 0) publish(c, r);
      }
    };
    if (sx) {
      load_group(c_first);  // in flight while the span lands
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncthreads();
      auto count_s = [&](uint32_t b, const uint4& q, uint32_t m) {
        uint32_t n = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint32_t i = b + off16(q, k);
          if ((m >> k) & 1u) n += (xs[(i >> 5) - xlo] >> (i & 31u)) & 1u;
        }
        return n;
      };
      for (uint32_t c0 = c_first; c0 < c_end; c0 += COLS * c_step) {
        if (c0 != c_first) load_group(c0);
        run_group(c0, count_s);
      }
      __syncthreads();  // the span becomes the last CTA's working memory
    } else {
      auto count_g = [&](uint32_t b, const uint4& q, uint32_t m) {
        return compact_count(a.x, b, q, m);
      };
      for (uint32_t c0 = c_first; c0 < c_end; c0 += COLS * c_step) {
        load_group(c0);
        run_group(c0, count_g);
      }
    }
  } else if (STAGE && VEC == 4 && a.S <= 512u &&
      kStepWarps * stage_ring_bytes(a.S) <= stage_cap) {
    // Each warp streams its columns' pool and permanence rows through a ring
    // of kRing shared-memory slots with bulk copies: the copies of the next
    // columns are in flight while this one is counted.
    __shared__ __align__(8) uint64_t s_mbar[kStepWarps][kRing];
    const uint32_t row = a.S * 4u;
    uint8_t* ring = reinterpret_cast<uint8_t*>(dyn_smem) + warp * stage_ring_bytes(a.S);
    uint64_t* mb = s_mbar[warp];
    const uint32_t n_mine = c_first < c_end ? (c_end - c_first + c_step - 1u) / c_step : 0u;
    auto issue = [&](uint32_t i) {  // lane 0
      const uint32_t c = c_first + i * c_step;
      uint8_t* dst = ring + (i % kRing) * 2u * row;
      uint64_t* bar = mb + (i % kRing);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(
                       smem_addr(bar)),
                   "r"(2u * row)
                   : "memory");
      bulk_g2s(dst, a.idx + (uint64_t)c * a.S, row, bar);
      bulk_g2s(dst + row, a.perm + (uint64_t)c * a.S, row, bar);
    };
    if (lane == 0) {
      for (uint32_t k = 0; k < kRing; ++k)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(mb + k))
                     : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
      for (uint32_t i = 0; i < n_mine && i < kRing; ++i) issue(i);
    }
    __syncwarp();
    uint32_t i = 0;
    for (; i < n_mine; ++i) {
      const uint32_t c = c_first + i * c_step;
      const bool ok = stage_wait(mb + (i % kRing), (i / kRing) & 1u);
      if (__any_sync(kFull, !ok)) break;
      const uint8_t* slot = ring + (i % kRing) * 2u * row;
      const uint4* id4 = reinterpret_cast<const uint4*>(slot);
      const float4* p4 = reinterpret_cast<const float4*>(slot + row);
      float4* g4 = reinterpret_cast<float4*>(a.perm + (uint64_t)c * a.S);
      const bool learn_now = learning(c);
      uint32_t cnt = 0;
      for (uint32_t j = lane; j < (a.S >> 2); j += 32) {
        const uint4 id = id4[j];
        float4 p = p4[j];
        if (learn_now) {
          learn4(p, id, a);
          g4[j] = p;
        }
        cnt += count4(p, id, a.thr, a.x);
      }
      cnt = __reduce_add_sync(kFull, cnt);
      if (lane == 0) publish(c, cnt);
      __syncwarp();  // every lane is done with the slot before it is refilled
      if (lane == 0 && i + kRing < n_mine) issue(i + kRing);
    }
    if (i < n_mine) {
      // a copy did not complete in time: report it, publish nothing useful,
      // and wait (bounded) for the copies still in flight before leaving
      if (lane == 0 && err) atomicExch(err, 1u);
      for (uint32_t k = i; k < n_mine && k < i + kRing; ++k) stage_wait(mb + (k % kRing), (k / kRing) & 1u);
      for (uint32_t k = i; k < n_mine; ++k)
        if (lane == 0) publish(c_first + k * c_step, 0u);
    }
    __syncwarp();
    if (lane == 0)
      for (uint32_t k = 0; k < kRing; ++k)
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_addr(mb + k)) : "memory");
    __syncthreads();  // the rings become the last CTA's working memory
  } else {
    uint32_t xlo = 0u, xhi = 0u;
    if (STAGE && VEC == 4 && a.xspan) {
      xlo = __ldg(a.xspan + 2u * bid);
      xhi = __ldg(a.xspan + 2u * bid + 1u);
    }
    if (xhi > xlo && (xhi - xlo) * 4u <= xspan_cap) {
      // copy the input words this CTA's pools index into shared memory once;
      // every bit gather of its columns then reads shared memory
      uint32_t* xs = dyn_smem;
      const uint32_t n = xhi - xlo;
      for (uint32_t w = threadIdx.x; w < n; w += kStepThreads) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(xs + w)),
                     "l"(a.x + xlo + w)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
      __syncthreads();
      for (uint32_t c = c_first; c < c_end; c += c_step) {
        const uint32_t raw = column_overlap<VEC, STREAM, true>(a, c, learning(c), lane, xs, xlo);
        if (lane == 0) publish(c, raw);
      }
      __syncthreads();  // the span becomes the last CTA's working memory
    } else {
      for (uint32_t c = c_first; c < c_end; c += c_step) {
        const uint32_t raw = column_overlap<VEC, STREAM>(a, c, learning(c), lane);
        if (lane == 0) publish(c, raw);
      }
    }
  }
  // publish this CTA's overlaps and histogram counts, then take a ticket:
  // the last CTA runs the inhibition.  The barrier orders every thread's
  // writes before thread 0's fence, which releases them (cumulatively) ahead
  // of its ticket; the other stores are read only by the next launch.
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_ticket = atomicAdd(a.counter, 1u);
  }
  __syncthreads();
  if (s_ticket != nb - 1u) return;
  __threadfence();
  last_cta_inhibit(a, dyn_smem, dyn_smem + a.C);
  if (threadIdx.x == 0) atomicExch(a.counter, 0u);
  if (done) {
    // release this frame's results (mask, list, reset counter and
    // histogram) to the CTAs of the SP's next frame in the same launch
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicExch(done, done_value);
    }
  }
}

template <int VEC>
__global__ void __launch_bounds__(kStepThreads) sp_step_kernel(const StepArgs a) {
  extern __shared__ __align__(128) uint32_t dyn_smem[];
  step_body<VEC, false>(a, blockIdx.x, gridDim.x, dyn_smem);
}

// Resident CTAs per SM the batch kernel is compiled for (register budget).
#ifndef SP_BATCH_MIN_BLOCKS
#define SP_BATCH_MIN_BLOCKS 10
#endif

// One frame for every SP of a batch: CTA b works on SP cta_inst[b].
//
// Launched with programmatic stream serialization: every CTA lets the next
// launch in the stream start at once, reads only the batch's static tables
// (descriptors and CTA map, written at batch creation) and then waits for
// the previous grid to complete and flush before it touches any frame or
// state, so the next frame's CTAs take SM slots freed during this frame's
// tail.  Without a programmatic predecessor the wait returns at once.
__global__ void __launch_bounds__(kStepThreads, SP_BATCH_MIN_BLOCKS) sp_batch_step_kernel(const BatchArgs ba) {
  extern __shared__ __align__(128) uint32_t dyn_smem[];
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  // serving launches copy their tables right before the launch: wait first
  if (ba.tick) asm volatile("griddepcontrol.wait;\n" ::: "memory");
  const uint32_t inst = __ldg(ba.cta_inst + blockIdx.x);
  const BatchDesc& d = ba.desc[inst];
  StepArgs a;
  a.learn_next = 0u;
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
  a.ov_copy = (ba.ov_out && !ba.tick) ? ba.ov_out + d.ov_off : nullptr;
  a.result = d.result;
  a.counter = d.counter;
  a.hist = d.hist;
  a.duty = d.duty;
  a.duty_period = d.duty_period;
  a.xspan = d.xspan;
  a.cidx = d.cidx;
  a.cbase = d.cbase;
  a.conn = d.conn;
  a.worg = d.worg;
  a.wbits = d.wbits;
  a.wband = d.wband;
  a.wpr = d.wpr;
  a.win_w = d.win_w;
  if (!ba.tick) asm volatile("griddepcontrol.wait;\n" ::: "memory");
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
  if ((a.S & 3u) == 0u || a.cidx)
    step_body<4, true, true>(a, bid, d.n_ctas, dyn_smem, ba.stage_cap, ba.err, ba.xspan_cap);
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

// Persistent launch over a whole sequence of batch frames.  CTAs take work
// items in order from a counter: item (t, k) is CTA k of frame t's grid.  An
// item of frame t > 0 first waits until its SP's frame t - 1 is complete
// (the SP's last CTA of that frame releases done[inst] = epoch + t).  The
// items it waits for were taken earlier by CTAs that are running, so the
// wait always ends; it is bounded all the same (1 s of %globaltimer, then
// the launch is aborted and the error word set; r.wait_ns sets the bound).
// Frame t + 1 of one SP thus overlaps frame t of the others instead of
// waiting for a whole grid.

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// MINB resident CTAs per SM (the register budget a thread gets) and COLS
// columns per warp in flight: one compiled schedule of the persistent batch
// pass (batch_schedule lists those compiled; the autotuner picks one).
template <int MINB, int COLS>
__global__ void __launch_bounds__(kStepThreads, MINB) sp_batch_run_kernel(const BatchRunArgs r) {
  extern __shared__ __align__(128) uint32_t dyn_smem[];
  __shared__ uint32_t s_t, s_k, s_go;
  const unsigned long long total = (unsigned long long)r.items_per_frame * r.n_frames;
  for (;;) {
    if (threadIdx.x == 0) {
      uint32_t go = 0u;
      if (ld_acquire(r.abort) == 0u) {
        const unsigned long long it = atomicAdd(r.work, 1ull);
        if (it < total) {
          s_t = (uint32_t)(it / r.items_per_frame);
          s_k = (uint32_t)(it % r.items_per_frame);
          go = 1u;
        }
      }
      s_go = go;
    }
    __syncthreads();
    if (!s_go) return;
    const uint32_t t = s_t, k = s_k;
    const uint32_t inst = __ldg(r.cta_inst + k);
    const BatchDesc& d = r.desc[inst];
    if (t > 0u) {
      if (threadIdx.x == 0) {
        const uint32_t target = r.epoch + t;
        const unsigned long long t0 = global_ns();
        uint32_t ok = 1u;
        for (uint32_t i = 0;; ++i) {
          if ((int32_t)(ld_acquire(r.done + inst) - target) >= 0) break;
          if (ld_acquire(r.abort) != 0u || global_ns() - t0 > r.wait_ns) {
            ok = 0u;
            break;
          }
          __nanosleep(i < 64u ? 32u : 256u);
        }
        if (!ok) {
          atomicExch(r.abort, 1u);
          if (r.err) atomicExch(r.err, 1u);
        }
        s_go = ok;
      }
      __syncthreads();
      if (!s_go) return;
    }
    StepArgs a;
    a.learn_next = r.learn;
    const uint32_t cur = r.cur0 ^ (t & 1u);
    const uint32_t pending = t > 0u ? r.learn : r.pending0;
    const uint32_t save = t + 1u == r.n_frames ? 1u : 0u;
    a.idx = d.idx;
    a.perm = d.perm;
    a.boost = d.boost;
    a.ov = d.ov;
    a.result_copy = nullptr;
    a.x = r.frames + (uint64_t)t * r.stride + d.frame_off;
    a.x_prev = !pending ? nullptr
               : (t > 0u ? r.frames + (uint64_t)(t - 1u) * r.stride + d.frame_off
                         : (cur ? d.xsave0 : d.xsave1));
    a.mask_prev = pending ? (cur ? d.mask0 : d.mask1) : nullptr;
    a.x_save = (r.learn && save) ? (cur ? d.xsave1 : d.xsave0) : nullptr;
    a.mask_out = cur ? d.mask1 : d.mask0;
    a.mask_copy = r.masks_out ? r.masks_out + (uint64_t)t * r.mstride + d.mask_off : nullptr;
    a.ov_copy = r.ov_out ? r.ov_out + (uint64_t)t * r.ov_stride + d.ov_off : nullptr;
    a.result = d.result;
    a.counter = d.counter;
    a.hist = d.hist;
    a.duty = d.duty;
    a.duty_period = d.duty_period;
    a.xspan = d.xspan;
    a.cidx = d.cidx;
    a.cbase = d.cbase;
    a.conn = d.conn;
    a.worg = d.worg;
    a.wbits = d.wbits;
    a.wband = d.wband;
    a.wpr = d.wpr;
    a.win_w = d.win_w;
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
    const uint32_t bid = k - d.cta_first;
    if ((a.S & 3u) == 0u || a.cidx)
      step_body<4, true, true, COLS>(a, bid, d.n_ctas, dyn_smem, r.stage_cap, r.err,
                                     r.xspan_cap, r.done + inst, r.epoch + t + 1u);
    else
      step_body<1, true, false, COLS>(a, bid, d.n_ctas, dyn_smem, 0u, nullptr, 0u,
                                      r.done + inst, r.epoch + t + 1u);
    __syncthreads();  // shared memory is reused by the next item
  }
}

namespace {

// The compiled schedules of the persistent batch pass; entry 0 is the default.
struct RunSchedule {
  void (*kernel)(const BatchRunArgs);
  uint32_t ctas_per_sm, cols_in_flight;
};
const RunSchedule kRunSchedules[] = {
    {sp_batch_run_kernel<SP_BATCH_MIN_BLOCKS, kCompactCols>, SP_BATCH_MIN_BLOCKS, kCompactCols},
    {sp_batch_run_kernel<12, 2>, 12, 2},
    {sp_batch_run_kernel<8, 4>, 8, 4},
    {sp_batch_run_kernel<8, 6>, 8, 6},
    {sp_batch_run_kernel<10, 2>, 10, 2},
};
constexpr uint32_t kNumRunSchedules = sizeof(kRunSchedules) / sizeof(kRunSchedules[0]);

}  // namespace

uint32_t batch_schedule_count() { return kNumRunSchedules; }

bool batch_schedule(uint32_t i, uint32_t* ctas_per_sm, uint32_t* cols_in_flight) {
  if (i >= kNumRunSchedules) return false;
  if (ctas_per_sm) *ctas_per_sm = kRunSchedules[i].ctas_per_sm;
  if (cols_in_flight) *cols_in_flight = kRunSchedules[i].cols_in_flight;
  return true;
}

cudaError_t kernels_init() {
  const int bytes = (int)step_smem_bytes(SP_MAX_COLUMNS);
  cudaError_t e = cudaFuncSetAttribute(sp_step_kernel<4>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(sp_batch_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           bytes);
  if (e != cudaSuccess) return e;
  for (uint32_t i = 0; i < kNumRunSchedules && e == cudaSuccess; ++i)
    e = cudaFuncSetAttribute(kRunSchedules[i].kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sp_step_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

// One warp per column: base, 16-bit offsets and connected bits.
__global__ void __launch_bounds__(256) sp_compact_kernel(const uint32_t* idx, const float* perm,
                                                         uint32_t C, uint32_t S, float thr,
                                                         uint16_t* cidx, uint32_t* cbase,
                                                         uint32_t* conn, uint32_t* wide) {
  const uint32_t c = blockIdx.x * 8u + (threadIdx.x >> 5), lane = threadIdx.x & 31u;
  if (c >= C) return;
  const uint32_t* row = idx + (uint64_t)c * S;
  uint32_t lo = 0xffffffffu, hi = 0u;
  for (uint32_t s = lane; s < S; s += 32) {
    lo = min(lo, row[s]);
    hi = max(hi, row[s]);
  }
  lo = __reduce_min_sync(kFull, lo);
  hi = __reduce_max_sync(kFull, hi);
  if (hi - lo > 0xffffu) {
    if (lane == 0) atomicOr(wide, 1u);
    return;
  }
  const uint32_t cS = (S + 31u) & ~31u;
  const uint32_t L = cS >> 3;  // lanes in use; synapse s sits with lane s % L, slot s / L
  for (uint32_t s = lane; s < cS; s += 32)
    cidx[(uint64_t)c * cS + (s % L) * 8u + s / L] = s < S ? (uint16_t)(row[s] - lo) : (uint16_t)0;
  uint8_t* cb8 = reinterpret_cast<uint8_t*>(conn + (uint64_t)c * (cS >> 5));
  for (uint32_t l = lane; l < L; l += 32) {
    uint32_t byte = 0;
    for (uint32_t k = 0; k < 8u; ++k) {
      const uint32_t s = l + k * L;
      byte |= (s < S && perm[(uint64_t)c * S + s] >= thr ? 1u : 0u) << k;
    }
    cb8[l] = (uint8_t)byte;
  }
  if (lane == 0) cbase[c] = lo;
}

cudaError_t launch_compact(const uint32_t* idx, const float* perm, uint32_t C, uint32_t S,
                           float thr, uint16_t* cidx, uint32_t* cbase, uint32_t* conn,
                           uint32_t* wide, cudaStream_t stream) {
  sp_compact_kernel<<<(C + 7u) / 8u, 256, 0, stream>>>(idx, perm, C, S, thr, cidx, cbase, conn,
                                                      wide);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

// One warp per column: the pool's bounding box, then its connected synapses
// as bits of a 64 x 64 bitmap (built in shared memory, written lane-wise).
__global__ void __launch_bounds__(256) sp_window_kernel(const uint32_t* idx, const float* perm,
                                                        uint32_t C, uint32_t S, uint32_t W,
                                                        float thr, uint32_t* worg,
                                                        uint32_t* wbits, uint32_t* bad) {
  __shared__ uint32_t s_bits[8][kWinWords];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t c = blockIdx.x * 8u + warp;
  if (c >= C) return;
  const uint64_t row = (uint64_t)c * S;
  uint32_t x0 = 0xffffffffu, x1 = 0u, y0 = 0xffffffffu, y1 = 0u;
  for (uint32_t s = lane; s < S; s += 32) {
    const uint32_t id = idx[row + s], y = id / W, x = id - y * W;
    x0 = min(x0, x);
    x1 = max(x1, x);
    y0 = min(y0, y);
    y1 = max(y1, y);
  }
  x0 = __reduce_min_sync(kFull, x0);
  x1 = __reduce_max_sync(kFull, x1);
  y0 = __reduce_min_sync(kFull, y0);
  y1 = __reduce_max_sync(kFull, y1);
  if (x1 - x0 >= 64u || y1 - y0 >= 64u || x0 > 0xffffu || y0 > 0xffffu) {
    if (lane == 0) atomicOr(bad, 1u);
    return;
  }
  uint32_t* sb = s_bits[warp];
  reinterpret_cast<uint4*>(sb)[lane] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
  for (uint32_t s = lane; s < S; s += 32) {
    if (perm[row + s] >= thr) {
      const uint32_t id = idx[row + s], y = id / W, x = id - y * W;
      const uint32_t j = x - x0;
      atomicOr(sb + 2u * (y - y0) + (j >> 5), 1u << (j & 31u));
    }
  }
  __syncwarp();
  reinterpret_cast<uint4*>(wbits + (uint64_t)c * kWinWords)[lane] =
      make_uint4(sb[2 * lane], sb[2 * lane + 1], sb[2 * lane + 64], sb[2 * lane + 65]);
  if (lane == 0) worg[c] = (y0 << 16) | x0;
}

cudaError_t launch_window(const uint32_t* idx, const float* perm, uint32_t C, uint32_t S,
                          uint32_t W, float thr, uint32_t* worg, uint32_t* wbits, uint32_t* bad,
                          cudaStream_t stream) {
  sp_window_kernel<<<(C + 7u) / 8u, 256, 0, stream>>>(idx, perm, C, S, W, thr, worg, wbits, bad);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

// Thread b: the frame rows block b of `per` consecutive columns reads: from
// its lowest box origin to 64 rows past its highest.
__global__ void __launch_bounds__(128) sp_window_band_kernel(const uint32_t* worg, uint32_t C,
                                                             uint32_t H, uint32_t per,
                                                             uint32_t n_ctas, uint32_t* out) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_ctas) return;
  const uint32_t c0 = min(C, b * per), c1 = min(C, c0 + per);
  uint32_t y0 = 0xffffffffu, y1 = 0u;
  for (uint32_t c = c0; c < c1; ++c) {
    const uint32_t oy = worg[c] >> 16;
    y0 = min(y0, oy);
    y1 = max(y1, oy + 63u);  // rows past the frame are staged as zeros
  }
  out[2u * b] = c0 < c1 ? y0 : 0u;
  out[2u * b + 1u] = c0 < c1 ? y1 - y0 + 1u : 0u;
}

cudaError_t launch_window_bands(const uint32_t* worg, uint32_t C, uint32_t H, uint32_t n_ctas,
                                uint32_t* out, cudaStream_t stream) {
  const uint32_t per = (C + n_ctas - 1u) / n_ctas;
  sp_window_band_kernel<<<(n_ctas + 127u) / 128u, 128, 0, stream>>>(worg, C, H, per, n_ctas, out);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

uint32_t window_smem_bytes(uint32_t rows, uint32_t wpr) {
  // band (rounded out to 16-byte ends, plus slack for the last row's third
  // word) and the learning scratch
  return (((rows * wpr + 12u + 3u) & ~3u) + kWinLearn * kWinWords) * 4u;
}

// Block b of `per` consecutive columns: lowest and one past the highest input
// word its pools index.
__global__ void __launch_bounds__(256) sp_xspan_kernel(const uint32_t* idx, uint32_t C,
                                                       uint32_t S, uint32_t per, uint32_t* out) {
  __shared__ uint32_t s_lo[8], s_hi[8];
  const uint32_t c0 = min(C, blockIdx.x * per), c1 = min(C, (blockIdx.x + 1u) * per);
  uint32_t lo = 0xffffffffu, hi = 0u;
  for (uint64_t e = (uint64_t)c0 * S + threadIdx.x; e < (uint64_t)c1 * S; e += blockDim.x) {
    const uint32_t w = __ldg(idx + e) >> 5;
    lo = min(lo, w);
    hi = max(hi, w + 1u);
  }
  lo = __reduce_min_sync(kFull, lo);
  hi = __reduce_max_sync(kFull, hi);
  if ((threadIdx.x & 31u) == 0u) {
    s_lo[threadIdx.x >> 5] = lo;
    s_hi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (uint32_t w = 1; w < blockDim.x / 32u; ++w) {
      lo = min(lo, s_lo[w]);
      hi = max(hi, s_hi[w]);
    }
    out[2u * blockIdx.x] = hi > 0u ? lo : 0u;
    out[2u * blockIdx.x + 1u] = hi;
  }
}

cudaError_t launch_xspan(const uint32_t* idx, uint32_t C, uint32_t S, uint32_t n_ctas,
                         uint32_t* out, cudaStream_t stream) {
  const uint32_t per = (C + n_ctas - 1u) / n_ctas;
  sp_xspan_kernel<<<n_ctas, 256, 0, stream>>>(idx, C, S, per, out);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_batch_run(const BatchRunArgs& r, uint32_t max_C, uint32_t schedule,
                             cudaStream_t stream) {
  const RunSchedule& rs = kRunSchedules[schedule < kNumRunSchedules ? schedule : 0u];
  const size_t smem = std::max<size_t>(step_smem_bytes(max_C),
                                       std::max(std::max(r.stage_cap, r.xspan_cap), r.win_cap));
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rs.kernel, kStepThreads, smem);
  if (e != cudaSuccess) return e;
  const unsigned long long total = (unsigned long long)r.items_per_frame * r.n_frames;
  const unsigned long long resident = (unsigned long long)std::max(1, sms * std::max(1, per_sm));
  const uint32_t grid = (uint32_t)std::min(total, resident);
  rs.kernel<<<grid, kStepThreads, smem, stream>>>(r);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

uint32_t batch_stage_bytes(uint32_t C, uint32_t S, uint32_t n_ctas) {
  (void)C;
  (void)n_ctas;
  if (S % 4u || S > 512u) return 0u;
  return kStepWarps * stage_ring_bytes(S);
}

cudaError_t launch_batch_step(const BatchArgs& a, uint32_t n_ctas, uint32_t max_C,
                              cudaStream_t stream) {
  const size_t smem = std::max<size_t>(step_smem_bytes(max_C),
                                       std::max(std::max(a.stage_cap, a.xspan_cap), a.win_cap));
  static const bool pdl = [] {
    const char* e = std::getenv("SP_DISABLE_PDL");
    return !(e && e[0] == '1');
  }();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_ctas);
  cfg.blockDim = dim3(kStepThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, sp_batch_step_kernel, a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e != cudaSuccess ? e : cudaGetLastError();
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
