// Dense potential pools on the tensor cores (sm_103a tcgen05).
//
// When every column's pool is the whole input (S = n_in, idx[c][s] = s) and a
// run of frames is computed without learning, Alg. 1's raw overlaps of F
// frames are one matrix product:
//
//     raw[f][c] = sum_i X[f][i] * Conn[c][i],   Conn[c][i] = [perm[c][i] >= thr],
//
// with X and Conn in {0, 1}.  Both operands are exact in fp8 (e4m3: 1.0 is
// 0x38), each product is 0 or 1 and every partial sum is an integer <= n_in <
// 2^24, exact in the fp32 accumulator, so the tensor-core result equals the
// integer count bit for bit.
//
// Operands live in global memory as images of the tensor core's shared-memory
// operand layout (K-major, no swizzle: 8-row x 16-byte core matrices, 128 B
// apart along K, 1024 B apart along M/N), one contiguous block per (tile of
// rows, slice of 128 inputs), zero past the ends:
//   sp_conn_image_kernel  Conn blocks (256 columns x 128 inputs, 32 KB) from
//                         perm; the image is part of the SP's state and is
//                         rebuilt only after the permanences changed;
//   sp_frame_image_kernel X blocks (128 frames x 128 inputs, 16 KB) from the
//                         packed frame bits of the run.
// sp_dense_overlap_kernel: one CTA (256 threads) per tile of 128 frames x 256
// columns.  Warp 0 streams the tile's blocks into four shared-memory stages
// with bulk copies (cp.async.bulk, completion counted on an mbarrier); warp 1
// issues four tcgen05.mma (kind::f8f6f4, M=128, N=256, K=32) per slice into a
// 128-lane x 256-column fp32 accumulator in tensor memory and commits each
// slice to the stage's "free" mbarrier.  All eight warps then read the
// accumulator with tcgen05.ld and write the boosted overlaps (min_overlap,
// boost: Alg. 1's tail) of every frame through a shared-memory transpose.
//
// sp_frame_select_warp_kernel: one warp per frame runs Alg. 2 with global
// inhibition on its overlaps; sp_frame_inhibit_kernel (one CTA per frame)
// the other inhibition modes and wider SPs.
//
// Every mbarrier wait is bounded (1 s of %globaltimer): on expiry the kernel
// records an error, stops issuing, waits (bounded) for the copies and MMAs it
// issued, frees its tensor memory and returns.
#include <algorithm>
#include <atomic>
#include <cstdlib>

#include "../../include/sp.h"
#include "sp_device.cuh"
#include "sp_kernels.cuh"

namespace sp {

extern std::atomic<uint64_t> g_launches;

namespace {

using dev::kFull;

constexpr uint32_t kTM = 128;       // frames per tile (MMA M)
constexpr uint32_t kTN = 256;       // columns per tile (MMA N)
constexpr uint32_t kTK = 128;       // inputs per slice (one byte each)
constexpr uint32_t kMmaK = 32;      // K of one kind::f8f6f4 MMA
constexpr uint32_t kStages = 4;
constexpr uint32_t kThreads = 256;  // warp 0 copies, warp 1 issues; all 8 read the accumulator
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kABytes = kTM * kTK;  // 16 KB
constexpr uint32_t kBBytes = kTN * kTK;  // 32 KB
constexpr uint32_t kLBO = 128;           // bytes between core matrices along K
constexpr uint32_t kSBO = (kTK / 16) * 128;  // bytes between 8-row groups
constexpr uint64_t kWaitNs = 1000000000ull;  // bound of every mbarrier wait
constexpr uint32_t kFp8One = 0x38;           // 1.0 in e4m3

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// tcgen05 shared-memory matrix descriptor: start address, leading (K) and
// stride (M/N) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(kLBO >> 4) << 16;
  d |= (uint64_t)(kSBO >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f8f6f4: fp32 accumulator, e4m3 A and B
// (format code 0), both K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | ((kTN >> 3) << 17) | ((kTM >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

// Wait for the phase with the given parity to complete; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < (1u << 30); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Global -> shared bulk copy (16-byte aligned ends, size a multiple of 16)
// whose bytes complete on bar.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_f8(uint32_t taddr, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// Four {0,1} bits -> four e4m3 bytes (bit i -> byte i): the multiply places
// bit i at bit 8i (the four shifted copies do not overlap), the mask keeps
// those bits and the second multiply turns each into 0x38.
__device__ __forceinline__ uint32_t fp8_nibble(uint32_t n4) {
  return ((n4 * 0x00204081u) & 0x01010101u) * kFp8One;
}

// One SP's arguments by value, or a device array of several SPs (one per
// blockIdx.z / blockIdx.y).
struct DenseLaunch {
  const DenseArgs* many;
  DenseArgs one;
};

__global__ void __launch_bounds__(kThreads, 1) sp_dense_overlap_kernel(const DenseLaunch L) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[kStages], freed[kStages], done;
  __shared__ uint32_t s_taddr;
  __shared__ volatile uint32_t s_fail;
  __shared__ uint32_t s_issued, s_consumed;
  __shared__ __align__(16) float s_boost[kTN];
  DenseArgs a;  // kept in registers
  if (L.many)
    a = L.many[blockIdx.z];
  else
    a = L.one;
  const uint32_t t = threadIdx.x, warp = t >> 5, lane = t & 31u;
  const uint32_t f0 = blockIdx.y * kTM, c0 = blockIdx.x * kTN;
  // the per-frame selection may be scheduled now: it waits for this grid
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  if (f0 >= a.n_frames || c0 >= a.C) return;  // a smaller SP of the launch
  s_boost[t] = c0 + t < a.C ? __ldg(a.boost + c0 + t) : 0.0f;  // kThreads == kTN

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&s_taddr)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (t == 0) {
    for (uint32_t i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&freed[i], 1);
    }
    mbar_init(&done, 1);
    s_fail = 0u;
    s_issued = 0u;
    s_consumed = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  // the frame image (and everything before it) is complete from here on
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  const uint32_t taddr = s_taddr;
  const uint32_t n = a.n_slices;
  const uint8_t* ablk = a.aimg + (uint64_t)blockIdx.y * n * kABytes;
  const uint8_t* bblk = a.bimg + (uint64_t)blockIdx.x * n * kBBytes;

  if (t == 0) {
    // ---- producer: slice kc into stage kc % kStages once its MMAs are done
    uint32_t kc = 0;
    for (; kc < n && !s_fail; ++kc) {
      const uint32_t st = kc % kStages;
      if (kc >= kStages && !mbar_wait_bounded(&freed[st], ((kc / kStages) - 1u) & 1u)) {
        s_fail = 1u;
        break;
      }
      uint8_t* sA = smem + st * (kABytes + kBBytes);
      mbar_expect_tx(&full[st], kABytes + kBBytes);
      bulk_copy(sA, ablk + (uint64_t)kc * kABytes, kABytes, &full[st]);
      bulk_copy(sA + kABytes, bblk + (uint64_t)kc * kBBytes, kBBytes, &full[st]);
    }
    s_issued = kc;
  } else if (t == 32) {
    // ---- MMA issuer
    uint32_t kc = 0;
    for (; kc < n && !s_fail; ++kc) {
      const uint32_t st = kc % kStages;
      if (!mbar_wait_bounded(&full[st], (kc / kStages) & 1u)) {
        s_fail = 1u;
        break;
      }
      fence_after_sync();
      const uint8_t* sA = smem + st * (kABytes + kBBytes);
      const uint64_t ad = smem_desc(smem_u32(sA)), bd = smem_desc(smem_u32(sA + kABytes));
#pragma unroll
      for (uint32_t s = 0; s < kTK / kMmaK; ++s) {
        // K advances by two core matrices (32 bytes of each row) per MMA
        const uint64_t step = (uint64_t)((2u * kLBO * s) >> 4);
        mma_f8(taddr, ad + step, bd + step, (kc | s) != 0u ? 1u : 0u);
      }
      mma_commit(&freed[st]);
    }
    s_consumed = kc;
    mma_commit(&done);  // arrives when every MMA issued above has completed
  }
  __syncthreads();
  bool ok = !s_fail;
  if (!ok) {
    // copies issued but never consumed still land in shared memory: wait for them
    if (t == 0)
      for (uint32_t kc = s_consumed; kc < s_issued; ++kc)
        mbar_wait_bounded(&full[kc % kStages], (kc / kStages) & 1u);
  }
  // every thread: the accumulator (and the stages' last readers) are done
  if (!mbar_wait_bounded(&done, 0u)) ok = false;
  ok = __syncthreads_and(ok) != 0;  // one decision for the whole CTA (warp-wide loads below)
  fence_after_sync();
  if (!ok) {
    if (t == 0) atomicExch(a.err, 1u);
  } else {
    // ---- epilogue: warp w reads accumulator lanes 32(w % 4) .. + 31 (lane i:
    // frame f0 + 32(w % 4) + i) and columns 128(w / 4) .. + 127, 32 at a time
    // (register j: column cb + j).  The raw counts are exact integers in
    // fp32, so the comparison with min_overlap (counts never reach 2^24) and
    // the one multiply by the boost are Alg. 1's tail as written.  Each 32 x
    // 32 block goes through a 4 KB shared-memory tile (the stages are free
    // now) whose 16-byte chunk j of row i sits at chunk j ^ (i % 8): lanes
    // write their rows and read back 8 lanes per row without bank conflicts,
    // and every store instruction then writes four whole 128-byte rows.
    const uint32_t q = warp & 3u, h = warp >> 2;
    const uint32_t fr0 = f0 + q * 32u;
    const float m = (float)min(a.min_overlap, 1u << 24);
    const bool vec = (a.C & 3u) == 0u;
    float4* tile = reinterpret_cast<float4*>(smem) + warp * 256u;  // [32 rows][8 chunks]
#pragma unroll 1
    for (uint32_t cb = h * 128u; cb < h * 128u + 128u; cb += 32u) {
      uint32_t r[32];
      tmem_ld32(taddr + ((q * 32u) << 16) + cb, r);
      float v[32];
#pragma unroll
      for (uint32_t j = 0; j < 32u; ++j) {
        const float raw = __uint_as_float(r[j]);
        v[j] = raw < m ? 0.0f : __fmul_rn(raw, s_boost[cb + j]);
      }
      const uint32_t c = c0 + cb;
      if (vec && c + 32u <= a.C) {
#pragma unroll
        for (uint32_t j = 0; j < 8u; ++j)
          tile[lane * 8u + (j ^ (lane & 7u))] =
              make_float4(v[4u * j], v[4u * j + 1u], v[4u * j + 2u], v[4u * j + 3u]);
        __syncwarp();
        const uint32_t chunk = lane & 7u;
#pragma unroll
        for (uint32_t i = 0; i < 8u; ++i) {
          const uint32_t row = 4u * i + (lane >> 3);
          const float4 x = tile[row * 8u + (chunk ^ (row & 7u))];
          if (fr0 + row < a.n_frames)
            *reinterpret_cast<float4*>(a.ov + (uint64_t)(fr0 + row) * a.C + c + 4u * chunk) = x;
        }
      } else if (fr0 + lane < a.n_frames) {
        float* out = a.ov + (uint64_t)(fr0 + lane) * a.C;
#pragma unroll
        for (uint32_t j = 0; j < 32u; ++j)
          if (c + j < a.C) out[c + j] = v[j];
      }
      __syncwarp();  // tile reused; converged again before the next tcgen05.ld
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr),
                 "r"(kTmemCols)
                 : "memory");
}

// Alg. 2 for frame blockIdx.x of a run whose overlaps are rows of a.ov.
struct InhibitLaunch {
  const FrameInhibitArgs* many;
  FrameInhibitArgs one;
};

__global__ void __launch_bounds__(kStepThreads) sp_frame_inhibit_kernel(const InhibitLaunch L) {
  extern __shared__ uint32_t dyn[];
  FrameInhibitArgs a;  // kept in registers
  if (L.many)
    a = L.many[blockIdx.y];
  else
    a = L.one;
  if (blockIdx.x >= a.n_frames) return;
  __shared__ uint32_t s_wmax[kStepWarps];
  __shared__ uint32_t sh[2 * kStepWarps];
  __shared__ uint32_t s2[2];
  uint32_t* sv = dyn;
  uint32_t* smask = dyn + a.C;
  uint32_t* shist = smask + a.mask_words;
  const uint32_t f = blockIdx.x, t = threadIdx.x;
  const float* ov = a.ov + (uint64_t)f * a.C;
  uint32_t nz = 0, vmax = 0;
  for (uint32_t i = t; i < a.C; i += kStepThreads) {
    const uint32_t v = __float_as_uint(__ldg(ov + i));
    sv[i] = v;
    nz += v != 0u;
    vmax = max(vmax, v);
  }
  // with unit boosts the histogram only needs bins up to the largest count
  vmax = __reduce_max_sync(dev::kFull, vmax);
  if ((t & 31u) == 0u) s_wmax[t >> 5] = vmax;
  for (uint32_t i = t; i < a.mask_words; i += kStepThreads) smask[i] = 0u;
  const bool last = f + 1u == a.n_frames;
  uint32_t* list = last ? a.result + 1 : nullptr;
  uint32_t total;
  if (a.inhibition == 0u) {
    uint32_t e0, e1, nz_tot, z;
    dev::block_scan2<kStepWarps>(nz, 0u, e0, e1, nz_tot, z, sh);
    uint32_t top = 0;
#pragma unroll
    for (int w = 0; w < kStepWarps; ++w) top = max(top, s_wmax[w]);
    const uint32_t unit_S = a.unit_S ? min(a.unit_S, (uint32_t)__uint_as_float(top)) : 0u;
    uint32_t T, need;
    dev::select_threshold<kStepThreads>(sv, a.C, a.k, nz_tot, nullptr, unit_S ? unit_S : 0u,
                                        shist, sh, s2, T, need);
    total = dev::mark_global<kStepThreads>(sv, a.C, T, need, smask, list, sh);
  } else if (a.inhibition == 1u) {
    __syncthreads();
    total = dev::mark_local<kStepThreads>(sv, 0u, a.C, a.gw, a.gh, a.radius, a.k, smask, list, sh);
  } else {
    __syncthreads();
    total = dev::mark_paper_literal<kStepThreads>(sv, a.C, a.k, smask, list, shist, sh, s2);
  }
  __syncthreads();
  for (uint32_t i = t; i < a.mask_words; i += kStepThreads) {
    if (a.masks_out) a.masks_out[(uint64_t)f * a.masks_stride + i] = smask[i];
    if (last) a.mask_last[i] = smask[i];
  }
  if (last) {
    if (t == 0) a.result[0] = total;
    for (uint32_t i = t; i < a.C; i += kStepThreads) a.ov_last[i] = __uint_as_float(sv[i]);
  }
}

// Alg. 2 with global inhibition, one warp per frame.  Lane l holds overlaps
// l, l + 32, l + 64, ... in registers, so a ballot over step j is mask word j.
// With unit boosts the overlaps are exact small integers and are compared as
// such, otherwise as fp32 bit patterns (non-negative, so integer order is
// value order).  T, the k-th largest overlap, is the largest t with at least
// k overlaps >= t; it lies between a lower bound (for k <= 32: k lanes hold a
// value >= the k-th largest lane maximum) and the maximum, so it shares their
// common leading bits and only the bits below are searched, most significant
// first.  Winners are the overlaps above T and the first k - #(> T) equal to
// T in column order (none when T is 0: fewer than k nonzero overlaps).
constexpr uint32_t kSelectWarps = 4;  // frames per CTA

template <int V>  // overlaps per lane: at most 32 * V columns
__global__ void __launch_bounds__(kSelectWarps * 32, V <= 32 ? 7 : 3) sp_frame_select_warp_kernel(
    const InhibitLaunch L) {
  constexpr int Q = (V + 31) / 32;  // mask words per lane
  FrameInhibitArgs a;  // kept in registers
  if (L.many)
    a = L.many[blockIdx.y];
  else
    a = L.one;
  __shared__ uint32_t s_hist[kSelectWarps][64];
  // the overlaps are the previous kernel's output; the next run's frame
  // image may be prepared once this run's overlaps are final
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t f = blockIdx.x * kSelectWarps + (threadIdx.x >> 5);
  if (f >= a.n_frames) return;
  const float* ov = a.ov + (uint64_t)f * a.C;
  uint32_t key[V];
  uint32_t lmax = 0;
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const uint32_t i = (uint32_t)j * 32u + lane;
    const float x = i < a.C ? __ldg(ov + i) : 0.0f;
    key[j] = a.unit_S ? __float2uint_rz(x) : __float_as_uint(x);
    lmax = max(lmax, key[j]);
  }
  const uint32_t vmax = __reduce_max_sync(kFull, lmax);
  const uint32_t k = a.k;
  uint32_t T = 0u;
  if (k == 0u) {
    T = 0xffffffffu;  // nothing exceeds or equals it: no column wins
  } else if (vmax != 0u) {
    uint32_t lo = 0u;
    if (k <= 32u) {
      for (int b = 31 - __clz(vmax); b >= 0; --b) {
        const uint32_t cand = lo | (1u << b);
        if ((uint32_t)__popc(__ballot_sync(kFull, lmax >= cand)) >= k) lo = cand;
      }
    }
    if (lo == vmax) {
      T = vmax;
    } else if (a.unit_S && k <= 32u && vmax - lo < 64u) {
      // integer overlaps in a short range [lo, vmax]: count them per value
      // (only those >= lo) and take T as the largest value with at least k
      // overlaps at or above it; lane l holds values lo + 2l and lo + 2l + 1
      uint32_t* hist = s_hist[threadIdx.x >> 5];
      hist[lane] = 0u;
      hist[lane + 32u] = 0u;
      __syncwarp();
#pragma unroll
      for (int j = 0; j < V; ++j)
        if (key[j] >= lo) atomicAdd(hist + (key[j] - lo), 1u);
      __syncwarp();
      const uint32_t h0 = hist[2u * lane], h1 = hist[2u * lane + 1u];
      uint32_t suf = h0 + h1;  // becomes the count of overlaps >= lo + 2 lane
#pragma unroll
      for (uint32_t o = 1; o < 32u; o <<= 1) {
        const uint32_t y = __shfl_down_sync(kFull, suf, o);
        if (lane + o < 32u) suf += y;
      }
      const uint32_t best = suf - h0 >= k ? 2u * lane + 2u : (suf >= k ? 2u * lane + 1u : 0u);
      T = lo + __reduce_max_sync(kFull, best) - 1u;  // count(>= lo) >= k: best >= 1 somewhere
    } else {
      const int d = 31 - __clz(lo ^ vmax);  // highest bit where the bounds differ
      T = d == 31 ? 0u : vmax & ~((2u << d) - 1u);
      for (int b = d; b >= 0; --b) {
        const uint32_t cand = T | (1u << b);
        uint32_t ge = 0;
#pragma unroll
        for (int j = 0; j < V; ++j) ge += key[j] >= cand;
        if (__reduce_add_sync(kFull, ge) >= k) T = cand;
      }
    }
  }
  uint32_t G[Q], E[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) G[q] = E[q] = 0u;
#pragma unroll
  for (int j = 0; j < V; ++j) {
    if ((uint32_t)j * 32u >= a.C) break;
    const uint32_t g = __ballot_sync(kFull, key[j] > T);
    const uint32_t e = __ballot_sync(kFull, key[j] == T);
    if (lane == ((uint32_t)j & 31u)) {
      G[j >> 5] = g;
      E[j >> 5] = e;
    }
  }
  uint32_t gt = 0;
#pragma unroll
  for (int q = 0; q < Q; ++q) gt += __popc(G[q]);
  gt = __reduce_add_sync(kFull, gt);
  const uint32_t need = (T == 0u || T == 0xffffffffu) ? 0u : k - gt;
  uint32_t W[Q];
  uint32_t before = 0;  // ties in earlier words (word order: q major, lane minor)
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    W[q] = G[q];
    if (need != 0u) {
      const uint32_t ce = __popc(E[q]);
      uint32_t inc = ce;
#pragma unroll
      for (uint32_t o = 1; o < 32u; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
      }
      const uint32_t ex = before + inc - ce;
      before += __shfl_sync(kFull, inc, 31);
      const uint32_t take = need > ex ? min(need - ex, ce) : 0u;
      uint32_t e = E[q], keep = 0u;
      if (take == ce) {
        keep = e;
      } else {
        for (uint32_t n = 0; n < take; ++n) {  // the lowest `take` tied columns
          const uint32_t low = e & (0u - e);
          keep |= low;
          e ^= low;
        }
      }
      W[q] |= keep;
    }
  }
  const bool last = f + 1u == a.n_frames;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const uint32_t w = (uint32_t)q * 32u + lane;
    if (w < a.mask_words) {
      if (a.masks_out) a.masks_out[(uint64_t)f * a.masks_stride + w] = W[q];
      if (last) a.mask_last[w] = W[q];
    }
  }
  if (last) {
    uint32_t base = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const uint32_t c = __popc(W[q]);
      uint32_t inc = c;
#pragma unroll
      for (uint32_t o = 1; o < 32u; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
      }
      uint32_t pos = base + inc - c;
      base += __shfl_sync(kFull, inc, 31);
      for (uint32_t w = W[q]; w != 0u; w &= w - 1u)
        a.result[1 + pos++] = ((uint32_t)q * 32u + lane) * 32u + (uint32_t)(__ffs(w) - 1);
    }
    if (lane == 0u) a.result[0] = gt + need;
    for (uint32_t i = lane; i < a.C; i += 32u) a.ov_last[i] = __ldg(ov + i);
  }
}

// Duty cycles over a run of frames, in frame order (one thread per column).
__global__ void sp_duty_run_kernel(const uint32_t* masks, uint32_t n_frames, uint32_t mask_words,
                                   uint32_t C, float* duty, float period) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  float d = duty[c];
  for (uint32_t f = 0; f < n_frames; ++f) {
    const float act =
        ((__ldg(masks + (uint64_t)f * mask_words + (c >> 5)) >> (c & 31u)) & 1u) ? 1.0f : 0.0f;
    d = __fadd_rn(d, __fdiv_rn(__fsub_rn(act, d), period));
  }
  duty[c] = d;
}

// Image blocks of one dense SP.  Unit u of a block (16 bytes: one row, 16
// consecutive inputs) sits at byte 16u of the block: u = 8 Q (r / 8) +
// 8 (chunk) + r % 8 for row r and 16-input chunk of the slice (Q = kTK / 16
// chunks per row), which is the core-matrix layout; unit g of the whole image
// is block g / U, unit g % U (U = rows per tile x Q), so consecutive threads
// write consecutive 16 bytes.
__device__ __forceinline__ void image_unit(uint64_t g, uint32_t rows, uint32_t n_slices,
                                           uint32_t& row, uint32_t& k0) {
  constexpr uint32_t kChunks = kTK / 16u;  // 16-input chunks per row of a slice
  const uint32_t per = rows * kChunks;     // units per block
  const uint64_t blk = g / per;
  const uint32_t u = (uint32_t)(g - blk * per);
  const uint32_t tile = (uint32_t)(blk / n_slices), slice = (uint32_t)(blk % n_slices);
  row = tile * rows + (u / (8u * kChunks)) * 8u + (u & 7u);
  k0 = slice * kTK + ((u >> 3) % kChunks) * 16u;
}

// Conn[c][i] = [perm[c][i] >= thr] as e4m3 {0, 1}; only SPs whose pack flag
// is set (their permanences changed since the image was built).
__global__ void __launch_bounds__(256) sp_conn_image_kernel(const DenseLaunch L) {
  DenseArgs a;
  if (L.many)
    a = L.many[blockIdx.y];
  else
    a = L.one;
  if (!a.pack) return;
  const uint32_t n_ct = (a.C + kTN - 1) / kTN;
  const uint64_t units = (uint64_t)n_ct * a.n_slices * kTN * (kTK / 16u);  // 16-byte units
  const bool vec = (a.K & 3u) == 0u;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < units;
       g += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t c, k0;
    image_unit(g, kTN, a.n_slices, c, k0);
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (c < a.C) {
      const float* p = a.perm + (uint64_t)c * a.K;
      if (vec && k0 + 16u <= a.K) {
#pragma unroll
        for (uint32_t q = 0; q < 4u; ++q) {
          const float4 v = __ldcs(reinterpret_cast<const float4*>(p + k0 + 4u * q));
          w[q] = (v.x >= a.thr ? kFp8One : 0u) | (v.y >= a.thr ? kFp8One << 8 : 0u) |
                 (v.z >= a.thr ? kFp8One << 16 : 0u) | (v.w >= a.thr ? kFp8One << 24 : 0u);
        }
      } else {
        uint64_t lo = 0u, hi = 0u;
        for (uint32_t i = 0; i < 16u && k0 + i < a.K; ++i) {
          const uint64_t byte = __ldcs(p + k0 + i) >= a.thr ? (uint64_t)kFp8One << (8u * (i & 7u)) : 0u;
          if (i < 8u)
            lo |= byte;
          else
            hi |= byte;
        }
        w[0] = (uint32_t)lo;
        w[1] = (uint32_t)(lo >> 32);
        w[2] = (uint32_t)hi;
        w[3] = (uint32_t)(hi >> 32);
      }
    }
    *reinterpret_cast<uint4*>(a.bimg + g * 16u) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// X[f][i] = bit i of frame f as e4m3 {0, 1}; bits at or past K are zero
// whatever the frame's unused high bits hold.
__global__ void __launch_bounds__(256) sp_frame_image_kernel(const DenseLaunch L) {
  // the product may be scheduled now (it waits for this grid).  The image is
  // written at once: this grid starts only after the previous kernel on the
  // stream let it, and a run's selection does so only after its own wait on
  // that run's product, the image's last reader.  The wait for the previous
  // kernel comes at the end, so that the product, which waits for this grid,
  // also finds the previous run's selection complete before it overwrites
  // the overlaps the selection reads.
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  DenseArgs a;
  if (L.many)
    a = L.many[blockIdx.y];
  else
    a = L.one;
  const uint32_t n_ft = (a.n_frames + kTM - 1) / kTM;
  const uint64_t units = (uint64_t)n_ft * a.n_slices * kTM * (kTK / 16u);  // 16-byte units
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < units;
       g += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t f, k0;
    image_unit(g, kTM, a.n_slices, f, k0);
    uint32_t bits = 0u;
    if (f < a.n_frames && k0 < a.K) {
      bits = (__ldg(a.frames + (uint64_t)f * a.stride + (k0 >> 5)) >> (k0 & 31u)) & 0xFFFFu;
      if (a.K - k0 < 16u) bits &= (1u << (a.K - k0)) - 1u;
    }
    *reinterpret_cast<uint4*>(a.aimg + g * 16u) =
        make_uint4(fp8_nibble(bits & 15u), fp8_nibble((bits >> 4) & 15u),
                   fp8_nibble((bits >> 8) & 15u), fp8_nibble(bits >> 12));
  }
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

}  // namespace

namespace {

// Launch with programmatic stream serialization: the kernel may start while
// the previous kernel on the stream finishes; it orders itself with
// griddepcontrol.wait where it reads that kernel's output (SP_DISABLE_PDL=1:
// plain stream order).
template <typename Arg>
cudaError_t launch_pdl(void (*kernel)(Arg), dim3 grid, uint32_t threads, size_t smem,
                       cudaStream_t stream, const Arg& arg) {
  static const bool pdl = [] {
    const char* e = std::getenv("SP_DISABLE_PDL");
    return !(e && e[0] == '1');
  }();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, arg);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

size_t dense_bimg_bytes(uint32_t C, uint32_t K) {
  return (size_t)((C + kTN - 1) / kTN) * kTN * ((K + kTK - 1) / kTK) * kTK;
}

size_t dense_aimg_bytes(uint32_t n_frames, uint32_t K) {
  return (size_t)((n_frames + kTM - 1) / kTM) * kTM * ((K + kTK - 1) / kTK) * kTK;
}

uint32_t dense_slices(uint32_t K) { return (K + kTK - 1) / kTK; }

namespace {

// A grid-stride launch over `units` 16-byte units: at most 8 CTAs of 256
// threads per SM in all.
dim3 image_grid(uint64_t units, uint32_t n) {
  const uint64_t want = (units + 255u) / 256u;
  const uint32_t cap = std::max<uint32_t>(1u, 152u * 8u / std::max<uint32_t>(1u, n));
  return dim3((uint32_t)std::max<uint64_t>(1u, std::min<uint64_t>(want, cap)), n, 1);
}

}  // namespace

cudaError_t launch_conn_image(const DenseArgs* args, uint32_t n, uint32_t max_C, uint32_t max_K,
                              cudaStream_t stream) {
  DenseLaunch L{args, DenseArgs{}};
  sp_conn_image_kernel<<<image_grid(dense_bimg_bytes(max_C, max_K) / 16u, n), 256, 0, stream>>>(L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_conn_image_one(const DenseArgs& a, cudaStream_t stream) {
  DenseLaunch L{nullptr, a};
  sp_conn_image_kernel<<<image_grid(dense_bimg_bytes(a.C, a.K) / 16u, 1u), 256, 0, stream>>>(L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_frame_image(const DenseArgs* args, uint32_t n, uint32_t max_frames,
                               uint32_t max_K, cudaStream_t stream) {
  const DenseLaunch L{args, DenseArgs{}};
  return launch_pdl(sp_frame_image_kernel, image_grid(dense_aimg_bytes(max_frames, max_K) / 16u, n),
                    256, 0, stream, L);
}

cudaError_t launch_frame_image_one(const DenseArgs& a, cudaStream_t stream) {
  const DenseLaunch L{nullptr, a};
  return launch_pdl(sp_frame_image_kernel, image_grid(dense_aimg_bytes(a.n_frames, a.K) / 16u, 1u),
                    256, 0, stream, L);
}

// Four stages of 48 KB: one CTA per SM, so its 256-column accumulator never
// waits for tensor memory.
size_t dense_smem_bytes() { return kStages * (kABytes + kBBytes); }

cudaError_t dense_init() {
  return cudaFuncSetAttribute(sp_dense_overlap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)dense_smem_bytes());
}

cudaError_t launch_dense_overlap(const DenseArgs& a, cudaStream_t stream) {
  const dim3 grid((a.C + kTN - 1) / kTN, (a.n_frames + kTM - 1) / kTM, 1);
  const DenseLaunch L{nullptr, a};
  return launch_pdl(sp_dense_overlap_kernel, grid, kThreads, dense_smem_bytes(), stream, L);
}

cudaError_t launch_dense_overlap_many(const DenseArgs* args, uint32_t n, uint32_t max_C,
                                      uint32_t max_frames, cudaStream_t stream) {
  const dim3 grid((max_C + kTN - 1) / kTN, (max_frames + kTM - 1) / kTM, n);
  const DenseLaunch L{args, DenseArgs{}};
  return launch_pdl(sp_dense_overlap_kernel, grid, kThreads, dense_smem_bytes(), stream, L);
}

size_t frame_inhibit_smem(uint32_t C, uint32_t unit_S) {
  const uint32_t hist = unit_S + 1u > 256u ? unit_S + 1u : 256u;
  return ((size_t)C + (C + 31u) / 32u + hist) * 4u;
}

size_t frame_inhibit_smem_limit() { return 226u * 1024u; }

cudaError_t frame_inhibit_init() {
  return cudaFuncSetAttribute(sp_frame_inhibit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)frame_inhibit_smem_limit());
}

namespace {

// Warp-per-frame select: global inhibition over at most 2048 columns.
cudaError_t launch_select_warp(const InhibitLaunch& L, uint32_t max_C, uint32_t max_frames,
                               uint32_t n, cudaStream_t stream) {
  const dim3 grid((max_frames + kSelectWarps - 1) / kSelectWarps, n, 1);
  if (max_C <= 1024u)
    return launch_pdl(sp_frame_select_warp_kernel<32>, grid, kSelectWarps * 32, 0, stream, L);
  return launch_pdl(sp_frame_select_warp_kernel<64>, grid, kSelectWarps * 32, 0, stream, L);
}

bool select_warp_fits(uint32_t max_C) { return max_C <= 2048u; }

}  // namespace

cudaError_t launch_frame_inhibit(const FrameInhibitArgs& a, cudaStream_t stream) {
  InhibitLaunch L{nullptr, a};
  if (a.inhibition == 0u && select_warp_fits(a.C))
    return launch_select_warp(L, a.C, a.n_frames, 1u, stream);
  sp_frame_inhibit_kernel<<<a.n_frames, kStepThreads, frame_inhibit_smem(a.C, a.unit_S), stream>>>(L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_frame_inhibit_many(const FrameInhibitArgs* args, uint32_t n, uint32_t max_C,
                                      uint32_t max_unit_S, uint32_t max_frames, bool all_global,
                                      cudaStream_t stream) {
  InhibitLaunch L{args, FrameInhibitArgs{}};
  if (all_global && select_warp_fits(max_C))
    return launch_select_warp(L, max_C, max_frames, n, stream);
  const dim3 grid(max_frames, n, 1);
  sp_frame_inhibit_kernel<<<grid, kStepThreads, frame_inhibit_smem(max_C, max_unit_S), stream>>>(L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_duty_run(const uint32_t* masks, uint32_t n_frames, uint32_t mask_words,
                            uint32_t C, float* duty, float period, cudaStream_t stream) {
  sp_duty_run_kernel<<<(C + 127) / 128, 128, 0, stream>>>(masks, n_frames, mask_words, C, duty,
                                                          period);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace sp
