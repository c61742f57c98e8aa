// Dense potential pools on the tensor cores (sm_103a tcgen05).
//
// When every column's pool is the whole input (S = n_in, idx[c][s] = s) and a
// run of frames is computed without learning, Alg. 1's raw overlaps of F
// frames are one matrix product:
//
//     raw[f][c] = sum_i X[f][i] * Conn[c][i],   Conn[c][i] = [perm[c][i] >= thr],
//
// with X and Conn in {0, 1}.  Both operands are exact in bf16 and every
// partial sum is an integer <= n_in < 2^24, exact in the fp32 accumulator,
// so the tensor-core result equals the integer count bit for bit.
//
// sp_conn_pack_kernel packs [perm >= thr] into bits once per run.
// sp_dense_overlap_kernel: one CTA (128 threads) per tile of 128 frames x 256
// columns.  For each 64-input slice of K the threads expand the packed frame
// bits and the packed connected bits into bf16 operand tiles in shared
// memory (two stages: a slice is expanded while the previous slice's MMAs
// run) (canonical K-major layout without swizzle: 8-row x 16-byte core
// matrices, 128 B apart along K, 1024 B apart along M/N); one thread issues
// four tcgen05.mma (M=128, N=256, K=16) into a 128-lane x 256-column fp32
// accumulator in tensor memory and commits them to an mbarrier.  The
// epilogue reads the accumulator with tcgen05.ld and writes the boosted
// overlaps (min_overlap, boost: Alg. 1's tail) of every frame.
//
// sp_frame_inhibit_kernel: one CTA per frame runs Alg. 2 on its overlaps.
//
// The only wait is on the mbarrier the MMAs complete, bounded by an
// iteration limit: on expiry the kernel records an error, stops issuing,
// waits (bounded) for what it issued, frees its tensor memory and returns.
#include <algorithm>
#include <atomic>

#include "../../include/sp.h"
#include "sp_device.cuh"
#include "sp_kernels.cuh"

namespace sp {

extern std::atomic<uint64_t> g_launches;

namespace {

using dev::kFull;

constexpr uint32_t kTM = 128;   // frames per tile (MMA M)
constexpr uint32_t kTN = 256;   // columns per tile (MMA N)
constexpr uint32_t kTK = 64;    // inputs per shared-memory slice
constexpr uint32_t kMmaK = 16;  // K of one kind::f16 MMA
constexpr uint32_t kThreads = 256;  // 8 warps expand operands; warps 0-3 read the accumulator
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kABytes = kTM * kTK * 2;  // 16 KB
constexpr uint32_t kBBytes = kTN * kTK * 2;  // 32 KB
constexpr uint32_t kSuperK = 1024;           // inputs whose packed bits are staged at once
constexpr uint32_t kSuperW = kSuperK / 32;   // words per row of a staged slab
constexpr uint32_t kSlabStride = kSuperW + 1;  // padded: rows fall in different banks
constexpr uint32_t kBitsBytes = (kTM + kTN) * kSlabStride * 4;  // ~49.5 KB
constexpr uint32_t kLBO = 128;               // bytes between core matrices along K
constexpr uint32_t kSBO = (kTK / 8) * 128;   // bytes between 8-row groups
constexpr uint32_t kWaitLimit = 1u << 26;    // mbarrier polls before giving up
constexpr uint16_t kBf16One = 0x3F80;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
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

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((kTN >> 3) << 17) |
                            ((kTM >> 4) << 24);

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

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t taddr, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
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
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
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

// Offset of element (row, k) of an operand tile in the canonical layout.
__device__ __forceinline__ uint32_t tile_off(uint32_t row, uint32_t k) {
  return (row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7u) * 16u + (k & 7u) * 2u;
}

__device__ __forceinline__ uint32_t two_bf16(bool lo, bool hi) {
  return (lo ? (uint32_t)kBf16One : 0u) | (hi ? ((uint32_t)kBf16One << 16) : 0u);
}

// One SP's arguments by value, or a device array of several SPs (one per
// blockIdx.z).
struct DenseLaunch {
  const DenseArgs* many;
  DenseArgs one;
};

__global__ void __launch_bounds__(kThreads, 1) sp_dense_overlap_kernel(const DenseLaunch L) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t s_taddr;
  __shared__ uint32_t s_fail;
  DenseArgs a;  // kept in registers
  if (L.many)
    a = L.many[blockIdx.z];
  else
    a = L.one;
  uint32_t* s_abits = reinterpret_cast<uint32_t*>(smem + 2u * (kABytes + kBBytes));
  uint32_t* s_bbits = s_abits + kTM * kSlabStride;
  const uint32_t t = threadIdx.x, warp = t >> 5, lane = t & 31u;
  const uint32_t f0 = blockIdx.y * kTM, c0 = blockIdx.x * kTN;
  if (f0 >= a.n_frames || c0 >= a.C) return;  // a smaller SP of the launch

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&s_taddr)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (t == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    s_fail = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t taddr = s_taddr;

  const uint32_t n_chunks = (a.K + kTK - 1) / kTK;
  uint32_t phase[2] = {0u, 0u};
  for (uint32_t kc = 0; kc < n_chunks; ++kc) {
    const uint32_t st = kc & 1u;
    uint8_t* sA = smem + st * (kABytes + kBBytes);
    uint8_t* sB = sA + kABytes;
    // this stage was last read by the MMAs of slice kc - 2
    if (kc >= 2u) {
      if (!mbar_wait_bounded(&mbar[st], phase[st])) s_fail = 1u;
      phase[st] ^= 1u;
    }
    const uint32_t k0 = kc * kTK;
    // ---- every kSuperK inputs: stage the packed bits of the CTA's rows
    if ((k0 % kSuperK) == 0u) {
      __syncthreads();  // the previous slab has been expanded
      const uint32_t w0 = k0 >> 5;
      for (uint32_t i = t; i < kTM * kSuperW; i += kThreads) {
        const uint32_t r = i / kSuperW, w = i % kSuperW, f = f0 + r, wi = w0 + w;
        uint32_t v = 0u;
        if (f < a.n_frames && wi < a.n_words) {
          v = __ldg(a.frames + (uint64_t)f * a.stride + wi);
          // inputs at or beyond n_in are zero whatever the unused bits hold
          const uint32_t base = wi * 32u;
          if (base + 32u > a.K) v &= (a.K > base) ? ((1u << (a.K - base)) - 1u) : 0u;
        }
        s_abits[r * kSlabStride + w] = v;
      }
      for (uint32_t i = t; i < kTN * kSuperW; i += kThreads) {
        const uint32_t r = i / kSuperW, w = i % kSuperW, c = c0 + r, wi = w0 + w;
        s_bbits[r * kSlabStride + w] = (c < a.C && wi < a.conn_words)
                                           ? __ldg(a.conn + (uint64_t)c * a.conn_words + wi)
                                           : 0u;
      }
      __syncthreads();
    }
    const uint32_t ws = (k0 % kSuperK) >> 5;  // word of this slice in the slab
    // ---- expand: a thread takes whole rows of the slice (64 inputs = two
    // words of bits -> eight 16-byte units of 8 bf16); rows 0..127 are A
    // (frames), 128..383 B (columns); consecutive threads write consecutive
    // 16-byte rows of a core matrix
    for (uint32_t row = t; row < kTM + kTN; row += kThreads) {
      const bool is_a = row < kTM;
      const uint32_t r = is_a ? row : row - kTM;
      const uint32_t* bitsrow = is_a ? s_abits + r * kSlabStride : s_bbits + r * kSlabStride;
      const uint32_t w0 = bitsrow[ws], w1 = bitsrow[ws + 1u];
      uint8_t* dst = (is_a ? sA : sB) + tile_off(r, 0u);
#pragma unroll
      for (uint32_t j = 0; j < 8u; ++j) {
        const uint32_t bits = ((j < 4u ? w0 : w1) >> ((j & 3u) * 8u)) & 0xFFu;
        uint4 v;
        v.x = two_bf16(bits & 1u, bits & 2u);
        v.y = two_bf16(bits & 4u, bits & 8u);
        v.z = two_bf16(bits & 16u, bits & 32u);
        v.w = two_bf16(bits & 64u, bits & 128u);
        *reinterpret_cast<uint4*>(dst + j * kLBO) = v;
      }
    }
    // make the tiles visible to the tensor core, then one thread issues
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (s_fail) break;
    if (t == 0) {
      const uint64_t ad = smem_desc(smem_u32(sA)), bd = smem_desc(smem_u32(sB));
#pragma unroll
      for (uint32_t s = 0; s < kTK / kMmaK; ++s) {
        // K advances by two core matrices (32 bytes of each row) per MMA
        const uint64_t step = (uint64_t)((2u * kLBO * s) >> 4);
        mma_bf16(taddr, ad + step, bd + step, (kc | s) != 0u ? 1u : 0u);
      }
      mma_commit(&mbar[st]);
    }
  }
  // the last one or two commits are still outstanding
  if (!s_fail) {
    for (uint32_t st = 0; st < 2u; ++st) {
      const uint32_t issued = n_chunks > st ? (n_chunks - st + 1u) / 2u : 0u;
      const uint32_t waited = n_chunks > st + 2u ? (n_chunks - st - 1u) / 2u : 0u;
      if (issued > waited && !mbar_wait_bounded(&mbar[st], phase[st])) s_fail = 1u;
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();

  if (s_fail) {
    // let whatever was issued finish (bounded) before the memory is released
    mbar_wait_bounded(&mbar[0], phase[0]);
    mbar_wait_bounded(&mbar[1], phase[1]);
    if (t == 0) atomicExch(a.err, 1u);
  } else if (warp < 4u) {
    // ---- epilogue: warp w holds frames f0 + 32w .. f0 + 32w + 31; each 32 x
    // 32 block goes through shared memory (the operand stages are free now)
    // so that every store writes 32 consecutive columns of one frame
    float* tr = reinterpret_cast<float*>(smem) + warp * 32u * 33u;
    const uint32_t c = c0 + lane;  // this lane's column within the block, below
#pragma unroll 1
    for (uint32_t cb = 0; cb < kTN; cb += 32u) {
      uint32_t r[32];
      tmem_ld32(taddr + ((warp * 32u) << 16) + cb, r);
#pragma unroll
      for (uint32_t j = 0; j < 32; ++j) tr[lane * 33u + j] = __uint_as_float(r[j]);
      __syncwarp();
      const bool col_ok = c + cb < a.C;
      const float b = col_ok ? __ldg(a.boost + c + cb) : 0.0f;
#pragma unroll 4
      for (uint32_t i = 0; i < 32u; ++i) {
        const uint32_t f = f0 + warp * 32u + i;
        if (f < a.n_frames && col_ok) {
          const uint32_t raw = (uint32_t)tr[i * 33u + lane];
          a.ov[(uint64_t)f * a.C + c + cb] = dev::boosted(raw, a.min_overlap, b);
        }
      }
      __syncwarp();
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
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

// Connected bits of one dense SP: word w of column c holds [perm >= thr] of
// inputs 32w .. 32w+31 (LSB first; zero beyond K and in the padding word).
// One warp per word: lane i reads input 32w + i (coalesced) and a ballot packs.
__global__ void __launch_bounds__(256) sp_conn_pack_kernel(const DenseLaunch L) {
  DenseArgs a;
  if (L.many)
    a = L.many[blockIdx.y];
  else
    a = L.one;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (blockDim.x >> 5) * gridDim.x;
  const uint32_t first = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  uint32_t* conn = const_cast<uint32_t*>(a.conn);
  if ((a.K & 3u) == 0u) {
    // a warp takes 4 words (128 synapses) per row block: one 16-byte load per
    // lane (4 synapses, 4 bits); 8 lanes OR their nibbles into a word; four
    // blocks' loads are in flight together
    const uint32_t blocks_per_row = (a.conn_words + 3u) / 4u;
    const uint32_t total = a.C * blocks_per_row;
    for (uint32_t b0 = first; b0 < total; b0 += 4u * warps) {
      uint32_t nib[4];
#pragma unroll
      for (uint32_t q = 0; q < 4u; ++q) {
        const uint32_t b = b0 + q * warps;
        const uint32_t c = b / blocks_per_row, blk = b - c * blocks_per_row;
        const uint32_t k = blk * 128u + lane * 4u;
        nib[q] = 0u;
        if (b < total && k < a.K) {
          const float4 p = __ldcs(reinterpret_cast<const float4*>(a.perm + (uint64_t)c * a.K + k));
          nib[q] = (p.x >= a.thr ? 1u : 0u) | (p.y >= a.thr ? 2u : 0u) |
                   (p.z >= a.thr ? 4u : 0u) | (p.w >= a.thr ? 8u : 0u);
        }
      }
#pragma unroll
      for (uint32_t q = 0; q < 4u; ++q) {
        const uint32_t b = b0 + q * warps;
        uint32_t word = nib[q] << (4u * (lane & 7u));
        word |= __shfl_xor_sync(kFull, word, 1);
        word |= __shfl_xor_sync(kFull, word, 2);
        word |= __shfl_xor_sync(kFull, word, 4);
        if (b < total && (lane & 7u) == 0u) {
          const uint32_t c = b / blocks_per_row, blk = b - c * blocks_per_row;
          const uint32_t w = blk * 4u + (lane >> 3);
          if (w < a.conn_words) conn[(uint64_t)c * a.conn_words + w] = word;
        }
      }
    }
    return;
  }
  const uint32_t total = a.C * a.conn_words;
  // four words per round, their loads issued together
  for (uint32_t gw0 = first; gw0 < total; gw0 += 4u * warps) {
    bool on[4];
#pragma unroll
    for (uint32_t q = 0; q < 4u; ++q) {
      const uint32_t gw = gw0 + q * warps;
      const uint32_t c = gw / a.conn_words, w = gw % a.conn_words;
      const uint32_t k = w * 32u + lane;
      on[q] = gw < total && k < a.K && __ldg(a.perm + (uint64_t)c * a.K + k) >= a.thr;
    }
#pragma unroll
    for (uint32_t q = 0; q < 4u; ++q) {
      const uint32_t gw = gw0 + q * warps;
      const uint32_t bits = __ballot_sync(kFull, on[q]);
      if (lane == 0 && gw < total) conn[gw] = bits;
    }
  }
}

}  // namespace

cudaError_t launch_conn_pack(const DenseArgs* args, uint32_t n, uint32_t max_C,
                             uint32_t max_conn_words, cudaStream_t stream) {
  const uint32_t words = max_C * max_conn_words;  // 8 warps per CTA, 16 words per warp-round
  const dim3 grid(std::max<uint32_t>(1u, std::min<uint32_t>((words + 127u) / 128u, 64u)), n, 1);
  DenseLaunch L{args, DenseArgs{}};
  sp_conn_pack_kernel<<<grid, 256, 0, stream>>>(L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_conn_pack_one(const DenseArgs& a, cudaStream_t stream) {
  const uint32_t words = a.C * a.conn_words;
  DenseLaunch L{nullptr, a};
  sp_conn_pack_kernel<<<std::max<uint32_t>(1u, std::min<uint32_t>((words + 127u) / 128u, 608u)), 256, 0, stream>>>(L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

// Two stages of 48 KB operand tiles and a 48 KB slab of packed bits: one CTA
// per SM, so its 256-column accumulator never waits for tensor memory.
size_t dense_smem_bytes() { return 2u * (kABytes + kBBytes) + kBitsBytes; }

cudaError_t dense_init() {
  return cudaFuncSetAttribute(sp_dense_overlap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)dense_smem_bytes());
}

cudaError_t launch_dense_overlap(const DenseArgs& a, cudaStream_t stream) {
  const dim3 grid((a.C + kTN - 1) / kTN, (a.n_frames + kTM - 1) / kTM, 1);
  DenseLaunch L{nullptr, a};
  sp_dense_overlap_kernel<<<grid, kThreads, dense_smem_bytes(), stream>>>(L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_dense_overlap_many(const DenseArgs* args, uint32_t n, uint32_t max_C,
                                      uint32_t max_frames, cudaStream_t stream) {
  const dim3 grid((max_C + kTN - 1) / kTN, (max_frames + kTM - 1) / kTM, n);
  DenseLaunch L{args, DenseArgs{}};
  sp_dense_overlap_kernel<<<grid, kThreads, dense_smem_bytes(), stream>>>(L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
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

cudaError_t launch_frame_inhibit(const FrameInhibitArgs& a, cudaStream_t stream) {
  InhibitLaunch L{nullptr, a};
  sp_frame_inhibit_kernel<<<a.n_frames, kStepThreads, frame_inhibit_smem(a.C, a.unit_S), stream>>>(L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_frame_inhibit_many(const FrameInhibitArgs* args, uint32_t n, uint32_t max_C,
                                      uint32_t max_unit_S, uint32_t max_frames,
                                      cudaStream_t stream) {
  InhibitLaunch L{args, FrameInhibitArgs{}};
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
