// Frame sequences of one Spatial Pooler in a single persistent launch: the
// SP state lives in the distributed shared memory of one thread-block
// cluster for the whole sequence.
//
// A sequence with learning is inherently serial (frame t+1 reads the
// permanences frame t wrote), so one SP is latency-bound, not bandwidth-bound.
// Instead of one kernel per frame reading the state from L2 each time, a
// cluster of Q CTAs (Q = 16 for 1024 columns x 256 synapses) loads the state
// once into shared memory -- CTA q owns columns [q*Cq, (q+1)*Cq) with their
// pools, permanences and boosts -- and loops over the frames:
//
//   1. the input band its columns' pools cover (a contiguous word range of
//      the packed frame) arrives in shared memory by cp.async, issued during
//      the previous frame (double-buffered);
//   2. Alg. 1 for its columns from shared memory, each warp counting four
//      columns side by side; the boosted overlaps are published in shared
//      memory;
//   3. one cluster barrier (barrier.cluster arrive.release / wait.acquire);
//   4. with global inhibition and unit boosts (counts are the overlaps),
//      each CTA has published a count histogram of its columns in step 2;
//      warp 0 of every CTA reads the cluster's histograms from the top, 32
//      bins a round, until it reaches the k-th largest count, and decides its
//      own columns; otherwise every CTA gathers all C overlaps through DSMEM
//      and runs Alg. 2 on them (the same deterministic answer in every CTA),
//      keeping the decisions for its own columns;
//   5. learning (Section 1.1) of its winning columns in shared memory, with
//      the frame band still resident.
//
// Outputs per frame: this CTA's words of the active mask and, when asked
// for, its columns' boosted overlaps; the last frame's list and overlaps.
//
// The published overlaps are double-buffered by frame parity, so one
// barrier per frame orders both the gather of frame t and the overwrite at
// frame t+2.  Permanence rows that changed are written back at the end.
// There is no software spin-wait anywhere: the cluster barrier and
// cp.async.wait_all are hardware waits, and every CTA runs the same frame
// loop, so every barrier is reached by all CTAs.
#include <cooperative_groups.h>

#include <atomic>

#include "../../include/sp.h"
#include "sp_device.cuh"
#include "sp_kernels.cuh"

namespace cg = cooperative_groups;

namespace sp {

extern std::atomic<uint64_t> g_launches;

namespace {

using dev::kFull;
using dev::learn_one;

constexpr int kSeqWarps = kSeqThreads / 32;
constexpr int kSeqCols = 4;  // columns a warp counts side by side

__device__ __forceinline__ void cp_async4(uint32_t* smem_dst, const uint32_t* gmem_src) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t* smem_dst, const uint32_t* gmem_src) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Start copying words [w_lo, w_lo + nw) of one frame into a band buffer.
__device__ __forceinline__ void issue_band(uint32_t* dst, const uint32_t* frame, uint32_t w_lo,
                                           uint32_t nw, bool vec16) {
  if (vec16) {
    for (uint32_t i = threadIdx.x * 4u; i < nw; i += kSeqThreads * 4u)
      cp_async16(dst + i, frame + w_lo + i);
  } else {
    for (uint32_t i = threadIdx.x; i < nw; i += kSeqThreads) cp_async4(dst + i, frame + w_lo + i);
  }
  cp_async_commit();
}

// Shared-memory layout of one CTA (all offsets in 4-byte words).
struct SeqLayout {
  uint32_t idx, perm, boost, band, ov, raw, hstride, hpub, all, hist, mask, dirty, total;
  __host__ __device__ SeqLayout(uint32_t Cq, uint32_t S, uint32_t band_max, uint32_t C) {
    const uint32_t CqS = Cq * S;
    idx = 0;
    perm = idx + CqS;
    boost = perm + CqS;
    band = (boost + Cq + 3u) & ~3u;  // 16-byte aligned
    ov = band + 2u * band_max;
    raw = ov + 2u * Cq;
    hstride = (S + 4u) & ~3u;         // bins 0..S, rounded up to whole 16-byte words
    hpub = (raw + Cq + 3u) & ~3u;     // [2][hstride] published count histograms, bin 0 the max
    all = hpub + 2u * hstride;
    hist = all + C;
    const uint32_t hw = (S + 1u) > 256u ? (S + 1u) : 256u;
    mask = hist + hw;
    dirty = mask + (C + 31u) / 32u;
    total = dirty + Cq / 32u;
  }
};

// Global inhibition with unit boosts, decided by warp 0 of each CTA for the
// CTA's own columns from the count histograms the CTAs publish in shared
// memory (hpub: bin b holds how many of the publishing CTA's columns count b;
// bin 0 holds its largest count).  The warp reads the Q largest counts, then
// gathers 32 bins at a time from the top (lane l: bin top - l, from every
// CTA; usually one or two rounds reach the k-th largest count T), with one
// warp scan per round for the columns above each bin, in the whole cluster
// and in the lower-ranked CTAs.  That gives T, the ties at T that still win
// (`need`) and the winners and ties of the lower-ranked CTAs.  The CTA's
// columns (count in s_raw, 0 below min_overlap) are then decided 32 at a
// time: a ballot ranks the ties in column order, another gives the mask
// word.  When list != nullptr the winners' slots of the ascending list are
// written.  Returns the cluster-wide number of winners (every lane gets it).
template <typename Cluster>
__device__ uint32_t decide_unit_global(const Cluster& cluster, const uint32_t* hpub,
                                       const uint32_t* s_raw, uint32_t k, uint32_t q,
                                       uint32_t c0, uint32_t nc, uint32_t* s_mask,
                                       uint32_t* list) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t Q = cluster.num_blocks();
  const uint32_t top0 = __reduce_max_sync(kFull, lane < Q ? cluster.map_shared_rank(hpub, lane)[0] : 0u);
  // T: 0xffffffff nobody wins; 0 every counted column wins (at most k)
  uint32_t T = 0xffffffffu, need = 0u, above_lower = 0u, ties_lower = 0u;
  uint32_t acc_g = 0u, acc_p = 0u;  // columns above the current round's bins
  if (k != 0u) {
    T = 0u;                           // reaching bin 0: at most k counted columns
    for (uint32_t top = top0; top >= 1u; top = top > 32u ? top - 32u : 0u) {
      const uint32_t bin = top >= lane + 1u ? top - lane : 0u;  // 0: past the last bin
      uint32_t v[kSeqMaxCluster];
#pragma unroll
      for (uint32_t r = 0; r < kSeqMaxCluster; ++r)
        v[r] = (r < Q && bin != 0u) ? cluster.map_shared_rank(hpub, r)[bin] : 0u;
      uint32_t g = 0u, p = 0u;
#pragma unroll
      for (uint32_t r = 0; r < kSeqMaxCluster; ++r) {
        g += v[r];
        p += r < q ? v[r] : 0u;
      }
      uint32_t ig = g, ip = p;  // inclusive sums from the top
#pragma unroll
      for (uint32_t o = 1; o < 32u; o <<= 1) {
        const uint32_t yg = __shfl_up_sync(kFull, ig, o), yp = __shfl_up_sync(kFull, ip, o);
        if (lane >= o) {
          ig += yg;
          ip += yp;
        }
      }
      const uint32_t hit = __ballot_sync(kFull, acc_g + ig - g < k && acc_g + ig >= k);
      if (hit) {
        const int src = __ffs(hit) - 1;
        T = __shfl_sync(kFull, bin, src);
        need = k - (acc_g + __shfl_sync(kFull, ig - g, src));
        above_lower = acc_p + __shfl_sync(kFull, ip - p, src);
        ties_lower = __shfl_sync(kFull, p, src);
        break;
      }
      acc_g += __shfl_sync(kFull, ig, 31);
      acc_p += __shfl_sync(kFull, ip, 31);
    }
    if (T == 0u) above_lower = acc_p;  // every counted column of the lower CTAs wins
  }
  const bool real_T = T != 0u && T != 0xffffffffu;
  const uint32_t base = above_lower + min(ties_lower, need);  // this CTA's first list slot
  uint32_t ties_before = 0u, wins_before = 0u;
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t j = 0; j < nc; j += 32u) {
    const uint32_t r = j + lane < nc ? s_raw[j + lane] : 0u;
    const bool tie = real_T && r == T;
    const uint32_t tm = __ballot_sync(kFull, tie);
    const bool win = r != 0u && T != 0xffffffffu &&
                     (T == 0u || r > T ||
                      (tie && ties_lower + ties_before + (uint32_t)__popc(tm & lt) < need));
    const uint32_t wm = __ballot_sync(kFull, win);
    if (lane == 0u) s_mask[(c0 >> 5) + (j >> 5)] = wm;
    if (list && win) list[base + wins_before + (uint32_t)__popc(wm & lt)] = c0 + j + lane;
    ties_before += (uint32_t)__popc(tm);
    wins_before += (uint32_t)__popc(wm);
  }
  // T = 0: every counted column wins, acc_g of them (every bin was summed)
  return T == 0xffffffffu ? 0u : (T == 0u ? acc_g : k);
}

__global__ void __launch_bounds__(kSeqThreads, 1) sp_seq_cluster_kernel(const SeqArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ uint32_t sh[2 * kSeqWarps];
  __shared__ uint32_t s2[8];

  const uint32_t q = cluster.block_rank();
  const uint32_t t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const uint32_t C = a.C, S = a.S, Cq = a.Cq;
  const uint32_t c0 = q * Cq;
  const uint32_t nc = C > c0 ? min(Cq, C - c0) : 0u;
  const SeqLayout L(Cq, S, a.band_max, C);
  uint32_t* s_idx = sm + L.idx;
  float* s_perm = reinterpret_cast<float*>(sm + L.perm);
  float* s_boost = reinterpret_cast<float*>(sm + L.boost);
  uint32_t* s_band = sm + L.band;
  float* s_ov = reinterpret_cast<float*>(sm + L.ov);
  uint32_t* s_raw = sm + L.raw;
  uint32_t* s_hpub = sm + L.hpub;
  uint32_t* s_all = sm + L.all;
  uint32_t* s_hist = sm + L.hist;
  uint32_t* s_mask = sm + L.mask;
  uint32_t* s_dirty = sm + L.dirty;

  // ---- load this CTA's state: pools, permanences, boosts -----------------
  const uint64_t g0 = (uint64_t)c0 * S;
  const uint32_t nCS = nc * S;
  if ((S & 3u) == 0u) {
    const uint4* gi = reinterpret_cast<const uint4*>(a.idx + g0);
    const uint4* gp = reinterpret_cast<const uint4*>(a.perm + g0);
    for (uint32_t i = t; i < nCS / 4u; i += kSeqThreads) {
      reinterpret_cast<uint4*>(s_idx)[i] = __ldg(gi + i);
      reinterpret_cast<uint4*>(s_perm)[i] = gp[i];
    }
  } else {
    for (uint32_t i = t; i < nCS; i += kSeqThreads) {
      s_idx[i] = __ldg(a.idx + g0 + i);
      s_perm[i] = a.perm[g0 + i];
    }
  }
  for (uint32_t i = t; i < nc; i += kSeqThreads) s_boost[i] = __ldg(a.boost + c0 + i);
  for (uint32_t i = t; i < Cq / 32u; i += kSeqThreads) s_dirty[i] = 0u;
  for (uint32_t i = t; i < 2u * L.hstride; i += kSeqThreads) s_hpub[i] = 0u;
  const bool fast = a.inhibition == 0u && a.unit_boost != 0u;
  // input band of this CTA: the 16-byte aligned word range covering its pools
  uint32_t mn = 0xffffffffu, mx = 0u;
  for (uint32_t i = t; i < nCS; i += kSeqThreads) {
    const uint32_t id = __ldg(a.idx + g0 + i);
    mn = min(mn, id);
    mx = max(mx, id);
  }
  mn = __reduce_min_sync(kFull, mn);
  mx = __reduce_max_sync(kFull, mx);
  if (lane == 0) {
    sh[warp] = mn;
    sh[kSeqWarps + warp] = mx;
  }
  __syncthreads();
  if (t == 0) {
    uint32_t m0 = 0xffffffffu, m1 = 0u;
    for (int w = 0; w < kSeqWarps; ++w) {
      m0 = min(m0, sh[w]);
      m1 = max(m1, sh[kSeqWarps + w]);
    }
    if (m0 > m1) m0 = m1 = 0u;  // a CTA without columns
    const uint32_t w_lo = (m0 >> 5) & ~3u;
    uint32_t w_hi = ((m1 >> 5) + 4u) & ~3u;  // exclusive, multiple of 4
    if (!a.vec16 && w_hi > a.n_words) w_hi = a.n_words;
    s2[0] = w_lo;
    s2[1] = min(w_hi - w_lo, a.band_max);
  }
  __syncthreads();
  const uint32_t w_lo = s2[0], nbw = s2[1];
  __syncthreads();

  // ---- learning left pending by the previous call ------------------------
  if (a.pend_mask) {
    for (uint32_t lc = warp; lc < nc; lc += kSeqWarps) {
      const uint32_t c = c0 + lc;
      if (!((__ldg(a.pend_mask + (c >> 5)) >> (c & 31u)) & 1u)) continue;
      for (uint32_t s = lane; s < S; s += 32) {
        const uint32_t e = lc * S + s;
        s_perm[e] = learn_one(s_perm[e], dev::input_bit(a.pend_x, s_idx[e]), a.inc, a.dec);
      }
      if (lane == 0) atomicOr(s_dirty + (lc >> 5), 1u << (lc & 31u));
    }
  }
  issue_band(s_band, a.frames, w_lo, nbw, a.vec16);

  for (uint32_t f = 0; f < a.n_frames; ++f) {
    const uint32_t par = f & 1u;
    uint32_t* band = s_band + par * a.band_max;
    float* ov_pub = s_ov + par * Cq;
    cp_async_wait_all();
    __syncthreads();  // band f visible; frame f-1 finished in this CTA
    if (f + 1u < a.n_frames)
      issue_band(s_band + (par ^ 1u) * a.band_max, a.frames + (uint64_t)(f + 1u) * a.stride,
                 w_lo, nbw, a.vec16);

    // ---- Alg. 1 for this CTA's columns --------------------------------------
    // warp w counts columns w, w + 16, w + 32, w + 48 (kSeqCols of them) side
    // by side, so the loads of all four are in flight together; lane j then
    // publishes column j's count
    uint32_t* hpub = s_hpub + par * L.hstride;
    for (uint32_t lc0 = warp; lc0 < nc; lc0 += kSeqWarps * kSeqCols) {
      uint32_t cnt[kSeqCols];
#pragma unroll
      for (int j = 0; j < kSeqCols; ++j) {
        const uint32_t lc = lc0 + (uint32_t)j * kSeqWarps;
        cnt[j] = 0u;
        if (lc < nc) {
          const uint32_t* ri = s_idx + lc * S;
          const float* rp = s_perm + lc * S;
#pragma unroll 8
          for (uint32_t s = lane; s < S; s += 32) {
            const uint32_t id = ri[s];
            const uint32_t w = (id >> 5) - w_lo;
            cnt[j] += (rp[s] >= a.thr) ? ((band[w] >> (id & 31u)) & 1u) : 0u;
          }
        }
      }
      uint32_t mine = 0u;
#pragma unroll
      for (int j = 0; j < kSeqCols; ++j) {
        const uint32_t c = __reduce_add_sync(kFull, cnt[j]);
        if (lane == (uint32_t)j) mine = c;
      }
      const uint32_t lc = lc0 + lane * kSeqWarps;
      if (lane < (uint32_t)kSeqCols && lc < nc) {
        const bool keep = mine >= a.min_overlap && mine != 0u;
        s_raw[lc] = keep ? mine : 0u;
        if (fast) {
          if (keep) {
            atomicAdd(hpub + mine, 1u);
            atomicMax(hpub, mine);  // bin 0: this CTA's largest count
          }
        } else {
          ov_pub[lc] = dev::boosted(mine, a.min_overlap, s_boost[lc]);
        }
      }
    }
    cluster.sync();  // every CTA's overlaps (or count histogram) of frame f are published
    const bool last = f + 1u == a.n_frames;
    uint32_t total;
    if (fast) {
      total = 0u;
      if (warp == 0)
        total = decide_unit_global(cluster, hpub, s_raw, a.k, q, c0, nc, s_mask,
                                   last ? a.result + 1 : nullptr);
      // the previous frame's published histogram is no longer read by anyone
      for (uint32_t b = t; b < L.hstride; b += kSeqThreads) s_hpub[(par ^ 1u) * L.hstride + b] = 0u;
    } else {

    // ---- gather all overlaps through DSMEM -------------------------------------
    {
    uint32_t nz = 0;
#pragma unroll 4
    for (uint32_t i = t; i < C; i += kSeqThreads) {
      const uint32_t owner = i / Cq;
      const float* src = cluster.map_shared_rank(ov_pub, owner);
      const uint32_t v = __float_as_uint(src[i - owner * Cq]);
      s_all[i] = v;
      nz += v != 0u;
    }
    for (uint32_t i = t; i < a.mask_words; i += kSeqThreads) s_mask[i] = 0u;
    if (a.inhibition == 0u) {
      uint32_t e0, e1, nz_tot, z;
      dev::block_scan2<kSeqWarps>(nz, 0u, e0, e1, nz_tot, z, sh);
      uint32_t T, need;
      dev::select_threshold<kSeqThreads>(s_all, C, a.k, nz_tot, nullptr,
                                         a.unit_boost ? S : 0u, s_hist, sh, s2, T, need);
      total = dev::mark_global<kSeqThreads>(s_all, C, T, need, s_mask,
                                            (last && q == 0u) ? a.result + 1 : nullptr, sh);
    } else {
      __syncthreads();
      // every CTA marks all columns: the list offsets then need no exchange
      total = dev::mark_local<kSeqThreads>(s_all, 0u, C, a.gw, a.gh, a.radius, a.k, s_mask,
                                           (last && q == 0u) ? a.result + 1 : nullptr, sh);
    }
    }
    }
    __syncthreads();
    // ---- outputs: this CTA's mask words; the last frame's list and overlaps
    const uint32_t mw0 = c0 / 32u, mw1 = min(a.mask_words, (c0 + nc + 31u) / 32u);
    if (a.masks_out)
      for (uint32_t i = mw0 + t; i < mw1; i += kSeqThreads)
        a.masks_out[(uint64_t)f * a.mask_words + i] = s_mask[i];
    if (a.ov_all)
      for (uint32_t i = t; i < nc; i += kSeqThreads)
        a.ov_all[(uint64_t)f * C + c0 + i] = fast ? __uint2float_rn(s_raw[i]) : ov_pub[i];
    if (last) {
      for (uint32_t i = mw0 + t; i < mw1; i += kSeqThreads) a.mask_last[i] = s_mask[i];
      for (uint32_t i = t; i < nc; i += kSeqThreads)
        a.ov_out[c0 + i] = fast ? __uint2float_rn(s_raw[i]) : ov_pub[i];
      if (q == 0u && t == 0u) a.result[0] = total;
    }

    if (a.duty) {
      for (uint32_t lc = t; lc < nc; lc += kSeqThreads) {
        const uint32_t c = c0 + lc;
        const float act = ((s_mask[c >> 5] >> (c & 31u)) & 1u) ? 1.0f : 0.0f;
        const float d = a.duty[c];
        a.duty[c] = __fadd_rn(d, __fdiv_rn(__fsub_rn(act, d), a.duty_period));
      }
    }

    // ---- learning of this CTA's winners (frame band still resident) ---------
    if (a.learn) {
      for (uint32_t lc = warp; lc < nc; lc += kSeqWarps) {
        const uint32_t c = c0 + lc;
        if (!((s_mask[c >> 5] >> (c & 31u)) & 1u)) continue;
        float* rp = s_perm + lc * S;
        const uint32_t* ri = s_idx + lc * S;
#pragma unroll 8
        for (uint32_t s = lane; s < S; s += 32) {
          const uint32_t id = ri[s];
          const uint32_t bit = (band[(id >> 5) - w_lo] >> (id & 31u)) & 1u;
          rp[s] = learn_one(rp[s], bit, a.inc, a.dec);
        }
        if (lane == 0) atomicOr(s_dirty + (lc >> 5), 1u << (lc & 31u));
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // ---- write back the permanence rows that changed ---------------------------
  for (uint32_t lc = warp; lc < nc; lc += kSeqWarps) {
    if (!((s_dirty[lc >> 5] >> (lc & 31u)) & 1u)) continue;
    float* gp = a.perm + g0 + (uint64_t)lc * S;
    for (uint32_t s = lane; s < S; s += 32) gp[s] = s_perm[lc * S + s];
  }
  // no CTA may exit while another can still read its shared memory
  cluster.sync();
}

}  // namespace

size_t seq_smem_bytes(uint32_t C, uint32_t S, uint32_t Cq, uint32_t band_max) {
  return (size_t)SeqLayout(Cq, S, band_max, C).total * 4u;
}

cudaError_t seq_kernel_init(size_t smem_bytes) {
  cudaError_t e = cudaFuncSetAttribute(sp_seq_cluster_kernel,
                                       cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sp_seq_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes);
}

cudaError_t seq_max_active_clusters(uint32_t Q, size_t smem_bytes, int* out) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(Q, 1, 1);
  cfg.blockDim = dim3(kSeqThreads, 1, 1);
  cfg.dynamicSmemBytes = smem_bytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(out, sp_seq_cluster_kernel, &cfg);
}

cudaError_t launch_seq(const SeqArgs& a, uint32_t Q, size_t smem_bytes, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(Q, 1, 1);
  cfg.blockDim = dim3(kSeqThreads, 1, 1);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, sp_seq_cluster_kernel, a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

}  // namespace sp
