// Host runtime behind include/sp.h: handle state on the device, stream
// ordering, pinned staging, bounded waits and argument validation.
//
// Device layout of one handle (a single cudaMalloc, every part 256-byte
// aligned): idx[C][S] u32 | perm[C][S] f32 | boost[C] | ov[C] |
// xsave[2][n_words] | mask[2][mask_words] | result[1 + C] | counter.
// The double-buffered input copies and winner masks carry one frame's
// learning over to the next frame's kernel (deferred learning).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/sp.h"
#include "../../include/sp_synth.h"
#include "sp_kernels.cuh"

namespace sp {
extern std::atomic<uint64_t> g_launches;
}

namespace {
thread_local std::string t_last_error;
}

void sp::set_last_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_last_error = buf;
}

#include "sp_internal.h"

using namespace sp::rt;

namespace sp {
namespace rt {

sp_status validate_config(const sp_config* c) {
  if (!c) return fail(SP_EINVAL, "config is NULL");
  if (c->abi_version != SP_ABI_VERSION)
    return fail(SP_EINVAL, "abi_version %u, library is %u", c->abi_version, SP_ABI_VERSION);
  const uint64_t n_in = (uint64_t)c->input_w * c->input_h;
  if (n_in == 0 || n_in > SP_MAX_INPUT_BITS) return fail(SP_EINVAL, "input size %llu", (unsigned long long)n_in);
  if (c->num_columns == 0 || c->num_columns > SP_MAX_COLUMNS)
    return fail(SP_EINVAL, "num_columns %u not in [1, %u]", c->num_columns, SP_MAX_COLUMNS);
  if (c->synapses_per_column == 0 || c->synapses_per_column > SP_MAX_SYNAPSES)
    return fail(SP_EINVAL, "synapses_per_column %u not in [1, %u]", c->synapses_per_column,
                SP_MAX_SYNAPSES);
  if ((uint64_t)c->num_columns * c->synapses_per_column > (1ull << 31))
    return fail(SP_EINVAL, "C*S too large");
  if (!std::isfinite(c->connect_threshold)) return fail(SP_EINVAL, "connect_threshold not finite");
  if (!(c->perm_inc >= 0.0f) || !(c->perm_dec >= 0.0f) || !std::isfinite(c->perm_inc) ||
      !std::isfinite(c->perm_dec))
    return fail(SP_EINVAL, "perm_inc / perm_dec must be finite and >= 0");
  if (c->inhibition > SP_INHIBIT_PAPER_LITERAL) return fail(SP_EINVAL, "inhibition %u", c->inhibition);
  if (!(c->duty_period >= 0.0f) || std::isinf(c->duty_period) || c->reserved != 0u)
    return fail(SP_EINVAL, "duty_period must be finite and >= 0, reserved 0");
  const bool grid = c->col_grid_w != 0 || c->col_grid_h != 0;
  if (grid && (uint64_t)c->col_grid_w * c->col_grid_h != c->num_columns)
    return fail(SP_EINVAL, "col_grid %ux%u != num_columns %u", c->col_grid_w, c->col_grid_h,
                c->num_columns);
  if (c->inhibition == SP_INHIBIT_LOCAL && !grid)
    return fail(SP_EINVAL, "local inhibition needs a column grid");
  return SP_OK;
}

}  // namespace rt
}  // namespace sp

namespace {

sp_status validate_seeded(const sp_config* c) {
  const uint64_t n_in = (uint64_t)c->input_w * c->input_h;
  if (!(c->perm_init_lo >= 0.0f && c->perm_init_lo <= c->perm_init_hi && c->perm_init_hi <= 1.0f))
    return fail(SP_EINVAL, "perm_init range [%g, %g] not inside [0, 1]", c->perm_init_lo,
                c->perm_init_hi);
  switch (c->pool_mode) {
    case SP_POOL_UNIFORM:
      if (c->synapses_per_column > n_in) return fail(SP_EINVAL, "S > n_in");
      return SP_OK;
    case SP_POOL_WINDOW:
      if (c->col_grid_w == 0) return fail(SP_EINVAL, "windowed pools need a column grid");
      if (c->rf_w == 0 || c->rf_h == 0 || c->rf_w > c->input_w || c->rf_h > c->input_h)
        return fail(SP_EINVAL, "receptive field %ux%u does not fit the %ux%u input", c->rf_w,
                    c->rf_h, c->input_w, c->input_h);
      if ((uint64_t)c->rf_w * c->rf_h < c->synapses_per_column)
        return fail(SP_EINVAL, "S larger than the receptive field");
      return SP_OK;
    case SP_POOL_DENSE:
      if (c->synapses_per_column != n_in) return fail(SP_EINVAL, "dense pools need S == n_in");
      return SP_OK;
    default:
      return fail(SP_EINVAL, "pool_mode %u", c->pool_mode);
  }
}

void free_handle(sp_handle* h) {
  if (!h) return;
  DeviceGuard g(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->own_stream) cudaStreamSynchronize(h->own_stream);
  if (h->s_in) cudaStreamSynchronize(h->s_in);
  if (h->s_out) cudaStreamSynchronize(h->s_out);
  for (int i = 0; i < kSlots; ++i) {
    if (h->ev_h2d[i]) cudaEventDestroy(h->ev_h2d[i]);
    if (h->ev_comp[i]) cudaEventDestroy(h->ev_comp[i]);
    if (h->ev_d2h[i]) cudaEventDestroy(h->ev_d2h[i]);
  }
  if (h->s_in) cudaStreamDestroy(h->s_in);
  if (h->s_out) cudaStreamDestroy(h->s_out);
  if (h->d_stage) cudaFree(h->d_stage);
  if (h->d_mstage) cudaFree(h->d_mstage);
  if (h->d_run_ov) cudaFree(h->d_run_ov);
  if (h->d_run_masks) cudaFree(h->d_run_masks);
  if (h->d_bimg) cudaFree(h->d_bimg);
  if (h->d_aimg) cudaFree(h->d_aimg);
  if (h->d_xspan) cudaFree(h->d_xspan);
  if (h->d_compact) cudaFree(h->d_compact);
  if (h->d_window) cudaFree(h->d_window);
  if (h->d_wband) cudaFree(h->d_wband);
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->ev_switch) cudaEventDestroy(h->ev_switch);
  if (h->ev_wait) cudaEventDestroy(h->ev_wait);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  if (h->h_result) cudaFreeHost(h->h_result);
  if (h->h_err) cudaFreeHost(h->h_err);
  if (h->d_block) cudaFree(h->d_block);
  delete h;
}

// Decide whether whole frame sequences of this SP can run in one persistent
// cluster launch: Q CTAs of Cq columns (a multiple of 32) must hold their
// pools, permanences and input bands in shared memory, and the device must
// be able to schedule such a cluster.  Failure only disables the path.
void plan_cluster_path(sp_handle* h, const uint32_t* idx) {
  h->seq_ok = false;
  if (h->cfg.inhibition == SP_INHIBIT_PAPER_LITERAL) return;  // per-frame kernel only
  uint32_t Q = (h->C + 31u) / 32u;
  if (Q > sp::kSeqMaxCluster) Q = sp::kSeqMaxCluster;
  if (Q < 2u) Q = 2u;
  const uint32_t Cq = (((h->C + Q - 1u) / Q) + 31u) & ~31u;
  if (Cq > (uint32_t)sp::kSeqThreads) return;  // one column per thread in the decision
  uint32_t band_max = 4u;
  for (uint32_t q = 0; q < Q; ++q) {
    const uint32_t c0 = q * Cq;
    if (c0 >= h->C) break;
    const uint32_t c1 = std::min(h->C, c0 + Cq);
    uint32_t mn = 0xffffffffu, mx = 0u;
    for (size_t e = (size_t)c0 * h->S; e < (size_t)c1 * h->S; ++e) {
      mn = std::min(mn, idx[e]);
      mx = std::max(mx, idx[e]);
    }
    const uint32_t w_lo = (mn >> 5) & ~3u;
    const uint32_t w_hi = ((mx >> 5) + 4u) & ~3u;
    band_max = std::max(band_max, w_hi - w_lo);
  }
  const size_t smem = sp::seq_smem_bytes(h->C, h->S, Cq, band_max);
  if (smem > kSeqSmemLimit) return;
  if (sp::seq_kernel_init(smem) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  int clusters = 0;
  if (sp::seq_max_active_clusters(Q, smem, &clusters) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return;
  }
  h->seq_ok = true;
  h->seq_Q = Q;
  h->seq_Cq = Cq;
  h->seq_band_max = band_max;
  h->seq_smem = smem;
}

// Allocate the device block, streams and events; copy idx/perm/boost.
sp_status init_handle(sp_handle* h, const sp_config* cfg, const uint32_t* idx, const float* perm,
                      const float* boost) {
  h->cfg = *cfg;
  h->C = cfg->num_columns;
  h->S = cfg->synapses_per_column;
  h->n_in = (uint64_t)cfg->input_w * cfg->input_h;
  h->n_words = (uint32_t)((h->n_in + 31) / 32);
  h->mask_words = (h->C + 31) / 32;
  h->max_active = cfg->inhibition == SP_INHIBIT_LOCAL
                      ? h->C
                      : (cfg->winners_set_size < h->C ? cfg->winners_set_size : h->C);
  if (cfg->inhibition == SP_INHIBIT_PAPER_LITERAL && cfg->winners_set_size >= h->C)
    h->max_active = h->C;  // no k-th largest among the others: the floor alone decides
  h->timeout_ms = default_timeout_ms();
  SP_CUDA(cudaGetDevice(&h->device));
  SP_CUDA(sp::kernels_init());
  SP_CUDA(sp::dense_init());
  SP_CUDA(sp::frame_inhibit_init());
  const size_t CS = (size_t)h->C * h->S;
  size_t off[11];
  size_t total = 0;
  const size_t sizes[11] = {CS * 4, CS * 4, (size_t)h->C * 4, (size_t)h->C * 4,
                            (size_t)h->n_words * 4 * 2, (size_t)h->mask_words * 4 * 2,
                            ((size_t)h->C + 1) * 4, 4, ((size_t)h->S + 1) * 4,
                            (size_t)h->C * 4, 4};
  for (int i = 0; i < 11; ++i) {
    off[i] = total;
    total += align256(sizes[i]);
  }
  SP_CUDA(device_malloc((void**)&h->d_block, total));
  h->device_bytes = total;
  char* b = static_cast<char*>(h->d_block);
  h->d_idx = reinterpret_cast<uint32_t*>(b + off[0]);
  h->d_perm = reinterpret_cast<float*>(b + off[1]);
  h->d_boost = reinterpret_cast<float*>(b + off[2]);
  h->d_ov = reinterpret_cast<float*>(b + off[3]);
  h->d_xsave[0] = reinterpret_cast<uint32_t*>(b + off[4]);
  h->d_xsave[1] = h->d_xsave[0] + h->n_words;
  h->d_mask[0] = reinterpret_cast<uint32_t*>(b + off[5]);
  h->d_mask[1] = h->d_mask[0] + h->mask_words;
  h->d_result = reinterpret_cast<uint32_t*>(b + off[6]);
  h->d_counter = reinterpret_cast<uint32_t*>(b + off[7]);
  h->d_hist = reinterpret_cast<uint32_t*>(b + off[8]);
  h->d_duty = reinterpret_cast<float*>(b + off[9]);
  h->d_err = reinterpret_cast<uint32_t*>(b + off[10]);
  SP_CUDA(cudaMallocHost(&h->h_result, ((size_t)h->C + 1) * 4));
  SP_CUDA(cudaMallocHost(&h->h_err, 4));
  *h->h_err = 0u;
  SP_CUDA(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
  h->stream = h->own_stream;
  SP_CUDA(cudaEventCreateWithFlags(&h->ev_switch, cudaEventDisableTiming));
  SP_CUDA(cudaEventCreateWithFlags(&h->ev_wait, cudaEventDisableTiming));
  SP_CUDA(cudaMemsetAsync(h->d_block, 0, total, h->stream));
  SP_CUDA(cudaMemcpyAsync(h->d_idx, idx, CS * 4, cudaMemcpyHostToDevice, h->stream));
  SP_CUDA(cudaMemcpyAsync(h->d_perm, perm, CS * 4, cudaMemcpyHostToDevice, h->stream));
  std::vector<float> ones;
  if (!boost) {
    ones.assign(h->C, 1.0f);
    boost = ones.data();
  }
  h->unit_boost = all_ones(boost, h->C);
  h->dense = h->S == h->n_in;
  for (size_t e = 0; h->dense && e < CS; ++e) h->dense = idx[e] == (uint32_t)(e % h->S);
  SP_CUDA(cudaMemcpyAsync(h->d_boost, boost, (size_t)h->C * 4, cudaMemcpyHostToDevice, h->stream));
  SP_CUDA(cudaStreamSynchronize(h->stream));
  h->grid = sp::step_grid(h->C);
  plan_cluster_path(h, idx);
  return SP_OK;
}

// Bounded wait for everything enqueued so far on the handle's stream.
sp_status wait_handle(sp_handle* h) {
  if (h->dense_used) {
    // a tensor-core run reports an expired bounded wait through d_err
    SP_CUDA(cudaMemcpyAsync(h->h_err, h->d_err, 4, cudaMemcpyDeviceToHost, h->stream));
  }
  SP_CUDA(cudaEventRecord(h->ev_wait, h->stream));
  const auto deadline =
      std::chrono::steady_clock::now() + std::chrono::milliseconds(h->timeout_ms);
  for (uint32_t spin = 0;; ++spin) {
    const cudaError_t e = cudaEventQuery(h->ev_wait);
    if (e == cudaSuccess) {
      if (h->dense_used && *h->h_err != 0u)
        return fail(SP_ETIMEOUT, "a tensor-core kernel gave up waiting for its MMAs");
      return SP_OK;
    }
    if (e != cudaErrorNotReady)
      return fail(SP_ECUDA, "device work failed: %s", cudaGetErrorString(e));
    if (std::chrono::steady_clock::now() > deadline)
      return fail(SP_ETIMEOUT, "wait exceeded %u ms", h->timeout_ms);
    if (spin < 2000)
      std::this_thread::yield();
    else
      std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// Order the handle's work on stream s after everything enqueued before.
sp_status use_stream(sp_handle* h, cudaStream_t s) {
  if (!s) s = h->own_stream;
  if (s != h->stream) {
    SP_CUDA(cudaEventRecord(h->ev_switch, h->stream));
    SP_CUDA(cudaStreamWaitEvent(s, h->ev_switch, 0));
    h->stream = s;
  }
  return SP_OK;
}

sp::StepArgs base_args(const sp_handle* h) {
  sp::StepArgs a{};
  a.idx = h->d_idx;
  a.perm = h->d_perm;
  a.boost = h->d_boost;
  a.ov = h->d_ov;
  a.result = h->d_result;
  a.counter = h->d_counter;
  a.hist = (h->unit_boost && h->cfg.inhibition == SP_INHIBIT_GLOBAL) ? h->d_hist : nullptr;
  a.duty = h->cfg.duty_period > 0.0f ? h->d_duty : nullptr;
  a.duty_period = h->cfg.duty_period;
  a.C = h->C;
  a.S = h->S;
  a.n_words = h->n_words;
  a.mask_words = h->mask_words;
  a.thr = h->cfg.connect_threshold;
  a.inc = h->cfg.perm_inc;
  a.dec = h->cfg.perm_dec;
  a.min_overlap = h->cfg.min_overlap;
  a.k = h->cfg.winners_set_size;
  a.inhibition = h->cfg.inhibition;
  a.gw = h->cfg.col_grid_w;
  a.gh = h->cfg.col_grid_h;
  a.radius = h->cfg.local_radius;
  return a;
}

// Enqueue one frame: x is this frame's input (device); x_prev the previous
// frame's (used iff learning is pending); x_save, if set, receives a copy of
// x for the next frame's learning.
sp_status enqueue_frame(sp_handle* h, cudaStream_t st, const uint32_t* x, const uint32_t* x_prev,
                        uint32_t* x_save, int learn, uint32_t* mask_copy, float* ov_copy = nullptr) {
  sp::StepArgs a = base_args(h);
  a.ov_copy = ov_copy;
  const int cur = h->cur;
  a.x = x;
  if (h->pending) {
    a.x_prev = x_prev;
    a.mask_prev = h->d_mask[cur ^ 1];
  }
  a.x_save = x_save;
  a.mask_out = h->d_mask[cur];
  a.mask_copy = mask_copy;
  SP_CUDA(sp::launch_step(a, h->grid, st));
  h->pending = learn != 0;
  if (learn) h->bimg_stale = true;  // the deferred update will change the permanences
  h->cur = cur ^ 1;
  h->frames++;
  return SP_OK;
}

// Apply pending learning now (before reading permanences).
sp_status flush_learning(sp_handle* h) {
  if (!h->pending) return SP_OK;
  sp::LearnArgs l{};
  l.idx = h->d_idx;
  l.perm = h->d_perm;
  l.x = h->d_xsave[h->cur ^ 1];
  l.mask = h->d_mask[h->cur ^ 1];
  l.C = h->C;
  l.S = h->S;
  l.inc = h->cfg.perm_inc;
  l.dec = h->cfg.perm_dec;
  SP_CUDA(sp::launch_learn(l, h->stream));
  h->pending = false;
  return SP_OK;
}

// Enqueue frames x_base + t * stride (t < n) on `st`, from the handle's
// current (parity, pending) state.  Within the call the previous frame is
// read in place; the last frame is saved when learning, for the next call.
sp_status enqueue_sequence(sp_handle* h, cudaStream_t st, const uint32_t* x_base, uint32_t n,
                           uint64_t stride, int learn, uint32_t* masks, float* ovs) {
  for (uint32_t t = 0; t < n; ++t) {
    const uint32_t* x = x_base + (uint64_t)t * stride;
    const uint32_t* x_prev = t ? x - stride : h->d_xsave[h->cur ^ 1];
    uint32_t* x_save = (learn && t + 1 == n) ? h->d_xsave[h->cur] : nullptr;
    uint32_t* mc = masks ? masks + (uint64_t)t * h->mask_words : nullptr;
    float* oc = ovs ? ovs + (uint64_t)t * h->C : nullptr;
    sp_status s = enqueue_frame(h, st, x, x_prev, x_save, learn, mc, oc);
    if (s != SP_OK) return s;
  }
  return SP_OK;
}

// Run a frame sequence on the handle's stream: replay its recorded graph if
// this exact sequence was seen before, else record it on the private capture
// stream first.  Short sequences, or SP_DISABLE_GRAPHS=1, launch directly.
// Scratch of a dense inference run of n frames: overlaps, masks, connected bits.
sp_status ensure_dense_buffers(sp_handle* h, uint32_t n) {
  if (n > h->run_cap) {
    if (h->d_run_ov) cudaFree(h->d_run_ov);
    if (h->d_run_masks) cudaFree(h->d_run_masks);
    h->d_run_ov = nullptr;
    h->d_run_masks = nullptr;
    h->run_cap = 0;
    SP_CUDA(device_malloc((void**)&h->d_run_ov, (size_t)n * h->C * 4));
    SP_CUDA(device_malloc((void**)&h->d_run_masks, (size_t)n * h->mask_words * 4));
    h->run_cap = n;
    h->run_gen += 1;
  }
  const size_t abytes = sp::dense_aimg_bytes(n, h->S);
  if (abytes > h->aimg_cap) {
    if (h->d_aimg) cudaFree(h->d_aimg);
    h->d_aimg = nullptr;
    h->aimg_cap = 0;
    SP_CUDA(device_malloc((void**)&h->d_aimg, abytes));
    h->aimg_cap = abytes;
  }
  if (!h->d_bimg) {
    SP_CUDA(device_malloc((void**)&h->d_bimg, sp::dense_bimg_bytes(h->C, h->S)));
    h->bimg_stale = true;
  }
  return SP_OK;
}

// The arguments of a dense run of n frames at x_base (the connection image is
// rebuilt first when the permanences may have changed since it was built).
sp::DenseArgs dense_args(sp_handle* h, const uint32_t* x_base, uint32_t n, uint64_t stride) {
  sp::DenseArgs d{};
  d.perm = h->d_perm;
  d.bimg = h->d_bimg;
  d.aimg = h->d_aimg;
  d.n_slices = sp::dense_slices(h->S);
  d.pack = h->bimg_stale ? 1u : 0u;
  d.boost = h->d_boost;
  d.frames = x_base;
  d.stride = stride;
  d.n_frames = n;
  d.C = h->C;
  d.K = h->S;
  d.n_words = h->n_words;
  d.thr = h->cfg.connect_threshold;
  d.min_overlap = h->cfg.min_overlap;
  d.ov = h->d_run_ov;
  d.err = h->d_err;
  return d;
}

sp_status run_dense(sp_handle* h, const uint32_t* x_base, uint32_t n, uint64_t stride,
                    uint32_t* masks, float* ovs) {
  sp_status s = flush_learning(h);
  if (s != SP_OK) return s;
  if ((s = ensure_dense_buffers(h, n)) != SP_OK) return s;
  const sp::DenseArgs d = dense_args(h, x_base, n, stride);
  if (d.pack) SP_CUDA(sp::launch_conn_image_one(d, h->stream));
  h->bimg_stale = false;
  SP_CUDA(sp::launch_frame_image_one(d, h->stream));
  SP_CUDA(sp::launch_dense_overlap(d, h->stream));
  h->dense_used = true;
  const bool duty = h->cfg.duty_period > 0.0f;
  sp::FrameInhibitArgs f{};
  f.ov = h->d_run_ov;
  f.n_frames = n;
  f.C = h->C;
  f.mask_words = h->mask_words;
  f.k = h->cfg.winners_set_size;
  f.inhibition = h->cfg.inhibition;
  f.gw = h->cfg.col_grid_w;
  f.gh = h->cfg.col_grid_h;
  f.radius = h->cfg.local_radius;
  f.unit_S = h->unit_boost ? h->S : 0u;
  if (sp::frame_inhibit_smem(h->C, f.unit_S) > sp::frame_inhibit_smem_limit()) f.unit_S = 0u;
  if (sp::frame_inhibit_smem(h->C, 0u) > sp::frame_inhibit_smem_limit())
    return fail(SP_ENOTSUP, "too many columns for the per-frame inhibition kernel");
  f.masks_out = masks ? masks : (duty ? h->d_run_masks : nullptr);
  f.masks_stride = h->mask_words;
  f.mask_last = h->d_mask[h->cur];
  f.result = h->d_result;
  f.ov_last = h->d_ov;
  SP_CUDA(sp::launch_frame_inhibit(f, h->stream));
  if (duty)
    SP_CUDA(sp::launch_duty_run(f.masks_out, n, h->mask_words, h->C, h->d_duty,
                                h->cfg.duty_period, h->stream));
  if (ovs)  // the run's overlaps, every frame, for the caller's record
    SP_CUDA(cudaMemcpyAsync(ovs, h->d_run_ov, (size_t)n * h->C * 4, cudaMemcpyDeviceToDevice,
                            h->stream));
  h->pending = false;
  h->cur ^= 1;
  h->frames += n;
  return SP_OK;
}

sp_status run_sequence(sp_handle* h, const uint32_t* x_base, uint32_t n, uint64_t stride,
                       int learn, uint32_t* masks, float* ovs = nullptr) {
  if (learn) h->bimg_stale = true;
  if (!learn && h->dense && n >= kDenseMinFrames && dense_enabled())
    return run_dense(h, x_base, n, stride, masks, ovs);
  if (h->seq_ok && n >= kSeqMinFrames && seq_enabled()) {
    sp::SeqArgs a{};
    a.idx = h->d_idx;
    a.perm = h->d_perm;
    a.boost = h->d_boost;
    a.frames = x_base;
    a.stride = stride;
    a.n_frames = n;
    a.learn = learn;
    if (h->pending) {
      a.pend_mask = h->d_mask[h->cur ^ 1];
      a.pend_x = h->d_xsave[h->cur ^ 1];
    }
    a.masks_out = masks;
    a.mask_last = h->d_mask[h->cur];
    a.result = h->d_result;
    a.ov_out = h->d_ov;
    a.ov_all = ovs;
    a.C = h->C;
    a.S = h->S;
    a.n_words = h->n_words;
    a.mask_words = h->mask_words;
    a.Cq = h->seq_Cq;
    a.band_max = h->seq_band_max;
    a.vec16 = (h->n_words % 4u == 0u && stride % 4u == 0u &&
               reinterpret_cast<uintptr_t>(x_base) % 16u == 0u) ? 1u : 0u;
    a.thr = h->cfg.connect_threshold;
    a.inc = h->cfg.perm_inc;
    a.dec = h->cfg.perm_dec;
    a.min_overlap = h->cfg.min_overlap;
    a.k = h->cfg.winners_set_size;
    a.inhibition = h->cfg.inhibition;
    a.gw = h->cfg.col_grid_w;
    a.gh = h->cfg.col_grid_h;
    a.radius = h->cfg.local_radius;
    a.unit_boost = h->unit_boost ? 1u : 0u;
    a.duty = h->cfg.duty_period > 0.0f ? h->d_duty : nullptr;
    a.duty_period = h->cfg.duty_period;
    SP_CUDA(sp::launch_seq(a, h->seq_Q, h->seq_smem, h->stream));
    h->pending = false;  // learning of every frame is already applied
    h->cur ^= 1;
    h->frames += n;
    return SP_OK;
  }
  if (n < kGraphMinFrames || !graphs_enabled())
    return enqueue_sequence(h, h->stream, x_base, n, stride, learn, masks, ovs);
  const GraphKey key{x_base, n, stride, learn, masks, h->cur, h->pending, h->unit_boost, 0, 0,
                     ovs};
  GraphEntry* e = nullptr;
  for (auto& g : h->graphs)
    if (g.key == key) e = &g;
  if (!e) {
    if (!h->cap_stream) SP_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const int cur0 = h->cur;
    const bool pending0 = h->pending;
    const uint64_t frames0 = h->frames;
    SP_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    sp_status s = enqueue_sequence(h, h->cap_stream, x_base, n, stride, learn, masks, ovs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &graph);
    sp::g_launches.fetch_sub(n, std::memory_order_relaxed);  // recorded, not launched
    h->cur = cur0;
    h->pending = pending0;
    h->frames = frames0;
    if (s != SP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (ec != cudaSuccess) return fail(SP_ECUDA, "recording the frame sequence: %s", cudaGetErrorString(ec));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(SP_ECUDA, "instantiating the frame sequence: %s", cudaGetErrorString(ei));
    if (h->graphs.size() >= kGraphCacheSize) {
      size_t lru = 0;
      for (size_t i = 1; i < h->graphs.size(); ++i)
        if (h->graphs[i].last_use < h->graphs[lru].last_use) lru = i;
      cudaGraphExecDestroy(h->graphs[lru].exec);
      h->graphs.erase(h->graphs.begin() + lru);
    }
    h->graphs.push_back(GraphEntry{key, exec, 0});
    e = &h->graphs.back();
  }
  e->last_use = ++h->graph_clock;
  SP_CUDA(cudaGraphLaunch(e->exec, h->stream));
  sp::g_launches.fetch_add(n, std::memory_order_relaxed);
  h->pending = learn != 0;
  h->cur ^= (int)(n & 1u);
  h->frames += n;
  return SP_OK;
}


bool finite_nonneg(const float* v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!(v[i] >= 0.0f) || std::isinf(v[i])) return false;
  return true;
}

}  // namespace

namespace sp {
namespace rt {

bool all_ones(const float* v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (v[i] != 1.0f) return false;
  return true;
}

sp_status handle_wait(sp_handle* h) { return wait_handle(h); }
sp_status handle_flush_learning(sp_handle* h) { return flush_learning(h); }

// The descriptor of one SP inside a multi-SP launch.
// The input-word span of each of the handle's batch CTAs (computed once per
// CTA split, since pools never change); nullptr if it cannot be had, which
// only turns the staging of input words off.
const uint32_t* handle_xspan(sp_handle* h, uint32_t n_ctas) {
  if (h->d_xspan && h->xspan_ctas == n_ctas) return h->d_xspan;
  if (h->d_xspan) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->d_xspan);
    h->d_xspan = nullptr;
    h->xspan_ctas = 0;
  }
  DeviceGuard g(h->device);
  if (device_malloc((void**)&h->d_xspan, (size_t)n_ctas * 8) != cudaSuccess) {
    h->d_xspan = nullptr;
    return nullptr;
  }
  if (sp::launch_xspan(h->d_idx, h->C, h->S, n_ctas, h->d_xspan, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaFree(h->d_xspan);
    h->d_xspan = nullptr;
    return nullptr;
  }
  h->xspan_ctas = n_ctas;
  return h->d_xspan;
}

// Derive the compact form of the handle's pools and connectivity from its
// current state (S <= 256, every pool spanning at most 65536 inputs; rows
// padded to a multiple of 32 synapses); false if the SP does not qualify or
// the form cannot be had, which leaves batches on the full form.
// SP_BATCH_COMPACT=0 turns it off.
bool handle_compact(sp_handle* h) {
  if (const char* e = std::getenv("SP_BATCH_COMPACT"))
    if (e[0] == '0') return false;
  if (h->S > 256u) return false;
  DeviceGuard g(h->device);
  const size_t CS = (size_t)h->C * ((h->S + 31u) & ~31u);  // rows padded to 32 synapses
  const size_t b_cidx = align256(CS * 2), b_base = align256((size_t)h->C * 4),
               b_conn = align256(CS / 8);
  if (!h->d_compact) {
    if (device_malloc(&h->d_compact, b_cidx + b_base + b_conn + 256) != cudaSuccess) {
      h->d_compact = nullptr;
      return false;
    }
    char* p = static_cast<char*>(h->d_compact);
    h->d_cidx = reinterpret_cast<uint16_t*>(p);
    h->d_cbase = reinterpret_cast<uint32_t*>(p + b_cidx);
    h->d_cconn = reinterpret_cast<uint32_t*>(p + b_cidx + b_base);
    h->d_cwide = reinterpret_cast<uint32_t*>(p + b_cidx + b_base + b_conn);
  }
  uint32_t wide = 1;
  if (cudaMemsetAsync(h->d_cwide, 0, 4, h->stream) != cudaSuccess ||
      sp::launch_compact(h->d_idx, h->d_perm, h->C, h->S, h->cfg.connect_threshold, h->d_cidx,
                         h->d_cbase, h->d_cconn, h->d_cwide, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(&wide, h->d_cwide, 4, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return false;
  return wide == 0;
}

// Shared memory a batch launch may give a window-form CTA for its frame
// rows, bitmap rings and learning scratch (SP_BATCH_WINDOW_KB, 0..160; 0
// turns the window form off).  An SP whose CTAs would need more runs on the
// compact form: the whole launch takes the largest member's figure, so a
// wide band would cost every CTA occupancy.
uint32_t window_cap_bytes() {
  uint32_t kb = 48u;
  if (const char* e = std::getenv("SP_BATCH_WINDOW_KB")) {
    const long v = std::strtol(e, nullptr, 10);
    if (v >= 0 && v <= 160) kb = (uint32_t)v;
  }
  return kb << 10;
}

// Frame bands of the handle's window form for an n_ctas split; the shared
// memory the widest needs, or 0 if they cannot be had.
uint32_t window_bands(sp_handle* h, uint32_t n_ctas) {
  if (h->wband_ctas != n_ctas) {
    if (h->d_wband) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->d_wband);
      h->d_wband = nullptr;
      h->wband_ctas = 0;
    }
    if (device_malloc((void**)&h->d_wband, (size_t)n_ctas * 8) != cudaSuccess) {
      h->d_wband = nullptr;
      return 0u;
    }
    h->wband_ctas = n_ctas;
  }
  std::vector<uint32_t> band((size_t)n_ctas * 2);
  if (sp::launch_window_bands(h->d_worg, h->C, h->cfg.input_h, n_ctas, h->d_wband, h->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(band.data(), h->d_wband, band.size() * 4, cudaMemcpyDeviceToHost,
                      h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return 0u;
  uint32_t rows = 0;
  for (uint32_t b = 0; b < n_ctas; ++b) rows = std::max(rows, band[2 * b + 1]);
  return sp::window_smem_bytes(rows, h->cfg.input_w / 32u);
}

// Derive the window form of the handle's pools and connectivity from its
// current state (every pool inside a 64 x 64 box of a frame whose width is a
// multiple of 32) and the frame bands of an n_ctas split; false if the SP
// does not qualify, the bands exceed the cap or the form cannot be had.
// SP_BATCH_WINDOW_KB=0 turns it off.
bool handle_window(sp_handle* h, uint32_t n_ctas, uint32_t* win_bytes) {
  const uint32_t cap = window_cap_bytes();
  if (cap == 0u || h->window_geom == 0) return false;
  // a column streams 516 bytes in the window form; it pays only where the
  // other forms stream about as much (large pools), since a small pool is
  // cheaper as offsets (2 bytes and a bit per synapse) or indices and
  // permanences (8 bytes per synapse)
  const bool compact_shape = h->S <= 256u;
  const double other = compact_shape ? 2.125 * ((h->S + 31u) & ~31u) + 4.0 : 8.0 * h->S;
  if (516.0 > 1.1 * other) return false;
  const uint32_t W = h->cfg.input_w;
  if (W % 32u != 0u || h->S > 4096u) {
    h->window_geom = 0;
    return false;
  }
  if ((h->C + n_ctas - 1u) / n_ctas > 256u) return false;  // a CTA holds at most 256 columns
  DeviceGuard g(h->device);
  if (!h->d_window) {
    const size_t b_org = align256((size_t)h->C * 4), b_bits = align256((size_t)h->C * 512);
    if (device_malloc(&h->d_window, b_org + b_bits + 256) != cudaSuccess) {
      h->d_window = nullptr;
      return false;
    }
    char* p = static_cast<char*>(h->d_window);
    h->d_worg = reinterpret_cast<uint32_t*>(p);
    h->d_wbits = reinterpret_cast<uint32_t*>(p + b_org);
    h->d_wbad = reinterpret_cast<uint32_t*>(p + b_org + b_bits);
  }
  uint32_t bad = 1;
  if (cudaMemsetAsync(h->d_wbad, 0, 4, h->stream) != cudaSuccess ||
      sp::launch_window(h->d_idx, h->d_perm, h->C, h->S, W, h->cfg.connect_threshold, h->d_worg,
                        h->d_wbits, h->d_wbad, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(&bad, h->d_wbad, 4, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return false;
  h->window_geom = bad ? 0 : 1;
  if (bad) return false;
  const uint32_t need = window_bands(h, n_ctas);
  if (need == 0u || need > cap) return false;
  if (win_bytes) *win_bytes = need;
  return true;
}

bool window_rebands(sp_handle* h, sp::BatchDesc* d, uint32_t* win_bytes) {
  if (!d->worg) return false;
  DeviceGuard g(h->device);
  const uint32_t need = (h->C + d->n_ctas - 1u) / d->n_ctas > 256u ? 0u : window_bands(h, d->n_ctas);
  if (need == 0u || need > window_cap_bytes()) {
    d->worg = nullptr;
    d->wbits = nullptr;
    d->wband = nullptr;
    return false;
  }
  d->wband = h->d_wband;
  if (win_bytes) *win_bytes = need;
  return true;
}

void fill_desc(sp_handle* h, sp::BatchDesc* d, uint32_t cols_per_warp, uint32_t* win_bytes) {
  *d = sp::BatchDesc{};
  d->idx = h->d_idx;
  d->perm = h->d_perm;
  d->boost = h->d_boost;
  d->ov = h->d_ov;
  d->xsave0 = h->d_xsave[0];
  d->xsave1 = h->d_xsave[1];
  d->mask0 = h->d_mask[0];
  d->mask1 = h->d_mask[1];
  d->result = h->d_result;
  d->counter = h->d_counter;
  d->hist = (h->unit_boost && h->cfg.inhibition == SP_INHIBIT_GLOBAL) ? h->d_hist : nullptr;
  d->duty = h->cfg.duty_period > 0.0f ? h->d_duty : nullptr;
  d->duty_period = h->cfg.duty_period;
  d->C = h->C;
  d->S = h->S;
  d->n_words = h->n_words;
  d->mask_words = h->mask_words;
  d->thr = h->cfg.connect_threshold;
  d->inc = h->cfg.perm_inc;
  d->dec = h->cfg.perm_dec;
  d->min_overlap = h->cfg.min_overlap;
  d->k = h->cfg.winners_set_size;
  d->inhibition = h->cfg.inhibition;
  d->gw = h->cfg.col_grid_w;
  d->gh = h->cfg.col_grid_h;
  d->radius = h->cfg.local_radius;
  d->n_ctas = batch_ctas(h->C, h->S, cols_per_warp);
  d->xspan = batch_xspan_cap() > 0u ? handle_xspan(h, d->n_ctas) : nullptr;
  if (win_bytes) *win_bytes = 0u;
  if (handle_window(h, d->n_ctas, win_bytes)) {
    d->worg = h->d_worg;
    d->wbits = h->d_wbits;
    d->wband = h->d_wband;
    d->wpr = h->cfg.input_w / 32u;
    d->win_w = h->cfg.input_w;
  } else if (handle_compact(h)) {
    d->cidx = h->d_cidx;
    d->cbase = h->d_cbase;
    d->conn = h->d_cconn;
  }
}

}  // namespace rt
}  // namespace sp

extern "C" {

SP_API sp_status sp_config_init(sp_config* cfg) {
  if (!cfg) return fail(SP_EINVAL, "cfg is NULL");
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->abi_version = SP_ABI_VERSION;
  cfg->input_w = 240;
  cfg->input_h = 134;
  cfg->num_columns = 2048;
  cfg->synapses_per_column = 128;
  cfg->pool_mode = SP_POOL_UNIFORM;
  cfg->connect_threshold = 0.2f;
  cfg->perm_inc = 0.1f;
  cfg->perm_dec = 0.1f;
  cfg->perm_init_lo = 0.21f;
  cfg->perm_init_hi = 0.21f;
  cfg->min_overlap = 8;
  cfg->winners_set_size = 40;
  cfg->inhibition = SP_INHIBIT_GLOBAL;
  cfg->seed = 1;
  return SP_OK;
}

SP_API sp_status sp_create(const sp_config* cfg, sp_handle** out) {
  if (!out) return fail(SP_EINVAL, "out is NULL");
  *out = nullptr;
  sp_status s = validate_config(cfg);
  if (s != SP_OK) return s;
  if ((s = validate_seeded(cfg)) != SP_OK) return s;
  const uint32_t C = cfg->num_columns, S = cfg->synapses_per_column;
  const uint64_t n_in = (uint64_t)cfg->input_w * cfg->input_h;
  std::vector<uint32_t> idx((size_t)C * S);
  std::vector<float> perm((size_t)C * S);
  const uint64_t pool_seed = synth_derive_seed(cfg->seed, SYNTH_PURPOSE_POOL, 0);
  const uint64_t perm_seed = synth_derive_seed(cfg->seed, SYNTH_PURPOSE_PERM, 0);
  int rc = -1;
  if (cfg->pool_mode == SP_POOL_UNIFORM) {
    std::vector<uint32_t> scratch(n_in);
    rc = synth_pool_uniform(pool_seed, C, S, (uint32_t)n_in, idx.data(), scratch.data());
  } else if (cfg->pool_mode == SP_POOL_WINDOW) {
    std::vector<uint32_t> scratch((size_t)cfg->rf_w * cfg->rf_h);
    rc = synth_pool_window(pool_seed, cfg->col_grid_w, cfg->col_grid_h, cfg->input_w,
                           cfg->input_h, cfg->rf_w, cfg->rf_h, S, idx.data(), scratch.data());
  } else {
    rc = synth_pool_dense(C, (uint32_t)n_in, idx.data());
  }
  if (rc != 0) return fail(SP_EINVAL, "pool generation rejected the configuration");
  if (synth_perm_uniform(perm_seed, (uint64_t)C * S, cfg->perm_init_lo, cfg->perm_init_hi,
                         perm.data()) != 0)
    return fail(SP_EINVAL, "permanence generation rejected the configuration");
  sp_handle* h = new (std::nothrow) sp_handle();
  if (!h) return fail(SP_ENOMEM, "host allocation");
  s = init_handle(h, cfg, idx.data(), perm.data(), nullptr);
  if (s != SP_OK) {
    free_handle(h);
    return s;
  }
  *out = h;
  return SP_OK;
}

SP_API sp_status sp_create_from_state(const sp_config* cfg, const uint32_t* idx, const float* perm,
                                      const float* boost, sp_handle** out) {
  if (!out) return fail(SP_EINVAL, "out is NULL");
  *out = nullptr;
  sp_status s = validate_config(cfg);
  if (s != SP_OK) return s;
  if (!idx || !perm) return fail(SP_EINVAL, "idx / perm is NULL");
  const size_t CS = (size_t)cfg->num_columns * cfg->synapses_per_column;
  const uint64_t n_in = (uint64_t)cfg->input_w * cfg->input_h;
  for (size_t i = 0; i < CS; ++i) {
    if (idx[i] >= n_in) return fail(SP_EINVAL, "idx[%zu] = %u >= n_in %llu", i, idx[i], (unsigned long long)n_in);
    if (!(perm[i] >= 0.0f && perm[i] <= 1.0f)) return fail(SP_EINVAL, "perm[%zu] not in [0, 1]", i);
  }
  if (boost && !finite_nonneg(boost, cfg->num_columns))
    return fail(SP_EINVAL, "boost must be finite and >= 0");
  sp_handle* h = new (std::nothrow) sp_handle();
  if (!h) return fail(SP_ENOMEM, "host allocation");
  s = init_handle(h, cfg, idx, perm, boost);
  if (s != SP_OK) {
    free_handle(h);
    return s;
  }
  *out = h;
  return SP_OK;
}

SP_API void sp_destroy(sp_handle* h) {
  if (h && h->batch) return;  // still a batch member: the batch must be destroyed first
  free_handle(h);
}

SP_API sp_status sp_get_info(const sp_handle* h, sp_info* out) {
  if (!h || !out) return fail(SP_EINVAL, "NULL argument");
  out->num_columns = h->C;
  out->synapses_per_column = h->S;
  out->input_bits = h->n_in;
  out->input_words = h->n_words;
  out->mask_words = h->mask_words;
  out->max_active = h->max_active;
  out->device = h->device;
  out->device_bytes = h->device_bytes;
  out->frames = h->frames;
  return SP_OK;
}

SP_API sp_status sp_compute(sp_handle* h, const uint32_t* input_bits, int learn) {
  if (!h || !input_bits) return fail(SP_EINVAL, "NULL argument");
  if (h->batch) return fail(SP_EBUSY, "the handle is a member of a batch");
  DeviceGuard g(h->device);
  sp_status s = use_stream(h, h->own_stream);
  if (s != SP_OK) return s;
  uint32_t* dst = h->d_xsave[h->cur];
  SP_CUDA(cudaMemcpyAsync(dst, input_bits, (size_t)h->n_words * 4, cudaMemcpyHostToDevice,
                          h->stream));
  return enqueue_frame(h, h->stream, dst, h->d_xsave[h->cur ^ 1], nullptr, learn, nullptr);
}

SP_API sp_status sp_compute_device(sp_handle* h, const uint32_t* d_bits, int learn, void* stream) {
  if (!h || !d_bits) return fail(SP_EINVAL, "NULL argument");
  if (h->batch) return fail(SP_EBUSY, "the handle is a member of a batch");
  if (reinterpret_cast<uintptr_t>(d_bits) % 4u) return fail(SP_EINVAL, "d_bits not 4-byte aligned");
  DeviceGuard g(h->device);
  sp_status s = use_stream(h, static_cast<cudaStream_t>(stream));
  if (s != SP_OK) return s;
  return enqueue_frame(h, h->stream, d_bits, h->d_xsave[h->cur ^ 1],
                       learn ? h->d_xsave[h->cur] : nullptr, learn, nullptr);
}

SP_API sp_status sp_compute_frames_overlaps_device(sp_handle* h, const uint32_t* d_frames,
                                                   uint32_t n_frames, uint64_t stride, int learn,
                                                   uint32_t* d_active_masks, float* d_overlaps,
                                                   void* stream) {
  if (!h || (!d_frames && n_frames)) return fail(SP_EINVAL, "NULL argument");
  if (h->batch) return fail(SP_EBUSY, "the handle is a member of a batch");
  if (n_frames == 0) return SP_OK;
  if (stride < h->n_words) return fail(SP_EINVAL, "frame stride %llu < %u words", (unsigned long long)stride, h->n_words);
  if (reinterpret_cast<uintptr_t>(d_frames) % 4u || reinterpret_cast<uintptr_t>(d_active_masks) % 4u ||
      reinterpret_cast<uintptr_t>(d_overlaps) % 4u)
    return fail(SP_EINVAL, "device pointers must be 4-byte aligned");
  DeviceGuard g(h->device);
  sp_status s = use_stream(h, static_cast<cudaStream_t>(stream));
  if (s != SP_OK) return s;
  return run_sequence(h, d_frames, n_frames, stride, learn, d_active_masks, d_overlaps);
}

SP_API sp_status sp_compute_frames_device(sp_handle* h, const uint32_t* d_frames, uint32_t n_frames,
                                          uint64_t stride, int learn, uint32_t* d_active_masks,
                                          void* stream) {
  return sp_compute_frames_overlaps_device(h, d_frames, n_frames, stride, learn, d_active_masks,
                                           nullptr, stream);
}

SP_API sp_status sp_compute_frames(sp_handle* h, const uint32_t* h_frames, uint32_t n_frames,
                                   uint64_t stride, int learn, uint32_t* h_active_masks) {
  if (!h || (!h_frames && n_frames)) return fail(SP_EINVAL, "NULL argument");
  if (h->batch) return fail(SP_EBUSY, "the handle is a member of a batch");
  if (n_frames == 0) return SP_OK;
  if (stride < h->n_words) return fail(SP_EINVAL, "frame stride %llu < %u words", (unsigned long long)stride, h->n_words);
  DeviceGuard g(h->device);
  sp_status s = use_stream(h, h->own_stream);
  if (s != SP_OK) return s;
  if (!h->d_stage) {
    SP_CUDA(device_malloc((void**)&h->d_stage, (size_t)kSlots * kChunkFrames * h->n_words * 4));
    SP_CUDA(device_malloc((void**)&h->d_mstage, (size_t)kSlots * kChunkFrames * h->mask_words * 4));
    SP_CUDA(cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking));
    SP_CUDA(cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking));
    for (int i = 0; i < kSlots; ++i) {
      SP_CUDA(cudaEventCreateWithFlags(&h->ev_h2d[i], cudaEventDisableTiming));
      SP_CUDA(cudaEventCreateWithFlags(&h->ev_comp[i], cudaEventDisableTiming));
      SP_CUDA(cudaEventCreateWithFlags(&h->ev_d2h[i], cudaEventDisableTiming));
      SP_CUDA(cudaEventRecord(h->ev_comp[i], h->stream));
      SP_CUDA(cudaEventRecord(h->ev_d2h[i], h->stream));
    }
  }
  const size_t fbytes = (size_t)h->n_words * 4;
  const size_t mbytes = (size_t)h->mask_words * 4;
  for (uint32_t f0 = 0, ci = 0; f0 < n_frames; f0 += kChunkFrames, ++ci) {
    const int slot = (int)(ci % kSlots);
    const uint32_t nf = (n_frames - f0) < kChunkFrames ? (n_frames - f0) : kChunkFrames;
    uint32_t* dst = h->d_stage + (size_t)slot * kChunkFrames * h->n_words;
    uint32_t* mdst = h->d_mstage + (size_t)slot * kChunkFrames * h->mask_words;
    // H2D of this chunk once the kernels that read this slot two chunks ago are done
    SP_CUDA(cudaStreamWaitEvent(h->s_in, h->ev_comp[slot], 0));
    SP_CUDA(cudaMemcpy2DAsync(dst, fbytes, h_frames + (uint64_t)f0 * stride, stride * 4, fbytes,
                              nf, cudaMemcpyHostToDevice, h->s_in));
    SP_CUDA(cudaEventRecord(h->ev_h2d[slot], h->s_in));
    // compute once the chunk is in and the previous masks of this slot were read
    SP_CUDA(cudaStreamWaitEvent(h->stream, h->ev_h2d[slot], 0));
    SP_CUDA(cudaStreamWaitEvent(h->stream, h->ev_d2h[slot], 0));
    s = run_sequence(h, dst, nf, h->n_words, learn, h_active_masks ? mdst : nullptr);
    if (s != SP_OK) return s;
    SP_CUDA(cudaEventRecord(h->ev_comp[slot], h->stream));
    if (h_active_masks) {
      SP_CUDA(cudaStreamWaitEvent(h->s_out, h->ev_comp[slot], 0));
      SP_CUDA(cudaMemcpyAsync(h_active_masks + (uint64_t)f0 * h->mask_words, mdst, nf * mbytes,
                              cudaMemcpyDeviceToHost, h->s_out));
      SP_CUDA(cudaEventRecord(h->ev_d2h[slot], h->s_out));
    }
  }
  if (h_active_masks) {
    // the handle's stream waits for the last D2H so a later sync covers it
    SP_CUDA(cudaEventRecord(h->ev_switch, h->s_out));
    SP_CUDA(cudaStreamWaitEvent(h->stream, h->ev_switch, 0));
  }
  return wait_handle(h);
}

SP_API sp_status sp_active_columns(sp_handle* h, uint32_t* out, uint32_t cap, uint32_t* n) {
  if (!h || !n || (!out && cap)) return fail(SP_EINVAL, "NULL argument");
  if (h->batch) return fail(SP_EBUSY, "the handle is a member of a batch");
  DeviceGuard g(h->device);
  SP_CUDA(cudaMemcpyAsync(h->h_result, h->d_result, ((size_t)h->max_active + 1) * 4,
                          cudaMemcpyDeviceToHost, h->stream));
  sp_status s = wait_handle(h);
  if (s != SP_OK) return s;
  const uint32_t cnt = h->h_result[0];
  *n = cnt;
  if (cnt > h->max_active) return fail(SP_ECUDA, "winner count %u exceeds bound %u", cnt, h->max_active);
  if (cap < cnt) return fail(SP_EINVAL, "cap %u < %u active columns", cap, cnt);
  if (cnt) std::memcpy(out, h->h_result + 1, (size_t)cnt * 4);
  return SP_OK;
}

SP_API sp_status sp_get_overlaps(sp_handle* h, float* out) {
  if (!h || !out) return fail(SP_EINVAL, "NULL argument");
  if (h->batch) return fail(SP_EBUSY, "the handle is a member of a batch");
  DeviceGuard g(h->device);
  SP_CUDA(cudaMemcpyAsync(out, h->d_ov, (size_t)h->C * 4, cudaMemcpyDeviceToHost, h->stream));
  return wait_handle(h);
}

SP_API sp_status sp_get_permanences(sp_handle* h, float* out) {
  if (!h || !out) return fail(SP_EINVAL, "NULL argument");
  if (h->batch) return fail(SP_EBUSY, "the handle is a member of a batch");
  DeviceGuard g(h->device);
  sp_status s = flush_learning(h);
  if (s != SP_OK) return s;
  SP_CUDA(cudaMemcpyAsync(out, h->d_perm, (size_t)h->C * h->S * 4, cudaMemcpyDeviceToHost,
                          h->stream));
  return wait_handle(h);
}

SP_API sp_status sp_get_pool(sp_handle* h, uint32_t* out) {
  if (!h || !out) return fail(SP_EINVAL, "NULL argument");
  if (h->batch) return fail(SP_EBUSY, "the handle is a member of a batch");
  DeviceGuard g(h->device);
  SP_CUDA(cudaMemcpyAsync(out, h->d_idx, (size_t)h->C * h->S * 4, cudaMemcpyDeviceToHost,
                          h->stream));
  return wait_handle(h);
}

SP_API sp_status sp_get_boost(sp_handle* h, float* out) {
  if (!h || !out) return fail(SP_EINVAL, "NULL argument");
  if (h->batch) return fail(SP_EBUSY, "the handle is a member of a batch");
  DeviceGuard g(h->device);
  SP_CUDA(cudaMemcpyAsync(out, h->d_boost, (size_t)h->C * 4, cudaMemcpyDeviceToHost, h->stream));
  return wait_handle(h);
}

SP_API sp_status sp_get_duty_cycles(sp_handle* h, float* out) {
  if (!h || !out) return fail(SP_EINVAL, "NULL argument");
  if (h->batch) return fail(SP_EBUSY, "the handle is a member of a batch");
  if (!(h->cfg.duty_period > 0.0f)) return fail(SP_EINVAL, "duty cycles are not tracked (duty_period 0)");
  DeviceGuard g(h->device);
  SP_CUDA(cudaMemcpyAsync(out, h->d_duty, (size_t)h->C * 4, cudaMemcpyDeviceToHost, h->stream));
  return wait_handle(h);
}

namespace {
constexpr char kCkptMagic[8] = {'S', 'P', 'G', 'B', '3', '0', '0', '\0'};
constexpr uint32_t kCkptVersion = 1;

struct CkptHeader {
  char magic[8];
  uint32_t version;
  uint32_t config_bytes;
  sp_config cfg;
  uint32_t C, S;
  uint64_t frames;
};
}  // namespace

SP_API sp_status sp_save(sp_handle* h, const char* path) {
  if (!h || !path) return fail(SP_EINVAL, "NULL argument");
  if (h->batch) return fail(SP_EBUSY, "the handle is a member of a batch");
  DeviceGuard g(h->device);
  const size_t CS = (size_t)h->C * h->S;
  std::vector<uint32_t> idx(CS);
  std::vector<float> perm(CS), boost(h->C), duty(h->C, 0.0f);
  sp_status s = flush_learning(h);
  if (s != SP_OK) return s;
  SP_CUDA(cudaMemcpyAsync(idx.data(), h->d_idx, CS * 4, cudaMemcpyDeviceToHost, h->stream));
  SP_CUDA(cudaMemcpyAsync(perm.data(), h->d_perm, CS * 4, cudaMemcpyDeviceToHost, h->stream));
  SP_CUDA(cudaMemcpyAsync(boost.data(), h->d_boost, (size_t)h->C * 4, cudaMemcpyDeviceToHost,
                          h->stream));
  SP_CUDA(cudaMemcpyAsync(duty.data(), h->d_duty, (size_t)h->C * 4, cudaMemcpyDeviceToHost,
                          h->stream));
  if ((s = wait_handle(h)) != SP_OK) return s;
  CkptHeader hd{};
  std::memcpy(hd.magic, kCkptMagic, sizeof(kCkptMagic));
  hd.version = kCkptVersion;
  hd.config_bytes = (uint32_t)sizeof(sp_config);
  hd.cfg = h->cfg;
  hd.C = h->C;
  hd.S = h->S;
  hd.frames = h->frames;
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(SP_EINVAL, "cannot open %s for writing", path);
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 &&
            std::fwrite(idx.data(), 4, CS, f) == CS && std::fwrite(perm.data(), 4, CS, f) == CS &&
            std::fwrite(boost.data(), 4, h->C, f) == h->C &&
            std::fwrite(duty.data(), 4, h->C, f) == h->C;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? SP_OK : fail(SP_EINVAL, "writing %s failed", path);
}

SP_API sp_status sp_load(const char* path, sp_handle** out) {
  if (!path || !out) return fail(SP_EINVAL, "NULL argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(SP_EINVAL, "cannot open %s", path);
  CkptHeader hd{};
  bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1 &&
            std::memcmp(hd.magic, kCkptMagic, sizeof(kCkptMagic)) == 0 &&
            hd.version == kCkptVersion && hd.config_bytes == sizeof(sp_config) &&
            hd.C == hd.cfg.num_columns && hd.S == hd.cfg.synapses_per_column &&
            hd.C <= SP_MAX_COLUMNS && hd.S <= SP_MAX_SYNAPSES;
  const size_t CS = ok ? (size_t)hd.C * hd.S : 0;
  std::vector<uint32_t> idx(CS);
  std::vector<float> perm(CS), boost(ok ? hd.C : 0), duty(ok ? hd.C : 0);
  ok = ok && std::fread(idx.data(), 4, CS, f) == CS && std::fread(perm.data(), 4, CS, f) == CS &&
       std::fread(boost.data(), 4, hd.C, f) == hd.C && std::fread(duty.data(), 4, hd.C, f) == hd.C;
  std::fclose(f);
  if (!ok) return fail(SP_EINVAL, "%s is not a readable SP checkpoint", path);
  sp_handle* h = nullptr;
  sp_status s = sp_create_from_state(&hd.cfg, idx.data(), perm.data(), boost.data(), &h);
  if (s != SP_OK) return s;
  h->frames = hd.frames;
  {
    DeviceGuard g(h->device);
    const cudaError_t e = cudaMemcpyAsync(h->d_duty, duty.data(), (size_t)h->C * 4,
                                          cudaMemcpyHostToDevice, h->stream);
    s = e == cudaSuccess ? wait_handle(h) : fail(SP_ECUDA, "restoring duty cycles failed");
  }
  if (s != SP_OK) {
    sp_destroy(h);
    return s;
  }
  *out = h;
  return SP_OK;
}

SP_API sp_status sp_set_boost(sp_handle* h, const float* boost) {
  if (!h || !boost) return fail(SP_EINVAL, "NULL argument");
  if (h->batch) return fail(SP_EBUSY, "the handle is a member of a batch");
  if (!finite_nonneg(boost, h->C)) return fail(SP_EINVAL, "boost must be finite and >= 0");
  DeviceGuard g(h->device);
  SP_CUDA(cudaMemcpyAsync(h->d_boost, boost, (size_t)h->C * 4, cudaMemcpyHostToDevice, h->stream));
  sp_status s = wait_handle(h);
  if (s == SP_OK) h->unit_boost = all_ones(boost, h->C);
  return s;
}

SP_API sp_status sp_sync(sp_handle* h) {
  if (!h) return fail(SP_EINVAL, "NULL handle");
  DeviceGuard g(h->device);
  return wait_handle(h);
}

SP_API sp_status sp_set_timeout_ms(sp_handle* h, uint32_t ms) {
  if (!h) return fail(SP_EINVAL, "NULL handle");
  h->timeout_ms = ms ? ms : default_timeout_ms();
  return SP_OK;
}

SP_API uint64_t sp_kernel_launch_count(void) {
  return sp::g_launches.load(std::memory_order_relaxed);
}

SP_API const char* sp_status_str(sp_status s) {
  switch (s) {
    case SP_OK: return "ok";
    case SP_EINVAL: return "invalid argument";
    case SP_ENOMEM: return "out of memory";
    case SP_ECUDA: return "CUDA error";
    case SP_ETIMEOUT: return "timed out";
    case SP_EBUSY: return "busy";
    case SP_ENOTSUP: return "not supported";
  }
  return "unknown status";
}

SP_API const char* sp_last_error(void) { return t_last_error.c_str(); }

}  // extern "C"

// ============================== batches ======================================

struct sp_batch {
  std::vector<sp_handle*> members;
  int device = 0;
  void* d_block = nullptr;  // descriptors + CTA map
  sp::BatchDesc* d_desc = nullptr;
  uint32_t* d_cta_inst = nullptr;
  uint32_t n_ctas = 0, max_C = 0;
  // inference of a batch that mixes dense members (tensor cores) with others:
  // the CTA map of the others alone, for their persistent launch
  uint32_t* d_cta_sparse = nullptr;
  uint32_t n_ctas_sparse = 0, max_C_sparse = 0;
  std::vector<sp::BatchDesc> h_desc;  // host copy of the descriptors
  void* d_sync = nullptr;             // persistent launches: work counter, abort, done[n]
  std::vector<uint32_t> member_cpw;   // columns per warp of each member (0: batch_ctas' default)
  uint32_t sched = 0;                 // compiled schedule of the persistent pass (0: default)
  uint32_t stage_cap = 0;             // shared memory for staging state by bulk copy
  uint32_t xspan_cap = 0;             // shared memory for each CTA's input words
  uint32_t win_cap = 0;               // shared memory of the widest window-form CTA
  uint32_t* h_err = nullptr;          // mapped host word: a bounded wait expired
  uint64_t wait_ns = kDeviceWaitNs;   // bound of a persistent launch's per-SP frame wait
  uint32_t* d_err = nullptr;
  uint64_t frame_words = 0, mask_words = 0, ov_words = 0;
  std::vector<uint64_t> frame_off, mask_off, ov_off;
  int cur = 0;
  bool pending = false;
  uint64_t frames = 0;
  uint32_t timeout_ms = 10000;
  cudaStream_t own_stream = nullptr, stream = nullptr, cap_stream = nullptr;
  cudaEvent_t ev_switch = nullptr, ev_wait = nullptr;
  std::vector<GraphEntry> graphs;
  uint64_t graph_clock = 0;
  // sp_batch_infer_device: per-member kernel arguments on the device, staged
  // through two pinned host halves used in turn (each reused only after the
  // copy that read it two calls ago has run)
  void* d_infer_args = nullptr;
  void* h_infer_args = nullptr;
  size_t infer_half = 0;
  int infer_turn = 0;
  cudaEvent_t ev_infer[2] = {nullptr, nullptr};
  std::vector<char> infer_last[2];  // the argument bytes last uploaded to each slot
  // sp_batch_compute staging
  uint32_t* d_stage = nullptr;
  uint32_t* d_mstage = nullptr;
  uint32_t stage_frames = 0;
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_h2d[kSlots] = {}, ev_comp[kSlots] = {}, ev_d2h[kSlots] = {};
};

namespace sp {
namespace rt {

// CTAs given to one SP in a batch launch: every warp takes several columns
// so each CTA streams a few tens of KB of state (fewer, fatter CTAs keep the
// per-CTA ticket and fence cost small).  SP_BATCH_COLS_PER_WARP overrides.
uint32_t batch_ctas(uint32_t C, uint32_t S, uint32_t cols_per_warp) {
  uint32_t cpw = S >= 128u ? 32u : (S >= 32u ? 8u : 16u);
  if (const char* e = std::getenv("SP_BATCH_COLS_PER_WARP")) {
    const long v = std::strtol(e, nullptr, 10);
    if (v >= 1 && v <= 64) cpw = (uint32_t)v;
  }
  if (cols_per_warp) cpw = cols_per_warp;
  const uint32_t per_cta = (uint32_t)sp::kStepWarps * cpw;
  return (C + per_cta - 1u) / per_cta;
}

// Dynamic shared memory a batch launch offers for staging each CTA's
// pools and permanences by bulk copy (0: the CTAs stream them from global
// memory into registers).  Off unless SP_BATCH_STAGE_KB (1..64) allows it:
// on 256 SPs of 1024x256 the staged form measured 0.29-0.47 of HBM peak
// against 0.63 for the streamed one, since a CTA waits for all of its state
// before its first gather and fewer CTAs fit on an SM.
// Shared memory a batch launch offers each CTA for the input words its
// columns index, copied in once so the bit gathers read shared memory.  Off
// unless SP_BATCH_XSPAN_KB (1..48) allows it: on 256 SPs of 1024x256 it
// measured 0.53-0.61 of HBM peak against 0.63 without, the copy adding two
// dependent memory latencies to every CTA's start.
uint32_t batch_xspan_cap() {
  uint32_t kb = 0u;
  if (const char* e = std::getenv("SP_BATCH_XSPAN_KB")) {
    const long v = std::strtol(e, nullptr, 10);
    if (v >= 0 && v <= 48) kb = (uint32_t)v;
  }
  return kb << 10;
}

uint32_t batch_stage_cap(uint32_t need) {
  uint32_t limit = 0u;
  if (const char* e = std::getenv("SP_BATCH_STAGE_KB")) {
    const long v = std::strtol(e, nullptr, 10);
    if (v >= 0 && v <= 64) limit = (uint32_t)v << 10;
  }
  return need <= limit ? need : 0u;
}

}  // namespace rt
}  // namespace sp

namespace {

sp_status batch_wait(sp_batch* b) {
  SP_CUDA(cudaEventRecord(b->ev_wait, b->stream));
  const auto deadline =
      std::chrono::steady_clock::now() + std::chrono::milliseconds(b->timeout_ms);
  for (uint32_t spin = 0;; ++spin) {
    const cudaError_t e = cudaEventQuery(b->ev_wait);
    if (e == cudaSuccess) {
      if (b->h_err && *reinterpret_cast<volatile uint32_t*>(b->h_err)) {
        *b->h_err = 0u;
        // a launch gave up part way: frames of some members stopped after
        // some CTAs took their tickets and counted their histograms, so
        // both are cleared for the next launch
        for (sp_handle* h : b->members) {
          SP_CUDA(cudaMemsetAsync(h->d_counter, 0, 4, b->stream));
          if (h->d_hist) SP_CUDA(cudaMemsetAsync(h->d_hist, 0, ((size_t)h->S + 1) * 4, b->stream));
        }
        SP_CUDA(cudaStreamSynchronize(b->stream));
        return fail(SP_ETIMEOUT, "a bounded device wait expired (the launch stopped early)");
      }
      return SP_OK;
    }
    if (e != cudaErrorNotReady)
      return fail(SP_ECUDA, "device work failed: %s", cudaGetErrorString(e));
    if (std::chrono::steady_clock::now() > deadline)
      return fail(SP_ETIMEOUT, "wait exceeded %u ms", b->timeout_ms);
    if (spin < 2000)
      std::this_thread::yield();
    else
      std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// The CTA map of the members without dense pools, when the batch also has
// dense ones (their inference runs on the tensor cores).
sp_status build_sparse_map(sp_batch* b, const std::vector<uint32_t>& cta_inst) {
  bool any_dense = false;
  for (sp_handle* h : b->members) any_dense = any_dense || h->dense;
  std::vector<uint32_t> sparse;
  uint32_t max_C = 0;
  if (any_dense)
    for (uint32_t i : cta_inst)
      if (!b->members[i]->dense) {
        sparse.push_back(i);
        max_C = std::max(max_C, b->members[i]->C);
      }
  if (b->d_cta_sparse) {
    cudaStreamSynchronize(b->stream);
    cudaFree(b->d_cta_sparse);
    b->d_cta_sparse = nullptr;
  }
  b->n_ctas_sparse = 0;
  b->max_C_sparse = max_C;
  if (sparse.empty()) return SP_OK;
  SP_CUDA(device_malloc((void**)&b->d_cta_sparse, sparse.size() * 4));
  SP_CUDA(cudaMemcpy(b->d_cta_sparse, sparse.data(), sparse.size() * 4, cudaMemcpyHostToDevice));
  b->n_ctas_sparse = (uint32_t)sparse.size();
  return SP_OK;
}

void free_batch(sp_batch* b) {
  if (!b) return;
  DeviceGuard g(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->s_in) cudaStreamSynchronize(b->s_in);
  if (b->s_out) cudaStreamSynchronize(b->s_out);
  for (auto& e : b->graphs) cudaGraphExecDestroy(e.exec);
  for (int i = 0; i < kSlots; ++i) {
    if (b->ev_h2d[i]) cudaEventDestroy(b->ev_h2d[i]);
    if (b->ev_comp[i]) cudaEventDestroy(b->ev_comp[i]);
    if (b->ev_d2h[i]) cudaEventDestroy(b->ev_d2h[i]);
  }
  if (b->s_in) cudaStreamDestroy(b->s_in);
  if (b->s_out) cudaStreamDestroy(b->s_out);
  if (b->d_stage) cudaFree(b->d_stage);
  if (b->d_mstage) cudaFree(b->d_mstage);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->ev_switch) cudaEventDestroy(b->ev_switch);
  if (b->ev_wait) cudaEventDestroy(b->ev_wait);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  if (b->d_block) cudaFree(b->d_block);
  if (b->d_cta_sparse) cudaFree(b->d_cta_sparse);
  if (b->d_infer_args) cudaFree(b->d_infer_args);
  if (b->h_infer_args) cudaFreeHost(b->h_infer_args);
  for (int i = 0; i < 2; ++i)
    if (b->ev_infer[i]) cudaEventDestroy(b->ev_infer[i]);
  if (b->d_sync) cudaFree(b->d_sync);
  if (b->h_err) cudaFreeHost(b->h_err);
  for (sp_handle* h : b->members) {
    if (h->batch != b) continue;
    h->cur = b->cur;  // the members' buffers follow the batch's parity
    h->pending = b->pending;
    h->stream = h->own_stream;
    h->frames += b->frames;
    h->batch = nullptr;
  }
  delete b;
}

sp_status batch_use_stream(sp_batch* b, cudaStream_t s) {
  if (!s) s = b->own_stream;
  if (s != b->stream) {
    SP_CUDA(cudaEventRecord(b->ev_switch, b->stream));
    SP_CUDA(cudaStreamWaitEvent(s, b->ev_switch, 0));
    b->stream = s;
  }
  return SP_OK;
}

// Enqueue n batch frames on `st` from the batch's current (parity, pending).
sp_status batch_enqueue(sp_batch* b, cudaStream_t st, const uint32_t* x_base, uint32_t n,
                        uint64_t stride, int learn, uint32_t* masks, uint64_t mstride,
                        float* ovs, uint64_t ovstride) {
  for (uint32_t t = 0; t < n; ++t) {
    sp::BatchArgs a{};
    a.desc = b->d_desc;
    a.cta_inst = b->d_cta_inst;
    a.frames = x_base + (uint64_t)t * stride;
    a.prev_frames = t ? x_base + (uint64_t)(t - 1) * stride : nullptr;
    a.masks_out = masks ? masks + (uint64_t)t * mstride : nullptr;
    a.ov_out = ovs ? ovs + (uint64_t)t * ovstride : nullptr;
    a.cur = (uint32_t)b->cur;
    a.pending = b->pending ? 1u : 0u;
    a.learn = learn ? 1u : 0u;
    a.save = (t + 1 == n) ? 1u : 0u;
    a.stage_cap = b->stage_cap;
    a.xspan_cap = b->xspan_cap;
    a.win_cap = b->win_cap;
    a.err = b->d_err;
    SP_CUDA(sp::launch_batch_step(a, b->n_ctas, b->max_C, st));
    b->pending = learn != 0;
    b->cur ^= 1;
  }
  return SP_OK;
}

// Whether sequences of batch frames run as one persistent launch
// (SP_DISABLE_PERSISTENT=1 keeps one launch per frame).
bool persistent_enabled() {
  const char* e = std::getenv("SP_DISABLE_PERSISTENT");
  return !(e && e[0] == '1');
}

sp_status batch_run(sp_batch* b, const uint32_t* x_base, uint32_t n, uint64_t stride, int learn,
                    uint32_t* masks, uint64_t mstride, float* ovs = nullptr,
                    uint64_t ovstride = 0) {
  if (learn)
    for (sp_handle* h : b->members) h->bimg_stale = true;
  if (n >= 2 && persistent_enabled()) {
    sp::BatchRunArgs r{};
    r.desc = b->d_desc;
    r.cta_inst = b->d_cta_inst;
    r.items_per_frame = b->n_ctas;
    r.n_frames = n;
    r.frames = x_base;
    r.stride = stride;
    r.masks_out = masks;
    r.mstride = mstride;
    r.ov_out = ovs;
    r.ov_stride = ovstride;
    r.cur0 = (uint32_t)b->cur;
    r.pending0 = b->pending ? 1u : 0u;
    r.learn = learn ? 1u : 0u;
    r.epoch = 0u;
    r.work = static_cast<unsigned long long*>(b->d_sync);
    r.abort = reinterpret_cast<uint32_t*>(static_cast<char*>(b->d_sync) + 8);
    r.done = reinterpret_cast<uint32_t*>(static_cast<char*>(b->d_sync) + 16);
    r.err = b->d_err;
    r.stage_cap = b->stage_cap;
    r.xspan_cap = b->xspan_cap;
    r.win_cap = b->win_cap;
    r.wait_ns = b->wait_ns;
    // counter, abort word and done flags start at 0 in every launch, so a
    // launch recorded into a graph and replayed sees no stale flags
    SP_CUDA(cudaMemsetAsync(b->d_sync, 0, 16 + b->members.size() * 4, b->stream));
    SP_CUDA(sp::launch_batch_run(r, b->max_C, b->sched, b->stream));
    b->pending = learn != 0;
    b->cur ^= (int)(n & 1u);
    b->frames += n;
    return SP_OK;
  }
  if (n < kGraphMinFrames || !graphs_enabled()) {
    sp_status s = batch_enqueue(b, b->stream, x_base, n, stride, learn, masks, mstride, ovs,
                                ovstride);
    if (s == SP_OK) b->frames += n;
    return s;
  }
  const GraphKey key{x_base, n, stride, learn, masks, b->cur, b->pending, false, mstride, 0, ovs,
                     ovstride};
  GraphEntry* e = nullptr;
  for (auto& g : b->graphs)
    if (g.key == key) e = &g;
  if (!e) {
    if (!b->cap_stream) SP_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    const int cur0 = b->cur;
    const bool pending0 = b->pending;
    SP_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    sp_status s = batch_enqueue(b, b->cap_stream, x_base, n, stride, learn, masks, mstride, ovs,
                                ovstride);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->cap_stream, &graph);
    sp::g_launches.fetch_sub(n, std::memory_order_relaxed);
    b->cur = cur0;
    b->pending = pending0;
    if (s != SP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (ec != cudaSuccess) return fail(SP_ECUDA, "recording the batch sequence: %s", cudaGetErrorString(ec));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(SP_ECUDA, "instantiating the batch sequence: %s", cudaGetErrorString(ei));
    if (b->graphs.size() >= kGraphCacheSize) {
      size_t lru = 0;
      for (size_t i = 1; i < b->graphs.size(); ++i)
        if (b->graphs[i].last_use < b->graphs[lru].last_use) lru = i;
      cudaGraphExecDestroy(b->graphs[lru].exec);
      b->graphs.erase(b->graphs.begin() + lru);
    }
    b->graphs.push_back(GraphEntry{key, exec, 0});
    e = &b->graphs.back();
  }
  e->last_use = ++b->graph_clock;
  SP_CUDA(cudaGraphLaunch(e->exec, b->stream));
  sp::g_launches.fetch_add(n, std::memory_order_relaxed);
  b->pending = learn != 0;
  b->cur ^= (int)(n & 1u);
  b->frames += n;
  return SP_OK;
}

}  // namespace

extern "C" {

SP_API sp_status sp_batch_create(sp_handle* const* members, uint32_t n, sp_batch** out) {
  if (!out) return fail(SP_EINVAL, "out is NULL");
  *out = nullptr;
  if (!members || n == 0) return fail(SP_EINVAL, "empty member list");
  for (uint32_t i = 0; i < n; ++i) {
    if (!members[i]) return fail(SP_EINVAL, "member %u is NULL", i);
    if (members[i]->batch) return fail(SP_EBUSY, "member %u is already batched", i);
    if (members[i]->device != members[0]->device)
      return fail(SP_EINVAL, "members live on different devices");
    for (uint32_t j = 0; j < i; ++j)
      if (members[j] == members[i]) return fail(SP_EINVAL, "member %u repeats member %u", i, j);
  }
  sp_batch* b = new (std::nothrow) sp_batch();
  if (!b) return fail(SP_ENOMEM, "host allocation");
  b->device = members[0]->device;
  b->timeout_ms = default_timeout_ms();
  DeviceGuard g(b->device);
  // apply every member's pending learning so the batch starts with none
  for (uint32_t i = 0; i < n; ++i) {
    sp_handle* h = members[i];
    sp_status s = flush_learning(h);
    if (s == SP_OK) s = wait_handle(h);
    if (s != SP_OK) {
      delete b;
      return s;
    }
  }
  std::vector<sp::BatchDesc> desc(n);
  std::vector<uint32_t> cta_inst;
  uint64_t foff = 0, moff = 0, ooff = 0;
  for (uint32_t i = 0; i < n; ++i) {
    sp_handle* h = members[i];
    sp::BatchDesc& d = desc[i];
    uint32_t wb = 0;
    fill_desc(h, &d, 0, &wb);
    b->win_cap = std::max(b->win_cap, wb);
    d.frame_off = foff;
    d.mask_off = moff;
    d.ov_off = ooff;
    b->ov_off.push_back(ooff);
    ooff += h->C;
    d.cta_first = (uint32_t)cta_inst.size();
    for (uint32_t c = 0; c < d.n_ctas; ++c) cta_inst.push_back(i);
    b->frame_off.push_back(foff);
    b->mask_off.push_back(moff);
    foff += ((uint64_t)h->n_words + 3u) & ~uint64_t(3);  // 16-byte aligned members
    moff += h->mask_words;
    b->max_C = std::max(b->max_C, h->C);
    b->stage_cap = std::max(b->stage_cap, sp::batch_stage_bytes(h->C, h->S, d.n_ctas));
  }
  b->stage_cap = batch_stage_cap(b->stage_cap);
  b->xspan_cap = batch_xspan_cap();
  b->frame_words = foff;
  b->mask_words = moff;
  b->ov_words = ooff;
  b->n_ctas = (uint32_t)cta_inst.size();
  b->h_desc = desc;
  const size_t desc_bytes = align256(sizeof(sp::BatchDesc) * n);
  cudaError_t e = device_malloc((void**)&b->d_block, desc_bytes + cta_inst.size() * 4);
  if (e == cudaSuccess) {
    b->d_desc = static_cast<sp::BatchDesc*>(b->d_block);
    b->d_cta_inst = reinterpret_cast<uint32_t*>(static_cast<char*>(b->d_block) + desc_bytes);
    e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_switch, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_wait, cudaEventDisableTiming);
  if (e == cudaSuccess) e = device_malloc(&b->d_sync, 16 + (size_t)n * 4);
  if (e == cudaSuccess) e = cudaMemset(b->d_sync, 0, 16 + (size_t)n * 4);
  if (e == cudaSuccess) {
    e = cudaHostAlloc((void**)&b->h_err, 4, cudaHostAllocMapped);
    if (e == cudaSuccess) {
      *b->h_err = 0u;
      e = cudaHostGetDevicePointer((void**)&b->d_err, b->h_err, 0);
    }
  }
  if (e == cudaSuccess) {
    b->stream = b->own_stream;
    e = cudaMemcpyAsync(b->d_desc, desc.data(), sizeof(sp::BatchDesc) * n, cudaMemcpyHostToDevice,
                        b->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_cta_inst, cta_inst.data(), cta_inst.size() * 4,
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    free_batch(b);
    return fail(e == cudaErrorMemoryAllocation ? SP_ENOMEM : SP_ECUDA, "batch set-up: %s",
                cudaGetErrorString(e));
  }
  for (uint32_t i = 0; i < n; ++i) {
    members[i]->batch = b;
    members[i]->pending = false;
    b->members.push_back(members[i]);
  }
  if (build_sparse_map(b, cta_inst) != SP_OK) {
    const std::string msg = sp_last_error();
    sp_batch_destroy(b);
    return fail(SP_ENOMEM, "%s", msg.c_str());
  }
  *out = b;
  return SP_OK;
}

SP_API void sp_batch_destroy(sp_batch* b) { free_batch(b); }

SP_API sp_status sp_batch_get_info(const sp_batch* b, sp_batch_info* out) {
  if (!b || !out) return fail(SP_EINVAL, "NULL argument");
  out->members = (uint32_t)b->members.size();
  out->ctas = b->n_ctas;
  out->frame_words = b->frame_words;
  out->mask_words = b->mask_words;
  out->frames = b->frames;
  return SP_OK;
}

SP_API sp_status sp_batch_offsets(const sp_batch* b, uint64_t* frame_off, uint64_t* mask_off) {
  if (!b) return fail(SP_EINVAL, "NULL batch");
  for (size_t i = 0; i < b->members.size(); ++i) {
    if (frame_off) frame_off[i] = b->frame_off[i];
    if (mask_off) mask_off[i] = b->mask_off[i];
  }
  return SP_OK;
}

SP_API sp_status sp_batch_forms(const sp_batch* b, uint32_t* forms) {
  if (!b || !forms) return fail(SP_EINVAL, "NULL argument");
  for (size_t i = 0; i < b->members.size(); ++i) {
    const sp::BatchDesc& d = b->h_desc[i];
    forms[i] = d.worg ? SP_FORM_WINDOW : (d.cidx ? SP_FORM_COMPACT : SP_FORM_FULL);
  }
  return SP_OK;
}

SP_API sp_status sp_batch_overlap_offsets(const sp_batch* b, uint64_t* ov_off, uint64_t* ov_words) {
  if (!b) return fail(SP_EINVAL, "NULL batch");
  for (size_t i = 0; i < b->members.size(); ++i)
    if (ov_off) ov_off[i] = b->ov_off[i];
  if (ov_words) *ov_words = b->ov_words;
  return SP_OK;
}

SP_API sp_status sp_batch_compute_overlaps_device(sp_batch* b, const uint32_t* d_frames,
                                                  uint32_t n_frames, uint64_t stride, int learn,
                                                  uint32_t* d_masks, uint64_t mstride,
                                                  float* d_overlaps, uint64_t ov_stride,
                                                  void* stream) {
  if (!b || (!d_frames && n_frames)) return fail(SP_EINVAL, "NULL argument");
  if (n_frames == 0) return SP_OK;
  if (stride < b->frame_words) return fail(SP_EINVAL, "frame stride %llu < %llu words", (unsigned long long)stride, (unsigned long long)b->frame_words);
  if (d_masks && mstride < b->mask_words) return fail(SP_EINVAL, "mask stride %llu < %llu words", (unsigned long long)mstride, (unsigned long long)b->mask_words);
  if (d_overlaps && ov_stride < b->ov_words)
    return fail(SP_EINVAL, "overlap stride %llu < %llu", (unsigned long long)ov_stride, (unsigned long long)b->ov_words);
  if (reinterpret_cast<uintptr_t>(d_frames) % 16u || reinterpret_cast<uintptr_t>(d_masks) % 4u ||
      (n_frames > 1 && stride % 4u))
    return fail(SP_EINVAL, "batch frames must be 16-byte aligned (stride a multiple of 4 words)");
  if (reinterpret_cast<uintptr_t>(d_overlaps) % 4u)
    return fail(SP_EINVAL, "d_overlaps not 4-byte aligned");
  DeviceGuard g(b->device);
  sp_status s = batch_use_stream(b, static_cast<cudaStream_t>(stream));
  if (s != SP_OK) return s;
  return batch_run(b, d_frames, n_frames, stride, learn, d_masks, mstride, d_overlaps, ov_stride);
}

SP_API sp_status sp_batch_compute_device(sp_batch* b, const uint32_t* d_frames, uint32_t n_frames,
                                         uint64_t stride, int learn, uint32_t* d_masks,
                                         uint64_t mstride, void* stream) {
  return sp_batch_compute_overlaps_device(b, d_frames, n_frames, stride, learn, d_masks, mstride,
                                          nullptr, 0, stream);
}

SP_API sp_status sp_batch_compute(sp_batch* b, const uint32_t* h_frames, uint32_t n_frames,
                                  uint64_t stride, int learn, uint32_t* h_masks, uint64_t mstride) {
  if (!b || (!h_frames && n_frames)) return fail(SP_EINVAL, "NULL argument");
  if (n_frames == 0) return SP_OK;
  if (stride < b->frame_words) return fail(SP_EINVAL, "frame stride below frame_words");
  if (h_masks && mstride < b->mask_words) return fail(SP_EINVAL, "mask stride below mask_words");
  DeviceGuard g(b->device);
  sp_status s = batch_use_stream(b, b->own_stream);
  if (s != SP_OK) return s;
  const uint64_t fw = (b->frame_words + 3u) & ~uint64_t(3);
  if (!b->d_stage) {
    // about 64 MiB of staged batch frames per slot
    uint64_t per = (64ull << 20) / (fw * 4u);
    b->stage_frames = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(per, kChunkFrames));
    SP_CUDA(device_malloc((void**)&b->d_stage, (size_t)kSlots * b->stage_frames * fw * 4));
    SP_CUDA(device_malloc((void**)&b->d_mstage, (size_t)kSlots * b->stage_frames * b->mask_words * 4));
    SP_CUDA(cudaStreamCreateWithFlags(&b->s_in, cudaStreamNonBlocking));
    SP_CUDA(cudaStreamCreateWithFlags(&b->s_out, cudaStreamNonBlocking));
    for (int i = 0; i < kSlots; ++i) {
      SP_CUDA(cudaEventCreateWithFlags(&b->ev_h2d[i], cudaEventDisableTiming));
      SP_CUDA(cudaEventCreateWithFlags(&b->ev_comp[i], cudaEventDisableTiming));
      SP_CUDA(cudaEventCreateWithFlags(&b->ev_d2h[i], cudaEventDisableTiming));
      SP_CUDA(cudaEventRecord(b->ev_comp[i], b->stream));
      SP_CUDA(cudaEventRecord(b->ev_d2h[i], b->stream));
    }
  }
  const uint32_t cf = b->stage_frames;
  for (uint32_t f0 = 0, ci = 0; f0 < n_frames; f0 += cf, ++ci) {
    const int slot = (int)(ci % kSlots);
    const uint32_t nf = std::min(cf, n_frames - f0);
    uint32_t* dst = b->d_stage + (size_t)slot * cf * fw;
    uint32_t* mdst = b->d_mstage + (size_t)slot * cf * b->mask_words;
    SP_CUDA(cudaStreamWaitEvent(b->s_in, b->ev_comp[slot], 0));
    SP_CUDA(cudaMemcpy2DAsync(dst, fw * 4, h_frames + (uint64_t)f0 * stride, stride * 4,
                              b->frame_words * 4, nf, cudaMemcpyHostToDevice, b->s_in));
    SP_CUDA(cudaEventRecord(b->ev_h2d[slot], b->s_in));
    SP_CUDA(cudaStreamWaitEvent(b->stream, b->ev_h2d[slot], 0));
    SP_CUDA(cudaStreamWaitEvent(b->stream, b->ev_d2h[slot], 0));
    s = batch_run(b, dst, nf, fw, learn, h_masks ? mdst : nullptr, b->mask_words);
    if (s != SP_OK) return s;
    SP_CUDA(cudaEventRecord(b->ev_comp[slot], b->stream));
    if (h_masks) {
      SP_CUDA(cudaStreamWaitEvent(b->s_out, b->ev_comp[slot], 0));
      SP_CUDA(cudaMemcpy2DAsync(h_masks + (uint64_t)f0 * mstride, mstride * 4, mdst,
                                b->mask_words * 4, b->mask_words * 4, nf, cudaMemcpyDeviceToHost,
                                b->s_out));
      SP_CUDA(cudaEventRecord(b->ev_d2h[slot], b->s_out));
    }
  }
  if (h_masks) {
    SP_CUDA(cudaEventRecord(b->ev_switch, b->s_out));
    SP_CUDA(cudaStreamWaitEvent(b->stream, b->ev_switch, 0));
  }
  return batch_wait(b);
}

SP_API sp_status sp_batch_infer_overlaps_device(sp_batch* b, const uint32_t* d_frames,
                                                uint32_t n_frames, uint64_t stride,
                                                uint32_t* d_masks, uint64_t mstride,
                                                float* d_overlaps, uint64_t ov_stride,
                                                void* stream) {
  if (!b || (!d_frames && n_frames)) return fail(SP_EINVAL, "NULL argument");
  if (n_frames == 0) return SP_OK;
  if (stride < b->frame_words) return fail(SP_EINVAL, "frame stride below frame_words");
  if (d_masks && mstride < b->mask_words) return fail(SP_EINVAL, "mask stride below mask_words");
  if (d_overlaps && ov_stride < b->ov_words) return fail(SP_EINVAL, "overlap stride below the record length");
  if (reinterpret_cast<uintptr_t>(d_frames) % 4u || reinterpret_cast<uintptr_t>(d_masks) % 4u ||
      reinterpret_cast<uintptr_t>(d_overlaps) % 4u)
    return fail(SP_EINVAL, "device pointers must be 4-byte aligned");
  DeviceGuard g(b->device);
  sp_status st = batch_use_stream(b, static_cast<cudaStream_t>(stream));
  if (st != SP_OK) return st;
  // dense members on the tensor cores, the others in one persistent launch
  std::vector<uint32_t> dm;
  for (uint32_t i = 0; i < (uint32_t)b->members.size(); ++i)
    if (b->members[i]->dense) dm.push_back(i);
  if (dm.size() < b->members.size() && (reinterpret_cast<uintptr_t>(d_frames) % 16u ||
                                        (n_frames > 1 && stride % 4u)))
    return fail(SP_EINVAL, "a batch with members of sparse pools needs 16-byte aligned frames");
  const uint32_t n = (uint32_t)dm.size();
  // learning left pending by the last batch step is applied first: by a
  // learning pass for the dense members, by the persistent launch (which
  // also keeps their compact or window form in step) for the others
  const bool pend = b->pending;
  if (pend) {
    for (uint32_t i : dm) {
      sp_handle* h = b->members[i];
      sp::LearnArgs l{};
      l.idx = h->d_idx;
      l.perm = h->d_perm;
      l.x = h->d_xsave[b->cur ^ 1];
      l.mask = h->d_mask[b->cur ^ 1];
      l.C = h->C;
      l.S = h->S;
      l.inc = h->cfg.perm_inc;
      l.dec = h->cfg.perm_dec;
      SP_CUDA(sp::launch_learn(l, b->stream));
    }
    b->pending = false;
  }
  // the members without dense pools: one persistent launch of their CTAs
  // (no learning; frame 0 applies what was pending), before the tensor-core
  // launches
  const uint32_t cur0 = (uint32_t)b->cur;
  const uint32_t last_par = cur0 ^ ((n_frames - 1u) & 1u);  // the last frame's mask slot
  if (b->n_ctas_sparse) {
    sp::BatchRunArgs r{};
    r.desc = b->d_desc;
    r.cta_inst = b->d_cta_sparse;
    r.items_per_frame = b->n_ctas_sparse;
    r.n_frames = n_frames;
    r.frames = d_frames;
    r.stride = stride;
    r.masks_out = d_masks;
    r.mstride = mstride;
    r.ov_out = d_overlaps;
    r.ov_stride = ov_stride;
    r.cur0 = cur0;
    r.pending0 = pend ? 1u : 0u;
    r.learn = 0u;
    r.epoch = 0u;
    r.work = static_cast<unsigned long long*>(b->d_sync);
    r.abort = reinterpret_cast<uint32_t*>(static_cast<char*>(b->d_sync) + 8);
    r.done = reinterpret_cast<uint32_t*>(static_cast<char*>(b->d_sync) + 16);
    r.err = b->d_err;
    r.stage_cap = b->stage_cap;
    r.xspan_cap = b->xspan_cap;
    r.win_cap = b->win_cap;
    r.wait_ns = b->wait_ns;
    SP_CUDA(cudaMemsetAsync(b->d_sync, 0, 16 + b->members.size() * 4, b->stream));
    SP_CUDA(sp::launch_batch_run(r, b->max_C_sparse, b->sched, b->stream));
  }
  if (n == 0) {
    b->cur ^= (int)(n_frames & 1u);
    b->frames += n_frames;
    return SP_OK;
  }
  std::vector<sp::DenseArgs> dargs(n);
  std::vector<sp::FrameInhibitArgs> fargs(n);
  uint32_t max_C = 0, max_S = 0, max_K = 0;
  bool all_global = true, any_pack = false;
  for (uint32_t ii = 0; ii < n; ++ii) {
    const uint32_t i = dm[ii];
    sp_handle* h = b->members[i];
    if ((st = ensure_dense_buffers(h, n_frames)) != SP_OK) return st;
    sp::DenseArgs& d = dargs[ii];
    d = dense_args(h, d_frames + b->frame_off[i], n_frames, stride);
    any_pack = any_pack || d.pack != 0u;
    max_K = std::max(max_K, h->S);
    h->dense_used = true;
    sp::FrameInhibitArgs& f = fargs[ii];
    f.ov = h->d_run_ov;
    f.n_frames = n_frames;
    f.C = h->C;
    f.mask_words = h->mask_words;
    f.k = h->cfg.winners_set_size;
    f.inhibition = h->cfg.inhibition;
    f.gw = h->cfg.col_grid_w;
    f.gh = h->cfg.col_grid_h;
    f.radius = h->cfg.local_radius;
    f.unit_S = h->unit_boost ? h->S : 0u;
    if (sp::frame_inhibit_smem(h->C, f.unit_S) > sp::frame_inhibit_smem_limit()) f.unit_S = 0u;
    const bool duty = h->cfg.duty_period > 0.0f;
    f.masks_out = d_masks ? d_masks + b->mask_off[i] : (duty ? h->d_run_masks : nullptr);
    f.masks_stride = d_masks ? mstride : h->mask_words;
    f.mask_last = h->d_mask[last_par];
    f.result = h->d_result;
    f.ov_last = h->d_ov;
    max_C = std::max(max_C, h->C);
    max_S = std::max(max_S, f.unit_S);
    all_global = all_global && f.inhibition == 0u;
  }
  if (sp::frame_inhibit_smem(max_C, max_S) > sp::frame_inhibit_smem_limit())
    return fail(SP_ENOTSUP, "members too large for one per-frame inhibition launch");
  const size_t arg_bytes = (sizeof(sp::DenseArgs) + sizeof(sp::FrameInhibitArgs)) * n;
  if (!b->d_infer_args) {
    b->infer_half = align256(arg_bytes);
    SP_CUDA(device_malloc((void**)&b->d_infer_args, 2 * b->infer_half));
    SP_CUDA(cudaMallocHost(&b->h_infer_args, 2 * b->infer_half));
    for (int i = 0; i < 2; ++i) SP_CUDA(cudaEventCreateWithFlags(&b->ev_infer[i], cudaEventDisableTiming));
  }
  // one device slot of arguments per buffer parity (the members' last-frame
  // masks alternate with it), so a repeated run finds its arguments in place
  const int slot = b->cur;
  sp::DenseArgs* d_dargs = reinterpret_cast<sp::DenseArgs*>(static_cast<char*>(b->d_infer_args) +
                                                            (size_t)slot * b->infer_half);
  sp::FrameInhibitArgs* d_fargs = reinterpret_cast<sp::FrameInhibitArgs*>(d_dargs + n);
  const size_t dbytes = sizeof(sp::DenseArgs) * n;
  std::vector<char>& last = b->infer_last[slot];
  const bool same = last.size() == arg_bytes &&
                    std::memcmp(last.data(), dargs.data(), dbytes) == 0 &&
                    std::memcmp(last.data() + dbytes, fargs.data(), arg_bytes - dbytes) == 0;
  if (!same) {
    // through the stream (earlier launches keep their arguments) from a
    // pinned half whose previous copy has completed
    const int turn = b->infer_turn;
    b->infer_turn ^= 1;
    SP_CUDA(cudaEventSynchronize(b->ev_infer[turn]));
    char* h_args = static_cast<char*>(b->h_infer_args) + (size_t)turn * b->infer_half;
    std::memcpy(h_args, dargs.data(), dbytes);
    std::memcpy(h_args + dbytes, fargs.data(), arg_bytes - dbytes);
    SP_CUDA(cudaMemcpyAsync(d_dargs, h_args, arg_bytes, cudaMemcpyHostToDevice, b->stream));
    SP_CUDA(cudaEventRecord(b->ev_infer[turn], b->stream));
    last.assign(h_args, h_args + arg_bytes);
  }
  if (any_pack) SP_CUDA(sp::launch_conn_image(d_dargs, n, max_C, max_K, b->stream));
  for (uint32_t i : dm) b->members[i]->bimg_stale = false;
  // frame images, product, selection and duty cycles: the same launches for
  // the same frames, masks and slot, so they are recorded once and replayed
  uint64_t n_launch = 3;
  for (uint32_t i : dm) n_launch += b->members[i]->cfg.duty_period > 0.0f ? 1u : 0u;
  auto enqueue = [&](cudaStream_t st) -> sp_status {
    SP_CUDA(sp::launch_frame_image(d_dargs, n, n_frames, max_K, st));
    SP_CUDA(sp::launch_dense_overlap_many(d_dargs, n, max_C, n_frames, st));
    SP_CUDA(sp::launch_frame_inhibit_many(d_fargs, n, max_C, max_S, n_frames, all_global, st));
    for (uint32_t ii = 0; ii < n; ++ii) {
      sp_handle* h = b->members[dm[ii]];
      if (h->cfg.duty_period > 0.0f)
        SP_CUDA(sp::launch_duty_run(fargs[ii].masks_out, n_frames, (uint32_t)fargs[ii].masks_stride,
                                    h->C, h->d_duty, h->cfg.duty_period, st));
    }
    return SP_OK;
  };
  if (!graphs_enabled()) {
    if ((st = enqueue(b->stream)) != SP_OK) return st;
  } else {
    // learn = 2 marks a dense inference run in the batch's graph cache; the
    // selection's histogram size and the members' run buffers (the duty
    // launches hold their masks' address) are part of the recorded launches
    uint64_t gens = 0;
    for (uint32_t i : dm) gens += b->members[i]->run_gen;
    GraphKey key{d_frames, n_frames, stride, 2, d_masks, b->cur, false, all_global, mstride};
    key.extra = (uint64_t)max_S | (gens << 32);
    GraphEntry* e = nullptr;
    for (auto& g : b->graphs)
      if (g.key == key) e = &g;
    if (!e) {
      if (!b->cap_stream) SP_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
      SP_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
      const sp_status s = enqueue(b->cap_stream);
      cudaGraph_t graph = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(b->cap_stream, &graph);
      sp::g_launches.fetch_sub(n_launch, std::memory_order_relaxed);
      if (s != SP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
      }
      if (ec != cudaSuccess)
        return fail(SP_ECUDA, "recording the dense run: %s", cudaGetErrorString(ec));
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess)
        return fail(SP_ECUDA, "instantiating the dense run: %s", cudaGetErrorString(ei));
      if (b->graphs.size() >= kGraphCacheSize) {
        size_t lru = 0;
        for (size_t i = 1; i < b->graphs.size(); ++i)
          if (b->graphs[i].last_use < b->graphs[lru].last_use) lru = i;
        cudaGraphExecDestroy(b->graphs[lru].exec);
        b->graphs.erase(b->graphs.begin() + lru);
      }
      b->graphs.push_back(GraphEntry{key, exec, 0});
      e = &b->graphs.back();
    }
    e->last_use = ++b->graph_clock;
    SP_CUDA(cudaGraphLaunch(e->exec, b->stream));
    sp::g_launches.fetch_add(n_launch, std::memory_order_relaxed);
  }
  if (d_overlaps) {
    // each dense member's [n_frames][C] run overlaps into its columns of the record
    for (uint32_t i : dm) {
      sp_handle* h = b->members[i];
      SP_CUDA(cudaMemcpy2DAsync(d_overlaps + b->ov_off[i], ov_stride * 4, h->d_run_ov,
                                (size_t)h->C * 4, (size_t)h->C * 4, n_frames,
                                cudaMemcpyDeviceToDevice, b->stream));
    }
  }
  b->cur ^= (int)(n_frames & 1u);
  b->frames += n_frames;
  return SP_OK;
}

SP_API sp_status sp_batch_infer_device(sp_batch* b, const uint32_t* d_frames, uint32_t n_frames,
                                       uint64_t stride, uint32_t* d_masks, uint64_t mstride,
                                       void* stream) {
  return sp_batch_infer_overlaps_device(b, d_frames, n_frames, stride, d_masks, mstride, nullptr,
                                        0, stream);
}

namespace {

// Re-split member i into CTAs of 4 * cols_per_warp[i] columns (0: the
// member's default) and upload the descriptors and CTA map.  The batch must
// be idle.
sp_status batch_relayout(sp_batch* b, const std::vector<uint32_t>& cols_per_warp) {
  std::vector<uint32_t> cta_inst;
  uint32_t win_cap = 0;
  for (size_t i = 0; i < b->members.size(); ++i) {
    sp_handle* h = b->members[i];
    sp::BatchDesc& d = b->h_desc[i];
    d.n_ctas = batch_ctas(h->C, h->S, cols_per_warp[i]);
    d.cta_first = (uint32_t)cta_inst.size();
    d.xspan = batch_xspan_cap() > 0u ? handle_xspan(h, d.n_ctas) : nullptr;
    uint32_t wb = 0;
    if (d.worg && !window_rebands(h, &d, &wb) && handle_compact(h)) {
      // the bands of this split do not fit: the compact form, derived from
      // the permanences as they are now (the window form kept them current)
      d.cidx = h->d_cidx;
      d.cbase = h->d_cbase;
      d.conn = h->d_cconn;
    }
    win_cap = std::max(win_cap, wb);
    for (uint32_t c = 0; c < d.n_ctas; ++c) cta_inst.push_back((uint32_t)i);
  }
  const size_t n = b->members.size();
  const size_t desc_bytes = align256(sizeof(sp::BatchDesc) * n);
  if (cta_inst.size() > b->n_ctas) {  // the CTA map grows: a new block
    void* blk = nullptr;
    SP_CUDA(device_malloc(&blk, desc_bytes + cta_inst.size() * 4));
    cudaFree(b->d_block);
    b->d_block = blk;
    b->d_desc = static_cast<sp::BatchDesc*>(blk);
    b->d_cta_inst = reinterpret_cast<uint32_t*>(static_cast<char*>(blk) + desc_bytes);
  }
  SP_CUDA(cudaMemcpyAsync(b->d_desc, b->h_desc.data(), sizeof(sp::BatchDesc) * n,
                          cudaMemcpyHostToDevice, b->stream));
  SP_CUDA(cudaMemcpyAsync(b->d_cta_inst, cta_inst.data(), cta_inst.size() * 4,
                          cudaMemcpyHostToDevice, b->stream));
  SP_CUDA(cudaStreamSynchronize(b->stream));
  b->n_ctas = (uint32_t)cta_inst.size();
  b->member_cpw = cols_per_warp;
  b->win_cap = win_cap;
  sp_status sm = build_sparse_map(b, cta_inst);
  if (sm != SP_OK) return sm;
  for (auto& e : b->graphs) cudaGraphExecDestroy(e.exec);  // recorded with the old grid
  b->graphs.clear();
  return SP_OK;
}

// Tuning bucket of a member: its synapses per column (S <= 32, <= 128, more)
// and its input (at most 4096 bits, more), the two sizes that set how a
// column's pass streams its state and gathers its inputs.
uint32_t tune_bucket(const sp_handle* h) {
  const uint32_t sb = h->S <= 32u ? 0u : (h->S <= 128u ? 1u : 2u);
  const uint32_t nb = h->n_words * 32u <= 4096u ? 0u : 1u;
  return sb * 2u + nb;
}

}  // namespace

SP_API sp_status sp_batch_autotune(sp_batch* b, const uint32_t* d_frames, uint32_t n_frames,
                                   uint64_t stride, uint32_t* cols_per_warp) {
  if (!b || !d_frames || n_frames == 0) return fail(SP_EINVAL, "NULL argument or no frames");
  if (stride < b->frame_words && n_frames > 1)
    return fail(SP_EINVAL, "frame stride below the batch frame");
  if (reinterpret_cast<uintptr_t>(d_frames) % 16u || (n_frames > 1 && stride % 4u))
    return fail(SP_EINVAL, "batch frames must be 16-byte aligned (stride a multiple of 4 words)");
  if (b->pending) return fail(SP_EBUSY, "learning is pending: tune before learning frames");
  DeviceGuard g(b->device);
  sp_status s = batch_wait(b);
  if (s != SP_OK) return s;
  // The tuning frames learn, as the batch's own frames do: the state that
  // learning writes (permanences, window bitmaps, compact connected bits)
  // and the duty cycles, which advance on every frame, are copied aside and
  // put back after.  Without room for the copy the frames are timed as
  // inference and only the duty cycles are kept.
  std::vector<std::pair<void*, size_t>> duty, learnt;
  size_t duty_bytes = 0, learnt_bytes = 0;
  for (sp_handle* h : b->members) {
    if (h->cfg.duty_period > 0.0f) {
      duty.emplace_back(h->d_duty, (size_t)h->C * 4);
      duty_bytes += align256((size_t)h->C * 4);
    }
    learnt.emplace_back(h->d_perm, (size_t)h->C * h->S * 4);
    if (h->d_wbits) learnt.emplace_back(h->d_wbits, (size_t)h->C * 512);
    if (h->d_cconn) learnt.emplace_back(h->d_cconn, (size_t)h->C * ((h->S + 31u) & ~31u) / 8);
  }
  for (auto& d : learnt) learnt_bytes += align256(d.second);
  char* d_keep = nullptr;
  bool learn_tune = n_frames >= 2 && persistent_enabled() &&
                    device_malloc((void**)&d_keep, duty_bytes + learnt_bytes) == cudaSuccess;
  if (!learn_tune) {
    cudaGetLastError();  // a failed allocation is not an error here
    d_keep = nullptr;
    learnt.clear();
    if (duty_bytes) SP_CUDA(device_malloc((void**)&d_keep, duty_bytes));
  }
  std::vector<std::pair<void*, size_t>> kept = duty;
  kept.insert(kept.end(), learnt.begin(), learnt.end());
  size_t off = 0;
  for (auto& d : kept) {
    SP_CUDA(cudaMemcpyAsync(d_keep + off, d.first, d.second, cudaMemcpyDeviceToDevice, b->stream));
    off += align256(d.second);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SP_CUDA(cudaEventCreate(&e0));
  SP_CUDA(cudaEventCreate(&e1));
  const bool persistent = n_frames >= 2 && persistent_enabled();
  // the fastest of three runs of the tuning frames in the current layout and
  // schedule, in the launch form sequences use (one persistent launch of
  // inference frames), or one launch per frame for a single frame
  auto time_layout = [&](float* best_of3) -> sp_status {
    float ms_min = 0.0f;
    sp_status st = SP_OK;
    for (int rep = 0; rep < 3 && st == SP_OK; ++rep) {
      cudaError_t e = cudaEventRecord(e0, b->stream);
      if (persistent) {
        sp::BatchRunArgs r{};
        r.desc = b->d_desc;
        r.cta_inst = b->d_cta_inst;
        r.items_per_frame = b->n_ctas;
        r.n_frames = n_frames;
        r.frames = d_frames;
        r.stride = stride;
        r.cur0 = (uint32_t)b->cur;
        r.pending0 = 0u;  // every timing run starts with nothing pending
        r.learn = learn_tune ? 1u : 0u;
        r.epoch = 0u;
        r.work = static_cast<unsigned long long*>(b->d_sync);
        r.abort = reinterpret_cast<uint32_t*>(static_cast<char*>(b->d_sync) + 8);
        r.done = reinterpret_cast<uint32_t*>(static_cast<char*>(b->d_sync) + 16);
        r.err = b->d_err;
        r.stage_cap = b->stage_cap;
        r.xspan_cap = b->xspan_cap;
        r.win_cap = b->win_cap;
        r.wait_ns = b->wait_ns;
        if (e == cudaSuccess)
          e = cudaMemsetAsync(b->d_sync, 0, 16 + b->members.size() * 4, b->stream);
        if (e == cudaSuccess) e = sp::launch_batch_run(r, b->max_C, b->sched, b->stream);
      } else {
        for (uint32_t t = 0; t < n_frames && e == cudaSuccess; ++t) {
          sp::BatchArgs a{};
          a.desc = b->d_desc;
          a.cta_inst = b->d_cta_inst;
          a.frames = d_frames + (uint64_t)t * stride;
          a.cur = (uint32_t)b->cur;  // inference with nothing pending: parity unchanged
          a.stage_cap = b->stage_cap;
          a.xspan_cap = b->xspan_cap;
          a.win_cap = b->win_cap;
          a.err = b->d_err;
          e = sp::launch_batch_step(a, b->n_ctas, b->max_C, b->stream);
        }
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) st = batch_wait(b);
      else st = fail(SP_ECUDA, "autotune launch: %s", cudaGetErrorString(e));
      float ms = 0.0f;
      if (st == SP_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        ms_min = rep == 0 ? ms : std::min(ms_min, ms);
    }
    *best_of3 = ms_min;
    return st;
  };
  // A change is kept only if it is more than 3 % faster than the best so far
  // (inference frames leave out learning, so small gains are not trusted).
  constexpr float kGain = 1.03f;
  const size_t n = b->members.size();
  std::vector<uint32_t> cpw(n, 0u);
  b->sched = 0u;
  s = batch_relayout(b, cpw);
  float best_ms = 0.0f;
  if (s == SP_OK) s = time_layout(&best_ms);
  const uint32_t candidates[] = {2u, 4u, 8u, 16u};
  // 1. one split for every member
  uint32_t uniform = 0u;
  for (uint32_t c : candidates) {
    if (s != SP_OK) break;
    s = batch_relayout(b, std::vector<uint32_t>(n, c));
    float ms = 0.0f;
    if (s == SP_OK) s = time_layout(&ms);
    if (s == SP_OK && ms * kGain < best_ms) {
      best_ms = ms;
      uniform = c;
    }
  }
  std::fill(cpw.begin(), cpw.end(), uniform);
  if (s == SP_OK) s = batch_relayout(b, cpw);
  // 2. the compiled schedule (resident CTAs per SM x columns in flight)
  uint32_t best_sched = 0u;
  for (uint32_t i = 1; persistent && s == SP_OK && i < sp::batch_schedule_count(); ++i) {
    b->sched = i;
    float ms = 0.0f;
    s = time_layout(&ms);
    if (s == SP_OK && ms * kGain < best_ms) {
      best_ms = ms;
      best_sched = i;
    }
  }
  b->sched = best_sched;
  // 3. the split of each bucket of members (members of one bucket share it),
  // largest bucket first, the others as chosen so far
  std::vector<uint32_t> bucket(n), count(6, 0u);
  for (size_t i = 0; i < n; ++i) count[bucket[i] = tune_bucket(b->members[i])]++;
  std::vector<uint32_t> order;
  for (uint32_t k = 0; k < 6; ++k)
    if (count[k]) order.push_back(k);
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t x, uint32_t y) { return count[x] > count[y]; });
  for (uint32_t k : order) {
    if (order.size() < 2u) break;  // one bucket: step 1 has tried its splits
    uint32_t keep = uniform;
    for (uint32_t c : {0u, 2u, 4u, 8u, 16u}) {
      if (s != SP_OK || c == uniform) continue;
      std::vector<uint32_t> trial = cpw;
      for (size_t i = 0; i < n; ++i)
        if (bucket[i] == k) trial[i] = c;
      s = batch_relayout(b, trial);
      float ms = 0.0f;
      if (s == SP_OK) s = time_layout(&ms);
      if (s == SP_OK && ms * kGain < best_ms) {
        best_ms = ms;
        keep = c;
      }
    }
    for (size_t i = 0; i < n; ++i)
      if (bucket[i] == k) cpw[i] = keep;
  }
  off = 0;
  for (auto& d : kept) {
    cudaMemcpyAsync(d.first, d_keep + off, d.second, cudaMemcpyDeviceToDevice, b->stream);
    off += align256(d.second);
  }
  cudaStreamSynchronize(b->stream);
  if (d_keep) cudaFree(d_keep);
  // the final split after the state is back, so that forms derived from the
  // permanences (a compact form a split needs) derive from the kept ones
  if (s == SP_OK) s = batch_relayout(b, cpw);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == SP_OK && cols_per_warp) {
    uint32_t one = cpw.empty() ? 0u : cpw[0];
    for (uint32_t c : cpw)
      if (c != one) one = SP_MIXED_SPLIT;
    *cols_per_warp = one;
  }
  return s;
}

SP_API sp_status sp_batch_schedule_list(uint32_t* ctas_per_sm, uint32_t* cols_in_flight,
                                        uint32_t cap, uint32_t* count) {
  const uint32_t n = sp::batch_schedule_count();
  if (count) *count = n;
  if (cap < n && (ctas_per_sm || cols_in_flight))
    return fail(SP_EINVAL, "room for %u schedules needed, %u given", n, cap);
  for (uint32_t i = 0; i < n; ++i)
    sp::batch_schedule(i, ctas_per_sm ? ctas_per_sm + i : nullptr,
                       cols_in_flight ? cols_in_flight + i : nullptr);
  return SP_OK;
}

SP_API sp_status sp_batch_set_schedule(sp_batch* b, uint32_t ctas_per_sm, uint32_t cols_in_flight,
                                       const uint32_t* member_cols_per_warp) {
  if (!b) return fail(SP_EINVAL, "NULL batch");
  uint32_t found = UINT32_MAX;
  for (uint32_t i = 0; i < sp::batch_schedule_count(); ++i) {
    uint32_t c = 0, f = 0;
    sp::batch_schedule(i, &c, &f);
    if (c == ctas_per_sm && f == cols_in_flight) found = i;
  }
  if (found == UINT32_MAX)
    return fail(SP_ENOTSUP, "no compiled schedule of %u CTAs per SM x %u columns in flight",
                ctas_per_sm, cols_in_flight);
  std::vector<uint32_t> cpw(b->members.size(), 0u);
  if (member_cols_per_warp)
    for (size_t i = 0; i < cpw.size(); ++i) {
      cpw[i] = member_cols_per_warp[i];
      if (cpw[i] > 64u) return fail(SP_EINVAL, "member %zu: columns per warp above 64", i);
    }
  if (b->pending) return fail(SP_EBUSY, "learning is pending: set the schedule before learning");
  DeviceGuard g(b->device);
  sp_status s = batch_wait(b);
  if (s != SP_OK) return s;
  b->sched = found;
  return batch_relayout(b, cpw);
}

SP_API sp_status sp_batch_schedule(const sp_batch* b, uint32_t* ctas_per_sm,
                                   uint32_t* cols_in_flight, uint32_t* member_cols_per_warp) {
  if (!b) return fail(SP_EINVAL, "NULL batch");
  if (!sp::batch_schedule(b->sched, ctas_per_sm, cols_in_flight))
    return fail(SP_EINVAL, "no such schedule");
  if (member_cols_per_warp)
    for (size_t i = 0; i < b->members.size(); ++i)
      member_cols_per_warp[i] = i < b->member_cpw.size() ? b->member_cpw[i] : 0u;
  return SP_OK;
}

SP_API sp_status sp_batch_set_device_wait_ns(sp_batch* b, uint64_t ns) {
  if (!b) return fail(SP_EINVAL, "NULL batch");
  b->wait_ns = ns ? ns : kDeviceWaitNs;
  // recorded launches carry the old bound
  for (auto& e : b->graphs) cudaGraphExecDestroy(e.exec);
  b->graphs.clear();
  return SP_OK;
}

SP_API sp_status sp_batch_sync(sp_batch* b) {
  if (!b) return fail(SP_EINVAL, "NULL batch");
  DeviceGuard g(b->device);
  return batch_wait(b);
}

}  // extern "C"
