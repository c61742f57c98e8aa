// Internal definitions shared by the host runtime files (not part of the ABI):
// the handle's layout, error helpers, device guard and graph-cache keys.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../include/sp.h"
#include "sp_kernels.cuh"

struct sp_handle;
struct sp_batch;

namespace sp {
namespace rt {

inline sp_status fail(sp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  sp::set_last_error("%s", buf);
  return s;
}

#define SP_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(e_ == cudaErrorMemoryAllocation ? SP_ENOMEM : SP_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                      \
  } while (0)

inline uint32_t default_timeout_ms() {
  const char* s = std::getenv("SP_TIMEOUT_MS");
  if (s && *s) {
    long v = std::strtol(s, nullptr, 10);
    if (v > 0) return (uint32_t)v;
  }
  return 10000u;
}

// Make `dev` current for the scope and restore the caller's device after.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

inline size_t align256(size_t x) { return (x + 255u) & ~size_t(255u); }

// Checks every field of a configuration that the compute paths use (sizes,
// finite parameters, inhibition mode, column grid, reserved fields); sets the
// calling thread's message and returns SP_EINVAL on the first violation.
sp_status validate_config(const sp_config* c);
bool all_ones(const float* v, size_t n);
sp_status handle_wait(sp_handle* h);
sp_status handle_flush_learning(sp_handle* h);
uint32_t batch_ctas(uint32_t C, uint32_t S, uint32_t cols_per_warp = 0);
uint32_t batch_stage_cap(uint32_t need);
// The descriptor of one SP inside a multi-SP launch, in the best form it
// qualifies for (window, compact, else full); *win_bytes (nullable) receives
// the shared memory a CTA of this SP needs in the window form, 0 otherwise.
void fill_desc(sp_handle* h, sp::BatchDesc* d, uint32_t cols_per_warp = 0,
               uint32_t* win_bytes = nullptr);
// Recompute the window form's per-CTA frame bands for a new CTA split; false
// (the descriptor then leaves the window form) if they no longer fit.
bool window_rebands(sp_handle* h, sp::BatchDesc* d, uint32_t* win_bytes);
uint32_t batch_xspan_cap();

constexpr uint32_t kChunkFrames = 32;  // frames per staged chunk in sp_compute_frames
constexpr int kSlots = 2;
constexpr uint32_t kGraphMinFrames = 4;  // shorter sequences are launched directly
constexpr uint32_t kSeqMinFrames = 8;    // shorter sequences use the per-frame kernel
constexpr size_t kSeqSmemLimit = 226u * 1024u;  // 227 KiB per CTA, less static shared memory

inline bool seq_enabled() {
  const char* s = std::getenv("SP_DISABLE_CLUSTER");
  return !(s && s[0] == '1');
}
constexpr size_t kGraphCacheSize = 8;

// A recorded frame sequence is valid for exactly the buffers, sizes and
// starting (buffer parity, pending learning) state it was recorded with.
struct GraphKey {
  const uint32_t* x;
  uint64_t n, stride;
  int learn;
  uint32_t* masks;
  int cur;
  bool pending;
  bool unit_boost;  // selects the histogram path baked into the recorded launches
  uint64_t mstride; // mask stride (batches)
  uint64_t extra = 0;  // dense runs: launch shape and buffer generations baked into the launches
  const float* ovs = nullptr;  // the caller's per-frame overlap record, or nullptr
  uint64_t ovstride = 0;
  bool operator==(const GraphKey& o) const {
    return x == o.x && n == o.n && stride == o.stride && learn == o.learn && masks == o.masks &&
           cur == o.cur && pending == o.pending && unit_boost == o.unit_boost &&
           mstride == o.mstride && extra == o.extra && ovs == o.ovs && ovstride == o.ovstride;
  }
};

struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec;
  uint64_t last_use;
};

constexpr uint32_t kDenseMinFrames = 16;  // shorter inference runs use the per-frame kernel
constexpr uint64_t kDeviceWaitNs = 1000000000ull;  // default bound of an in-kernel wait: 1 s

inline bool dense_enabled() {
  const char* s = std::getenv("SP_DISABLE_TENSOR_CORES");
  return !(s && s[0] == '1');
}

// Device allocation used by the whole runtime.  SP_INJECT_ALLOC_FAILURE=1
// makes it fail as an out-of-memory device would (host-side fault injection
// for tests: nothing reaches the GPU).
inline cudaError_t device_malloc(void** p, size_t bytes) {
  const char* s = std::getenv("SP_INJECT_ALLOC_FAILURE");
  if (s && s[0] == '1') {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

inline bool graphs_enabled() {
  const char* s = std::getenv("SP_DISABLE_GRAPHS");
  return !(s && s[0] == '1');
}

}  // namespace rt
}  // namespace sp

struct sp_handle {
  sp_config cfg{};
  int device = 0;
  uint32_t C = 0, S = 0, n_words = 0, mask_words = 0, max_active = 0;
  uint64_t n_in = 0;
  void* d_block = nullptr;
  size_t device_bytes = 0;
  uint32_t* d_idx = nullptr;
  float* d_perm = nullptr;
  float* d_boost = nullptr;
  float* d_ov = nullptr;
  uint32_t* d_xsave[2] = {nullptr, nullptr};
  uint32_t* d_mask[2] = {nullptr, nullptr};
  uint32_t* d_result = nullptr;
  uint32_t* d_counter = nullptr;
  uint32_t* d_hist = nullptr;  // [S + 1], used when every boost is 1
  float* d_duty = nullptr;     // [C] active-duty cycles (tracked when duty_period > 0)
  uint32_t* d_err = nullptr;   // set by a kernel whose bounded wait expired
  uint32_t* h_err = nullptr;   // pinned copy of d_err
  // dense pools (every column sees the whole input): inference runs of frames
  // go through the tensor cores
  bool dense = false;
  bool dense_used = false;
  float* d_run_ov = nullptr;        // [run_cap][C] overlaps of a run
  uint32_t* d_run_masks = nullptr;  // [run_cap][mask_words]
  uint32_t run_cap = 0;
  void* d_compact = nullptr;        // batch compact form: cidx | cbase | conn | wide flag
  uint16_t* d_cidx = nullptr;
  uint32_t* d_cbase = nullptr;
  uint32_t* d_cconn = nullptr;
  uint32_t* d_cwide = nullptr;
  void* d_window = nullptr;         // batch window form: worg [C] | wbits [C][128] | flag
  uint32_t* d_worg = nullptr;
  uint32_t* d_wbits = nullptr;
  uint32_t* d_wbad = nullptr;
  uint32_t* d_wband = nullptr;      // [2][wband_ctas] frame rows of each batch CTA
  uint32_t wband_ctas = 0;
  int window_geom = -1;             // pools fit 64 x 64 boxes: -1 unknown, 0 no, 1 yes
  uint32_t* d_xspan = nullptr;      // [2][xspan_ctas] input-word span of each batch CTA
  uint32_t xspan_ctas = 0;
  uint8_t* d_bimg = nullptr;        // e4m3 connection image of a dense SP (tensor-core layout)
  uint8_t* d_aimg = nullptr;        // e4m3 frame image of a dense run
  size_t aimg_cap = 0;              // bytes of d_aimg
  bool bimg_stale = true;           // the permanences may have changed since d_bimg was built
  uint32_t run_gen = 0;             // bumped whenever d_run_ov / d_run_masks are reallocated
  bool unit_boost = true;
  uint32_t* h_result = nullptr;  // pinned [1 + C]
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;  // stream of the last call
  cudaEvent_t ev_switch = nullptr;
  cudaEvent_t ev_wait = nullptr;
  int cur = 0;
  bool pending = false;  // the previous frame's learning is not applied yet
  uint64_t frames = 0;
  uint32_t timeout_ms = 10000;
  int grid = 1;
  // sp_compute_frames staging (allocated on first use)
  uint32_t* d_stage = nullptr;   // [sp::rt::kSlots][kChunkFrames][n_words]
  uint32_t* d_mstage = nullptr;  // [sp::rt::kSlots][kChunkFrames][mask_words]
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_h2d[sp::rt::kSlots] = {}, ev_comp[sp::rt::kSlots] = {}, ev_d2h[sp::rt::kSlots] = {};
  // recorded frame sequences (CUDA graphs), replayed instead of n launches
  std::vector<sp::rt::GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;  // private stream used only for recording
  uint64_t graph_clock = 0;
  sp_batch* batch = nullptr;  // set while the handle is a member of a batch
  // persistent cluster path for frame sequences (state in shared memory)
  bool seq_ok = false;
  uint32_t seq_Q = 0, seq_Cq = 0, seq_band_max = 0;
  size_t seq_smem = 0;
};
