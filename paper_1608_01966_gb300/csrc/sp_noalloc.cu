// sp_step_noalloc: one Spatial Pooler frame on caller-owned device state,
// with no memory allocation of any kind.
//
// Why it exists: some callers cannot allocate device memory when they run a
// frame.  A real-time video pipeline stage, for instance, handles each frame
// in a callback that must not block, and cudaMalloc / cudaFree may
// synchronise the whole device; a host that admits work against a fixed
// device-memory budget, or a plugin host that owns every allocation itself,
// cannot let the library grow its footprint behind its back.  Such callers
// keep the SP state (pools, permanences, boosts) in their own buffers and
// call this entry point.
//
// The only memory the fused step kernel needs beyond the caller's inputs
// and outputs -- the per-column boosted overlaps read back by the last CTA,
// and that CTA's ticket counter -- lives in the file-scope array below.  It
// is reserved when the library is loaded (every GPU that loads the library
// holds it until the process exits) and is shared by every call.
#include <cuda_runtime.h>

#include "../../include/sp.h"
#include "sp_internal.h"
#include "sp_kernels.cuh"

namespace {

// [0, SP_NOALLOC_MAX_COLUMNS): boosted overlaps of the current call;
// [SP_NOALLOC_MAX_COLUMNS]: the last-CTA ticket counter (cleared every call).
constexpr uint32_t kScratchWords = SP_NOALLOC_MAX_COLUMNS + 64u;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

sp_status noalloc_fail(sp_status s, const char* msg) {
  sp::set_last_error("sp_step_noalloc: %s", msg);
  return s;
}

// The device address of the scratch array in the current device's context.
// In host code g_noalloc_scratch names a host-side stand-in, never a device
// address, so it is not passed to a kernel directly.  The address is looked
// up on every call (a lookup, no allocation): a context that was destroyed
// and created again -- a device reset between calls -- loads the library's
// device code again, possibly at another address, so a remembered address
// could be stale.  The kernels' attributes are set again for the same reason.
sp_status scratch_address(uint32_t** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    sp::set_last_error("sp_step_noalloc: cudaGetSymbolAddress failed: %s",
                       cudaGetErrorString(e));
    return SP_ECUDA;
  }
  if (sp::kernels_init() != cudaSuccess)
    return noalloc_fail(SP_ECUDA, "kernel attribute set-up failed");
  *out = static_cast<uint32_t*>(p);
  return SP_OK;
}

bool aligned(const void* p, uintptr_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; }

}  // namespace

extern "C" {

SP_API sp_status sp_step_noalloc(const sp_config* cfg, const uint32_t* d_idx, float* d_perm,
                                 const float* d_boost, const uint32_t* d_input, int learn,
                                 uint32_t* d_active_mask, uint32_t* d_active_list,
                                 void* stream) {
  if (!cfg || !d_idx || !d_perm || !d_boost || !d_input || !d_active_mask || !d_active_list)
    return noalloc_fail(SP_EINVAL, "NULL argument");
  if (cfg->num_columns > SP_NOALLOC_MAX_COLUMNS)
    return noalloc_fail(SP_EINVAL, "num_columns must be in [1, SP_NOALLOC_MAX_COLUMNS]");
  // the same configuration checks as sp_create (the message names the field)
  if (sp::rt::validate_config(cfg) != SP_OK) return SP_EINVAL;
  const uint64_t n_in = (uint64_t)cfg->input_w * cfg->input_h;
  const uint32_t C = cfg->num_columns, S = cfg->synapses_per_column;
  const bool vec = S % 4u == 0u;
  if (!aligned(d_idx, vec ? 16 : 4) || !aligned(d_perm, vec ? 16 : 4) || !aligned(d_boost, 4) ||
      !aligned(d_input, 4) || !aligned(d_active_mask, 4) || !aligned(d_active_list, 4))
    return noalloc_fail(SP_EINVAL, "device pointers misaligned (16 bytes for idx/perm when S % 4 == 0)");

  uint32_t* scratch = nullptr;
  sp_status s = scratch_address(&scratch);
  if (s != SP_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* counter = scratch + SP_NOALLOC_MAX_COLUMNS;
  // the ticket counter must start at zero; the overlaps are fully rewritten
  if (cudaMemsetAsync(counter, 0, sizeof(uint32_t), st) != cudaSuccess)
    return noalloc_fail(SP_ECUDA, "clearing the scratch counter failed");

  sp::StepArgs a{};
  a.idx = d_idx;
  a.perm = d_perm;
  a.boost = d_boost;
  a.ov = reinterpret_cast<float*>(scratch);
  a.x = d_input;
  a.mask_out = d_active_mask;
  a.result = d_active_list;
  a.counter = counter;
  a.C = C;
  a.S = S;
  a.n_words = (uint32_t)((n_in + 31) / 32);
  a.mask_words = (C + 31) / 32;
  a.thr = cfg->connect_threshold;
  a.inc = cfg->perm_inc;
  a.dec = cfg->perm_dec;
  a.min_overlap = cfg->min_overlap;
  a.k = cfg->winners_set_size;
  a.inhibition = cfg->inhibition;
  a.gw = cfg->col_grid_w;
  a.gh = cfg->col_grid_h;
  a.radius = cfg->local_radius;
  if (sp::launch_step(a, sp::step_grid(C), st) != cudaSuccess)
    return noalloc_fail(SP_ECUDA, "step kernel launch failed");
  if (learn) {
    sp::LearnArgs l{};
    l.idx = d_idx;
    l.perm = d_perm;
    l.x = d_input;
    l.mask = d_active_mask;
    l.C = C;
    l.S = S;
    l.inc = cfg->perm_inc;
    l.dec = cfg->perm_dec;
    if (sp::launch_learn(l, st) != cudaSuccess)
      return noalloc_fail(SP_ECUDA, "learning kernel launch failed");
  }
  return SP_OK;
}

}  // extern "C"
