// Device-side argument blocks and launchers of the Spatial Pooler kernels.
//
// One fused kernel per frame (sp_step): every CTA computes Alg. 1 for a
// strided set of columns (one warp per column), after first applying the
// previous frame's learning to the columns that won it; the last CTA to
// finish (ticket counter, no spinning) runs Alg. 2 over all overlaps and
// publishes the ascending winner list and the winner bitmask.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sp {

constexpr int kStepThreads = 128;  // 4 warps: one column per warp at a time
constexpr int kStepWarps = kStepThreads / 32;

// Everything one frame of one SP needs.  Passed by value.
struct StepArgs {
  const uint32_t* idx;       // [C][S] input indices
  float* perm;               // [C][S] permanences (updated for pending learning)
  const float* boost;        // [C]
  float* ov;                 // [C] boosted overlaps (out)
  const uint32_t* x;         // this frame, packed bits
  const uint32_t* x_prev;    // previous frame (pending learning), or nullptr
  const uint32_t* mask_prev; // previous frame's winners (pending learning), or nullptr
  uint32_t* x_save;          // copy of x kept for next-frame learning, or nullptr
  uint32_t* mask_out;        // this frame's winner mask [mask_words]
  uint32_t* mask_copy;       // optional second copy of the mask (caller array), or nullptr
  uint32_t* result;          // [0] = number of winners, [1..] ascending winners
  uint32_t* counter;         // last-CTA ticket, 0 between launches
  uint32_t* hist;            // [S + 1] counts of surviving raw overlaps, 0 between
                             // launches; used (global inhibition) when every boost
                             // is exactly 1, else nullptr (radix select instead)
  uint32_t C, S, n_words, mask_words;
  float thr, inc, dec;
  uint32_t min_overlap, k;
  uint32_t inhibition;       // 0 global, 1 local
  uint32_t gw, gh, radius;   // column grid for local inhibition
};

// Learning of one frame applied on its own (used to flush pending learning).
struct LearnArgs {
  const uint32_t* idx;
  float* perm;
  const uint32_t* x;     // the frame the winners won on
  const uint32_t* mask;  // its winner mask
  uint32_t C, S;
  float inc, dec;
};

// Dynamic shared memory of the fused kernel for C columns.
size_t step_smem_bytes(uint32_t C);

// Launch the fused step on `stream`.  Returns the launch error.
cudaError_t launch_step(const StepArgs& a, int grid, cudaStream_t stream);
cudaError_t launch_learn(const LearnArgs& a, cudaStream_t stream);

// Grid of the fused step for C columns on the current device.
int step_grid(uint32_t C);

// One-time per-process attribute set-up (max dynamic shared memory).
cudaError_t kernels_init();

// Record the calling thread's message for sp_last_error().
void set_last_error(const char* fmt, ...);

}  // namespace sp
