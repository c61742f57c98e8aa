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
  uint32_t* result_copy;     // optional second copy of result[0..n] (serving), or nullptr
  float* ov_copy;            // optional copy of this frame's boosted overlaps [C] (a
                             // caller's per-frame overlap record), or nullptr
  float* duty;               // [C] active-duty cycles updated each frame, or nullptr
  float duty_period;
  const uint32_t* xspan;     // per CTA: [lo, hi) input words its columns read, or nullptr
  // compact form (batches; nullptr = use idx/perm only), laid out as described
  // at launch_compact
  const uint16_t* cidx;
  const uint32_t* cbase;
  uint32_t* conn;
  // window form (batches; nullptr = not used), laid out as described at
  // launch_window: per column the origin of a 64 x 64 box holding its pool
  // and a bitmap of its connected synapses inside the box
  const uint32_t* worg;
  uint32_t* wbits;
  const uint32_t* wband;  // per CTA: first frame row and row count its columns read
  uint32_t wpr;           // frame words per row (input_w / 32)
  uint32_t win_w;         // input_w
  uint32_t C, S, n_words, mask_words;
  float thr, inc, dec;
  uint32_t min_overlap, k;
  uint32_t inhibition;       // 0 global, 1 local
  uint32_t gw, gh, radius;   // column grid for local inhibition
  uint32_t learn_next;       // 1: the SP's next frame learns this frame's winners, so
                             // the last CTA asks L2 for their indices and permanences
};

// One SP of a batch (device-resident descriptor; pointers into its handle).
struct BatchDesc {
  const uint32_t* idx;
  float* perm;
  const float* boost;
  float* ov;
  uint32_t *xsave0, *xsave1, *mask0, *mask1;
  uint32_t* result;
  uint32_t* counter;
  uint32_t* hist;       // nullptr unless global inhibition with unit boosts
  float* duty;          // nullptr unless duty cycles are tracked
  float duty_period;
  const uint32_t* xspan;  // per CTA of this SP: [lo, hi) input words read (nullable)
  const uint16_t* cidx;   // compact form (nullable), as in StepArgs
  const uint32_t* cbase;
  uint32_t* conn;
  const uint32_t* worg;   // window form (nullable), as in StepArgs
  uint32_t* wbits;
  const uint32_t* wband;
  uint32_t wpr, win_w;
  uint64_t frame_off;   // words: this SP's frame inside one batch frame
  uint64_t mask_off;    // words: this SP's mask inside one batch mask record
  uint64_t ov_off;      // floats: this SP's overlaps inside one batch overlap record
  uint32_t C, S, n_words, mask_words;
  float thr, inc, dec;
  uint32_t min_overlap, k, inhibition, gw, gh, radius;
  uint32_t cta_first, n_ctas;  // this SP's CTAs in the batch grid
};

// A sequence of batch frames in one persistent launch (see sp_batch_run_kernel).
struct BatchRunArgs {
  const BatchDesc* desc;
  const uint32_t* cta_inst;     // [items_per_frame] SP of each CTA of one frame's grid
  uint32_t items_per_frame;
  uint32_t n_frames;
  const uint32_t* frames;       // batch frame t at frames + t * stride
  uint64_t stride;
  uint32_t* masks_out;          // batch mask record t at masks_out + t * mstride (nullable)
  uint64_t mstride;
  float* ov_out;                // batch overlap record t at ov_out + t * ov_stride (nullable)
  uint64_t ov_stride;
  uint32_t cur0, pending0, learn;  // parity and pending learning before frame 0
  uint32_t epoch;               // base of the done values (0: flags cleared per launch)
  unsigned long long* work;     // item counter, 0 at launch
  uint32_t* abort;              // 0 at launch; set when a wait gives up
  uint32_t* done;               // per SP: epoch + t + 1 once frame t is complete
  uint32_t* err;                // set to 1 if a bounded wait expired (nullable)
  uint32_t stage_cap, xspan_cap;
  uint32_t win_cap;             // bytes of shared memory for a window-form CTA's band
  uint64_t wait_ns;             // bound of an item's wait for its SP's previous frame
};

// Per-launch entry of one SP when a launch steps a chosen subset of SPs,
// each with its own state (serving: streams advance independently).
struct TickMember {
  const uint32_t* x;   // this SP's frame (device)
  uint32_t flags;      // bit 0 parity, bit 1 learning pending, bit 2 learn, bit 3 save frame
  uint32_t cta_first;  // this SP's first CTA in this launch
  uint32_t out_off;    // words: its [count, list...] in results_out
  uint32_t pad;
};
enum : uint32_t { kTickCur = 1u, kTickPending = 2u, kTickLearn = 4u, kTickSave = 8u };

// One frame for every SP of a batch.  All members share the buffer parity
// `cur` and the pending-learning flag (they advance in lockstep).
struct BatchArgs {
  const BatchDesc* desc;
  const uint32_t* cta_inst;     // [grid] SP of each CTA
  const uint32_t* frames;       // one batch frame (members at their frame_off)
  const uint32_t* prev_frames;  // the previous batch frame, or nullptr (saved copies)
  uint32_t* masks_out;          // one batch mask record, or nullptr
  float* ov_out;                // one batch overlap record, or nullptr
  uint32_t cur, pending, learn;
  uint32_t save;                // copy each member's frame for next-call learning
  const TickMember* tick;       // if set: per-SP frame/state (indexed like desc); the
                                // uniform fields above are then ignored
  uint32_t* results_out;        // with tick: per-SP [count, ascending list]
  uint32_t stage_cap;           // bytes of dynamic shared memory for staging state (0: none)
  uint32_t xspan_cap;           // bytes of shared memory for a CTA's input span (0: none)
  uint32_t win_cap;             // bytes of shared memory for a window-form CTA's band
  uint32_t* err;                // set to 1 if a bounded wait expired (nullable)
};

cudaError_t launch_batch_step(const BatchArgs& a, uint32_t n_ctas, uint32_t max_C,
                              cudaStream_t stream);
// One persistent launch over r.n_frames batch frames (grid sized to the
// resident CTAs) with compiled schedule `schedule` (0: the default; out of
// range: the default); r.work and r.abort must be 0.
cudaError_t launch_batch_run(const BatchRunArgs& r, uint32_t max_C, uint32_t schedule,
                             cudaStream_t stream);
// The compiled schedules of the persistent batch pass: how many, and the
// resident CTAs per SM and columns per warp in flight of schedule i (false
// when i is out of range).
uint32_t batch_schedule_count();
bool batch_schedule(uint32_t i, uint32_t* ctas_per_sm, uint32_t* cols_in_flight);
// Compact form of an SP's pools and connectivity (S <= 256), rows padded to
// cS = S rounded up to a multiple of 32 synapses and laid out lane-strided
// (see sp_step.cu): cbase[c] = min_s idx[c][s], 16-bit offsets idx[c][s] -
// cbase[c], one connected bit (perm[c][s] >= thr) per synapse, padding
// never connected.  *wide is set to 1 if some column's pool spans more than
// 65536 inputs (the form is unusable then).
cudaError_t launch_compact(const uint32_t* idx, const float* perm, uint32_t C, uint32_t S,
                           float thr, uint16_t* cidx, uint32_t* cbase, uint32_t* conn,
                           uint32_t* wide, cudaStream_t stream);

// Window form of an SP whose input is W pixels wide (W % 32 == 0): for every
// column, worg[c] = (oy << 16) | ox, the smallest row and column of its pool's
// pixels, and wbits[c][128] the connected synapses (perm >= thr) as a 64 x 64
// bitmap of the box starting there -- row r, pixel ox + j is bit j % 32 of
// word 2r + j / 32 of the row pair, stored so that lane l of a warp loads one
// 16-byte vector {row l low, row l high, row l + 32 low, row l + 32 high} at
// word 4l.  *bad is set to 1 if a pool does not fit a 64 x 64 box (or the
// box origin does not fit 16 bits); the form is unusable then.
cudaError_t launch_window(const uint32_t* idx, const float* perm, uint32_t C, uint32_t S,
                          uint32_t W, float thr, uint32_t* worg, uint32_t* wbits, uint32_t* bad,
                          cudaStream_t stream);
// The frame rows each of n_ctas blocks of consecutive columns reads in the
// window form: out[2b] = first row, out[2b + 1] = row count (0 for an empty
// block); rows past H - 1 are never read.
cudaError_t launch_window_bands(const uint32_t* worg, uint32_t C, uint32_t H, uint32_t n_ctas,
                                uint32_t* out, cudaStream_t stream);
// Shared memory of a window-form CTA: `rows` staged frame rows of wpr words
// (input_w / 32), the per-warp rings of bitmap slots and the learning
// scratch.
uint32_t window_smem_bytes(uint32_t rows, uint32_t wpr);

// Per-CTA input-word spans of an SP split into n_ctas blocks of consecutive
// columns: out[2b], out[2b+1] = lowest and one past the highest input word
// that block b's pools index (0, 0 for an empty block).
cudaError_t launch_xspan(const uint32_t* idx, uint32_t C, uint32_t S, uint32_t n_ctas,
                         uint32_t* out, cudaStream_t stream);

// Shared memory a batch CTA needs for its warps' rings of column slots (pool and
// permanence rows staged by bulk copy); 0 when the SP cannot be staged.
uint32_t batch_stage_bytes(uint32_t C, uint32_t S, uint32_t n_ctas);

// Learning of one frame applied on its own (used to flush pending learning).
struct LearnArgs {
  const uint32_t* idx;
  float* perm;
  const uint32_t* x;     // the frame the winners won on
  const uint32_t* mask;  // its winner mask
  uint32_t C, S;
  float inc, dec;
};

// A whole frame sequence of one SP in one persistent cluster launch
// (sp_seq_cluster.cu): the state stays in the cluster's shared memory.
constexpr int kSeqThreads = 512;
constexpr uint32_t kSeqMaxCluster = 16;

struct SeqArgs {
  const uint32_t* idx;        // [C][S]
  float* perm;                // [C][S], rows that learned are written back at the end
  const float* boost;         // [C]
  const uint32_t* frames;     // frame f at frames + f * stride
  uint64_t stride;
  uint32_t n_frames;
  int learn;
  const uint32_t* pend_mask;  // learning left pending by the previous call, or nullptr
  const uint32_t* pend_x;     // ... and the frame it belongs to
  uint32_t* masks_out;        // [n_frames][mask_words] or nullptr
  uint32_t* mask_last;        // last frame's mask [mask_words]
  uint32_t* result;           // last frame: [0] count, [1..] ascending winners
  float* ov_out;              // last frame's boosted overlaps [C]
  float* ov_all;              // [n_frames][C] boosted overlaps of every frame, or nullptr
  uint32_t C, S, n_words, mask_words;
  uint32_t Cq;                // columns per CTA (multiple of 32)
  uint32_t band_max;          // words of the largest per-CTA input band (multiple of 4)
  uint32_t vec16;             // frames 16-byte aligned with stride, n_words % 4 == 0
  float thr, inc, dec;
  uint32_t min_overlap, k, inhibition, gw, gh, radius;
  uint32_t unit_boost;
  float* duty;                // [C] active-duty cycles, or nullptr
  float duty_period;
};

size_t seq_smem_bytes(uint32_t C, uint32_t S, uint32_t Cq, uint32_t band_max);
cudaError_t seq_kernel_init(size_t smem_bytes);
cudaError_t seq_max_active_clusters(uint32_t Q, size_t smem_bytes, int* out);
cudaError_t launch_seq(const SeqArgs& a, uint32_t Q, size_t smem_bytes, cudaStream_t stream);

// Dense pools on the tensor cores (sp_dense_tc.cu): the raw overlaps of a run
// of frames without learning as one {0,1} matrix product.  Both operands are
// e4m3 images laid out block by block as the tensor core reads them from
// shared memory: block (tile, slice) covers rows tile * R .. + R - 1 (R = 256
// columns for the connection image, 128 frames for the frame image) and
// inputs slice * 128 .. + 127, zero past the ends.
struct DenseArgs {
  const float* perm;        // [C][K]
  uint8_t* bimg;            // connection image, dense_bimg_bytes(C, K)
  uint8_t* aimg;            // frame image, dense_aimg_bytes(n_frames, K)
  uint32_t n_slices;        // dense_slices(K)
  uint32_t pack;            // 1: rebuild bimg from perm (the permanences changed)
  const float* boost;       // [C]
  const uint32_t* frames;   // frame f at frames + f * stride
  uint64_t stride;
  uint32_t n_frames, C, K, n_words;
  float thr;
  uint32_t min_overlap;
  float* ov;                // [n_frames][C] boosted overlaps (out)
  uint32_t* err;            // set to 1 if a bounded wait expired
};

// Alg. 2 for every frame of a run whose overlaps are rows of ov.
struct FrameInhibitArgs {
  const float* ov;          // [n_frames][C]
  uint32_t n_frames, C, mask_words, k, inhibition, gw, gh, radius;
  uint32_t unit_S;          // S when every boost is 1 (histogram select), else 0
  uint32_t* masks_out;      // frame f's mask at masks_out + f * masks_stride, or nullptr
  uint64_t masks_stride;    // words between consecutive frames' masks
  uint32_t* mask_last;      // the last frame's mask
  uint32_t* result;         // the last frame's [count, list...]
  float* ov_last;           // the last frame's overlaps [C]
};

size_t dense_smem_bytes();
cudaError_t dense_init();
size_t dense_bimg_bytes(uint32_t C, uint32_t K);
size_t dense_aimg_bytes(uint32_t n_frames, uint32_t K);
uint32_t dense_slices(uint32_t K);
// Connection images of the SPs whose pack flag is set / frame images of the
// run (args: a device array of n entries, or one SP by value).
cudaError_t launch_conn_image(const DenseArgs* args, uint32_t n, uint32_t max_C, uint32_t max_K,
                              cudaStream_t stream);
cudaError_t launch_conn_image_one(const DenseArgs& a, cudaStream_t stream);
cudaError_t launch_frame_image(const DenseArgs* args, uint32_t n, uint32_t max_frames,
                               uint32_t max_K, cudaStream_t stream);
cudaError_t launch_frame_image_one(const DenseArgs& a, cudaStream_t stream);
cudaError_t launch_dense_overlap(const DenseArgs& a, cudaStream_t stream);
// Several SPs in one launch: args is a device array of n entries; every SP
// covers at most max_C columns and max_frames frames.
cudaError_t launch_dense_overlap_many(const DenseArgs* args, uint32_t n, uint32_t max_C,
                                      uint32_t max_frames, cudaStream_t stream);
cudaError_t frame_inhibit_init();
size_t frame_inhibit_smem(uint32_t C, uint32_t unit_S);
size_t frame_inhibit_smem_limit();
cudaError_t launch_frame_inhibit(const FrameInhibitArgs& a, cudaStream_t stream);
// all_global: every member inhibits globally (one warp per frame then
// selects the winners when max_C <= 2048).
cudaError_t launch_frame_inhibit_many(const FrameInhibitArgs* args, uint32_t n, uint32_t max_C,
                                      uint32_t max_unit_S, uint32_t max_frames, bool all_global,
                                      cudaStream_t stream);
cudaError_t launch_duty_run(const uint32_t* masks, uint32_t n_frames, uint32_t mask_words,
                            uint32_t C, float* duty, float period, cudaStream_t stream);

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
