/*
 * sp.h — C ABI of the GB300 (sm_103a) Spatial Pooler library, libsp_gb300.so.
 *
 * The library runs the data-parallel hot path of the HTM Spatial Pooler of
 * Wielgosz & Pietron, "OpenCL-accelerated object classification in video
 * streams using Spatial Pooler of Hierarchical Temporal Memory":
 *
 *   overlap     Alg. 1 (Section 1.1): per column, the number of connected
 *               potential synapses (permanence >= connect_threshold, fp32)
 *               whose input bit is 1; zero when below min_overlap, else
 *               multiplied by the column's boost (one fp32 multiply, as the
 *               paper's overlap unit does, Section 3 "Hardware architecture");
 *   inhibition  Alg. 2 (Section 1.1) read as a rank count: a column is active
 *               iff its overlap is > 0 and fewer than winners_set_size columns
 *               of its neighbourhood beat it (higher overlap, or equal overlap
 *               and lower index); the neighbourhood is the whole SP (global)
 *               or the (2r+1)^2 window on the column grid, clipped at the
 *               edges (local);
 *   learning    Section 1.1 (kept on the CPU in the paper; increments of
 *               Table 2): every potential synapse of an active column moves
 *               to min(1, p + perm_inc) when its input bit is 1, else to
 *               max(0, p - perm_dec), each add one fp32 round-to-nearest op.
 *
 * A binary frame goes in, the sparse set of active columns comes out
 * (Section 2, "Processing flow"), in learning or inference mode (Section 4.1).
 * Results are bit-identical to the plain CPU definition: overlaps are integer
 * counts, fp32 steps are single round-to-nearest operations (no FMA), and
 * the winner set is unique under the total order above.
 *
 * Input format (Section 4.4 proposes boolean instead of integer input to cut
 * transfers ~32x): input bit i is bit (i & 31) of 32-bit word i >> 5, LSB
 * first; a W x H frame is flattened row-major, i = y*W + x.  A frame is
 * n_words = ceil(W*H / 32) words; unused high bits of the last word are
 * ignored.  Active-column masks use the same packing over columns,
 * mask_words = ceil(C / 32) words.
 *
 * State: each handle owns its state on the GPU it was created on (the
 * current CUDA device at sp_create): pools idx[C][S] (uint32), permanences perm[C][S] (fp32), boost[C] (fp32),
 * the last frame's overlaps, and double-buffered masks/inputs.  State never
 * returns to the host except through the getters.
 *
 * Ordering: a handle is bound to one CUDA stream (its own, or the one passed
 * to the *_device calls) and is NOT thread-safe; separate handles are
 * independent.  Compute calls are asynchronous; sp_active_columns, the
 * getters and sp_sync wait (bounded, see sp_set_timeout_ms) for the work
 * they read.  Learning of a frame is applied lazily, before the next frame's
 * overlap on the same pass over the state, or by any getter that reads
 * permanences; the observable results are those of applying it at the end
 * of its own frame.
 *
 * Buffers: caller buffers are borrowed only for the call, or, for the
 * asynchronous calls, until the next sp_sync / sp_active_columns / getter /
 * sp_destroy of that handle.  The library never frees caller memory.
 *
 * Errors: every call returns an sp_status; no C++ exception crosses the
 * ABI.  On error nothing observable changes unless stated.  sp_last_error()
 * gives a human-readable message for the calling thread's last failure.
 */
#ifndef SP_H
#define SP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(SP_BUILD_LIBRARY)
#define SP_API __attribute__((visibility("default")))
#else
#define SP_API
#endif

#define SP_ABI_VERSION 2u
#define SP_MAX_COLUMNS 16384u        /* per SP instance */
#define SP_MAX_SYNAPSES 65536u       /* per column */
#define SP_MAX_INPUT_BITS (1u << 28) /* per frame */

typedef struct sp_handle sp_handle; /* opaque, owned by the library */

typedef enum {
  SP_OK = 0,
  SP_EINVAL = 1,   /* invalid argument or configuration */
  SP_ENOMEM = 2,   /* device or pinned host allocation failed */
  SP_ECUDA = 3,    /* a CUDA runtime call failed (see sp_last_error) */
  SP_ETIMEOUT = 4, /* a bounded wait on device work expired */
  SP_EBUSY = 5,    /* resource in use (e.g. capacity exhausted) */
  SP_ENOTSUP = 6   /* valid but unsupported combination */
} sp_status;

enum { SP_POOL_UNIFORM = 0, SP_POOL_WINDOW = 1, SP_POOL_DENSE = 2 };
/* SP_INHIBIT_PAPER_LITERAL: Alg. 2 word for word over the whole SP, for
 * comparison with the rank count: a column is active iff its overlap exceeds
 * both 1 and the k-th largest overlap among the other columns (ties at the
 * boundary all lose, so fewer than k columns may win). */
enum { SP_INHIBIT_GLOBAL = 0, SP_INHIBIT_LOCAL = 1, SP_INHIBIT_PAPER_LITERAL = 2 };

/* Configuration of one SP (Table 2 names the paper's defaults). */
typedef struct {
  uint32_t abi_version;         /* must be SP_ABI_VERSION */
  uint32_t input_w, input_h;    /* n_in = input_w * input_h bits; h = 1 for flat input */
  uint32_t num_columns;         /* C */
  uint32_t col_grid_w, col_grid_h; /* column grid (C = w*h) for windowed pools and
                                      local inhibition; 0,0 = none */
  uint32_t synapses_per_column; /* S (= n_in for SP_POOL_DENSE) */
  uint32_t pool_mode;           /* SP_POOL_* (sp_create only) */
  uint32_t rf_w, rf_h;          /* receptive-field window for SP_POOL_WINDOW */
  float connect_threshold;      /* connected iff perm >= threshold (fp32) */
  float perm_inc, perm_dec;     /* learning steps */
  float perm_init_lo, perm_init_hi; /* initial permanences U[lo, hi) (sp_create) */
  uint32_t min_overlap;         /* counts below this are zeroed (Alg. 1) */
  uint32_t winners_set_size;    /* k of Alg. 2 */
  uint32_t inhibition;          /* SP_INHIBIT_* */
  uint32_t local_radius;        /* r: (2r+1)^2 window for SP_INHIBIT_LOCAL */
  uint64_t seed;                /* pools / permanences for sp_create */
  float duty_period;            /* > 0: track each column's active-duty cycle,
                                   d <- d + (a - d) / duty_period per frame (a = 1 if
                                   active); 0 = off.  The paper only cites the
                                   Numenta duty-cycle rules; this moving average is
                                   the library's own definition. */
  uint32_t reserved;            /* must be 0 */
} sp_config;

/* Sizes of a handle's state and buffers. */
typedef struct {
  uint32_t num_columns, synapses_per_column;
  uint64_t input_bits;
  uint32_t input_words;  /* ceil(input_bits / 32) */
  uint32_t mask_words;   /* ceil(num_columns / 32) */
  uint32_t max_active;   /* upper bound on active columns per frame */
  int device;            /* CUDA device the state lives on */
  uint64_t device_bytes; /* device memory held by the handle */
  uint64_t frames;       /* frames computed so far */
} sp_info;

/* Fill *cfg with the paper's Table 2 defaults: 2048 columns, 128 synapses,
 * perm_inc = perm_dec = 0.1, min_overlap 8, winners_set_size 40, initial
 * permanence 0.21, over a 240 x 134 input (Table 1 frame size) with uniform
 * pools and global inhibition; connect_threshold 0.2 (not given by the
 * paper).  Returns SP_EINVAL if cfg is NULL. */
SP_API sp_status sp_config_init(sp_config* cfg);

/* Create an SP on the current CUDA device, drawing pools and permanences
 * from cfg->seed (include/sp_synth.h recipes: uniform, windowed or dense
 * pools; permanences U[perm_init_lo, perm_init_hi)); boosts start at 1.
 * *out receives the handle (NULL on failure). SP_EINVAL on a bad config,
 * SP_ENOMEM / SP_ECUDA on allocation failure. */
SP_API sp_status sp_create(const sp_config* cfg, sp_handle** out);

/* Create an SP from caller state (host arrays, copied as given): idx[C][S]
 * input indices (each < n_in; ascending rows give the best locality),
 * perm[C][S] in [0, 1], boost[C] finite and >= 0 (NULL = all 1). */
SP_API sp_status sp_create_from_state(const sp_config* cfg, const uint32_t* idx,
                                      const float* perm, const float* boost,
                                      sp_handle** out);

/* Free the handle and its device state after its pending work (bounded
 * wait).  NULL-safe. */
SP_API void sp_destroy(sp_handle* h);

SP_API sp_status sp_get_info(const sp_handle* h, sp_info* out);

/* One frame from host memory (input_words words; pinned memory gives a true
 * asynchronous copy).  learn != 0 applies the learning rule for this frame.
 * Asynchronous on the handle's stream. */
SP_API sp_status sp_compute(sp_handle* h, const uint32_t* input_bits, int learn);

/* One frame already on the device (input_words words at d_bits, 4-byte
 * aligned), enqueued on `stream` (a cudaStream_t; NULL = the handle's own
 * stream, cudaStreamLegacy = the legacy default stream).  The handle then stays on that stream until its next call. */
SP_API sp_status sp_compute_device(sp_handle* h, const uint32_t* d_bits, int learn,
                                   void* stream);

/* n_frames frames on the device, frame t at d_frames + t * frame_stride_words
 * (stride >= input_words), in order, all with the same learn flag, with the
 * results of n_frames single-frame calls.  Execution: inference runs of an SP
 * with dense pools go through the tensor cores (as sp_batch_infer_device);
 * otherwise one persistent launch of a thread-block cluster holding the SP's
 * state runs the whole sequence when the state fits, else one fused kernel
 * per frame (replayed as a recorded graph for repeated sequences).  If
 * d_active_masks is not NULL, frame t's active set is written there as
 * mask_words words at d_active_masks + t * mask_words.  Asynchronous on
 * `stream` (NULL = the handle's stream). */
SP_API sp_status sp_compute_frames_device(sp_handle* h, const uint32_t* d_frames,
                                          uint32_t n_frames, uint64_t frame_stride_words,
                                          int learn, uint32_t* d_active_masks,
                                          void* stream);

/* sp_compute_frames_device that also records the boosted overlaps of every
 * frame -- Alg. 1's output (Section 1.1) before inhibition, the values
 * Alg. 2 ranks -- so that each frame's overlaps, not only the last one's
 * (sp_get_overlaps), can be checked: frame t's C floats go to
 * d_overlaps + t * C (device, 4-byte aligned, caller-owned, n_frames * C
 * floats).  d_overlaps NULL records nothing; every other argument, the
 * execution and the results are those of sp_compute_frames_device.
 * SP_EINVAL for a misaligned pointer (nothing enqueued). */
SP_API sp_status sp_compute_frames_overlaps_device(sp_handle* h, const uint32_t* d_frames,
                                                   uint32_t n_frames, uint64_t frame_stride_words,
                                                   int learn, uint32_t* d_active_masks,
                                                   float* d_overlaps, void* stream);

/* n_frames frames from host memory (frame t at h_frames + t * stride words)
 * with their active masks written to host memory h_active_masks
 * ([n_frames][mask_words], NULL = not returned).  Copies are staged in
 * chunks and overlapped with compute on a second stream.  Synchronous:
 * returns when the masks are in host memory. */
SP_API sp_status sp_compute_frames(sp_handle* h, const uint32_t* h_frames, uint32_t n_frames,
                                   uint64_t frame_stride_words, int learn,
                                   uint32_t* h_active_masks);

/* Wait (bounded) for the last frame and copy its active columns, ascending,
 * into out[0..n).  If cap < n, nothing is copied, *n is set and SP_EINVAL is
 * returned. */
SP_API sp_status sp_active_columns(sp_handle* h, uint32_t* out, uint32_t cap, uint32_t* n);

/* Boosted overlaps of the last frame (C floats, host). */
SP_API sp_status sp_get_overlaps(sp_handle* h, float* out);

/* Permanences [C][S] (host), in the pool order, after all learning so far. */
SP_API sp_status sp_get_permanences(sp_handle* h, float* out);

/* Potential pools [C][S] (host). */
SP_API sp_status sp_get_pool(sp_handle* h, uint32_t* out);

/* Active-duty cycles [C] (host); SP_EINVAL unless duty_period > 0. */
SP_API sp_status sp_get_duty_cycles(sp_handle* h, float* out);

/* Checkpoint: write the SP (configuration, pools, permanences with all
 * learning so far applied, boosts, duty cycles, frame count) to a file.
 * Bounded wait for the handle's work.  SP_EINVAL on I/O errors. */
SP_API sp_status sp_save(sp_handle* h, const char* path);

/* Create an SP on the current device from a file written by sp_save;
 * continuing it gives the results of never having stopped. */
SP_API sp_status sp_load(const char* path, sp_handle** out);

/* Boosts [C] (host). */
SP_API sp_status sp_get_boost(sp_handle* h, float* out);

/* Replace the boosts (host array of C finite values >= 0). */
SP_API sp_status sp_set_boost(sp_handle* h, const float* boost);

/* Wait (bounded) until all work enqueued on the handle has finished. */
SP_API sp_status sp_sync(sp_handle* h);

/* Bound, in milliseconds, of every wait of this handle (default 10000;
 * 0 restores the default).  An expired wait returns SP_ETIMEOUT and leaves
 * the work running. */
SP_API sp_status sp_set_timeout_ms(sp_handle* h, uint32_t ms);

/* ---- Batches of SPs ------------------------------------------------------
 *
 * The paper's 'Multiple HTMs' setup (Section 3, "Outer Structure") runs one
 * SP per object class; a video server runs one per stream.  A batch steps
 * many independent SPs -- of any shapes and parameters -- with one kernel
 * launch per frame: every member computes one frame (overlap, inhibition,
 * learning) exactly as sp_compute would, and its results are bit-identical
 * to running it alone.
 *
 * Members are existing handles on the same device.  While a handle belongs
 * to a batch, its own compute calls and getters return SP_EBUSY; the batch
 * advances all members in lockstep.  sp_batch_destroy hands the members back
 * (state, overlaps, last active list and pending learning intact).
 *
 * Layout: one "batch frame" holds every member's packed input frame, member
 * i at word offset frame_off[i] (16-byte aligned), frame_words words in all;
 * one "batch mask record" holds every member's active mask, member i at word
 * offset mask_off[i], mask_words words in all (sp_batch_offsets). */
typedef struct sp_batch sp_batch;

typedef struct {
  uint32_t members;
  uint32_t ctas;          /* CTAs of one batch step launch */
  uint64_t frame_words;   /* words of one batch frame */
  uint64_t mask_words;    /* words of one batch mask record */
  uint64_t frames;        /* batch frames computed so far */
} sp_batch_info;

/* Group n distinct handles (none already batched, all on one device) into a
 * batch.  Pending learning of each member is applied first.  The handles
 * stay owned by the caller and must outlive the batch.  SP_EINVAL for a bad
 * member list, SP_EBUSY if a member is already batched. */
SP_API sp_status sp_batch_create(sp_handle* const* members, uint32_t n, sp_batch** out);

/* Wait (bounded) for the batch's work and release the members.  NULL-safe. */
SP_API void sp_batch_destroy(sp_batch* b);

SP_API sp_status sp_batch_get_info(const sp_batch* b, sp_batch_info* out);

/* Autotune the batch pass's schedule and CTA shapes on the caller's frames:
 * run n_frames learning frames from d_frames (device batch frames laid out
 * as for sp_batch_compute_device, stride in words) three times per candidate
 * and keep the fastest, in three steps:
 *   1. one CTA split for every member: each member's default, or 4 warps x
 *      {2, 4, 8, 16} columns per warp;
 *   2. the compiled schedule of the persistent pass (resident CTAs per SM,
 *      which sets each thread's register budget, x columns per warp in
 *      flight; sp_batch_schedule reports the choice);
 *   3. when the members fall in several buckets (synapses per column <= 32,
 *      <= 128 or more x input of at most 4096 bits or more), the split of
 *      each bucket, largest bucket first, the others as chosen so far.
 * A candidate replaces the best so far only if more than 3 % faster.  The
 * state learning writes (permanences, the derived window and compact forms)
 * and the duty cycles are copied aside on the device first and put back
 * after (a temporary allocation of that size); if it cannot be had, or
 * n_frames == 1 (which tunes the splits of single-frame launches only), the
 * frames are timed as inference.  So the members' permanences, learning and
 * duty cycles are left as they were; their last-frame overlaps and active
 * columns are those of the last tuning frame.  *cols_per_warp (nullable)
 * receives the columns per warp chosen when every member has the same (0:
 * the defaults), else SP_MIXED_SPLIT.  Tuning is a property of the workload
 * and the device (Section 4.4's sweeps show the cost moving with columns and
 * synapses), so call it once after sp_batch_create.  SP_EBUSY if learning is
 * pending (tune before the first learning frame); blocks until done (bounded
 * waits). */
#define SP_MIXED_SPLIT 0xFFFFFFFFu
SP_API sp_status sp_batch_autotune(sp_batch* b, const uint32_t* d_frames, uint32_t n_frames,
                                   uint64_t stride, uint32_t* cols_per_warp);

/* The batch's schedule as set by sp_batch_autotune (before tuning: the
 * default): resident CTAs per SM and columns per warp in flight of the
 * persistent pass, and each member's columns per warp (an array of
 * `members` entries, 0 for the member's default).  Any output may be NULL.
 * Tuning machinery: the paper has no counterpart. */
SP_API sp_status sp_batch_schedule(const sp_batch* b, uint32_t* ctas_per_sm,
                                   uint32_t* cols_in_flight, uint32_t* member_cols_per_warp);

/* The compiled schedules of the persistent pass (needs no device): *count
 * (nullable) receives how many; ctas_per_sm[i] and cols_in_flight[i]
 * (either nullable, room for cap entries, else SP_EINVAL) receive each.
 * Entry 0 is the default.  Tuning machinery: the paper has no counterpart. */
SP_API sp_status sp_batch_schedule_list(uint32_t* ctas_per_sm, uint32_t* cols_in_flight,
                                        uint32_t cap, uint32_t* count);

/* Set the batch's schedule without tuning (for instance one that
 * sp_batch_autotune chose earlier on the same workload): the compiled
 * schedule of ctas_per_sm x cols_in_flight (SP_ENOTSUP if none is
 * compiled) and each member's columns per warp (array of `members` entries,
 * 0 or NULL: the defaults; at most 64, else SP_EINVAL).  SP_EBUSY if
 * learning is pending; blocks until the batch is idle.  Results do not
 * depend on the schedule.  Tuning machinery: the paper has no counterpart. */
SP_API sp_status sp_batch_set_schedule(sp_batch* b, uint32_t ctas_per_sm, uint32_t cols_in_flight,
                                       const uint32_t* member_cols_per_warp);

/* Per-member word offsets inside a batch frame and a batch mask record
 * (arrays of `members` entries; either may be NULL). */
SP_API sp_status sp_batch_offsets(const sp_batch* b, uint64_t* frame_off, uint64_t* mask_off);

/* n_frames batch frames on the device, batch frame t at
 * d_frames + t * frame_stride_words (stride >= frame_words, d_frames 16-byte
 * aligned); every member computes its frames in order with the same learn
 * flag, one launch per batch frame (recorded as a CUDA graph for repeated
 * calls).  If d_masks is not NULL, batch frame t's mask record goes to
 * d_masks + t * mask_stride_words (stride >= mask_words).  Asynchronous on
 * `stream` (NULL = the batch's own stream, cudaStreamLegacy = the legacy
 * default stream). */
SP_API sp_status sp_batch_compute_device(sp_batch* b, const uint32_t* d_frames, uint32_t n_frames,
                                         uint64_t frame_stride_words, int learn, uint32_t* d_masks,
                                         uint64_t mask_stride_words, void* stream);

/* Batch overlap records: one record holds every member's boosted overlaps of
 * one batch frame (Alg. 1, Section 1.1), member i's C_i floats at
 * ov_off[i] (the sum of the earlier members' column counts); *ov_words
 * receives the record's length.  Either pointer may be NULL. */
SP_API sp_status sp_batch_overlap_offsets(const sp_batch* b, uint64_t* ov_off, uint64_t* ov_words);

/* sp_batch_compute_device that also writes batch frame t's overlap record to
 * d_overlaps + t * ov_stride floats (ov_stride >= the record length;
 * device, 4-byte aligned, caller-owned); NULL records nothing.  Execution and
 * results are otherwise those of sp_batch_compute_device.  SP_EINVAL for a
 * short stride or a misaligned pointer. */
SP_API sp_status sp_batch_compute_overlaps_device(sp_batch* b, const uint32_t* d_frames,
                                                  uint32_t n_frames, uint64_t frame_stride_words,
                                                  int learn, uint32_t* d_masks,
                                                  uint64_t mask_stride_words, float* d_overlaps,
                                                  uint64_t ov_stride, void* stream);

/* The form each member's state takes in batch launches (one entry per
 * member, in member order):
 *   SP_FORM_FULL     the SP's own pools and permanences, 8 bytes a synapse;
 *   SP_FORM_COMPACT  16-bit pool offsets and one connected bit a synapse
 *                    (S a multiple of 32 up to 256, pools spanning at most
 *                    65536 inputs);
 *   SP_FORM_WINDOW   per column the origin of a 64 x 64 box of the frame
 *                    holding its pool and a 512-byte bitmap of its connected
 *                    synapses there (frames 32k pixels wide, large pools).
 * The permanences stay authoritative in every form; learning rewrites the
 * derived form of the columns it changes. */
enum { SP_FORM_FULL = 0, SP_FORM_COMPACT = 1, SP_FORM_WINDOW = 2 };
SP_API sp_status sp_batch_forms(const sp_batch* b, uint32_t* forms);

/* The same from host memory: batch frames copied in (pinned memory gives
 * overlapped copies), mask records copied back to h_masks (NULL = not
 * returned).  Synchronous: returns when the masks are in host memory. */
SP_API sp_status sp_batch_compute(sp_batch* b, const uint32_t* h_frames, uint32_t n_frames,
                                  uint64_t frame_stride_words, int learn, uint32_t* h_masks,
                                  uint64_t mask_stride_words);

/* Inference (no learning) over n_frames batch frames.  Members with dense
 * pools (every column's pool is its whole input, S = n_in): the overlaps of
 * every such member and frame are one {0,1} matrix product per member on the
 * tensor cores (tcgen05, e4m3 operands, fp32 accumulation; exact), all of
 * them in one launch, then Alg. 2 for every frame of every member in a second
 * launch; the frames are first laid out as operands in one more launch, and
 * a member's connection operand is rebuilt (one launch for all such members)
 * only when its permanences may have changed since it was last built.  The
 * other members run all n_frames in one persistent launch of the batch step
 * (their CTAs only), before the tensor-core launches; such batches need
 * d_frames 16-byte aligned and the stride a multiple of 4 words.  Learning
 * pending from an earlier batch step is applied first.  Results are those of
 * n_frames calls of sp_batch_compute_device with learn = 0.  Frame and mask
 * layout as sp_batch_compute_device. */
SP_API sp_status sp_batch_infer_device(sp_batch* b, const uint32_t* d_frames, uint32_t n_frames,
                                       uint64_t frame_stride_words, uint32_t* d_masks,
                                       uint64_t mask_stride_words, void* stream);

/* sp_batch_infer_device that also writes batch frame t's overlap record (as
 * sp_batch_compute_overlaps_device) to d_overlaps + t * ov_stride: the
 * tensor-core product's boosted overlaps of every member and frame.  NULL
 * records nothing. */
SP_API sp_status sp_batch_infer_overlaps_device(sp_batch* b, const uint32_t* d_frames,
                                                uint32_t n_frames, uint64_t frame_stride_words,
                                                uint32_t* d_masks, uint64_t mask_stride_words,
                                                float* d_overlaps, uint64_t ov_stride,
                                                void* stream);

/* Bound, in nanoseconds of the GPU's global timer, of the one wait inside a
 * persistent batch launch: a CTA item of a member's frame t + 1 waits for
 * that member's frame t, which CTAs already running compute, so the wait
 * ends by itself; if it has not ended within the bound, the launch stops
 * taking work and the next sp_batch_sync (or synchronous call) returns
 * SP_ETIMEOUT.  The members then hold a partially computed run (frames of
 * some members done, others not); the batch's per-launch counters are reset,
 * so later calls run normally.  0 restores the default of 1 s. */
SP_API sp_status sp_batch_set_device_wait_ns(sp_batch* b, uint64_t ns);

/* Wait (bounded) until the batch's enqueued work has finished. */
SP_API sp_status sp_batch_sync(sp_batch* b);

/* ---- Serving many video streams (continuous batching) ---------------------
 *
 * The paper feeds a system frame by frame (Section 2) and runs one SP per
 * class or video (Section 3); a server does the same for many live streams.
 * Each stream owns an SP kept on the device (pools, permanences, boosts,
 * duty cycles) and submits frames as they arrive.  A worker thread inside
 * the library forms a launch from every stream that has a frame waiting and
 * no frame on the GPU -- streams that arrive while others are being computed
 * join the next launch -- with up to two launches in flight on separate
 * CUDA streams.  Frames of one stream are computed in submission order; each
 * result is bit-identical to computing the stream alone with sp_compute.
 * Streams are admitted against a device-memory budget (SP_EBUSY when full). */
typedef struct sp_server sp_server;

typedef struct {
  uint32_t abi_version;          /* SP_ABI_VERSION */
  uint32_t max_streams;          /* open streams at once, 1..4096 */
  uint32_t queue_depth;          /* frames one stream may have waiting or in flight, 1..64 */
  uint32_t max_input_words;      /* largest frame of any stream, in 32-bit words */
  uint64_t device_budget_bytes;  /* device memory the open streams may hold in total */
  uint32_t max_active;           /* room for one frame's active list; every stream's
                                    upper bound (k, or C for local inhibition) must fit */
  uint32_t reserved;             /* 0 */
} sp_server_config;

typedef struct {
  uint64_t request_id;     /* from sp_server_submit */
  uint64_t frame_seq;      /* frame number within its stream, from 0 */
  uint32_t stream_id;
  uint32_t n_active;       /* active columns of the frame */
  uint32_t active_offset;  /* their ascending list starts here in the poll's buffer */
  sp_status status;        /* SP_OK, or the failure of its launch */
  double latency_us;       /* submit -> result available on the host */
} sp_server_result;

typedef struct {
  uint64_t submitted, completed, launches, frames_in_launches;
  uint64_t device_bytes_used;
  uint32_t open_streams;
  uint32_t reserved;
  double p50_us, p99_us;   /* latency percentiles over the results since the last reset */
} sp_server_stats;

/* Create a server on the current device (starts its worker thread). */
SP_API sp_status sp_server_create(const sp_server_config* cfg, sp_server** out);

/* Stop the worker after the work in flight (bounded wait), free every stream. */
SP_API void sp_server_destroy(sp_server* s);

/* Open a stream with an SP drawn from cfg (as sp_create) or from caller state
 * (as sp_create_from_state).  SP_EBUSY if no slot is free or the stream would
 * exceed the device-memory budget (nothing is allocated then). */
SP_API sp_status sp_server_open_stream(sp_server* s, const sp_config* cfg, uint32_t* stream_id);
SP_API sp_status sp_server_open_stream_from_state(sp_server* s, const sp_config* cfg,
                                                  const uint32_t* idx, const float* perm,
                                                  const float* boost, uint32_t* stream_id);

/* Close an idle stream (SP_EBUSY while it has frames waiting or in flight)
 * and release its memory. */
SP_API sp_status sp_server_close_stream(sp_server* s, uint32_t stream_id);

/* Queue one frame (host memory, the stream's input_words words, copied before
 * return) with its learn flag.  SP_EBUSY if the stream's queue is full. */
SP_API sp_status sp_server_submit(sp_server* s, uint32_t stream_id, const uint32_t* frame_bits,
                                  int learn, uint64_t* request_id);

/* Queue frames for several streams in one call (one lock, one wake-up of the
 * worker): entry i is the frame at frames[i] (host, stream ids[i]'s
 * input_words words, copied before return) with learn[i] (NULL = no
 * learning).  statuses[i] receives SP_OK, SP_EBUSY (that stream's queue is
 * full; nothing queued for it), SP_EINVAL (closed stream or NULL frame) or
 * SP_ECUDA; request_ids[i] (nullable array) the request id or 0.  Entries
 * for one stream are queued in order.  Returns SP_EINVAL only for NULL
 * arrays. */
SP_API sp_status sp_server_submit_many(sp_server* s, uint32_t n, const uint32_t* stream_ids,
                                       const uint32_t* const* frames, const int* learn,
                                       uint64_t* request_ids, sp_status* statuses);

/* sp_server_submit_many for frames already on the device (d_frames[i]: the
 * stream's input_words words, 4-byte aligned): each is copied into the
 * stream's queue on `stream` (a cudaStream_t; NULL = legacy default), so
 * work the caller queued earlier on `stream` (say, an encoder producing the
 * frame) is finished first, and the caller may reuse its buffer once
 * `stream` has passed the call.  Statuses as for sp_server_submit_many. */
SP_API sp_status sp_server_submit_many_device(sp_server* s, uint32_t n, const uint32_t* stream_ids,
                                              const uint32_t* const* d_frames, const int* learn,
                                              uint64_t* request_ids, sp_status* statuses,
                                              void* stream);

/* Take up to max_results finished frames (oldest first), their active lists
 * copied into active[0..active_cap); waits up to wait_ms for the first one.
 * *n_results may be 0.  Results whose lists do not fit stay queued. */
SP_API sp_status sp_server_poll(sp_server* s, sp_server_result* results, uint32_t max_results,
                                uint32_t* active, uint32_t active_cap, uint32_t* n_results,
                                uint32_t wait_ms);

/* Permanences [C][S] of an idle stream (bounded wait for its frames). */
SP_API sp_status sp_server_get_permanences(sp_server* s, uint32_t stream_id, float* out);

/* Counters and latency percentiles; reset != 0 restarts the latency window. */
SP_API sp_status sp_server_get_stats(sp_server* s, sp_server_stats* out, int reset);

/* ---- Frame encoder (Section 2; "Adaptive Video Encoder", Section 3.1) -----
 *
 * Turns colour (or gray) 8-bit frames into the SP's packed binary input on
 * the GPU, so raw frames rather than bits cross the host link:
 *   1. reduction by an integer factor f: the output is floor(src_w / f) x
 *      floor(src_h / f) pixels, each channel the mean of its f x f source
 *      block rounded half up, (sum + f*f/2) / (f*f);
 *   2. grayscale: g = (77 R + 150 G + 29 B + 128) >> 8 (one-channel frames
 *      are their own gray);
 *   3. adaptive Gaussian threshold (the paper uses OpenCV's
 *      ADAPTIVE_THRESH_GAUSSIAN_C; this is its exact integer form): over a
 *      block x block window with binomial weights C(block-1, i) per axis and
 *      edge pixels replicated outside the image, the local mean is the
 *      weighted sum divided by 4^(block-1), rounded half up; the bit of a
 *      pixel is g > mean - offset;
 *   4. packing: output pixel p = y * out_w + x is bit p & 31 of word p >> 5
 *      (LSB first); the unused high bits of the last word are zero.
 * All of it is integer arithmetic, so results are exact.
 *
 * Source frames are [src_h][src_w][channels] bytes, row-major, channels 1 or
 * 3 (R, G, B interleaved). */
typedef struct {
  uint32_t src_w, src_h;  /* source frame size in pixels (1..65535) */
  uint32_t channels;      /* 1 or 3 */
  uint32_t reduce;        /* f, 1..8; the output must be at least 1 x 1 */
  uint32_t block;         /* window size: odd, 3..13 */
  int32_t offset;         /* subtracted from the local mean */
  uint32_t reserved[2];   /* zero */
} sp_encoder_config;

typedef struct {
  uint32_t out_w, out_h;  /* floor(src / reduce) */
  uint64_t out_bits;      /* out_w * out_h: the SP's input_w * input_h */
  uint32_t out_words;     /* ceil(out_bits / 32) words per encoded frame */
  uint64_t src_bytes;     /* src_w * src_h * channels bytes per source frame */
} sp_encoder_info;

typedef struct sp_encoder sp_encoder;

/* Defaults: 960 x 540 RGB, reduce 1, block 11, offset 2. */
SP_API sp_status sp_encoder_config_init(sp_encoder_config* cfg);

/* Validates cfg and creates an encoder on the current device (it owns a
 * stream and, once used, staging buffers).  SP_EINVAL for an invalid cfg. */
SP_API sp_status sp_encoder_create(const sp_encoder_config* cfg, sp_encoder** out);
SP_API void sp_encoder_destroy(sp_encoder* e);  /* NULL-safe; waits for its work */
SP_API sp_status sp_encoder_get_info(const sp_encoder* e, sp_encoder_info* out);

/* Encodes n_frames device frames (frame t at d_src + t * src_stride bytes,
 * src_stride >= src_bytes) into d_bits (frame t at d_bits + t * bits_stride
 * words, bits_stride >= out_words, 4-byte aligned).  Asynchronous on
 * `stream` (a cudaStream_t; NULL = the encoder's own stream, cudaStreamLegacy
 * = the legacy default stream).  SP_EINVAL on NULL or
 * misaligned pointers or short strides (nothing enqueued). */
SP_API sp_status sp_encode_device(sp_encoder* e, const uint8_t* d_src, uint32_t n_frames,
                                  uint64_t src_stride, uint32_t* d_bits, uint64_t bits_stride,
                                  void* stream);

/* Encoder then SP, frame by frame in order, as sp_compute_frames_device
 * would on the encoded bits (learning, masks and the handle's state
 * included): d_active_masks (nullable) receives ceil(C / 32) words per frame.
 * The SP's input must be out_w x out_h bits (SP_EINVAL otherwise).  The
 * encoded bits go through the encoder's own device buffer (up to 32 frames
 * at a time).  Asynchronous on `stream`. */
SP_API sp_status sp_encode_compute_device(sp_encoder* e, sp_handle* h, const uint8_t* d_src,
                                          uint32_t n_frames, uint64_t src_stride, int learn,
                                          uint32_t* d_active_masks, void* stream);

/* The same from host frames (n_frames x src_bytes contiguous; pinned memory
 * lets the copies overlap the kernels): copies in, encoding, SP and the copy
 * out of h_active_masks (nullable; ceil(C / 32) words per frame) are
 * pipelined in chunks; returns after all of it finished (bounded wait). */
SP_API sp_status sp_encode_compute(sp_encoder* e, sp_handle* h, const uint8_t* h_src,
                                   uint32_t n_frames, int learn, uint32_t* h_active_masks);

/* ---- Allocation-free frame (no counterpart in the paper) ------------------
 *
 * sp_step_noalloc runs one frame -- overlap, inhibition and, if learn != 0,
 * learning -- on SP state that the caller keeps in its own device buffers,
 * and allocates nothing: no cudaMalloc, no cudaFree, no pinned or managed
 * memory, no allocating library routine.  It is for callers that cannot
 * allocate device memory at the point where they process a frame: a real-time
 * video pipeline stage whose per-frame callback must not block (cudaMalloc
 * and cudaFree may synchronise the whole device), or a host that runs work
 * against a fixed device-memory budget, or owns every allocation itself, and
 * so cannot let the library grow its footprint.
 *
 * The kernel's scratch (C boosted overlaps and a ticket counter) lives in a
 * static device array of SP_NOALLOC_SCRATCH_BYTES inside the library, which
 * every GPU that loads the library holds until the process exits.  Every call
 * shares that array and it keeps the last call's contents (the counter is
 * cleared at the start of each call), so calls whose work overlaps on a GPU
 * -- different streams, or different threads without ordering -- race and
 * give wrong results: order them, e.g. all on one stream.
 *
 * Every call looks up the array's device address in the current device's
 * context (a lookup that allocates nothing), so a device reset between calls
 * needs no extra step from the caller.  The first call on a device may also
 * load the library's device code into that context; make that first call
 * before any stream capture on that device.
 *
 * Arguments (device pointers on the current device; caller-owned; the call
 * is asynchronous on `stream`, a cudaStream_t, NULL = legacy default):
 *   cfg            scalars of the SP (input_w * input_h bits, num_columns C
 *                  <= SP_NOALLOC_MAX_COLUMNS, synapses_per_column S,
 *                  connect_threshold, perm_inc, perm_dec, min_overlap,
 *                  winners_set_size, inhibition, column grid, local_radius),
 *                  checked as sp_create checks them; pool_mode, rf_*,
 *                  perm_init_*, seed and duty_period are ignored (no duty
 *                  cycles are kept);
 *   d_idx          [C][S] input indices, each < input_w * input_h (not
 *                  checked: out-of-range indices read out of bounds);
 *   d_perm         [C][S] permanences, updated in place when learn != 0;
 *   d_boost        [C] boosts (finite, >= 0);
 *   d_input        ceil(n_in / 32) packed input words (this frame);
 *   d_active_mask  out: ceil(C / 32) words, bit c = column c active;
 *   d_active_list  out: [0] = number of active columns n, [1..n] their
 *                  indices ascending (room for 1 + C words).
 * d_idx and d_perm must be 16-byte aligned when S % 4 == 0, every other
 * pointer 4-byte aligned.
 *
 * Results equal those of sp_compute on a handle holding the same state.
 * Returns SP_EINVAL (nothing enqueued) for a NULL or misaligned pointer, an
 * invalid configuration or C > SP_NOALLOC_MAX_COLUMNS; SP_ECUDA when a launch
 * fails.  sp_last_error() explains. */
#define SP_NOALLOC_MAX_COLUMNS 16384u
#define SP_NOALLOC_SCRATCH_BYTES ((SP_NOALLOC_MAX_COLUMNS + 64u) * 4u)
SP_API sp_status sp_step_noalloc(const sp_config* cfg, const uint32_t* d_idx, float* d_perm,
                                 const float* d_boost, const uint32_t* d_input, int learn,
                                 uint32_t* d_active_mask, uint32_t* d_active_list,
                                 void* stream);

/* Number of kernels this library has launched in the calling process. */
SP_API uint64_t sp_kernel_launch_count(void);

SP_API const char* sp_status_str(sp_status s);

/* Message of the calling thread's last failing call ("" if none). */
SP_API const char* sp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SP_H */
