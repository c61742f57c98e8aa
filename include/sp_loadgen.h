/*
 * sp_loadgen.h — native load generator for the Spatial Pooler server
 * (part of libsp_gb300.so).
 *
 * The paper feeds its system frame by frame from video (Section 2,
 * "Processing flow") and runs one SP per video or class (Section 3, "Outer
 * Structure").  A server of many live streams (sp_server_*) is measured by
 * driving it the way cameras would: every stream delivers frames as a
 * Poisson process at a given rate, and each frame is submitted when it
 * arrives.  Doing that from an interpreted language caps the offered load
 * at the interpreter's speed, so this generator runs the producers and the
 * result collector as native threads.
 *
 * Open loop (rate_per_stream > 0): stream i's inter-arrival times are
 * exponential with mean 1 / rate_per_stream, drawn from SplitMix64 seeded
 * by (seed, i); a frame that arrives while its stream's queue is full is
 * refused and counted (a live camera's frame is dropped, not delayed).
 * Closed loop (rate_per_stream == 0): every stream's queue is kept full --
 * the server's saturation throughput.  Frames cycle through each stream's
 * pool.  Latency is the server's own (submit -> result on the host, see
 * sp_server_result.latency_us), collected for every completed frame.
 *
 * The streams must be open on the server, idle, with pools of their own
 * input size; the call returns after `seconds` of offered load and the
 * completion (bounded wait) of every frame submitted.  Statuses: SP_EINVAL
 * for invalid arguments, SP_ETIMEOUT if submitted frames did not complete
 * within 30 s after the load stopped, SP_ECUDA / other server failures as
 * reported by the server.
 */
#ifndef SP_LOADGEN_H
#define SP_LOADGEN_H

#include <stdint.h>

#include "sp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint32_t n_streams;
  const uint32_t* stream_ids;        /* [n_streams] open, idle streams */
  const uint32_t* const* pools;      /* [n_streams] host frame pools (caller-owned) */
  const uint32_t* pool_frames;       /* [n_streams] frames in each pool (>= 1) */
  const uint64_t* pool_stride_words; /* [n_streams] words between frames of a pool */
  double rate_per_stream;            /* frames per second per stream; 0 = closed loop */
  double seconds;                    /* duration of the offered load (> 0) */
  uint32_t producers;                /* producer threads, 1..64 */
  uint32_t learn;                    /* learn flag of every frame */
  uint64_t seed;
} sp_loadgen_config;

typedef struct {
  uint64_t offered;      /* frames that arrived (open loop) or were offered */
  uint64_t submitted;    /* frames the server accepted */
  uint64_t refused;      /* arrivals refused because the stream's queue was full */
  uint64_t completed;    /* results collected */
  uint64_t errors;       /* results with a failing status */
  uint64_t launches;     /* server launches during the run */
  double seconds;        /* first arrival -> last result */
  double offered_per_s;  /* offered / seconds of load */
  double frames_per_s;   /* completed / seconds */
  double p50_us, p90_us, p99_us, p999_us, max_us;  /* latency of completed frames */
  double frames_per_launch;
} sp_loadgen_report;

SP_API sp_status sp_loadgen_run(sp_server* s, const sp_loadgen_config* cfg,
                                sp_loadgen_report* out);

#ifdef __cplusplus
}
#endif

#endif /* SP_LOADGEN_H */
