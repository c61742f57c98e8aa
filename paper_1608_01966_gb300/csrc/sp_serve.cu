// Serving many streams with continuous batching (include/sp.h, sp_server_*).
//
// Client threads submit frames: each frame is copied into its stream's pinned
// ring slot and its host-to-device copy is enqueued at once on the server's
// copy stream.  One worker thread forms launches: every open stream with a
// frame waiting and none in flight joins the next launch, which steps that
// subset of SPs with the batch kernel (a per-launch member table gives each
// SP its frame, buffer parity, pending-learning flag and CTA range).  Two
// launch slots, each with its own CUDA stream, let a new launch start while
// the previous one runs.  Results (count + ascending list per SP) come back
// into pinned memory; the worker records each request's latency and hands
// the results to sp_server_poll.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <iterator>
#include <mutex>
#include <thread>
#include <vector>

#include "sp_internal.h"

using namespace sp::rt;
using Clock = std::chrono::steady_clock;

namespace {

constexpr int kLaunchSlots = 2;
constexpr uint32_t kServeColsPerWarp = 4;
constexpr uint32_t kMaxServerStreams = 4096;

struct Request {
  uint64_t id;
  uint64_t seq;
  uint32_t ring;  // ring slot of its frame
  bool learn;
  Clock::time_point t_submit;
  bool copied = true;  // false: its frame could not be copied (failed, never launched)
  bool device = false;  // copied on a caller's stream: the launch waits for its event
};

struct Stream {
  bool open = false;
  sp_handle* h = nullptr;
  uint64_t bytes = 0;          // charged against the budget
  uint32_t* h_ring = nullptr;  // pinned [depth][input_words]
  uint32_t* d_ring = nullptr;  // device mirror
  std::vector<cudaEvent_t> ev_h2d;
  std::deque<Request> queue;   // submitted, not yet launched
  uint32_t outstanding = 0;    // queued + in flight (ring slots in use)
  uint32_t head = 0;           // next ring slot
  uint32_t in_flight = 0;      // launches holding a frame of this stream (at most 2)
  int cur = 0;
  bool pending = false;
  uint64_t next_seq = 0;       // next sequence number to reserve
  uint64_t launch_seq = 0;     // the request that may launch next
  uint32_t n_ctas = 0, max_active = 0, input_words = 0;
  uint32_t stage_bytes = 0;    // shared memory to stage its CTAs' state
  uint32_t win_bytes = 0;      // shared memory of its CTAs in the window form (0: other forms)
};

struct Done {
  sp_server_result r;
  std::vector<uint32_t> active;
};

struct LaunchSlot {
  bool busy = false;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  sp::TickMember* h_table = nullptr;  // pinned [max_streams]
  uint32_t* h_cta = nullptr;          // pinned [max_ctas]
  uint32_t* h_results = nullptr;      // pinned [max_streams][1 + max_active]
  sp::TickMember* d_table = nullptr;
  uint32_t* d_cta = nullptr;
  uint32_t* d_results = nullptr;
  uint32_t* h_err = nullptr;          // mapped host word: a bounded wait expired
  uint32_t* d_err = nullptr;
  cudaEvent_t copies = nullptr;       // host frame copies issued before this launch
  uint64_t launch_no = 0;             // order of the launches (results are delivered in it)
  std::vector<std::pair<uint32_t, Request>> members;  // (slot, request)
};

}  // namespace

struct sp_server {
  sp_server_config cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  std::atomic<bool> stop{false};
  std::vector<Stream> streams;
  sp::BatchDesc* d_desc = nullptr;
  cudaStream_t copy_stream = nullptr;
  LaunchSlot slots[kLaunchSlots];
  uint32_t max_ctas = 0;
  uint32_t rr = 0;  // round-robin start
  uint64_t next_id = 1;
  uint64_t used_bytes = 0;
  std::deque<Done> done;
  std::vector<double> lat_us;
  uint64_t submitted = 0, completed = 0, launches = 0, frames_launched = 0;
};

namespace {

uint64_t estimate_bytes(const sp_config* c, uint32_t depth, uint32_t words) {
  const uint64_t C = c->num_columns, S = c->synapses_per_column;
  const uint64_t n_words = ((uint64_t)c->input_w * c->input_h + 31) / 32;
  const uint64_t mw = (C + 31) / 32;
  uint64_t b = 0;
  for (uint64_t part : {C * S * 4, C * S * 4, C * 4, C * 4, n_words * 8, mw * 8, (C + 1) * 4,
                        (uint64_t)4, (S + 1) * 4, C * 4})
    b += (part + 255) & ~uint64_t(255);
  return b + (uint64_t)depth * words * 4;
}

// Deliver a finished launch: results to the completion queue, streams idle.
void finish_launch(sp_server* s, LaunchSlot& L, sp_status st) {
  const auto now = Clock::now();
  const uint32_t row = 1u + s->cfg.max_active;
  uint32_t pos = 0;
  for (auto& m : L.members) {
    Stream& S = s->streams[m.first];
    Done d;
    d.r.request_id = m.second.id;
    d.r.frame_seq = m.second.seq;
    d.r.stream_id = m.first;
    d.r.status = st;
    d.r.latency_us =
        std::chrono::duration<double, std::micro>(now - m.second.t_submit).count();
    const uint32_t* res = L.h_results + (size_t)pos * row;
    const uint32_t n = st == SP_OK ? std::min(res[0], s->cfg.max_active) : 0u;
    d.r.n_active = n;
    d.active.assign(res + 1, res + 1 + n);
    s->lat_us.push_back(d.r.latency_us);
    s->done.push_back(std::move(d));
    S.in_flight -= 1;
    S.outstanding -= 1;
    ++pos;
    ++s->completed;
  }
  L.members.clear();
  L.busy = false;
}

// Form and enqueue one launch from the waiting streams (caller holds mu).  A
// stream whose previous frame is still in the other slot's launch may take
// part: this launch then waits on the GPU for that one.
sp_status start_launch(sp_server* s, LaunchSlot& L, const LaunchSlot& other) {
  bool chained = false, host_copies = false;
  const uint32_t n = (uint32_t)s->streams.size();
  const uint32_t row = 1u + s->cfg.max_active;
  uint32_t ctas = 0, count = 0;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t i = (s->rr + k) % n;
    Stream& S = s->streams[i];
    // a request whose frame could not be copied fails without a launch
    while (!S.queue.empty() && S.queue.front().seq == S.launch_seq &&
           !S.queue.front().copied) {
      const Request& bad = S.queue.front();
      Done d;
      d.r.request_id = bad.id;
      d.r.frame_seq = bad.seq;
      d.r.stream_id = i;
      d.r.status = SP_ECUDA;
      d.r.latency_us = 0.0;
      s->done.push_back(std::move(d));
      S.queue.pop_front();
      S.launch_seq += 1;
      S.outstanding -= 1;
      ++s->completed;
    }
    // requests launch in sequence order; one still being copied holds back
    // the ones after it
    if (!S.open || S.in_flight >= 2u || S.queue.empty() || S.queue.front().seq != S.launch_seq)
      continue;
    if (ctas + S.n_ctas > s->max_ctas) break;
    Request r = S.queue.front();
    S.queue.pop_front();
    S.launch_seq += 1;
    sp::TickMember& tm = L.h_table[i];
    tm.x = S.d_ring + (size_t)r.ring * S.input_words;
    tm.flags = (S.cur ? sp::kTickCur : 0u) | (S.pending ? sp::kTickPending : 0u) |
               (r.learn ? sp::kTickLearn : 0u) | sp::kTickSave;
    tm.cta_first = ctas;
    tm.out_off = count * row;
    for (uint32_t c = 0; c < S.n_ctas; ++c) L.h_cta[ctas + c] = i;
    ctas += S.n_ctas;
    chained = chained || S.in_flight > 0u;
    S.in_flight += 1;
    S.pending = r.learn;
    if (r.learn) S.h->bimg_stale = true;
    S.cur ^= 1;
    L.members.emplace_back(i, r);
    ++count;
    // the launch waits for this frame's copy: frames copied on a caller's
    // stream one by one, host frames all at once below
    if (r.device)
      SP_CUDA(cudaStreamWaitEvent(L.st, S.ev_h2d[r.ring], 0));
    else
      host_copies = true;
  }
  if (count == 0) return SP_OK;
  if (host_copies) {
    // every published host frame's copy was issued on the copy stream before
    // its request was published
    SP_CUDA(cudaEventRecord(L.copies, s->copy_stream));
    SP_CUDA(cudaStreamWaitEvent(L.st, L.copies, 0));
  }
  if (chained) SP_CUDA(cudaStreamWaitEvent(L.st, other.done, 0));
  s->rr = (s->rr + 1) % n;
  SP_CUDA(cudaMemcpyAsync(L.d_table, L.h_table, sizeof(sp::TickMember) * n,
                          cudaMemcpyHostToDevice, L.st));
  SP_CUDA(cudaMemcpyAsync(L.d_cta, L.h_cta, (size_t)ctas * 4, cudaMemcpyHostToDevice, L.st));
  sp::BatchArgs a{};
  a.desc = s->d_desc;
  a.cta_inst = L.d_cta;
  a.tick = L.d_table;
  a.results_out = L.d_results;
  uint32_t max_C = 1, stage = 0, win = 0;
  for (auto& m : L.members) {
    max_C = std::max(max_C, s->streams[m.first].h->C);
    stage = std::max(stage, s->streams[m.first].stage_bytes);
    win = std::max(win, s->streams[m.first].win_bytes);
  }
  a.stage_cap = batch_stage_cap(stage);
  a.xspan_cap = batch_xspan_cap();
  a.win_cap = win;
  a.err = L.d_err;
  SP_CUDA(sp::launch_batch_step(a, ctas, max_C, L.st));
  SP_CUDA(cudaMemcpyAsync(L.h_results, L.d_results, (size_t)count * row * 4,
                          cudaMemcpyDeviceToHost, L.st));
  SP_CUDA(cudaEventRecord(L.done, L.st));
  L.busy = true;
  L.launch_no = ++s->launches;
  s->frames_launched += count;
  return SP_OK;
}

void worker_main(sp_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  uint32_t idle_spins = 0;
  while (!s->stop.load()) {
    bool progress = false;
    // deliver finished launches oldest first: a stream's frames can be in both
    for (int pass = 0; pass < kLaunchSlots; ++pass) {
      LaunchSlot* oldest = nullptr;
      for (auto& L : s->slots)
        if (L.busy && (!oldest || L.launch_no < oldest->launch_no)) oldest = &L;
      if (!oldest) break;
      const cudaError_t e = cudaEventQuery(oldest->done);
      if (e == cudaErrorNotReady) break;
      sp_status st = e == cudaSuccess ? SP_OK : SP_ECUDA;
      if (st == SP_OK && *reinterpret_cast<volatile uint32_t*>(oldest->h_err)) {
        *oldest->h_err = 0u;
        st = SP_ETIMEOUT;
      }
      finish_launch(s, *oldest, st);
      progress = true;
    }
    if (progress) s->cv_done.notify_all();
    for (int li = 0; li < kLaunchSlots; ++li) {
      LaunchSlot& L = s->slots[li];
      if (L.busy) continue;
      const uint64_t before = s->launches;
      const sp_status st = start_launch(s, L, s->slots[(li + 1) % kLaunchSlots]);
      if (st != SP_OK) {
        // the members of a launch that could not be enqueued fail
        finish_launch(s, L, st);
        s->cv_done.notify_all();
      }
      if (s->launches != before) progress = true;
    }
    const bool in_flight = s->slots[0].busy || s->slots[1].busy;
    if (progress) {
      idle_spins = 0;
      continue;
    }
    if (in_flight) {
      // poll the launches in flight: yield for a few milliseconds (a launch
      // takes tens of microseconds; a sleep would overshoot it), then sleep
      lk.unlock();
      if (++idle_spins < 20000)
        std::this_thread::yield();
      else
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    } else {
      idle_spins = 0;
      s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

sp_status validate_server_config(const sp_server_config* c) {
  if (!c) return fail(SP_EINVAL, "server config is NULL");
  if (c->abi_version != SP_ABI_VERSION) return fail(SP_EINVAL, "abi_version mismatch");
  if (c->max_streams == 0 || c->max_streams > kMaxServerStreams)
    return fail(SP_EINVAL, "max_streams must be in [1, %u]", kMaxServerStreams);
  if (c->queue_depth == 0 || c->queue_depth > 64) return fail(SP_EINVAL, "queue_depth in [1, 64]");
  if (c->max_input_words == 0) return fail(SP_EINVAL, "max_input_words is 0");
  if (c->max_active == 0 || c->max_active > SP_MAX_COLUMNS)
    return fail(SP_EINVAL, "max_active in [1, SP_MAX_COLUMNS]");
  if (c->reserved != 0) return fail(SP_EINVAL, "reserved must be 0");
  return SP_OK;
}

void free_server(sp_server* s) {
  if (!s) return;
  DeviceGuard g(s->device);
  if (s->worker.joinable()) {
    s->stop.store(true);
    s->cv_work.notify_all();
    s->worker.join();
  }
  for (auto& L : s->slots) {
    if (L.st) cudaStreamSynchronize(L.st);
    if (L.done) cudaEventDestroy(L.done);
    if (L.st) cudaStreamDestroy(L.st);
    if (L.h_table) cudaFreeHost(L.h_table);
    if (L.h_cta) cudaFreeHost(L.h_cta);
    if (L.h_results) cudaFreeHost(L.h_results);
    if (L.h_err) cudaFreeHost(L.h_err);
    if (L.copies) cudaEventDestroy(L.copies);
    if (L.d_table) cudaFree(L.d_table);
    if (L.d_cta) cudaFree(L.d_cta);
    if (L.d_results) cudaFree(L.d_results);
  }
  if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
  for (auto& S : s->streams) {
    if (!S.open) continue;
    for (auto e : S.ev_h2d) cudaEventDestroy(e);
    if (S.h_ring) cudaFreeHost(S.h_ring);
    if (S.d_ring) cudaFree(S.d_ring);
    S.h->cur = S.cur;
    S.h->pending = S.pending;
    sp_destroy(S.h);
  }
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->d_desc) cudaFree(s->d_desc);
  delete s;
}

// Admit a created handle into a free slot (caller holds no lock).
sp_status admit(sp_server* s, sp_handle* h, uint32_t* stream_id) {
  sp_info info{};
  sp_get_info(h, &info);
  if (info.input_words > s->cfg.max_input_words) {
    sp_destroy(h);
    return fail(SP_EINVAL, "stream input (%u words) exceeds max_input_words", info.input_words);
  }
  if (info.max_active > s->cfg.max_active) {
    sp_destroy(h);
    return fail(SP_EINVAL, "stream may activate %u columns, server holds %u", info.max_active,
                s->cfg.max_active);
  }
  Stream S;
  S.h = h;
  S.input_words = info.input_words;
  S.max_active = info.max_active;
  sp::BatchDesc d;
  // a launch carries one frame of a few tens of streams: small CTAs (16
  // columns) keep every SM busy and the latency low
  fill_desc(h, &d, kServeColsPerWarp, &S.win_bytes);
  S.n_ctas = d.n_ctas;
  S.stage_bytes = sp::batch_stage_bytes(h->C, h->S, d.n_ctas);
  const size_t ring_bytes = (size_t)s->cfg.queue_depth * info.input_words * 4;
  cudaError_t e = cudaMallocHost(&S.h_ring, ring_bytes);
  if (e == cudaSuccess) e = device_malloc((void**)&S.d_ring, ring_bytes);
  S.ev_h2d.assign(s->cfg.queue_depth, nullptr);
  for (uint32_t i = 0; e == cudaSuccess && i < s->cfg.queue_depth; ++i)
    e = cudaEventCreateWithFlags(&S.ev_h2d[i], cudaEventDisableTiming);
  std::unique_lock<std::mutex> lk(s->mu);
  uint32_t slot = UINT32_MAX;
  for (uint32_t i = 0; i < s->streams.size(); ++i)
    if (!s->streams[i].open) {
      slot = i;
      break;
    }
  S.bytes = info.device_bytes + ring_bytes;
  if (e == cudaSuccess && slot != UINT32_MAX && s->used_bytes + S.bytes <= s->cfg.device_budget_bytes &&
      S.n_ctas <= s->max_ctas)
    e = cudaMemcpyAsync(s->d_desc + slot, &d, sizeof(d), cudaMemcpyHostToDevice, s->copy_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
  if (e != cudaSuccess || slot == UINT32_MAX || s->used_bytes + S.bytes > s->cfg.device_budget_bytes ||
      S.n_ctas > s->max_ctas) {
    lk.unlock();
    for (auto ev : S.ev_h2d)
      if (ev) cudaEventDestroy(ev);
    if (S.h_ring) cudaFreeHost(S.h_ring);
    if (S.d_ring) cudaFree(S.d_ring);
    sp_destroy(h);
    if (e != cudaSuccess) return fail(SP_ECUDA, "stream set-up: %s", cudaGetErrorString(e));
    return fail(SP_EBUSY, "no free slot or the device-memory budget is exhausted");
  }
  S.open = true;
  // the handle's pending learning (none after creation) travels with the stream
  S.cur = h->cur;
  S.pending = h->pending;
  s->used_bytes += S.bytes;
  s->streams[slot] = std::move(S);
  *stream_id = slot;
  return SP_OK;
}

sp_status pre_admit(sp_server* s, const sp_config* cfg) {
  const uint64_t est = estimate_bytes(cfg, s->cfg.queue_depth,
                                      (uint32_t)(((uint64_t)cfg->input_w * cfg->input_h + 31) / 32));
  std::lock_guard<std::mutex> lk(s->mu);
  bool free_slot = false;
  for (auto& S : s->streams) free_slot |= !S.open;
  if (!free_slot) return fail(SP_EBUSY, "all %u stream slots are open", s->cfg.max_streams);
  if (s->used_bytes + est > s->cfg.device_budget_bytes)
    return fail(SP_EBUSY, "device-memory budget exhausted (%llu of %llu bytes used)",
                (unsigned long long)s->used_bytes, (unsigned long long)s->cfg.device_budget_bytes);
  return SP_OK;
}

// Wait (bounded) until a stream has nothing queued or in flight.
sp_status wait_idle(sp_server* s, std::unique_lock<std::mutex>& lk, uint32_t id) {
  const auto deadline = Clock::now() + std::chrono::milliseconds(default_timeout_ms());
  while (s->streams[id].outstanding > 0) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
        s->streams[id].outstanding > 0)
      return fail(SP_ETIMEOUT, "stream %u did not drain", id);
  }
  return SP_OK;
}

}  // namespace

extern "C" {

SP_API sp_status sp_server_create(const sp_server_config* cfg, sp_server** out) {
  if (!out) return fail(SP_EINVAL, "out is NULL");
  *out = nullptr;
  sp_status st = validate_server_config(cfg);
  if (st != SP_OK) return st;
  sp_server* s = new (std::nothrow) sp_server();
  if (!s) return fail(SP_ENOMEM, "host allocation");
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  s->streams.resize(cfg->max_streams);
  s->max_ctas = cfg->max_streams * batch_ctas(SP_MAX_COLUMNS, 128u, kServeColsPerWarp);  // the largest share
  const uint32_t row = 1u + cfg->max_active;
  cudaError_t e = sp::kernels_init();
  if (e == cudaSuccess) e = device_malloc((void**)&s->d_desc, sizeof(sp::BatchDesc) * cfg->max_streams);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  for (auto& L : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&L.h_table, sizeof(sp::TickMember) * cfg->max_streams);
    if (e == cudaSuccess) e = cudaMallocHost(&L.h_cta, (size_t)s->max_ctas * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&L.h_results, (size_t)cfg->max_streams * row * 4);
    if (e == cudaSuccess) e = device_malloc((void**)&L.d_table, sizeof(sp::TickMember) * cfg->max_streams);
    if (e == cudaSuccess) e = device_malloc((void**)&L.d_cta, (size_t)s->max_ctas * 4);
    if (e == cudaSuccess) e = device_malloc((void**)&L.d_results, (size_t)cfg->max_streams * row * 4);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.copies, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&L.h_err, 4, cudaHostAllocMapped);
    if (e == cudaSuccess) {
      *L.h_err = 0u;
      e = cudaHostGetDevicePointer((void**)&L.d_err, L.h_err, 0);
    }
  }
  if (e != cudaSuccess) {
    free_server(s);
    return fail(e == cudaErrorMemoryAllocation ? SP_ENOMEM : SP_ECUDA, "server set-up: %s",
                cudaGetErrorString(e));
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return SP_OK;
}

SP_API void sp_server_destroy(sp_server* s) { free_server(s); }

SP_API sp_status sp_server_open_stream(sp_server* s, const sp_config* cfg, uint32_t* stream_id) {
  if (!s || !cfg || !stream_id) return fail(SP_EINVAL, "NULL argument");
  DeviceGuard g(s->device);
  sp_status st = pre_admit(s, cfg);
  if (st != SP_OK) return st;
  sp_handle* h = nullptr;
  if ((st = sp_create(cfg, &h)) != SP_OK) return st;
  return admit(s, h, stream_id);
}

SP_API sp_status sp_server_open_stream_from_state(sp_server* s, const sp_config* cfg,
                                                  const uint32_t* idx, const float* perm,
                                                  const float* boost, uint32_t* stream_id) {
  if (!s || !cfg || !stream_id) return fail(SP_EINVAL, "NULL argument");
  DeviceGuard g(s->device);
  sp_status st = pre_admit(s, cfg);
  if (st != SP_OK) return st;
  sp_handle* h = nullptr;
  if ((st = sp_create_from_state(cfg, idx, perm, boost, &h)) != SP_OK) return st;
  return admit(s, h, stream_id);
}

SP_API sp_status sp_server_close_stream(sp_server* s, uint32_t id) {
  if (!s) return fail(SP_EINVAL, "NULL server");
  DeviceGuard g(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  if (id >= s->streams.size() || !s->streams[id].open) return fail(SP_EINVAL, "stream %u is not open", id);
  Stream& S = s->streams[id];
  if (S.outstanding > 0) return fail(SP_EBUSY, "stream %u has frames waiting or in flight", id);
  for (auto e : S.ev_h2d) cudaEventDestroy(e);
  cudaFreeHost(S.h_ring);
  cudaFree(S.d_ring);
  S.h->cur = S.cur;
  S.h->pending = S.pending;
  sp_destroy(S.h);
  s->used_bytes -= S.bytes;
  s->streams[id] = Stream();
  return SP_OK;
}

namespace {

// One frame being submitted: its slot and sequence number are reserved under
// the lock, its copies are made without it, and it is published under the
// lock again in sequence order, so the worker never waits for a copy.
struct Pending {
  uint32_t entry, stream, ring;
  uint64_t seq;
  bool learn;
  bool device;
};

void publish(sp_server* s, const std::vector<Pending>& ps, const std::vector<bool>& copied,
             const Clock::time_point t, uint64_t* request_ids) {
  std::unique_lock<std::mutex> lk(s->mu);
  for (size_t k = 0; k < ps.size(); ++k) {
    Stream& S = s->streams[ps[k].stream];
    Request r{s->next_id++, ps[k].seq, ps[k].ring, ps[k].learn, t, copied[k], ps[k].device};
    auto it = S.queue.end();
    while (it != S.queue.begin() && std::prev(it)->seq > r.seq) --it;
    S.queue.insert(it, r);
    ++s->submitted;
    if (request_ids) request_ids[ps[k].entry] = r.id;
  }
}

}  // namespace

SP_API sp_status sp_server_submit(sp_server* s, uint32_t id, const uint32_t* bits, int learn,
                                  uint64_t* request_id) {
  if (!s || !bits) return fail(SP_EINVAL, "NULL argument");
  const int lf = learn != 0 ? 1 : 0;
  sp_status st = SP_OK;
  uint64_t rid = 0;
  const sp_status call = sp_server_submit_many(s, 1, &id, &bits, &lf, &rid, &st);
  if (call != SP_OK) return call;
  if (st == SP_EINVAL) return fail(SP_EINVAL, "stream %u is not open", id);
  if (st == SP_EBUSY) return fail(SP_EBUSY, "stream %u queue is full", id);
  if (st != SP_OK) return fail(st, "copying the frame of stream %u failed", id);
  if (request_id) *request_id = rid;
  return SP_OK;
}

namespace {

// Reserve, copy (host frames through the pinned ring on the copy stream, or
// device frames on the caller's stream), publish.
sp_status submit_impl(sp_server* s, uint32_t n, const uint32_t* ids,
                      const uint32_t* const* frames, const int* learn, uint64_t* request_ids,
                      sp_status* statuses, bool device, cudaStream_t cst) {
  if (!s || (n && (!ids || !frames || !statuses))) return fail(SP_EINVAL, "NULL argument");
  DeviceGuard g(s->device);
  std::vector<Pending> ps;
  ps.reserve(n);
  {
    std::unique_lock<std::mutex> lk(s->mu);
    for (uint32_t i = 0; i < n; ++i) {
      statuses[i] = SP_OK;
      if (request_ids) request_ids[i] = 0;
      const uint32_t id = ids[i];
      if (id >= s->streams.size() || !s->streams[id].open || !frames[i]) {
        statuses[i] = SP_EINVAL;
        continue;
      }
      Stream& S = s->streams[id];
      if (S.outstanding >= s->cfg.queue_depth) {
        statuses[i] = SP_EBUSY;
        continue;
      }
      ps.push_back(Pending{i, id, S.head, S.next_seq++, learn && learn[i] != 0, device});
      S.head = (S.head + 1) % s->cfg.queue_depth;
      S.outstanding += 1;  // the slot stays reserved until its frame is done
    }
  }
  if (ps.empty()) return SP_OK;
  const Clock::time_point t = Clock::now();
  std::vector<bool> copied(ps.size(), true);
  for (size_t k = 0; k < ps.size(); ++k) {
    // the stream cannot close while it has a reserved slot (outstanding > 0)
    Stream& S = s->streams[ps[k].stream];
    uint32_t* dst = S.d_ring + (size_t)ps[k].ring * S.input_words;
    cudaError_t e;
    if (device) {
      e = cudaMemcpyAsync(dst, frames[ps[k].entry], (size_t)S.input_words * 4,
                          cudaMemcpyDeviceToDevice, cst);
      if (e == cudaSuccess) e = cudaEventRecord(S.ev_h2d[ps[k].ring], cst);
    } else {
      uint32_t* hs = S.h_ring + (size_t)ps[k].ring * S.input_words;
      std::memcpy(hs, frames[ps[k].entry], (size_t)S.input_words * 4);
      e = cudaMemcpyAsync(dst, hs, (size_t)S.input_words * 4, cudaMemcpyHostToDevice,
                          s->copy_stream);
    }
    if (e != cudaSuccess) {
      copied[k] = false;
      statuses[ps[k].entry] = SP_ECUDA;
    }
  }
  publish(s, ps, copied, t, request_ids);
  s->cv_work.notify_one();
  return SP_OK;
}

}  // namespace

SP_API sp_status sp_server_submit_many(sp_server* s, uint32_t n, const uint32_t* ids,
                                       const uint32_t* const* frames, const int* learn,
                                       uint64_t* request_ids, sp_status* statuses) {
  return submit_impl(s, n, ids, frames, learn, request_ids, statuses, false, nullptr);
}

SP_API sp_status sp_server_submit_many_device(sp_server* s, uint32_t n, const uint32_t* ids,
                                              const uint32_t* const* d_frames, const int* learn,
                                              uint64_t* request_ids, sp_status* statuses,
                                              void* stream) {
  return submit_impl(s, n, ids, d_frames, learn, request_ids, statuses, true,
                     static_cast<cudaStream_t>(stream));
}

SP_API sp_status sp_server_poll(sp_server* s, sp_server_result* results, uint32_t max_results,
                                uint32_t* active, uint32_t active_cap, uint32_t* n_results,
                                uint32_t wait_ms) {
  if (!s || !n_results || (!results && max_results)) return fail(SP_EINVAL, "NULL argument");
  *n_results = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  uint32_t used = 0, n = 0;
  while (n < max_results && !s->done.empty()) {
    Done& d = s->done.front();
    if (d.r.n_active > 0 && (!active || used + d.r.n_active > active_cap)) break;
    results[n] = d.r;
    results[n].active_offset = used;
    if (d.r.n_active) std::memcpy(active + used, d.active.data(), (size_t)d.r.n_active * 4);
    used += d.r.n_active;
    ++n;
    s->done.pop_front();
  }
  *n_results = n;
  return SP_OK;
}

SP_API sp_status sp_server_get_permanences(sp_server* s, uint32_t id, float* out) {
  if (!s || !out) return fail(SP_EINVAL, "NULL argument");
  DeviceGuard g(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  if (id >= s->streams.size() || !s->streams[id].open) return fail(SP_EINVAL, "stream %u is not open", id);
  sp_status st = wait_idle(s, lk, id);
  if (st != SP_OK) return st;
  Stream& S = s->streams[id];
  S.h->cur = S.cur;
  S.h->pending = S.pending;
  st = sp_get_permanences(S.h, out);  // applies the stream's pending learning
  S.cur = S.h->cur;
  S.pending = S.h->pending;
  return st;
}

SP_API sp_status sp_server_get_stats(sp_server* s, sp_server_stats* out, int reset) {
  if (!s || !out) return fail(SP_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->launches = s->launches;
  out->frames_in_launches = s->frames_launched;
  out->device_bytes_used = s->used_bytes;
  out->open_streams = 0;
  for (auto& S : s->streams) out->open_streams += S.open ? 1u : 0u;
  out->reserved = 0;
  std::vector<double> v = s->lat_us;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) {
    if (v.empty()) return 0.0;
    size_t i = (size_t)(p * (double)(v.size() - 1) + 0.5);
    return v[std::min(i, v.size() - 1)];
  };
  out->p50_us = pct(0.50);
  out->p99_us = pct(0.99);
  if (reset) s->lat_us.clear();
  return SP_OK;
}

}  // extern "C"
