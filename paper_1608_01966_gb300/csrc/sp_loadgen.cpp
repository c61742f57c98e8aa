// Native load generator for the Spatial Pooler server (include/sp_loadgen.h):
// producer threads submit every stream's frames at Poisson arrival times (or
// keep every queue full), a collector thread takes the results and keeps
// their latencies.
#include "../../include/sp_loadgen.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/sp_synth.h"

namespace sp {
void set_last_error(const char* fmt, ...);
}

namespace {

using Clock = std::chrono::steady_clock;

sp_status lg_fail(sp_status s, const char* msg) {
  sp::set_last_error("sp_loadgen_run: %s", msg);
  return s;
}

struct Shared {
  std::atomic<uint64_t> offered{0}, submitted{0}, refused{0}, failed{0};
  std::atomic<uint32_t> producers_left{0};
  std::atomic<int> status{SP_OK};
};

// Exponential inter-arrival time (seconds) of rate `rate` from a SplitMix64
// stream: u in (0, 1], -ln(u) / rate.
double exp_draw(uint64_t* st, double rate) {
  const uint64_t x = synth_splitmix64(st);
  const double u = (double)((x >> 11) + 1u) * (1.0 / 9007199254740992.0);
  return -std::log(u) / rate;
}

void sleep_until_s(Clock::time_point t0, double t) {
  const auto when = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(t));
  for (;;) {
    const auto now = Clock::now();
    if (now >= when) return;
    const auto left = when - now;
    if (left > std::chrono::microseconds(300))
      std::this_thread::sleep_for(left - std::chrono::microseconds(200));
    else
      std::this_thread::yield();
  }
}

void producer_open(sp_server* s, const sp_loadgen_config* c, uint32_t p, Clock::time_point t0,
                   Shared* sh) {
  std::vector<uint32_t> mine;
  for (uint32_t i = p; i < c->n_streams; i += c->producers) mine.push_back(i);
  const size_t m = mine.size();
  std::vector<uint64_t> rng(m);
  std::vector<double> next(m);
  std::vector<uint64_t> seq(m, 0);
  for (size_t j = 0; j < m; ++j) {
    rng[j] = synth_derive_seed(c->seed, SYNTH_PURPOSE_INSTANCE, mine[j]);
    next[j] = exp_draw(&rng[j], c->rate_per_stream);
  }
  std::vector<uint32_t> ids;
  std::vector<const uint32_t*> frames;
  std::vector<int> learn;
  std::vector<size_t> which;
  std::vector<sp_status> st;
  for (;;) {
    double t_min = 1e300;
    for (size_t j = 0; j < m; ++j) t_min = std::min(t_min, next[j]);
    if (t_min >= c->seconds || sh->status.load() != SP_OK) break;
    sleep_until_s(t0, t_min);
    const double now = std::chrono::duration<double>(Clock::now() - t0).count();
    ids.clear();
    frames.clear();
    learn.clear();
    which.clear();
    for (size_t j = 0; j < m; ++j) {
      while (next[j] <= now && next[j] < c->seconds) {
        // one arrival of stream mine[j]; several due arrivals of a stream
        // are offered in order within the call
        const uint32_t i = mine[j];
        ids.push_back(c->stream_ids[i]);
        frames.push_back(c->pools[i] + (seq[j] % c->pool_frames[i]) * c->pool_stride_words[i]);
        learn.push_back(c->learn ? 1 : 0);
        which.push_back(j);
        ++seq[j];
        next[j] += exp_draw(&rng[j], c->rate_per_stream);
      }
    }
    if (ids.empty()) continue;
    st.assign(ids.size(), SP_OK);
    const sp_status r = sp_server_submit_many(s, (uint32_t)ids.size(), ids.data(), frames.data(),
                                              learn.data(), nullptr, st.data());
    if (r != SP_OK) {
      sh->status.store(r);
      break;
    }
    sh->offered.fetch_add(ids.size());
    for (sp_status x : st) {
      if (x == SP_OK)
        sh->submitted.fetch_add(1);
      else if (x == SP_EBUSY)
        sh->refused.fetch_add(1);
      else
        sh->failed.fetch_add(1);
    }
  }
  sh->producers_left.fetch_sub(1);
}

void producer_closed(sp_server* s, const sp_loadgen_config* c, uint32_t p, Clock::time_point t0,
                     Shared* sh) {
  std::vector<uint32_t> mine;
  for (uint32_t i = p; i < c->n_streams; i += c->producers) mine.push_back(i);
  const size_t m = mine.size();
  std::vector<uint64_t> seq(m, 0);
  std::vector<uint32_t> ids(m);
  std::vector<const uint32_t*> frames(m);
  std::vector<int> learn(m, c->learn ? 1 : 0);
  std::vector<sp_status> st(m);
  for (size_t j = 0; j < m; ++j) ids[j] = c->stream_ids[mine[j]];
  while (m && sh->status.load() == SP_OK &&
         std::chrono::duration<double>(Clock::now() - t0).count() < c->seconds) {
    for (size_t j = 0; j < m; ++j) {
      const uint32_t i = mine[j];
      frames[j] = c->pools[i] + (seq[j] % c->pool_frames[i]) * c->pool_stride_words[i];
    }
    const sp_status r = sp_server_submit_many(s, (uint32_t)m, ids.data(), frames.data(),
                                              learn.data(), nullptr, st.data());
    if (r != SP_OK) {
      sh->status.store(r);
      break;
    }
    uint64_t ok = 0;
    for (size_t j = 0; j < m; ++j) {
      if (st[j] == SP_OK) {
        ++seq[j];
        ++ok;
      } else if (st[j] != SP_EBUSY) {
        sh->failed.fetch_add(1);
      }
    }
    sh->offered.fetch_add(ok);
    sh->submitted.fetch_add(ok);
    if (!ok) std::this_thread::yield();
  }
  sh->producers_left.fetch_sub(1);
}

double percentile(const std::vector<double>& v, double q) {
  if (v.empty()) return 0.0;
  const size_t i = std::min(v.size() - 1, (size_t)std::floor(q * (double)(v.size() - 1) + 0.5));
  return v[i];
}

}  // namespace

extern "C" {

SP_API sp_status sp_loadgen_run(sp_server* s, const sp_loadgen_config* c, sp_loadgen_report* out) {
  if (!s || !c || !out || !c->stream_ids || !c->pools || !c->pool_frames ||
      !c->pool_stride_words)
    return lg_fail(SP_EINVAL, "NULL argument");
  if (c->n_streams == 0 || c->producers == 0 || c->producers > 64 || !(c->seconds > 0.0) ||
      !(c->rate_per_stream >= 0.0) || std::isinf(c->rate_per_stream) || std::isinf(c->seconds))
    return lg_fail(SP_EINVAL, "invalid streams, producers, seconds or rate");
  for (uint32_t i = 0; i < c->n_streams; ++i)
    if (!c->pools[i] || c->pool_frames[i] == 0)
      return lg_fail(SP_EINVAL, "a stream without frames");
  std::memset(out, 0, sizeof(*out));
  sp_server_stats st0{};
  sp_status r = sp_server_get_stats(s, &st0, 1);
  if (r != SP_OK) return r;
  Shared sh;
  sh.producers_left.store(c->producers);
  std::vector<double> lat;
  lat.reserve(1u << 16);
  uint64_t completed = 0, errors = 0;
  Clock::time_point t_last;
  const Clock::time_point t0 = Clock::now();
  t_last = t0;
  std::vector<std::thread> prod;
  for (uint32_t p = 0; p < c->producers; ++p)
    prod.emplace_back(c->rate_per_stream > 0.0 ? producer_open : producer_closed, s, c, p, t0,
                      &sh);
  // the collector runs here: results until the producers are done and every
  // accepted frame has come back (bounded)
  std::vector<sp_server_result> res(1024);
  std::vector<uint32_t> act(1u << 18);
  Clock::time_point deadline = Clock::time_point::max();
  for (;;) {
    uint32_t n = 0;
    r = sp_server_poll(s, res.data(), (uint32_t)res.size(), act.data(), (uint32_t)act.size(), &n,
                       2);
    if (r != SP_OK) {
      sh.status.store(r);
      break;
    }
    if (n) t_last = Clock::now();
    for (uint32_t k = 0; k < n; ++k) {
      if (res[k].status == SP_OK) {
        lat.push_back(res[k].latency_us);
        ++completed;
      } else {
        ++errors;
      }
    }
    if (sh.producers_left.load() == 0) {
      if (deadline == Clock::time_point::max()) deadline = Clock::now() + std::chrono::seconds(30);
      if (completed + errors >= sh.submitted.load()) break;
      if (Clock::now() > deadline) {
        sh.status.store(SP_ETIMEOUT);
        break;
      }
    }
  }
  for (auto& t : prod) t.join();
  sp_server_stats st1{};
  sp_server_get_stats(s, &st1, 0);
  std::sort(lat.begin(), lat.end());
  out->offered = sh.offered.load();
  out->submitted = sh.submitted.load();
  out->refused = sh.refused.load();
  out->completed = completed;
  out->errors = errors + sh.failed.load();
  out->launches = st1.launches - st0.launches;
  out->seconds = std::chrono::duration<double>(t_last - t0).count();
  out->offered_per_s = (double)out->offered / c->seconds;
  out->frames_per_s = out->seconds > 0.0 ? (double)completed / out->seconds : 0.0;
  out->p50_us = percentile(lat, 0.50);
  out->p90_us = percentile(lat, 0.90);
  out->p99_us = percentile(lat, 0.99);
  out->p999_us = percentile(lat, 0.999);
  out->max_us = lat.empty() ? 0.0 : lat.back();
  out->frames_per_launch =
      out->launches ? (double)(st1.frames_in_launches - st0.frames_in_launches) / out->launches
                    : 0.0;
  const int stv = sh.status.load();
  if (stv != SP_OK) return lg_fail((sp_status)stv, "the server failed or results did not complete");
  return SP_OK;
}

}  // extern "C"
