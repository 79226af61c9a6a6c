// Amplitude server: a request loop over resident plans (Sec. 2: many
// amplitudes per run; here queries arrive over time).
//
// Plans stay bound to their workspaces (tables and constants resident); each
// admitted query gets its own scratch part carved from the caller's arena and
// its own stream, so queries that arrive while others run are admitted as
// soon as a slot and enough arena are free, and their launches overlap on the
// device. A worker thread admits queued queries (first fit, in arrival order)
// and retires finished ones; results wait in pinned host memory until polled.
//
// A query runs in chunks of its slice range (about chunk_ms of estimated
// work each; Sec. 1's subtasks are independent, so any cut is exact). When a
// chunk ends while queries wait for a slot, the running query yields: it
// keeps its scratch part (its partial sums and group state) and resumes, on
// whichever slot frees up next, after the waiting queries have been started.
// So a query of thousands of slices does not hold a slot while small queries
// queue behind it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "plan.h"

namespace {

using Clock = std::chrono::steady_clock;

enum QState { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2, Q_FAILED = 3, Q_PAUSED = 4 };

struct Query {
  uint64_t ticket = 0;
  tz_plan *plan = nullptr;
  std::vector<uint8_t> bits;
  int64_t n = 0;
  std::vector<double> out;
  int state = Q_QUEUED;
  int slot = -1;
  int64_t arena_off = -1;
  size_t bytes = 0;
  int err = TZ_OK;
  std::string msg;
  Clock::time_point t_submit, t_done;
  int64_t lo = 0, hi = 0;   // the plan's slice range at submission
  int64_t next = 0;         // first slice not yet launched
  int64_t chunk = 1;        // slices per chunk
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  uint8_t *pin_in = nullptr;
  double *pin_out = nullptr;
  size_t cap_in = 0, cap_out = 0;
  uint64_t ticket = 0;  // query running here, 0 = free
  bool last = false;    // the work in flight ends the query (its copy-out included)
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct tz_server {
  tz_server_opts opts{};
  std::vector<Slot> slots;
  std::map<uint64_t, Query> queries;
  std::deque<uint64_t> queue;
  std::deque<uint64_t> paused;  // started queries waiting for a slot
  std::vector<std::pair<int64_t, int64_t>> used;  // arena intervals (offset, size)
  size_t in_use = 0;
  uint64_t next_ticket = 1;
  std::vector<double> latencies;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::thread worker;
  std::string fatal;

  // first fit in the arena; -1 if no room
  int64_t arena_alloc(size_t bytes) {
    if (in_use + bytes > opts.hbm_budget) return -1;
    std::sort(used.begin(), used.end());
    int64_t cur = 0;
    for (auto &u : used) {
      if (u.first - cur >= (int64_t)bytes) break;
      cur = std::max(cur, u.first + u.second);
    }
    if (cur + (int64_t)bytes > (int64_t)opts.arena_bytes) return -1;
    used.push_back({cur, (int64_t)bytes});
    in_use += bytes;
    return cur;
  }
  void arena_free(int64_t off) {
    for (size_t i = 0; i < used.size(); i++)
      if (used[i].first == off) {
        in_use -= (size_t)used[i].second;
        used.erase(used.begin() + i);
        return;
      }
  }

  void ensure_pinned(Slot &sl, size_t in, size_t out) {
    if (sl.cap_in < in) {
      if (sl.pin_in) cudaFreeHost(sl.pin_in);
      tz::cuda_check(cudaMallocHost(&sl.pin_in, in), "pinned staging");
      sl.cap_in = in;
    }
    if (sl.cap_out < out) {
      if (sl.pin_out) cudaFreeHost(sl.pin_out);
      tz::cuda_check(cudaMallocHost(reinterpret_cast<void **>(&sl.pin_out), out), "pinned staging");
      sl.cap_out = out;
    }
  }

  // Launch the next chunk of query q on slot s (called with the lock held):
  // the first chunk also copies the bitstrings in and clears the partial
  // sums; the last one also copies the amplitudes and the error word out.
  void launch_chunk(Query &q, int s) {
    Slot &sl = slots[s];
    tz_plan *p = q.plan;
    const int nq = p->net.n_qubits;
    char *scratch = static_cast<char *>(opts.arena) + q.arena_off;
    tz::RunCtx ctx{scratch, sl.stream};
    const bool first = q.next == q.lo;
    const size_t n_out = (size_t)q.n << p->net.n_open;  // amplitudes of the query
    if (first) {
      ensure_pinned(sl, (size_t)q.n * nq, n_out * 16 + 16);
      std::memcpy(sl.pin_in, q.bits.data(), (size_t)q.n * nq);
      tz::cuda_check(cudaMemcpyAsync(scratch + p->s_bits, sl.pin_in, (size_t)q.n * nq, cudaMemcpyHostToDevice,
                                     sl.stream),
                     "query bitstrings in");
    }
    const int64_t lo = q.next, hi = std::min(q.hi, q.next + q.chunk);
    tz::plan_run(p, ctx, q.n, lo, hi, first);
    q.next = hi;
    sl.last = hi == q.hi;
    if (sl.last) {
      // pinned out: the amplitudes, then the scratch part's error word
      ensure_pinned(sl, (size_t)q.n * nq, n_out * 16 + 16);
      tz::cuda_check(cudaMemcpyAsync(sl.pin_out, scratch + p->s_acc, n_out * 16, cudaMemcpyDeviceToHost,
                                     sl.stream),
                     "query amplitudes out");
      const auto *gs = reinterpret_cast<const tz::dev::GroupState *>(scratch + p->s_gs);
      tz::cuda_check(cudaMemcpyAsync(sl.pin_out + 2 * n_out, &gs->tc_error, sizeof(int), cudaMemcpyDeviceToHost,
                                     sl.stream),
                     "query error word out");
    }
    tz::cuda_check(cudaEventRecord(sl.done, sl.stream), "query event");
    sl.ticket = q.ticket;
    q.slot = s;
    q.state = Q_RUNNING;
  }

  int free_slot() const {
    for (size_t s = 0; s < slots.size(); s++)
      if (!slots[s].ticket) return (int)s;
    return -1;
  }

  void fail_query(Query &q, int code, const std::string &m) {
    q.state = Q_FAILED;
    q.err = code;
    q.msg = m;
    q.t_done = Clock::now();
    latencies.push_back(std::chrono::duration<double>(q.t_done - q.t_submit).count());
    if (q.arena_off >= 0) arena_free(q.arena_off);
    q.arena_off = -1;
  }

  void step() {  // one pass of retire + continue/yield + admit, lock held
    for (size_t s = 0; s < slots.size(); s++) {
      Slot &sl = slots[s];
      if (!sl.ticket) continue;
      cudaError_t e = cudaEventQuery(sl.done);
      if (e == cudaErrorNotReady) continue;
      Query &q = queries[sl.ticket];
      sl.ticket = 0;
      if (e != cudaSuccess) {
        fail_query(q, TZ_ECUDA, cudaGetErrorString(e));
        continue;
      }
      if (!sl.last) {
        // more slices: yield the slot to a waiting query, else go on here
        if (!queue.empty()) {
          q.state = Q_PAUSED;
          q.slot = -1;
          paused.push_back(q.ticket);
        } else {
          try {
            launch_chunk(q, (int)s);
          } catch (const tz::Error &err) {
            fail_query(q, err.code, err.what());
          }
        }
        continue;
      }
      int tc_error = 0;
      const size_t n_out = (size_t)q.n << q.plan->net.n_open;
      std::memcpy(&tc_error, sl.pin_out + 2 * n_out, sizeof(int));
      if (tc_error) {
        fail_query(q, TZ_ETIMEOUT, "a bounded wait (tensor-core product or direct-step queue) of this query ran out");
        continue;
      }
      q.out.assign(sl.pin_out, sl.pin_out + 2 * n_out);
      q.state = Q_DONE;
      q.t_done = Clock::now();
      latencies.push_back(std::chrono::duration<double>(q.t_done - q.t_submit).count());
      arena_free(q.arena_off);
      q.arena_off = -1;
    }
    // new queries first (first fit in arrival order), then paused ones
    for (auto it = queue.begin(); it != queue.end();) {
      const int fs = free_slot();
      if (fs < 0) break;
      Query &q = queries[*it];
      int64_t off = arena_alloc(q.bytes);
      if (off < 0) {
        ++it;  // does not fit yet: later, smaller queries may
        continue;
      }
      q.arena_off = off;
      try {
        launch_chunk(q, fs);
      } catch (const tz::Error &e) {
        fail_query(q, e.code, e.what());
      }
      it = queue.erase(it);
    }
    while (!paused.empty()) {
      const int fs = free_slot();
      if (fs < 0) break;
      Query &q = queries[paused.front()];
      paused.pop_front();
      try {
        launch_chunk(q, fs);
      } catch (const tz::Error &e) {
        fail_query(q, e.code, e.what());
      }
    }
  }

  void loop() {
    cudaSetDevice(opts.device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
      step();
      bool busy = !queue.empty() || !paused.empty();
      for (auto &sl : slots) busy |= sl.ticket != 0;
      cv.wait_for(lk, busy ? std::chrono::microseconds(20) : std::chrono::milliseconds(2));
    }
  }
};

#define SRV_TRY try {
#define SRV_CATCH                                \
  }                                              \
  catch (const tz::Error &e) {                   \
    tz_set_error_message(e.what());              \
    return e.code;                               \
  }                                              \
  catch (const std::exception &e) {              \
    tz_set_error_message(e.what());              \
    return TZ_EINVAL;                            \
  }                                              \
  return TZ_OK;

void tz_set_error_message(const std::string &m);  // api.cpp

extern "C" {

int tz_server_create(const tz_server_opts *o, tz_server **out) {
  SRV_TRY
  if (!o || !out) tz::fail(TZ_EINVAL, "NULL argument");
  *out = nullptr;
  if (o->max_inflight < 1 || o->max_inflight > 32) tz::fail(TZ_EINVAL, "max_inflight must be in 1..32");
  if (!o->arena || o->arena_bytes == 0) tz::fail(TZ_EINVAL, "server needs a device arena");
  if ((reinterpret_cast<uintptr_t>(o->arena) & 255) != 0) tz::fail(TZ_EINVAL, "arena must be 256-byte aligned");
  auto srv = std::make_unique<tz_server>();
  srv->opts = *o;
  if (srv->opts.hbm_budget == 0 || srv->opts.hbm_budget > o->arena_bytes) srv->opts.hbm_budget = o->arena_bytes;
  tz::cuda_check(cudaSetDevice(o->device), "cudaSetDevice");
  srv->slots.resize(o->max_inflight);
  for (auto &sl : srv->slots) {
    tz::cuda_check(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking), "server stream");
    tz::cuda_check(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming), "server event");
  }
  tz_server *raw = srv.get();
  srv->worker = std::thread([raw] { raw->loop(); });
  *out = srv.release();
  SRV_CATCH
}

int tz_server_submit(tz_server *srv, tz_plan *plan, const uint8_t *bitstrings, int64_t n, uint64_t *ticket) {
  SRV_TRY
  if (!srv || !plan || !bitstrings || !ticket) tz::fail(TZ_EINVAL, "NULL argument");
  if (!plan->bound) tz::fail(TZ_EINVAL, "plan has no workspace bound");
  if (plan->opts.device != srv->opts.device) tz::fail(TZ_EINVAL, "plan and server are on different devices");
  if (n < 1 || n > plan->max_rows) tz::fail(TZ_EINVAL, "bitstring count outside 1..max_bitstrings of the plan");
  const int nq = plan->net.n_qubits;
  for (int64_t i = 0; i < n * nq; i++)
    if (bitstrings[i] > 1) tz::fail(TZ_EINVAL, "bitstring bytes must be 0 or 1");
  const size_t bytes = align256(plan->scratch_bytes);
  std::lock_guard<std::mutex> lk(srv->mu);
  if (bytes > srv->opts.hbm_budget)
    tz::fail(TZ_EHBM_ADMIT, "query scratch (" + std::to_string(bytes) + " B) exceeds the server budget");
  if (!srv->opts.wait_admit) {
    // admit now or refuse
    bool slot_free = false;
    for (auto &sl : srv->slots) slot_free |= sl.ticket == 0;
    if (!slot_free || srv->in_use + bytes > srv->opts.hbm_budget || !srv->queue.empty())
      tz::fail(TZ_EHBM_ADMIT, "query does not fit now (slots or budget in use)");
  }
  Query q;
  q.ticket = srv->next_ticket++;
  q.plan = plan;
  q.bits.assign(bitstrings, bitstrings + n * nq);
  q.n = n;
  q.lo = q.next = plan->lo;
  q.hi = plan->hi;
  // slices per chunk: about chunk_ms of work by the plan's own estimate
  // (useful flops at a modest rate plus a few microseconds per launch, for
  // every bitstring group of the query)
  {
    const tz_plan_stats &st = plan->stats;
    const double groups = (double)((n + (int64_t(1) << plan->net.batch_log2) - 1) >> plan->net.batch_log2);
    const double group_s = st.flops_per_group / 100e12 + st.n_launches_per_group * 4e-6;
    const double chunk_s = (srv->opts.chunk_ms > 0 ? srv->opts.chunk_ms : 4.0) * 1e-3;
    q.chunk = std::max<int64_t>(1, (int64_t)(chunk_s / std::max(group_s * groups, 1e-9)));
  }
  q.bytes = bytes;
  q.t_submit = Clock::now();
  *ticket = q.ticket;
  srv->queries[q.ticket] = std::move(q);
  srv->queue.push_back(*ticket);
  srv->step();
  srv->cv.notify_one();
  SRV_CATCH
}

int tz_server_poll(tz_server *srv, uint64_t ticket, double *out, int *done) {
  SRV_TRY
  if (!srv || !out || !done) tz::fail(TZ_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->step();
  auto it = srv->queries.find(ticket);
  if (it == srv->queries.end()) tz::fail(TZ_EINVAL, "unknown ticket");
  Query &q = it->second;
  *done = 0;
  if (q.state == Q_DONE) {
    std::memcpy(out, q.out.data(), q.out.size() * sizeof(double));
    *done = 1;
    srv->queries.erase(it);
  } else if (q.state == Q_FAILED) {
    int code = q.err;
    std::string m = q.msg;
    srv->queries.erase(it);
    tz::fail(code, "query failed: " + m);
  }
  SRV_CATCH
}

int tz_server_latency(tz_server *srv, double *p50, double *p99, int64_t *n_done) {
  SRV_TRY
  if (!srv || !p50 || !p99 || !n_done) tz::fail(TZ_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  std::vector<double> v = srv->latencies;
  *n_done = (int64_t)v.size();
  *p50 = *p99 = 0;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    *p50 = v[(size_t)(0.50 * (v.size() - 1) + 0.5)];
    *p99 = v[(size_t)(0.99 * (v.size() - 1) + 0.5)];
  }
  SRV_CATCH
}

void tz_server_destroy(tz_server *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv.notify_all();
  if (srv->worker.joinable()) srv->worker.join();
  cudaSetDevice(srv->opts.device);
  for (auto &sl : srv->slots) {
    if (sl.stream) {
      cudaStreamSynchronize(sl.stream);
      cudaStreamDestroy(sl.stream);
    }
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.pin_in) cudaFreeHost(sl.pin_in);
    if (sl.pin_out) cudaFreeHost(sl.pin_out);
  }
  delete srv;
}

}  // extern "C"
