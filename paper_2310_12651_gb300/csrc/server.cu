// Serving engine: many independent mobility products from many host threads on
// one GPU.
//
// The paper computes one system per call. A service sees a stream of requests
// of every size and box; launching each alone leaves the GPU idle between small
// launches and re-plans FFTs for every box. Here:
//
//   * requests with identical parameters (a "grid class": box, grid, kernel
//     widths, cutoff, precision, torques or not) waiting at the same time are
//     stacked into one fcm_batch_apply pass (continuous batching: whatever is
//     queued when a launch slot frees up goes into the next pass);
//   * a class has at most one pass in flight: requests that arrive while their
//     class is on the GPU wait for that pass and join the class's next one (its
//     passes would run one after the other anyway, since they share the cached
//     handle's workspace), while other classes use the remaining slots;
//   * batch handles (workspace, cell lists, cuFFT plans) stay resident in a
//     cache keyed by grid class and capacity bucket, so a class's second pass
//     plans and allocates nothing;
//   * the cache is bounded by an HBM budget: before a new handle is created,
//     idle handles are evicted least recently used first; a request whose
//     handle alone exceeds the budget is rejected (FCM_ERR_OOM);
//   * four launch slots, each with its own stream and pinned staging, so one
//     pass's copies and kernels overlap the next pass's (also across classes);
//   * every wait is bounded (poll timeouts; the worker polls events).
//
// One worker thread owns every CUDA object; submit/poll/cancel/stats only take
// the request table's lock.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/fcm.h"
#include "fcm_internal.cuh"

namespace fcm {
int check_params(const fcm_params* p, std::string* why);
size_t workspace_estimate(const fcm_params& p, int max_systems);
int capture_batch_graph(fcm_handle* h, int bucket, const void* pos, const void* F, const void* T, void* U, void* W,
                        cudaStream_t s, cudaGraphExec_t* out);
int handle_max_n(const fcm_handle* h);
int* handle_sys_off(fcm_handle* h);
}  // namespace fcm

using namespace fcm;
using Clock = std::chrono::steady_clock;

namespace {

int fail(int code, const std::string& msg) { return record_error(code, msg.c_str()); }

size_t pow2_at_least(size_t v, size_t lo) {
  size_t p = lo;
  while (p < v) p <<= 1;
  return p;
}

enum State { kPending = 0, kRunning = 1, kDone = 2 };

struct Request {
  long long id = 0;
  fcm_request r{};
  std::string key;
  bool torque = false;
  size_t rsz = 4;
  int state = kPending;
  int status = FCM_OK;
  Clock::time_point t_submit, t_done;
};

struct Buffer {
  void* p = nullptr;
  size_t bytes = 0;
};

// A cached batch handle with two sets of device staging: pos, F, T (and U, W) occupy max_n rows
// each, so a captured pass sees the same addresses whatever the batch's size. Consecutive passes
// alternate sets, so one pass's copies overlap the previous pass's kernels; the kernels of passes
// on one handle are ordered by `computed` (they share its workspace).
struct CachedHandle {
  std::string key;
  fcm_handle* h = nullptr;
  int max_systems = 0;
  int max_n = 0;
  size_t bytes = 0;                 // handle workspace + staging
  cudaEvent_t computed = nullptr;   // kernels of the last pass enqueued on this handle
  cudaEvent_t set_free[2] = {nullptr, nullptr};   // staging set no longer read or written
  int next_set = 0;
  int in_flight = 0;                // slots whose pass uses it
  unsigned long long last_use = 0;
  bool fp32 = true;
  bool torque = false;
  size_t rsz = 4;
  Buffer d_in[2], d_out[2];
  bool graphs_ok = true;            // cleared if a capture ever fails: direct launches from then on
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;   // (bucket, staging set) -> captured pass
};

// A launch slot: a stream and pinned host staging (pos, F, T, then U, W, each `cap` rows).
struct Slot {
  int index = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Buffer h_in, h_out;                // pinned host staging
  int* h_off = nullptr;              // pinned offsets copied ahead of a pass
  std::vector<std::shared_ptr<Request>> reqs;
  std::vector<int> offsets;
  CachedHandle* ch = nullptr;
  bool busy = false;
  bool torque = false;
  size_t rsz = 4;
  int n = 0;
  size_t cap = 0;
};

constexpr int kSlots = 4;
constexpr size_t kLatencyWindow = 1 << 17;

}  // namespace

struct fcm_server {
  int device = 0;
  size_t budget = 0;
  int max_batch = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  long long next_id = 1;
  std::deque<std::shared_ptr<Request>> pending;
  std::unordered_map<long long, std::shared_ptr<Request>> table;
  // stats (under mu)
  long long submitted = 0, completed = 0, rejected = 0, canceled = 0, failed = 0;
  long long batches = 0, batched_requests = 0, handles_created = 0, handles_evicted = 0, graph_passes = 0;
  std::vector<double> latency_us;   // ring of the latest completions
  size_t latency_next = 0;
  size_t hbm_bytes = 0;             // written by the worker, read under mu
  // worker-owned
  std::list<CachedHandle> cache;
  std::unordered_map<std::string, int> class_in_flight;   // passes on the GPU per grid class (worker only)
  Slot slots[kSlots];
  size_t used = 0;                  // handles + staging device bytes
  unsigned long long tick = 0;
  cudaStream_t capture = nullptr;   // stream that graphs are captured on (nothing runs on it)
  std::thread worker;
  int init_status = FCM_OK;
  std::string init_error;
};

namespace {

// The grid class of a request: every parameter that shapes the pass, field by field (the
// struct's padding bytes are not part of it).
std::string class_key(const fcm_params& p, bool torque) {
  const double d[9] = {p.L[0], p.L[1], p.L[2], p.a, p.eta, p.Sigma, p.Sigma_D == 0.0 ? p.Sigma : p.Sigma_D, p.r_c,
                       torque ? 1.0 : 0.0};
  const int i[5] = {p.M[0], p.M[1], p.M[2], p.M_G, p.precision};
  std::string k(reinterpret_cast<const char*>(d), sizeof(d));
  k.append(reinterpret_cast<const char*>(i), sizeof(i));
  return k;
}

void record_latency(fcm_server* s, double us) {
  if (s->latency_us.size() < kLatencyWindow) s->latency_us.push_back(us);
  else s->latency_us[s->latency_next] = us;
  s->latency_next = (s->latency_next + 1) % kLatencyWindow;
}

// Completes requests (state, status, latency) and wakes pollers. Caller holds no lock.
void finish_requests(fcm_server* s, std::vector<std::shared_ptr<Request>>& reqs, int status) {
  std::lock_guard<std::mutex> lock(s->mu);
  const Clock::time_point now = Clock::now();
  for (auto& r : reqs) {
    r->state = kDone;
    r->status = status;
    r->t_done = now;
    if (status == FCM_OK) {
      ++s->completed;
      record_latency(s, std::chrono::duration<double, std::micro>(now - r->t_submit).count());
    } else if (status == FCM_ERR_OOM) {
      ++s->rejected;
    } else {
      ++s->failed;
    }
  }
  s->hbm_bytes = s->used;
  s->cv_done.notify_all();
}

int grow(Buffer* b, size_t bytes, bool host, size_t* used, bool* moved) {
  if (b->bytes >= bytes) return FCM_OK;
  *moved = true;
  const size_t want = pow2_at_least(bytes, 1 << 16);
  if (b->p) {
    if (host) cudaFreeHost(b->p);
    else { cudaFree(b->p); *used -= b->bytes; }
    b->p = nullptr;
    b->bytes = 0;
  }
  cudaError_t e = host ? cudaMallocHost(&b->p, want) : cudaMalloc(&b->p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->p = nullptr;
    return fail(FCM_ERR_OOM, std::string("staging allocation failed: ") + cudaGetErrorString(e));
  }
  b->bytes = want;
  if (!host) *used += want;
  return FCM_OK;
}

void destroy_handle(fcm_server* s, std::list<CachedHandle>::iterator it) {
  for (auto& gr : it->graphs) cudaGraphExecDestroy(gr.second);
  for (int k = 0; k < 2; ++k) {
    if (it->d_in[k].p) cudaFree(it->d_in[k].p);
    if (it->d_out[k].p) cudaFree(it->d_out[k].p);
    if (it->set_free[k]) cudaEventDestroy(it->set_free[k]);
  }
  if (it->computed) cudaEventDestroy(it->computed);
  fcm_destroy(it->h);
  s->used -= it->bytes;
  s->cache.erase(it);
}

// Completes a slot whose pass has finished: results to the callers' buffers.
void complete_slot(fcm_server* s, Slot& sl, int status) {
  if (status == FCM_OK) {
    const size_t row = 3 * sl.rsz;
    const char* U = static_cast<const char*>(sl.h_out.p);
    const char* W = U + sl.cap * row;
    for (size_t k = 0; k < sl.reqs.size(); ++k) {
      Request& r = *sl.reqs[k];
      const size_t o = (size_t)sl.offsets[k] * row, bytes = (size_t)r.r.n * row;
      if (bytes == 0) continue;
      std::memcpy(r.r.U, U + o, bytes);
      if (r.r.W) std::memcpy(r.r.W, W + o, bytes);
    }
  }
  if (sl.ch) sl.ch->in_flight -= 1;
  sl.ch = nullptr;
  sl.busy = false;
  if (!sl.reqs.empty()) {
    auto it = s->class_in_flight.find(sl.reqs.front()->key);
    if (it != s->class_in_flight.end() && it->second > 0) it->second -= 1;
  }
  finish_requests(s, sl.reqs, status);
  sl.reqs.clear();
}

// Polls the slots; completes finished passes. Returns true if any finished.
bool reap(fcm_server* s) {
  bool any = false;
  for (Slot& sl : s->slots) {
    if (!sl.busy) continue;
    cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) {
      record_error(FCM_ERR_CUDA, cudaGetErrorString(q));
      complete_slot(s, sl, FCM_ERR_CUDA);
    } else {
      complete_slot(s, sl, FCM_OK);
    }
    any = true;
  }
  return any;
}

bool any_busy(const fcm_server* s) {
  for (const Slot& sl : s->slots)
    if (sl.busy) return true;
  return false;
}

// A cached handle for the class with room for (systems, n), creating one within the budget.
int get_handle(fcm_server* s, const fcm_params& p, const std::string& key, bool torque, int systems, int n,
               CachedHandle** out) {
  *out = nullptr;
  for (auto it = s->cache.begin(); it != s->cache.end(); ++it) {
    if (it->key == key && it->max_systems >= systems && it->max_n >= n) {
      it->last_use = ++s->tick;
      *out = &*it;
      return FCM_OK;
    }
  }
  fcm_params q = p;
  const int want_sys = (int)std::min<size_t>(pow2_at_least(systems, 1), s->max_batch);
  q.max_n = (int)std::min<size_t>(pow2_at_least((size_t)n, 1024), (size_t)1 << 30);
  q.tile[0] = q.tile[1] = q.tile[2] = 0;
  q.spread_kernel = 0;
  const size_t rsz = q.precision == FCM_FP64 ? sizeof(double) : sizeof(float);
  const size_t stage_bytes = 2 * (size_t)q.max_n * 3 * rsz * ((torque ? 3 : 2) + 2);
  const size_t est = workspace_estimate(q, want_sys) + stage_bytes;
  if (est > s->budget)
    return fail(FCM_ERR_OOM, "the request's workspace (" + std::to_string(est) + " bytes) exceeds the HBM budget (" +
                                 std::to_string(s->budget) + " bytes)");
  // evict idle handles, least recently used first; wait for passes in flight if that is not enough
  for (;;) {
    if (s->used + est <= s->budget) break;
    auto victim = s->cache.end();
    for (auto it = s->cache.begin(); it != s->cache.end(); ++it)
      if (it->in_flight == 0 && (victim == s->cache.end() || it->last_use < victim->last_use)) victim = it;
    if (victim != s->cache.end()) {
      destroy_handle(s, victim);
      std::lock_guard<std::mutex> lock(s->mu);
      ++s->handles_evicted;
      continue;
    }
    if (!any_busy(s)) break;   // only staging remains; try anyway
    if (!reap(s)) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  fcm_handle* h = nullptr;
  int rc = fcm_create_batch(&q, want_sys, s->device, &h);
  if (rc != FCM_OK) return rc;
  CachedHandle ch;
  ch.key = key;
  ch.h = h;
  ch.max_systems = want_sys;
  ch.max_n = q.max_n;
  ch.fp32 = q.precision == FCM_FP32;
  ch.torque = torque;
  ch.rsz = rsz;
  ch.last_use = ++s->tick;
  const size_t row = 3 * rsz;
  cudaError_t ce = cudaEventCreateWithFlags(&ch.computed, cudaEventDisableTiming);
  for (int k = 0; k < 2; ++k) {
    ch.d_in[k].bytes = (size_t)q.max_n * row * (torque ? 3 : 2);
    ch.d_out[k].bytes = (size_t)q.max_n * row * 2;
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ch.set_free[k], cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaMalloc(&ch.d_in[k].p, ch.d_in[k].bytes);
    if (ce == cudaSuccess) ce = cudaMalloc(&ch.d_out[k].p, ch.d_out[k].bytes);
  }
  if (ce != cudaSuccess) {
    cudaGetLastError();
    for (int k = 0; k < 2; ++k) {
      if (ch.d_in[k].p) cudaFree(ch.d_in[k].p);
      if (ch.d_out[k].p) cudaFree(ch.d_out[k].p);
      if (ch.set_free[k]) cudaEventDestroy(ch.set_free[k]);
    }
    if (ch.computed) cudaEventDestroy(ch.computed);
    fcm_destroy(h);
    return fail(ce == cudaErrorMemoryAllocation ? FCM_ERR_OOM : FCM_ERR_CUDA,
                std::string("handle staging: ") + cudaGetErrorString(ce));
  }
  ch.bytes = fcm_workspace_bytes(h) + 2 * (ch.d_in[0].bytes + ch.d_out[0].bytes);
  s->used += ch.bytes;
  s->cache.push_back(ch);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    ++s->handles_created;
  }
  *out = &s->cache.back();
  return FCM_OK;
}

// Takes the oldest pending request and every pending request of its class (FIFO), up to the
// batch limits. Called with s->mu held.
std::vector<std::shared_ptr<Request>> take_batch(fcm_server* s) {
  std::vector<std::shared_ptr<Request>> b;
  // the oldest request whose class has no pass in flight picks the class
  const std::string* key = nullptr;
  for (const auto& q : s->pending) {
    auto it = s->class_in_flight.find(q->key);
    if (it == s->class_in_flight.end() || it->second == 0) {
      key = &q->key;
      break;
    }
  }
  if (!key) return b;
  const std::string k = *key;
  long long total = 0;
  for (auto it = s->pending.begin(); it != s->pending.end() && (int)b.size() < s->max_batch;) {
    if ((*it)->key == k && (b.empty() || total + (*it)->r.n <= (1LL << 28))) {
      total += (*it)->r.n;
      (*it)->state = kRunning;
      b.push_back(*it);
      it = s->pending.erase(it);
    } else {
      ++it;
    }
  }
  return b;
}

// The captured pass of (handle, bucket, staging set), captured on first use.
int graph_for(CachedHandle* ch, int bucket, int set, cudaStream_t stream, cudaGraphExec_t* out) {
  *out = nullptr;
  const auto key = std::make_pair(bucket, set);
  auto it = ch->graphs.find(key);
  if (it != ch->graphs.end()) {
    *out = it->second;
    return FCM_OK;
  }
  const size_t row = 3 * ch->rsz, cap = (size_t)ch->max_n;
  char* din = static_cast<char*>(ch->d_in[set].p);
  char* dout = static_cast<char*>(ch->d_out[set].p);
  cudaGraphExec_t exec = nullptr;
  int rc = capture_batch_graph(ch->h, bucket, din, din + cap * row, ch->torque ? din + 2 * cap * row : nullptr, dout,
                               ch->torque ? dout + cap * row : nullptr, stream, &exec);
  if (rc != FCM_OK) return rc;
  ch->graphs[key] = exec;
  *out = exec;
  return FCM_OK;
}

// Stages a batch into a slot and enqueues its pass on the slot's stream, after the handle's
// previous pass: inputs into the handle's staging, a replay of the captured pass for FP32 classes
// (direct fcm_batch_apply otherwise, and if a capture ever failed), results back to the slot.
int launch(fcm_server* s, Slot& sl, std::vector<std::shared_ptr<Request>>& reqs) {
  const Request& r0 = *reqs.front();
  sl.rsz = r0.rsz;
  sl.torque = r0.torque;
  sl.offsets.assign(reqs.size() + 1, 0);
  for (size_t k = 0; k < reqs.size(); ++k) sl.offsets[k + 1] = sl.offsets[k] + reqs[k]->r.n;
  sl.n = sl.offsets.back();
  CachedHandle* ch = nullptr;
  int rc = get_handle(s, r0.r.params, r0.key, r0.torque, (int)reqs.size(), sl.n, &ch);
  if (rc != FCM_OK) return rc;
  const size_t row = 3 * sl.rsz, ntot = (size_t)sl.n;
  sl.cap = (size_t)std::max(ch->max_n, 1);
  const size_t in_bytes = (sl.torque ? 3 : 2) * sl.cap * row, out_bytes = 2 * sl.cap * row;
  bool moved = false;
  if ((rc = grow(&sl.h_in, in_bytes, true, &s->used, &moved)) || (rc = grow(&sl.h_out, out_bytes, true, &s->used, &moved)))
    return rc;
  char* hin = static_cast<char*>(sl.h_in.p);
  for (size_t k = 0; k < reqs.size(); ++k) {
    const fcm_request& q = reqs[k]->r;
    const size_t o = (size_t)sl.offsets[k] * row, bytes = (size_t)q.n * row;
    if (bytes == 0) continue;
    std::memcpy(hin + o, q.pos, bytes);
    std::memcpy(hin + sl.cap * row + o, q.F, bytes);
    if (sl.torque) {
      if (q.T) std::memcpy(hin + 2 * sl.cap * row + o, q.T, bytes);
      else std::memset(hin + 2 * sl.cap * row + o, 0, bytes);
    }
  }
  const int set = ch->next_set;
  ch->next_set ^= 1;
  char* din = static_cast<char*>(ch->d_in[set].p);
  char* dout = static_cast<char*>(ch->d_out[set].p);
  auto cuda = [&](cudaError_t e, const char* what) -> int {
    if (e == cudaSuccess) return FCM_OK;
    cudaGetLastError();
    return fail(FCM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  const int nsys = (int)reqs.size();
  if (ch->max_systems < nsys) return fail(FCM_ERR_ARG, "batch larger than the handle");
  // inputs into the staging set once its previous pass is done with it; kernels (and the offsets
  // they read) once the handle's previous pass has computed
  if ((rc = cuda(cudaStreamWaitEvent(sl.stream, ch->set_free[set], 0), "staging ordering"))) return rc;
  for (int a = 0; a < (sl.torque ? 3 : 2); ++a) {
    if ((rc = cuda(cudaMemcpyAsync(din + a * sl.cap * row, hin + a * sl.cap * row, ntot * row, cudaMemcpyHostToDevice,
                                   sl.stream), "input copy")))
      return rc;
  }
  bool replayed = false;
  if (ch->fp32 && ch->graphs_ok) {
    int bucket = 1;
    while (bucket < nsys) bucket <<= 1;
    bucket = std::min(bucket, ch->max_systems);
    for (int k = 0; k <= bucket; ++k) sl.h_off[k] = k <= nsys ? sl.offsets[k] : sl.n;
    cudaGraphExec_t exec = nullptr;
    if (graph_for(ch, bucket, set, s->capture, &exec) == FCM_OK) {
      if ((rc = cuda(cudaStreamWaitEvent(sl.stream, ch->computed, 0), "handle ordering"))) return rc;
      if ((rc = cuda(cudaMemcpyAsync(handle_sys_off(ch->h), sl.h_off, sizeof(int) * (size_t)(bucket + 1),
                                     cudaMemcpyHostToDevice, sl.stream), "offsets copy")))
        return rc;
      if ((rc = cuda(cudaGraphLaunch(exec, sl.stream), "graph launch"))) return rc;
      replayed = true;
    } else {
      ch->graphs_ok = false;   // capture is not available here: direct launches from now on
    }
  }
  if (!replayed) {
    if ((rc = cuda(cudaStreamWaitEvent(sl.stream, ch->computed, 0), "handle ordering"))) return rc;
    rc = fcm_batch_apply(ch->h, nsys, sl.offsets.data(), din, din + sl.cap * row,
                         sl.torque ? din + 2 * sl.cap * row : nullptr, dout, sl.torque ? dout + sl.cap * row : nullptr,
                         sl.stream);
    if (rc != FCM_OK) return rc;
  }
  if ((rc = cuda(cudaEventRecord(ch->computed, sl.stream), "event"))) return rc;
  char* hout = static_cast<char*>(sl.h_out.p);
  if ((rc = cuda(cudaMemcpyAsync(hout, dout, ntot * row, cudaMemcpyDeviceToHost, sl.stream), "output copy"))) return rc;
  if (sl.torque &&
      (rc = cuda(cudaMemcpyAsync(hout + sl.cap * row, dout + sl.cap * row, ntot * row, cudaMemcpyDeviceToHost, sl.stream),
                 "output copy")))
    return rc;
  if ((rc = cuda(cudaEventRecord(ch->set_free[set], sl.stream), "event"))) return rc;
  if ((rc = cuda(cudaEventRecord(sl.done, sl.stream), "event"))) return rc;
  ch->in_flight += 1;
  ch->last_use = ++s->tick;
  sl.ch = ch;
  sl.reqs = reqs;
  sl.busy = true;
  (void)moved;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    ++s->batches;
    s->batched_requests += (long long)reqs.size();
    if (replayed) ++s->graph_passes;
    s->hbm_bytes = s->used;
  }
  return FCM_OK;
}

void worker_main(fcm_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    bool progressed = reap(s);
    Slot* free_slot = nullptr;
    for (Slot& sl : s->slots)
      if (!sl.busy) { free_slot = &sl; break; }
    std::vector<std::shared_ptr<Request>> batch;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      if (s->stop) break;
      if (free_slot) batch = take_batch(s);
      if (batch.empty() && !progressed) {
        if (any_busy(s)) {
          lock.unlock();
          std::this_thread::sleep_for(std::chrono::microseconds(20));
        } else {
          s->cv_work.wait_for(lock, std::chrono::milliseconds(5), [&] { return s->stop || !s->pending.empty(); });
        }
        continue;
      }
    }
    if (!batch.empty()) {
      const std::string key = batch.front()->key;
      int rc = launch(s, *free_slot, batch);
      if (rc != FCM_OK) {
        finish_requests(s, batch, rc);
      } else {
        s->class_in_flight[key] += 1;   // worker-owned, like the slots
      }
    }
  }
  // shutdown: let passes in flight end (kernels are finite), then release everything
  for (Slot& sl : s->slots) {
    if (sl.busy) {
      cudaError_t e = cudaEventSynchronize(sl.done);
      complete_slot(s, sl, e == cudaSuccess ? FCM_OK : FCM_ERR_CUDA);
    }
  }
}

void release_server(fcm_server* s) {
  cudaSetDevice(s->device);
  while (!s->cache.empty()) destroy_handle(s, s->cache.begin());
  if (s->capture) cudaStreamDestroy(s->capture);
  for (Slot& sl : s->slots) {
    if (sl.h_in.p) cudaFreeHost(sl.h_in.p);
    if (sl.h_out.p) cudaFreeHost(sl.h_out.p);
    if (sl.h_off) cudaFreeHost(sl.h_off);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
}

}  // namespace

#pragma GCC visibility push(default)
extern "C" {

int fcm_server_create(int device, size_t hbm_budget, int max_batch, fcm_server** out) {
  if (!out) return fail(FCM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (max_batch < 1 || max_batch > FCM_MAX_BATCH)
    return fail(FCM_ERR_ARG, "max_batch must be in [1, " + std::to_string(FCM_MAX_BATCH) + "]");
  if (hbm_budget == 0) return fail(FCM_ERR_ARG, "hbm_budget must be > 0");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(FCM_ERR_CUDA, "CUDA device " + std::to_string(device) + " is not available");
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  fcm_server* s = new fcm_server();
  s->device = device;
  s->budget = hbm_budget;
  s->max_batch = max_batch;
  s->latency_us.reserve(1024);
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < kSlots; ++k) {
    Slot& sl = s->slots[k];
    sl.index = k;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_off, sizeof(int) * (FCM_MAX_BATCH + 1));
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking);
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release_server(s);
    return fail(FCM_ERR_CUDA, std::string("server setup: ") + cudaGetErrorString(e));
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return FCM_OK;
}

int fcm_server_submit(fcm_server* s, const fcm_request* r, long long* id) {
  if (!s || !r || !id) return fail(FCM_ERR_ARG, "server, request and id must be non-NULL");
  *id = 0;
  std::string why;
  if (!check_params(&r->params, &why)) {
    std::lock_guard<std::mutex> lock(s->mu);
    ++s->rejected;
    return fail(FCM_ERR_ARG, why);
  }
  if (r->n < 0 || (r->n > 0 && (!r->pos || !r->F || !r->U))) {
    std::lock_guard<std::mutex> lock(s->mu);
    ++s->rejected;
    return fail(FCM_ERR_ARG, "n must be >= 0 and pos, F, U non-NULL when n > 0");
  }
  auto q = std::make_shared<Request>();
  q->r = *r;
  q->torque = (r->T != nullptr) || (r->W != nullptr);
  q->key = class_key(r->params, q->torque);
  q->rsz = r->params.precision == FCM_FP64 ? sizeof(double) : sizeof(float);
  q->t_submit = Clock::now();
  std::lock_guard<std::mutex> lock(s->mu);
  q->id = s->next_id++;
  ++s->submitted;
  s->table.emplace(q->id, q);
  if (r->n == 0) {   // nothing to compute
    q->state = kDone;
    q->status = FCM_OK;
    q->t_done = q->t_submit;
    ++s->completed;
    record_latency(s, 0.0);
  } else {
    s->pending.push_back(q);
    s->cv_work.notify_one();
  }
  *id = q->id;
  return FCM_OK;
}

int fcm_server_poll(fcm_server* s, long long id, long long timeout_us, int* status) {
  if (!s || !status) return fail(FCM_ERR_ARG, "server and status must be non-NULL");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->table.find(id);
  if (it == s->table.end()) return fail(FCM_ERR_ARG, "unknown request id " + std::to_string(id));
  std::shared_ptr<Request> q = it->second;
  if (q->state != kDone && timeout_us > 0)
    s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), [&] { return q->state == kDone; });
  if (q->state != kDone) return fail(FCM_ERR_TIMEOUT, "request " + std::to_string(id) + " not finished");
  *status = q->status;
  s->table.erase(id);
  return FCM_OK;
}

int fcm_server_cancel(fcm_server* s, long long id) {
  if (!s) return fail(FCM_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->table.find(id);
  if (it == s->table.end()) return fail(FCM_ERR_ARG, "unknown request id " + std::to_string(id));
  std::shared_ptr<Request> q = it->second;
  if (q->state != kPending) return fail(FCM_ERR_BUSY, "request " + std::to_string(id) + " already launched or done");
  for (auto p = s->pending.begin(); p != s->pending.end(); ++p)
    if ((*p)->id == id) { s->pending.erase(p); break; }
  q->state = kDone;
  q->status = FCM_ERR_CANCELED;
  q->t_done = Clock::now();
  ++s->canceled;
  s->cv_done.notify_all();
  return FCM_OK;
}

int fcm_server_get_stats(fcm_server* s, fcm_server_stats* out) {
  if (!s || !out) return fail(FCM_ERR_ARG, "server and out must be non-NULL");
  std::vector<double> lat;
  std::lock_guard<std::mutex> lock(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->rejected = s->rejected;
  out->canceled = s->canceled;
  out->failed = s->failed;
  out->pending = (long long)s->pending.size();
  out->batches = s->batches;
  out->batched_requests = s->batched_requests;
  out->handles_created = s->handles_created;
  out->handles_evicted = s->handles_evicted;
  out->graph_passes = s->graph_passes;
  out->hbm_bytes = s->hbm_bytes;
  out->hbm_budget = s->budget;
  lat = s->latency_us;
  if (!lat.empty()) {
    auto pct = [&](double f) {
      size_t k = (size_t)std::min<double>((double)lat.size() - 1, f * (double)(lat.size() - 1) + 0.5);
      std::nth_element(lat.begin(), lat.begin() + k, lat.end());
      return lat[k];
    };
    out->latency_p50_us = pct(0.50);
    out->latency_p99_us = pct(0.99);
    out->latency_max_us = *std::max_element(lat.begin(), lat.end());
  }
  return FCM_OK;
}

int fcm_server_reset_latency(fcm_server* s) {
  if (!s) return fail(FCM_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  s->latency_us.clear();
  s->latency_next = 0;
  return FCM_OK;
}

int fcm_server_destroy(fcm_server* s) {
  if (!s) return FCM_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    for (auto& q : s->pending) {
      q->state = kDone;
      q->status = FCM_ERR_CANCELED;
      ++s->canceled;
    }
    s->pending.clear();
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  release_server(s);
  return FCM_OK;
}

}  // extern "C"
#pragma GCC visibility pop
