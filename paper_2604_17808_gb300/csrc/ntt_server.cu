// ntt_server.cu -- request-serving runtime with continuous batching.
//
// A prover that serves many clients submits transforms of mixed sizes,
// kinds and fields as they arrive.  The server keeps a plan (with its
// twiddle tables) resident for every (field, size) it serves, admits
// requests against a device-memory budget, and runs admitted requests as
// batches (one persistent kernel per field and batch, ntt_batch.cu) on
// several streams, so that requests arriving while others are on the GPU
// are admitted as soon as memory and an in-flight slot free up and their
// work overlaps with the running batches.
//
// Flow of one request: submit (host buffers, timestamp "arrive") -> queue
// -> admission (device buffers reserved from the budget, "admit") -> batch
// on a free stream: host-to-device copy, kernel, device-to-host copy ->
// stream callback marks the batch done -> the worker retires it
// ("finish"), returns the device buffers and admits more.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <set>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ntt_launch.h"
#include "ntt_plan.h"
#include "nvtx_range.h"

using namespace gb300ntt;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int field = 0;
  int kind = 0;
  uint32_t log_n = 0;
  const void *h_in = nullptr;
  void *h_out = nullptr;
  double arrive = 0, admit = 0, finish = 0;
  void *d_in = nullptr, *d_out = nullptr;
  bool done = false;
};

// Buddy allocator over one device arena.  Request buffers are 32 * 2^log_n
// bytes, so blocks of order k (32 * 2^k bytes) split and coalesce exactly;
// the arena is reserved once at server creation, so serving never calls
// cudaMalloc / cudaFree (cudaFree synchronises the whole device).
class BuddyArena {
 public:
  ntt_status init(uint64_t bytes, uint32_t max_order) {
    max_order_ = max_order;
    const uint64_t top = kUnit << max_order;
    const uint64_t n_top = bytes / top;
    if (n_top == 0) return NTT_ERR_BUDGET;
    if (cudaMalloc(&base_, n_top * top) != cudaSuccess) {
      cudaGetLastError();
      base_ = nullptr;
      return NTT_ERR_OOM;
    }
    capacity_ = n_top * top;
    free_.assign(max_order + 1, {});
    for (uint64_t i = 0; i < n_top; ++i) free_[max_order].insert(i << max_order);
    return NTT_OK;
  }
  ~BuddyArena() {
    if (base_) cudaFree(base_);
  }
  // nullptr when no block of this order can be formed right now
  void *alloc(uint32_t order) {
    uint32_t o = order;
    while (o <= max_order_ && free_[o].empty()) ++o;
    if (o > max_order_) return nullptr;
    uint64_t off = *free_[o].begin();
    free_[o].erase(free_[o].begin());
    while (o > order) {  // split, keep the lower half
      --o;
      free_[o].insert(off + (1ull << o));
    }
    used_ += kUnit << order;
    peak_ = std::max(peak_, used_);
    return static_cast<char *>(base_) + off * kUnit;
  }
  void release(void *p, uint32_t order) {
    uint64_t off = (uint64_t)(static_cast<char *>(p) - static_cast<char *>(base_)) / kUnit;
    used_ -= kUnit << order;
    while (order < max_order_) {
      const uint64_t buddy = off ^ (1ull << order);
      auto it = free_[order].find(buddy);
      if (it == free_[order].end()) break;
      free_[order].erase(it);
      off = std::min(off, buddy);
      ++order;
    }
    free_[order].insert(off);
  }
  uint64_t capacity() const { return capacity_; }
  uint64_t peak() const { return peak_; }

 private:
  static constexpr uint64_t kUnit = 32;
  void *base_ = nullptr;
  uint32_t max_order_ = 0;
  uint64_t capacity_ = 0, used_ = 0, peak_ = 0;
  std::vector<std::set<uint64_t>> free_;
};

// One in-flight batch slot: a stream, its segment staging and device tables.
struct Slot {
  cudaStream_t stream = nullptr;
  BatchSeg *h_segs[2] = {nullptr, nullptr};  // pinned staging per field
  BatchSeg *d_segs[2] = {nullptr, nullptr};
  uint32_t *d_ctl[2] = {nullptr, nullptr};
  uint32_t cap = 0;                          // segments per field
  std::vector<uint64_t> tickets;
  std::atomic<int> complete{0};
  bool busy = false;
};

}  // namespace

struct ntt_server_s {
  ntt_server_config cfg{};
  int device = 0;
  int sm_count = 0;
  Clock::time_point t0;
  ntt_plan plans[2][32] = {};
  uint64_t resident_bytes = 0;
  BuddyArena arena;            // request buffers (budget - resident tables)
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;  // tickets waiting for admission
  std::deque<uint64_t> admitted;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<Slot *> slots;
  uint64_t next_ticket = 1;
  uint64_t submitted = 0, completed = 0, batches = 0;
  bool stop = false;
  ntt_status error = NTT_OK;
  std::thread worker;
};

namespace {

double now_s(const ntt_server_s *s) {
  return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

uint64_t job_bytes(uint32_t log_n) { return 32ull << log_n; }

void CUDART_CB slot_done(void *arg) {
  static_cast<Slot *>(arg)->complete.store(1, std::memory_order_release);
}

// Dispatch the admitted requests (up to the batch limits) on slot `sl`.
void dispatch(ntt_server_s *s, Slot *sl) {
  NvtxRange range("ntt_server_dispatch");
  std::vector<BatchJobRef> jobs;
  uint64_t elems = 0;
  sl->tickets.clear();
  while (!s->admitted.empty() && jobs.size() < s->cfg.max_batch_jobs) {
    Request &r = s->reqs[s->admitted.front()];
    if (!jobs.empty() && elems + (1ull << r.log_n) > s->cfg.max_batch_elements) break;
    s->admitted.pop_front();
    jobs.push_back(BatchJobRef{s->plans[r.field][r.log_n], r.kind, r.d_in, r.d_out});
    sl->tickets.push_back(r.ticket);
    elems += 1ull << r.log_n;
  }
  if (jobs.empty()) return;
  cudaStream_t st = sl->stream;
  for (uint64_t t : sl->tickets) {
    Request &r = s->reqs[t];
    cudaMemcpyAsync(r.d_in, r.h_in, job_bytes(r.log_n), cudaMemcpyHostToDevice, st);
  }
  uint32_t *err = nullptr;
  batch_error_word(&err);
  for (int field = 0; field < 2; ++field) {
    uint32_t total = 0;
    std::vector<BatchSeg> segs = build_segments(jobs, field, &total);
    if (segs.empty()) continue;
    if (segs.size() > sl->cap) {  // cannot happen with the configured limits
      s->error = NTT_ERR_INVALID_ARG;
      continue;
    }
    std::memcpy(sl->h_segs[field], segs.data(), segs.size() * sizeof(BatchSeg));
    cudaMemcpyAsync(sl->d_segs[field], sl->h_segs[field], segs.size() * sizeof(BatchSeg), cudaMemcpyHostToDevice,
                    st);
    cudaMemsetAsync(sl->d_ctl[field], 0, (1 + segs.size()) * sizeof(uint32_t), st);
    BatchLaunch b;
    b.segs = sl->d_segs[field];
    b.num_segs = (uint32_t)segs.size();
    b.total_items = total;
    b.head = sl->d_ctl[field];
    b.done = sl->d_ctl[field] + 1;
    b.err = err;
    b.wait_ns = batch_wait_limit_ns();
    b.grid = (uint32_t)(s->sm_count * kPassCtasPerSm);
    if (launchers(field).batch(b, st) != cudaSuccess) s->error = NTT_ERR_CUDA;
  }
  for (uint64_t t : sl->tickets) {
    Request &r = s->reqs[t];
    cudaMemcpyAsync(r.h_out, r.d_out, job_bytes(r.log_n), cudaMemcpyDeviceToHost, st);
  }
  sl->complete.store(0);
  sl->busy = true;
  cudaLaunchHostFunc(st, slot_done, sl);
  s->batches += 1;
}

void worker_loop(ntt_server_s *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool progress = false;
    // retire finished batches
    for (Slot *sl : s->slots) {
      if (sl->busy && sl->complete.load(std::memory_order_acquire)) {
        const double t = now_s(s);
        for (uint64_t tk : sl->tickets) {
          Request &r = s->reqs[tk];
          r.finish = t;
          r.done = true;
          s->arena.release(r.d_in, r.log_n);
          s->arena.release(r.d_out, r.log_n);
          r.d_in = r.d_out = nullptr;
          s->completed += 1;
        }
        sl->tickets.clear();
        sl->busy = false;
        progress = true;
      }
    }
    if (progress) s->cv.notify_all();
    // admit waiting requests while memory allows (in arrival order)
    while (!s->queue.empty()) {
      Request &r = s->reqs[s->queue.front()];
      void *in = s->arena.alloc(r.log_n);
      if (!in) break;
      void *out = s->arena.alloc(r.log_n);
      if (!out) {
        s->arena.release(in, r.log_n);
        break;
      }
      r.d_in = in;
      r.d_out = out;
      r.admit = now_s(s);
      s->admitted.push_back(r.ticket);
      s->queue.pop_front();
      progress = true;
    }
    // dispatch on free slots
    for (Slot *sl : s->slots) {
      if (s->admitted.empty()) break;
      if (!sl->busy) {
        dispatch(s, sl);
        progress = true;
      }
    }
    bool inflight = false;
    for (Slot *sl : s->slots) inflight |= sl->busy;
    if (s->stop && s->queue.empty() && s->admitted.empty() && !inflight) break;
    if (!progress) {
      // poll in-flight batches every 20 us; otherwise sleep until a submit
      if (inflight) s->cv.wait_for(lk, std::chrono::microseconds(20));
      else s->cv.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

void destroy_server(ntt_server_s *s) {
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv.notify_all();
    s->worker.join();
  }
  cudaDeviceSynchronize();
  for (Slot *sl : s->slots) {
    if (sl->stream) cudaStreamDestroy(sl->stream);
    for (int f = 0; f < 2; ++f) {
      if (sl->h_segs[f]) cudaFreeHost(sl->h_segs[f]);
      if (sl->d_segs[f]) cudaFree(sl->d_segs[f]);
      if (sl->d_ctl[f]) cudaFree(sl->d_ctl[f]);
    }
    delete sl;
  }
  for (auto &row : s->plans)
    for (ntt_plan p : row)
      if (p) ntt_plan_destroy(p);
  delete s;
}

}  // namespace

extern "C" {

ntt_status ntt_server_create(const ntt_server_config *cfg, ntt_server *out) {
  if (!out) return NTT_ERR_INVALID_ARG;
  *out = nullptr;
  ntt_server_config c{};
  c.memory_budget_bytes = 64ull << 30;
  c.min_log_n = 12;
  c.max_log_n = 24;
  c.max_inflight = 3;
  c.max_batch_jobs = 64;
  c.max_batch_elements = 1ull << 26;
  if (cfg) {
    if (cfg->memory_budget_bytes) c.memory_budget_bytes = cfg->memory_budget_bytes;
    if (cfg->min_log_n) c.min_log_n = cfg->min_log_n;
    if (cfg->max_log_n) c.max_log_n = cfg->max_log_n;
    if (cfg->max_inflight) c.max_inflight = cfg->max_inflight;
    if (cfg->max_batch_jobs) c.max_batch_jobs = cfg->max_batch_jobs;
    if (cfg->max_batch_elements) c.max_batch_elements = cfg->max_batch_elements;
  }
  if (c.min_log_n < 1 || c.max_log_n > 28 || c.min_log_n > c.max_log_n || c.max_inflight > 16)
    return NTT_ERR_INVALID_ARG;
  ntt_server_s *s = new (std::nothrow) ntt_server_s();
  if (!s) return NTT_ERR_OOM;
  s->cfg = c;
  s->t0 = Clock::now();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return NTT_ERR_NO_DEVICE;
  }
  cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  // resident plans (with coset tables) for every served size and field
  for (int f = 0; f < 2; ++f) {
    for (uint32_t ln = c.min_log_n; ln <= c.max_log_n; ++ln) {
      if (f == 1 && ln > 28) continue;
      ntt_status st = ntt_plan_create(&s->plans[f][ln], (ntt_field)f, ln, 1);
      if (st != NTT_OK) {
        destroy_server(s);
        return st;
      }
      s->resident_bytes += s->plans[f][ln]->device_bytes;
    }
  }
  if (s->resident_bytes + 2 * job_bytes(c.max_log_n) > c.memory_budget_bytes) {
    destroy_server(s);
    return NTT_ERR_BUDGET;
  }
  {
    const ntt_status st = s->arena.init(c.memory_budget_bytes - s->resident_bytes, c.max_log_n);
    if (st != NTT_OK) {
      destroy_server(s);
      return st;
    }
  }
  // in-flight slots: worst-case segment count per field = jobs * passes
  const uint32_t cap = c.max_batch_jobs * 4;
  for (uint32_t i = 0; i < c.max_inflight; ++i) {
    Slot *sl = new Slot();
    s->slots.push_back(sl);
    ntt_status st = cuda_status(cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking));
    sl->cap = cap;
    for (int f = 0; f < 2 && st == NTT_OK; ++f) {
      st = cuda_status(cudaMallocHost(&sl->h_segs[f], cap * sizeof(BatchSeg)));
      if (st == NTT_OK) st = cuda_status(cudaMalloc(&sl->d_segs[f], cap * sizeof(BatchSeg)));
      if (st == NTT_OK) st = cuda_status(cudaMalloc(&sl->d_ctl[f], (1 + cap) * sizeof(uint32_t)));
    }
    if (st != NTT_OK) {
      destroy_server(s);
      return st;
    }
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return NTT_OK;
}

ntt_status ntt_server_submit(ntt_server s, ntt_field field, ntt_kind kind, uint32_t log_n, const void *h_in,
                             void *h_out, uint64_t *ticket) {
  if (!s || !h_in || !h_out || !ticket) return NTT_ERR_INVALID_ARG;
  if (field != NTT_FIELD_BLS12_381_FR && field != NTT_FIELD_BN254_FR) return NTT_ERR_INVALID_ARG;
  if (!kind_is_valid((int)kind, true)) return NTT_ERR_INVALID_ARG;
  if (log_n < s->cfg.min_log_n || log_n > s->cfg.max_log_n || !s->plans[field][log_n]) return NTT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->error != NTT_OK) return s->error;
  Request r;
  r.ticket = s->next_ticket++;
  r.field = (int)field;
  r.kind = (int)kind;
  r.log_n = log_n;
  r.h_in = h_in;
  r.h_out = h_out;
  r.arrive = now_s(s);
  s->reqs[r.ticket] = r;
  s->queue.push_back(r.ticket);
  s->submitted += 1;
  *ticket = r.ticket;
  s->cv.notify_all();
  return NTT_OK;
}

ntt_status ntt_server_query(ntt_server s, uint64_t ticket, int *done) {
  if (!s || !done) return NTT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return NTT_ERR_INVALID_ARG;
  *done = it->second.done ? 1 : 0;
  return NTT_OK;
}

ntt_status ntt_server_wait(ntt_server s, uint64_t ticket, double timeout_s) {
  if (!s) return NTT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return NTT_ERR_INVALID_ARG;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9));
  while (!s->reqs[ticket].done) {
    if (s->error != NTT_OK) return s->error;
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && !s->reqs[ticket].done) return NTT_ERR_TIMEOUT;
  }
  return NTT_OK;
}

ntt_status ntt_server_request_times(ntt_server s, uint64_t ticket, double *arrive_s, double *admit_s,
                                    double *finish_s) {
  if (!s || !arrive_s || !admit_s || !finish_s) return NTT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return NTT_ERR_INVALID_ARG;
  *arrive_s = it->second.arrive;
  *admit_s = it->second.admit;
  *finish_s = it->second.finish;
  return NTT_OK;
}

ntt_status ntt_server_release(ntt_server s, uint64_t ticket) {
  if (!s) return NTT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end() || !it->second.done) return NTT_ERR_INVALID_ARG;
  s->reqs.erase(it);
  return NTT_OK;
}

ntt_status ntt_server_get_stats(ntt_server s, ntt_server_stats *out) {
  if (!s || !out) return NTT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->batches = s->batches;
  out->queued = s->queue.size() + s->admitted.size();
  out->resident_bytes = s->resident_bytes;
  out->peak_device_bytes = s->resident_bytes + s->arena.peak();
  out->budget_bytes = s->cfg.memory_budget_bytes;
  return NTT_OK;
}

ntt_status ntt_server_destroy(ntt_server s) {
  if (!s) return NTT_OK;
  destroy_server(s);
  return NTT_OK;
}

}  // extern "C"
