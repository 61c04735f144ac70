// ntt_batch.cu -- many independent transforms in one persistent launch.
//
// The paper batches NTTs to keep its matrix units busy (Sec. 4.4, Fig. 7).
// On GB300 a single small transform leaves most of the 152 SMs idle (a
// 2^14-point pass has 8 tiles), so a batch is run as one persistent kernel
// per field: every (job, pass, tile) is an item in one queue ordered by pass
// level, CTAs (3 per SM) claim items with an atomic counter, and an item of
// pass j waits (time-bounded) for the completion counter of pass j-1 of its
// own job.  The segment table and counters of a job list are built once; the
// launch sequence (counter reset + kernels) is captured into a CUDA graph and
// replayed on later submissions of the same job list.
#include <cuda_runtime.h>

#include <algorithm>
#include <list>
#include <mutex>
#include <tuple>
#include <vector>

#include "ntt_launch.h"
#include "ntt_plan.h"

using namespace gb300ntt;

namespace {

struct JobKey {
  ntt_plan plan;
  int32_t kind;
  const void *in;
  void *out;
  bool operator==(const JobKey &o) const {
    return plan == o.plan && kind == o.kind && in == o.in && out == o.out;
  }
};

struct Part {
  int field = 0;
  BatchSeg *d_segs = nullptr;
  uint32_t *d_ctl = nullptr;  // [0] = head, [1 + s] = done tiles of segment s
  uint32_t num_segs = 0;
  uint32_t total_items = 0;
};

struct Entry {
  std::vector<JobKey> key;
  int device = 0;
  std::vector<Part> parts;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

constexpr size_t kCacheEntries = 16;
std::mutex g_mu;
std::list<Entry> g_cache;                 // most recently used first
uint64_t g_wait_ns = 2000000000ull;       // 2 s per dependency wait
bool g_stall = false;                     // test hook: one unsatisfiable wait
uint32_t *g_err[64] = {};                 // per-device batch error word

void free_entry(Entry &e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.graph) cudaGraphDestroy(e.graph);
  for (Part &p : e.parts) {
    if (p.d_segs) cudaFree(p.d_segs);
    if (p.d_ctl) cudaFree(p.d_ctl);
  }
  e.parts.clear();
  e.exec = nullptr;
  e.graph = nullptr;
}

void clear_cache_locked() {
  if (!g_cache.empty()) cudaDeviceSynchronize();
  for (Entry &e : g_cache) free_entry(e);
  g_cache.clear();
}

ntt_status device_err_word(int dev, uint32_t **out) {
  if (dev < 0 || dev >= 64) return NTT_ERR_INVALID_ARG;
  if (!g_err[dev]) {
    uint32_t *p = nullptr;
    if (cudaMalloc(&p, sizeof(uint32_t)) != cudaSuccess) return NTT_ERR_OOM;
    if (cudaMemset(p, 0, sizeof(uint32_t)) != cudaSuccess) return NTT_ERR_CUDA;
    g_err[dev] = p;
  }
  *out = g_err[dev];
  return NTT_OK;
}

}  // namespace

namespace gb300ntt {

// Segment table of the jobs of one field: every pass of every job, ordered
// by pass level (larger jobs first within a level).  Pure host code.
std::vector<BatchSeg> build_segments(const std::vector<BatchJobRef> &jobs, int field, uint32_t *total_items) {
  std::vector<BatchSeg> segs;
  std::vector<std::vector<int>> seg_of(jobs.size());  // [job][pass] -> segment index
  uint32_t max_passes = 0;
  for (const BatchJobRef &j : jobs)
    if (j.plan->field == field) max_passes = std::max(max_passes, j.plan->num_passes);
  std::vector<size_t> order;
  for (size_t i = 0; i < jobs.size(); ++i)
    if (jobs[i].plan->field == field) order.push_back(i);
  std::stable_sort(order.begin(), order.end(),
                   [&](size_t a, size_t b) { return jobs[a].plan->log_n > jobs[b].plan->log_n; });
  for (size_t i : order) seg_of[i].assign(jobs[i].plan->num_passes, -1);
  uint32_t item = 0;
  for (uint32_t level = 0; level < max_passes; ++level) {
    for (size_t i : order) {
      const BatchJobRef &j = jobs[i];
      if (level >= j.plan->num_passes) continue;
      BatchSeg s{};
      int mode = 0;
      build_pass_args(j.plan, j.kind, j.in, j.out, level, &s.a, &mode);
      s.logs = j.plan->pass_log[level];
      s.mode = (uint32_t)mode;
      s.first_item = item;
      s.num_tiles = (uint32_t)pass_tiles(j.plan->log_n, s.logs, kTileLog);
      if (level > 0) {
        s.dep_seg = seg_of[i][level - 1];
        s.dep_tiles = segs[s.dep_seg].num_tiles;
      } else {
        s.dep_seg = -1;
        s.dep_tiles = 0;
      }
      seg_of[i][level] = (int)segs.size();
      item += s.num_tiles;
      segs.push_back(s);
    }
  }
  *total_items = item;
  return segs;
}

uint64_t batch_wait_limit_ns() { return g_wait_ns; }

bool batch_debug_stall() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_stall;
}

ntt_status batch_error_word(uint32_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NTT_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lk(g_mu);
  return device_err_word(dev, out);
}

}  // namespace gb300ntt

namespace {

// Build the segment table of the jobs of one field and upload it.
ntt_status build_part(const std::vector<JobKey> &jobs, int field, Part *part) {
  std::vector<BatchJobRef> refs;
  for (const JobKey &j : jobs) refs.push_back(BatchJobRef{j.plan, j.kind, j.in, j.out});
  uint32_t item = 0;
  std::vector<BatchSeg> segs = build_segments(refs, field, &item);
  if (segs.empty()) return NTT_OK;
  if (g_stall) {
    // test hook: the last segment waits for one tile more than exists
    for (int k = (int)segs.size() - 1; k >= 0; --k)
      if (segs[k].dep_seg >= 0) {
        segs[k].dep_tiles += 1;
        break;
      }
  }
  part->field = field;
  part->num_segs = (uint32_t)segs.size();
  part->total_items = item;
  ntt_status st = cuda_status(cudaMalloc(&part->d_segs, segs.size() * sizeof(BatchSeg)));
  if (st == NTT_OK) st = cuda_status(cudaMalloc(&part->d_ctl, (1 + segs.size()) * sizeof(uint32_t)));
  if (st == NTT_OK)
    st = cuda_status(cudaMemcpy(part->d_segs, segs.data(), segs.size() * sizeof(BatchSeg), cudaMemcpyHostToDevice));
  return st;
}

ntt_status build_entry(Entry &e, int sm_count) {
  cudaGetDevice(&e.device);
  uint32_t *err = nullptr;
  ntt_status st = device_err_word(e.device, &err);
  if (st != NTT_OK) return st;
  for (int field = 0; field < 2; ++field) {
    bool any = false;
    for (const JobKey &j : e.key) any |= j.plan->field == field;
    if (!any) continue;
    Part part;
    st = build_part(e.key, field, &part);
    e.parts.push_back(part);
    if (st != NTT_OK) return st;
  }
  cudaStream_t cs = nullptr;
  st = cuda_status(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  if (st != NTT_OK) return st;
  st = cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  if (st == NTT_OK) {
    for (const Part &part : e.parts) {
      if (!part.total_items) continue;
      cudaMemsetAsync(part.d_ctl, 0, (1 + part.num_segs) * sizeof(uint32_t), cs);
      BatchLaunch b;
      b.segs = part.d_segs;
      b.num_segs = part.num_segs;
      b.total_items = part.total_items;
      b.head = part.d_ctl;
      b.done = part.d_ctl + 1;
      b.err = err;
      b.wait_ns = g_wait_ns;
      b.grid = (uint32_t)(sm_count * kPassCtasPerSm);
      launchers(part.field).batch(b, cs);
    }
    const cudaError_t ce = cudaStreamEndCapture(cs, &e.graph);
    st = cuda_status(ce);
    if (st == NTT_OK) st = cuda_status(cudaGraphInstantiate(&e.exec, e.graph, 0));
  }
  cudaStreamDestroy(cs);
  return st;
}

}  // namespace

extern "C" {

ntt_status ntt_batch_submit(const ntt_job *jobs, size_t n, ntt_stream stream) {
  if (!jobs && n) return NTT_ERR_INVALID_ARG;
  if (n == 0) return NTT_OK;
  std::vector<JobKey> key(n);
  for (size_t i = 0; i < n; ++i) {
    const ntt_job &j = jobs[i];
    if (!j.plan || j.in == j.out) return NTT_ERR_INVALID_ARG;
    if (!kind_is_valid(j.kind, j.plan->has_coset)) return NTT_ERR_INVALID_ARG;
    if (j.plan->path == NTT_PATH_MATRIX) return NTT_ERR_UNSUPPORTED;
    ntt_status s = check_buffer(j.in);
    if (s == NTT_OK) s = check_buffer(j.out);
    if (s != NTT_OK) return s;
    key[i] = JobKey{j.plan, j.kind, j.in, j.out};
  }
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  auto it = std::find_if(g_cache.begin(), g_cache.end(),
                         [&](const Entry &e) { return e.device == dev && e.key == key; });
  if (it == g_cache.end()) {
    if (g_cache.size() >= kCacheEntries) {
      cudaDeviceSynchronize();
      free_entry(g_cache.back());
      g_cache.pop_back();
    }
    Entry e;
    e.key = key;
    const ntt_status s = build_entry(e, key[0].plan->sm_count);
    if (s != NTT_OK) {
      free_entry(e);
      return s;
    }
    g_cache.push_front(std::move(e));
    it = g_cache.begin();
  } else if (it != g_cache.begin()) {
    g_cache.splice(g_cache.begin(), g_cache, it);
    it = g_cache.begin();
  }
  return cuda_status(cudaGraphLaunch(it->exec, (cudaStream_t)stream));
}

ntt_status ntt_batch_poll_error(uint32_t *code) {
  if (!code) return NTT_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NTT_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lk(g_mu);
  uint32_t *err = nullptr;
  ntt_status s = device_err_word(dev, &err);
  if (s != NTT_OK) return s;
  s = cuda_status(cudaDeviceSynchronize());
  if (s != NTT_OK) return s;
  s = cuda_status(cudaMemcpy(code, err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (s == NTT_OK) s = cuda_status(cudaMemset(err, 0, sizeof(uint32_t)));
  // the word of allocation-free calls made without a status pointer
  uint32_t scode = 0;
  if (s == NTT_OK) s = static_batch_take_error(dev, &scode);
  if (s == NTT_OK && !*code) *code = scode;
  return s;
}

ntt_status ntt_batch_set_wait_limit(uint64_t ns) {
  if (ns == 0) return NTT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  g_wait_ns = ns;
  clear_cache_locked();
  return NTT_OK;
}

ntt_status ntt_batch_debug_stall(int enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_stall = enable != 0;
  clear_cache_locked();
  return NTT_OK;
}

ntt_status ntt_batch_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  clear_cache_locked();
  static_batch_forget_addresses();
  return NTT_OK;
}

}  // extern "C"

namespace gb300ntt {

// Drop cached job lists that reference `plan` (called by ntt_plan_destroy).
void batch_forget_plan(ntt_plan plan) {
  std::lock_guard<std::mutex> lk(g_mu);
  bool any = false;
  for (const Entry &e : g_cache)
    for (const JobKey &k : e.key) any |= k.plan == plan;
  if (!any) return;
  cudaDeviceSynchronize();
  for (auto it = g_cache.begin(); it != g_cache.end();) {
    bool uses = false;
    for (const JobKey &k : it->key) uses |= k.plan == plan;
    if (uses) {
      free_entry(*it);
      it = g_cache.erase(it);
    } else {
      ++it;
    }
  }
}

}  // namespace gb300ntt
