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
//
// A batch policy (chosen by ntt_batch_autotune per job-list signature: the
// multiset of (field, size, kind, path) of its jobs) may take the larger jobs
// out of the persistent kernel: jobs of 2^split_log points and more (and
// every job whose plan is on the matrix path) then run as ordinary
// transforms, each on its plan's own (tuned) path, spread over parallel
// branches of the same graph, concurrently with the persistent kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "ntt_launch.h"
#include "ntt_plan.h"
#include "nvtx_range.h"

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

// How a job list is run: jobs of 2^split_log points and more (and matrix-path
// jobs) as individual transforms over `branches` parallel graph branches,
// the rest in the persistent kernel.  split_log = kNoSplit: all in the
// persistent kernel (matrix-path jobs still individually).
constexpr uint32_t kNoSplit = 64;
struct Policy {
  uint32_t split_log = kNoSplit;
  uint32_t branches = 1;
  double ms = 0;
  bool operator==(const Policy &o) const { return split_log == o.split_log && branches == o.branches; }
};

struct Entry {
  std::vector<JobKey> key;
  Policy policy;
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
std::map<std::string, Policy> g_policy;   // job-list signature -> tuned policy
bool g_policy_loaded = false;

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

bool runs_alone(const JobKey &j, const Policy &pol) {
  return j.plan->path == NTT_PATH_MATRIX || j.plan->log_n >= pol.split_log;
}

std::string signature(int dev, const std::vector<JobKey> &key) {
  std::vector<std::string> items;
  for (const JobKey &j : key) {
    char buf[64];
    std::snprintf(buf, sizeof buf, "%d.%u.%d.%d", j.plan->field, j.plan->log_n, j.kind, (int)j.plan->path);
    items.push_back(buf);
  }
  std::sort(items.begin(), items.end());
  std::string sig = std::to_string(dev) + ":";
  for (const std::string &it : items) sig += it + ",";
  return sig;
}

// Policies persist in "<NTT_TUNE_CACHE>.batch", one "<signature> <split_log>
// <branches> <ms>" line each (the device is the process's device index).
std::string policy_file() {
  const char *path = std::getenv("NTT_TUNE_CACHE");
  return (path && *path) ? std::string(path) + ".batch" : std::string();
}

void load_policies_locked() {
  if (g_policy_loaded) return;
  g_policy_loaded = true;
  const std::string path = policy_file();
  if (path.empty()) return;
  FILE *f = std::fopen(path.c_str(), "r");
  if (!f) return;
  static char sig[1 << 16];
  Policy pol;
  while (std::fscanf(f, "%65535s %u %u %lf", sig, &pol.split_log, &pol.branches, &pol.ms) == 4) {
    if (pol.branches >= 1 && pol.branches <= 8) g_policy[sig] = pol;
  }
  std::fclose(f);
}

void save_policies_locked() {
  const std::string path = policy_file();
  if (path.empty()) return;
  const std::string tmp = path + ".tmp";
  FILE *f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  for (const auto &kv : g_policy)
    std::fprintf(f, "%s %u %u %.6f\n", kv.first.c_str(), kv.second.split_log, kv.second.branches, kv.second.ms);
  std::fclose(f);
  std::rename(tmp.c_str(), path.c_str());
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
ntt_status build_part(const std::vector<JobKey> &jobs, const Policy &pol, int field, Part *part) {
  std::vector<BatchJobRef> refs;
  for (const JobKey &j : jobs)
    if (!runs_alone(j, pol)) refs.push_back(BatchJobRef{j.plan, j.kind, j.in, j.out});
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
    for (const JobKey &j : e.key) any |= j.plan->field == field && !runs_alone(j, e.policy);
    if (!any) continue;
    Part part;
    st = build_part(e.key, e.policy, field, &part);
    e.parts.push_back(part);
    if (st != NTT_OK) return st;
  }
  // individual jobs, larger first, dealt round-robin over the branches
  std::vector<size_t> alone;
  for (size_t i = 0; i < e.key.size(); ++i)
    if (runs_alone(e.key[i], e.policy)) alone.push_back(i);
  std::stable_sort(alone.begin(), alone.end(),
                   [&](size_t a, size_t b) { return e.key[a].plan->log_n > e.key[b].plan->log_n; });
  const uint32_t nb = alone.empty() ? 0 : std::min<uint32_t>(e.policy.branches, (uint32_t)alone.size());
  cudaStream_t cs = nullptr;
  std::vector<cudaStream_t> bs(nb, nullptr);
  std::vector<cudaEvent_t> ev(1 + nb, nullptr);
  st = cuda_status(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  for (uint32_t b = 0; st == NTT_OK && b < nb; ++b) st = cuda_status(cudaStreamCreateWithFlags(&bs[b], cudaStreamNonBlocking));
  for (size_t k = 0; st == NTT_OK && k < ev.size(); ++k)
    st = cuda_status(cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming));
  if (st == NTT_OK) st = cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  if (st == NTT_OK) {
    // fork: the branches start with the graph
    if (nb) cudaEventRecord(ev[0], cs);
    for (uint32_t b = 0; b < nb; ++b) cudaStreamWaitEvent(bs[b], ev[0], 0);
    for (size_t k = 0; k < alone.size() && st == NTT_OK; ++k) {
      const JobKey &j = e.key[alone[k]];
      st = ntt_execute(j.plan, (ntt_kind)j.kind, j.in, j.out, (ntt_stream)bs[k % nb]);
    }
    for (const Part &part : e.parts) {
      if (!part.total_items || st != NTT_OK) continue;
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
    // join
    for (uint32_t b = 0; b < nb; ++b) {
      cudaEventRecord(ev[1 + b], bs[b]);
      cudaStreamWaitEvent(cs, ev[1 + b], 0);
    }
    const cudaError_t ce = cudaStreamEndCapture(cs, &e.graph);
    if (st == NTT_OK) st = cuda_status(ce);
    if (st == NTT_OK) st = cuda_status(cudaGraphInstantiate(&e.exec, e.graph, 0));
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  for (cudaStream_t x : bs)
    if (x) cudaStreamDestroy(x);
  if (cs) cudaStreamDestroy(cs);
  return st;
}

// Run job list `key` under `pol` on `stream` (cached graph, built on first use).
ntt_status submit_locked(const std::vector<JobKey> &key, const Policy &pol, cudaStream_t stream) {
  int dev = 0;
  cudaGetDevice(&dev);
  auto it = std::find_if(g_cache.begin(), g_cache.end(),
                         [&](const Entry &e) { return e.device == dev && e.key == key && e.policy == pol; });
  if (it == g_cache.end()) {
    if (g_cache.size() >= kCacheEntries) {
      cudaDeviceSynchronize();
      free_entry(g_cache.back());
      g_cache.pop_back();
    }
    Entry e;
    e.key = key;
    e.policy = pol;
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
  return cuda_status(cudaGraphLaunch(it->exec, stream));
}

ntt_status make_key(const ntt_job *jobs, size_t n, std::vector<JobKey> *key) {
  key->resize(n);
  for (size_t i = 0; i < n; ++i) {
    const ntt_job &j = jobs[i];
    if (!j.plan || j.in == j.out) return NTT_ERR_INVALID_ARG;
    if (!kind_is_valid(j.kind, j.plan->has_coset)) return NTT_ERR_INVALID_ARG;
    ntt_status s = check_buffer(j.in);
    if (s == NTT_OK) s = check_buffer(j.out);
    if (s != NTT_OK) return s;
    (*key)[i] = JobKey{j.plan, j.kind, j.in, j.out};
  }
  return NTT_OK;
}

}  // namespace

extern "C" {

ntt_status ntt_batch_submit(const ntt_job *jobs, size_t n, ntt_stream stream) {
  NvtxRange range("ntt_batch_submit");
  if (!jobs && n) return NTT_ERR_INVALID_ARG;
  if (n == 0) return NTT_OK;
  std::vector<JobKey> key;
  ntt_status s = make_key(jobs, n, &key);
  if (s != NTT_OK) return s;
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  load_policies_locked();
  Policy pol;
  auto pit = g_policy.find(signature(dev, key));
  if (pit != g_policy.end()) pol = pit->second;
  return submit_locked(key, pol, (cudaStream_t)stream);
}

ntt_status ntt_batch_autotune(const ntt_job *jobs, size_t n, uint32_t reps, ntt_batch_tune_result *result) {
  NvtxRange range("ntt_batch_autotune");
  if (!jobs || n == 0) return NTT_ERR_INVALID_ARG;
  if (reps == 0) reps = 3;
  std::vector<JobKey> key;
  ntt_status s = make_key(jobs, n, &key);
  if (s != NTT_OK) return s;
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  load_policies_locked();
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  s = cuda_status(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  if (s == NTT_OK) s = cuda_status(cudaEventCreate(&a));
  if (s == NTT_OK) s = cuda_status(cudaEventCreate(&b));
  // candidates: everything in the persistent kernel; jobs of 2^t points and
  // more alone, for every distinct size t of the list, over 1, 2 or 4 branches
  std::vector<Policy> cands(1);
  std::vector<uint32_t> sizes;
  for (const JobKey &j : key) sizes.push_back(j.plan->log_n);
  std::sort(sizes.begin(), sizes.end());
  sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
  for (uint32_t t : sizes)
    for (uint32_t br : {1u, 2u, 4u}) {
      Policy p;
      p.split_log = t;
      p.branches = br;
      cands.push_back(p);
    }
  Policy best;
  best.ms = 1e30;
  double persistent_ms = 0, loop_ms = 0;
  uint32_t tried = 0;
  auto time_it = [&](auto &&run) -> double {
    ntt_status r = run();   // warm-up (builds the graph)
    if (r != NTT_OK) return -1;
    cudaEventRecord(a, st);
    for (uint32_t i = 0; i < reps; ++i) run();
    cudaEventRecord(b, st);
    float ms = 0;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return -1;
    return (double)ms / reps;
  };
  if (s == NTT_OK) {
    loop_ms = time_it([&]() {
      ntt_status r = NTT_OK;
      for (const JobKey &j : key)
        if (r == NTT_OK) r = ntt_execute(j.plan, (ntt_kind)j.kind, j.in, j.out, (ntt_stream)st);
      return r;
    });
    for (const Policy &c : cands) {
      const double ms = time_it([&]() { return submit_locked(key, c, st); });
      if (ms < 0) {
        s = NTT_ERR_CUDA;
        break;
      }
      ++tried;
      if (c.split_log == kNoSplit) persistent_ms = ms;
      if (ms < best.ms) {
        best = c;
        best.ms = ms;
      }
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  // drop the candidates' graphs of this list; keep the winner's policy
  cudaDeviceSynchronize();
  for (auto it = g_cache.begin(); it != g_cache.end();) {
    if (it->key == key && !(it->policy == best)) {
      free_entry(*it);
      it = g_cache.erase(it);
    } else {
      ++it;
    }
  }
  if (s != NTT_OK) return s;
  g_policy[signature(dev, key)] = best;
  save_policies_locked();
  if (result) {
    result->split_log = best.split_log == kNoSplit ? 0 : best.split_log;
    result->branches = best.split_log == kNoSplit ? 0 : best.branches;
    result->candidates = tried;
    result->best_ms = best.ms;
    result->persistent_ms = persistent_ms;
    result->loop_ms = loop_ms;
  }
  return NTT_OK;
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
  g_policy.clear();
  g_policy_loaded = false;
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
