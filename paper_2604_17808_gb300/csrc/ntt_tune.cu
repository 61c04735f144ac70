// ntt_tune.cu -- the autotuner: pick the pass split, tile shape and path of
// a plan by timing candidates on the device.
//
// Candidates for N = 2^log_n:
//   * butterfly path: balanced splits for every maximum pass size 2^4..2^11
//     (distinct ones), each also with its passes in reverse order, each with
//     the 1024-element tile (7 CTAs/SM) or the 2048-element tile (3 CTAs/SM);
//   * matrix path (tensor-core passes of at most 2^3 points).
// Each candidate builds its own tables, runs one untimed forward transform,
// then `reps` timed ones (CUDA events); the fastest wins and the plan is
// rebuilt with it.  Results are cached per (GPU name, SM count, field,
// log_n) in memory and, when the environment variable NTT_TUNE_CACHE names
// a file, in that file (one line per entry), which ntt_plan_create reads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "ntt_launch.h"
#include "ntt_plan.h"
#include "nvtx_range.h"

using namespace gb300ntt;

namespace gb300ntt {

namespace {

std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;
bool g_tune_loaded = false;

std::string device_key(int dev) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  std::string name = prop.name;
  for (char &c : name)
    if (c == ' ' || c == '|') c = '_';
  return name + "|" + std::to_string(prop.multiProcessorCount);
}

std::string entry_key(int dev, int field, uint32_t log_n) {
  return device_key(dev) + "|" + std::to_string(field) + "|" + std::to_string(log_n);
}

// File format, one entry per line:
//   <device>|<sms>|<field>|<log_n> <path> <tile_log> <ms> <P> <s_0> ... <s_P-1>
void load_file_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *path = std::getenv("NTT_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = std::fopen(path, "r");
  if (!f) return;
  char key[256];
  TuneChoice c;
  unsigned P = 0;
  while (std::fscanf(f, "%255s %d %u %lf %u", key, &c.path, &c.tile_log, &c.ms, &P) == 5) {
    c.split.assign(P, 0);
    bool ok = P >= 1 && P <= (unsigned)kMaxPasses;
    for (unsigned i = 0; i < P && ok; ++i) ok = std::fscanf(f, "%u", &c.split[i]) == 1;
    if (!ok) break;
    g_tune_cache[key] = c;
  }
  std::fclose(f);
}

void save_file_locked() {
  const char *path = std::getenv("NTT_TUNE_CACHE");
  if (!path || !*path) return;
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  for (const auto &kv : g_tune_cache) {
    const TuneChoice &c = kv.second;
    std::fprintf(f, "%s %d %u %.6f %zu", kv.first.c_str(), c.path, c.tile_log, c.ms, c.split.size());
    for (uint32_t s : c.split) std::fprintf(f, " %u", s);
    std::fprintf(f, "\n");
  }
  std::fclose(f);
  std::rename(tmp.c_str(), path);
}

void free_plan_memory(ntt_plan p) {
  release_matrix_resources(p);
  release_plan_tables(p);
}

// (Re)build plan p's tables for a butterfly choice.
ntt_status apply_butterfly(ntt_plan p, const std::vector<uint32_t> &split, uint32_t tile_log, cudaStream_t st) {
  batch_forget_plan(p);  // cached batch graphs point at the old tables
  cudaDeviceSynchronize();
  const U256 shift = p->coset_shift;
  free_plan_memory(p);
  ntt_status s = build_plan(p, st, &split);
  if (s == NTT_OK && p->has_coset && !u256_is_zero(shift)) s = build_coset_tables(p, shift, st);
  if (s != NTT_OK) return s;
  for (uint32_t j = 0; j < p->num_passes; ++j) p->pass_tl[j] = p->pass_log[j] <= 10 ? tile_log : 11;
  return cuda_status(cudaStreamSynchronize(st));
}

std::vector<std::pair<std::vector<uint32_t>, uint32_t>> butterfly_candidates(uint32_t log_n) {
  std::vector<std::vector<uint32_t>> splits;
  for (uint32_t mx = 4; mx <= 11; ++mx) {
    if (mx > log_n && mx != 4) continue;
    std::vector<uint32_t> s = split_passes_max(log_n, mx);
    if ((int)s.size() > kMaxPasses) continue;
    std::vector<uint32_t> r(s.rbegin(), s.rend());
    for (const auto &c : {s, r})
      if (std::find(splits.begin(), splits.end(), c) == splits.end()) splits.push_back(c);
  }
  std::vector<std::pair<std::vector<uint32_t>, uint32_t>> out;
  for (const auto &s : splits) {
    const bool any_le10 = std::any_of(s.begin(), s.end(), [](uint32_t x) { return x <= 10; });
    out.push_back({s, 11});
    if (any_le10) out.push_back({s, 10});
  }
  return out;
}

double time_forward(ntt_plan p, const void *in, void *out, int reps, cudaStream_t st) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  ntt_execute(p, NTT_KIND_FORWARD, in, out, (ntt_stream)st);
  cudaEventRecord(a, st);
  for (int i = 0; i < reps; ++i) ntt_execute(p, NTT_KIND_FORWARD, in, out, (ntt_stream)st);
  cudaEventRecord(b, st);
  float ms = 0;
  const bool ok = cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ok ? ms / reps : 1e30;
}

}  // namespace

// Cached choice for a new plan, if any (called by ntt_plan_create).
bool tune_lookup(int dev, int field, uint32_t log_n, TuneChoice *out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  load_file_locked();
  auto it = g_tune_cache.find(entry_key(dev, field, log_n));
  if (it == g_tune_cache.end()) return false;
  *out = it->second;
  return true;
}

ntt_status tune_apply(ntt_plan p, const TuneChoice &c) {
  cudaStream_t st = nullptr;
  ntt_status s = cuda_status(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  if (s != NTT_OK) return s;
  if (!c.split.empty()) s = apply_butterfly(p, c.split, c.tile_log, st);
  cudaStreamDestroy(st);
  if (s == NTT_OK) s = ntt_plan_set_path(p, c.path == NTT_PATH_MATRIX ? NTT_PATH_MATRIX : NTT_PATH_BUTTERFLY);
  return s;
}

}  // namespace gb300ntt

extern "C" ntt_status ntt_plan_autotune(ntt_plan plan, uint32_t reps, ntt_tune_result *result) {
  NvtxRange range("ntt_plan_autotune");
  if (!plan) return NTT_ERR_INVALID_ARG;
  if (reps == 0) reps = 3;
  const uint32_t log_n = plan->log_n;
  const uint64_t bytes = 32ull << log_n;
  void *in = nullptr, *out = nullptr;
  ntt_status s = cuda_status(cudaMalloc(&in, bytes));
  if (s == NTT_OK) s = cuda_status(cudaMalloc(&out, bytes));
  if (s == NTT_OK) s = cuda_status(cudaMemset(in, 0, bytes));  // zeros are canonical
  cudaStream_t st = nullptr;
  if (s == NTT_OK) s = cuda_status(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  TuneChoice best;
  best.ms = 1e30;
  double default_ms = 0;
  uint32_t tried = 0;
  if (s == NTT_OK) {
    plan->path = NTT_PATH_BUTTERFLY;
    default_ms = time_forward(plan, in, out, (int)reps, st);
    for (const auto &cand : butterfly_candidates(log_n)) {
      s = apply_butterfly(plan, cand.first, cand.second, st);
      if (s != NTT_OK) break;
      const double ms = time_forward(plan, in, out, (int)reps, st);
      ++tried;
      if (ms < best.ms) {
        best.ms = ms;
        best.path = NTT_PATH_BUTTERFLY;
        best.split = cand.first;
        best.tile_log = cand.second;
      }
    }
  }
  if (s == NTT_OK && matrix_path_available(plan)) {
    s = ntt_plan_set_path(plan, NTT_PATH_MATRIX);
    if (s == NTT_OK) {
      const double ms = time_forward(plan, in, out, (int)reps, st);
      ++tried;
      if (ms < best.ms) {
        best.ms = ms;
        best.path = NTT_PATH_MATRIX;
      }
      plan->path = NTT_PATH_BUTTERFLY;
    }
  }
  if (s == NTT_OK) {
    TuneChoice apply = best;
    if (best.path == NTT_PATH_MATRIX) apply.split = split_passes(log_n), apply.tile_log = 10;
    s = tune_apply(plan, apply);
    if (s == NTT_OK) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      load_file_locked();
      g_tune_cache[entry_key(plan->device, plan->field, log_n)] = apply.path == NTT_PATH_MATRIX ? best : apply;
      save_file_locked();
    }
  }
  if (st) cudaStreamDestroy(st);
  if (in) cudaFree(in);
  if (out) cudaFree(out);
  if (s == NTT_OK && result) {
    std::memset(result, 0, sizeof *result);
    result->path = (uint32_t)plan->path;
    result->num_passes = plan->num_passes;
    for (uint32_t j = 0; j < plan->num_passes && j < NTT_MAX_PASSES; ++j) {
      result->pass_log[j] = plan->pass_log[j];
      result->tile_log[j] = plan->pass_tl[j];
    }
    result->best_ms = best.ms;
    result->default_ms = default_ms;
    result->candidates = tried;
  }
  return s;
}

extern "C" ntt_status ntt_plan_set_passes(ntt_plan plan, uint32_t num_passes, const uint32_t *pass_log,
                                          uint32_t tile_log) {
  if (!plan || !pass_log) return NTT_ERR_INVALID_ARG;
  if (num_passes < 1 || num_passes > (uint32_t)kMaxPasses) return NTT_ERR_INVALID_ARG;
  if (tile_log != 10 && tile_log != 11) return NTT_ERR_INVALID_ARG;
  std::vector<uint32_t> split(pass_log, pass_log + num_passes);
  uint32_t sum = 0;
  for (uint32_t s : split) {
    if (s < 1 || s > (uint32_t)kMaxPassLog) return NTT_ERR_INVALID_ARG;
    sum += s;
  }
  if (sum != plan->log_n) return NTT_ERR_INVALID_ARG;
  cudaStream_t st = nullptr;
  ntt_status s = cuda_status(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  if (s != NTT_OK) return s;
  s = apply_butterfly(plan, split, tile_log, st);
  cudaStreamDestroy(st);
  if (s == NTT_OK) plan->path = NTT_PATH_BUTTERFLY;
  return s;
}
