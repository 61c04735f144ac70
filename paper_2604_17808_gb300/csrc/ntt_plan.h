// ntt_plan.h -- the plan object behind the C ABI's opaque ntt_plan.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <utility>
#include <vector>

#include "../../include/ntt_gb300.h"
#include "host_field.h"
#include "ntt_pass.cuh"

namespace gb300ntt {

enum Kind : int { kForward = 0, kInverse = 1, kCoset = 2, kCosetInverse = 3 };

// The coset inverse runs the inverse's passes (its tables index kInverse)
// and multiplies every output x_n by s^-n in the store of the last pass.
inline int table_kind(int kind) { return kind == kCosetInverse ? kInverse : kind; }
inline bool kind_is_valid(int kind, bool has_coset) {
  if (kind < kForward || kind > kCosetInverse) return false;
  return has_coset || (kind != kCoset && kind != kCosetInverse);
}

struct MatrixResources;  // tensor-core path (ntt_matrix.cu)

}  // namespace gb300ntt

struct ntt_plan_s {
  int device = 0;
  int field = 0;
  uint32_t log_n = 0;
  bool has_coset = false;
  ntt_path path = NTT_PATH_AUTO;
  int sm_count = 0;
  uint32_t num_passes = 0;
  uint32_t pass_log[gb300ntt::kMaxPasses] = {};
  uint32_t pass_tl[gb300ntt::kMaxPasses] = {};  // log2 tile size of each pass (10 or 11)
  uint32_t launches = 0;
  gb300ntt::U256 omega{}, omega_inv{}, coset_shift{};
  // device tables, Montgomery form, 32 bytes per entry
  uint4 *dft_tw[2][12] = {};     // [direction][log S]: omega_S^(+-i), i < S/2
  uint4 *tw[3][gb300ntt::kMaxPasses] = {};  // [kind][pass >= 1]: inter-pass multipliers [S_j][Mp]
  uint4 *pre[3] = {};            // [kind]: pass-0 multipliers [S_0] (coset; single-pass inverse)
  uint4 *fac_coset[gb300ntt::kMaxPasses] = {};  // [pass >= 1]: s^(n N / M_j), n < S_j
  uint4 *post_coset_inv = nullptr;  // s^-n, n < N: output multipliers of the coset inverse
  uint4 *scratch = nullptr;      // N elements (in-place transforms with > 1 pass)
  uint32_t *d_err = nullptr;     // device error word
  bool debug_shrink = false;     // debug builds: next transform with its vector extent halved
  std::vector<void *> allocations;
  uint64_t device_bytes = 0;
  gb300ntt::MatrixResources *matrix = nullptr;
  // per-pass launch timing (ntt_plan_enable_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;             // all events created for timing
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;  // (pass, start/stop)
  size_t ev_next = 0;
};

namespace gb300ntt {

// Resources of the matrix-form path (ntt_matrix.cu): a nested plan with
// passes of at most 2^3 points, the byte matrices E (fp16, B-operand
// layout) of its passes and their ByteMerge offsets.
struct MatrixResources {
  ntt_plan nested = nullptr;
  // [..][scaled]: scaled = 1 for passes ending in the 9-row Montgomery
  // product (E carries 2^32), 0 for a last pass reduced by Barrett
  uint4 *e_inner[2][4][2] = {};     // [direction][log S][scaled]: DFT matrix of passes >= 1
  uint32_t off_inner[2][4][2][8][8] = {};
  uint4 *e_first[3][2] = {};        // [table kind][scaled]: pass 0, its factors folded in
  uint32_t off_first[3][2][8][8] = {};
  // Folded passes 1..fold: all 128 rows of a tile share q, and the pass's
  // input factors c(q, n) are folded into one matrix E_q per q
  uint32_t fold = 0;
  uint4 *e_fold[3][kMaxPasses] = {};       // [table kind][pass]: Mp matrices E_q
  uint32_t *off_fold[3][kMaxPasses] = {};  // [table kind][pass]: Mp x S offsets (8 words each)
  uint32_t one[8] = {};             // 2^256 mod p
  uint64_t mu = 0;                  // floor(2^288 / p)
  uint32_t *err = nullptr;          // device error word of matrix launches
};

std::vector<uint32_t> split_passes(uint32_t log_n);
std::vector<uint32_t> split_passes_max(uint32_t log_n, uint32_t max_log);
// Build tables and scratch of plan p (fields device, field, log_n,
// has_coset, sm_count set) for the given pass split (nullptr = default).
ntt_status build_plan(ntt_plan p, cudaStream_t st, const std::vector<uint32_t> *forced_split);
uint64_t pass_tiles(uint32_t log_n, uint32_t logs, uint32_t tl);
ntt_status enqueue_transform(ntt_plan p, int kind, const void *in, void *out, cudaStream_t st);
ntt_status cuda_status(cudaError_t e);
struct PassArgs;
void build_pass_args(ntt_plan p, int kind, const void *in, void *out, uint32_t j, PassArgs *a, int *mode);
ntt_status check_buffer(const void *ptr);
// Timing hooks around one launch of pass `pass` (no-ops unless timing is on).
cudaError_t timing_begin(ntt_plan p, int pass, cudaStream_t st);
cudaError_t timing_end(ntt_plan p, cudaStream_t st);

ntt_status build_coset_tables(ntt_plan p, const U256 &s, cudaStream_t st);
// Free all device tables of p and null their pointers (see ntt_plan.cu).
void release_plan_tables(ntt_plan p);

// matrix (tensor-core) path, ntt_matrix.cu
bool matrix_path_available(ntt_plan p);
ntt_status prepare_matrix_path(ntt_plan p);
ntt_status matrix_build_coset(ntt_plan p);  // after a coset-shift change
ntt_status matrix_poll_error(ntt_plan p, uint32_t *code);
ntt_status enqueue_matrix_transform(ntt_plan p, int kind, const void *in, void *out, cudaStream_t st);
uint32_t matrix_launches(ntt_plan p);
void release_matrix_resources(ntt_plan p);

// autotuner, ntt_tune.cu
struct TuneChoice {
  int path = 1;                  // NTT_PATH_BUTTERFLY or NTT_PATH_MATRIX
  std::vector<uint32_t> split;   // butterfly pass sizes (log2)
  uint32_t tile_log = 10;        // 10 or 11 (butterfly)
  double ms = 0;
};

bool tune_lookup(int dev, int field, uint32_t log_n, TuneChoice *out);
ntt_status tune_apply(ntt_plan p, const TuneChoice &c);

// batched path, ntt_batch.cu
void batch_forget_plan(ntt_plan plan);
struct BatchSeg;
struct BatchJobRef {
  ntt_plan plan;
  int32_t kind;
  const void *in;
  void *out;
};
std::vector<BatchSeg> build_segments(const std::vector<BatchJobRef> &jobs, int field, uint32_t *total_items);
uint64_t batch_wait_limit_ns();
bool batch_debug_stall();  // the ntt_batch_debug_stall test hook is on
ntt_status batch_error_word(uint32_t **out);
// allocation-free batch (ntt_batch_static.cu)
ntt_status static_batch_take_error(int dev, uint32_t *code);
void static_batch_forget_addresses();

}  // namespace gb300ntt
