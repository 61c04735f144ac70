// ntt_plan.cu -- plans, resident twiddle tables and the C ABI.
//
// A plan fixes (field, log_n), splits N into passes of at most 2^8 points
// (the four-step / six-step decomposition of ntt_pass.cuh), and builds on
// the device every constant the passes multiply by, in Montgomery form:
//   * per distinct pass size S: omega_S^i and omega_S^-i, i < S/2;
//   * per pass j >= 1 and kind: the inter-pass table omega_M^(n q) [S_j][Mp]
//     (inverse: omega^-1 and, in the last pass, N^-1; coset: times
//     s^(n * N/M) for the digit the pass transforms);
//   * pass 0 multipliers for coset (s^(n N/S_0)) and, for single-pass
//     plans, the inverse scale N^-1.
// The paper precomputes its twiddle matrices (Fig. 5); here they are
// generated once per plan by kernels and stay in HBM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <utility>
#include <vector>

#include "../../include/ntt_gb300.h"
#include "host_field.h"
#include "ntt_launch.h"
#include "ntt_matrix.cuh"
#include "ntt_plan.h"
#include "nvtx_range.h"

using namespace gb300ntt;

namespace gb300ntt {

namespace {

Fe32 to_fe32(const U256 &a) {
  Fe32 r;
  for (int i = 0; i < 4; ++i) {
    r.w[2 * i] = (uint32_t)a.w[i];
    r.w[2 * i + 1] = (uint32_t)(a.w[i] >> 32);
  }
  return r;
}

U256 from_limbs(const uint64_t *l) { return U256{{l[0], l[1], l[2], l[3]}}; }

Pow2Table make_ladder(const HostField &F, const U256 &base) {
  Pow2Table t;
  U256 b = base;
  for (int i = 0; i < 32; ++i) {
    t.v[i] = to_fe32(F.to_mont(b));
    b = F.mul(b, b);
  }
  return t;
}

// omega^(2^k)
U256 square_times(const HostField &F, U256 a, unsigned k) {
  for (unsigned i = 0; i < k; ++i) a = F.mul(a, a);
  return a;
}

std::mutex g_prep_mu;
std::set<std::pair<int, int>> g_prepared;  // (device, field)

ntt_status prepare_device(int device, int field) {
  std::lock_guard<std::mutex> lk(g_prep_mu);
  if (g_prepared.count({device, field})) return NTT_OK;
  if (launchers(field).prepare() != cudaSuccess) return NTT_ERR_CUDA;
  g_prepared.insert({device, field});
  return NTT_OK;
}

}  // namespace

ntt_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return NTT_OK;
  if (e == cudaErrorMemoryAllocation) return NTT_ERR_OOM;
  return NTT_ERR_CUDA;
}

// Default split of log_n into passes of at most kDefaultPassLog bits, as
// equal as possible, larger ones first.  (Sub-transforms of up to 2^10
// points keep at least two per tile, so the strided reads of a pass still
// touch two adjacent elements; the autotuner may pick other splits.)
constexpr uint32_t kDefaultPassLog = 10;

std::vector<uint32_t> split_passes(uint32_t log_n) {
  const uint32_t P = (log_n + kDefaultPassLog - 1) / kDefaultPassLog;
  std::vector<uint32_t> s(P, log_n / P);
  for (uint32_t i = 0; i < log_n % P; ++i) s[i] += 1;
  return s;
}

uint64_t pass_tiles(uint32_t log_n, uint32_t logs, uint32_t tl) {
  const uint64_t num_sub = 1ull << (log_n - logs);
  const uint64_t g = 1ull << (tl - logs);
  return (num_sub + g - 1) / g;
}

// Default tile shape of a pass: the 1024-element tile (7 CTAs per SM) when
// the sub-transform fits in it, else the 2048-element tile.
uint32_t default_tile_log(uint32_t logs) { return logs <= 10 ? 10 : 11; }

// Balanced split of log_n into passes of at most max_log bits, larger first.
std::vector<uint32_t> split_passes_max(uint32_t log_n, uint32_t max_log) {
  const uint32_t P = (log_n + max_log - 1) / max_log;
  std::vector<uint32_t> s(P, log_n / P);
  for (uint32_t i = 0; i < log_n % P; ++i) s[i] += 1;
  return s;
}

static ntt_status alloc_tab(ntt_plan p, uint4 **out, uint64_t elems) {
  void *ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, elems * 32);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  p->allocations.push_back(ptr);
  p->device_bytes += elems * 32;
  *out = (uint4 *)ptr;
  return NTT_OK;
}

// Free every device table of plan p and clear every pointer to one (the
// plan keeps its device, field, size and error word), so that build_plan
// can run again.  Every table allocated by alloc_tab must be listed here.
void release_plan_tables(ntt_plan p) {
  for (void *ptr : p->allocations) cudaFree(ptr);
  p->allocations.clear();
  p->device_bytes = 0;
  std::memset(p->dft_tw, 0, sizeof p->dft_tw);
  std::memset(p->tw, 0, sizeof p->tw);
  std::memset(p->pre, 0, sizeof p->pre);
  std::memset(p->fac_coset, 0, sizeof p->fac_coset);
  p->post_coset_inv = nullptr;
  p->scratch = nullptr;
}

#define NTT_TRY(expr)                  \
  do {                                 \
    ntt_status _s = (expr);            \
    if (_s != NTT_OK) return _s;       \
  } while (0)

#define NTT_CUDA(expr) NTT_TRY(cuda_status(expr))

// (Re)build the coset tables for shift s (standard form).
ntt_status build_coset_tables(ntt_plan p, const U256 &s, cudaStream_t st) {
  const HostField F = host_field(p->field);
  const FieldLaunchers &L = launchers(p->field);
  const uint32_t log_n = p->log_n, P = p->num_passes;
  const Fe32 one = to_fe32(F.to_mont(u256(1)));
  uint32_t log_m = 0;
  for (uint32_t j = 0; j < P; ++j) {
    const uint32_t logs = p->pass_log[j];
    log_m += logs;
    // s^(N/M_j): the coset factor of one step of digit j
    const U256 step = F.pow(s, 1ull << (log_n - log_m));
    if (j == 0) {
      if (!p->pre[kCoset]) NTT_TRY(alloc_tab(p, &p->pre[kCoset], 1ull << logs));
      NTT_CUDA(L.gen_1d(p->pre[kCoset], 1ull << logs, make_ladder(F, step), one, st));
    } else {
      if (!p->fac_coset[j]) NTT_TRY(alloc_tab(p, &p->fac_coset[j], 1ull << logs));
      NTT_CUDA(L.gen_1d(p->fac_coset[j], 1ull << logs, make_ladder(F, step), one, st));
      const uint32_t log_mp = log_m - logs;
      const U256 w = square_times(F, p->omega, log_n - log_m);
      if (!p->tw[kCoset][j]) NTT_TRY(alloc_tab(p, &p->tw[kCoset][j], 1ull << log_m));
      NTT_CUDA(L.gen_2d(p->tw[kCoset][j], logs, log_mp, make_ladder(F, w), p->fac_coset[j], one, st));
    }
  }
  // coset inverse: x_n *= s^-n on the output of the last pass
  if (!p->post_coset_inv) NTT_TRY(alloc_tab(p, &p->post_coset_inv, 1ull << log_n));
  NTT_CUDA(L.gen_1d(p->post_coset_inv, 1ull << log_n, make_ladder(F, F.inv(s)), one, st));
  p->coset_shift = s;
  return NTT_OK;
}

ntt_status build_plan(ntt_plan p, cudaStream_t st, const std::vector<uint32_t> *forced_split) {
  const HostField F = host_field(p->field);
  const FieldLaunchers &L = launchers(p->field);
  const uint32_t log_n = p->log_n;
  const std::vector<uint32_t> passes = forced_split ? *forced_split : split_passes(log_n);
  if (passes.empty() || passes.size() > (size_t)kMaxPasses) return NTT_ERR_UNSUPPORTED;
  p->num_passes = (uint32_t)passes.size();
  for (uint32_t j = 0; j < p->num_passes; ++j) {
    p->pass_log[j] = passes[j];
    p->pass_tl[j] = default_tile_log(passes[j]);
  }
  const uint32_t P = p->num_passes;

  p->omega = F.root_of_unity(log_n);
  p->omega_inv = F.inv(p->omega);
  const U256 n_inv = F.inv(F.reduce_small(1ull << log_n));
  const Fe32 one = to_fe32(F.to_mont(u256(1)));
  const Fe32 n_inv_m = to_fe32(F.to_mont(n_inv));

  // DFT twiddles per distinct pass size
  for (uint32_t j = 0; j < P; ++j) {
    const uint32_t logs = passes[j];
    for (int dir = 0; dir < 2; ++dir) {
      if (p->dft_tw[dir][logs]) continue;
      const U256 w = square_times(F, dir ? p->omega_inv : p->omega, log_n - logs);
      const uint64_t count = std::max<uint64_t>(1, (1ull << logs) / 2);
      NTT_TRY(alloc_tab(p, &p->dft_tw[dir][logs], count));
      NTT_CUDA(L.gen_1d(p->dft_tw[dir][logs], count, make_ladder(F, w), one, st));
    }
  }
  // inter-pass tables (forward, inverse)
  uint32_t log_m = passes[0];
  for (uint32_t j = 1; j < P; ++j) {
    const uint32_t logs = passes[j];
    const uint32_t log_mp = log_m;
    log_m += logs;
    for (int dir = 0; dir < 2; ++dir) {
      const U256 w = square_times(F, dir ? p->omega_inv : p->omega, log_n - log_m);
      const Fe32 init = (dir == 1 && j == P - 1) ? n_inv_m : one;
      NTT_TRY(alloc_tab(p, &p->tw[dir][j], 1ull << log_m));
      NTT_CUDA(L.gen_2d(p->tw[dir][j], logs, log_mp, make_ladder(F, w), nullptr, init, st));
    }
  }
  // single-pass inverse: N^-1 as a pass-0 multiplier
  if (P == 1) {
    NTT_TRY(alloc_tab(p, &p->pre[kInverse], 1ull << passes[0]));
    NTT_CUDA(L.gen_1d(p->pre[kInverse], 1ull << passes[0], make_ladder(F, u256(1)), n_inv_m, st));
  }
  if (p->has_coset) NTT_TRY(build_coset_tables(p, F.reduce_small(F.generator), st));
  if (P > 1) NTT_TRY(alloc_tab(p, &p->scratch, 1ull << log_n));
  p->launches = P;
  return NTT_OK;
}

// Arguments of pass j of one transform: pass 0 reads `in`; every later pass
// works in place on `work` (out, or the plan's scratch for in-place calls);
// the last pass writes `out`.
void build_pass_args(ntt_plan p, int kind, const void *in, void *out, uint32_t j, PassArgs *a, int *mode) {
  const uint32_t P = p->num_passes, log_n = p->log_n;
  const int tk = table_kind(kind);
  const int dir = tk == kInverse ? 1 : 0;
  uint4 *work = (P > 1 && in == out) ? p->scratch : (uint4 *)out;
  const uint32_t logs = p->pass_log[j];
  *a = PassArgs{};
  a->dft_tw = p->dft_tw[dir][logs];
  a->num_sub = 1ull << (log_n - logs);
  if (j == 0) {
    a->src = (const uint4 *)in;
    a->dst = P == 1 ? (uint4 *)out : work;
    a->log_mp = log_n - logs;
    a->num_digits = P - 1;
    uint32_t shift = 0;
    for (uint32_t d = 1; d < P; ++d) {
      a->digit_log[d - 1] = (uint8_t)p->pass_log[d];
      a->digit_shift[d - 1] = (uint8_t)shift;
      shift += p->pass_log[d];
    }
    a->mul = p->pre[tk];
    *mode = a->mul ? kModeFirstPre : kModeFirst;
  } else {
    uint32_t log_mp = 0;
    for (uint32_t i = 0; i < j; ++i) log_mp += p->pass_log[i];
    a->src = work;
    a->dst = j == P - 1 ? (uint4 *)out : work;
    a->log_mp = log_mp;
    a->mul = p->tw[tk][j];
    *mode = kModeInner;
  }
  if (kind == kCosetInverse && j == P - 1) a->post = p->post_coset_inv;
  // extents for the bounds checks of debug builds
  a->n_vec = 1ull << log_n;
  if (j == 0) {
    a->n_mul = a->mul ? (1ull << logs) : 0;
  } else {
    a->n_mul = 1ull << (a->log_mp + logs);
  }
  a->dbg_err = p->d_err;
}

// Tile structure of a pass: the fused tile when the pass is one wave of
// 1024-element tiles (every CTA resident at once, 7 per SM), the staged
// tile otherwise (see pass_tile in ntt_pass.cuh for the measurements).
bool use_fused_tile(ntt_plan p, uint32_t logs, uint32_t tl) {
  return tl == 10 && logs >= 4 &&
         pass_tiles(p->log_n, logs, tl) <= (uint64_t)p->sm_count * (uint64_t)TileCfg<10>::kMinBlocks;
}

// Enqueue one transform: one kernel launch per pass.
ntt_status enqueue_transform(ntt_plan p, int kind, const void *in, void *out, cudaStream_t st) {
  const FieldLaunchers &L = launchers(p->field);
  const bool shrink = p->debug_shrink;   // debug-build test hook (see ntt_debug_shrink_next_extent)
  p->debug_shrink = false;
  for (uint32_t j = 0; j < p->num_passes; ++j) {
    PassArgs a;
    int mode;
    build_pass_args(p, kind, in, out, j, &a, &mode);
    if (shrink) a.n_vec >>= 1;
    const uint32_t logs = p->pass_log[j];
    cudaError_t e = timing_begin(p, (int)j, st);
    const uint32_t tl = p->pass_tl[j];
    if (e == cudaSuccess)
      e = L.pass((int)logs, mode, (int)tl, use_fused_tile(p, logs, tl), a, pass_tiles(p->log_n, logs, tl), st);
    if (e == cudaSuccess) e = timing_end(p, st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return NTT_OK;
}

static cudaEvent_t next_event(ntt_plan p) {
  if (p->ev_next == p->ev_pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    p->ev_pool.push_back(e);
  }
  return p->ev_pool[p->ev_next++];
}

cudaError_t timing_begin(ntt_plan p, int pass, cudaStream_t st) {
  if (!p->timing) return cudaSuccess;
  cudaEvent_t a = next_event(p), b = next_event(p);
  if (!a || !b) return cudaErrorMemoryAllocation;
  p->ev_used.push_back({pass, {a, b}});
  return cudaEventRecord(a, st);
}

cudaError_t timing_end(ntt_plan p, cudaStream_t st) {
  if (!p->timing) return cudaSuccess;
  return cudaEventRecord(p->ev_used.back().second.second, st);
}

ntt_status check_buffer(const void *ptr) {
  if (!ptr) return NTT_ERR_INVALID_ARG;
  if ((uintptr_t)ptr % 32) return NTT_ERR_INVALID_ARG;   // one element
  return NTT_OK;
}

}  // namespace gb300ntt

// ===================================================================== C ABI

extern "C" {

ntt_status ntt_plan_create(ntt_plan *out, ntt_field field, uint32_t log_n, int coset) {
  NvtxRange range("ntt_plan_create");
  if (!out) return NTT_ERR_INVALID_ARG;
  *out = nullptr;
  if (field != NTT_FIELD_BLS12_381_FR && field != NTT_FIELD_BN254_FR) return NTT_ERR_INVALID_ARG;
  const uint32_t adicity = field == NTT_FIELD_BLS12_381_FR ? 32 : 28;
  if (log_n < 1 || log_n > adicity || log_n > 28) return NTT_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return NTT_ERR_NO_DEVICE;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return NTT_ERR_NO_DEVICE;
  }
  if (prop.major != 10 || prop.minor != 3) return NTT_ERR_NO_DEVICE;
  NTT_TRY(prepare_device(dev, (int)field));
  ntt_plan p = new (std::nothrow) ntt_plan_s();
  if (!p) return NTT_ERR_OOM;
  p->device = dev;
  p->field = (int)field;
  p->log_n = log_n;
  p->has_coset = coset != 0;
  p->path = NTT_PATH_AUTO;
  p->sm_count = prop.multiProcessorCount;
  cudaStream_t st = nullptr;
  ntt_status s = cuda_status(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  if (s == NTT_OK) s = build_plan(p, st, nullptr);
  if (st) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (s == NTT_OK) s = cuda_status(e);
    cudaStreamDestroy(st);
  }
  if (s == NTT_OK) {
    TuneChoice tc;
    if (tune_lookup(dev, (int)field, log_n, &tc)) s = tune_apply(p, tc);
  }
  if (s == NTT_OK) s = cuda_status(cudaMalloc(&p->d_err, sizeof(uint32_t)));
  if (s == NTT_OK) s = cuda_status(cudaMemset(p->d_err, 0, sizeof(uint32_t)));
  if (s != NTT_OK) {
    ntt_plan_destroy(p);
    return s;
  }
  *out = p;
  return NTT_OK;
}

ntt_status ntt_plan_set_path(ntt_plan plan, ntt_path path) {
  if (!plan) return NTT_ERR_INVALID_ARG;
  if (path != NTT_PATH_AUTO && path != NTT_PATH_BUTTERFLY && path != NTT_PATH_MATRIX) return NTT_ERR_INVALID_ARG;
  if (path == NTT_PATH_MATRIX) {
    if (!matrix_path_available(plan)) return NTT_ERR_UNSUPPORTED;
    NTT_TRY(prepare_matrix_path(plan));
  }
  plan->path = path;
  return NTT_OK;
}

ntt_status ntt_plan_set_coset_shift(ntt_plan plan, const uint64_t shift[4]) {
  if (!plan || !shift) return NTT_ERR_INVALID_ARG;
  if (!plan->has_coset) return NTT_ERR_INVALID_ARG;
  const HostField F = host_field(plan->field);
  const U256 s = from_limbs(shift);
  if (u256_geq(s, F.p) || u256_is_zero(s)) return NTT_ERR_INVALID_ARG;
  cudaStream_t st = nullptr;
  NTT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  ntt_status r = build_coset_tables(plan, s, st);
  if (r == NTT_OK && plan->matrix && plan->matrix->nested) r = build_coset_tables(plan->matrix->nested, s, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (r == NTT_OK) r = cuda_status(e);
  if (r == NTT_OK) r = matrix_build_coset(plan);
  return r;
}

ntt_status ntt_plan_destroy(ntt_plan plan) {
  if (!plan) return NTT_OK;
  batch_forget_plan(plan);
  cudaDeviceSynchronize();
  for (void *ptr : plan->allocations) cudaFree(ptr);
  if (plan->d_err) cudaFree(plan->d_err);
  for (cudaEvent_t e : plan->ev_pool) cudaEventDestroy(e);
  release_matrix_resources(plan);
  delete plan;
  return NTT_OK;
}

ntt_status ntt_execute(ntt_plan plan, ntt_kind kind, const void *d_in, void *d_out, ntt_stream stream) {
  NvtxRange range("ntt_execute");
  if (!plan) return NTT_ERR_INVALID_ARG;
  if (!kind_is_valid((int)kind, plan->has_coset)) return NTT_ERR_INVALID_ARG;
  NTT_TRY(check_buffer(d_in));
  NTT_TRY(check_buffer(d_out));
  if (plan->path == NTT_PATH_MATRIX) return enqueue_matrix_transform(plan, (int)kind, d_in, d_out, (cudaStream_t)stream);
  return enqueue_transform(plan, (int)kind, d_in, d_out, (cudaStream_t)stream);
}

ntt_status ntt_forward(ntt_plan plan, const void *d_in, void *d_out, ntt_stream stream) {
  return ntt_execute(plan, NTT_KIND_FORWARD, d_in, d_out, stream);
}
ntt_status ntt_inverse(ntt_plan plan, const void *d_in, void *d_out, ntt_stream stream) {
  return ntt_execute(plan, NTT_KIND_INVERSE, d_in, d_out, stream);
}
ntt_status ntt_coset_inverse(ntt_plan plan, const void *d_in, void *d_out, ntt_stream stream) {
  return ntt_execute(plan, NTT_KIND_COSET_INVERSE, d_in, d_out, stream);
}
ntt_status ntt_coset_forward(ntt_plan plan, const void *d_in, void *d_out, ntt_stream stream) {
  return ntt_execute(plan, NTT_KIND_COSET, d_in, d_out, stream);
}

ntt_status ntt_transform_host(ntt_plan plan, ntt_kind kind, const void *h_in, void *h_out, void *d_work,
                              ntt_stream stream) {
  if (!plan || !h_in || !h_out) return NTT_ERR_INVALID_ARG;
  NTT_TRY(check_buffer(d_work));
  const size_t bytes = (size_t)32 << plan->log_n;
  cudaStream_t st = (cudaStream_t)stream;
  NTT_CUDA(cudaMemcpyAsync(d_work, h_in, bytes, cudaMemcpyHostToDevice, st));
  NTT_TRY(ntt_execute(plan, kind, d_work, d_work, stream));
  NTT_CUDA(cudaMemcpyAsync(h_out, d_work, bytes, cudaMemcpyDeviceToHost, st));
  NTT_CUDA(cudaStreamSynchronize(st));
  return NTT_OK;
}

ntt_status ntt_transform_host_async(ntt_plan plan, ntt_kind kind, const void *h_in, void *h_out, void *d_work,
                                    ntt_stream stream) {
  if (!plan || !h_in || !h_out) return NTT_ERR_INVALID_ARG;
  NTT_TRY(check_buffer(d_work));
  const size_t bytes = (size_t)32 << plan->log_n;
  cudaStream_t st = (cudaStream_t)stream;
  NTT_CUDA(cudaMemcpyAsync(d_work, h_in, bytes, cudaMemcpyHostToDevice, st));
  NTT_TRY(ntt_execute(plan, kind, d_work, d_work, stream));
  NTT_CUDA(cudaMemcpyAsync(h_out, d_work, bytes, cudaMemcpyDeviceToHost, st));
  return NTT_OK;
}

ntt_status ntt_plan_describe(ntt_plan plan, ntt_plan_desc *out) {
  if (!plan || !out) return NTT_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof *out);
  out->field = (uint32_t)plan->field;
  out->log_n = plan->log_n;
  // the passes of the path that runs: the matrix path's own split when it is selected
  const ntt_plan run = plan->path == NTT_PATH_MATRIX && plan->matrix && plan->matrix->nested ? plan->matrix->nested : plan;
  out->num_passes = run->num_passes;
  for (uint32_t j = 0; j < run->num_passes && j < NTT_MAX_PASSES; ++j) out->pass_log[j] = run->pass_log[j];
  out->launches_per_transform = plan->path == NTT_PATH_MATRIX ? matrix_launches(plan) : plan->launches;
  out->path = (uint32_t)plan->path;
  out->device_bytes = plan->device_bytes;
  out->matrix_folded_passes = plan->path == NTT_PATH_MATRIX && plan->matrix ? plan->matrix->fold : 0;
  return NTT_OK;
}

ntt_status ntt_plan_read_table(ntt_plan plan, ntt_kind kind, uint32_t pass, uint32_t table, uint64_t first,
                               uint64_t count, void *h_out) {
  if (!plan || !h_out) return NTT_ERR_INVALID_ARG;
  if (!kind_is_valid((int)kind, true)) return NTT_ERR_INVALID_ARG;
  if (pass >= plan->num_passes) return NTT_ERR_INVALID_ARG;
  const int tk = table_kind((int)kind);
  const uint32_t logs = plan->pass_log[pass];
  const uint4 *src = nullptr;
  uint64_t size = 0;
  if (table == 0) {
    src = plan->dft_tw[tk == kInverse ? 1 : 0][logs];
    size = std::max<uint64_t>(1, (1ull << logs) / 2);
  } else if (table == 1) {
    if (pass == 0) {
      src = plan->pre[tk];
      size = 1ull << logs;
    } else {
      src = plan->tw[tk][pass];
      uint32_t log_m = 0;
      for (uint32_t i = 0; i <= pass; ++i) log_m += plan->pass_log[i];
      size = 1ull << log_m;
    }
  } else if (table == 2) {
    if (kind == NTT_KIND_COSET_INVERSE && pass == plan->num_passes - 1) src = plan->post_coset_inv;
    size = 1ull << plan->log_n;
  } else {
    return NTT_ERR_INVALID_ARG;
  }
  if (!src || first > size || count > size - first) return NTT_ERR_INVALID_ARG;
  std::vector<uint64_t> buf(count * 4);
  NTT_CUDA(cudaMemcpy(buf.data(), src + 2 * first, count * 32, cudaMemcpyDeviceToHost));
  const HostField F = host_field(plan->field);
  const U256 rinv = F.r_inv();
  uint64_t *o = (uint64_t *)h_out;
  for (uint64_t i = 0; i < count; ++i) {
    const U256 v = F.mul(from_limbs(&buf[4 * i]), rinv);
    std::memcpy(o + 4 * i, v.w, 32);
  }
  return NTT_OK;
}

ntt_status ntt_plan_enable_timing(ntt_plan plan, int enable) {
  if (!plan) return NTT_ERR_INVALID_ARG;
  plan->timing = enable != 0;
  return NTT_OK;
}

ntt_status ntt_plan_read_timing(ntt_plan plan, double ms_per_pass[NTT_MAX_PASSES],
                                uint64_t launches_per_pass[NTT_MAX_PASSES]) {
  if (!plan || !ms_per_pass || !launches_per_pass) return NTT_ERR_INVALID_ARG;
  for (int j = 0; j < NTT_MAX_PASSES; ++j) {
    ms_per_pass[j] = 0;
    launches_per_pass[j] = 0;
  }
  ntt_status s = NTT_OK;
  for (auto &u : plan->ev_used) {
    float ms = 0;
    const cudaError_t e = cudaEventSynchronize(u.second.second);
    if (e == cudaSuccess && cudaEventElapsedTime(&ms, u.second.first, u.second.second) == cudaSuccess) {
      if (u.first >= 0 && u.first < NTT_MAX_PASSES) {
        ms_per_pass[u.first] += ms;
        launches_per_pass[u.first] += 1;
      }
    } else {
      s = NTT_ERR_CUDA;
    }
  }
  plan->ev_used.clear();
  plan->ev_next = 0;
  return s;
}

ntt_status ntt_plan_poll_error(ntt_plan plan, uint32_t *code) {
  if (!plan || !code) return NTT_ERR_INVALID_ARG;
  NTT_CUDA(cudaDeviceSynchronize());
  NTT_CUDA(cudaMemcpy(code, plan->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  NTT_CUDA(cudaMemset(plan->d_err, 0, sizeof(uint32_t)));
  uint32_t mcode = 0;
  NTT_TRY(matrix_poll_error(plan, &mcode));
  if (!*code) *code = mcode;
  return NTT_OK;
}

ntt_status ntt_field_mont_mul(ntt_field field, const void *d_a, const void *d_b, void *d_out, uint64_t count,
                              ntt_stream stream) {
  if (field != NTT_FIELD_BLS12_381_FR && field != NTT_FIELD_BN254_FR) return NTT_ERR_INVALID_ARG;
  if (count == 0) return NTT_OK;
  NTT_TRY(check_buffer(d_a));
  NTT_TRY(check_buffer(d_b));
  NTT_TRY(check_buffer(d_out));
  return cuda_status(
      launchers((int)field).mul_vec((uint4 *)d_out, (const uint4 *)d_a, (const uint4 *)d_b, count, (cudaStream_t)stream));
}

ntt_status ntt_pointwise_quotient(ntt_field field, const void *d_a, const void *d_b, const void *d_c,
                                  const uint64_t *h_z, uint32_t z_len, void *d_out, uint64_t count, ntt_stream stream) {
  if (field != NTT_FIELD_BLS12_381_FR && field != NTT_FIELD_BN254_FR) return NTT_ERR_INVALID_ARG;
  if (!h_z || z_len == 0 || z_len > (uint32_t)kMaxQuotientZ || (z_len & (z_len - 1))) return NTT_ERR_INVALID_ARG;
  NTT_TRY(check_buffer(d_a));
  NTT_TRY(check_buffer(d_b));
  NTT_TRY(check_buffer(d_c));
  NTT_TRY(check_buffer(d_out));
  const HostField F = host_field((int)field);
  QuotientZ z{};
  z.len = z_len;
  for (uint32_t j = 0; j < z_len; ++j) {
    const U256 v = from_limbs(h_z + 4 * j);
    if (u256_geq(v, F.p)) return NTT_ERR_INVALID_ARG;
    z.z[j] = to_fe32(F.to_mont(F.to_mont(v)));   // z 2^512 mod M
  }
  if (count == 0) return NTT_OK;
  return cuda_status(launchers((int)field).quotient((uint4 *)d_out, (const uint4 *)d_a, (const uint4 *)d_b,
                                                    (const uint4 *)d_c, z, count, (cudaStream_t)stream));
}

ntt_status ntt_field_mont_mul_rep(ntt_field field, const void *d_a, const void *d_b, void *d_out, uint64_t count,
                                  uint32_t reps, int variant, ntt_stream stream) {
  if (field != NTT_FIELD_BLS12_381_FR && field != NTT_FIELD_BN254_FR) return NTT_ERR_INVALID_ARG;
  if (reps == 0 || (variant != 0 && variant != 1)) return NTT_ERR_INVALID_ARG;
  if (count == 0) return NTT_OK;
  if (count > (1ull << 28)) return NTT_ERR_UNSUPPORTED;
  NTT_TRY(check_buffer(d_a));
  NTT_TRY(check_buffer(d_b));
  NTT_TRY(check_buffer(d_out));
  return cuda_status(launchers((int)field).mul_rep((uint4 *)d_out, (const uint4 *)d_a, (const uint4 *)d_b, count, reps,
                                                   variant, (cudaStream_t)stream));
}

const char *ntt_status_string(ntt_status status) {
  switch (status) {
    case NTT_OK: return "NTT_OK";
    case NTT_ERR_INVALID_ARG: return "NTT_ERR_INVALID_ARG";
    case NTT_ERR_UNSUPPORTED: return "NTT_ERR_UNSUPPORTED";
    case NTT_ERR_OOM: return "NTT_ERR_OOM";
    case NTT_ERR_CUDA: return "NTT_ERR_CUDA";
    case NTT_ERR_TIMEOUT: return "NTT_ERR_TIMEOUT";
    case NTT_ERR_BUDGET: return "NTT_ERR_BUDGET";
    case NTT_ERR_NO_DEVICE: return "NTT_ERR_NO_DEVICE";
    case NTT_ERR_BOUNDS: return "NTT_ERR_BOUNDS";
  }
  return "NTT_ERR_UNKNOWN";
}

uint32_t ntt_version(void) { return 100; }

int ntt_build_is_debug(void) {
#ifdef NTT_DEBUG
  return 1;
#else
  return 0;
#endif
}

ntt_status ntt_debug_shrink_next_extent(ntt_plan plan) {
  if (!plan) return NTT_ERR_INVALID_ARG;
#ifdef NTT_DEBUG
  plan->debug_shrink = true;
  return NTT_OK;
#else
  return NTT_ERR_UNSUPPORTED;
#endif
}

}  // extern "C"
