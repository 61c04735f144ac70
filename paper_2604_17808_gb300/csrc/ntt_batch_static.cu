// ntt_batch_static.cu -- batched submission that allocates nothing.
//
// ntt_batch_submit allocates a work-item table and counters for every new
// job list (cudaMalloc).  Some callers cannot allocate on their submission
// path: services that reserve all device memory up front and must not
// allocate once they serve requests, and submitters on a latency path,
// where cudaMalloc's implicit device synchronisation would stall work
// already queued on other streams.  For them,
// ntt_batch_submit_static runs the same persistent batched kernel with its
// work-item table and counters in one file-scope device array of fixed size,
// instead of allocated memory.  Its host side uses only fixed-size stack
// arrays: no cudaMalloc, cudaFree or heap allocation.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "ntt_launch.h"
#include "ntt_plan.h"
#include "nvtx_range.h"

using namespace gb300ntt;

namespace {

constexpr uint32_t kStaticMaxJobs = 64;
// Segments (passes of jobs) per field per call: four per job on average.
// A job has at most kMaxPasses passes; a call whose jobs need more than
// kStaticMaxSegs segments in one field is rejected (NTT_ERR_UNSUPPORTED).
constexpr uint32_t kStaticMaxSegs = kStaticMaxJobs * 4;

struct StaticScratch {
  BatchSeg segs[2][kStaticMaxSegs];       // work-item tables, one per field
  uint32_t ctl[2][1 + kStaticMaxSegs];    // [0] = next item, [1 + s] = tiles done of segment s
  uint32_t err;                           // error word when the caller passes no status
                                          // (read and cleared by ntt_batch_poll_error)
};

// Work-item table of the jobs of one field into `out` (capacity
// kStaticMaxSegs), ordered by pass level, larger jobs first within a level.
// Fixed-size arrays only.
ntt_status static_segments(const ntt_job *jobs, size_t n, int field, BatchSeg *out, uint32_t *count,
                           uint32_t *total_items) {
  uint32_t order[kStaticMaxJobs];
  int seg_of[kStaticMaxJobs][kMaxPasses];  // [job][pass] -> segment index
  uint32_t m = 0, max_passes = 0;
  for (size_t i = 0; i < n; ++i) {
    if (jobs[i].plan->field != field) continue;
    order[m++] = (uint32_t)i;
    max_passes = std::max(max_passes, jobs[i].plan->num_passes);
  }
  std::stable_sort(order, order + m, [&](uint32_t a, uint32_t b) { return jobs[a].plan->log_n > jobs[b].plan->log_n; });
  uint32_t segs = 0, item = 0;
  for (uint32_t level = 0; level < max_passes; ++level) {
    for (uint32_t oi = 0; oi < m; ++oi) {
      const uint32_t i = order[oi];
      const ntt_job &j = jobs[i];
      if (level >= j.plan->num_passes) continue;
      if (segs >= kStaticMaxSegs) return NTT_ERR_UNSUPPORTED;
      BatchSeg &s = out[segs];
      s = BatchSeg{};
      int mode = 0;
      build_pass_args(j.plan, j.kind, j.in, j.out, level, &s.a, &mode);
      s.logs = j.plan->pass_log[level];
      s.mode = (uint32_t)mode;
      s.first_item = item;
      s.num_tiles = (uint32_t)pass_tiles(j.plan->log_n, s.logs, kTileLog);
      s.dep_seg = level > 0 ? seg_of[i][level - 1] : -1;
      s.dep_tiles = level > 0 ? out[s.dep_seg].num_tiles : 0;
      seg_of[i][level] = (int)segs;
      item += s.num_tiles;
      ++segs;
    }
  }
  if (batch_debug_stall()) {
    // test hook (as in ntt_batch_submit): the last segment with a dependency
    // waits for one tile more than exists, so its bounded wait runs out
    for (int k = (int)segs - 1; k >= 0; --k)
      if (out[k].dep_seg >= 0) {
        out[k].dep_tiles += 1;
        break;
      }
  }
  *count = segs;
  *total_items = item;
  return NTT_OK;
}

}  // namespace

// The scratch, resident on every device that loads the library until the
// process exits (about 55 KB).
static __device__ __align__(256) StaticScratch g_static_scratch;

namespace {

std::mutex g_static_mu;
StaticScratch *g_static_addr[64] = {};  // device address of g_static_scratch, per device

// Once per device, with that device current: the device address of the
// array (its name in host code is only a host-side stand-in).  The address
// is kept until ntt_batch_cache_clear (after a cudaDeviceReset the module
// is loaded anew and the address must be looked up again).
ntt_status static_scratch_address(int dev, StaticScratch **out) {
  if (dev < 0 || dev >= 64) return NTT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return NTT_ERR_CUDA;
    g_static_addr[dev] = static_cast<StaticScratch *>(p);
  }
  *out = g_static_addr[dev];
  return NTT_OK;
}

}  // namespace

namespace gb300ntt {

// The error word of calls made without a status pointer, read and cleared
// for ntt_batch_poll_error (0 when this device never ran such a call).
ntt_status static_batch_take_error(int dev, uint32_t *code) {
  *code = 0;
  if (dev < 0 || dev >= 64) return NTT_ERR_INVALID_ARG;
  StaticScratch *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    scratch = g_static_addr[dev];
  }
  if (!scratch) return NTT_OK;
  ntt_status s = cuda_status(cudaMemcpy(code, &scratch->err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (s == NTT_OK && *code) s = cuda_status(cudaMemset(&scratch->err, 0, sizeof(uint32_t)));
  return s;
}

void static_batch_forget_addresses() {
  std::lock_guard<std::mutex> lk(g_static_mu);
  for (StaticScratch *&a : g_static_addr) a = nullptr;
}

}  // namespace gb300ntt

extern "C" ntt_status ntt_batch_submit_static(const ntt_job *jobs, size_t n, uint32_t *d_status, ntt_stream stream) {
  NvtxRange range("ntt_batch_submit_static");
  if (!jobs && n) return NTT_ERR_INVALID_ARG;
  if (n > kStaticMaxJobs) return NTT_ERR_UNSUPPORTED;
  for (size_t i = 0; i < n; ++i) {
    const ntt_job &j = jobs[i];
    if (!j.plan || j.in == j.out) return NTT_ERR_INVALID_ARG;
    if (!kind_is_valid(j.kind, j.plan->has_coset)) return NTT_ERR_INVALID_ARG;
    if (j.plan->path == NTT_PATH_MATRIX) return NTT_ERR_UNSUPPORTED;
    ntt_status s = check_buffer(j.in);
    if (s == NTT_OK) s = check_buffer(j.out);
    if (s != NTT_OK) return s;
  }
  if (d_status && (uintptr_t)d_status % 4) return NTT_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NTT_ERR_NO_DEVICE;
  StaticScratch *scratch = nullptr;
  ntt_status st = static_scratch_address(dev, &scratch);
  if (st != NTT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // With a status pointer the call reports into it (cleared first); without
  // one, into the array's error word, which keeps the first error until
  // ntt_batch_poll_error reads it (as the word of ntt_batch_submit does).
  uint32_t *err = d_status ? d_status : &scratch->err;
  if (d_status && cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s) != cudaSuccess) return NTT_ERR_CUDA;
  if (n == 0) return NTT_OK;
  BatchSeg host_segs[kStaticMaxSegs];
  for (int field = 0; field < 2; ++field) {
    uint32_t count = 0, total = 0;
    st = static_segments(jobs, n, field, host_segs, &count, &total);
    if (st != NTT_OK) return st;
    if (count == 0) continue;
    // from pageable stack memory: the call returns once the bytes are staged
    if (cudaMemcpyAsync(scratch->segs[field], host_segs, count * sizeof(BatchSeg), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return NTT_ERR_CUDA;
    // counters must start at zero on every call (the array keeps the last call's values)
    if (cudaMemsetAsync(scratch->ctl[field], 0, (1 + count) * sizeof(uint32_t), s) != cudaSuccess) return NTT_ERR_CUDA;
    BatchLaunch b;
    b.segs = scratch->segs[field];
    b.num_segs = count;
    b.total_items = total;
    b.head = scratch->ctl[field];
    b.done = scratch->ctl[field] + 1;
    b.err = err;
    b.wait_ns = batch_wait_limit_ns();
    b.grid = (uint32_t)(jobs[0].plan->sm_count * kPassCtasPerSm);
    if (launchers(field).batch(b, s) != cudaSuccess) return NTT_ERR_CUDA;
  }
  return NTT_OK;
}
