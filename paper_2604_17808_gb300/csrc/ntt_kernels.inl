// ntt_kernels.inl -- kernel instantiations and launchers for one field.
//
// Included by the kernels_<field>*.cu files with NTT_FIELD (the field type),
// NTT_NS (a namespace for the field's launchers) and one NTT_PART_* macro,
// so that the kernel families of a field compile in parallel, one nvcc
// process each:
//   NTT_PART_PASS = 10 or 11  the pass kernels of one tile shape;
//   NTT_PART_BATCH            the persistent batched kernel;
//   NTT_PART_MATRIX           the matrix-form (tensor-core) pass;
//   NTT_PART_MISC             table generators, element-wise kernels and
//                             the launcher table.
#include "../../include/ntt_gb300.h"
#include "ntt_launch.h"

namespace gb300ntt {
namespace NTT_NS {

// launchers defined by the other parts of this field
cudaError_t prepare_pass10();
cudaError_t prepare_pass11();
cudaError_t pass10(int logs, int mode, bool fused, const PassArgs &a, uint64_t tiles, cudaStream_t st);
cudaError_t pass11(int logs, int mode, bool fused, const PassArgs &a, uint64_t tiles, cudaStream_t st);
cudaError_t prepare_batch();
cudaError_t batch(const BatchLaunch &b, cudaStream_t st);
cudaError_t prepare_matrix();
cudaError_t matrix_pass(int logs, int mode, const MatrixPassArgs &ma, const CUtensorMap &in_map, uint32_t grid,
                        cudaStream_t st);

namespace {

using F = NTT_FIELD;

__device__ __forceinline__ void fe_from_param(uint32_t r[8], const Fe32 &a) {
#pragma unroll
  for (int j = 0; j < 8; ++j) r[j] = a.w[j];
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Launch with programmatic stream serialisation (see pdl_trigger_and_wait):
// consecutive passes overlap their launch latency and CTA scheduling.
template <class K, class... A>
cudaError_t launch_pdl(K kernel, dim3 grid, dim3 block, int smem, cudaStream_t st, const A &...a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, a...);
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

}  // namespace

#if defined(NTT_PART_PASS)

namespace {

// The fused tile is instantiated for the 1024-element tile only: that is
// the shape of the one-wave passes it is chosen for (sizes up to 2^20).
template <int LOGS, int TL>
constexpr bool has_fused() {
  return TL == 10 && LOGS >= 4;
}

template <int LOGS, int MODE, int TL>
cudaError_t set_pass_attr() {
  cudaError_t e = cudaFuncSetAttribute(ntt_pass_kernel<F, LOGS, MODE, TL, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, TileCfg<TL>::kBytes);
  if constexpr (has_fused<LOGS, TL>()) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ntt_pass_kernel<F, LOGS, MODE, TL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TileCfg<TL>::kBytes);
  }
  return e;
}

template <int LOGS, int TL>
cudaError_t set_pass_attrs() {
  cudaError_t e = set_pass_attr<LOGS, kModeInner, TL>();
  if (e == cudaSuccess) e = set_pass_attr<LOGS, kModeFirst, TL>();
  if (e == cudaSuccess) e = set_pass_attr<LOGS, kModeFirstPre, TL>();
  return e;
}

template <int TL>
cudaError_t set_all_pass_attrs() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = set_pass_attrs<1, TL>();
  if (e == cudaSuccess) e = set_pass_attrs<2, TL>();
  if (e == cudaSuccess) e = set_pass_attrs<3, TL>();
  if (e == cudaSuccess) e = set_pass_attrs<4, TL>();
  if (e == cudaSuccess) e = set_pass_attrs<5, TL>();
  if (e == cudaSuccess) e = set_pass_attrs<6, TL>();
  if (e == cudaSuccess) e = set_pass_attrs<7, TL>();
  if (e == cudaSuccess) e = set_pass_attrs<8, TL>();
  if (e == cudaSuccess) e = set_pass_attrs<9, TL>();
  if (e == cudaSuccess) e = set_pass_attrs<10, TL>();
  if constexpr (TL >= 11) {
    if (e == cudaSuccess) e = set_pass_attrs<11, TL>();
  }
  return e;
}

template <int LOGS, int TL, bool FUSED>
cudaError_t pass_launch(int mode, const PassArgs &a, uint64_t tiles, cudaStream_t st) {
  const dim3 grid((unsigned)tiles), block(TileCfg<TL>::kThreads);
  const int smem = TileCfg<TL>::kBytes;
  switch (mode) {
    case kModeInner: return launch_pdl(ntt_pass_kernel<F, LOGS, kModeInner, TL, FUSED>, grid, block, smem, st, a);
    case kModeFirst: return launch_pdl(ntt_pass_kernel<F, LOGS, kModeFirst, TL, FUSED>, grid, block, smem, st, a);
    case kModeFirstPre:
      return launch_pdl(ntt_pass_kernel<F, LOGS, kModeFirstPre, TL, FUSED>, grid, block, smem, st, a);
    default: return cudaErrorInvalidValue;
  }
}

template <int LOGS, int TL>
cudaError_t pass_logs(int mode, bool fused, const PassArgs &a, uint64_t tiles, cudaStream_t st) {
  if constexpr (has_fused<LOGS, TL>()) {
    if (fused) return pass_launch<LOGS, TL, true>(mode, a, tiles, st);
  }
  return pass_launch<LOGS, TL, false>(mode, a, tiles, st);
}

template <int TL>
cudaError_t pass_tl(int logs, int mode, bool fused, const PassArgs &a, uint64_t tiles, cudaStream_t st) {
  switch (logs) {
    case 1: return pass_logs<1, TL>(mode, fused, a, tiles, st);
    case 2: return pass_logs<2, TL>(mode, fused, a, tiles, st);
    case 3: return pass_logs<3, TL>(mode, fused, a, tiles, st);
    case 4: return pass_logs<4, TL>(mode, fused, a, tiles, st);
    case 5: return pass_logs<5, TL>(mode, fused, a, tiles, st);
    case 6: return pass_logs<6, TL>(mode, fused, a, tiles, st);
    case 7: return pass_logs<7, TL>(mode, fused, a, tiles, st);
    case 8: return pass_logs<8, TL>(mode, fused, a, tiles, st);
    case 9: return pass_logs<9, TL>(mode, fused, a, tiles, st);
    case 10: return pass_logs<10, TL>(mode, fused, a, tiles, st);
    case 11:
      if constexpr (TL >= 11) return pass_logs<11, TL>(mode, fused, a, tiles, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

#if NTT_PART_PASS == 10
cudaError_t prepare_pass10() { return set_all_pass_attrs<10>(); }
cudaError_t pass10(int logs, int mode, bool fused, const PassArgs &a, uint64_t tiles, cudaStream_t st) {
  return pass_tl<10>(logs, mode, fused, a, tiles, st);
}
#else
cudaError_t prepare_pass11() { return set_all_pass_attrs<11>(); }
cudaError_t pass11(int logs, int mode, bool fused, const PassArgs &a, uint64_t tiles, cudaStream_t st) {
  return pass_tl<11>(logs, mode, fused, a, tiles, st);
}
#endif

#elif defined(NTT_PART_BATCH)

namespace {

// One tile of one segment.  Each (size, mode) variant is a separate,
// non-inlined function: the call costs nothing next to a 2048-element tile,
// and ptxas then compiles 33 small functions instead of one kernel holding
// every variant inline (which took minutes).
template <int LOGS, int MODE>
__device__ __noinline__ void batch_tile_fn(const BatchSeg &sg, uint64_t tile, uint4 *smem) {
  pass_tile<F, LOGS, MODE, true, 11, true>(sg.a, tile, smem);
}

template <int LOGS>
__device__ __forceinline__ void batch_tile_logs(const BatchSeg &sg, uint64_t tile, uint4 *smem) {
  switch (sg.mode) {
    case kModeInner: batch_tile_fn<LOGS, kModeInner>(sg, tile, smem); break;
    case kModeFirst: batch_tile_fn<LOGS, kModeFirst>(sg, tile, smem); break;
    default: batch_tile_fn<LOGS, kModeFirstPre>(sg, tile, smem); break;
  }
}

__device__ __forceinline__ void batch_tile(const BatchSeg &sg, uint64_t tile, uint4 *smem) {
  switch (sg.logs) {
    case 1: batch_tile_logs<1>(sg, tile, smem); break;
    case 2: batch_tile_logs<2>(sg, tile, smem); break;
    case 3: batch_tile_logs<3>(sg, tile, smem); break;
    case 4: batch_tile_logs<4>(sg, tile, smem); break;
    case 5: batch_tile_logs<5>(sg, tile, smem); break;
    case 6: batch_tile_logs<6>(sg, tile, smem); break;
    case 7: batch_tile_logs<7>(sg, tile, smem); break;
    case 8: batch_tile_logs<8>(sg, tile, smem); break;
    case 9: batch_tile_logs<9>(sg, tile, smem); break;
    case 10: batch_tile_logs<10>(sg, tile, smem); break;
    default: batch_tile_logs<11>(sg, tile, smem); break;
  }
}

// CTAs claim items (one tile of one pass of one job) in increasing order.
// An item of pass j waits until every tile of pass j-1 of its job is done;
// those tiles have smaller item indices, so they are held by CTAs that have
// already started and never wait on later items: no deadlock.  Every wait
// is bounded by b.wait_ns (globaltimer); on timeout the CTA records
// NTT_ERR_TIMEOUT in *b.err and returns, and every CTA stops claiming
// items once *b.err is set.
__global__ void __launch_bounds__(kPassThreads, kPassCtasPerSm) batch_kernel(const BatchLaunch b) {
  extern __shared__ uint4 smem[];
  __shared__ uint32_t s_item;
  __shared__ int32_t s_seg;
  __shared__ int s_abort;
  for (;;) {
    if (threadIdx.x == 0) {
      uint32_t item = atomicAdd(b.head, 1u);
      if (*(volatile uint32_t *)b.err != 0) item = b.total_items;
      int32_t seg = -1;
      int abort = 0;
      if (item < b.total_items) {
        int lo = 0, hi = (int)b.num_segs - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (b.segs[mid].first_item <= item) lo = mid;
          else hi = mid - 1;
        }
        seg = lo;
        const int32_t dep = b.segs[lo].dep_seg;
        if (dep >= 0) {
          const uint32_t need = b.segs[lo].dep_tiles;
          const uint64_t t0 = global_ns();
          while (ld_acquire_gpu(b.done + dep) < need) {
            if (global_ns() - t0 > b.wait_ns) {
              atomicCAS(b.err, 0u, (uint32_t)NTT_ERR_TIMEOUT);
              abort = 1;
              break;
            }
            __nanosleep(128);
          }
        }
      }
      s_item = item;
      s_seg = seg;
      s_abort = abort;
    }
    __syncthreads();
    if (s_item >= b.total_items || s_abort) return;
    const BatchSeg &sg = b.segs[s_seg];
    batch_tile(sg, s_item - sg.first_item, smem);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(b.done + s_seg, 1u);
    }
  }
}

}  // namespace

cudaError_t batch(const BatchLaunch &b, cudaStream_t st) {
  batch_kernel<<<b.grid, kPassThreads, kTileBytes, st>>>(b);
  return cudaGetLastError();
}


cudaError_t prepare_batch() {
  return cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileBytes);
}

#elif defined(NTT_PART_MATRIX)

namespace {

template <int LOGS, int MODE, bool BARRETT>
cudaError_t set_matrix_attr() {
  return cudaFuncSetAttribute(ntt_matrix_pass_kernel<F, LOGS, MODE, BARRETT>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, matrix_smem_bytes<LOGS>());
}

template <int LOGS>
cudaError_t set_matrix_attrs() {
  cudaError_t e = set_matrix_attr<LOGS, kModeInner, false>();
  if (e == cudaSuccess) e = set_matrix_attr<LOGS, kModeInner, true>();
  if (e == cudaSuccess) e = set_matrix_attr<LOGS, kModeFirst, false>();
  if (e == cudaSuccess) e = set_matrix_attr<LOGS, kModeFirst, true>();
  return e;
}

template <int LOGS, int MODE>
cudaError_t matrix_mode(const MatrixPassArgs &ma, const CUtensorMap &in_map, uint32_t grid, cudaStream_t st) {
  const int smem = matrix_smem_bytes<LOGS>();
  if (ma.barrett)
    return launch_pdl(ntt_matrix_pass_kernel<F, LOGS, MODE, true>, grid, kMatThreads, smem, st, ma, in_map);
  return launch_pdl(ntt_matrix_pass_kernel<F, LOGS, MODE, false>, grid, kMatThreads, smem, st, ma, in_map);
}

template <int LOGS>
cudaError_t matrix_logs(int mode, const MatrixPassArgs &ma, const CUtensorMap &in_map, uint32_t grid,
                        cudaStream_t st) {
  switch (mode) {
    case kModeInner: return matrix_mode<LOGS, kModeInner>(ma, in_map, grid, st);
    case kModeFirst: return matrix_mode<LOGS, kModeFirst>(ma, in_map, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t matrix_pass(int logs, int mode, const MatrixPassArgs &ma, const CUtensorMap &in_map, uint32_t grid,
                        cudaStream_t st) {
  switch (logs) {
    case 1: return matrix_logs<1>(mode, ma, in_map, grid, st);
    case 2: return matrix_logs<2>(mode, ma, in_map, grid, st);
    case 3: return matrix_logs<3>(mode, ma, in_map, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t prepare_matrix() {
  cudaError_t e = set_matrix_attrs<1>();
  if (e == cudaSuccess) e = set_matrix_attrs<2>();
  if (e == cudaSuccess) e = set_matrix_attrs<3>();
  return e;
}

#elif defined(NTT_PART_MISC)

namespace {

// acc *= base^e using the ladder pw (bits of e below 32).
__device__ __forceinline__ void ladder_mul(uint32_t acc[8], uint64_t e, const Pow2Table &pw) {
  for (int b = 0; b < 32 && (e >> b) != 0; ++b) {
    if ((e >> b) & 1) {
      uint32_t w[8];
      fe_from_param(w, pw.v[b]);
      mont_mul<F>(acc, acc, w);
    }
  }
}

__global__ void gen_2d_kernel(uint4 *out, uint32_t log_s, uint32_t log_mp, const Pow2Table pw,
                              const uint4 *fac, const Fe32 init) {
  const uint64_t total = 1ull << (log_s + log_mp);
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t n = idx >> log_mp, q = idx & ((1ull << log_mp) - 1);
    uint32_t acc[8];
    fe_from_param(acc, init);
    if (fac) {
      uint32_t f[8];
      fe_load_global(f, fac, n);
      mont_mul<F>(acc, acc, f);
    }
    ladder_mul(acc, n * q, pw);
    fe_store_global(out, idx, acc);
  }
}

__global__ void gen_1d_kernel(uint4 *out, uint64_t count, const Pow2Table pw, const Fe32 init) {
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < count;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t acc[8];
    fe_from_param(acc, init);
    ladder_mul(acc, idx, pw);
    fe_store_global(out, idx, acc);
  }
}

__global__ void mul_vec_kernel(uint4 *out, const uint4 *a, const uint4 *b, uint64_t count) {
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < count;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x[8], y[8];
    fe_load_global(x, a, idx);
    fe_load_global(y, b, idx);
    mont_mul<F>(x, x, y);
    fe_store_global(out, idx, x);
  }
}

// Pointwise quotient of a prover on coset evaluations:
//   out[i] = (a[i] b[i] - c[i]) z[i mod len]
// in one pass over the vectors (3 reads, 1 write, two products and one
// reduction per element): u = a b 2^-256, v = c 2^-256, and the multiplier
// z 2^512 turns (u - v) back into standard form.
__global__ void quotient_kernel(uint4 *out, const uint4 *a, const uint4 *b, const uint4 *c, const QuotientZ z,
                                uint64_t count) {
  const uint64_t zmask = z.len - 1;
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < count;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x[8], y[8], w[8];
    fe_load_global(x, a, idx);
    fe_load_global(y, b, idx);
    mont_mul<F>(x, x, y);          // a b 2^-256
    fe_load_global(y, c, idx);
    mont_redc<F>(y, y);            // c 2^-256
    sub_mod<F>(x, x, y);
    fe_from_param(w, z.z[idx & zmask]);
    mont_mul<F>(x, x, w);          // (a b - c) z
    fe_store_global(out, idx, x);
  }
}

// out[i] = a[i] * (b[i] * 2^-256)^reps: `reps` dependent Montgomery products
// per element, per-thread carry chains (variant 0) or 8 lanes per element
// with shuffle carries (variant 1).
__global__ void mul_rep_kernel(uint4 *out, const uint4 *a, const uint4 *b, uint64_t count, uint32_t reps) {
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < count;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x[8], y[8];
    fe_load_global(x, a, idx);
    fe_load_global(y, b, idx);
    for (uint32_t r = 0; r < reps; ++r) mont_mul<F>(x, x, y);
    fe_store_global(out, idx, x);
  }
}

__global__ void mul_rep_coop_kernel(uint32_t *out, const uint32_t *a, const uint32_t *b, uint64_t count,
                                    uint32_t reps) {
  // 8 lanes per element; the grid covers every element exactly (no early exit
  // of part of a warp: the shuffles need all 32 lanes)
  const uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint32_t j = threadIdx.x & 7u;
  const uint64_t elem = gid >> 3;
  const bool live = elem < count;
  uint32_t x = live ? a[elem * 8 + j] : 0u;
  const uint32_t y = live ? b[elem * 8 + j] : 0u;
  for (uint32_t r = 0; r < reps; ++r) x = mont_mul_coop<F>(x, y, j);
  if (live) out[elem * 8 + j] = x;
}

cudaError_t prepare() {
  cudaError_t e = prepare_pass11();
  if (e == cudaSuccess) e = prepare_matrix();
  if (e == cudaSuccess) e = prepare_pass10();
  if (e == cudaSuccess) e = prepare_batch();
  return e;
}

cudaError_t pass(int logs, int mode, int tl, bool fused, const PassArgs &a, uint64_t tiles, cudaStream_t st) {
  if (tl == 11) return pass11(logs, mode, fused, a, tiles, st);
  if (tl == 10) return pass10(logs, mode, fused, a, tiles, st);
  return cudaErrorInvalidValue;
}

unsigned grid_for(uint64_t count) {
  uint64_t blocks = (count + 255) / 256;
  if (blocks > 152ull * 64) blocks = 152ull * 64;
  return (unsigned)(blocks ? blocks : 1);
}

cudaError_t gen_2d(uint4 *out, uint32_t log_s, uint32_t log_mp, const Pow2Table &pw, const uint4 *fac,
                   Fe32 init, cudaStream_t st) {
  gen_2d_kernel<<<grid_for(1ull << (log_s + log_mp)), 256, 0, st>>>(out, log_s, log_mp, pw, fac, init);
  return cudaGetLastError();
}

cudaError_t gen_1d(uint4 *out, uint64_t count, const Pow2Table &pw, Fe32 init, cudaStream_t st) {
  gen_1d_kernel<<<grid_for(count), 256, 0, st>>>(out, count, pw, init);
  return cudaGetLastError();
}

cudaError_t mul_vec(uint4 *out, const uint4 *a, const uint4 *b, uint64_t count, cudaStream_t st) {
  mul_vec_kernel<<<grid_for(count), 256, 0, st>>>(out, a, b, count);
  return cudaGetLastError();
}

cudaError_t mul_rep(uint4 *out, const uint4 *a, const uint4 *b, uint64_t count, uint32_t reps, int variant,
                    cudaStream_t st) {
  if (variant == 0) {
    mul_rep_kernel<<<grid_for(count), 256, 0, st>>>(out, a, b, count, reps);
  } else {
    const uint64_t threads = count * 8;
    mul_rep_coop_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        (uint32_t *)out, (const uint32_t *)a, (const uint32_t *)b, count, reps);
  }
  return cudaGetLastError();
}

cudaError_t quotient(uint4 *out, const uint4 *a, const uint4 *b, const uint4 *c, const QuotientZ &z, uint64_t count,
                     cudaStream_t st) {
  quotient_kernel<<<grid_for(count), 256, 0, st>>>(out, a, b, c, z, count);
  return cudaGetLastError();
}

const FieldLaunchers kLaunchers = {prepare, pass, gen_2d, gen_1d, mul_vec, batch, mul_rep, matrix_pass, quotient};

}  // namespace

const FieldLaunchers &launchers() { return kLaunchers; }

#endif

}  // namespace NTT_NS
}  // namespace gb300ntt
