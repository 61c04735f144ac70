// ntt_matrix.cuh -- matrix-form sub-transforms on the tcgen05 tensor cores.
//
// The paper's reformulation (Sec. 3.2.3-3.2.4, Alg. 1; Sec. 3.3.2, Fig. 5b-c):
// high-precision modular arithmetic becomes a low-precision matrix product
// over byte limbs (ByteDecompose -> uint8 "Einsum" against a precomputed
// byte matrix E -> ByteMerge), and the NTT's sub-transforms become matrix
// products with twiddle matrices.  Here one pass of the multi-pass NTT
// computes, for 128 sub-transforms of size S at once,
//
//   y_k = sum_n x_n omega_S^(nk)
//       = sum_{n,b} a_{n,b} W[(n,b), k],  x_n = sum_b a_{n,b} 2^(8b)
//   W[(n,b), k] = omega_S^(nk) * 2^(8b) * 2^256 mod p       (precomputed)
//   W[(n,b), k] = sum_h E[(k,h), (n,b)] 2^(8h)              (signed digits)
//   acc[k,h]   = sum_{n,b} a_{n,b} E[(k,h), (n,b)]           <- tensor cores
//   y_k        = REDC( sum_h acc[k,h] 2^(8h) + 2^18 p )      <- ByteMerge + Montgomery
//
// Digits are balanced (signed, in [-128, 127]) so |a * E| <= 2^14 and, with
// K = 32 S <= 256 terms, every partial sum stays within 2^22: bf16 holds the
// digits exactly and the fp32 accumulators hold every partial sum exactly
// (checked on GB300 with adversarial all -128 operands).  The 2^256 in W
// cancels the REDC factor, so the output is the standard-form y_k, canonical.
//
// Shapes per CTA tile: M = 128 (sub-transforms), N = K = 32 S (S <= 8),
// one tcgen05.mma.cta_group::1.kind::f16 (bf16 x bf16 -> f32) per 16 of K,
// accumulator in TMEM (N columns), operands in shared memory in the K-major
// no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix, LBO =
// 128 bytes along K, SBO = K/8 * 128 bytes along M/N).
#pragma once

#include <cstdint>

#include "../../include/ntt_gb300.h"
#include "fp256.cuh"
#include "ntt_pass.cuh"

namespace gb300ntt {

constexpr int kMatThreads = 512;
constexpr int kMatRows = 128;  // sub-transforms per tile (MMA M)

struct MatrixPassArgs {
  PassArgs a;                // src, dst, mul, num_sub, log_mp, digits (dft_tw unused)
  const uint4 *e;            // E in the B-operand layout, N x K bf16
  uint32_t offset[9];        // 2^18 * p, 9 limbs
  uint32_t *err;             // device error word
  uint64_t wait_ns;          // bound of the MMA-completion wait
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major, no swizzle.
__device__ __forceinline__ uint64_t mat_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Byte offset of element (row, col) of a K-major bf16 operand with K columns.
__host__ __device__ __forceinline__ uint32_t core_offset(uint32_t row, uint32_t col, uint32_t K) {
  return ((row >> 3) * (K >> 3) + (col >> 3)) * 128 + (row & 7) * 16 + (col & 7) * 2;
}

// bf16 bit pattern of a small integer v in [-128, 127] (exact).
__device__ __forceinline__ uint32_t bf16_of_small_int(int v) {
  if (v == 0) return 0;
  const uint32_t s = v < 0 ? 0x8000u : 0u;
  const uint32_t a = (uint32_t)(v < 0 ? -v : v);  // 1..128
  const uint32_t e = 31 - __clz(a);                // 0..7
  return s | ((127 + e) << 7) | ((a << (7 - e)) & 0x7Fu);
}

// Signed (balanced) base-256 digits of a canonical element (< 2^255), packed
// as bf16 pairs: out[w] = digit 2w | digit 2w+1 << 16.
__device__ __forceinline__ void signed_digits_bf16(uint32_t out[16], const uint32_t x[8]) {
  int carry = 0;
#pragma unroll
  for (int w = 0; w < 16; ++w) {
    uint32_t pair = 0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int b = 2 * w + j;
      int d = (int)((x[b >> 2] >> (8 * (b & 3))) & 0xFFu) + carry;
      carry = d >= 128 ? 1 : 0;
      d -= carry << 8;
      pair |= bf16_of_small_int(d) << (16 * j);
    }
    out[w] = pair;
  }
}

// Exact integer of an fp32 accumulator with |v| <= 2^22.
__device__ __forceinline__ int acc_to_int(uint32_t bits) {
  return __float_as_int(__uint_as_float(bits) + 12582912.0f) - 0x4B400000;
}

// y = REDC(sum_h acc[h] 2^(8h) + offset) for the 32 accumulators of one output.
template <class F>
__device__ __forceinline__ void merge_reduce(uint32_t y[8], const uint32_t acc_bits[32], const uint32_t offset[9]) {
  int64_t col[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    col[l] = (int64_t)acc_to_int(acc_bits[4 * l]) + ((int64_t)acc_to_int(acc_bits[4 * l + 1]) << 8) +
             ((int64_t)acc_to_int(acc_bits[4 * l + 2]) << 16) + ((int64_t)acc_to_int(acc_bits[4 * l + 3]) << 24);
  }
  uint32_t t[9];
  int64_t carry = 0;
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    const int64_t v = col[l] + (int64_t)offset[l] + carry;
    t[l] = (uint32_t)v;
    carry = v >> 32;
  }
  t[8] = (uint32_t)((int64_t)offset[8] + carry);
  // Montgomery reduction of the 9-limb value (< 2^274 < p * 2^256)
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t m = mont_m<F>(t[0]);
    row_even_p<F>(t, m);
    row_odd_p<F>(t, m);
#pragma unroll
    for (int j = 0; j < 8; ++j) t[j] = t[j + 1];
    t[8] = 0;
  }
  reduce_once<F>(y, t);
}

__device__ __forceinline__ uint64_t mat_global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One matrix pass: persistent CTAs (one per SM) loop over tiles of 128
// sub-transforms.  MODE as in ntt_pass.cuh (input multiplier variants).
template <class F, int LOGS, int MODE>
__global__ void __launch_bounds__(kMatThreads, 1) ntt_matrix_pass_kernel(const MatrixPassArgs ma) {
  constexpr uint32_t S = 1u << LOGS;
  constexpr uint32_t K = 32 * S;                 // (n, b)
  constexpr uint32_t NCOL = 32 * S;              // (k, h)
  constexpr uint32_t TMEM_COLS = NCOL < 32 ? 32 : NCOL;
  constexpr uint32_t E_BYTES = NCOL * K * 2;
  constexpr uint32_t A_BYTES = kMatRows * K * 2;
  static_assert(NCOL <= 256, "one MMA per K step");
  static_assert(E_BYTES + A_BYTES <= 227u * 1024u, "E and the A tile fit in shared memory");
  extern __shared__ __align__(1024) uint8_t mat_smem[];
  uint8_t *sE = mat_smem;
  uint8_t *sA = mat_smem + E_BYTES;                   // also the output staging area
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ int s_abort;
  const PassArgs &a = ma.a;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // resident E
  for (uint32_t i = tid; i < E_BYTES / 16; i += kMatThreads)
    reinterpret_cast<uint4 *>(sE)[i] = __ldg(ma.e + i);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_taddr)),
                 "n"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = s_taddr;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((NCOL >> 3) << 17) | ((uint32_t)(kMatRows >> 4) << 24);
  const uint64_t num_tiles = (a.num_sub + kMatRows - 1) / kMatRows;
  const uint64_t mp_mask = (1ull << a.log_mp) - 1;
  uint32_t phase = 0;

  for (uint64_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
    const uint64_t d0 = tile * kMatRows;
    // ---- A: load, multiply, split into signed digits (row m, K range 32n..32n+31)
    for (uint32_t e = tid; e < kMatRows * S; e += kMatThreads) {
      const uint32_t n = e / kMatRows, m = e % kMatRows;   // consecutive threads: consecutive m
      const uint64_t d = d0 + m;
      uint32_t v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (d < a.num_sub) {
        if constexpr (MODE == kModeInner) {
          const uint64_t q = d & mp_mask, o = d >> a.log_mp;
          fe_load_global(v, a.src, q + ((uint64_t)n << a.log_mp) + (o << (a.log_mp + LOGS)));
          uint32_t w[8];
          fe_load_global(w, a.mul, ((uint64_t)n << a.log_mp) + q);
          mont_mul<F>(v, v, w);
        } else {
          fe_load_global(v, a.src, d + ((uint64_t)n << a.log_mp));
          if constexpr (MODE == kModeFirstPre) {
            uint32_t w[8];
            fe_load_global(w, a.mul, n);
            mont_mul<F>(v, v, w);
          }
        }
      }
      uint32_t dg[16];
      signed_digits_bf16(dg, v);
#pragma unroll
      for (int c = 0; c < 4; ++c) {   // 4 core-matrix rows of 8 digits each
        *reinterpret_cast<uint4 *>(sA + core_offset(m, 32 * n + 8 * c, K)) =
            make_uint4(dg[4 * c], dg[4 * c + 1], dg[4 * c + 2], dg[4 * c + 3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- tensor cores: acc[m][(k,h)] = sum over K of A[m][(n,b)] * E[(k,h)][(n,b)]
    if (tid == 0) {
      const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sE);
      const uint32_t sbo = (K >> 3) * 128;
#pragma unroll 1
      for (uint32_t ks = 0; ks < K / 16; ++ks) {
        const uint64_t da = mat_desc(a0 + ks * 256, 128, sbo);
        const uint64_t db = mat_desc(b0 + ks * 256, 128, sbo);
        const uint32_t accum = ks ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
            "l"(da), "l"(db), "r"(idesc), "r"(accum));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(&s_mbar)));
    }
    // ---- bounded wait for the MMAs
    {
      uint32_t done = 0;
      const uint64_t t0 = mat_global_ns();
      for (;;) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(&s_mbar)), "r"(phase));
        if (done || mat_global_ns() - t0 > ma.wait_ns) break;
      }
      if (!done) {
        atomicCAS(ma.err, 0u, (uint32_t)NTT_ERR_TIMEOUT);
        s_abort = 1;
      }
    }
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (s_abort) break;
    // ---- epilogue: warps w, w+4, w+8, w+12 share TMEM lanes 32*(w%4)..; they
    // split the S outputs of each row.
    {
      const uint32_t lg = warp & 3, part = warp >> 2;  // part in 0..3
      const uint32_t m = 32 * lg + lane;
      for (uint32_t k = part; k < S; k += 4) {
        uint32_t r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr + ((32 * lg) << 16) + 32 * k));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        uint32_t y[8];
        merge_reduce<F>(y, r, ma.offset);
        tile_store(reinterpret_cast<uint4 *>(sA), m * S + k, y);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // ---- store phase: element (m, k) of the tile
    for (uint32_t e = tid; e < kMatRows * S; e += kMatThreads) {
      if constexpr (MODE == kModeInner) {
        const uint32_t k = e / kMatRows, m = e % kMatRows;
        const uint64_t d = d0 + m;
        if (d < a.num_sub) {
          const uint64_t q = d & mp_mask, o = d >> a.log_mp;
          const uint64_t pos = q + ((uint64_t)k << a.log_mp) + (o << (a.log_mp + LOGS));
          uint32_t v[8];
          tile_load(v, reinterpret_cast<const uint4 *>(sA), m * S + k);
          if (a.post) post_mul<F>(v, a.post, pos);
          fe_store_global(a.dst, pos, v);
        }
      } else {
        const uint32_t m = e / S, k = e % S;
        const uint64_t d = d0 + m;
        if (d < a.num_sub) {
          const uint64_t rev = reverse_digits(a, d);
          uint32_t v[8];
          tile_load(v, reinterpret_cast<const uint4 *>(sA), m * S + k);
          if (a.post) post_mul<F>(v, a.post, (rev << LOGS) | k);
          fe_store_global(a.dst, (rev << LOGS) | k, v);
        }
      }
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(TMEM_COLS));
  }
}

template <int LOGS>
constexpr int matrix_smem_bytes() {
  return (32 << LOGS) * (32 << LOGS) * 2 + kMatRows * (32 << LOGS) * 2;
}

}  // namespace gb300ntt
