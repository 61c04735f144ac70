// ntt_rns.cuh -- the paper's RNS lazy modular multiplication on tcgen05.
//
// MORPH (Sec. 3.2.3-3.2.4, Alg. 1 "MXU RNS Lazy") multiplies elements of
// the prime field F_M inside a residue number system over a larger,
// non-prime modulus, so that the product needs no carry chains, and turns
// the reduction modulo M into a low-precision matrix product over bytes
// (ByteDecompose -> Einsum -> ByteMerge) plus a few vector operations.
// This kernel runs that scheme on GB300: the residue work on the CUDA
// cores, the two byte products on the tensor cores.
//
// Representation: an element is an integer in [0, L), L = (sum q + I) M,
// congruent to the field element, carried as its residues in base
// Q = q_0 ... q_{I-1} (31-bit primes, Q > 4 L^2); a second base
// P = p_0 ... p_{J-1} (P > 2^20 L) serves the reduction.  One product:
//
//   xi_i  = x_i y_i (Q/q_i)^-1 mod q_i          two 32-bit Montgomery products
//   k     = floor(sum_i xi_i f_i / 2^58)         the CRT quotient (exact)
//   D1    = A1 E1   (128 x 80) x (80 x 48)       bytes of xi  x  bytes of constants
//   eta_j = (ByteMerge(D1 row) + k g_j) mod p_j  = R (P/p_j)^-1 mod p_j,
//           R = sum_i xi_i ((Q/q_i) mod M) + k (M - Q mod M) == x y (mod M), R < L
//   k2    = floor(sum_j eta_j f2_j / 2^58)
//   D2    = A2 E2   (128 x 48) x (48 x 80)       exact extension of R to base Q
//   r_i   = (ByteMerge(D2 row) + k2 g2_i) mod q_i
//
// One CTA of 128 threads holds 128 elements, one per thread and per TMEM
// lane; each GEMM is one tcgen05.mma.cta_group::1.kind::f16 (bf16 x bf16 ->
// f32, exact: bytes are exact in bf16 and every accumulator stays below
// 2^24) per 16 of K, issued by one thread, accumulators read back with
// tcgen05.ld.  `reps` dependent products per element (out = x y^reps,
// lazily) measure the arithmetic without the memory traffic.
#pragma once

#include <cstdint>

#include "../../include/ntt_gb300.h"
#include "ntt_matrix.cuh"

namespace gb300ntt {

constexpr int kRnsI = 19;          // residues in base Q (both fields)
constexpr int kRnsMaxJ = 11;       // residues in base P (11 for BLS12-381 Fr, 10 for BN254 Fr)
constexpr int kRnsWords = 20;      // 32-bit words per element in memory (80 bytes)
constexpr int kRnsK1 = 80;         // GEMM1 K: 4 bytes x 19 residues, padded to 16
constexpr int kRnsN1 = 48;         // GEMM1 N: 4 bytes x J residues, padded to 16
constexpr int kRnsK2 = 48;         // GEMM2 K
constexpr int kRnsN2 = 80;         // GEMM2 N
constexpr int kRnsThreads = 128;
constexpr int kRnsShift = 58;      // scale of the quotient estimates

struct RnsConst {
  uint32_t q[kRnsI], q_ninv[kRnsI];     // q_i, -q_i^-1 mod 2^32
  uint32_t q_hat_inv_m[kRnsI];          // (Q/q_i)^-1 * 2^64 mod q_i (Montgomery-scaled)
  uint32_t f[kRnsI];                    // ceil(2^58 / q_i)
  uint32_t g2[kRnsI];                   // (-P) mod q_i
  uint64_t q_mu[kRnsI];                 // floor((2^64 - 1) / q_i)
  uint32_t p[kRnsMaxJ], g[kRnsMaxJ], f2[kRnsMaxJ];
  uint64_t p_mu[kRnsMaxJ];
};

struct RnsArgs {
  const uint4 *x, *y;                   // kRnsWords words per element
  uint4 *out;
  uint64_t count;
  uint32_t reps;
  const uint4 *e1;                      // B operand of GEMM1, N1 x K1 bf16, core-matrix layout
  const uint4 *e2;                      // B operand of GEMM2, N2 x K2 bf16
  uint32_t *err;
  uint64_t wait_ns;
};

// x * y * 2^-32 mod q (x, y < q < 2^31): 32-bit Montgomery product.
__device__ __forceinline__ uint32_t rns_mont(uint32_t x, uint32_t y, uint32_t q, uint32_t ninv) {
  const uint64_t t = (uint64_t)x * y;
  const uint32_t m = (uint32_t)t * ninv;
  const uint32_t u = (uint32_t)((t + (uint64_t)m * q) >> 32);
  return u >= q ? u - q : u;
}

// s mod q for s < 2^63, q < 2^31 (Barrett with mu = floor((2^64 - 1) / q)).
__device__ __forceinline__ uint32_t rns_mod64(uint64_t s, uint32_t q, uint64_t mu) {
  const uint64_t qt = __umul64hi(s, mu);
  uint64_t r = s - qt * q;
  if (r >= q) r -= q;
  if (r >= q) r -= q;
  return (uint32_t)r;
}

// bf16 pair of two bytes (exact: 0..255 have at most 8 significant bits).
__device__ __forceinline__ uint32_t bf16x2_of_bytes(uint32_t b0, uint32_t b1) {
  const float f0 = __uint_as_float(0x4B000000u | b0) - 8388608.0f;
  const float f1 = __uint_as_float(0x4B000000u | b1) - 8388608.0f;
  return (__float_as_uint(f0) >> 16) | (__float_as_uint(f1) & 0xFFFF0000u);
}

// The four bytes of w as two bf16 pairs.
__device__ __forceinline__ void bf16_bytes(uint32_t &lo, uint32_t &hi, uint32_t w) {
  lo = bf16x2_of_bytes(w & 0xFFu, (w >> 8) & 0xFFu);
  hi = bf16x2_of_bytes((w >> 16) & 0xFFu, w >> 24);
}

// Exact integer of an fp32 accumulator in [0, 2^23).
__device__ __forceinline__ uint32_t rns_acc(uint32_t bits) {
  return __float_as_uint(__uint_as_float(bits) + 8388608.0f) - 0x4B000000u;
}

__device__ __forceinline__ uint64_t rns_merge4(const uint32_t a[4]) {
  return (uint64_t)rns_acc(a[0]) + ((uint64_t)rns_acc(a[1]) << 8) + ((uint64_t)rns_acc(a[2]) << 16) +
         ((uint64_t)rns_acc(a[3]) << 24);
}

__device__ __forceinline__ void tmem_ld16(uint32_t r[16], uint32_t addr) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
}

// One thread issues the MMAs of a (128 x K) x (K x N) product into TMEM
// columns [col, col + N) and commits them to the mbarrier.
template <int K, int N>
__device__ __forceinline__ void rns_issue_gemm(uint32_t taddr, uint32_t col, const uint8_t *sA, const uint8_t *sB,
                                               uint32_t mbar) {
  constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                             ((uint32_t)(kRnsThreads >> 4) << 24);
  const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
  constexpr uint32_t sbo = (K >> 3) * 128;
#pragma unroll
  for (uint32_t ks = 0; ks < K / 16; ++ks) {
    const uint64_t da = mat_desc(a0 + ks * 256, 128, sbo);
    const uint64_t db = mat_desc(b0 + ks * 256, 128, sbo);
    const uint32_t accum = ks ? 1u : 0u;
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr + col),
        "l"(da), "l"(db), "r"(idesc), "r"(accum));
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

// Bounded wait for the mbarrier phase; false on timeout.
__device__ __forceinline__ bool rns_wait(uint32_t mbar, uint32_t phase, uint64_t wait_ns) {
  const uint64_t t0 = mat_global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(phase));
    if (done) return true;
    if (mat_global_ns() - t0 > wait_ns) return false;
  }
}

template <int J>
__global__ void __launch_bounds__(kRnsThreads, 4) rns_mul_kernel(const RnsArgs args, const RnsConst C) {
  static_assert(4 * J <= kRnsN1 && 4 * J <= kRnsK2, "base P too large for the GEMM shapes");
  constexpr uint32_t E1_BYTES = kRnsN1 * kRnsK1 * 2, E2_BYTES = kRnsN2 * kRnsK2 * 2;
  constexpr uint32_t A1_BYTES = kRnsThreads * kRnsK1 * 2, A2_BYTES = kRnsThreads * kRnsK2 * 2;
  extern __shared__ __align__(1024) uint8_t rns_smem[];
  uint8_t *sE1 = rns_smem, *sE2 = sE1 + E1_BYTES, *sA1 = sE2 + E2_BYTES, *sA2 = sA1 + A1_BYTES;
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ int s_abort;
  const uint32_t tid = threadIdx.x, warp = tid >> 5;

  for (uint32_t i = tid; i < E1_BYTES / 16; i += kRnsThreads) reinterpret_cast<uint4 *>(sE1)[i] = __ldg(args.e1 + i);
  for (uint32_t i = tid; i < E2_BYTES / 16; i += kRnsThreads) reinterpret_cast<uint4 *>(sE2)[i] = __ldg(args.e2 + i);
  // zero the K padding of both A tiles once (columns 76..79 and 4J..47)
  for (uint32_t i = tid; i < A1_BYTES / 16; i += kRnsThreads) reinterpret_cast<uint4 *>(sA1)[i] = make_uint4(0, 0, 0, 0);
  for (uint32_t i = tid; i < A2_BYTES / 16; i += kRnsThreads) reinterpret_cast<uint4 *>(sA2)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_taddr)),
                 "n"(kRnsN1 + kRnsN2));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = s_taddr;
  const uint32_t lane_addr = taddr + ((32u * warp) << 16);
  const uint32_t mbar = smem_addr(&s_mbar);
  uint32_t phase = 0;
  const uint64_t num_tiles = (args.count + kRnsThreads - 1) / kRnsThreads;

  for (uint64_t tile = blockIdx.x; tile < num_tiles && !s_abort; tile += gridDim.x) {
    const uint64_t e = tile * kRnsThreads + tid;
    const bool live = e < args.count;
    uint32_t x[kRnsWords], y[kRnsWords];
#pragma unroll
    for (int w = 0; w < kRnsWords / 4; ++w) {
      uint4 a = make_uint4(0, 0, 0, 0), b = make_uint4(0, 0, 0, 0);
      if (live) {
        a = __ldg(args.x + e * (kRnsWords / 4) + w);
        b = __ldg(args.y + e * (kRnsWords / 4) + w);
      }
      x[4 * w] = a.x; x[4 * w + 1] = a.y; x[4 * w + 2] = a.z; x[4 * w + 3] = a.w;
      y[4 * w] = b.x; y[4 * w + 1] = b.y; y[4 * w + 2] = b.z; y[4 * w + 3] = b.w;
    }
#pragma unroll 1
    for (uint32_t rep = 0; rep < args.reps; ++rep) {
      // ---- VecMul, CRT digits, quotient estimate; A1 row = bytes of xi
      uint64_t v = 0;
#pragma unroll
      for (int i = 0; i < kRnsI; i += 2) {
        uint32_t lo0, hi0, lo1 = 0, hi1 = 0;
        const uint32_t c0 = rns_mont(x[i], y[i], C.q[i], C.q_ninv[i]);
        const uint32_t xi0 = rns_mont(c0, C.q_hat_inv_m[i], C.q[i], C.q_ninv[i]);
        v += (uint64_t)xi0 * C.f[i];
        bf16_bytes(lo0, hi0, xi0);
        if (i + 1 < kRnsI) {
          const uint32_t c1 = rns_mont(x[i + 1], y[i + 1], C.q[i + 1], C.q_ninv[i + 1]);
          const uint32_t xi1 = rns_mont(c1, C.q_hat_inv_m[i + 1], C.q[i + 1], C.q_ninv[i + 1]);
          v += (uint64_t)xi1 * C.f[i + 1];
          bf16_bytes(lo1, hi1, xi1);
        }
        // K columns 4i .. 4i+7 = one 16-byte core-matrix row
        *reinterpret_cast<uint4 *>(sA1 + core_offset(tid, 4 * i, kRnsK1)) = make_uint4(lo0, hi0, lo1, hi1);
      }
      const uint32_t k = (uint32_t)(v >> kRnsShift);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) rns_issue_gemm<kRnsK1, kRnsN1>(taddr, 0, sA1, sE1, mbar);
      if (!rns_wait(mbar, phase, args.wait_ns)) {
        atomicCAS(args.err, 0u, (uint32_t)NTT_ERR_TIMEOUT);
        s_abort = 1;
      }
      phase ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // ---- ByteMerge + correction: eta_j; A2 row = bytes of eta
      uint32_t eta[J];
      uint64_t v2 = 0;
#pragma unroll
      for (int c = 0; c < kRnsN1 / 16; ++c) {
        uint32_t acc[16];
        tmem_ld16(acc, lane_addr + 16 * c);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int j = 4 * c + t;
          if (j < J) {
            const uint64_t s = rns_merge4(acc + 4 * t) + (uint64_t)k * C.g[j];
            eta[j] = rns_mod64(s, C.p[j], C.p_mu[j]);
            v2 += (uint64_t)eta[j] * C.f2[j];
          }
        }
      }
      const uint32_t k2 = (uint32_t)(v2 >> kRnsShift);
#pragma unroll
      for (int j = 0; j < J; j += 2) {
        uint32_t lo0, hi0, lo1 = 0, hi1 = 0;
        bf16_bytes(lo0, hi0, eta[j]);
        if (j + 1 < J) bf16_bytes(lo1, hi1, eta[j + 1]);
        *reinterpret_cast<uint4 *>(sA2 + core_offset(tid, 4 * j, kRnsK2)) = make_uint4(lo0, hi0, lo1, hi1);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (s_abort) break;
      if (tid == 0) rns_issue_gemm<kRnsK2, kRnsN2>(taddr, kRnsN1, sA2, sE2, mbar);
      if (!rns_wait(mbar, phase, args.wait_ns)) {
        atomicCAS(args.err, 0u, (uint32_t)NTT_ERR_TIMEOUT);
        s_abort = 1;
      }
      phase ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // ---- ByteMerge + correction: r_i in base Q (the next x)
#pragma unroll
      for (int c = 0; c < kRnsN2 / 16; ++c) {
        uint32_t acc[16];
        tmem_ld16(acc, lane_addr + kRnsN1 + 16 * c);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int i = 4 * c + t;
          if (i < kRnsI) {
            const uint64_t s = rns_merge4(acc + 4 * t) + (uint64_t)k2 * C.g2[i];
            x[i] = rns_mod64(s, C.q[i], C.q_mu[i]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (s_abort) break;
    }
    if (live && !s_abort) {
#pragma unroll
      for (int w = 0; w < kRnsWords / 4; ++w)
        args.out[e * (kRnsWords / 4) + w] = make_uint4(x[4 * w], x[4 * w + 1], x[4 * w + 2], x[4 * w + 3]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(kRnsN1 + kRnsN2));
  }
}

constexpr int rns_smem_bytes() {
  return kRnsN1 * kRnsK1 * 2 + kRnsN2 * kRnsK2 * 2 + kRnsThreads * kRnsK1 * 2 + kRnsThreads * kRnsK2 * 2;
}

}  // namespace gb300ntt
