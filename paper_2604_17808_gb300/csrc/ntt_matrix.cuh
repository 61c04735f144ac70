// ntt_matrix.cuh -- matrix-form sub-transforms on the tcgen05 tensor cores.
//
// The paper's reformulation (Sec. 3.2.3-3.2.4, Alg. 1; Sec. 3.3.2, Fig. 5b-c):
// high-precision modular arithmetic becomes a low-precision matrix product
// over byte limbs (ByteDecompose -> byte "Einsum" against a precomputed byte
// matrix -> ByteMerge), and the NTT's sub-transforms become products with
// twiddle matrices.  One pass of the multi-pass NTT computes, for 128
// sub-transforms of S points at once (S = 2, 4 or 8),
//
//   y_k = sum_n V[n,k] x_n,   V[n,k] = pre_n omega_S^(nk)   (pre_n: pass-0
//         coset / scale factors folded in; 1 for the other passes)
//   x_n = sum_b (a_{n,b} + 128) 2^(8b),   a_{n,b} = byte b of x_n - 128
//   W[(n,b),k] = V[n,k] 2^(8b) 2^32 mod p  = sum_h E[(k,h),(n,b)] 2^(8h)
//                 (E: balanced signed byte digits of W, in [-128, 127])
//   acc[k,h] = sum_{n,b} a_{n,b} E[(k,h),(n,b)]     <- tcgen05.mma kind::f16
//   Z_k = sum_h (acc[k,h] + 2^23 1.5 (as fp32 bits)) 2^(8h) + O_k
//       = 2^32 y_k (mod p),   O_k = (2^32 C sum_n V[n,k] - B sum_h 2^(8h)) mod p
//   out = Z_k * T * 2^-288 mod p                      <- 9-row Montgomery
//
// where C = 128 sum_b 2^(8b) undoes the digit offset and B = 0x4B400000 is
// the fp32 bit pattern of 1.5 * 2^23.  T is the Montgomery form c 2^256 of the
// factor the element needs next: the NEXT pass's inter-pass twiddle (looked
// up by the output position), the coset inverse's s^-n in the last pass, or
// 1.  So the inter-pass twiddle product of the paper's 3-/5-step NTT is fused
// with the reduction of the ByteMerge result: one Montgomery product per
// element per pass, nothing else on the integer multiply pipe.
//
// Exactness: |a E| <= 2^14 and K = 32 S <= 256 terms keep every partial sum
// within 2^22; fp16 holds the byte digits exactly (integers up to 2^11).
// Each accumulator starts at the bias 1.5 * 2^23 (written into TMEM by the
// epilogue), so every running value the tensor core forms is an integer in
// [2^23, 2^24], exact in fp32, and the final fp32 bit pattern is 0x4B400000
// + acc: the accumulators are read as integers with no conversion at all.
// Z < 2^31 2^248 (256/255) + p < 2^280, so the 9-row Montgomery product (R =
// 2^288) of Z and T < p ends below 2p; the last pass (no factor) uses a
// Barrett reduction instead, which also ends below 2p.  Only the last pass
// subtracts p once more to make its outputs canonical: a value in [0, 2p) is
// below 2^256, and a pass takes the bytes of any 256-bit input (its digits,
// offsets and bounds do not assume x < p).
//
// Folded passes (early passes: few q, many rows each): the rows d = q + o Mp
// of a tile share q, and the pass's own input factors c(q, n) are folded
// into E_q (V[n,k] c(q, n) in place of V[n,k]) with per-q offsets; the pass
// before needs no factor and ends in Barrett.
//
// Kernel structure (persistent, one CTA per SM, warp-specialised):
//   warp 0       MMA issuer: two tcgen05.mma (K = 16 each) per chunk into a
//                double-buffered TMEM accumulator (N = 32 S columns each);
//                also loads E by cp.async.bulk (E_q of a folded pass, again
//                whenever q changes, once the MMAs reading the previous one
//                are complete);
//   warps 1-3    converter-loaders: chunk g (the 128 rows of one input n of
//                a tile, whatever their stride) is loaded by one tensor-map
//                copy (cp.async.bulk.tensor) into a staging ring and
//                converted -- staging element -> 32 fp16 digits by byte
//                permutes (0x64 | byte = 1024 + byte as fp16) and one packed
//                fp16 subtraction -- into the A operand ring, both by warp
//                g mod 3 (four rows per thread), which issues the copy of
//                chunk g + 12 into the slot once its lanes have read it;
//   warps 4-19   epilogue: tcgen05.ld of one output's 32 accumulators (and
//                tcgen05.st of the bias back into them for the buffer's next
//                tile), ByteMerge by funnel shifts and carry chains, the
//                Montgomery product with T (or Barrett), store.
// Every wait is an mbarrier wait bounded by %globaltimer; on timeout the CTA
// records NTT_ERR_TIMEOUT, every role stops, copies in flight are waited for
// (bounded) and TMEM is freed before the kernel returns.
#pragma once

#include <cuda.h>   // CUtensorMap (the kernel's TMA descriptor parameter)

#include <cstdint>

#include "../../include/ntt_gb300.h"
#include "fp256.cuh"
#include "ntt_pass.cuh"

namespace gb300ntt {

constexpr int kMatRows = 128;                 // sub-transforms per tile (MMA M)
// Converter warps (1-3, one on each of three SM sub-partitions; the MMA
// warp is on the fourth): chunk g goes to converter g mod 3, which also
// loads it, so every ring slot always belongs to the same converter.
constexpr int kMatConvWarps = 3;
constexpr int kMatEpiWarps = 16;              // four per TMEM lane quarter
constexpr int kMatFirstEpiWarp = 1 + kMatConvWarps;
// 20 warps: five per SM sub-partition, so up to 102 registers per thread
// fit its 16K-entry register file (22 warps would cap them at 80)
constexpr int kMatThreads = 32 * (kMatFirstEpiWarp + kMatEpiWarps);   // 640
// Chunks in flight: the staging ring covers the latency of the input loads
// from HBM (12 x 4 KiB, one and a half tiles ahead); the A-operand ring the
// hand-off from the converters to the MMA issuer, two slots per converter so
// that it converts its next chunk while the MMAs read the last one.  Both
// are multiples of the converter count.
constexpr int kMatStageRing = 12;
constexpr int kMatRing = 6;
constexpr uint32_t kMatChunkBytes = kMatRows * 32 * 2;   // A chunk: 128 rows x 32 fp16 digits
constexpr uint32_t kMatStageBytes = kMatRows * 32;       // staging: 128 elements
constexpr uint32_t kMatFp32Magic = 0x4B400000u;          // bits of 1.5 * 2^23

struct MatrixPassArgs {
  PassArgs a;             // src, dst, num_sub, log_mp, digits (mul, dft_tw, post unused)
  const uint4 *e;         // E, fp16, B-operand layout (N x K = 32 S x 32 S)
  const uint4 *next;      // epilogue factor table indexed by pos mod 2^next_log, or null
  const uint4 *post;      // epilogue factor table indexed by pos (coset inverse), or null
  uint32_t next_log;
  uint32_t off[8][8];     // O_k (canonical), k < S
  uint32_t one[8];        // 2^256 mod p: the factor when no table applies
  uint32_t barrett;       // 1: no factor, E without the 2^32: Barrett reduction
  uint64_t mu;            // floor(2^288 / p)
  // Folded passes: all 128 rows of a tile share the index q (d = q + o Mp,
  // 128 consecutive o), so the pass's own input factors, which depend on
  // (q, n) only, are folded into a per-q matrix E_q (e: Mp matrices of E
  // bytes each) with per-q merge offsets (off_fold: S x 8 words per q).
  // The CTAs work in groups of fold_group: CTA i of a group takes q = i
  // (mod fold_group) of the same o blocks at the same time, so the group's
  // 32-byte rows of neighbouring q meet in L2 as whole lines.
  uint32_t fold;
  uint32_t fold_group;
  uint32_t tiles_per_q_log;   // log2 of the 128-row blocks of o per q
  const uint32_t *off_fold;
  uint32_t lazy;          // 1: outputs left in [0, 2p) (every pass but the last)
  uint32_t *err;          // device error word
  uint64_t wait_ns;       // bound of every wait
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

// Byte offset of element (row, col) of a K-major 16-bit operand with K
// columns (core matrices of 8 rows x 16 bytes, K-direction neighbours 128
// bytes apart, 8-row groups K/8 * 128 bytes apart).
__host__ __device__ __forceinline__ uint32_t core_offset(uint32_t row, uint32_t col, uint32_t K) {
  return ((row >> 3) * (K >> 3) + (col >> 3)) * 128 + (row & 7) * 16 + (col & 7) * 2;
}

__device__ __forceinline__ uint64_t mat_global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// The same test, but the thread may sleep in hardware (up to about 0.1 ms)
// until the phase completes, instead of issuing instructions while it polls.
__device__ __forceinline__ bool mbar_try_sleep(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity), "r"(100000u)
      : "memory");
  return done != 0;
}

// Wait for completion of the phase of `bar` with the given parity, bounded
// by wait_ns; gives up early when another role has aborted.  On timeout the
// CTA's abort flag and the device error word are set.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, const MatrixPassArgs &ma,
                                          volatile int *abort) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = mat_global_ns();
  for (;;) {
    if (mbar_try_sleep(bar, parity)) return true;
    if (*abort) return false;
    if (mat_global_ns() - t0 > ma.wait_ns) {
      *abort = 1;
      atomicCAS(ma.err, 0u, (uint32_t)NTT_ERR_TIMEOUT);
      return false;
    }
  }
}

// Global -> shared bulk copy (TMA, this GPU's memory only, no multicast),
// completing on `bar` (bytes counted by its expect_tx).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Tensor-map (TMA) load of a 4-D box into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

// 32 fp16 digits (byte - 128) of one element, packed in 16 words: word 2i
// holds bytes 4i, 4i+1 of limb i, word 2i+1 bytes 4i+2, 4i+3.  The byte
// permute builds the fp16 pattern 0x64bb = 1024 + byte; subtracting 1152
// (0x6480) in packed fp16 leaves byte - 128 exactly.
__device__ __forceinline__ void digits_f16(uint32_t w[16], const uint32_t x[8]) {
  const uint32_t k1152 = 0x64806480u, k64 = 0x64646464u;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    uint32_t lo, hi;
    asm("prmt.b32 %0, %1, %2, 0x4140;" : "=r"(lo) : "r"(x[i]), "r"(k64));
    asm("prmt.b32 %0, %1, %2, 0x4342;" : "=r"(hi) : "r"(x[i]), "r"(k64));
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(w[2 * i]) : "r"(lo), "r"(k1152));
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(w[2 * i + 1]) : "r"(hi), "r"(k1152));
  }
}

// 32 consecutive TMEM columns of this warp's 32 lanes into r (completes at
// the next tcgen05.wait::ld).
__device__ __forceinline__ void tmem_ld32(uint32_t r[32], uint32_t taddr) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// Write the bias 1.5 * 2^23 (fp32 bits 0x4B400000) into 32 consecutive TMEM
// columns of this warp's 32 lanes: accumulating on top of it, every MMA
// result is already the pattern 0x4B400000 + acc (see the header).
__device__ __forceinline__ void tmem_store_bias(uint32_t taddr) {
  const uint32_t b = kMatFp32Magic;
#pragma unroll
  for (uint32_t c = 0; c < 32; c += 8)
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr + c), "r"(b)
                 : "memory");
}

// Z = sum_h u_h 2^(8h) + off, u_h = fp32 bits of acc_h + 1.5 2^23 (< 2^31).
// Four non-overlapping 9-limb terms: A = u_{4l} at limb l, and for the
// byte shifts 8, 16, 24 the funnel-shifted limbs (u_{4l+j} << 8j) |
// (u_{4l+j-4} >> (32 - 8j)); summed with carry chains.
__device__ __forceinline__ void byte_merge(uint32_t z[9], const uint32_t u[32], const uint32_t off[8]) {
  uint32_t b[9], c[9], d[9];
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const uint32_t b_lo = l < 8 ? u[4 * l + 1] : 0u, b_hi = l > 0 ? u[4 * l - 3] : 0u;
    const uint32_t c_lo = l < 8 ? u[4 * l + 2] : 0u, c_hi = l > 0 ? u[4 * l - 2] : 0u;
    const uint32_t d_lo = l < 8 ? u[4 * l + 3] : 0u, d_hi = l > 0 ? u[4 * l - 1] : 0u;
    b[l] = __funnelshift_l(b_hi, b_lo, 8);
    c[l] = __funnelshift_l(c_hi, c_lo, 16);
    d[l] = __funnelshift_l(d_hi, d_lo, 24);
  }
  asm("add.cc.u32  %0, %9,  %18;\n\t"
      "addc.cc.u32 %1, %10, %19;\n\t"
      "addc.cc.u32 %2, %11, %20;\n\t"
      "addc.cc.u32 %3, %12, %21;\n\t"
      "addc.cc.u32 %4, %13, %22;\n\t"
      "addc.cc.u32 %5, %14, %23;\n\t"
      "addc.cc.u32 %6, %15, %24;\n\t"
      "addc.cc.u32 %7, %16, %25;\n\t"
      "addc.u32    %8, %17, %26;"
      : "=r"(z[0]), "=r"(z[1]), "=r"(z[2]), "=r"(z[3]), "=r"(z[4]), "=r"(z[5]), "=r"(z[6]), "=r"(z[7]), "=r"(z[8])
      : "r"(u[0]), "r"(u[4]), "r"(u[8]), "r"(u[12]), "r"(u[16]), "r"(u[20]), "r"(u[24]), "r"(u[28]), "r"(0u),
        "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]));
  asm("add.cc.u32  %0, %0, %9;\n\t"
      "addc.cc.u32 %1, %1, %10;\n\t"
      "addc.cc.u32 %2, %2, %11;\n\t"
      "addc.cc.u32 %3, %3, %12;\n\t"
      "addc.cc.u32 %4, %4, %13;\n\t"
      "addc.cc.u32 %5, %5, %14;\n\t"
      "addc.cc.u32 %6, %6, %15;\n\t"
      "addc.cc.u32 %7, %7, %16;\n\t"
      "addc.u32    %8, %8, %17;"
      : "+r"(z[0]), "+r"(z[1]), "+r"(z[2]), "+r"(z[3]), "+r"(z[4]), "+r"(z[5]), "+r"(z[6]), "+r"(z[7]), "+r"(z[8])
      : "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(c[5]), "r"(c[6]), "r"(c[7]), "r"(c[8]));
  asm("add.cc.u32  %0, %0, %9;\n\t"
      "addc.cc.u32 %1, %1, %10;\n\t"
      "addc.cc.u32 %2, %2, %11;\n\t"
      "addc.cc.u32 %3, %3, %12;\n\t"
      "addc.cc.u32 %4, %4, %13;\n\t"
      "addc.cc.u32 %5, %5, %14;\n\t"
      "addc.cc.u32 %6, %6, %15;\n\t"
      "addc.cc.u32 %7, %7, %16;\n\t"
      "addc.u32    %8, %8, %17;"
      : "+r"(z[0]), "+r"(z[1]), "+r"(z[2]), "+r"(z[3]), "+r"(z[4]), "+r"(z[5]), "+r"(z[6]), "+r"(z[7]), "+r"(z[8])
      : "r"(d[0]), "r"(d[1]), "r"(d[2]), "r"(d[3]), "r"(d[4]), "r"(d[5]), "r"(d[6]), "r"(d[7]), "r"(d[8]));
  asm("add.cc.u32  %0, %0, %9;\n\t"
      "addc.cc.u32 %1, %1, %10;\n\t"
      "addc.cc.u32 %2, %2, %11;\n\t"
      "addc.cc.u32 %3, %3, %12;\n\t"
      "addc.cc.u32 %4, %4, %13;\n\t"
      "addc.cc.u32 %5, %5, %14;\n\t"
      "addc.cc.u32 %6, %6, %15;\n\t"
      "addc.cc.u32 %7, %7, %16;\n\t"
      "addc.u32    %8, %8, 0;"
      : "+r"(z[0]), "+r"(z[1]), "+r"(z[2]), "+r"(z[3]), "+r"(z[4]), "+r"(z[5]), "+r"(z[6]), "+r"(z[7]), "+r"(z[8])
      : "r"(off[0]), "r"(off[1]), "r"(off[2]), "r"(off[3]), "r"(off[4]), "r"(off[5]), "r"(off[6]), "r"(off[7]));
}

// r = z * t * 2^-288 mod p for z < 2^280 (nine limbs) and canonical t: the
// CIOS rows of mont_mul (fp256.cuh) over the nine limbs of z.  The running
// value stays below 2^288 (as in mont_mul: t < p, one limb of z per row) and
// the result is below 2p; one conditional subtraction makes it canonical
// (lazy: left in [0, 2p) for a pass that is not the last).
template <class F>
__device__ __forceinline__ void mont_mul_z9(uint32_t r[8], const uint32_t z[9], const uint32_t t[8], bool lazy) {
  uint32_t acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    row_even(acc, t, z[i]);
    row_odd(acc, t, z[i]);
    const uint32_t m = mont_m<F>(acc[0]);
    row_even_p<F>(acc, m);
    row_odd_p<F>(acc, m);
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = acc[j + 1];
    acc[8] = 0;
  }
  if (lazy) {
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = acc[j];   // in [0, 2p): the next pass takes any 256-bit input
  } else {
    reduce_once<F>(r, acc);
  }
}

// r = z mod p for z < 2^280 (nine limbs): q = floor(floor(z / 2^224) mu /
// 2^64) with mu = floor(2^288 / p) is floor(z / p) or one less (the
// truncations lose less than 2^-30 + 2^-8), so z - q p lies in [0, 2p) and
// one conditional subtraction makes it canonical (lazy: left in [0, 2p)).
// q < 2^27.
template <class F>
__device__ __forceinline__ void barrett_z9(uint32_t r[8], const uint32_t z[9], uint64_t mu, bool lazy) {
  const uint64_t zt = ((uint64_t)z[8] << 32) | z[7];
  const uint32_t q = (uint32_t)__umul64hi(zt, mu);
  uint32_t qp[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  row_even_p<F>(qp, q);
  row_odd_p<F>(qp, q);
  uint32_t d[8];
  asm("sub.cc.u32  %0, %8,  %16;\n\t"
      "subc.cc.u32 %1, %9,  %17;\n\t"
      "subc.cc.u32 %2, %10, %18;\n\t"
      "subc.cc.u32 %3, %11, %19;\n\t"
      "subc.cc.u32 %4, %12, %20;\n\t"
      "subc.cc.u32 %5, %13, %21;\n\t"
      "subc.cc.u32 %6, %14, %22;\n\t"
      "subc.u32    %7, %15, %23;"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7])
      : "r"(z[0]), "r"(z[1]), "r"(z[2]), "r"(z[3]), "r"(z[4]), "r"(z[5]), "r"(z[6]), "r"(z[7]), "r"(qp[0]),
        "r"(qp[1]), "r"(qp[2]), "r"(qp[3]), "r"(qp[4]), "r"(qp[5]), "r"(qp[6]), "r"(qp[7]));
  if (lazy) {
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = d[j];
  } else {
    reduce_once<F>(r, d);
  }
}

// Position of input n (or, for inner passes, output n) of sub-transform d.
template <int LOGS, int MODE>
__device__ __forceinline__ uint64_t mat_in_pos(const PassArgs &a, uint64_t d, uint32_t n) {
  if constexpr (MODE == kModeInner) {
    const uint64_t q = d & ((1ull << a.log_mp) - 1), o = d >> a.log_mp;
    return q + ((uint64_t)n << a.log_mp) + (o << (a.log_mp + LOGS));
  } else {
    return d + ((uint64_t)n << a.log_mp);
  }
}

template <int LOGS, int MODE>
__device__ __forceinline__ uint64_t mat_out_pos(const PassArgs &a, uint64_t d, uint32_t k) {
  if constexpr (MODE == kModeInner) return mat_in_pos<LOGS, MODE>(a, d, k);
  else return (reverse_digits(a, d) << LOGS) | k;
}

template <int LOGS>
__host__ __device__ constexpr uint32_t matrix_tmem_cols() {
  // two accumulators of 32 S columns, at least 32 columns in all, power of two
  return (64u << LOGS) < 32u ? 32u : (64u << LOGS);
}

template <int LOGS>
__host__ __device__ constexpr int matrix_smem_bytes() {
  return (32 << LOGS) * (32 << LOGS) * 2 + kMatRing * (int)kMatChunkBytes + kMatStageRing * (int)kMatStageBytes;
}

// One matrix pass (MODE: kModeInner or kModeFirst; pass-0 multipliers are
// folded into E).  BARRETT: the pass ends in the Barrett reduction (no
// factor); its epilogue issues the second output's accumulator load before
// the first output's reduction.
template <class F, int LOGS, int MODE, bool BARRETT>
__global__ void __launch_bounds__(kMatThreads, 1)
    ntt_matrix_pass_kernel(const MatrixPassArgs ma, const __grid_constant__ CUtensorMap in_map) {
  constexpr uint32_t S = 1u << LOGS;
  constexpr uint32_t K = 32 * S;                  // (n, b)
  constexpr uint32_t NC = 32 * S;                 // (k, h)
  constexpr uint32_t TMEM_COLS = matrix_tmem_cols<LOGS>();
  constexpr uint32_t E_BYTES = NC * K * 2;
  static_assert(NC <= 256 && NC % 16 == 0, "one MMA covers all outputs");
  static_assert(matrix_smem_bytes<LOGS>() <= 227 * 1024 - 1024, "shared memory");
  static_assert(kMatRing % kMatConvWarps == 0 && kMatStageRing % kMatConvWarps == 0, "slots of one converter");
  static_assert(kMatFirstEpiWarp == 4, "epilogue warps start on sub-partition 0");
  extern __shared__ __align__(1024) uint8_t mat_smem[];
  uint8_t *sE = mat_smem;
  uint8_t *sA = mat_smem + E_BYTES;
  uint8_t *sStage = sA + kMatRing * kMatChunkBytes;
  __shared__ __align__(8) uint64_t bar_e;
  __shared__ __align__(8) uint64_t stage_full[kMatStageRing], stage_empty[kMatStageRing];
  __shared__ __align__(8) uint64_t chunk_full[kMatRing], chunk_empty[kMatRing];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
  __shared__ __align__(8) uint64_t bar_done, bar_efree;
  __shared__ uint32_t s_taddr;
  __shared__ int s_abort;
  volatile int *abort = &s_abort;
  const PassArgs &a = ma.a;
  const bool lazy = ma.lazy != 0;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // Work units: tiles (128 consecutive rows d) of the plain pass; for a
  // folded pass (q group, o block) pairs of the CTA's group.  Each CTA takes
  // a contiguous range of units, so a folded pass changes q, and reloads E,
  // only a few times per CTA.
  const uint32_t groups = ma.fold ? gridDim.x / ma.fold_group : gridDim.x;
  const uint32_t group = ma.fold ? blockIdx.x / ma.fold_group : blockIdx.x;
  const uint32_t in_group = ma.fold ? blockIdx.x % ma.fold_group : 0;
  const uint64_t num_units = ma.fold ? ((1ull << a.log_mp) / ma.fold_group) << ma.tiles_per_q_log
                                     : (a.num_sub + kMatRows - 1) / kMatRows;
  const uint64_t u_begin = group < groups ? num_units * group / groups : 0;
  const uint64_t my_tiles = group < groups ? num_units * (group + 1) / groups - u_begin : 0;
  const uint64_t mp_mask = (1ull << a.log_mp) - 1;
  // q of unit u (folded passes), first row d of its tile and the step
  // between the tile's rows (the rows are d0 + m * step, m < 128)
  auto tile_q = [&](uint64_t u) -> uint64_t {
    return ma.fold ? (u >> ma.tiles_per_q_log) * ma.fold_group + in_group : 0;
  };
  auto tile_d0 = [&](uint64_t u) -> uint64_t {
    const uint64_t ob = u & ((1ull << ma.tiles_per_q_log) - 1);
    return ma.fold ? tile_q(u) + ((ob * kMatRows) << a.log_mp) : u * kMatRows;
  };
  const uint64_t row_step = ma.fold ? (1ull << a.log_mp) : 1;

  if (tid == 0) {
    mbar_init(&bar_e, 1);
    for (int i = 0; i < kMatStageRing; ++i) {
      mbar_init(&stage_full[i], 1);
      mbar_init(&stage_empty[i], 32);   // the lanes of the slot's converter warp
    }
    for (int i = 0; i < kMatRing; ++i) {
      mbar_init(&chunk_full[i], 32);
      mbar_init(&chunk_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 32 * kMatEpiWarps);
    }
    mbar_init(&bar_done, 1);
    mbar_init(&bar_efree, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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

  uint64_t e_issued = 0;       // (MMA thread) E loads, for the teardown
  uint64_t loads_issued = 0;   // (converter lane 0) last chunk it loaded + 1, for the teardown
  const uint32_t cw = warp - 1;   // converter index (warps 1 .. kMatConvWarps)
  // E (of a folded pass: E_q) into shared memory, completing on bar_e
  auto load_e = [&](uint64_t q) {
    const uint8_t *src = reinterpret_cast<const uint8_t *>(ma.e) + q * (uint64_t)E_BYTES;
    mbar_expect_tx(&bar_e, E_BYTES);
    for (uint32_t off = 0; off < E_BYTES; off += 16384u) {
      const uint32_t bytes = E_BYTES - off < 16384u ? E_BYTES - off : 16384u;
      bulk_g2s(sE + off, src + off, bytes, &bar_e);
    }
  };
  // Chunk g (input g mod S of tile g / S) into staging slot g mod
  // kMatStageRing: one tensor-map copy of the tile's 128 rows of that input,
  // whatever their stride in memory.
  const uint32_t chunk_bytes = (uint32_t)(a.num_sub < (uint64_t)kMatRows ? a.num_sub : kMatRows) * 32u;
  auto load_chunk = [&](uint64_t g) {
    const uint32_t sl = (uint32_t)(g % kMatStageRing);
    const uint64_t d0 = tile_d0(u_begin + g / S);
    mbar_expect_tx(&stage_full[sl], chunk_bytes);
    tma_load_4d(sStage + sl * kMatStageBytes, &in_map, 0, (int)(d0 & mp_mask), (int)(g % S), (int)(d0 >> a.log_mp),
                &stage_full[sl]);
  };
  const uint64_t chunks = my_tiles * S;
  // E and the factor tables are plan constants: the first E is requested
  // before the wait for the previous launch (programmatic dependent launch),
  // every access to the vector comes after it.
  if (tid == 0 && my_tiles) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&in_map)) : "memory");
    load_e(tile_q(u_begin));
    e_issued = 1;
  }
  pdl_trigger_and_wait();

  if (warp == 0) {
    // ------------------------------------------------------ MMA issuer
    // Lane 0; for a folded pass also E_q again whenever q changes, once the
    // MMAs reading the previous E are complete.
    if (lane == 0) {
      // fp32 accumulate (bit 4), fp16 A and B (formats 0), K-major both,
      // N >> 3 at bit 17, M >> 4 at bit 24
      constexpr uint32_t idesc = (1u << 4) | ((NC >> 3) << 17) | ((uint32_t)(kMatRows >> 4) << 24);
      bool ok = true;
      uint64_t e_used = 0;   // E loads consumed
      const uint32_t a_base = smem_addr(sA), b_base = smem_addr(sE);
      uint64_t g = 0;
      for (uint64_t it = 0; ok && it < my_tiles; ++it) {
        const uint64_t t = u_begin + it;
        const bool new_e = it == 0 || (ma.fold && tile_q(t) != tile_q(t - 1));
        if (it > 0 && new_e) {
          if (!mbar_wait(&bar_efree, (uint32_t)((e_issued - 1) & 1), ma, abort)) break;
          load_e(tile_q(t));
          ++e_issued;
        }
        if (new_e) {
          if (!mbar_wait(&bar_e, (uint32_t)(e_used & 1), ma, abort)) break;
          ++e_used;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        const uint32_t buf = (uint32_t)(it & 1);
        const uint64_t v = it >> 1;
        if (!mbar_wait(&acc_empty[buf], (uint32_t)(v & 1), ma, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dcol = taddr + buf * NC;
        for (uint32_t n = 0; n < S; ++n, ++g) {
          const uint32_t c = (uint32_t)(g % kMatRing);
          const uint64_t u = g / kMatRing;
          if (!mbar_wait(&chunk_full[c], (uint32_t)(u & 1), ma, abort)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (uint32_t ks = 0; ks < 2; ++ks) {
            const uint64_t da = mat_desc(a_base + c * kMatChunkBytes + ks * 256, 128, 4 * 128);
            const uint64_t db = mat_desc(b_base + (2 * n + ks) * 256, 128, (K >> 3) * 128);
            const uint32_t accum = 1u;   // on top of the bias the epilogue wrote
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
                "l"(da), "l"(db), "r"(idesc), "r"(accum));
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_addr(&chunk_empty[c]))
                       : "memory");
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&acc_full[buf]))
                     : "memory");
        // the last tile of a q: E may be replaced once these MMAs are done
        if (ma.fold && it + 1 < my_tiles && tile_q(t + 1) != tile_q(t))
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_addr(&bar_efree))
                       : "memory");
      }
    }
  } else if (warp < kMatFirstEpiWarp) {
    // ------------------------------------------------------ converter-loaders
    // Converter cw takes the chunks g = cw, cw + 3, ... (staging and operand
    // slots g mod 12 and g mod 6: always its own), each thread the rows
    // lane, lane + 32, lane + 64, lane + 96; lane 0 loads the converter's
    // chunks, the next one into a slot as soon as the warp has read it.
    if (lane == 0)
      for (uint64_t g = cw; g < chunks && g < (uint64_t)kMatStageRing; g += kMatConvWarps) {
        load_chunk(g);
        loads_issued = g + 1;
      }
    for (uint64_t g = cw; g < chunks && !*abort; g += kMatConvWarps) {
      const uint32_t sl = (uint32_t)(g % kMatStageRing);
      const uint64_t us = g / kMatStageRing;
      const uint32_t c = (uint32_t)(g % kMatRing);
      const uint64_t u = g / kMatRing;
      if (!mbar_wait(&stage_full[sl], (uint32_t)(us & 1), ma, abort)) break;
      if (u >= 1 && !mbar_wait(&chunk_empty[c], (uint32_t)((u - 1) & 1), ma, abort)) break;
      const uint4 *st = reinterpret_cast<const uint4 *>(sStage + sl * kMatStageBytes);
      uint8_t *dst = sA + c * kMatChunkBytes;
#pragma unroll
      for (uint32_t rr = 0; rr < 4; ++rr) {
        const uint32_t m = lane + 32 * rr;
        const uint4 lo = st[2 * m], hi = st[2 * m + 1];
        const uint32_t x[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
        uint32_t w[16];
        digits_f16(w, x);
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q)
          *reinterpret_cast<uint4 *>(dst + core_offset(m, 8 * q, 32)) =
              make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
      }
      // the operand writes before the MMA reads them (async proxy); every
      // lane's staging reads before lane 0 copies the next chunk into the slot
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&stage_empty[sl]);
      mbar_arrive(&chunk_full[c]);
      if (lane == 0 && g + kMatStageRing < chunks) {
        if (!mbar_wait(&stage_empty[sl], (uint32_t)(us & 1), ma, abort)) break;
        load_chunk(g + kMatStageRing);
        loads_issued = g + kMatStageRing + 1;
      }
    }
  } else {
    // ------------------------------------------------------ epilogue
    const uint32_t ew = warp - kMatFirstEpiWarp;   // 0..15
    const uint32_t quarter = warp & 3;              // TMEM lanes 32 quarter .. + 31
    const uint32_t part = ew >> 2;                  // 0..3: outputs k = part, part + 4
    const uint32_t m = 32 * quarter + lane;
    const uint64_t next_mask = (1ull << ma.next_log) - 1;
    const uint32_t lane_addr = taddr + ((32 * quarter) << 16);
    for (uint32_t buf = 0; buf < 2; ++buf) {
#pragma unroll
      for (int o = 0; o < 2; ++o)
        if (part + 4 * o < S) tmem_store_bias(lane_addr + buf * NC + 32 * (part + 4 * o));
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    mbar_arrive(&acc_empty[0]);
    mbar_arrive(&acc_empty[1]);
    // factors of this thread's outputs; a folded pass ending in Barrett
    // needs none and keeps its merge offsets here instead, loaded again only
    // when q changes
    uint32_t fac[2][8];
    uint64_t fac_q = ~0ull;
    if (!ma.post && !ma.next && !ma.fold) {
#pragma unroll
      for (int o = 0; o < 2; ++o)
#pragma unroll
        for (int j = 0; j < 8; ++j) fac[o][j] = ma.one[j];
    }
    for (uint64_t it = 0; it < my_tiles; ++it) {
      const uint32_t buf = (uint32_t)(it & 1);
      const uint64_t u = u_begin + it;
      const uint64_t d = tile_d0(u) + m * row_step;
      const bool live = ma.fold || d < a.num_sub;
      // positions and factors of the outputs k = part and part + 4 are
      // loaded before the accumulators are ready
      uint64_t pos[2] = {0, 0};
      const uint64_t q = tile_q(u);
      const uint4 *offq = reinterpret_cast<const uint4 *>(ma.off_fold + q * S * 8);   // S entries of q
      const bool new_off = BARRETT && ma.fold && q != fac_q;
      fac_q = q;
#pragma unroll
      for (int o = 0; o < 2; ++o) {
        const uint32_t k = part + 4 * o;
        if (k < S && live) {
          pos[o] = mat_out_pos<LOGS, MODE>(a, d, k);
          if (BARRETT && ma.fold) {
            if (new_off) fe_load_global(fac[o], offq, k);
          } else if (ma.post) {
            fe_load_global(fac[o], ma.post, pos[o]);
          } else if (ma.next) {
            fe_load_global(fac[o], ma.next, pos[o] & next_mask);
          }
        }
      }
      if (!mbar_wait(&acc_full[buf], (uint32_t)((it >> 1) & 1), ma, abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      constexpr int kOuts = S > 4 ? 2 : 1;
      if constexpr (BARRETT) {
        // output 0's accumulators, back to the bias, ByteMerge; output 1's
        // load is issued into the same registers before output 0's Barrett
        // reduction, so that its latency hides behind it
        uint32_t r[32];
        tmem_ld32(r, lane_addr + buf * NC + 32 * part);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int o = 0; o < kOuts; ++o) {
          const uint32_t k = part + 4 * o;
          if (k >= S) break;
          if (o > 0) asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          tmem_store_bias(lane_addr + buf * NC + 32 * k);   // for this buffer's next tile
          uint32_t z[9];
          if (ma.fold) byte_merge(z, r, fac[o]);
          else byte_merge(z, r, ma.off[k]);
          if (o + 1 < kOuts && k + 4 < S) tmem_ld32(r, lane_addr + buf * NC + 32 * (k + 4));
          if (live) {
            uint32_t y[8];
            barrett_z9<F>(y, z, ma.mu, lazy);
            fe_store_global(a.dst, pos[o], y);
          }
        }
      } else {
        // each output in turn: its accumulators (back to the bias as they
        // are read), ByteMerge, Montgomery product, store -- one output's
        // values live at a time
#pragma unroll
        for (int o = 0; o < kOuts; ++o) {
          const uint32_t k = part + 4 * o;
          if (k >= S) break;
          uint32_t z[9];
          {
            uint32_t r[32];
            tmem_ld32(r, lane_addr + buf * NC + 32 * k);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            tmem_store_bias(lane_addr + buf * NC + 32 * k);   // for this buffer's next tile
            if (ma.fold) {
              uint32_t off[8];
              fe_load_global(off, offq, k);
              byte_merge(z, r, off);
            } else {
              byte_merge(z, r, ma.off[k]);
            }
          }
          if (live) {
            uint32_t y[8];
            mont_mul_z9<F>(y, z, fac[o], lazy);
            fe_store_global(a.dst, pos[o], y);
          }
        }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&acc_empty[buf]);
    }
  }

  // ---------------------------------------------------------- teardown
  // Every copy into shared memory and every MMA must be complete before the
  // shared memory and TMEM go away.  Normally these waits return at once;
  // after an abort they are bounded like every other wait.
  __syncthreads();
  if (warp >= 1 && warp < kMatFirstEpiWarp && lane == 0) {
    // the last copy into each of this converter's staging slots
    const uint64_t t0 = mat_global_ns();
    for (uint64_t sl = cw; sl < (uint64_t)kMatStageRing && sl < loads_issued; sl += kMatConvWarps) {
      const uint64_t g = sl + ((loads_issued - 1 - sl) / kMatStageRing) * kMatStageRing;
      while (!mbar_try(&stage_full[sl], (uint32_t)((g / kMatStageRing) & 1)) && mat_global_ns() - t0 < ma.wait_ns) {
      }
    }
  }
  if (tid == 0) {
    const uint64_t t0 = mat_global_ns();
    while (e_issued && !mbar_try(&bar_e, (uint32_t)((e_issued - 1) & 1)) && mat_global_ns() - t0 < ma.wait_ns) {
    }
    // a commit tracks every MMA this thread issued before it
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(&bar_done))
                 : "memory");
    while (!mbar_try(&bar_done, 0) && mat_global_ns() - t0 < ma.wait_ns) {
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(TMEM_COLS));
  }
}

}  // namespace gb300ntt
