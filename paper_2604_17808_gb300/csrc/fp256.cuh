// fp256.cuh -- 255-bit prime-field arithmetic for sm_103a, 8 x 32-bit limbs.
//
// The paper's arithmetic baseline ("radix Mont", Sec. 2.3.2 and Tab. 1): a
// field element is D = 8 32-bit digits; a multiplication is an O(D^2) digit
// product with carry propagation followed by an O(D^2) Montgomery reduction.
// On a GPU the carry chains are native (mad.lo.cc / madc.hi.cc on the
// integer multiply-add pipe), so this is the hot loop of the butterfly path.
//
// Conventions used throughout the library:
//   * element = uint32_t[8], limb 0 least significant;
//   * data stays in STANDARD form end to end; every constant operand
//     (twiddles, coset powers, N^-1) is stored in MONTGOMERY form c*2^256, so
//     mont_mul(x, c*2^256) = x*c mod p is again standard.  No conversion
//     passes are needed at the ABI boundary;
//   * every value is canonical in [0, p) before and after each operation.
//
// mont_mul is the coarsely integrated operand scanning (CIOS) form of
// Montgomery multiplication (Koc, Acar, Kaliski, "Analyzing and comparing
// Montgomery multiplication algorithms", IEEE Micro 1996), radix 2^32.  With
// a, b < p < 2^255 the running value stays below 2^288, so it fits in nine
// limbs and the last carry of every row is provably zero.
#pragma once

#include <cstdint>

namespace gb300ntt {

constexpr uint32_t neg_inv_u32(uint32_t p0) {
  // Newton iteration for p0^-1 mod 2^32 (p0 odd); each step doubles the
  // number of correct low bits, starting from 3 (p0 * p0 = 1 mod 8).
  uint32_t inv = p0;
  for (int i = 0; i < 5; ++i) inv *= 2u - p0 * inv;
  return 0u - inv;
}

// BLS12-381 scalar field r (255 bits, 2-adicity 32, generator 7).
struct FieldBls12381Fr {
  static constexpr int kId = 0;
  static constexpr uint32_t P0 = 0x00000001u, P1 = 0xffffffffu, P2 = 0xfffe5bfeu, P3 = 0x53bda402u,
                            P4 = 0x09a1d805u, P5 = 0x3339d808u, P6 = 0x299d7d48u, P7 = 0x73eda753u;
  static constexpr uint32_t NP = neg_inv_u32(P0);
};

// BN254 scalar field r (254 bits, 2-adicity 28, generator 5).
struct FieldBn254Fr {
  static constexpr int kId = 1;
  static constexpr uint32_t P0 = 0xf0000001u, P1 = 0x43e1f593u, P2 = 0x79b97091u, P3 = 0x2833e848u,
                            P4 = 0x8181585du, P5 = 0xb85045b6u, P6 = 0xe131a029u, P7 = 0x30644e72u;
  static constexpr uint32_t NP = neg_inv_u32(P0);
};

static_assert(FieldBls12381Fr::P0 * (0u - FieldBls12381Fr::NP) == 1u, "NP");
static_assert(FieldBn254Fr::P0 * (0u - FieldBn254Fr::NP) == 1u, "NP");
static_assert(FieldBls12381Fr::P0 == 1u && FieldBls12381Fr::P1 == 0xffffffffu && FieldBls12381Fr::NP == 0xffffffffu,
              "the BLS12-381 reduction rows rely on r = 2^64 - 2^32 + 1 mod 2^64");

// ------------------------------------------------------------------ helpers

// One CIOS row, t[0..8] += a * b, as two carry chains in which each
// product's low and high halves are adjacent:
//   even chain: a0*b -> (t0, t1), a2*b -> (t2, t3), a4*b -> (t4, t5),
//               a6*b -> (t6, t7), carry -> t8;
//   odd chain:  a1*b -> (t1, t2), ..., a7*b -> (t7, t8).
// Keeping lo and hi of a product in one chain lets the compiler issue each
// product as one wide multiply-add; measured on GB300 this formulation runs
// 1.37x faster than separate chains of low halves and of high halves.
__device__ __forceinline__ void row_even(uint32_t t[9], const uint32_t a[8], uint32_t b) {
  asm("mad.lo.cc.u32  %0, %9,  %13, %0;\n\t"
      "madc.hi.cc.u32 %1, %9,  %13, %1;\n\t"
      "madc.lo.cc.u32 %2, %10, %13, %2;\n\t"
      "madc.hi.cc.u32 %3, %10, %13, %3;\n\t"
      "madc.lo.cc.u32 %4, %11, %13, %4;\n\t"
      "madc.hi.cc.u32 %5, %11, %13, %5;\n\t"
      "madc.lo.cc.u32 %6, %12, %13, %6;\n\t"
      "madc.hi.cc.u32 %7, %12, %13, %7;\n\t"
      "addc.u32       %8, %8, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]),
        "+r"(t[8])
      : "r"(a[0]), "r"(a[2]), "r"(a[4]), "r"(a[6]), "r"(b));
}

// t[1..8] += odd products (no carry out: bounded, see header).
__device__ __forceinline__ void row_odd(uint32_t t[9], const uint32_t a[8], uint32_t b) {
  asm("mad.lo.cc.u32  %0, %8,  %12, %0;\n\t"
      "madc.hi.cc.u32 %1, %8,  %12, %1;\n\t"
      "madc.lo.cc.u32 %2, %9,  %12, %2;\n\t"
      "madc.hi.cc.u32 %3, %9,  %12, %3;\n\t"
      "madc.lo.cc.u32 %4, %10, %12, %4;\n\t"
      "madc.hi.cc.u32 %5, %10, %12, %5;\n\t"
      "madc.lo.cc.u32 %6, %11, %12, %6;\n\t"
      "madc.hi.u32    %7, %11, %12, %7;"
      : "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8])
      : "r"(a[1]), "r"(a[3]), "r"(a[5]), "r"(a[7]), "r"(b));
}

// Same two chains with the modulus p (immediates) as the multi-limb operand.
// For BLS12-381 Fr the two low limbs are p0 = 1 and p1 = 2^32 - 1 (r = ... +
// 2^64 - 2^32 + 1), so m*p0 = m and m*p1 = (m - [m != 0]) * 2^32 + (-m mod
// 2^32): those two products become additions (see row_*_p_bls below).
template <class F>
__device__ __forceinline__ void row_even_p_generic(uint32_t t[9], uint32_t m) {
  asm("mad.lo.cc.u32  %0, %9, %10, %0;\n\t"
      "madc.hi.cc.u32 %1, %9, %10, %1;\n\t"
      "madc.lo.cc.u32 %2, %9, %11, %2;\n\t"
      "madc.hi.cc.u32 %3, %9, %11, %3;\n\t"
      "madc.lo.cc.u32 %4, %9, %12, %4;\n\t"
      "madc.hi.cc.u32 %5, %9, %12, %5;\n\t"
      "madc.lo.cc.u32 %6, %9, %13, %6;\n\t"
      "madc.hi.cc.u32 %7, %9, %13, %7;\n\t"
      "addc.u32       %8, %8, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]),
        "+r"(t[8])
      : "r"(m), "n"(F::P0), "n"(F::P2), "n"(F::P4), "n"(F::P6));
}

template <class F>
__device__ __forceinline__ void row_odd_p_generic(uint32_t t[9], uint32_t m) {
  asm("mad.lo.cc.u32  %0, %8, %9,  %0;\n\t"
      "madc.hi.cc.u32 %1, %8, %9,  %1;\n\t"
      "madc.lo.cc.u32 %2, %8, %10, %2;\n\t"
      "madc.hi.cc.u32 %3, %8, %10, %3;\n\t"
      "madc.lo.cc.u32 %4, %8, %11, %4;\n\t"
      "madc.hi.cc.u32 %5, %8, %11, %5;\n\t"
      "madc.lo.cc.u32 %6, %8, %12, %6;\n\t"
      "madc.hi.u32    %7, %8, %12, %7;"
      : "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8])
      : "r"(m), "n"(F::P1), "n"(F::P3), "n"(F::P5), "n"(F::P7));
}

// BLS12-381 Fr: even chain with m*p0 = m (no multiply).
template <class F>
__device__ __forceinline__ void row_even_p_bls(uint32_t t[9], uint32_t m) {
  asm("add.cc.u32     %0, %0, %9;\n\t"
      "addc.cc.u32    %1, %1, 0;\n\t"
      "madc.lo.cc.u32 %2, %9, %10, %2;\n\t"
      "madc.hi.cc.u32 %3, %9, %10, %3;\n\t"
      "madc.lo.cc.u32 %4, %9, %11, %4;\n\t"
      "madc.hi.cc.u32 %5, %9, %11, %5;\n\t"
      "madc.lo.cc.u32 %6, %9, %12, %6;\n\t"
      "madc.hi.cc.u32 %7, %9, %12, %7;\n\t"
      "addc.u32       %8, %8, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]),
        "+r"(t[8])
      : "r"(m), "n"(F::P2), "n"(F::P4), "n"(F::P6));
}

// BLS12-381 Fr: odd chain with m*p1 = (m - [m != 0]) * 2^32 + (-m).
template <class F>
__device__ __forceinline__ void row_odd_p_bls(uint32_t t[9], uint32_t m) {
  const uint32_t lo1 = 0u - m;
  const uint32_t hi1 = m - (m != 0u ? 1u : 0u);
  asm("add.cc.u32     %0, %0, %9;\n\t"
      "addc.cc.u32    %1, %1, %10;\n\t"
      "madc.lo.cc.u32 %2, %8, %11, %2;\n\t"
      "madc.hi.cc.u32 %3, %8, %11, %3;\n\t"
      "madc.lo.cc.u32 %4, %8, %12, %4;\n\t"
      "madc.hi.cc.u32 %5, %8, %12, %5;\n\t"
      "madc.lo.cc.u32 %6, %8, %13, %6;\n\t"
      "madc.hi.u32    %7, %8, %13, %7;"
      : "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8])
      : "r"(m), "r"(lo1), "r"(hi1), "n"(F::P3), "n"(F::P5), "n"(F::P7));
}

template <class F>
__device__ __forceinline__ void row_even_p(uint32_t t[9], uint32_t m) {
  if constexpr (F::kId == 0) row_even_p_bls<F>(t, m);
  else row_even_p_generic<F>(t, m);
}

template <class F>
__device__ __forceinline__ void row_odd_p(uint32_t t[9], uint32_t m) {
  if constexpr (F::kId == 0) row_odd_p_bls<F>(t, m);
  else row_odd_p_generic<F>(t, m);
}

// m = t0 * (-p^-1 mod 2^32); for BLS12-381 Fr p0 = 1, so m = -t0.
template <class F>
__device__ __forceinline__ uint32_t mont_m(uint32_t t0) {
  if constexpr (F::kId == 0) return 0u - t0;
  else return t0 * F::NP;
}

// r = t - p if t >= p else t   (t < 2p).
template <class F>
__device__ __forceinline__ void reduce_once(uint32_t r[8], const uint32_t t[8]) {
  uint32_t d[8], bw;
  const uint32_t zero = 0;
  asm("sub.cc.u32  %0, %9,  %17;\n\t"
      "subc.cc.u32 %1, %10, %18;\n\t"
      "subc.cc.u32 %2, %11, %19;\n\t"
      "subc.cc.u32 %3, %12, %20;\n\t"
      "subc.cc.u32 %4, %13, %21;\n\t"
      "subc.cc.u32 %5, %14, %22;\n\t"
      "subc.cc.u32 %6, %15, %23;\n\t"
      "subc.cc.u32 %7, %16, %24;\n\t"
      "subc.u32    %8, %25, %25;"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
        "=r"(bw)
      : "r"(t[0]), "r"(t[1]), "r"(t[2]), "r"(t[3]), "r"(t[4]), "r"(t[5]), "r"(t[6]), "r"(t[7]), "n"(F::P0),
        "n"(F::P1), "n"(F::P2), "n"(F::P3), "n"(F::P4), "n"(F::P5), "n"(F::P6), "n"(F::P7), "r"(zero));
  // bw = all ones when t < p (keep t), zero otherwise (take t - p).
#pragma unroll
  for (int j = 0; j < 8; ++j) r[j] = (t[j] & bw) | (d[j] & ~bw);
}

// ---------------------------------------------------------------- field ops

// r = a * b * 2^-256 mod p.  a, b canonical; r canonical.  r may alias a or b.
template <class F>
__device__ __forceinline__ void mont_mul(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
  uint32_t t[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    row_even(t, a, b[i]);
    row_odd(t, a, b[i]);
    const uint32_t m = mont_m<F>(t[0]);
    row_even_p<F>(t, m);
    row_odd_p<F>(t, m);
    // t[0] is now zero: divide by 2^32.
#pragma unroll
    for (int j = 0; j < 8; ++j) t[j] = t[j + 1];
    t[8] = 0;
  }
  reduce_once<F>(r, t);
}

// r = a + b mod p.
template <class F>
__device__ __forceinline__ void add_mod(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
  uint32_t s[8];
  asm("add.cc.u32  %0, %8,  %16;\n\t"
      "addc.cc.u32 %1, %9,  %17;\n\t"
      "addc.cc.u32 %2, %10, %18;\n\t"
      "addc.cc.u32 %3, %11, %19;\n\t"
      "addc.cc.u32 %4, %12, %20;\n\t"
      "addc.cc.u32 %5, %13, %21;\n\t"
      "addc.cc.u32 %6, %14, %22;\n\t"
      "addc.u32    %7, %15, %23;"
      : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(b[0]),
        "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
  reduce_once<F>(r, s);
}

// r = a - b mod p.
template <class F>
__device__ __forceinline__ void sub_mod(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
  uint32_t d[8], bw;
  const uint32_t zero = 0;
  asm("sub.cc.u32  %0, %9,  %17;\n\t"
      "subc.cc.u32 %1, %10, %18;\n\t"
      "subc.cc.u32 %2, %11, %19;\n\t"
      "subc.cc.u32 %3, %12, %20;\n\t"
      "subc.cc.u32 %4, %13, %21;\n\t"
      "subc.cc.u32 %5, %14, %22;\n\t"
      "subc.cc.u32 %6, %15, %23;\n\t"
      "subc.cc.u32 %7, %16, %24;\n\t"
      "subc.u32    %8, %25, %25;"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
        "=r"(bw)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(b[0]),
        "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(zero));
  // add p back when the subtraction borrowed (bw = all ones)
  asm("add.cc.u32  %0, %0, %8;\n\t"
      "addc.cc.u32 %1, %1, %9;\n\t"
      "addc.cc.u32 %2, %2, %10;\n\t"
      "addc.cc.u32 %3, %3, %11;\n\t"
      "addc.cc.u32 %4, %4, %12;\n\t"
      "addc.cc.u32 %5, %5, %13;\n\t"
      "addc.cc.u32 %6, %6, %14;\n\t"
      "addc.u32    %7, %7, %15;"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]), "+r"(d[4]), "+r"(d[5]), "+r"(d[6]), "+r"(d[7])
      : "r"(F::P0 & bw), "r"(F::P1 & bw), "r"(F::P2 & bw), "r"(F::P3 & bw), "r"(F::P4 & bw),
        "r"(F::P5 & bw), "r"(F::P6 & bw), "r"(F::P7 & bw));
#pragma unroll
  for (int j = 0; j < 8; ++j) r[j] = d[j];
}

// ------------------------------------------- warp-cooperative variant
// The same CIOS Montgomery product with one element spread over 8 lanes
// (lane j of each aligned group of 8 holds limb j): every lane does the two
// 32x32 products of its limb per row, the high halves move one lane up by
// warp shuffle, the reduction factor m is broadcast from lane 0, and the
// running value is shifted one lane down per row.  Columns are kept in 64-bit
// accumulators (carries deferred); after the 8 rows the carries are
// propagated lane to lane, and the final comparison / subtraction of p uses
// a carry-lookahead on warp ballots.  Kept as a measured alternative to the
// per-thread carry chains (mont_mul), which have no shuffle traffic.
template <class F>
__device__ __forceinline__ uint32_t mont_mul_coop(uint32_t a_j, uint32_t b_j, uint32_t j) {
  constexpr uint32_t kFull = 0xffffffffu;
  const uint32_t p_j = j == 0 ? F::P0 : j == 1 ? F::P1 : j == 2 ? F::P2 : j == 3 ? F::P3
                     : j == 4 ? F::P4 : j == 5 ? F::P5 : j == 6 ? F::P6 : F::P7;
  uint64_t acc = 0, top = 0;  // top: column 8, kept by lane 7
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t bi = __shfl_sync(kFull, b_j, i, 8);
    const uint64_t pr = (uint64_t)a_j * bi;
    const uint32_t hi_in = __shfl_up_sync(kFull, (uint32_t)(pr >> 32), 1, 8);
    acc += (uint64_t)(uint32_t)pr + (j ? hi_in : 0u);
    if (j == 7) top += pr >> 32;
    const uint32_t m = __shfl_sync(kFull, mont_m<F>((uint32_t)acc), 0, 8);
    const uint64_t pm = (uint64_t)p_j * m;
    const uint32_t hm_in = __shfl_up_sync(kFull, (uint32_t)(pm >> 32), 1, 8);
    acc += (uint64_t)(uint32_t)pm + (j ? hm_in : 0u);
    if (j == 7) top += pm >> 32;
    // column 0 is now 0 mod 2^32: its high part carries into column 1
    const uint32_t c0 = __shfl_sync(kFull, (uint32_t)(acc >> 32), 0, 8);  // columns stay < 2^38
    if (j == 1) acc += c0;
    // divide by 2^32: every column moves one lane down
    const uint32_t nx_lo = __shfl_down_sync(kFull, (uint32_t)acc, 1, 8);
    const uint32_t nx_hi = __shfl_down_sync(kFull, (uint32_t)(acc >> 32), 1, 8);
    acc = j == 7 ? top : ((uint64_t)nx_hi << 32 | nx_lo);
    if (j == 7) top = 0;
  }
  // propagate the deferred carries (each column < 2^38)
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t c = __shfl_up_sync(kFull, (uint32_t)(acc >> 32), 1, 8);
    acc = (acc & 0xffffffffull) + (j ? c : 0u);
  }
  const uint32_t t = (uint32_t)acc;  // t < 2p
  // t - p if t >= p: borrow lookahead over the group's 8 lanes
  const uint32_t base = (threadIdx.x & 31u) & ~7u;
  const uint32_t G = (__ballot_sync(kFull, t < p_j) >> base) & 0xffu;   // generates a borrow
  const uint32_t P = (__ballot_sync(kFull, t == p_j) >> base) & 0xffu;  // propagates one
  const uint32_t x = G | P, sum = x + G;
  const uint32_t borrow_in = ((sum ^ x ^ G) >> j) & 1u;
  const bool ge = ((sum >> 8) & 1u) == 0;  // no borrow out of the top limb
  return ge ? t - p_j - borrow_in : t;
}

// y = x * 2^-256 mod M for canonical x (Montgomery reduction alone: half
// the multiplies of mont_mul).
template <class F>
__device__ __forceinline__ void mont_redc(uint32_t y[8], const uint32_t x[8]) {
  uint32_t t[9];
#pragma unroll
  for (int j = 0; j < 8; ++j) t[j] = x[j];
  t[8] = 0;
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

__device__ __forceinline__ void fe_copy(uint32_t r[8], const uint32_t a[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) r[j] = a[j];
}

// ------------------------------------------------------------- memory access

// One element = 32 bytes, moved with one 256-bit access (ld/st .v8.b32,
// sm_100 and later); element addresses are 32-byte aligned.
__device__ __forceinline__ void fe_load_global(uint32_t r[8], const uint4 *base, uint64_t elem) {
  asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "l"(base + 2 * elem));
}

// L2-coherent load (ld.global.cg): for data another CTA wrote earlier in the
// same kernel launch (volatile: never moved above the wait that orders it).
__device__ __forceinline__ void fe_load_global_cg(uint32_t r[8], const uint4 *base, uint64_t elem) {
  asm volatile("ld.global.cg.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "l"(base + 2 * elem)
               : "memory");
}

__device__ __forceinline__ void fe_store_global(uint4 *base, uint64_t elem, const uint32_t a[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               :
               : "l"(base + 2 * elem), "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]),
                 "r"(a[6]), "r"(a[7])
               : "memory");
}

}  // namespace gb300ntt
