// fp384.cuh -- 381-bit prime-field arithmetic for sm_103a, 12 x 32-bit limbs:
// the base field of BLS12-381 G1 (for the multi-scalar multiplication).
//
// The same Montgomery product as fp256.cuh (CIOS, radix 2^32, Koc, Acar and
// Kaliski 1996) over twelve limbs: per row the a*b_i products run as two
// carry chains (even limbs, odd limbs; the low and high halves of a product
// adjacent in one chain), then m = t0 * (-q^-1 mod 2^32) and the m*q rows the
// same way.  With a, b < q < 2^381 the running value stays below 2^415, so it
// fits in thirteen limbs and the last carry of every odd chain is zero; the
// result is below 2q and one conditional subtraction makes it canonical.
//
// Conventions: element = uint32_t[12], limb 0 least significant; in memory
// 48 bytes, moved as three 128-bit accesses (an element is 16-byte aligned).
#pragma once

#include <cstdint>

namespace gb300ntt {

// BLS12-381 base field q (381 bits).
struct FieldBls12381Fq {
  static constexpr uint32_t P0 = 0xffffaaabu, P1 = 0xb9feffffu, P2 = 0xb153ffffu, P3 = 0x1eabfffeu,
                            P4 = 0xf6b0f624u, P5 = 0x6730d2a0u, P6 = 0xf38512bfu, P7 = 0x64774b84u,
                            P8 = 0x434bacd7u, P9 = 0x4b1ba7b6u, P10 = 0x397fe69au, P11 = 0x1a0111eau;
  static constexpr uint32_t NP = 0xfffcfffdu;  // -q^-1 mod 2^32
};
static_assert(FieldBls12381Fq::P0 * FieldBls12381Fq::NP == 0xffffffffu, "NP = -q^-1 mod 2^32");

namespace fp384 {

using F = FieldBls12381Fq;

// t[0..12] += (a0, a2, ..., a10) * b at limbs (0,1), (2,3), ..., (10,11), carry into t12.
__device__ __forceinline__ void row_even(uint32_t t[13], const uint32_t a[12], uint32_t b) {
  asm("mad.lo.cc.u32  %0,  %13, %19, %0;\n\t"
      "madc.hi.cc.u32 %1,  %13, %19, %1;\n\t"
      "madc.lo.cc.u32 %2,  %14, %19, %2;\n\t"
      "madc.hi.cc.u32 %3,  %14, %19, %3;\n\t"
      "madc.lo.cc.u32 %4,  %15, %19, %4;\n\t"
      "madc.hi.cc.u32 %5,  %15, %19, %5;\n\t"
      "madc.lo.cc.u32 %6,  %16, %19, %6;\n\t"
      "madc.hi.cc.u32 %7,  %16, %19, %7;\n\t"
      "madc.lo.cc.u32 %8,  %17, %19, %8;\n\t"
      "madc.hi.cc.u32 %9,  %17, %19, %9;\n\t"
      "madc.lo.cc.u32 %10, %18, %19, %10;\n\t"
      "madc.hi.cc.u32 %11, %18, %19, %11;\n\t"
      "addc.u32       %12, %12, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]),
        "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12])
      : "r"(a[0]), "r"(a[2]), "r"(a[4]), "r"(a[6]), "r"(a[8]), "r"(a[10]), "r"(b));
}

// t[1..12] += (a1, a3, ..., a11) * b at limbs (1,2), ..., (11,12); no carry out.
__device__ __forceinline__ void row_odd(uint32_t t[13], const uint32_t a[12], uint32_t b) {
  asm("mad.lo.cc.u32  %0,  %12, %18, %0;\n\t"
      "madc.hi.cc.u32 %1,  %12, %18, %1;\n\t"
      "madc.lo.cc.u32 %2,  %13, %18, %2;\n\t"
      "madc.hi.cc.u32 %3,  %13, %18, %3;\n\t"
      "madc.lo.cc.u32 %4,  %14, %18, %4;\n\t"
      "madc.hi.cc.u32 %5,  %14, %18, %5;\n\t"
      "madc.lo.cc.u32 %6,  %15, %18, %6;\n\t"
      "madc.hi.cc.u32 %7,  %15, %18, %7;\n\t"
      "madc.lo.cc.u32 %8,  %16, %18, %8;\n\t"
      "madc.hi.cc.u32 %9,  %16, %18, %9;\n\t"
      "madc.lo.cc.u32 %10, %17, %18, %10;\n\t"
      "madc.hi.u32    %11, %17, %18, %11;"
      : "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]),
        "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12])
      : "r"(a[1]), "r"(a[3]), "r"(a[5]), "r"(a[7]), "r"(a[9]), "r"(a[11]), "r"(b));
}

// The same two chains with q (immediates) as the multi-limb operand.
__device__ __forceinline__ void row_even_q(uint32_t t[13], uint32_t m) {
  asm("mad.lo.cc.u32  %0,  %13, %14, %0;\n\t"
      "madc.hi.cc.u32 %1,  %13, %14, %1;\n\t"
      "madc.lo.cc.u32 %2,  %13, %15, %2;\n\t"
      "madc.hi.cc.u32 %3,  %13, %15, %3;\n\t"
      "madc.lo.cc.u32 %4,  %13, %16, %4;\n\t"
      "madc.hi.cc.u32 %5,  %13, %16, %5;\n\t"
      "madc.lo.cc.u32 %6,  %13, %17, %6;\n\t"
      "madc.hi.cc.u32 %7,  %13, %17, %7;\n\t"
      "madc.lo.cc.u32 %8,  %13, %18, %8;\n\t"
      "madc.hi.cc.u32 %9,  %13, %18, %9;\n\t"
      "madc.lo.cc.u32 %10, %13, %19, %10;\n\t"
      "madc.hi.cc.u32 %11, %13, %19, %11;\n\t"
      "addc.u32       %12, %12, 0;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]),
        "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12])
      : "r"(m), "n"(F::P0), "n"(F::P2), "n"(F::P4), "n"(F::P6), "n"(F::P8), "n"(F::P10));
}

__device__ __forceinline__ void row_odd_q(uint32_t t[13], uint32_t m) {
  asm("mad.lo.cc.u32  %0,  %12, %13, %0;\n\t"
      "madc.hi.cc.u32 %1,  %12, %13, %1;\n\t"
      "madc.lo.cc.u32 %2,  %12, %14, %2;\n\t"
      "madc.hi.cc.u32 %3,  %12, %14, %3;\n\t"
      "madc.lo.cc.u32 %4,  %12, %15, %4;\n\t"
      "madc.hi.cc.u32 %5,  %12, %15, %5;\n\t"
      "madc.lo.cc.u32 %6,  %12, %16, %6;\n\t"
      "madc.hi.cc.u32 %7,  %12, %16, %7;\n\t"
      "madc.lo.cc.u32 %8,  %12, %17, %8;\n\t"
      "madc.hi.cc.u32 %9,  %12, %17, %9;\n\t"
      "madc.lo.cc.u32 %10, %12, %18, %10;\n\t"
      "madc.hi.u32    %11, %12, %18, %11;"
      : "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]),
        "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12])
      : "r"(m), "n"(F::P1), "n"(F::P3), "n"(F::P5), "n"(F::P7), "n"(F::P9), "n"(F::P11));
}

// d = a - q with borrow mask (all ones when a < q).
__device__ __forceinline__ uint32_t sub_q(uint32_t d[12], const uint32_t a[12]) {
  uint32_t bw;
  const uint32_t zero = 0;
  asm("sub.cc.u32  %0,  %13, %25;\n\t"
      "subc.cc.u32 %1,  %14, %26;\n\t"
      "subc.cc.u32 %2,  %15, %27;\n\t"
      "subc.cc.u32 %3,  %16, %28;\n\t"
      "subc.cc.u32 %4,  %17, %29;\n\t"
      "subc.cc.u32 %5,  %18, %30;\n\t"
      "subc.cc.u32 %6,  %19, %31;\n\t"
      "subc.cc.u32 %7,  %20, %32;\n\t"
      "subc.cc.u32 %8,  %21, %33;\n\t"
      "subc.cc.u32 %9,  %22, %34;\n\t"
      "subc.cc.u32 %10, %23, %35;\n\t"
      "subc.cc.u32 %11, %24, %36;\n\t"
      "subc.u32    %12, %37, %37;"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
        "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(bw)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]),
        "r"(a[9]), "r"(a[10]), "r"(a[11]), "n"(F::P0), "n"(F::P1), "n"(F::P2), "n"(F::P3), "n"(F::P4),
        "n"(F::P5), "n"(F::P6), "n"(F::P7), "n"(F::P8), "n"(F::P9), "n"(F::P10), "n"(F::P11), "r"(zero));
  return bw;
}

// r = t - q if t >= q else t  (t < 2q).
__device__ __forceinline__ void reduce_once(uint32_t r[12], const uint32_t t[12]) {
  uint32_t d[12];
  const uint32_t bw = sub_q(d, t);
#pragma unroll
  for (int j = 0; j < 12; ++j) r[j] = (t[j] & bw) | (d[j] & ~bw);
}

// r = a * b * 2^-384 mod q.  a, b canonical; r canonical; r may alias a or b.
__device__ __forceinline__ void mont_mul(uint32_t r[12], const uint32_t a[12], const uint32_t b[12]) {
  uint32_t t[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    row_even(t, a, b[i]);
    row_odd(t, a, b[i]);
    const uint32_t m = t[0] * F::NP;
    row_even_q(t, m);
    row_odd_q(t, m);
#pragma unroll
    for (int j = 0; j < 12; ++j) t[j] = t[j + 1];
    t[12] = 0;
  }
  reduce_once(r, t);
}

// y = x * 2^-384 mod q (Montgomery reduction alone).
__device__ __forceinline__ void mont_redc(uint32_t y[12], const uint32_t x[12]) {
  uint32_t t[13];
#pragma unroll
  for (int j = 0; j < 12; ++j) t[j] = x[j];
  t[12] = 0;
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const uint32_t m = t[0] * F::NP;
    row_even_q(t, m);
    row_odd_q(t, m);
#pragma unroll
    for (int j = 0; j < 12; ++j) t[j] = t[j + 1];
    t[12] = 0;
  }
  reduce_once(y, t);
}

// r = a + b mod q (a + b < 2q < 2^384: no carry out of the top limb).
__device__ __forceinline__ void add_mod(uint32_t r[12], const uint32_t a[12], const uint32_t b[12]) {
  uint32_t s[12];
  asm("add.cc.u32  %0,  %12, %24;\n\t"
      "addc.cc.u32 %1,  %13, %25;\n\t"
      "addc.cc.u32 %2,  %14, %26;\n\t"
      "addc.cc.u32 %3,  %15, %27;\n\t"
      "addc.cc.u32 %4,  %16, %28;\n\t"
      "addc.cc.u32 %5,  %17, %29;\n\t"
      "addc.cc.u32 %6,  %18, %30;\n\t"
      "addc.cc.u32 %7,  %19, %31;\n\t"
      "addc.cc.u32 %8,  %20, %32;\n\t"
      "addc.cc.u32 %9,  %21, %33;\n\t"
      "addc.cc.u32 %10, %22, %34;\n\t"
      "addc.u32    %11, %23, %35;"
      : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]),
        "=r"(s[8]), "=r"(s[9]), "=r"(s[10]), "=r"(s[11])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]),
        "r"(a[9]), "r"(a[10]), "r"(a[11]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]),
        "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]));
  reduce_once(r, s);
}

// r = a - b mod q.
__device__ __forceinline__ void sub_mod(uint32_t r[12], const uint32_t a[12], const uint32_t b[12]) {
  uint32_t d[12], bw;
  const uint32_t zero = 0;
  asm("sub.cc.u32  %0,  %13, %25;\n\t"
      "subc.cc.u32 %1,  %14, %26;\n\t"
      "subc.cc.u32 %2,  %15, %27;\n\t"
      "subc.cc.u32 %3,  %16, %28;\n\t"
      "subc.cc.u32 %4,  %17, %29;\n\t"
      "subc.cc.u32 %5,  %18, %30;\n\t"
      "subc.cc.u32 %6,  %19, %31;\n\t"
      "subc.cc.u32 %7,  %20, %32;\n\t"
      "subc.cc.u32 %8,  %21, %33;\n\t"
      "subc.cc.u32 %9,  %22, %34;\n\t"
      "subc.cc.u32 %10, %23, %35;\n\t"
      "subc.cc.u32 %11, %24, %36;\n\t"
      "subc.u32    %12, %37, %37;"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
        "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(bw)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]),
        "r"(a[9]), "r"(a[10]), "r"(a[11]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]),
        "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]), "r"(zero));
  // add q back when the subtraction borrowed (bw = all ones)
  asm("add.cc.u32  %0,  %0,  %12;\n\t"
      "addc.cc.u32 %1,  %1,  %13;\n\t"
      "addc.cc.u32 %2,  %2,  %14;\n\t"
      "addc.cc.u32 %3,  %3,  %15;\n\t"
      "addc.cc.u32 %4,  %4,  %16;\n\t"
      "addc.cc.u32 %5,  %5,  %17;\n\t"
      "addc.cc.u32 %6,  %6,  %18;\n\t"
      "addc.cc.u32 %7,  %7,  %19;\n\t"
      "addc.cc.u32 %8,  %8,  %20;\n\t"
      "addc.cc.u32 %9,  %9,  %21;\n\t"
      "addc.cc.u32 %10, %10, %22;\n\t"
      "addc.u32    %11, %11, %23;"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]), "+r"(d[4]), "+r"(d[5]), "+r"(d[6]), "+r"(d[7]),
        "+r"(d[8]), "+r"(d[9]), "+r"(d[10]), "+r"(d[11])
      : "r"(F::P0 & bw), "r"(F::P1 & bw), "r"(F::P2 & bw), "r"(F::P3 & bw), "r"(F::P4 & bw), "r"(F::P5 & bw),
        "r"(F::P6 & bw), "r"(F::P7 & bw), "r"(F::P8 & bw), "r"(F::P9 & bw), "r"(F::P10 & bw),
        "r"(F::P11 & bw));
#pragma unroll
  for (int j = 0; j < 12; ++j) r[j] = d[j];
}

// a < q for a raw 384-bit value.
__device__ __forceinline__ bool is_canonical(const uint32_t a[12]) {
  uint32_t d[12];
  return sub_q(d, a) != 0u;
}

// Element e of a 48-byte-element array (three 128-bit accesses).
__device__ __forceinline__ void load(uint32_t r[12], const uint4 *base, uint64_t e) {
  const uint4 *p = base + 3 * e;
#pragma unroll
  for (int h = 0; h < 3; ++h) {
    asm("ld.global.nc.v4.b32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r[4 * h]), "=r"(r[4 * h + 1]), "=r"(r[4 * h + 2]), "=r"(r[4 * h + 3])
        : "l"(p + h));
  }
}

__device__ __forceinline__ void store(uint4 *base, uint64_t e, const uint32_t a[12]) {
  uint4 *p = base + 3 * e;
#pragma unroll
  for (int h = 0; h < 3; ++h) {
    asm volatile("st.global.v4.b32 [%0], {%1,%2,%3,%4};"
                 :
                 : "l"(p + h), "r"(a[4 * h]), "r"(a[4 * h + 1]), "r"(a[4 * h + 2]), "r"(a[4 * h + 3])
                 : "memory");
  }
}

}  // namespace fp384
}  // namespace gb300ntt
