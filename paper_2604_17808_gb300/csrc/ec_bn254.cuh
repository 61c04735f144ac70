// ec_bn254.cuh -- BN254 G1 point arithmetic for sm_103a.
//
// The curve of the multi-scalar multiplication (MORPH, Sec. 2.3.1 and
// Algorithm 2, read as BN254 G1 for the paper's 256-bit MSM column):
// y^2 = x^3 + 3 over the 254-bit prime field F_q, a group of prime order r
// (the BN254 scalar field).  BN254 G1 has no point of order two, so it has no
// twisted Edwards model; the buckets use XYZZ coordinates of the short
// Weierstrass form instead: (X, Y, ZZ, ZZZ) stands for the affine point
// (X / ZZ, Y / ZZZ) with ZZ^3 = ZZZ^2, and ZZ = 0 marks the point at
// infinity O.  The formulas are the "xyzz" ones of the Explicit-Formulas
// Database (Bernstein and Lange): madd-2008-s (bucket += affine point,
// 8M + 2S), add-2008-s (12M + 2S), dbl-2008-s-1 (6M + 3S) and mdbl-2008-s-1,
// with the cases the formulas exclude (an operand O, P = Q, P = -Q) taken
// explicitly.
//
// Every coordinate is in Montgomery form x 2^256 mod q and canonical; the
// field product is the same CIOS routine as the transforms' (fp256.cuh).
#pragma once

#include "fp256.cuh"

namespace gb300ntt {

// BN254 base field q (254 bits).
struct FieldBn254Fq {
  static constexpr int kId = 2;
  static constexpr uint32_t P0 = 0xd87cfd47u, P1 = 0x3c208c16u, P2 = 0x6871ca8du, P3 = 0x97816a91u,
                            P4 = 0x8181585du, P5 = 0xb85045b6u, P6 = 0xe131a029u, P7 = 0x30644e72u;
  static constexpr uint32_t NP = neg_inv_u32(P0);
};
static_assert(FieldBn254Fq::P0 * (0u - FieldBn254Fq::NP) == 1u, "NP");

using Fq = FieldBn254Fq;

// The same product as an out-of-line call with the operands passed by value
// (they travel in registers; no stack frame).  The mixed addition of the
// bucket-accumulation loop uses it: one shared copy of the product's ~300
// instructions instead of ten inlined copies keeps the loop inside the
// instruction cache (measured on GB300: the whole MSM at 2^24 points 9%
// faster).  The other formulas keep the inlined product, which measured
// faster for them.
struct FeV {
  uint32_t v[8];
};

__device__ __noinline__ FeV fq_mul_call(FeV a, FeV b) {
  FeV r;
  mont_mul<Fq>(r.v, a.v, b.v);
  return r;
}

__device__ __forceinline__ void fq_mul_small(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
  FeV x, y;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    x.v[j] = a[j];
    y.v[j] = b[j];
  }
  const FeV z = fq_mul_call(x, y);
#pragma unroll
  for (int j = 0; j < 8; ++j) r[j] = z.v[j];
}

// Product used by a formula: inlined, or the out-of-line call (kCall).
template <bool kCall>
__device__ __forceinline__ void fq_mul(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
  if constexpr (kCall) fq_mul_small(r, a, b);
  else mont_mul<Fq>(r, a, b);
}

struct PointXyzz {
  uint32_t X[8], Y[8], ZZ[8], ZZZ[8];
};

__device__ __forceinline__ bool fe_is_zero(const uint32_t a[8]) {
  return (a[0] | a[1] | a[2] | a[3] | a[4] | a[5] | a[6] | a[7]) == 0u;
}

__device__ __forceinline__ bool fe_equal(const uint32_t a[8], const uint32_t b[8]) {
  return ((a[0] ^ b[0]) | (a[1] ^ b[1]) | (a[2] ^ b[2]) | (a[3] ^ b[3]) | (a[4] ^ b[4]) | (a[5] ^ b[5]) |
          (a[6] ^ b[6]) | (a[7] ^ b[7])) == 0u;
}

__device__ __forceinline__ void fe_zero(uint32_t a[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 0u;
}

// a < q for a raw 256-bit value
__device__ __forceinline__ bool fq_is_canonical(const uint32_t a[8]) {
  const uint32_t p[8] = {Fq::P0, Fq::P1, Fq::P2, Fq::P3, Fq::P4, Fq::P5, Fq::P6, Fq::P7};
#pragma unroll
  for (int j = 7; j >= 0; --j)
    if (a[j] != p[j]) return a[j] < p[j];
  return false;
}

__device__ __forceinline__ void xyzz_set_inf(PointXyzz &r) {
  fe_zero(r.X);
  fe_zero(r.Y);
  fe_zero(r.ZZ);
  fe_zero(r.ZZZ);
}

__device__ __forceinline__ bool xyzz_is_inf(const PointXyzz &p) { return fe_is_zero(p.ZZ); }

// r = 2 (x, y) for an affine point (x, y) (mdbl-2008-s-1, a = 0).
__device__ __forceinline__ void xyzz_mdbl(PointXyzz &r, const uint32_t x[8], const uint32_t y[8]) {
  uint32_t U[8], V[8], W[8], S[8], M[8];
  add_mod<Fq>(U, y, y);      // U = 2 y
  mont_mul<Fq>(V, U, U);     // V = U^2
  mont_mul<Fq>(W, U, V);     // W = U V
  mont_mul<Fq>(S, x, V);     // S = x V
  mont_mul<Fq>(M, x, x);
  add_mod<Fq>(U, M, M);
  add_mod<Fq>(M, U, M);      // M = 3 x^2
  mont_mul<Fq>(U, M, M);
  sub_mod<Fq>(U, U, S);
  sub_mod<Fq>(U, U, S);      // X3 = M^2 - 2 S
  sub_mod<Fq>(S, S, U);
  mont_mul<Fq>(S, M, S);     // M (S - X3)
  mont_mul<Fq>(M, W, y);
  sub_mod<Fq>(r.Y, S, M);    // Y3 = M (S - X3) - W y
  fe_copy(r.X, U);
  fe_copy(r.ZZ, V);          // ZZ3 = V
  fe_copy(r.ZZZ, W);         // ZZZ3 = W
}

// r = 2 p (dbl-2008-s-1, a = 0); r may alias p.  2 O = O follows from the
// formulas (ZZ3 = V ZZ1 = 0).
template <bool kCall = false>
__device__ __forceinline__ void xyzz_dbl(PointXyzz &r, const PointXyzz &p) {
  uint32_t U[8], V[8], W[8], S[8], M[8];
  add_mod<Fq>(U, p.Y, p.Y);  // U = 2 Y1
  fq_mul<kCall>(V, U, U);     // V = U^2
  fq_mul<kCall>(W, U, V);     // W = U V
  fq_mul<kCall>(S, p.X, V);   // S = X1 V
  fq_mul<kCall>(M, p.X, p.X);
  add_mod<Fq>(U, M, M);
  add_mod<Fq>(M, U, M);      // M = 3 X1^2
  fq_mul<kCall>(r.ZZ, V, p.ZZ);     // ZZ3 = V ZZ1
  fq_mul<kCall>(r.ZZZ, W, p.ZZZ);   // ZZZ3 = W ZZZ1
  fq_mul<kCall>(W, W, p.Y);         // W Y1
  fq_mul<kCall>(U, M, M);
  sub_mod<Fq>(U, U, S);
  sub_mod<Fq>(U, U, S);      // X3 = M^2 - 2 S
  sub_mod<Fq>(S, S, U);
  fq_mul<kCall>(S, M, S);
  sub_mod<Fq>(r.Y, S, W);    // Y3 = M (S - X3) - W Y1
  fe_copy(r.X, U);
}

// acc += (x2, y2), an affine point that is not O (madd-2008-s).
__device__ __forceinline__ void xyzz_madd(PointXyzz &acc, const uint32_t x2[8], const uint32_t y2[8],
                                          const uint32_t one[8]) {
  if (xyzz_is_inf(acc)) {
    fe_copy(acc.X, x2);
    fe_copy(acc.Y, y2);
    fe_copy(acc.ZZ, one);
    fe_copy(acc.ZZZ, one);
    return;
  }
  uint32_t P[8], R[8], PP[8], PPP[8], Q[8];
  fq_mul_small(P, x2, acc.ZZ);
  sub_mod<Fq>(P, P, acc.X);       // P = U2 - X1
  fq_mul_small(R, y2, acc.ZZZ);
  sub_mod<Fq>(R, R, acc.Y);       // R = S2 - Y1
  if (fe_is_zero(P)) {
    if (fe_is_zero(R)) xyzz_mdbl(acc, x2, y2);  // same point
    else xyzz_set_inf(acc);                     // opposite points
    return;
  }
  fq_mul_small(PP, P, P);
  fq_mul_small(PPP, P, PP);
  fq_mul_small(acc.ZZ, acc.ZZ, PP);     // ZZ3 = ZZ1 PP
  fq_mul_small(acc.ZZZ, acc.ZZZ, PPP);  // ZZZ3 = ZZZ1 PPP
  fq_mul_small(Q, acc.X, PP);           // Q = X1 PP
  fq_mul_small(P, R, R);
  sub_mod<Fq>(P, P, PPP);
  sub_mod<Fq>(P, P, Q);
  sub_mod<Fq>(P, P, Q);                 // X3 = R^2 - PPP - 2 Q
  sub_mod<Fq>(Q, Q, P);
  fq_mul_small(Q, R, Q);                // R (Q - X3)
  fq_mul_small(PPP, acc.Y, PPP);
  sub_mod<Fq>(acc.Y, Q, PPP);           // Y3 = R (Q - X3) - Y1 PPP
  fe_copy(acc.X, P);
}

// acc += q (add-2008-s).
template <bool kCall = false>
__device__ __forceinline__ void xyzz_add(PointXyzz &acc, const PointXyzz &q) {
  if (xyzz_is_inf(q)) return;
  if (xyzz_is_inf(acc)) {
    acc = q;
    return;
  }
  uint32_t U1[8], S1[8], P[8], R[8], PP[8], PPP[8];
  fq_mul<kCall>(U1, acc.X, q.ZZ);        // U1 = X1 ZZ2
  fq_mul<kCall>(S1, acc.Y, q.ZZZ);       // S1 = Y1 ZZZ2
  fq_mul<kCall>(P, q.X, acc.ZZ);
  sub_mod<Fq>(P, P, U1);                // P = U2 - U1
  fq_mul<kCall>(R, q.Y, acc.ZZZ);
  sub_mod<Fq>(R, R, S1);                // R = S2 - S1
  if (fe_is_zero(P)) {
    if (fe_is_zero(R)) xyzz_dbl<kCall>(acc, q);
    else xyzz_set_inf(acc);
    return;
  }
  fq_mul<kCall>(PP, P, P);
  fq_mul<kCall>(PPP, P, PP);
  fq_mul<kCall>(acc.ZZ, acc.ZZ, q.ZZ);
  fq_mul<kCall>(acc.ZZ, acc.ZZ, PP);     // ZZ3 = ZZ1 ZZ2 PP
  fq_mul<kCall>(acc.ZZZ, acc.ZZZ, q.ZZZ);
  fq_mul<kCall>(acc.ZZZ, acc.ZZZ, PPP);  // ZZZ3 = ZZZ1 ZZZ2 PPP
  fq_mul<kCall>(U1, U1, PP);             // Q = U1 PP
  fq_mul<kCall>(P, R, R);
  sub_mod<Fq>(P, P, PPP);
  sub_mod<Fq>(P, P, U1);
  sub_mod<Fq>(P, P, U1);                // X3 = R^2 - PPP - 2 Q
  sub_mod<Fq>(U1, U1, P);
  fq_mul<kCall>(U1, R, U1);              // R (Q - X3)
  fq_mul<kCall>(S1, S1, PPP);
  sub_mod<Fq>(acc.Y, U1, S1);           // Y3 = R (Q - X3) - S1 PPP
  fe_copy(acc.X, P);
}

// r = a^(q-2) = a^-1 (Fermat), Montgomery in and out; a = 0 gives 0.
__device__ __forceinline__ void fq_inverse(uint32_t r[8], const uint32_t a[8], const uint32_t one[8]) {
  const uint32_t e[8] = {Fq::P0 - 2u, Fq::P1, Fq::P2, Fq::P3, Fq::P4, Fq::P5, Fq::P6, Fq::P7};
  uint32_t acc[8];
  fe_copy(acc, one);
  for (int i = 253; i >= 0; --i) {
    mont_mul<Fq>(acc, acc, acc);
    if ((e[i >> 5] >> (i & 31)) & 1u) mont_mul<Fq>(acc, acc, a);
  }
  fe_copy(r, acc);
}

// Affine point of p in STANDARD form (x, y); O gives (0, 0).
__device__ __forceinline__ void xyzz_to_affine_std(uint32_t x[8], uint32_t y[8], const PointXyzz &p,
                                                   const uint32_t one[8]) {
  if (xyzz_is_inf(p)) {
    fe_zero(x);
    fe_zero(y);
    return;
  }
  uint32_t t[8], inv[8], zi[8];
  mont_mul<Fq>(t, p.ZZ, p.ZZZ);
  fq_inverse(inv, t, one);       // (ZZ ZZZ)^-1
  mont_mul<Fq>(zi, inv, p.ZZZ);  // ZZ^-1
  mont_mul<Fq>(t, p.X, zi);
  mont_redc<Fq>(x, t);
  mont_mul<Fq>(zi, inv, p.ZZ);   // ZZZ^-1
  mont_mul<Fq>(t, p.Y, zi);
  mont_redc<Fq>(y, t);
}

}  // namespace gb300ntt
