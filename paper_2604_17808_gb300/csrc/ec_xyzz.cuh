// ec_xyzz.cuh -- short-Weierstrass point arithmetic (y^2 = x^3 + b) for the
// multi-scalar multiplication, sm_103a, generic over the base field.
//
// Curves (MORPH, Sec. 2.3.1 and Algorithm 2; the paper's 256-bit MSM column
// read as BN254 G1): BN254 G1 (y^2 = x^3 + 3 over a 254-bit field) and
// BLS12-381 G1 (y^2 = x^3 + 4 over a 381-bit field).  Neither has a twisted
// Edwards model over its base field (no point of order two in the group the
// MSM uses), so the buckets use XYZZ coordinates: (X, Y, ZZ, ZZZ) stands for
// the affine point (X / ZZ, Y / ZZZ) with ZZ^3 = ZZZ^2, and ZZ = 0 marks the
// point at infinity O.  The formulas are the "xyzz" ones of the
// Explicit-Formulas Database (Bernstein and Lange): madd-2008-s (bucket +=
// affine point, 8M + 2S), add-2008-s (12M + 2S), dbl-2008-s-1 (6M + 3S) and
// mdbl-2008-s-1, with the cases the formulas exclude (an operand O, P = Q,
// P = -Q) taken explicitly.
//
// Every coordinate is in Montgomery form and canonical.  A field "traits"
// type T supplies the limb count T::L and the operations (product, sum,
// difference, reduction, canonical check, 32-byte or 48-byte memory access).
#pragma once

#include "fp256.cuh"
#include "fp384.cuh"

namespace gb300ntt {

// BN254 base field q (254 bits).
struct FieldBn254Fq {
  static constexpr int kId = 2;
  static constexpr uint32_t P0 = 0xd87cfd47u, P1 = 0x3c208c16u, P2 = 0x6871ca8du, P3 = 0x97816a91u,
                            P4 = 0x8181585du, P5 = 0xb85045b6u, P6 = 0xe131a029u, P7 = 0x30644e72u;
  static constexpr uint32_t NP = neg_inv_u32(P0);
};
static_assert(FieldBn254Fq::P0 * (0u - FieldBn254Fq::NP) == 1u, "NP");

// ------------------------------------------------------------ field traits

struct FqBn254 {
  static constexpr int L = 8;
  static constexpr int kTopBit = 253;  // q < 2^254
  using F = FieldBn254Fq;
  __device__ static void mul(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) { mont_mul<F>(r, a, b); }
  __device__ static void add(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) { add_mod<F>(r, a, b); }
  __device__ static void sub(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) { sub_mod<F>(r, a, b); }
  __device__ static void redc(uint32_t r[8], const uint32_t a[8]) { mont_redc<F>(r, a); }
  __device__ static bool canonical(const uint32_t a[8]) {
    const uint32_t p[8] = {F::P0, F::P1, F::P2, F::P3, F::P4, F::P5, F::P6, F::P7};
#pragma unroll
    for (int j = 7; j >= 0; --j)
      if (a[j] != p[j]) return a[j] < p[j];
    return false;
  }
  // exponent q - 2 (inversion by Fermat), limb j
  __device__ static uint32_t inv_exp(int j) {
    const uint32_t e[8] = {F::P0 - 2u, F::P1, F::P2, F::P3, F::P4, F::P5, F::P6, F::P7};
    return e[j];
  }
  __device__ static void load(uint32_t r[8], const uint4 *base, uint64_t e) { fe_load_global(r, base, e); }
  __device__ static void store(uint4 *base, uint64_t e, const uint32_t a[8]) { fe_store_global(base, e, a); }
};

struct FqBls381 {
  static constexpr int L = 12;
  static constexpr int kTopBit = 380;  // q < 2^381
  using F = FieldBls12381Fq;
  __device__ static void mul(uint32_t r[12], const uint32_t a[12], const uint32_t b[12]) { fp384::mont_mul(r, a, b); }
  __device__ static void add(uint32_t r[12], const uint32_t a[12], const uint32_t b[12]) { fp384::add_mod(r, a, b); }
  __device__ static void sub(uint32_t r[12], const uint32_t a[12], const uint32_t b[12]) { fp384::sub_mod(r, a, b); }
  __device__ static void redc(uint32_t r[12], const uint32_t a[12]) { fp384::mont_redc(r, a); }
  __device__ static bool canonical(const uint32_t a[12]) { return fp384::is_canonical(a); }
  __device__ static uint32_t inv_exp(int j) {
    const uint32_t e[12] = {F::P0 - 2u, F::P1, F::P2, F::P3, F::P4, F::P5, F::P6, F::P7, F::P8, F::P9, F::P10, F::P11};
    return e[j];
  }
  __device__ static void load(uint32_t r[12], const uint4 *base, uint64_t e) { fp384::load(r, base, e); }
  __device__ static void store(uint4 *base, uint64_t e, const uint32_t a[12]) { fp384::store(base, e, a); }
};

// ------------------------------------------------------ generic limb helpers

template <int L>
__device__ __forceinline__ bool fv_is_zero(const uint32_t a[L]) {
  uint32_t o = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) o |= a[j];
  return o == 0u;
}

template <int L>
__device__ __forceinline__ bool fv_equal(const uint32_t a[L], const uint32_t b[L]) {
  uint32_t o = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) o |= a[j] ^ b[j];
  return o == 0u;
}

template <int L>
__device__ __forceinline__ void fv_zero(uint32_t a[L]) {
#pragma unroll
  for (int j = 0; j < L; ++j) a[j] = 0u;
}

template <int L>
__device__ __forceinline__ void fv_copy(uint32_t r[L], const uint32_t a[L]) {
#pragma unroll
  for (int j = 0; j < L; ++j) r[j] = a[j];
}

// The field product as an out-of-line call with the operands passed by value
// (they travel in registers; no stack frame).  The mixed addition of the
// bucket-accumulation loop uses it: one shared copy of the product instead
// of ten inlined copies keeps the loop inside the instruction cache
// (measured on GB300, BN254: the whole MSM at 2^24 points 9% faster).
// xyzz_add / xyzz_dbl take the call when kCall is set (the reduction-tree
// and combine kernels, where it also measured faster); elsewhere the product
// is inlined.
template <class T>
struct FeV {
  uint32_t v[T::L];
};

template <class T>
__device__ __noinline__ FeV<T> f_mul_call(FeV<T> a, FeV<T> b) {
  FeV<T> r;
  T::mul(r.v, a.v, b.v);
  return r;
}

template <class T, bool kCall>
__device__ __forceinline__ void f_mul(uint32_t r[T::L], const uint32_t a[T::L], const uint32_t b[T::L]) {
  if constexpr (kCall) {
    FeV<T> x, y;
#pragma unroll
    for (int j = 0; j < T::L; ++j) {
      x.v[j] = a[j];
      y.v[j] = b[j];
    }
    const FeV<T> z = f_mul_call<T>(x, y);
#pragma unroll
    for (int j = 0; j < T::L; ++j) r[j] = z.v[j];
  } else {
    T::mul(r, a, b);
  }
}

template <class T>
struct Xyzz {
  uint32_t X[T::L], Y[T::L], ZZ[T::L], ZZZ[T::L];
};

template <class T>
__device__ __forceinline__ void xyzz_set_inf(Xyzz<T> &r) {
  fv_zero<T::L>(r.X);
  fv_zero<T::L>(r.Y);
  fv_zero<T::L>(r.ZZ);
  fv_zero<T::L>(r.ZZZ);
}

template <class T>
__device__ __forceinline__ bool xyzz_is_inf(const Xyzz<T> &p) { return fv_is_zero<T::L>(p.ZZ); }

// r = 2 (x, y) for an affine point (x, y) (mdbl-2008-s-1, a = 0).
template <class T>
__device__ __forceinline__ void xyzz_mdbl(Xyzz<T> &r, const uint32_t x[T::L], const uint32_t y[T::L]) {
  constexpr int L = T::L;
  uint32_t U[L], V[L], W[L], S[L], M[L];
  T::add(U, y, y);      // U = 2 y
  T::mul(V, U, U);      // V = U^2
  T::mul(W, U, V);      // W = U V
  T::mul(S, x, V);      // S = x V
  T::mul(M, x, x);
  T::add(U, M, M);
  T::add(M, U, M);      // M = 3 x^2
  T::mul(U, M, M);
  T::sub(U, U, S);
  T::sub(U, U, S);      // X3 = M^2 - 2 S
  T::sub(S, S, U);
  T::mul(S, M, S);      // M (S - X3)
  T::mul(M, W, y);
  T::sub(r.Y, S, M);    // Y3 = M (S - X3) - W y
  fv_copy<L>(r.X, U);
  fv_copy<L>(r.ZZ, V);  // ZZ3 = V
  fv_copy<L>(r.ZZZ, W); // ZZZ3 = W
}

// r = 2 p (dbl-2008-s-1, a = 0); r may alias p.  2 O = O follows from the
// formulas (ZZ3 = V ZZ1 = 0).
template <class T, bool kCall = false>
__device__ __forceinline__ void xyzz_dbl(Xyzz<T> &r, const Xyzz<T> &p) {
  constexpr int L = T::L;
  uint32_t U[L], V[L], W[L], S[L], M[L];
  T::add(U, p.Y, p.Y);            // U = 2 Y1
  f_mul<T, kCall>(V, U, U);       // V = U^2
  f_mul<T, kCall>(W, U, V);       // W = U V
  f_mul<T, kCall>(S, p.X, V);     // S = X1 V
  f_mul<T, kCall>(M, p.X, p.X);
  T::add(U, M, M);
  T::add(M, U, M);                // M = 3 X1^2
  f_mul<T, kCall>(r.ZZ, V, p.ZZ);    // ZZ3 = V ZZ1
  f_mul<T, kCall>(r.ZZZ, W, p.ZZZ);  // ZZZ3 = W ZZZ1
  f_mul<T, kCall>(W, W, p.Y);        // W Y1
  f_mul<T, kCall>(U, M, M);
  T::sub(U, U, S);
  T::sub(U, U, S);                // X3 = M^2 - 2 S
  T::sub(S, S, U);
  f_mul<T, kCall>(S, M, S);
  T::sub(r.Y, S, W);              // Y3 = M (S - X3) - W Y1
  fv_copy<L>(r.X, U);
}

// acc += (x2, y2), an affine point that is not O (madd-2008-s).
template <class T>
__device__ __forceinline__ void xyzz_madd(Xyzz<T> &acc, const uint32_t x2[T::L], const uint32_t y2[T::L],
                                          const uint32_t one[T::L]) {
  constexpr int L = T::L;
  if (xyzz_is_inf(acc)) {
    fv_copy<L>(acc.X, x2);
    fv_copy<L>(acc.Y, y2);
    fv_copy<L>(acc.ZZ, one);
    fv_copy<L>(acc.ZZZ, one);
    return;
  }
  uint32_t P[L], R[L], PP[L], PPP[L], Q[L];
  f_mul<T, true>(P, x2, acc.ZZ);
  T::sub(P, P, acc.X);            // P = U2 - X1
  f_mul<T, true>(R, y2, acc.ZZZ);
  T::sub(R, R, acc.Y);            // R = S2 - Y1
  if (fv_is_zero<L>(P)) {
    if (fv_is_zero<L>(R)) xyzz_mdbl<T>(acc, x2, y2);  // same point
    else xyzz_set_inf(acc);                          // opposite points
    return;
  }
  f_mul<T, true>(PP, P, P);
  f_mul<T, true>(PPP, P, PP);
  f_mul<T, true>(acc.ZZ, acc.ZZ, PP);     // ZZ3 = ZZ1 PP
  f_mul<T, true>(acc.ZZZ, acc.ZZZ, PPP);  // ZZZ3 = ZZZ1 PPP
  f_mul<T, true>(Q, acc.X, PP);           // Q = X1 PP
  f_mul<T, true>(P, R, R);
  T::sub(P, P, PPP);
  T::sub(P, P, Q);
  T::sub(P, P, Q);                        // X3 = R^2 - PPP - 2 Q
  T::sub(Q, Q, P);
  f_mul<T, true>(Q, R, Q);                // R (Q - X3)
  f_mul<T, true>(PPP, acc.Y, PPP);
  T::sub(acc.Y, Q, PPP);                  // Y3 = R (Q - X3) - Y1 PPP
  fv_copy<L>(acc.X, P);
}

// acc += q (add-2008-s).
template <class T, bool kCall = false>
__device__ __forceinline__ void xyzz_add(Xyzz<T> &acc, const Xyzz<T> &q) {
  constexpr int L = T::L;
  if (xyzz_is_inf(q)) return;
  if (xyzz_is_inf(acc)) {
    acc = q;
    return;
  }
  uint32_t U1[L], S1[L], P[L], R[L], PP[L], PPP[L];
  f_mul<T, kCall>(U1, acc.X, q.ZZ);       // U1 = X1 ZZ2
  f_mul<T, kCall>(S1, acc.Y, q.ZZZ);      // S1 = Y1 ZZZ2
  f_mul<T, kCall>(P, q.X, acc.ZZ);
  T::sub(P, P, U1);                       // P = U2 - U1
  f_mul<T, kCall>(R, q.Y, acc.ZZZ);
  T::sub(R, R, S1);                       // R = S2 - S1
  if (fv_is_zero<L>(P)) {
    if (fv_is_zero<L>(R)) xyzz_dbl<T, kCall>(acc, q);
    else xyzz_set_inf(acc);
    return;
  }
  f_mul<T, kCall>(PP, P, P);
  f_mul<T, kCall>(PPP, P, PP);
  f_mul<T, kCall>(acc.ZZ, acc.ZZ, q.ZZ);
  f_mul<T, kCall>(acc.ZZ, acc.ZZ, PP);    // ZZ3 = ZZ1 ZZ2 PP
  f_mul<T, kCall>(acc.ZZZ, acc.ZZZ, q.ZZZ);
  f_mul<T, kCall>(acc.ZZZ, acc.ZZZ, PPP); // ZZZ3 = ZZZ1 ZZZ2 PPP
  f_mul<T, kCall>(U1, U1, PP);            // Q = U1 PP
  f_mul<T, kCall>(P, R, R);
  T::sub(P, P, PPP);
  T::sub(P, P, U1);
  T::sub(P, P, U1);                       // X3 = R^2 - PPP - 2 Q
  T::sub(U1, U1, P);
  f_mul<T, kCall>(U1, R, U1);             // R (Q - X3)
  f_mul<T, kCall>(S1, S1, PPP);
  T::sub(acc.Y, U1, S1);                  // Y3 = R (Q - X3) - S1 PPP
  fv_copy<L>(acc.X, P);
}

// r = a^(q-2) = a^-1 (Fermat), Montgomery in and out; a = 0 gives 0.
template <class T>
__device__ __forceinline__ void f_inverse(uint32_t r[T::L], const uint32_t a[T::L], const uint32_t one[T::L]) {
  uint32_t acc[T::L];
  fv_copy<T::L>(acc, one);
  for (int i = T::kTopBit; i >= 0; --i) {
    T::mul(acc, acc, acc);
    if ((T::inv_exp(i >> 5) >> (i & 31)) & 1u) T::mul(acc, acc, a);
  }
  fv_copy<T::L>(r, acc);
}

// Affine point of p in STANDARD form (x, y); O gives (0, 0).
template <class T>
__device__ __forceinline__ void xyzz_to_affine_std(uint32_t x[T::L], uint32_t y[T::L], const Xyzz<T> &p,
                                                   const uint32_t one[T::L]) {
  constexpr int L = T::L;
  if (xyzz_is_inf(p)) {
    fv_zero<L>(x);
    fv_zero<L>(y);
    return;
  }
  uint32_t t[L], inv[L], zi[L];
  T::mul(t, p.ZZ, p.ZZZ);
  f_inverse<T>(inv, t, one);  // (ZZ ZZZ)^-1
  T::mul(zi, inv, p.ZZZ);     // ZZ^-1
  T::mul(t, p.X, zi);
  T::redc(x, t);
  T::mul(zi, inv, p.ZZ);      // ZZZ^-1
  T::mul(t, p.Y, zi);
  T::redc(y, t);
}

}  // namespace gb300ntt
