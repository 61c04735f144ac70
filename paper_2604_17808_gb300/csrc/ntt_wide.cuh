// ntt_wide.cuh -- NTT over the 377- and 753-bit fields (12 and 24 limbs).
//
// The paper evaluates its NTT at 256, 377 and 753 bits (Sec. 4.3.1,
// Tab. 3).  These fields reuse the pass decomposition of ntt_pass.cuh
// (four-/six-step passes, digit-reversed first pass, in-place inner passes
// with the inter-pass twiddle on load, bit-reversed store), with a
// generic-limb arithmetic: the modulus lives in constant memory, elements
// are held in 29-bit limbs inside the kernels, and the Montgomery product
// (CIOS in radix 2^29) accumulates limb products in 64-bit registers with
// one full-rate mad.wide each and no carry chain.  Elements are NL32
// consecutive 32-bit words in memory (48 or 96 bytes), standard form,
// canonical; constants are in Montgomery form, so mul(x, c R) = x c.
//
// Tile: 2^TL elements in shared memory (29-bit limbs plus one padding word
// per element: an odd stride keeps word accesses of consecutive elements
// conflict-free), 256 threads, one radix-2 DIF stage per barrier.
//
// Multipliers: the first pass's table (mode kModeFirstPre) is indexed by
// the input position (the coset factors s^i, or N^-1 for a one-pass
// inverse), the inner passes' by (n, q) as in ntt_pass.cuh, and the
// optional output table `post` by the output position (s^-i in the last
// pass of a coset inverse).
#pragma once

#include <cstdint>

#include "ntt_pass.cuh"

namespace gb300ntt {

// Internal limb layout: L limbs of 29 bits (14 for the 377-bit field, 26
// for the 753-bit one; 29 L >= the modulus bits), so that a limb product is
// below 2^58 and a 64-bit accumulator takes 2^6 of them: the Montgomery
// product needs no carry chain inside its rows (one full-rate mad.wide per
// limb product) and normalises once at the end.  Memory elements stay NL32
// 32-bit words (48 or 96 bytes); tables hold LP = L rounded up to 4 words.
template <int NL32>
struct WideShape {
  static constexpr int L = NL32 == 12 ? 14 : 26;
  static constexpr int LP = (L + 3) / 4 * 4;
  static constexpr int kLog = NL32 <= 12 ? 10 : 9;   // tile: 2^kLog elements
  static constexpr int kElems = 1 << kLog;
  static constexpr int kThreads = 256;
  static constexpr int kBytes = kElems * (L + 1) * 4;   // one padding word per element
};

constexpr uint32_t kM29 = (1u << 29) - 1;

template <int NL32>
struct WideConst {
  static constexpr int L = WideShape<NL32>::L;
  uint32_t p[L];            // modulus, 29-bit limbs
  uint32_t p32[NL32];       // modulus, 32-bit words
  uint32_t ninv;            // -p^-1 mod 2^29
  uint32_t one[L];          // R mod p, R = 2^(29 L)
  uint32_t r2[L];           // R^2 mod p
  uint32_t exp_c[NL32];     // (p - 1) / 2^32, 32-bit words
  uint32_t gen;             // generator (a quadratic non-residue)
};

// Field constants (filled once per device by the host; this header is
// included by one translation unit only).
__constant__ WideConst<12> c_wide12;
__constant__ WideConst<24> c_wide24;

template <int NL32>
__device__ __forceinline__ const WideConst<NL32> &wide_const();
template <>
__device__ __forceinline__ const WideConst<12> &wide_const<12>() { return c_wide12; }
template <>
__device__ __forceinline__ const WideConst<24> &wide_const<24>() { return c_wide24; }

// r = r - p if r >= p (limbs normalised, r < 2p).
template <int NL32>
__device__ __forceinline__ void wide_reduce_once(uint32_t r[WideShape<NL32>::L]) {
  constexpr int L = WideShape<NL32>::L;
  const WideConst<NL32> &C = wide_const<NL32>();
  uint32_t d[L];
  int32_t br = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int32_t v = (int32_t)r[j] - (int32_t)C.p[j] + br;
    br = v >> 29;                      // 0 or -1
    d[j] = (uint32_t)v & kM29;
  }
  if (br == 0) {
#pragma unroll
    for (int j = 0; j < L; ++j) r[j] = d[j];
  }
}

// r = a b R^-1 mod p (CIOS in radix 2^29; a, b < p; r canonical; may alias).
template <int NL32>
__device__ __forceinline__ void wide_mul(uint32_t r[WideShape<NL32>::L], const uint32_t a[WideShape<NL32>::L],
                                         const uint32_t b[WideShape<NL32>::L]) {
  constexpr int L = WideShape<NL32>::L;
  const WideConst<NL32> &C = wide_const<NL32>();
  uint64_t t[L];
#pragma unroll
  for (int j = 0; j < L; ++j) t[j] = 0;
#pragma unroll
  for (int i = 0; i < L; ++i) {
#pragma unroll
    for (int j = 0; j < L; ++j) t[j] += (uint64_t)a[i] * b[j];
    const uint32_t m = ((uint32_t)t[0] * C.ninv) & kM29;
#pragma unroll
    for (int j = 0; j < L; ++j) t[j] += (uint64_t)m * C.p[j];
    const uint64_t c = t[0] >> 29;     // the low 29 bits of t[0] are zero now
#pragma unroll
    for (int j = 0; j < L - 1; ++j) t[j] = t[j + 1];
    t[L - 1] = 0;
    t[0] += c;
  }
  uint64_t c = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const uint64_t v = t[j] + c;
    r[j] = (uint32_t)v & kM29;
    c = v >> 29;
  }
  wide_reduce_once<NL32>(r);
}

template <int NL32>
__device__ __forceinline__ void wide_add(uint32_t r[WideShape<NL32>::L], const uint32_t a[WideShape<NL32>::L],
                                         const uint32_t b[WideShape<NL32>::L]) {
  constexpr int L = WideShape<NL32>::L;
  uint32_t c = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const uint32_t v = a[j] + b[j] + c;
    r[j] = v & kM29;
    c = v >> 29;
  }
  wide_reduce_once<NL32>(r);   // a + b < 2p < 2^(29 L): no carry out of the top limb
}

template <int NL32>
__device__ __forceinline__ void wide_sub(uint32_t r[WideShape<NL32>::L], const uint32_t a[WideShape<NL32>::L],
                                         const uint32_t b[WideShape<NL32>::L]) {
  constexpr int L = WideShape<NL32>::L;
  const WideConst<NL32> &C = wide_const<NL32>();
  int32_t br = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int32_t v = (int32_t)a[j] - (int32_t)b[j] + br;
    br = v >> 29;
    r[j] = (uint32_t)v & kM29;
  }
  if (br != 0) {   // a < b: add p back
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const uint32_t v = r[j] + C.p[j] + c;
      r[j] = v & kM29;
      c = v >> 29;
    }
  }
}

// 32-bit words <-> 29-bit limbs (values below 2^(29 L)).
template <int NL32>
__device__ __forceinline__ void wide_from_words(uint32_t r[WideShape<NL32>::L], const uint32_t x[NL32]) {
  constexpr int L = WideShape<NL32>::L;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int bit = 29 * j, w = bit >> 5, sh = bit & 31;
    const uint32_t lo = w < NL32 ? x[w] : 0u;
    const uint32_t hi = w + 1 < NL32 ? x[w + 1] : 0u;
    r[j] = __funnelshift_r(lo, hi, sh) & kM29;
  }
}

template <int NL32>
__device__ __forceinline__ void wide_to_words(uint32_t x[NL32], const uint32_t r[WideShape<NL32>::L]) {
  constexpr int L = WideShape<NL32>::L;
#pragma unroll
  for (int w = 0; w < NL32; ++w) {
    const int bit = 32 * w, j = bit / 29, sh = bit % 29;
    uint32_t v = j < L ? r[j] >> sh : 0u;
    if (j + 1 < L) v |= r[j + 1] << (29 - sh);
    if (58 - sh < 32 && j + 2 < L) v |= r[j + 2] << (58 - sh);
    x[w] = v;
  }
}

// element (NL32 words) in memory -> 29-bit limbs, and back
template <int NL32>
__device__ __forceinline__ void wide_load_elem(uint32_t r[WideShape<NL32>::L], const uint4 *base, uint64_t elem) {
  uint32_t x[NL32];
  const uint4 *p = base + elem * (NL32 / 4);
#pragma unroll
  for (int k = 0; k < NL32 / 4; ++k) {
    const uint4 v = __ldg(p + k);
    x[4 * k] = v.x; x[4 * k + 1] = v.y; x[4 * k + 2] = v.z; x[4 * k + 3] = v.w;
  }
  wide_from_words<NL32>(r, x);
}

template <int NL32>
__device__ __forceinline__ void wide_store_elem(uint4 *base, uint64_t elem, const uint32_t r[WideShape<NL32>::L]) {
  uint32_t x[NL32];
  wide_to_words<NL32>(x, r);
  uint4 *p = base + elem * (NL32 / 4);
#pragma unroll
  for (int k = 0; k < NL32 / 4; ++k) p[k] = make_uint4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
}

// table entry (LP words, 29-bit limbs)
template <int NL32>
__device__ __forceinline__ void wide_load_tab(uint32_t r[WideShape<NL32>::L], const uint4 *base, uint64_t idx) {
  constexpr int L = WideShape<NL32>::L, LP = WideShape<NL32>::LP;
  const uint4 *p = base + idx * (LP / 4);
#pragma unroll
  for (int k = 0; k < LP / 4; ++k) {
    const uint4 v = __ldg(p + k);
    if (4 * k < L) r[4 * k] = v.x;
    if (4 * k + 1 < L) r[4 * k + 1] = v.y;
    if (4 * k + 2 < L) r[4 * k + 2] = v.z;
    if (4 * k + 3 < L) r[4 * k + 3] = v.w;
  }
}

template <int NL32>
__device__ __forceinline__ void wide_store_tab(uint4 *base, uint64_t idx, const uint32_t r[WideShape<NL32>::L]) {
  constexpr int L = WideShape<NL32>::L, LP = WideShape<NL32>::LP;
  uint4 *p = base + idx * (LP / 4);
#pragma unroll
  for (int k = 0; k < LP / 4; ++k)
    p[k] = make_uint4(4 * k < L ? r[4 * k] : 0u, 4 * k + 1 < L ? r[4 * k + 1] : 0u,
                      4 * k + 2 < L ? r[4 * k + 2] : 0u, 4 * k + 3 < L ? r[4 * k + 3] : 0u);
}

template <int NL32>
__device__ __forceinline__ void wide_tile_load(uint32_t r[WideShape<NL32>::L], const uint32_t *tile, uint32_t e) {
  constexpr int L = WideShape<NL32>::L;
#pragma unroll
  for (int j = 0; j < L; ++j) r[j] = tile[e * (L + 1) + j];
}

template <int NL32>
__device__ __forceinline__ void wide_tile_store(uint32_t *tile, uint32_t e, const uint32_t a[WideShape<NL32>::L]) {
  constexpr int L = WideShape<NL32>::L;
#pragma unroll
  for (int j = 0; j < L; ++j) tile[e * (L + 1) + j] = a[j];
}

template <int NL32, int LOGS, int MODE>
__global__ void __launch_bounds__(256, 2) wide_pass_kernel(const PassArgs a) {
  constexpr int L = WideShape<NL32>::L;
  constexpr int TL = WideShape<NL32>::kLog;
  constexpr int kThreads = WideShape<NL32>::kThreads;
  constexpr uint32_t S = 1u << LOGS;
  constexpr int LOGG = TL - LOGS;
  constexpr uint32_t G = 1u << LOGG;
  static_assert(LOGS <= TL, "sub-transform larger than the tile");
  extern __shared__ uint32_t wide_smem[];
  uint32_t *tile = wide_smem;
  const uint64_t d0 = (uint64_t)blockIdx.x << LOGG;
  const uint64_t mp_mask = (1ull << a.log_mp) - 1;

  // load phase: element e = (n, dl), sub-transforms fastest across threads
#pragma unroll 1
  for (uint32_t e = threadIdx.x; e < (1u << TL); e += kThreads) {
    const uint32_t n = e >> LOGG, dl = e & (G - 1);
    const uint64_t d = d0 + dl;
    if (d >= a.num_sub) continue;
    uint32_t v[L];
    if constexpr (MODE == kModeInner) {
      const uint64_t q = d & mp_mask, o = d >> a.log_mp;
      wide_load_elem<NL32>(v, a.src, q + ((uint64_t)n << a.log_mp) + (o << (a.log_mp + LOGS)));
      uint32_t w[L];
      wide_load_tab<NL32>(w, a.mul, ((uint64_t)n << a.log_mp) + q);
      wide_mul<NL32>(v, v, w);
    } else {
      const uint64_t i = d + ((uint64_t)n << a.log_mp);   // input position
      wide_load_elem<NL32>(v, a.src, i);
      if constexpr (MODE == kModeFirstPre) {
        uint32_t w[L];
        wide_load_tab<NL32>(w, a.mul, i);
        wide_mul<NL32>(v, v, w);
      }
    }
    wide_tile_store<NL32>(tile, (dl << LOGS) | n, v);
  }
  // DIF stages, top bit down: pairs (p, p + 2^T), twiddle omega_S^((p mod 2^T) S / 2^(T+1))
#pragma unroll 1
  for (int T = LOGS - 1; T >= 0; --T) {
    __syncthreads();
    const uint32_t h = 1u << T;
#pragma unroll 1
    for (uint32_t g = threadIdx.x; g < (1u << (TL - 1)); g += kThreads) {
      const uint32_t low = g & (h - 1);
      const uint32_t e0 = low | ((g >> T) << (T + 1));
      uint32_t x[L], y[L];
      wide_tile_load<NL32>(x, tile, e0);
      wide_tile_load<NL32>(y, tile, e0 | h);
      {
        uint32_t s[L];
        wide_add<NL32>(s, x, y);
        wide_tile_store<NL32>(tile, e0, s);   // the sum leaves the registers at once
      }
      wide_sub<NL32>(y, x, y);
      if (low != 0) {
        uint32_t w[L];
        wide_load_tab<NL32>(w, a.dft_tw, (uint64_t)low << (LOGS - 1 - T));
        wide_mul<NL32>(y, y, w);
      }
      wide_tile_store<NL32>(tile, e0 | h, y);
    }
  }
  __syncthreads();
  // store phase: the DIF output order is undone by reading bit-reversed positions
#pragma unroll 1
  for (uint32_t e = threadIdx.x; e < (1u << TL); e += kThreads) {
    uint32_t v[L];
    if constexpr (MODE == kModeInner) {
      const uint32_t k = e >> LOGG, dl = e & (G - 1);
      const uint64_t d = d0 + dl;
      if (d >= a.num_sub) continue;
      const uint64_t q = d & mp_mask, o = d >> a.log_mp;
      const uint64_t pos = q + ((uint64_t)k << a.log_mp) + (o << (a.log_mp + LOGS));
      wide_tile_load<NL32>(v, tile, (dl << LOGS) | (__brev(k) >> (32 - LOGS)));
      if (a.post) {   // output multipliers (uniform across the grid)
        uint32_t w[L];
        wide_load_tab<NL32>(w, a.post, pos);
        wide_mul<NL32>(v, v, w);
      }
      wide_store_elem<NL32>(a.dst, pos, v);
    } else {
      const uint32_t dl = e >> LOGS, k = e & (S - 1);
      const uint64_t d = d0 + dl;
      if (d >= a.num_sub) continue;
      const uint64_t pos = (reverse_digits(a, d) << LOGS) | k;
      wide_tile_load<NL32>(v, tile, (dl << LOGS) | (__brev(k) >> (32 - LOGS)));
      if (a.post) {
        uint32_t w[L];
        wide_load_tab<NL32>(w, a.post, pos);
        wide_mul<NL32>(v, v, w);
      }
      wide_store_elem<NL32>(a.dst, pos, v);
    }
  }
}

// ---------------------------------------------------------------- tables

// out = base^e (Montgomery form in and out; e as 32-bit words), one thread.
template <int NL32>
__device__ void wide_pow(uint32_t out[WideShape<NL32>::L], const uint32_t base[WideShape<NL32>::L], const uint32_t *e,
                         int words) {
  constexpr int L = WideShape<NL32>::L;
  const WideConst<NL32> &C = wide_const<NL32>();
  uint32_t acc[L], b[L];
  for (int j = 0; j < L; ++j) {
    acc[j] = C.one[j];
    b[j] = base[j];
  }
  for (int w = 0; w < words; ++w)
    for (int bit = 0; bit < 32; ++bit) {
      if ((e[w] >> bit) & 1) wide_mul<NL32>(acc, acc, b);
      wide_mul<NL32>(b, b, b);
    }
  for (int j = 0; j < L; ++j) out[j] = acc[j];
}

// Per transform size 2^log_m: writes to `k` (Montgomery form, L limbs each)
//   k[0..31]   omega_M^(2^b)      k[32..63]  omega_M^-(2^b)
//   k[64]      M^-1               k[65]      R mod p (one)
// One thread.
template <int NL32>
__global__ void wide_constants_kernel(uint32_t *k, uint32_t log_m) {
  constexpr int L = WideShape<NL32>::L;
  const WideConst<NL32> &C = wide_const<NL32>();
  uint32_t g[L], root[L], w[L];
  for (int j = 0; j < L; ++j) g[j] = j == 0 ? C.gen : 0u;
  wide_mul<NL32>(g, g, C.r2);                  // generator in Montgomery form
  wide_pow<NL32>(root, g, C.exp_c, NL32);      // primitive 2^32-th root
  for (uint32_t i = log_m; i < 32; ++i) wide_mul<NL32>(root, root, root);   // omega_M
  for (int j = 0; j < L; ++j) w[j] = root[j];
  for (int b = 0; b < 32; ++b) {
    for (int j = 0; j < L; ++j) k[b * L + j] = w[j];
    wide_mul<NL32>(w, w, w);
  }
  // omega^-1 = omega^(M - 1)
  const uint32_t e[1] = {(uint32_t)((1ull << log_m) - 1)};
  uint32_t inv[L];
  wide_pow<NL32>(inv, root, e, 1);
  for (int b = 0; b < 32; ++b) {
    for (int j = 0; j < L; ++j) k[(32 + b) * L + j] = inv[j];
    wide_mul<NL32>(inv, inv, inv);
  }
  // M^-1 = p - (p - 1) / M (32-bit words), then 29-bit limbs, then Montgomery form
  uint32_t mw[NL32];
  {
    uint32_t pm1[NL32];
    for (int j = 0; j < NL32; ++j) pm1[j] = C.p32[j];
    pm1[0] -= 1;   // p is odd: no borrow
    for (int j = 0; j < NL32; ++j) {
      const uint64_t lo = pm1[j], hi = j + 1 < NL32 ? pm1[j + 1] : 0u;
      mw[j] = (uint32_t)(((hi << 32) | lo) >> log_m);
    }
    int64_t br = 0;
    for (int j = 0; j < NL32; ++j) {
      const int64_t v = (int64_t)C.p32[j] - mw[j] + br;
      mw[j] = (uint32_t)v;
      br = v >> 32;
    }
  }
  uint32_t mi[L];
  wide_from_words<NL32>(mi, mw);
  wide_mul<NL32>(mi, mi, C.r2);
  for (int j = 0; j < L; ++j) k[64 * L + j] = mi[j];
  for (int j = 0; j < L; ++j) k[65 * L + j] = C.one[j];
}

// The coset shift s for wide_table_kernel.  Reads s from k[64] (NL32
// 32-bit words, standard form, 0 < s < p: the host checks) and writes
//   k[0..31]  s^(2^b)     k[32..63]  s^-(2^b)     k[65]  R mod p (one)
// (Montgomery form; s^-1 = s^(p-2) by Fermat's little theorem).  One thread.
template <int NL32>
__global__ void wide_coset_constants_kernel(uint32_t *k) {
  constexpr int L = WideShape<NL32>::L;
  const WideConst<NL32> &C = wide_const<NL32>();
  uint32_t s[L], w[L];
  {
    uint32_t sw[NL32];
    for (int j = 0; j < NL32; ++j) sw[j] = k[64 * L + j];
    wide_from_words<NL32>(s, sw);
  }
  wide_mul<NL32>(s, s, C.r2);
  uint32_t em2[NL32];   // p - 2
  int64_t br = -2;
  for (int j = 0; j < NL32; ++j) {
    const int64_t v = (int64_t)C.p32[j] + br;
    em2[j] = (uint32_t)v;
    br = v >> 32;
  }
  uint32_t inv[L];
  wide_pow<NL32>(inv, s, em2, NL32);
  for (int j = 0; j < L; ++j) w[j] = s[j];
  for (int b = 0; b < 32; ++b) {
    for (int j = 0; j < L; ++j) k[b * L + j] = w[j];
    wide_mul<NL32>(w, w, w);
  }
  for (int b = 0; b < 32; ++b) {
    for (int j = 0; j < L; ++j) k[(32 + b) * L + j] = inv[j];
    wide_mul<NL32>(inv, inv, inv);
  }
  for (int j = 0; j < L; ++j) k[65 * L + j] = C.one[j];
}

// out[n * Mp + q] = init * base^(n q)  (two_d: the inter-pass table), or
// out[i] = init * base^i; ladder[b] = base^(2^b); a null ladder gives the
// constant table out[i] = init.  Entries in the table layout (LP words).
template <int NL32>
__global__ void wide_table_kernel(uint4 *out, uint32_t log_mp, const uint32_t *ladder, const uint32_t *init,
                                  uint64_t count, int two_d) {
  constexpr int L = WideShape<NL32>::L;
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < count;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t e = !ladder ? 0 : two_d ? (idx >> log_mp) * (idx & ((1ull << log_mp) - 1)) : idx;
    uint32_t acc[L];
#pragma unroll
    for (int j = 0; j < L; ++j) acc[j] = init[j];
    for (int b = 0; b < 32 && (e >> b) != 0; ++b) {
      if ((e >> b) & 1) {
        uint32_t w[L];
#pragma unroll
        for (int j = 0; j < L; ++j) w[j] = ladder[b * L + j];
        wide_mul<NL32>(acc, acc, w);
      }
    }
    wide_store_tab<NL32>(out, idx, acc);
  }
}

}  // namespace gb300ntt
