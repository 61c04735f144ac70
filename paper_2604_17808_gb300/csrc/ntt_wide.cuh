// ntt_wide.cuh -- NTT over the 377- and 753-bit fields (12 and 24 limbs).
//
// The paper evaluates its NTT at 256, 377 and 753 bits (Sec. 4.3.1,
// Tab. 3).  These fields reuse the pass decomposition of ntt_pass.cuh
// (four-/six-step passes, digit-reversed first pass, in-place inner passes
// with the inter-pass twiddle on load, bit-reversed store), with a
// generic-limb arithmetic: the modulus lives in constant memory and the
// Montgomery product (CIOS, 32-bit limbs) is written with 64-bit
// accumulations, which compile to full-rate wide IMADs.  Elements are NL
// consecutive 32-bit words in memory (48 or 96 bytes), standard form,
// canonical; constants are in Montgomery form, so mul(x, c R) = x c.
//
// Tile: 2^TL elements in shared memory, one padding word per element (an
// odd stride keeps word accesses of consecutive elements conflict-free),
// 256 threads, one radix-2 DIF stage per barrier.
#pragma once

#include <cstdint>

#include "ntt_pass.cuh"

namespace gb300ntt {

template <int NL>
struct WideConst {
  uint32_t p[NL];
  uint32_t ninv;        // -p^-1 mod 2^32
  uint32_t one[NL];     // R mod p (Montgomery 1), R = 2^(32 NL)
  uint32_t r2[NL];      // R^2 mod p
  uint32_t exp_c[NL];   // c = (p - 1) / 2^32 (the odd part), for the root of order 2^32
  uint32_t gen;         // generator (a quadratic non-residue)
};

// Field constants (filled once per device by the host; this header is
// included by one translation unit only).
__constant__ WideConst<12> c_wide12;
__constant__ WideConst<24> c_wide24;

template <int NL>
__device__ __forceinline__ const WideConst<NL> &wide_const();
template <>
__device__ __forceinline__ const WideConst<12> &wide_const<12>() { return c_wide12; }
template <>
__device__ __forceinline__ const WideConst<24> &wide_const<24>() { return c_wide24; }

// r = a b R^-1 mod p (CIOS; a, b < p; r canonical; r may alias a or b).
template <int NL>
__device__ __forceinline__ void wide_mul(uint32_t r[NL], const uint32_t a[NL], const uint32_t b[NL]) {
  const WideConst<NL> &C = wide_const<NL>();
  uint32_t t[NL + 2];
#pragma unroll
  for (int j = 0; j < NL + 2; ++j) t[j] = 0;
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    uint64_t c = 0;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const uint64_t s = (uint64_t)a[i] * b[j] + t[j] + c;
      t[j] = (uint32_t)s;
      c = s >> 32;
    }
    uint64_t s = (uint64_t)t[NL] + c;
    t[NL] = (uint32_t)s;
    t[NL + 1] = (uint32_t)(s >> 32);
    const uint32_t m = t[0] * C.ninv;
    c = ((uint64_t)m * C.p[0] + t[0]) >> 32;
#pragma unroll
    for (int j = 1; j < NL; ++j) {
      const uint64_t u = (uint64_t)m * C.p[j] + t[j] + c;
      t[j - 1] = (uint32_t)u;
      c = u >> 32;
    }
    s = (uint64_t)t[NL] + c;
    t[NL - 1] = (uint32_t)s;
    t[NL] = t[NL + 1] + (uint32_t)(s >> 32);
    t[NL + 1] = 0;
  }
  // t < 2p: subtract p once if t >= p
  uint32_t d[NL];
  int64_t br = 0;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    const int64_t v = (int64_t)t[j] - C.p[j] + br;
    d[j] = (uint32_t)v;
    br = v >> 32;
  }
  const bool ge = (int64_t)t[NL] + br >= 0;
#pragma unroll
  for (int j = 0; j < NL; ++j) r[j] = ge ? d[j] : t[j];
}

template <int NL>
__device__ __forceinline__ void wide_add(uint32_t r[NL], const uint32_t a[NL], const uint32_t b[NL]) {
  const WideConst<NL> &C = wide_const<NL>();
  uint32_t s[NL], d[NL];
  uint64_t c = 0;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    const uint64_t v = (uint64_t)a[j] + b[j] + c;
    s[j] = (uint32_t)v;
    c = v >> 32;
  }
  int64_t br = 0;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    const int64_t v = (int64_t)s[j] - C.p[j] + br;
    d[j] = (uint32_t)v;
    br = v >> 32;
  }
  const bool ge = (int64_t)c + br >= 0;   // a + b >= p
#pragma unroll
  for (int j = 0; j < NL; ++j) r[j] = ge ? d[j] : s[j];
}

template <int NL>
__device__ __forceinline__ void wide_sub(uint32_t r[NL], const uint32_t a[NL], const uint32_t b[NL]) {
  const WideConst<NL> &C = wide_const<NL>();
  uint32_t d[NL];
  int64_t br = 0;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    const int64_t v = (int64_t)a[j] - b[j] + br;
    d[j] = (uint32_t)v;
    br = v >> 32;
  }
  if (br < 0) {   // a < b: add p back
    uint64_t c = 0;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const uint64_t v = (uint64_t)d[j] + C.p[j] + c;
      d[j] = (uint32_t)v;
      c = v >> 32;
    }
  }
#pragma unroll
  for (int j = 0; j < NL; ++j) r[j] = d[j];
}

template <int NL>
__device__ __forceinline__ void wide_load(uint32_t r[NL], const uint4 *base, uint64_t elem) {
  const uint4 *p = base + elem * (NL / 4);
#pragma unroll
  for (int k = 0; k < NL / 4; ++k) {
    const uint4 v = __ldg(p + k);
    r[4 * k] = v.x; r[4 * k + 1] = v.y; r[4 * k + 2] = v.z; r[4 * k + 3] = v.w;
  }
}

template <int NL>
__device__ __forceinline__ void wide_store(uint4 *base, uint64_t elem, const uint32_t a[NL]) {
  uint4 *p = base + elem * (NL / 4);
#pragma unroll
  for (int k = 0; k < NL / 4; ++k) p[k] = make_uint4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
}

template <int NL>
__device__ __forceinline__ void wide_tile_load(uint32_t r[NL], const uint32_t *tile, uint32_t e) {
#pragma unroll
  for (int j = 0; j < NL; ++j) r[j] = tile[e * (NL + 1) + j];
}

template <int NL>
__device__ __forceinline__ void wide_tile_store(uint32_t *tile, uint32_t e, const uint32_t a[NL]) {
#pragma unroll
  for (int j = 0; j < NL; ++j) tile[e * (NL + 1) + j] = a[j];
}

// Tile shape per limb count: 2^10 elements for 12 limbs, 2^9 for 24.
template <int NL>
struct WideTile {
  static constexpr int kLog = NL <= 12 ? 10 : 9;
  static constexpr int kElems = 1 << kLog;
  static constexpr int kThreads = 256;
  static constexpr int kBytes = kElems * (NL + 1) * 4;
};

template <int NL, int LOGS, int MODE>
__global__ void __launch_bounds__(256) wide_pass_kernel(const PassArgs a) {
  constexpr int TL = WideTile<NL>::kLog;
  constexpr int kThreads = WideTile<NL>::kThreads;
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
    uint32_t v[NL];
    if constexpr (MODE == kModeInner) {
      const uint64_t q = d & mp_mask, o = d >> a.log_mp;
      wide_load<NL>(v, a.src, q + ((uint64_t)n << a.log_mp) + (o << (a.log_mp + LOGS)));
      uint32_t w[NL];
      wide_load<NL>(w, a.mul, ((uint64_t)n << a.log_mp) + q);
      wide_mul<NL>(v, v, w);
    } else {
      wide_load<NL>(v, a.src, d + ((uint64_t)n << a.log_mp));
      if constexpr (MODE == kModeFirstPre) {
        uint32_t w[NL];
        wide_load<NL>(w, a.mul, n);
        wide_mul<NL>(v, v, w);
      }
    }
    wide_tile_store<NL>(tile, (dl << LOGS) | n, v);
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
      uint32_t x[NL], y[NL], dd[NL];
      wide_tile_load<NL>(x, tile, e0);
      wide_tile_load<NL>(y, tile, e0 | h);
      wide_sub<NL>(dd, x, y);
      wide_add<NL>(x, x, y);
      if (low != 0) {
        uint32_t w[NL];
        wide_load<NL>(w, a.dft_tw, (uint64_t)low << (LOGS - 1 - T));
        wide_mul<NL>(y, dd, w);
      } else {
#pragma unroll
        for (int j = 0; j < NL; ++j) y[j] = dd[j];
      }
      wide_tile_store<NL>(tile, e0, x);
      wide_tile_store<NL>(tile, e0 | h, y);
    }
  }
  __syncthreads();
  // store phase: the DIF output order is undone by reading bit-reversed positions
#pragma unroll 1
  for (uint32_t e = threadIdx.x; e < (1u << TL); e += kThreads) {
    uint32_t v[NL];
    if constexpr (MODE == kModeInner) {
      const uint32_t k = e >> LOGG, dl = e & (G - 1);
      const uint64_t d = d0 + dl;
      if (d >= a.num_sub) continue;
      const uint64_t q = d & mp_mask, o = d >> a.log_mp;
      wide_tile_load<NL>(v, tile, (dl << LOGS) | (LOGS ? (__brev(k) >> (32 - LOGS)) : 0u));
      wide_store<NL>(a.dst, q + ((uint64_t)k << a.log_mp) + (o << (a.log_mp + LOGS)), v);
    } else {
      const uint32_t dl = e >> LOGS, k = e & (S - 1);
      const uint64_t d = d0 + dl;
      if (d >= a.num_sub) continue;
      wide_tile_load<NL>(v, tile, (dl << LOGS) | (LOGS ? (__brev(k) >> (32 - LOGS)) : 0u));
      wide_store<NL>(a.dst, (reverse_digits(a, d) << LOGS) | k, v);
    }
  }
}

// ---------------------------------------------------------------- tables

// out[0] = base^e (Montgomery form in and out), one thread.
template <int NL>
__device__ void wide_pow(uint32_t out[NL], const uint32_t base[NL], const uint32_t *e, int words) {
  const WideConst<NL> &C = wide_const<NL>();
  uint32_t acc[NL], b[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    acc[j] = C.one[j];
    b[j] = base[j];
  }
  for (int w = 0; w < words; ++w)
    for (int bit = 0; bit < 32; ++bit) {
      if ((e[w] >> bit) & 1) wide_mul<NL>(acc, acc, b);
      wide_mul<NL>(b, b, b);
    }
#pragma unroll
  for (int j = 0; j < NL; ++j) out[j] = acc[j];
}

// Per transform size 2^log_m: writes to `k` (Montgomery form, NL words each)
//   k[0..31]   omega_M^(2^b)      k[32..63]  omega_M^-(2^b)
//   k[64]      M^-1               k[65]      R mod p (one)
// One thread.
template <int NL>
__global__ void wide_constants_kernel(uint32_t *k, uint32_t log_m) {
  const WideConst<NL> &C = wide_const<NL>();
  uint32_t g[NL], root[NL], w[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) g[j] = j == 0 ? C.gen : 0u;
  wide_mul<NL>(g, g, C.r2);                 // generator in Montgomery form
  wide_pow<NL>(root, g, C.exp_c, NL);       // primitive 2^32-th root
  for (uint32_t i = log_m; i < 32; ++i) wide_mul<NL>(root, root, root);   // omega_M
  for (int j = 0; j < NL; ++j) w[j] = root[j];
  for (int b = 0; b < 32; ++b) {
    for (int j = 0; j < NL; ++j) k[b * NL + j] = w[j];
    wide_mul<NL>(w, w, w);
  }
  // omega^-1 = omega^(M - 1)
  uint32_t e[1] = {(uint32_t)((1ull << log_m) - 1)};
  uint32_t inv[NL];
  wide_pow<NL>(inv, root, e, 1);
  for (int b = 0; b < 32; ++b) {
    for (int j = 0; j < NL; ++j) k[(32 + b) * NL + j] = inv[j];
    wide_mul<NL>(inv, inv, inv);
  }
  // M^-1 = p - (p - 1) / M, then to Montgomery form
  uint32_t mi[NL];
  {
    // (p - 1) >> log_m
    uint32_t pm1[NL];
    for (int j = 0; j < NL; ++j) pm1[j] = C.p[j];
    pm1[0] -= 1;   // p is odd: no borrow
    for (int j = 0; j < NL; ++j) {
      const uint64_t lo = pm1[j], hi = j + 1 < NL ? pm1[j + 1] : 0u;
      mi[j] = log_m ? (uint32_t)(((hi << 32) | lo) >> log_m) : (uint32_t)lo;
    }
    int64_t br = 0;
    for (int j = 0; j < NL; ++j) {
      const int64_t v = (int64_t)C.p[j] - mi[j] + br;
      mi[j] = (uint32_t)v;
      br = v >> 32;
    }
    wide_mul<NL>(mi, mi, C.r2);
  }
  for (int j = 0; j < NL; ++j) k[64 * NL + j] = mi[j];
  for (int j = 0; j < NL; ++j) k[65 * NL + j] = C.one[j];
}

// out[n * Mp + q] = init * base^(n q)  (two_d: the inter-pass table), or
// out[i] = init * base^i; ladder[b] = base^(2^b); a null ladder gives the
// constant table out[i] = init.
template <int NL>
__global__ void wide_table_kernel(uint4 *out, uint32_t log_s, uint32_t log_mp, const uint32_t *ladder,
                                  const uint32_t *init, uint64_t count, int two_d) {
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < count;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t e = !ladder ? 0 : two_d ? (idx >> log_mp) * (idx & ((1ull << log_mp) - 1)) : idx;
    uint32_t acc[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) acc[j] = init[j];
    for (int b = 0; b < 32 && (e >> b) != 0; ++b) {
      if ((e >> b) & 1) {
        uint32_t w[NL];
#pragma unroll
        for (int j = 0; j < NL; ++j) w[j] = ladder[b * NL + j];
        wide_mul<NL>(acc, acc, w);
      }
    }
    wide_store<NL>(out, idx, acc);
  }
  (void)log_s;
}

}  // namespace gb300ntt
