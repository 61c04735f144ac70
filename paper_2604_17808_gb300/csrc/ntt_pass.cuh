// ntt_pass.cuh -- one pass of the multi-pass (four-/six-step) NTT on sm_103a.
//
// Decomposition (the paper's 3-step / 5-step NTT, Sec. 3.3.2, Fig. 4b-c and
// Eq. 1, in the standard Cooley-Tukey index map): N = S_0 * S_1 * ... *
// S_{P-1}.  Write the input index as n = sum_j n_j * N / (S_0 ... S_j), so
// digit n_0 has the largest stride.  Then
//
//   pass 0:      for every value of the other digits, a size-S_0 DFT over
//                n_0 (input stride N/S_0); the result for output digit k_0
//                is stored at k_0 + S_0 * rev(n_1..n_{P-1}), i.e. the
//                untransformed digits are written in reversed significance
//                (this is the transpose of the four-step method);
//   pass j >= 1: in place, buffer position q + Mp*n_j + M*o with
//                Mp = S_0...S_{j-1}, M = Mp*S_j: each input is multiplied by
//                the inter-pass twiddle omega_M^(n_j*q) (the element-wise
//                "TF" product between the matrix steps of Eq. 1), then a
//                size-S_j DFT over n_j.  q is the already transformed low
//                part of the output index, o the untransformed rest.
//
// After the last pass the buffer holds X in natural order.  Coset and
// inverse scale factors are folded into the same per-element multipliers.
//
// Work split on the GPU: one CTA (256 threads, 8 warps) owns a tile of
// 2048 elements = G = 2048/S sub-transforms with consecutive sub-transform
// index, staged in shared memory.
//   load phase : consecutive threads read consecutive 32-byte elements
//                (coalesced), multiply by the input multiplier (pass >= 1:
//                omega_M^(n q), read with the same coalesced pattern), and
//                write the tile;
//   warp phase : warp w transforms tile elements [256w, 256w+256) -- one
//                sub-transform of 256 points or 256/S smaller ones -- as a
//                decimation-in-frequency (Gentleman-Sande) radix-2 network in
//                registers, 8 elements per lane, in rounds of up to three
//                stages (radix-8) with a shared-memory exchange between
//                rounds;
//   store phase: coalesced 32-byte stores of the tile in natural order.
// The shared tile is XOR-swizzled on 16-byte chunks so that the access
// patterns of all three phases are free of bank conflicts for S = 256.
#pragma once

#include <cstdint>

#include "fp256.cuh"

namespace gb300ntt {

constexpr int kPassThreads = 256;
constexpr int kTileLog = 11;                       // 2048 elements per CTA
constexpr int kTileElems = 1 << kTileLog;
constexpr int kTileBytes = kTileElems * 32;       // 64 KiB
constexpr int kMaxPassLog = 8;                     // sub-transforms up to 256 points

enum PassMode : int {
  kModeInner = 0,     // pass j >= 1: in place, 2-D input multiplier table [S][Mp]
  kModeFirst = 1,     // pass 0 without input multiplier
  kModeFirstPre = 2,  // pass 0 with a per-n_0 input multiplier table [S]
};

struct PassArgs {
  const uint4 *src;      // input elements (2 x uint4 each)
  uint4 *dst;            // output elements
  const uint4 *mul;      // input multipliers (Montgomery form) or nullptr
  const uint4 *dft_tw;   // omega_S^i, i < S/2 (Montgomery form)
  uint64_t num_sub;      // number of sub-transforms in the pass, N / S
  uint32_t log_mp;       // inner: log2 Mp; first: log2(N / S)
  uint32_t num_digits;   // first: P - 1 untransformed digits to reverse
  uint32_t digit_log[4];    // first: log2 S_j of digit j (j = 1..P-1) at index j-1
  uint32_t digit_shift[4];  // first: log2(S_1 ... S_{j-1}) at index j-1
};

// 16-byte chunk index of half h of tile element e (bank-conflict swizzle).
__device__ __forceinline__ uint32_t tile_chunk(uint32_t e, uint32_t h) {
  const uint32_t x = e >> 2;
  return ((e << 1) | h) ^ ((x ^ (x >> 3) ^ (x >> 6)) & 7u);
}

__device__ __forceinline__ void tile_store(uint4 *tile, uint32_t e, const uint32_t a[8]) {
  tile[tile_chunk(e, 0)] = make_uint4(a[0], a[1], a[2], a[3]);
  tile[tile_chunk(e, 1)] = make_uint4(a[4], a[5], a[6], a[7]);
}

__device__ __forceinline__ void tile_load(uint32_t r[8], const uint4 *tile, uint32_t e) {
  const uint4 lo = tile[tile_chunk(e, 0)];
  const uint4 hi = tile[tile_chunk(e, 1)];
  r[0] = lo.x; r[1] = lo.y; r[2] = lo.z; r[3] = lo.w;
  r[4] = hi.x; r[5] = hi.y; r[6] = hi.z; r[7] = hi.w;
}

// ------------------------------------------------------- round structure
// A size-2^LOGS DIF network is split into R = ceil(LOGS/3) rounds, from the
// top bit down; round sizes are as equal as possible with the larger ones
// first, so the last round has at least two bits whenever LOGS >= 2.

__host__ __device__ constexpr int num_rounds(int logs) { return (logs + 2) / 3; }

__host__ __device__ constexpr int round_bits(int logs, int r) {
  return logs / num_rounds(logs) + (r < logs % num_rounds(logs) ? 1 : 0);
}

__host__ __device__ constexpr int round_low(int logs, int r) {
  int hi = logs;
  for (int i = 0; i <= r; ++i) hi -= round_bits(logs, i);
  return hi;
}

// Warp-local position (8 bits) of register slot `slot` of `lane` in a round
// that owns position bits [T, T+B): slot bits 0..B-1 are the round bits, the
// five lane bits fill the lowest remaining position bits, and the remaining
// 3-B slot bits fill the rest.
template <int T, int B>
__device__ __forceinline__ uint32_t slot_pos(uint32_t lane, int slot) {
  uint32_t pos = 0;
  int li = 0, si = B;
#pragma unroll
  for (int bit = 0; bit < 8; ++bit) {
    if (bit >= T && bit < T + B) {
      pos |= (uint32_t)((slot >> (bit - T)) & 1) << bit;
    } else if (li < 5) {
      pos |= ((lane >> li) & 1u) << bit;
      ++li;
    } else {
      pos |= (uint32_t)((slot >> si) & 1) << bit;
      ++si;
    }
  }
  return pos;
}

template <int LOGS>
__device__ __forceinline__ uint32_t bit_reverse_local(uint32_t p) {
  return LOGS == 0 ? 0u : (__brev(p) >> (32 - LOGS));
}

// One round of DIF stages (bits T+B-1 down to T) on the lane's 8 registers.
template <class F, int LOGS, int T, int B>
__device__ __forceinline__ void dif_round(uint32_t (&x)[8][8], uint32_t lane, const uint4 *twt) {
  constexpr uint32_t S = 1u << LOGS;
#pragma unroll
  for (int beta = T + B - 1; beta >= T; --beta) {
    const int sb = beta - T;
#pragma unroll
    for (int s0 = 0; s0 < 8; ++s0) {
      if (s0 & (1 << sb)) continue;
      const int s1 = s0 | (1 << sb);
      uint32_t d[8];
      sub_mod<F>(d, x[s0], x[s1]);
      add_mod<F>(x[s0], x[s0], x[s1]);
      // twiddle omega_{2h}^(p mod h), h = 2^beta, as index into omega_S^i
      const bool trivial = (beta == 0) || (T == 0 && (s0 & ((1 << beta) - 1)) == 0);
      if (trivial) {
        fe_copy(x[s1], d);
      } else {
        const uint32_t p = slot_pos<T, B>(lane, s0) & (S - 1);
        const uint32_t idx = (p & ((1u << beta) - 1)) << (LOGS - 1 - beta);
        uint32_t w[8];
        tile_load(w, twt, idx);
        mont_mul<F>(x[s1], d, w);
      }
    }
  }
}

// The tile pointer passed around is the CTA's tile; warp w works on tile
// elements [256w, 256w + 256), so positions are offset by `base`.
struct WarpTile {
  uint4 *tile;
  uint32_t base;
};

__device__ __forceinline__ void wt_store(const WarpTile &t, uint32_t pos, const uint32_t a[8]) {
  tile_store(t.tile, t.base + pos, a);
}
__device__ __forceinline__ void wt_load(uint32_t r[8], const WarpTile &t, uint32_t pos) {
  tile_load(r, t.tile, t.base + pos);
}

template <int T, int B>
__device__ __forceinline__ void wround_store(const WarpTile &t, uint32_t lane, const uint32_t (&x)[8][8]) {
#pragma unroll
  for (int s = 0; s < 8; ++s) wt_store(t, slot_pos<T, B>(lane, s), x[s]);
}

template <int T, int B>
__device__ __forceinline__ void wround_load(uint32_t (&x)[8][8], uint32_t lane, const WarpTile &t) {
#pragma unroll
  for (int s = 0; s < 8; ++s) wt_load(x[s], t, slot_pos<T, B>(lane, s));
}

// Round r and everything after it; exchange through shared memory between
// rounds.  On entry the registers hold round r's layout.
template <class F, int LOGS, int R>
__device__ __forceinline__ void warp_rounds(uint32_t (&x)[8][8], uint32_t lane, const WarpTile &t,
                                            const uint4 *twt) {
  constexpr int T = round_low(LOGS, R);
  constexpr int B = round_bits(LOGS, R);
  dif_round<F, LOGS, T, B>(x, lane, twt);
  if constexpr (R + 1 < num_rounds(LOGS)) {
    constexpr int T2 = round_low(LOGS, R + 1);
    constexpr int B2 = round_bits(LOGS, R + 1);
    __syncwarp();
    wround_store<T, B>(t, lane, x);
    __syncwarp();
    wround_load<T2, B2>(x, lane, t);
    warp_rounds<F, LOGS, R + 1>(x, lane, t, twt);
  } else {
    // DIF leaves position p holding output bitrev(p): write it to its
    // natural place in the sub-transform.
    constexpr uint32_t S = 1u << LOGS;
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const uint32_t p = slot_pos<T, B>(lane, s);
      wt_store(t, (p & ~(S - 1)) | bit_reverse_local<LOGS>(p & (S - 1)), x[s]);
    }
  }
}

// Size-2^LOGS DFTs of all sub-transforms of the warp's 256 tile elements,
// in place in shared memory (natural order in and out).
template <class F, int LOGS>
__device__ __forceinline__ void warp_dft(const WarpTile &t, uint32_t lane, const uint4 *twt) {
  uint32_t x[8][8];
  constexpr int T0 = round_low(LOGS, 0);
  constexpr int B0 = round_bits(LOGS, 0);
  wround_load<T0, B0>(x, lane, t);
  warp_rounds<F, LOGS, 0>(x, lane, t, twt);
}

// ------------------------------------------------------------ pass kernel

template <class F, int LOGS, int MODE>
__global__ void __launch_bounds__(kPassThreads, 2) ntt_pass_kernel(const PassArgs a) {
  extern __shared__ uint4 smem[];
  uint4 *tile = smem;
  uint4 *twt = smem + 2 * kTileElems;
  constexpr uint32_t S = 1u << LOGS;
  constexpr int LOGG = kTileLog - LOGS;
  constexpr uint32_t G = 1u << LOGG;

  // DFT twiddles omega_S^i (i < S/2) into shared memory.
  for (uint32_t i = threadIdx.x; i < (S / 2) * 2; i += kPassThreads) {
    const uint32_t e = i >> 1, h = i & 1;
    twt[tile_chunk(e, h)] = __ldg(a.dft_tw + i);
  }

  const uint64_t d0 = (uint64_t)blockIdx.x << LOGG;
  const uint64_t mp_mask = (1ull << a.log_mp) - 1;

  // ---------------- load phase: element e of the tile = (n, dl), n-major
#pragma unroll 2
  for (int i = 0; i < kTileElems / kPassThreads; ++i) {
    const uint32_t e = threadIdx.x + kPassThreads * i;
    const uint32_t n = e >> LOGG, dl = e & (G - 1);
    const uint64_t d = d0 + dl;
    if (d < a.num_sub) {
      uint32_t v[8];
      if constexpr (MODE == kModeInner) {
        const uint64_t q = d & mp_mask, o = d >> a.log_mp;
        const uint64_t pos = q + ((uint64_t)n << a.log_mp) + (o << (a.log_mp + LOGS));
        fe_load_global(v, a.src, pos);
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
      tile_store(tile, (dl << LOGS) | n, v);
    }
  }
  __syncthreads();

  // ---------------- warp phase
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  warp_dft<F, LOGS>(WarpTile{tile, warp * 256u}, lane, twt);
  __syncthreads();

  // ---------------- store phase
#pragma unroll 2
  for (int i = 0; i < kTileElems / kPassThreads; ++i) {
    const uint32_t e = threadIdx.x + kPassThreads * i;
    if constexpr (MODE == kModeInner) {
      const uint32_t k = e >> LOGG, dl = e & (G - 1);
      const uint64_t d = d0 + dl;
      if (d < a.num_sub) {
        const uint64_t q = d & mp_mask, o = d >> a.log_mp;
        const uint64_t pos = q + ((uint64_t)k << a.log_mp) + (o << (a.log_mp + LOGS));
        uint32_t v[8];
        tile_load(v, tile, (dl << LOGS) | k);
        fe_store_global(a.dst, pos, v);
      }
    } else {
      const uint32_t dl = e >> LOGS, k = e & (S - 1);
      const uint64_t d = d0 + dl;
      if (d < a.num_sub) {
        // reverse the significance of the untransformed digits of d
        uint64_t rest = d, rev = 0;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
          if (j < (int)a.num_digits) {
            const uint64_t nj = rest & ((1ull << a.digit_log[j]) - 1);
            rest >>= a.digit_log[j];
            rev |= nj << a.digit_shift[j];
          }
        }
        uint32_t v[8];
        tile_load(v, tile, e);
        fe_store_global(a.dst, (rev << LOGS) | k, v);
      }
    }
  }
}

inline int pass_smem_bytes(int logs) { return kTileBytes + (1 << logs) / 2 * 32; }

}  // namespace gb300ntt
