// ntt_pass.cuh -- one pass of the multi-pass (four-/six-step) NTT on sm_103a.
//
// Decomposition (the paper's 3-step / 5-step NTT, Sec. 3.3.2, Fig. 5b-c and
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
// Work split on the GPU: one CTA owns a tile of 2^TL elements in shared
// memory (TL = 11: 2048 elements, 256 threads; TL = 10: 1024 elements, 128
// threads) = G = 2^TL / S sub-transforms with consecutive sub-transform
// index.
//   load phase : consecutive threads read consecutive 32-byte elements
//                (coalesced), multiply by the input multiplier (pass >= 1:
//                omega_M^(n q), read with the same coalesced pattern), and
//                write the tile;
//   rounds     : decimation-in-frequency (Gentleman-Sande) radix-2 network
//                over every sub-transform of the tile, two stages at a time
//                (radix-4: each thread loads 4 elements, does 4 butterflies,
//                writes them back), the whole CTA in lockstep with a barrier
//                between rounds.  The round loop runs at run time so that the
//                hot code is one radix-4 body (small enough for the
//                instruction cache).  An odd number of stages starts with a
//                radix-2 round; the last round (stages 1 and 0) knows its
//                trivial twiddles at compile time and does 1 multiply per 4
//                elements instead of 4;
//   store phase: coalesced 32-byte stores; the DIF output order is undone by
//                reading the tile at bit-reversed positions.
// The tile is XOR-swizzled on 16-byte chunks (swz); the swizzle was chosen
// by an exhaustive check so that every access pattern of the three phases,
// for every sub-transform size 2..2048, is free of bank conflicts.
#pragma once

#include <cstdint>

#include "fp256.cuh"

namespace gb300ntt {

// Two tile shapes, chosen per pass by the plan (and its autotuner):
//   TL = 11: 2048 elements (64 KiB), 256 threads, 3 CTAs per SM;
//   TL = 10: 1024 elements (32 KiB), 128 threads, 7 CTAs per SM (224 KiB of
//            shared memory: 7168 elements resident per SM, so a 2^20-point
//            pass fits in one wave of 152 SMs).
// Every thread owns 8 elements in the load and store phases and two radix-4
// groups per round.
template <int TL>
struct TileCfg {
  static constexpr int kLog = TL;
  static constexpr int kElems = 1 << TL;
  static constexpr int kBytes = kElems * 32;
  static constexpr int kThreads = kElems / 8;
  static constexpr int kMinBlocks = TL == 11 ? 3 : 7;
};

constexpr int kPassThreads = 256;                  // batched kernel (TL = 11)
constexpr int kPassCtasPerSm = 3;
constexpr int kTileLog = 11;
constexpr int kTileBytes = TileCfg<11>::kBytes;
constexpr int kMaxPassLog = 11;                    // sub-transforms up to 2048 points
constexpr int kElemsPerThread = 8;
constexpr int kGroupsPerThread = 2;                // radix-4 groups per thread per round

enum PassMode : int {
  kModeInner = 0,     // pass j >= 1: in place, 2-D input multiplier table [S][Mp]
  kModeFirst = 1,     // pass 0 without input multiplier
  kModeFirstPre = 2,  // pass 0 with a per-n_0 input multiplier table [S]
};

// At most this many passes per transform (the matrix path splits 2^28 into
// ten passes of at most 2^3 points).
constexpr int kMaxPasses = 12;

struct PassArgs {
  const uint4 *src;      // input elements (2 x uint4 each)
  uint4 *dst;            // output elements
  const uint4 *mul;      // input multipliers (Montgomery form) or nullptr
  const uint4 *dft_tw;   // omega_S^i, i < S/2 (Montgomery form)
  uint64_t num_sub;      // number of sub-transforms in the pass, N / S
  uint32_t log_mp;       // inner: log2 Mp; first: log2(N / S)
  uint32_t num_digits;   // first: P - 1 untransformed digits to reverse
  uint8_t digit_log[kMaxPasses];    // first: log2 S_j of digit j (j = 1..P-1) at index j-1
  uint8_t digit_shift[kMaxPasses];  // first: log2(S_1 ... S_{j-1}) at index j-1
};

// Output row of pass 0 for untransformed digits d (their significance reversed).
__device__ __forceinline__ uint64_t reverse_digits(const PassArgs &a, uint64_t d) {
  uint64_t rest = d, rev = 0;
#pragma unroll
  for (int j = kMaxPasses - 1; j >= 0; --j) {
    if (j < (int)a.num_digits) {
      const uint64_t nj = rest & ((1ull << a.digit_log[j]) - 1);
      rest >>= a.digit_log[j];
      rev |= nj << a.digit_shift[j];
    }
  }
  return rev;
}

// ------------------------------------------------------------- swizzle
// Chunk c = 2e + h (16-byte half h of tile element e) is stored at
// c ^ swz(e), swz(e) = XOR of f_b over the set bits b >= 2 of e, with
// f_2..f_10 = 1,7,3,5,7,1,3,4,1 (3-bit columns).  Packed as three 8-entry
// lookup tables (3 bits per entry) for e bits 2-4, 5-7 and 8-10.
constexpr uint32_t swz_lut(uint32_t fa, uint32_t fb, uint32_t fc) {
  uint32_t lut = 0;
  for (uint32_t x = 0; x < 8; ++x) {
    const uint32_t v = ((x & 1) ? fa : 0) ^ ((x & 2) ? fb : 0) ^ ((x & 4) ? fc : 0);
    lut |= v << (3 * x);
  }
  return lut;
}
constexpr uint32_t kSwzLut0 = swz_lut(1, 7, 3);
constexpr uint32_t kSwzLut1 = swz_lut(5, 7, 1);
constexpr uint32_t kSwzLut2 = swz_lut(3, 4, 1);

__device__ __forceinline__ uint32_t swz(uint32_t e) {
  const uint32_t x0 = (e >> 2) & 7, x1 = (e >> 5) & 7, x2 = (e >> 8) & 7;
  return ((kSwzLut0 >> (3 * x0)) ^ (kSwzLut1 >> (3 * x1)) ^ (kSwzLut2 >> (3 * x2))) & 7u;
}

__device__ __forceinline__ void tile_store(uint4 *tile, uint32_t e, const uint32_t a[8]) {
  const uint32_t s = swz(e), c = e << 1;
  tile[c ^ s] = make_uint4(a[0], a[1], a[2], a[3]);
  tile[(c | 1) ^ s] = make_uint4(a[4], a[5], a[6], a[7]);
}

__device__ __forceinline__ void tile_load(uint32_t r[8], const uint4 *tile, uint32_t e) {
  const uint32_t s = swz(e), c = e << 1;
  const uint4 lo = tile[c ^ s];
  const uint4 hi = tile[(c | 1) ^ s];
  r[0] = lo.x; r[1] = lo.y; r[2] = lo.z; r[3] = lo.w;
  r[4] = hi.x; r[5] = hi.y; r[6] = hi.z; r[7] = hi.w;
}

// ----------------------------------------------------------- butterflies

// DIF butterfly: (x, y) -> (x + y, (x - y) * w); w in Montgomery form.
template <class F>
__device__ __forceinline__ void dif_bfly(uint32_t x[8], uint32_t y[8], const uint32_t w[8]) {
  uint32_t d[8];
  sub_mod<F>(d, x, y);
  add_mod<F>(x, x, y);
  mont_mul<F>(y, d, w);
}

// DIF butterfly with twiddle 1.
template <class F>
__device__ __forceinline__ void dif_bfly1(uint32_t x[8], uint32_t y[8]) {
  uint32_t d[8];
  sub_mod<F>(d, x, y);
  add_mod<F>(x, x, y);
  fe_copy(y, d);
}

// Radix-2 round on bit T = LOGS - 1 (first round when LOGS is odd): pairs
// (p, p + S/2) with twiddle omega_S^(p mod S/2).
template <class F, int LOGS, int TL>
__device__ __forceinline__ void round_radix2_top(uint4 *tile, const uint4 *dft_tw) {
  constexpr uint32_t H = 1u << (LOGS - 1);
#pragma unroll 1
  for (int i = 0; i < kElemsPerThread / 2; ++i) {
    const uint32_t g = threadIdx.x + TileCfg<TL>::kThreads * i;   // pair index
    const uint32_t low = g & (H - 1);
    const uint32_t e0 = low | ((g >> (LOGS - 1)) << LOGS);
    uint32_t x[8], y[8];
    tile_load(x, tile, e0);
    tile_load(y, tile, e0 | H);
    if constexpr (LOGS == 1) {
      dif_bfly1<F>(x, y);
    } else {
      uint32_t w[8];
      fe_load_global(w, dft_tw, low);
      dif_bfly<F>(x, y, w);
    }
    tile_store(tile, e0, x);
    tile_store(tile, e0 | H, y);
  }
}

// Radix-4 round on bits [T, T+1], T >= 2 (run-time T).
template <class F, int LOGS, int TL>
__device__ __forceinline__ void round_radix4(uint4 *tile, const uint4 *dft_tw, uint32_t T) {
  const uint32_t step = 1u << T;
  const uint32_t sh = LOGS - 2 - T;
#pragma unroll 1
  for (int i = 0; i < kGroupsPerThread; ++i) {
    const uint32_t g = threadIdx.x + TileCfg<TL>::kThreads * i;   // group index
    const uint32_t low = g & (step - 1);
    const uint32_t e0 = low | ((g >> T) << (T + 2));
    uint32_t x0[8], x1[8], x2[8], x3[8], w[8];
    tile_load(x0, tile, e0);
    tile_load(x1, tile, e0 + step);
    tile_load(x2, tile, e0 + 2 * step);
    tile_load(x3, tile, e0 + 3 * step);
    // stage on bit T+1 (h = 2^(T+1)): twiddle omega_S^((p mod h) * S/(2h))
    fe_load_global(w, dft_tw, low << sh);
    dif_bfly<F>(x0, x2, w);
    fe_load_global(w, dft_tw, (low + step) << sh);
    dif_bfly<F>(x1, x3, w);
    // stage on bit T (h = 2^T)
    fe_load_global(w, dft_tw, low << (sh + 1));
    dif_bfly<F>(x0, x1, w);
    dif_bfly<F>(x2, x3, w);
    tile_store(tile, e0, x0);
    tile_store(tile, e0 + step, x1);
    tile_store(tile, e0 + 2 * step, x2);
    tile_store(tile, e0 + 3 * step, x3);
  }
}

// Last round, bits [0, 1]: stage 1 has twiddles 1 and omega_4, stage 0 only 1.
template <class F, int LOGS, int TL>
__device__ __forceinline__ void round_radix4_last(uint4 *tile, const uint4 *dft_tw) {
  uint32_t w4[8];
  fe_load_global(w4, dft_tw, 1u << (LOGS - 2));   // omega_S^(S/4) = omega_4
#pragma unroll 1
  for (int i = 0; i < kGroupsPerThread; ++i) {
    const uint32_t e0 = (threadIdx.x + TileCfg<TL>::kThreads * i) << 2;
    uint32_t x0[8], x1[8], x2[8], x3[8];
    tile_load(x0, tile, e0);
    tile_load(x1, tile, e0 + 1);
    tile_load(x2, tile, e0 + 2);
    tile_load(x3, tile, e0 + 3);
    dif_bfly1<F>(x0, x2);
    dif_bfly<F>(x1, x3, w4);
    dif_bfly1<F>(x0, x1);
    dif_bfly1<F>(x2, x3);
    tile_store(tile, e0, x0);
    tile_store(tile, e0 + 1, x1);
    tile_store(tile, e0 + 2, x2);
    tile_store(tile, e0 + 3, x3);
  }
}

template <int LOGS>
__device__ __forceinline__ uint32_t bit_reverse_local(uint32_t p) {
  return __brev(p) >> (32 - LOGS);
}

// ------------------------------------------------------------ pass tile

// Process tile `tile` of one pass.  All threads of the CTA call this.
// CG = true reads the pass input with ld.global.cg (L2, coherent), for data
// written earlier in the same kernel launch (the persistent batched kernel);
// otherwise through the read-only path.
template <class F, int LOGS, int MODE, bool CG, int TL>
__device__ __forceinline__ void pass_tile(const PassArgs &a, uint64_t tile, uint4 *smem) {
  static_assert(LOGS <= TL, "sub-transform larger than the tile");
  constexpr uint32_t S = 1u << LOGS;
  constexpr int LOGG = TL - LOGS;
  constexpr uint32_t G = 1u << LOGG;
  constexpr int kThreads = TileCfg<TL>::kThreads;

  const uint64_t d0 = tile << LOGG;
  const uint64_t mp_mask = (1ull << a.log_mp) - 1;

  // ---------------- load phase: element e of the tile = (n, dl), n-major
#pragma unroll 1
  for (int i = 0; i < kElemsPerThread; ++i) {
    const uint32_t e = threadIdx.x + kThreads * i;
    const uint32_t n = e >> LOGG, dl = e & (G - 1);
    const uint64_t d = d0 + dl;
    if (d < a.num_sub) {
      uint32_t v[8];
      if constexpr (MODE == kModeInner) {
        const uint64_t q = d & mp_mask, o = d >> a.log_mp;
        const uint64_t pos = q + ((uint64_t)n << a.log_mp) + (o << (a.log_mp + LOGS));
        if constexpr (CG) fe_load_global_cg(v, a.src, pos);
        else fe_load_global(v, a.src, pos);
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
      tile_store(smem, (dl << LOGS) | n, v);
    }
  }
  __syncthreads();

  // ---------------- DIF rounds, top bit down
  int T = LOGS;
  if constexpr (LOGS & 1) {
    round_radix2_top<F, LOGS, TL>(smem, a.dft_tw);
    __syncthreads();
    T -= 1;
  }
#pragma unroll 1
  for (T -= 2; T >= 2; T -= 2) {
    round_radix4<F, LOGS, TL>(smem, a.dft_tw, (uint32_t)T);
    __syncthreads();
  }
  if constexpr (LOGS >= 2) {
    round_radix4_last<F, LOGS, TL>(smem, a.dft_tw);
    __syncthreads();
  }

  // ---------------- store phase (read the tile at bit-reversed positions)
#pragma unroll 2
  for (int i = 0; i < kElemsPerThread; ++i) {
    const uint32_t e = threadIdx.x + kThreads * i;
    if constexpr (MODE == kModeInner) {
      const uint32_t k = e >> LOGG, dl = e & (G - 1);
      const uint64_t d = d0 + dl;
      if (d < a.num_sub) {
        const uint64_t q = d & mp_mask, o = d >> a.log_mp;
        const uint64_t pos = q + ((uint64_t)k << a.log_mp) + (o << (a.log_mp + LOGS));
        uint32_t v[8];
        tile_load(v, smem, (dl << LOGS) | bit_reverse_local<LOGS>(k));
        fe_store_global(a.dst, pos, v);
      }
    } else {
      const uint32_t dl = e >> LOGS, k = e & (S - 1);
      const uint64_t d = d0 + dl;
      if (d < a.num_sub) {
        const uint64_t rev = reverse_digits(a, d);
        uint32_t v[8];
        tile_load(v, smem, (dl << LOGS) | bit_reverse_local<LOGS>(k));
        fe_store_global(a.dst, (rev << LOGS) | k, v);
      }
    }
  }
}

// ------------------------------------------------------------ pass kernel

template <class F, int LOGS, int MODE, int TL>
__global__ void __launch_bounds__(TileCfg<TL>::kThreads, TileCfg<TL>::kMinBlocks)
    ntt_pass_kernel(const PassArgs a) {
  extern __shared__ uint4 smem[];
  pass_tile<F, LOGS, MODE, false, TL>(a, blockIdx.x, smem);
}

}  // namespace gb300ntt
