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
// index.  The DIF (Gentleman-Sande) radix-2 network over every
// sub-transform of the tile runs two stages at a time (radix-4: each thread
// takes 4 elements, does 4 butterflies, puts them back), the whole CTA in
// lockstep with a barrier between rounds:
//   load round : (S >= 16) the top two stages, on elements read straight
//                from global memory (one 256-bit load each, runs of
//                consecutive elements across a warp) and multiplied by the
//                input multiplier (pass >= 1: omega_M^(n q));
//   rounds     : the stages in between, read from and written back to the
//                tile; the round loop runs at run time so that the hot code
//                is one radix-4 body (small enough for the instruction
//                cache); an odd count starts with a radix-2 round;
//   store round: the last two stages, whose trivial twiddles are known at
//                compile time (1 multiply per 4 elements instead of 4),
//                written straight to global memory at the bit-reversed
//                output index (this undoes the DIF output order).
// Sub-transforms of 2..8 points use a staged variant (load phase, rounds,
// store phase through the tile).
// The tile is XOR-swizzled on 16-byte chunks (swz); the swizzle was chosen
// by simulating the shared-memory wavefronts of every access pattern above,
// for both tile sizes and every sub-transform size 4..2048: none has a bank
// conflict.
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

// At most this many passes per transform (NTT_MAX_PASSES of the C ABI: the
// matrix path splits 2^28 into ten passes of at most 2^3 points).
constexpr int kMaxPasses = 12;

struct PassArgs {
  const uint4 *src;      // input elements (2 x uint4 each)
  uint4 *dst;            // output elements
  const uint4 *mul;      // input multipliers (Montgomery form) or nullptr
  const uint4 *dft_tw;   // omega_S^i, i < S/2 (Montgomery form)
  const uint4 *post;     // output multipliers indexed by output position, or nullptr
                         // (last pass of a coset inverse: s^-n)
  uint64_t num_sub;      // number of sub-transforms in the pass, N / S
  uint32_t log_mp;       // inner: log2 Mp; first: log2(N / S)
  uint32_t num_digits;   // first: P - 1 untransformed digits to reverse
  uint8_t digit_log[kMaxPasses];    // first: log2 S_j of digit j (j = 1..P-1) at index j-1
  uint8_t digit_shift[kMaxPasses];  // first: log2(S_1 ... S_{j-1}) at index j-1
  uint64_t n_vec;        // elements of src, dst and post (debug bounds checks)
  uint64_t n_mul;        // entries of mul (debug bounds checks)
  uint32_t *dbg_err;     // device error word the debug checks report to
};

// Debug builds (NTT_DEBUG): an index is checked against the extent recorded
// for its buffer; out of range, NTT_ERR_BOUNDS goes to the plan's error word
// and the access is skipped (no trap: the context stays usable).  Release
// builds compile the checks away.
#ifdef NTT_DEBUG
__device__ __forceinline__ bool dbg_in(const PassArgs &a, uint64_t idx, uint64_t n) {
  if (idx < n) return true;
  if (a.dbg_err) atomicCAS(a.dbg_err, 0u, 8u /* NTT_ERR_BOUNDS */);
  return false;
}
#else
__device__ __forceinline__ constexpr bool dbg_in(const PassArgs &, uint64_t, uint64_t) { return true; }
#endif

__device__ __forceinline__ void fe_zero(uint32_t r[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) r[j] = 0;
}

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
// f_2..f_10 = 1,7,3,5,7,1,3,5,1 (3-bit columns).  Packed as three 8-entry
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
constexpr uint32_t kSwzLut2 = swz_lut(3, 5, 1);

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

// Radix-2 round on bit T (compile time): pairs (p, p + 2^T) with twiddle
// omega_S^((p mod 2^T) * S / 2^(T+1)).  The staged tile runs it first (T =
// LOGS - 1) when LOGS is odd, the fused tile right after its load round.
template <class F, int LOGS, int TL, int T>
__device__ __forceinline__ void round_radix2(uint4 *tile, const uint4 *dft_tw) {
  constexpr uint32_t H = 1u << T;
#pragma unroll 1
  for (int i = 0; i < kElemsPerThread / 2; ++i) {
    const uint32_t g = threadIdx.x + TileCfg<TL>::kThreads * i;   // pair index
    const uint32_t low = g & (H - 1);
    const uint32_t e0 = low | ((g >> T) << (T + 1));
    uint32_t x[8], y[8];
    tile_load(x, tile, e0);
    tile_load(y, tile, e0 | H);
    if constexpr (LOGS == 1) {
      dif_bfly1<F>(x, y);
    } else {
      uint32_t w[8];
      fe_load_global(w, dft_tw, low << (LOGS - 1 - T));
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
  // (the LOGS = 1 instantiation is never called: its rounds are radix-2)
  const uint32_t sh = static_cast<uint32_t>(LOGS - 2) - T;
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

// x *= post[pos] (Montgomery form multiplier: the result stays standard form).
template <class F>
__device__ __forceinline__ void post_mul(uint32_t x[8], const uint4 *post, uint64_t pos) {
  uint32_t w[8];
  fe_load_global(w, post, pos);
  mont_mul<F>(x, x, w);
}

template <int LOGS>
__device__ __forceinline__ uint32_t bit_reverse_local(uint32_t p) {
  return __brev(p) >> (32 - LOGS);
}

// ------------------------------------------------------------ pass tile

// Staged tile (sub-transforms of 2..8 points): load phase, rounds, store
// phase, each separated by a CTA barrier.
template <class F, int LOGS, int MODE, bool CG, int TL>
__device__ __forceinline__ void pass_tile_staged(const PassArgs &a, uint64_t tile, uint4 *smem) {
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
        if (!dbg_in(a, pos, a.n_vec)) fe_zero(v);
        else if constexpr (CG) fe_load_global_cg(v, a.src, pos);
        else fe_load_global(v, a.src, pos);
        uint32_t w[8];
        const uint64_t wi = ((uint64_t)n << a.log_mp) + q;
        if (dbg_in(a, wi, a.n_mul)) fe_load_global(w, a.mul, wi);
        else fe_zero(w);
        mont_mul<F>(v, v, w);
      } else {
        const uint64_t pos = d + ((uint64_t)n << a.log_mp);
        if (dbg_in(a, pos, a.n_vec)) fe_load_global(v, a.src, pos);
        else fe_zero(v);
        if constexpr (MODE == kModeFirstPre) {
          uint32_t w[8];
          if (dbg_in(a, n, a.n_mul)) fe_load_global(w, a.mul, n);
          else fe_zero(w);
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
    round_radix2<F, LOGS, TL, LOGS - 1>(smem, a.dft_tw);
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
        if (dbg_in(a, pos, a.n_vec)) {
          if (a.post) post_mul<F>(v, a.post, pos);
          fe_store_global(a.dst, pos, v);
        }
      }
    } else {
      const uint32_t dl = e >> LOGS, k = e & (S - 1);
      const uint64_t d = d0 + dl;
      if (d < a.num_sub) {
        const uint64_t rev = reverse_digits(a, d);
        uint32_t v[8];
        tile_load(v, smem, (dl << LOGS) | bit_reverse_local<LOGS>(k));
        const uint64_t pos = (rev << LOGS) | k;
        if (dbg_in(a, pos, a.n_vec)) {
          if (a.post) post_mul<F>(v, a.post, pos);
          fe_store_global(a.dst, pos, v);
        }
      }
    }
  }
}

// ------------------------------------------------ fused tile (S >= 16)
//
// The first radix-4 round (bits LOGS-1, LOGS-2) takes its four elements
// straight from global memory and the last one (bits 1, 0) writes its four
// results straight to global memory.  A warp starts its butterflies as soon
// as its own loads return and stores as soon as it is done, so in a pass that
// fits in one wave of CTAs (2^20 points: 1024 tiles on 1064 slots) the memory
// traffic overlaps the arithmetic of other warps instead of forming a load
// burst before and a store burst after it; two tile round trips through
// shared memory and two barriers go away.

// Global position of element n of sub-transform d (pass input; the in-place
// inner passes write output k of d to the same formula).
template <int LOGS, int MODE>
__device__ __forceinline__ uint64_t elem_pos(const PassArgs &a, uint64_t d, uint32_t n) {
  if constexpr (MODE == kModeInner) {
    const uint64_t q = d & ((1ull << a.log_mp) - 1), o = d >> a.log_mp;
    return q + ((uint64_t)n << a.log_mp) + (o << (a.log_mp + LOGS));
  } else {
    return d + ((uint64_t)n << a.log_mp);
  }
}

// Load round.  Group (dl, low): elements low + j*S/4 (j = 0..3) of
// sub-transform d0 + dl, sub-transforms varying fastest across threads so
// that a warp reads runs of consecutive elements.
template <class F, int LOGS, int MODE, bool CG, int TL>
__device__ __forceinline__ void round_radix4_load(const PassArgs &a, uint64_t d0, uint4 *tile) {
  constexpr int LOGG = TL - LOGS;
  constexpr uint32_t G = 1u << LOGG, Q = 1u << (LOGS - 2);
#pragma unroll 1
  for (int i = 0; i < kGroupsPerThread; ++i) {
    const uint32_t g = threadIdx.x + TileCfg<TL>::kThreads * i;
    const uint32_t dl = g & (G - 1), low = g >> LOGG;
    const uint64_t d = d0 + dl;
    if (d >= a.num_sub) continue;
    uint32_t x[4][8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t pos = elem_pos<LOGS, MODE>(a, d, low + j * Q);
      if (!dbg_in(a, pos, a.n_vec)) fe_zero(x[j]);
      else if constexpr (CG) fe_load_global_cg(x[j], a.src, pos);
      else fe_load_global(x[j], a.src, pos);
    }
    if constexpr (MODE != kModeFirst) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t n = low + j * Q;
        uint32_t w[8];
        const uint64_t wi = MODE == kModeInner ? ((uint64_t)n << a.log_mp) + (d & ((1ull << a.log_mp) - 1)) : n;
        if (dbg_in(a, wi, a.n_mul)) fe_load_global(w, a.mul, wi);
        else fe_zero(w);
        mont_mul<F>(x[j], x[j], w);
      }
    }
    uint32_t w[8];
    // stage on bit LOGS-1: pairs (low, low + S/2), (low + S/4, low + 3S/4)
    fe_load_global(w, a.dft_tw, low);
    dif_bfly<F>(x[0], x[2], w);
    fe_load_global(w, a.dft_tw, low + Q);
    dif_bfly<F>(x[1], x[3], w);
    // stage on bit LOGS-2: twiddle omega_S^(2 low) for both pairs
    fe_load_global(w, a.dft_tw, low << 1);
    dif_bfly<F>(x[0], x[1], w);
    dif_bfly<F>(x[2], x[3], w);
#pragma unroll
    for (int j = 0; j < 4; ++j) tile_store(tile, (dl << LOGS) | (low + j * Q), x[j]);
  }
}

// Store round.  Group t of sub-transform dl holds DIF positions
// p0 = 4 * rev(t) .. p0 + 3 (rev over LOGS-2 bits), whose outputs are
// k = t, t + S/2, t + S/4, t + 3S/4.  Inner passes vary sub-transforms
// fastest across threads (consecutive q), pass 0 varies t (consecutive k):
// either way a warp writes runs of consecutive elements.
template <class F, int LOGS, int MODE, int TL>
__device__ __forceinline__ void round_radix4_store(const PassArgs &a, uint64_t d0, const uint4 *tile) {
  constexpr int LOGG = TL - LOGS;
  constexpr uint32_t G = 1u << LOGG, Q = 1u << (LOGS - 2);
  uint32_t w4[8];
  fe_load_global(w4, a.dft_tw, Q);   // omega_S^(S/4) = omega_4
#pragma unroll 1
  for (int i = 0; i < kGroupsPerThread; ++i) {
    const uint32_t g = threadIdx.x + TileCfg<TL>::kThreads * i;
    uint32_t dl, t;
    if constexpr (MODE == kModeInner) {
      dl = g & (G - 1);
      t = g >> LOGG;
    } else {
      t = g & (Q - 1);
      dl = g >> (LOGS - 2);
    }
    const uint32_t e0 = (dl << LOGS) | (bit_reverse_local<LOGS - 2>(t) << 2);
    uint32_t x0[8], x1[8], x2[8], x3[8];
    tile_load(x0, tile, e0);
    tile_load(x1, tile, e0 + 1);
    tile_load(x2, tile, e0 + 2);
    tile_load(x3, tile, e0 + 3);
    dif_bfly1<F>(x0, x2);
    dif_bfly<F>(x1, x3, w4);
    dif_bfly1<F>(x0, x1);
    dif_bfly1<F>(x2, x3);
    const uint64_t d = d0 + dl;
    if (d < a.num_sub) {
      uint64_t base;
      uint32_t sh;
      if constexpr (MODE == kModeInner) {
        base = elem_pos<LOGS, MODE>(a, d, 0);
        sh = a.log_mp;
      } else {
        base = reverse_digits(a, d) << LOGS;
        sh = 0;
      }
      const uint64_t p0 = base + ((uint64_t)t << sh), p1 = base + ((uint64_t)(t + 2 * Q) << sh);
      const uint64_t p2 = base + ((uint64_t)(t + Q) << sh), p3 = base + ((uint64_t)(t + 3 * Q) << sh);
      // (the four positions are checked through the larger of each pair)
      if (dbg_in(a, p0 > p3 ? p0 : p3, a.n_vec) && dbg_in(a, p1 > p2 ? p1 : p2, a.n_vec)) {
        if (a.post) {   // output multipliers (uniform across the grid)
          post_mul<F>(x0, a.post, p0);
          post_mul<F>(x1, a.post, p1);
          post_mul<F>(x2, a.post, p2);
          post_mul<F>(x3, a.post, p3);
        }
        fe_store_global(a.dst, p0, x0);
        fe_store_global(a.dst, p1, x1);
        fe_store_global(a.dst, p2, x2);
        fe_store_global(a.dst, p3, x3);
      }
    }
  }
}

template <class F, int LOGS, int MODE, bool CG, int TL>
__device__ __forceinline__ void pass_tile_fused(const PassArgs &a, uint64_t tile, uint4 *smem) {
  static_assert(LOGS >= 4 && LOGS <= TL, "fused tile: 16 <= S <= tile");
  const uint64_t d0 = tile << (TL - LOGS);
  round_radix4_load<F, LOGS, MODE, CG, TL>(a, d0, smem);
  __syncthreads();
  // stages LOGS-3 .. 2 in between: a radix-2 round first if their count is odd
  constexpr int kMid = LOGS - 4;
  if constexpr (kMid & 1) {
    round_radix2<F, LOGS, TL, LOGS - 3>(smem, a.dft_tw);
    __syncthreads();
  }
#pragma unroll 1
  for (int T = (kMid & 1) ? LOGS - 5 : LOGS - 4; T >= 2; T -= 2) {
    round_radix4<F, LOGS, TL>(smem, a.dft_tw, (uint32_t)T);
    __syncthreads();
  }
  round_radix4_store<F, LOGS, MODE, TL>(a, d0, smem);
}

// Process tile `tile` of one pass.  All threads of the CTA call this; the
// caller separates two tiles on the same shared memory with a barrier.
// CG = true reads the pass input with ld.global.cg (L2, coherent), for data
// written earlier in the same kernel launch (the persistent batched kernel);
// otherwise through the read-only path.
//
// FUSED selects the fused tile (sub-transforms of 16 points and more) or the
// staged one.  Measured on GB300: the fused tile wins where a pass is one
// wave of CTAs (all CTAs in the same phase: 2^20 pass 0 -6%) and in the
// persistent batched kernel; the staged tile wins in many-wave passes
// (2^24: inner passes 1.42 vs 1.61 ms), where CTAs in different phases
// share the SM and the fused tile's larger hot code misses the
// instruction cache (no_instruction becomes the top stall).
template <class F, int LOGS, int MODE, bool CG, int TL, bool FUSED>
__device__ __forceinline__ void pass_tile(const PassArgs &a, uint64_t tile, uint4 *smem) {
  if constexpr (FUSED && LOGS >= 4) pass_tile_fused<F, LOGS, MODE, CG, TL>(a, tile, smem);
  else pass_tile_staged<F, LOGS, MODE, CG, TL>(a, tile, smem);
}

// ------------------------------------------------------------ pass kernel

// Programmatic dependent launch (the passes are launched with it): the next
// launch on the stream may start as soon as every CTA of this one has begun
// (its CTAs take SM slots as ours retire), and each thread waits here until
// the previous launch has completed and its memory is visible before it
// touches the vector.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger_and_wait() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <class F, int LOGS, int MODE, int TL, bool FUSED>
__global__ void __launch_bounds__(TileCfg<TL>::kThreads, TileCfg<TL>::kMinBlocks)
    ntt_pass_kernel(const PassArgs a) {
  extern __shared__ uint4 smem[];
  pdl_trigger_and_wait();
  pass_tile<F, LOGS, MODE, false, TL, FUSED>(a, blockIdx.x, smem);
}

}  // namespace gb300ntt
