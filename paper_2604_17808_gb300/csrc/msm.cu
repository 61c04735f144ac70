// msm.cu -- multi-scalar multiplication on BN254 G1 and BLS12-381 G1 by the
// paper's Layout-Stationary Pippenger (MORPH, Algorithm 2), GB300 form.
//
//   MSM = sum_{n<N} S_n P_n, S_n < r (254 or 255 bits), P_n affine points.
//
// Every kernel that touches points is a template over the curve (its base
// field's traits and its scalar field); the sort and scan kernels are shared.
// Each scalar is cut into K = ceil((S^BL + 1) / c) signed c-bit digits
// d_k in [-(2^(c-1) - 1), 2^(c-1)] (sum_k d_k 2^(k c) = S_n); window k keeps
// 2^(c-1) buckets, bucket j collecting the points whose digit has magnitude
// j + 1 (negated when the digit is negative).  The four phases of
// Algorithm 2 map to kernels:
//
//   Bucketize    msm_count_kernel      bucket sizes (one counter per bucket,
//                                      atomics in L2; zero digits skipped)
//                scan_*_kernel         exclusive scan -> bucket offsets
//                msm_scatter_kernel    point index (and digit sign) into the
//                                      next slot of its bucket: the argsort of
//                                      the digits as a counting sort
//   BA           msm_accumulate_kernel the bucket-sorted entries cut into
//                                      segments of exactly S; one thread adds
//                                      its S points (XYZZ += affine), writing a
//                                      bucket that lies inside its segment
//                                      straight to the bucket array and the
//                                      pieces of the (at most two) buckets
//                                      that cross its ends to piece slots;
//                msm_combine_kernel    a pairwise tree over the pieces of each
//                                      crossing bucket.  Every thread does the
//                                      same number of additions whatever the
//                                      bucket sizes (a skewed or constant
//                                      scalar set stays parallel and balanced)
//   BR           msm_reduce_level_kernel  the tree of Algorithm 2, one launch
//                                      per level, all windows at once:
//                                      W_b = W_2b + W_2b+1 + B_2b+1,
//                                      B_b = 2 (B_2b + B_2b+1); the leaves
//                                      start at W_j = B_j, so the root holds
//                                      sum_j (j + 1) B_j
//   WM           msm_merge_kernel      Horner over the windows, top one first
//                                      (MSM = 2^c MSM + W_k), then the affine
//                                      standard-form result.
//
// The paper streams the sorted points straight into bucket accumulation on
// the TPU; here the sort moves 4-byte point indices and the accumulation
// gathers the 64- or 96-byte points by index (a point is read once per
// window from HBM; the accumulation is bound by the integer multiply pipe,
// not by these reads).  Points are converted to Montgomery form once per
// call (msm_prepare_kernel), which also checks that every point lies on the
// curve.
//
// Two variants reuse the same kernels: a window range [kb, ke) (the count
// and scatter kernels skip the other windows' digits, the tree and merge run
// over the range only) gives one rank's part of a window-sharded MSM; and
// precomputed bases (msm_bases_kernel stores every point's window copies
// 2^(k c) P once) put all windows' digits into one bucket set ("flat" count
// and scatter), so one tree replaces K and the window merge disappears.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

#include "../../include/msm_gb300.h"
#include "ec_xyzz.cuh"
#include "nvtx_range.h"

namespace gb300ntt {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;
constexpr int kEcThreads = 128;
constexpr uint32_t kSignBit = 0x80000000u;

// Curves: base-field traits, the scalar modulus r (for the input check),
// the curve constant b, and the CTAs of 128 threads per SM that the register
// budget of the point kernels allows.  The scalar bit length and the
// generator are host-side (curve_scalar_bits, curve_generator).
struct CurveBn254 {
  using T = FqBn254;
  static constexpr int kMinBlocks = 4;
  static constexpr int kTreeMinBlocks = 4;  // reduction-tree and combine kernels
  static constexpr uint32_t kB = 3;
  __device__ static bool scalar_ok(const uint32_t s[8]) {
    const uint32_t r[8] = {0xf0000001u, 0x43e1f593u, 0x79b97091u, 0x2833e848u,
                           0x8181585du, 0xb85045b6u, 0xe131a029u, 0x30644e72u};
#pragma unroll
    for (int j = 7; j >= 0; --j)
      if (s[j] != r[j]) return s[j] < r[j];
    return false;
  }
};

struct CurveBls381 {
  using T = FqBls381;
  static constexpr int kMinBlocks = 3;
  static constexpr int kTreeMinBlocks = 2;  // two XYZZ points live: 255 registers, no spill
  static constexpr uint32_t kB = 4;
  __device__ static bool scalar_ok(const uint32_t s[8]) {
    const uint32_t r[8] = {0x00000001u, 0xffffffffu, 0xfffe5bfeu, 0x53bda402u,
                           0x09a1d805u, 0x3339d808u, 0x299d7d48u, 0x73eda753u};
#pragma unroll
    for (int j = 7; j >= 0; --j)
      if (s[j] != r[j]) return s[j] < r[j];
    return false;
  }
};

template <class T>
struct EcConst {
  uint32_t one[T::L];  // 2^(32 L) mod q (Montgomery 1)
  uint32_t r2[T::L];   // 2^(64 L) mod q (to Montgomery form)
  uint32_t b3[T::L];   // b 2^(32 L) mod q (curve constant, Montgomery)
  uint32_t gx[T::L];   // generator, standard form
  uint32_t gy[T::L];
};

struct MsmTotals {
  uint32_t entries;   // points placed in buckets (digit != 0)
  uint32_t max_span;  // most segment boundaries one bucket crosses
  uint32_t pad;
  uint32_t err;       // MSM_ERR_* bits
};

// ----------------------------------------------------------- small helpers

template <class T>
__device__ __forceinline__ void load_point_xyzz(Xyzz<T> &p, const uint4 *base, uint64_t i) {
  T::load(p.X, base, 4 * i + 0);
  T::load(p.Y, base, 4 * i + 1);
  T::load(p.ZZ, base, 4 * i + 2);
  T::load(p.ZZZ, base, 4 * i + 3);
}

template <class T>
__device__ __forceinline__ void store_point_xyzz(uint4 *base, uint64_t i, const Xyzz<T> &p) {
  T::store(base, 4 * i + 0, p.X);
  T::store(base, 4 * i + 1, p.Y);
  T::store(base, 4 * i + 2, p.ZZ);
  T::store(base, 4 * i + 3, p.ZZZ);
}

// Raw c-bit digit of window k of the scalar s (8 little-endian words); c <= 22.
__device__ __forceinline__ uint32_t raw_digit(const uint32_t s[8], uint32_t k, uint32_t c) {
  const uint32_t bit = k * c, w = bit >> 5, sh = bit & 31u;
  if (w >= 8) return 0u;
  uint64_t v = s[w];
  if (w + 1 < 8) v |= (uint64_t)s[w + 1] << 32;
  return (uint32_t)(v >> sh) & ((1u << c) - 1u);
}

// Next signed digit: v = raw + carry in [0, 2^c]; v > 2^(c-1) becomes
// v - 2^c (negative) with a carry into the next window.  Returns the
// magnitude (0 for a zero digit); neg is the sign.
__device__ __forceinline__ uint32_t signed_digit(const uint32_t s[8], uint32_t k, uint32_t c, uint32_t &carry,
                                                 bool &neg) {
  const uint32_t v = raw_digit(s, k, c) + carry;
  neg = v > (1u << (c - 1));
  carry = neg ? 1u : 0u;
  return neg ? (1u << c) - v : v;
}

// ---------------------------------------------------------------- kernels

// Points to Montgomery form (x R, y R); (0, 0) stays the point at infinity.
// Flags points that are not canonical or not on y^2 = x^3 + b (and treats
// them as O so that the arithmetic below never sees a value >= q).
template <class C>
__global__ void __launch_bounds__(kEcThreads) msm_prepare_kernel(const uint4 *pts, uint64_t n,
                                                                 EcConst<typename C::T> k, uint4 *pts_m,
                                                                 MsmTotals *tot) {
  using T = typename C::T;
  constexpr int L = T::L;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x[L], y[L];
    T::load(x, pts, 2 * i);
    T::load(y, pts, 2 * i + 1);
    if (fv_is_zero<L>(x) && fv_is_zero<L>(y)) {
      T::store(pts_m, 2 * i, x);
      T::store(pts_m, 2 * i + 1, y);
      continue;
    }
    bool ok = T::canonical(x) && T::canonical(y);
    if (ok) {
      T::mul(x, x, k.r2);
      T::mul(y, y, k.r2);
      uint32_t l[L], r[L];
      T::mul(l, y, y);
      T::mul(r, x, x);
      T::mul(r, r, x);
      T::add(r, r, k.b3);
      ok = fv_equal<L>(l, r);
    }
    if (!ok) {
      atomicOr(&tot->err, (uint32_t)MSM_ERR_POINT);
      fv_zero<L>(x);
      fv_zero<L>(y);
    }
    T::store(pts_m, 2 * i, x);
    T::store(pts_m, 2 * i + 1, y);
  }
}

// Bucketize, pass 1: one counter per (window, digit magnitude), windows
// [kb, ke) (the digits below kb are still recoded for their carries).
// With precomputed bases (flat = true) every window uses the same 2^(c-1)
// buckets: the point of digit k of scalar i is the copy 2^(k c) P_i.
template <class C>
__global__ void __launch_bounds__(256) msm_count_kernel(const uint4 *__restrict__ scalars, uint64_t n, uint32_t c,
                                                        uint32_t kb, uint32_t ke, bool flat,
                                                        uint32_t *__restrict__ counts, MsmTotals *tot) {
  const uint32_t lb = flat ? 0u : c - 1;  // window stride of the bucket index (log2)
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t s[8];
    fe_load_global(s, scalars, i);
    if (!C::scalar_ok(s)) atomicOr(&tot->err, (uint32_t)MSM_ERR_SCALAR);
    uint32_t carry = 0;
    for (uint32_t k = 0; k < ke; ++k) {
      bool neg;
      const uint32_t m = signed_digit(s, k, c, carry, neg);
      if (m && k >= kb) atomicAdd(&counts[(flat ? 0ull : ((uint64_t)k << lb)) + m - 1], 1u);
    }
  }
}

// Inclusive scan across a warp.
__device__ __forceinline__ uint32_t warp_scan(uint32_t v) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (uint32_t)o) v += a;
  }
  return v;
}

// Exclusive scan of v over the CTA (blockDim.x = kScanThreads); *total gets
// the CTA's sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total) {
  __shared__ uint32_t warp_sums[kScanThreads / 32];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t inc = warp_scan(v);
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0u;
    const uint32_t wi = warp_scan(w);
    if (lane < kScanThreads / 32) warp_sums[lane] = wi - w;
    if (lane == kScanThreads / 32 - 1) *total = wi;
  }
  __syncthreads();
  const uint32_t base = warp_sums[warp];
  __syncthreads();
  return base + inc - v;
}

// Scan pass 1: per-tile sums of the bucket sizes.
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t *counts, uint64_t nb,
                                                                   uint32_t *tile_sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanPer;
  uint32_t v = 0;
#pragma unroll
  for (int j = 0; j < kScanPer; ++j)
    if (base + j < nb) v += counts[base + j];
  __shared__ uint32_t total;
  block_excl_scan(v, &total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Scan pass 2 (one CTA): exclusive scan of the tile sums in place; the total
// goes to tot->entries and offsets[nb].
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(uint32_t *tile_sums, uint32_t num_tiles,
                                                                  uint64_t nb, uint32_t *offsets, MsmTotals *tot) {
  __shared__ uint32_t chunk_total;
  uint32_t carry = 0;
  for (uint32_t b0 = 0; b0 < num_tiles; b0 += kScanThreads) {
    const uint32_t i = b0 + threadIdx.x;
    const uint32_t v = i < num_tiles ? tile_sums[i] : 0u;
    const uint32_t ex = block_excl_scan(v, &chunk_total);
    if (i < num_tiles) tile_sums[i] = carry + ex;
    __syncthreads();
    carry += chunk_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    tot->entries = carry;
    offsets[nb] = carry;
  }
}

// Scan pass 3: bucket offsets, also copied to the scatter cursors.
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t *counts, uint64_t nb,
                                                                  const uint32_t *tile_sums, uint32_t *offsets,
                                                                  uint32_t *cursor) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanPer;
  uint32_t cnt[kScanPer];
  uint32_t v = 0;
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    cnt[j] = base + j < nb ? counts[base + j] : 0u;
    v += cnt[j];
  }
  __shared__ uint32_t total;
  uint32_t run = block_excl_scan(v, &total) + tile_sums[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    if (base + j < nb) {
      offsets[base + j] = run;
      cursor[base + j] = run;
    }
    run += cnt[j];
  }
}

// Bucketize, pass 2: each point index (sign in bit 31) into the next free
// slot of its bucket, windows [kb, ke); the atomics of eight windows are in
// flight at once.
__global__ void __launch_bounds__(256) msm_scatter_kernel(const uint4 *__restrict__ scalars, uint64_t n, uint32_t c,
                                                          uint32_t kb, uint32_t ke, uint32_t flat_stride,
                                                          uint32_t *__restrict__ cursor,
                                                          uint32_t *__restrict__ sorted) {
  // flat_stride > 0: precomputed bases, one bucket set, point copy k at k * flat_stride
  const uint32_t lb = c - 1;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t s[8];
    fe_load_global(s, scalars, i);
    uint32_t carry = 0;
    for (uint32_t k0 = 0; k0 < ke; k0 += 8) {
      uint32_t pos[8], val[8];
#pragma unroll
      for (uint32_t j = 0; j < 8; ++j) {
        const uint32_t k = k0 + j;
        bool neg = false;
        const uint32_t m = k < ke ? signed_digit(s, k, c, carry, neg) : 0u;
        const uint64_t bucket = (flat_stride ? 0ull : ((uint64_t)k << lb)) + m - 1;
        pos[j] = (m && k >= kb) ? atomicAdd(&cursor[bucket], 1u) : 0xffffffffu;
        val[j] = ((uint32_t)i + k * flat_stride) | (neg ? kSignBit : 0u);
      }
#pragma unroll
      for (uint32_t j = 0; j < 8; ++j)
        if (pos[j] != 0xffffffffu) sorted[pos[j]] = val[j];
    }
  }
}

// Largest b with offsets[b] <= e (offsets non-decreasing, offsets[0] = 0,
// e < offsets[nb]): the bucket holding sorted entry e.
__device__ __forceinline__ uint32_t bucket_of_entry(const uint32_t *offsets, uint64_t nb, uint32_t e) {
  uint64_t lo = 0, hi = nb;  // offsets[lo] <= e < offsets[hi]
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (__ldg(offsets + mid) <= e) lo = mid;
    else hi = mid;
  }
  return (uint32_t)lo;
}

// Where the partial sum of bucket b over segment t goes: a bucket inside the
// segment is complete (bucket array); a bucket that started in an earlier
// segment leaves its piece in slot 2t; one that starts here and continues
// leaves its head piece in slot 2t + 1.
template <class T>
__device__ __forceinline__ void emit_piece(const Xyzz<T> &acc, uint32_t b, uint32_t t, bool started_before,
                                           bool continues, uint4 *bucket_sum, uint4 *pieces) {
  if (!started_before && !continues) store_point_xyzz(bucket_sum, b, acc);
  else if (started_before) store_point_xyzz(pieces, 2 * (uint64_t)t, acc);
  else store_point_xyzz(pieces, 2 * (uint64_t)t + 1, acc);
}

// BA: segment t adds the points of sorted entries [t S, t S + S).
template <class C>
__global__ void __launch_bounds__(kEcThreads, C::kMinBlocks)
    msm_accumulate_kernel(const uint4 *__restrict__ pts_m, const uint32_t *__restrict__ sorted,
                          const uint32_t *__restrict__ offsets, uint64_t nb, uint32_t S, EcConst<typename C::T> k,
                          MsmTotals *tot, uint2 *__restrict__ seg_ends, uint4 *bucket_sum, uint4 *pieces) {
  using T = typename C::T;
  constexpr int L = T::L;
  const uint32_t n_entries = tot->entries;
  const uint32_t num_segs = (n_entries + S - 1) / S;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < num_segs; t += gridDim.x * blockDim.x) {
    const uint32_t e0 = t * S, e1 = min(e0 + S, n_entries);
    uint32_t b = bucket_of_entry(offsets, nb, e0);
    const uint32_t first = b;
    uint32_t end_b = __ldg(offsets + b + 1);
    bool started_before = __ldg(offsets + b) < e0;
    Xyzz<T> acc;
    xyzz_set_inf(acc);
    for (uint32_t e = e0; e < e1; ++e) {
      if (e == end_b) {  // bucket b ends inside the segment
        emit_piece(acc, b, t, started_before, false, bucket_sum, pieces);
        xyzz_set_inf(acc);
        do {
          ++b;
          end_b = __ldg(offsets + b + 1);
        } while (end_b == e);  // skip empty buckets
        started_before = false;
      }
      const uint32_t v = __ldg(sorted + e);
      const uint64_t idx = v & ~kSignBit;
      uint32_t x[L], y[L];
      T::load(x, pts_m, 2 * idx);
      T::load(y, pts_m, 2 * idx + 1);
      if (fv_is_zero<L>(x) && fv_is_zero<L>(y)) continue;  // point at infinity
      if (v & kSignBit) {
        uint32_t zero[L];
        fv_zero<L>(zero);
        T::sub(y, zero, y);
      }
      xyzz_madd<T>(acc, x, y, k.one);
    }
    const bool continues = end_b > e1;
    emit_piece(acc, b, t, started_before, continues, bucket_sum, pieces);
    if (continues && !started_before) {
      const uint32_t span = (end_b - 1) / S - t;  // segments after t that hold bucket b
      atomicMax(&tot->max_span, span);
    }
    seg_ends[t] = make_uint2(first, b);
  }
}

// BA, combine round r.  The pieces of a bucket that crosses segments
// t0 < t0+1 < ... < t1 form V[0] = head slot 2 t0 + 1, V[i] = slot 2 (t0 + i);
// round r adds V[i + 2^r] into V[i] for i a multiple of 2^(r+1), so after
// ceil(log2(t1 - t0 + 1)) rounds the bucket's sum is in V[0].
template <class C>
__global__ void __launch_bounds__(kEcThreads, C::kTreeMinBlocks)
    msm_combine_kernel(const uint32_t *__restrict__ offsets, const uint2 *__restrict__ seg_ends, uint32_t S,
                       const MsmTotals *tot, uint32_t r, uint4 *pieces) {
  using T = typename C::T;
  const uint32_t step = 1u << r;
  if (step > tot->max_span) return;
  const uint32_t n_entries = tot->entries;
  const uint32_t num_segs = (n_entries + S - 1) / S;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < num_segs; t += gridDim.x * blockDim.x) {
    const uint2 ends = seg_ends[t];
    const uint32_t e0 = t * S, e1 = min(e0 + S, n_entries);
    // role of V[0]: the last bucket starts in this segment and continues
    {
      const uint32_t b = ends.y;
      const uint32_t ob = __ldg(offsets + b), ob1 = __ldg(offsets + b + 1);
      if (ob >= e0 && ob1 > e1) {
        const uint32_t span = (ob1 - 1) / S - t;
        if (step <= span) {
          Xyzz<T> a, q;
          load_point_xyzz(a, pieces, 2 * (uint64_t)t + 1);
          load_point_xyzz(q, pieces, 2 * (uint64_t)(t + step));
          xyzz_add<T, true>(a, q);
          store_point_xyzz(pieces, 2 * (uint64_t)t + 1, a);
        }
      }
    }
    // role of V[i], i >= 1: the first bucket started in an earlier segment
    {
      const uint32_t b = ends.x;
      const uint32_t ob = __ldg(offsets + b), ob1 = __ldg(offsets + b + 1);
      if (ob < e0) {
        const uint32_t t0 = ob / S, span = (ob1 - 1) / S - t0, i = t - t0;
        if ((i & (2 * step - 1)) == 0 && i + step <= span) {
          Xyzz<T> a, q;
          load_point_xyzz(a, pieces, 2 * (uint64_t)t);
          load_point_xyzz(q, pieces, 2 * (uint64_t)(t + step));
          xyzz_add<T, true>(a, q);
          store_point_xyzz(pieces, 2 * (uint64_t)t, a);
        }
      }
    }
  }
}

// Bucket b's sum after accumulation: O, the complete sum, or the head piece.
template <class T>
__device__ __forceinline__ void load_bucket(Xyzz<T> &p, const uint4 *bucket_sum, const uint4 *pieces,
                                            const uint32_t *offsets, uint32_t S, uint64_t b) {
  const uint32_t ob = offsets[b], ob1 = offsets[b + 1];
  if (ob1 == ob) xyzz_set_inf(p);
  else if (ob / S == (ob1 - 1) / S) load_point_xyzz(p, bucket_sum, b);
  else load_point_xyzz(p, pieces, 2 * (uint64_t)(ob / S) + 1);
}

// BR, level s of the tree (all windows): node (k, b), b < 2^s, from its two
// children.  Window k has 2^(c-1) leaves (the buckets); level s of its tree
// is stored at heap index 2^s + b.  At the level above the leaves the
// children's W are the leaves themselves (W_j = B_j).
template <class C>
__global__ void __launch_bounds__(kEcThreads, C::kTreeMinBlocks)
    msm_reduce_level_kernel(uint32_t s, uint32_t lb, uint32_t kb, uint32_t nk, const uint4 *bucket_sum,
                            const uint4 *pieces, const uint32_t *offsets, uint32_t S, uint4 *heap_w,
                            uint4 *heap_b) {
  using T = typename C::T;
  const uint64_t per = 1ull << s, total = per * nk;  // windows kb .. kb + nk - 1
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = kb + (t >> s), b = t & (per - 1);
    const uint64_t heap0 = k << lb;  // window k's heap
    const uint64_t node = heap0 + per + b;
    Xyzz<T> a, br;
    if (s + 1 == lb) {
      const uint64_t leaf = heap0 + 2 * b;
      load_bucket(a, bucket_sum, pieces, offsets, S, leaf);
      load_bucket(br, bucket_sum, pieces, offsets, S, leaf + 1);
      xyzz_add<T, true>(a, br);                     // B_L + B_R
      Xyzz<T> w = a;
      xyzz_add<T, true>(w, br);                     // W = W_L + W_R + B_R with W_j = B_j
      store_point_xyzz(heap_w, node, w);
      if (s == 0) continue;                // the root's B is not needed
    } else {
      const uint64_t child = heap0 + 2 * per + 2 * b;
      load_point_xyzz(a, heap_w, child);
      load_point_xyzz(br, heap_w, child + 1);
      xyzz_add<T, true>(a, br);
      load_point_xyzz(br, heap_b, child + 1);
      xyzz_add<T, true>(a, br);
      store_point_xyzz(heap_w, node, a);   // W = W_L + W_R + B_R
      if (s == 0) continue;
      load_point_xyzz(a, heap_b, child);
      xyzz_add<T, true>(a, br);                     // B_L + B_R
    }
    xyzz_dbl<T, true>(a, a);
    store_point_xyzz(heap_b, node, a);     // B = 2 (B_L + B_R)
  }
}

// WM: sum_{kb <= k < ke} 2^(k c) W_k by Horner (then kb c doublings), in
// affine standard form; the whole MSM for [0, K).  With one bucket per
// window (c = 1) W_k is that bucket.
template <class C>
__global__ void msm_merge_kernel(uint32_t c, uint32_t kb, uint32_t ke, const uint4 *heap_w, const uint4 *bucket_sum,
                                 const uint4 *pieces, const uint32_t *offsets, uint32_t S,
                                 EcConst<typename C::T> kc, uint4 *result) {
  using T = typename C::T;
  constexpr int L = T::L;
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const uint32_t lb = c - 1;
  Xyzz<T> acc;
  xyzz_set_inf(acc);
  for (int k = (int)ke - 1; k >= (int)kb; --k) {
    if (!xyzz_is_inf(acc))
      for (uint32_t j = 0; j < c; ++j) xyzz_dbl(acc, acc);
    Xyzz<T> w;
    if (lb == 0) load_bucket(w, bucket_sum, pieces, offsets, S, (uint64_t)k);
    else load_point_xyzz(w, heap_w, ((uint64_t)k << lb) + 1);
    xyzz_add(acc, w);
  }
  if (!xyzz_is_inf(acc))
    for (uint32_t j = 0; j < c * kb; ++j) xyzz_dbl(acc, acc);
  uint32_t x[L], y[L];
  xyzz_to_affine_std<T>(x, y, acc, kc.one);
  T::store(result, 0, x);
  T::store(result, 1, y);
}

// Precomputed bases (fixed points reused across calls): for every point P_i
// the window copies 2^(k c) P_i, k < K, in affine Montgomery form at index
// k * stride + i; then all windows share one bucket set, and the
// per-window reduction trees and the window merge collapse into one window.
// The copies are normalised with one inversion per point (Montgomery's
// simultaneous inversion over its K copies).  Neither group has a point of
// order two, so no copy of a point other than O is O.  Invalid points are
// flagged and become O, as in msm_prepare_kernel.
constexpr uint32_t kMaxBaseWindows = 32;

template <class C>
__global__ void __launch_bounds__(kEcThreads) msm_bases_kernel(const uint4 *pts, uint64_t n, uint32_t c, uint32_t K,
                                                               uint64_t stride, EcConst<typename C::T> kc,
                                                               uint4 *bases, MsmTotals *tot) {
  using T = typename C::T;
  constexpr int L = T::L;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x[L], y[L];
    T::load(x, pts, 2 * i);
    T::load(y, pts, 2 * i + 1);
    bool inf = fv_is_zero<L>(x) && fv_is_zero<L>(y);
    if (!inf) {
      bool ok = T::canonical(x) && T::canonical(y);
      if (ok) {
        T::mul(x, x, kc.r2);
        T::mul(y, y, kc.r2);
        uint32_t l[L], r[L];
        T::mul(l, y, y);
        T::mul(r, x, x);
        T::mul(r, r, x);
        T::add(r, r, kc.b3);
        ok = fv_equal<L>(l, r);
      }
      if (!ok) {
        atomicOr(&tot->err, (uint32_t)MSM_ERR_POINT);
        inf = true;
      }
    }
    if (inf) {
      fv_zero<L>(x);
      for (uint32_t k = 0; k < K; ++k) {
        T::store(bases, 2 * (k * stride + i), x);
        T::store(bases, 2 * (k * stride + i) + 1, x);
      }
      continue;
    }
    Xyzz<T> q[kMaxBaseWindows];
    uint32_t pre[kMaxBaseWindows][L];
    fv_copy<L>(q[0].X, x);
    fv_copy<L>(q[0].Y, y);
    fv_copy<L>(q[0].ZZ, kc.one);
    fv_copy<L>(q[0].ZZZ, kc.one);
    fv_copy<L>(pre[0], kc.one);  // ZZ ZZZ of the affine copy
    for (uint32_t k = 1; k < K; ++k) {
      q[k] = q[k - 1];
      for (uint32_t j = 0; j < c; ++j) xyzz_dbl<T>(q[k], q[k]);
      uint32_t z[L];
      T::mul(z, q[k].ZZ, q[k].ZZZ);
      T::mul(pre[k], pre[k - 1], z);  // prefix products of z_k = ZZ_k ZZZ_k
    }
    uint32_t inv[L];
    f_inverse<T>(inv, pre[K - 1], kc.one);  // (z_0 ... z_{K-1})^-1
    for (int k = (int)K - 1; k >= 0; --k) {
      uint32_t ik[L], z[L], zi[L], ax[L], ay[L];
      if (k > 0) {
        T::mul(ik, inv, pre[k - 1]);        // z_k^-1
        T::mul(z, q[k].ZZ, q[k].ZZZ);
        T::mul(inv, inv, z);                // (z_0 ... z_{k-1})^-1
      } else {
        fv_copy<L>(ik, inv);
      }
      T::mul(zi, ik, q[k].ZZZ);             // ZZ^-1
      T::mul(ax, q[k].X, zi);
      T::mul(zi, ik, q[k].ZZ);              // ZZZ^-1
      T::mul(ay, q[k].Y, zi);
      T::store(bases, 2 * (k * stride + i), ax);
      T::store(bases, 2 * (k * stride + i) + 1, ay);
    }
  }
}

// ------------------------------------------------- fixed-base generation

// Comb table T[w][d] = d 2^(8 w) G (w < 32, d < 256), XYZZ, one thread per w.
template <class C>
__global__ void fixed_base_table_kernel(EcConst<typename C::T> kc, uint4 *table_xyzz) {
  using T = typename C::T;
  constexpr int L = T::L;
  const uint32_t w = threadIdx.x;
  if (blockIdx.x != 0 || w >= 32) return;
  Xyzz<T> base;
  T::mul(base.X, kc.gx, kc.r2);  // G in Montgomery form
  T::mul(base.Y, kc.gy, kc.r2);
  fv_copy<L>(base.ZZ, kc.one);
  fv_copy<L>(base.ZZZ, kc.one);
  for (uint32_t j = 0; j < 8 * w; ++j) xyzz_dbl<T>(base, base);
  Xyzz<T> acc;
  xyzz_set_inf(acc);
  store_point_xyzz(table_xyzz, 256 * w, acc);
  for (uint32_t d = 1; d < 256; ++d) {
    xyzz_add<T>(acc, base);
    store_point_xyzz(table_xyzz, 256 * w + d, acc);
  }
}

// Table entries to affine Montgomery form ((0, 0) for O).
template <class C>
__global__ void __launch_bounds__(kEcThreads) fixed_base_affine_kernel(EcConst<typename C::T> kc,
                                                                       const uint4 *table_xyzz, uint4 *table_aff) {
  using T = typename C::T;
  constexpr int L = T::L;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 32 * 256) return;
  Xyzz<T> p;
  load_point_xyzz(p, table_xyzz, i);
  uint32_t x[L], y[L];
  if (xyzz_is_inf(p)) {
    fv_zero<L>(x);
    fv_zero<L>(y);
  } else {
    uint32_t t[L], inv[L], zi[L];
    T::mul(t, p.ZZ, p.ZZZ);
    f_inverse<T>(inv, t, kc.one);
    T::mul(zi, inv, p.ZZZ);
    T::mul(x, p.X, zi);
    T::mul(zi, inv, p.ZZ);
    T::mul(y, p.Y, zi);
  }
  T::store(table_aff, 2 * i, x);
  T::store(table_aff, 2 * i + 1, y);
}

// P_n = t_n G = sum_w T[w][byte w of t_n], affine standard form.
template <class C>
__global__ void __launch_bounds__(kEcThreads) fixed_base_points_kernel(EcConst<typename C::T> kc,
                                                                       const uint4 *table_aff, const uint4 *ts,
                                                                       uint64_t n, uint4 *out) {
  using T = typename C::T;
  constexpr int L = T::L;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t t[8];
    fe_load_global(t, ts, i);
    Xyzz<T> acc;
    xyzz_set_inf(acc);
    for (uint32_t w = 0; w < 32; ++w) {
      const uint32_t d = (t[w >> 2] >> (8 * (w & 3))) & 0xffu;
      if (!d) continue;
      uint32_t x[L], y[L];
      T::load(x, table_aff, 2 * (256 * w + d));
      T::load(y, table_aff, 2 * (256 * w + d) + 1);
      xyzz_madd<T>(acc, x, y, kc.one);
    }
    uint32_t x[L], y[L];
    xyzz_to_affine_std<T>(x, y, acc, kc.one);
    T::store(out, 2 * i, x);
    T::store(out, 2 * i + 1, y);
  }
}

// ------------------------------------------------------------------ host

// x = 2 x mod q on L-limb numbers (x < q < 2^(32 L - 1)).
void host_double_mod(uint32_t *x, const uint32_t *q, int L) {
  uint32_t carry = 0;
  for (int j = 0; j < L; ++j) {
    const uint32_t nc = x[j] >> 31;
    x[j] = (x[j] << 1) | carry;
    carry = nc;
  }
  bool ge = true;
  for (int j = L - 1; j >= 0; --j)
    if (x[j] != q[j]) {
      ge = x[j] > q[j];
      break;
    }
  if (ge) {
    int64_t br = 0;
    for (int j = 0; j < L; ++j) {
      const int64_t v = (int64_t)x[j] - q[j] + br;
      x[j] = (uint32_t)v;
      br = v < 0 ? -1 : 0;
    }
  }
}

// x = x + y mod q (x, y < q)
void host_add_mod(uint32_t *x, const uint32_t *y, const uint32_t *q, int L) {
  uint64_t c = 0;
  for (int j = 0; j < L; ++j) {
    c += (uint64_t)x[j] + y[j];
    x[j] = (uint32_t)c;
    c >>= 32;
  }
  bool ge = true;
  for (int j = L - 1; j >= 0; --j)
    if (x[j] != q[j]) {
      ge = x[j] > q[j];
      break;
    }
  if (ge) {
    int64_t br = 0;
    for (int j = 0; j < L; ++j) {
      const int64_t v = (int64_t)x[j] - q[j] + br;
      x[j] = (uint32_t)v;
      br = v < 0 ? -1 : 0;
    }
  }
}

template <class C>
void curve_modulus(uint32_t *q);
template <>
void curve_modulus<CurveBn254>(uint32_t *q) {
  using F = FieldBn254Fq;
  const uint32_t v[8] = {F::P0, F::P1, F::P2, F::P3, F::P4, F::P5, F::P6, F::P7};
  std::memcpy(q, v, sizeof(v));
}
template <>
void curve_modulus<CurveBls381>(uint32_t *q) {
  using F = FieldBls12381Fq;
  const uint32_t v[12] = {F::P0, F::P1, F::P2, F::P3, F::P4, F::P5, F::P6, F::P7, F::P8, F::P9, F::P10, F::P11};
  std::memcpy(q, v, sizeof(v));
}

// Generators (public curve parameters), standard form.
template <class C>
void curve_generator(uint32_t *gx, uint32_t *gy);
template <>
void curve_generator<CurveBn254>(uint32_t *gx, uint32_t *gy) {
  for (int j = 0; j < 8; ++j) gx[j] = gy[j] = 0;
  gx[0] = 1;
  gy[0] = 2;
}
template <>
void curve_generator<CurveBls381>(uint32_t *gx, uint32_t *gy) {
  const uint32_t x[12] = {0xdb22c6bbu, 0xfb3af00au, 0xf97a1aefu, 0x6c55e83fu, 0x171bac58u, 0xa14e3a3fu,
                          0x9774b905u, 0xc3688c4fu, 0x4fa9ac0fu, 0x2695638cu, 0x3197d794u, 0x17f1d3a7u};
  const uint32_t y[12] = {0x46c5e7e1u, 0x0caa2329u, 0xa2888ae4u, 0xd03cc744u, 0x2c04b3edu, 0x00db18cbu,
                          0xd5d00af6u, 0xfcf5e095u, 0x741d8ae4u, 0xa09e30edu, 0xe3aaa0f1u, 0x08b3f481u};
  std::memcpy(gx, x, sizeof(x));
  std::memcpy(gy, y, sizeof(y));
}

// Montgomery constants from the modulus alone: R = 2^(32 L) mod q by
// doubling 1, R^2 by doubling R, b R by adding R.
template <class C>
EcConst<typename C::T> make_const() {
  constexpr int L = C::T::L;
  uint32_t q[L];
  curve_modulus<C>(q);
  EcConst<typename C::T> k;
  for (int j = 0; j < L; ++j) k.one[j] = 0;
  k.one[0] = 1;
  for (int i = 0; i < 32 * L; ++i) host_double_mod(k.one, q, L);
  std::memcpy(k.r2, k.one, sizeof(k.one));
  for (int i = 0; i < 32 * L; ++i) host_double_mod(k.r2, q, L);
  for (int j = 0; j < L; ++j) k.b3[j] = 0;
  for (uint32_t i = 0; i < C::kB; ++i) host_add_mod(k.b3, k.one, q, L);
  curve_generator<C>(k.gx, k.gy);
  return k;
}

ntt_status cuda_st(cudaError_t e) {
  if (e == cudaSuccess) return NTT_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? NTT_ERR_OOM : NTT_ERR_CUDA;
}

#define MSM_TRY(expr)               \
  do {                              \
    const ntt_status _s = (expr);   \
    if (_s != NTT_OK) return _s;    \
  } while (0)

ntt_status check_device(int *dev_out, int *sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return NTT_ERR_NO_DEVICE;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return NTT_ERR_NO_DEVICE;
  }
  if (prop.major != 10 || prop.minor != 3) return NTT_ERR_NO_DEVICE;
  *dev_out = dev;
  *sms = prop.multiProcessorCount;
  return NTT_OK;
}

// K c >= S^BL + 1 (signed digits)
uint32_t num_windows(uint32_t c, uint32_t scalar_bits) { return (scalar_bits + 1 + c - 1) / c; }

// Window size minimising the modelled multiply count K (10 n + 26 2^(c-1)):
// one 10-product mixed addition per point and window, about 26 products per
// bucket in the reduction tree.
uint32_t default_window(uint64_t n, uint32_t scalar_bits) {
  uint32_t best = 4;
  double best_cost = 1e300;
  for (uint32_t c = 4; c <= 21; ++c) {
    const double cost =
        (double)num_windows(c, scalar_bits) * (10.0 * (double)n + 26.0 * (double)(1u << (c - 1)));
    if (cost < best_cost) {
      best_cost = cost;
      best = c;
    }
  }
  return best;
}

// Entries per accumulation segment: enough segments to fill the GPU eight
// times over (512 resident threads per SM), 8..128 additions each.  Longer
// segments cut the buckets that cross a segment end, hence the combine work.
uint32_t segment_length(uint64_t max_n, uint32_t K, int sms) {
  const uint64_t entries = max_n * K;
  const uint64_t want = (uint64_t)sms * 512 * 8;
  return (uint32_t)std::max<uint64_t>(8, std::min<uint64_t>(128, entries / want));
}

uint32_t curve_scalar_bits(int curve) { return curve == MSM_CURVE_BLS12_381_G1 ? 255u : 254u; }
uint32_t curve_elem_bytes(int curve) { return curve == MSM_CURVE_BLS12_381_G1 ? 48u : 32u; }

}  // namespace
}  // namespace gb300ntt

using namespace gb300ntt;

struct msm_plan_s {
  int device = 0;
  int sms = 0;
  int curve = 0;
  uint32_t elem_bytes = 32;   // one coordinate
  uint64_t max_n = 0;
  uint32_t c = 0, K = 0, S = 0;
  uint64_t nb = 0;            // K 2^(c-1) buckets
  uint64_t max_segments = 0;
  uint32_t num_tiles = 0;
  EcConst<FqBn254> k254;
  EcConst<FqBls381> k381;
  uint4 *pts_m = nullptr;     // max_n points, Montgomery form
  uint32_t *counts = nullptr, *offsets = nullptr, *cursor = nullptr, *tile_sums = nullptr;
  MsmTotals *tot = nullptr;
  uint32_t *sorted = nullptr;
  uint2 *seg_ends = nullptr;  // first and last bucket of each segment
  uint4 *bucket_sum = nullptr, *pieces = nullptr;   // nb and 2 max_segments XYZZ points
  uint4 *heap_w = nullptr, *heap_b = nullptr;       // nb XYZZ points each
  uint4 *bases = nullptr;     // precomputed window copies: K x max_n points (msm_plan_set_bases)
  uint64_t bases_n = 0;       // points set (0: none)
  uint64_t device_bytes = 0;
};

namespace {

void free_plan(msm_plan p) {
  void *bufs[] = {p->pts_m, p->counts, p->offsets, p->cursor, p->tile_sums, p->tot, p->sorted,
                  p->seg_ends, p->bucket_sum, p->pieces, p->heap_w, p->heap_b, p->bases};
  for (void *b : bufs)
    if (b) cudaFree(b);
  delete p;
}

template <class T>
ntt_status alloc(T **ptr, uint64_t bytes, uint64_t *total) {
  *total += bytes;
  return cuda_st(cudaMalloc((void **)ptr, bytes ? bytes : 16));
}

int grid_for(uint64_t work, int threads, int sms, int per_sm) {
  const uint64_t blocks = (work + threads - 1) / threads;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(blocks, (uint64_t)sms * per_sm));
}

template <class C>
const EcConst<typename C::T> &plan_const(const msm_plan p);
template <>
const EcConst<FqBn254> &plan_const<CurveBn254>(const msm_plan p) { return p->k254; }
template <>
const EcConst<FqBls381> &plan_const<CurveBls381>(const msm_plan p) { return p->k381; }

// The launch sequence of one MSM (all on stream st).
// flat: the plan's precomputed bases (pt unused): one bucket set for all
// windows, the points gathered from the window copies, one reduction tree
// and no window merge.
template <class C>
ntt_status enqueue_msm(msm_plan p, const uint4 *sc, const uint4 *pt, uint64_t n, uint32_t kb, uint32_t ke,
                       uint4 *result, cudaStream_t st, bool flat = false) {
  const auto &k = plan_const<C>(p);
  const int sms = p->sms;
  const uint32_t lb = p->c - 1;
  const uint64_t nb = flat ? (1ull << lb) : p->nb;           // buckets in use
  const uint32_t num_tiles = (uint32_t)((nb + kScanTile - 1) / kScanTile);
  const uint4 *pts = flat ? p->bases : p->pts_m;
  const uint32_t tree_kb = flat ? 0 : kb, tree_ke = flat ? 1 : ke;
  MSM_TRY(cuda_st(cudaMemsetAsync(p->counts, 0, nb * 4, st)));
  // keep the error bits (read by msm_poll_error), reset the rest
  MSM_TRY(cuda_st(cudaMemsetAsync(p->tot, 0, offsetof(MsmTotals, err), st)));
  if (n > 0) {
    if (!flat)
      msm_prepare_kernel<C><<<grid_for(n, kEcThreads, sms, 16), kEcThreads, 0, st>>>(pt, n, k, p->pts_m, p->tot);
    msm_count_kernel<C><<<grid_for(n, 256, sms, 8), 256, 0, st>>>(sc, n, p->c, kb, ke, flat, p->counts, p->tot);
  }
  scan_reduce_kernel<<<num_tiles, kScanThreads, 0, st>>>(p->counts, nb, p->tile_sums);
  scan_tiles_kernel<<<1, kScanThreads, 0, st>>>(p->tile_sums, num_tiles, nb, p->offsets, p->tot);
  scan_apply_kernel<<<num_tiles, kScanThreads, 0, st>>>(p->counts, nb, p->tile_sums, p->offsets, p->cursor);
  if (n > 0) {
    msm_scatter_kernel<<<grid_for(n, 256, sms, 8), 256, 0, st>>>(sc, n, p->c, kb, ke,
                                                                 flat ? (uint32_t)p->max_n : 0u, p->cursor,
                                                                 p->sorted);
    const uint64_t segs = (n * p->K + p->S - 1) / p->S;
    const int g = grid_for(segs, kEcThreads, sms, C::kMinBlocks);
    msm_accumulate_kernel<C><<<g, kEcThreads, 0, st>>>(pts, p->sorted, p->offsets, nb, p->S, k, p->tot,
                                                       p->seg_ends, p->bucket_sum, p->pieces);
    // a bucket holds at most n entries, so it crosses at most ceil(n / S)
    // segment boundaries; rounds beyond the measured maximum exit at once
    const uint64_t max_span = (n + p->S - 1) / p->S;
    const int gt = grid_for(segs, kEcThreads, sms, C::kTreeMinBlocks);
    for (uint32_t r = 0; (1ull << r) <= max_span; ++r)
      msm_combine_kernel<C><<<gt, kEcThreads, 0, st>>>(p->offsets, p->seg_ends, p->S, p->tot, r, p->pieces);
  }
  for (int s = (int)lb - 1; s >= 0 && tree_ke > tree_kb; --s) {
    const uint64_t work = ((uint64_t)(tree_ke - tree_kb)) << s;
    msm_reduce_level_kernel<C><<<grid_for(work, kEcThreads, sms, C::kTreeMinBlocks), kEcThreads, 0, st>>>(
        (uint32_t)s, lb, tree_kb, tree_ke - tree_kb, p->bucket_sum, p->pieces, p->offsets, p->S, p->heap_w,
        p->heap_b);
  }
  msm_merge_kernel<C><<<1, 32, 0, st>>>(p->c, tree_kb, tree_ke, p->heap_w, p->bucket_sum, p->pieces, p->offsets,
                                        p->S, k, result);
  return cuda_st(cudaGetLastError());
}

std::mutex g_fb_mutex;
std::map<std::pair<int, int>, uint4 *> g_fb_tables;  // (device, curve) -> affine comb table (8192 points)

template <class C>
ntt_status fixed_base_table(int dev, int curve, const EcConst<typename C::T> &kc, cudaStream_t st, uint4 **out) {
  std::lock_guard<std::mutex> lock(g_fb_mutex);
  auto it = g_fb_tables.find({dev, curve});
  if (it != g_fb_tables.end()) {
    *out = it->second;
    return NTT_OK;
  }
  const uint64_t eb = 4ull * C::T::L;  // bytes per coordinate
  uint4 *xyzz = nullptr, *aff = nullptr;
  MSM_TRY(cuda_st(cudaMalloc((void **)&xyzz, 8192ull * 4 * eb)));
  ntt_status s = cuda_st(cudaMalloc((void **)&aff, 8192ull * 2 * eb));
  if (s == NTT_OK) {
    fixed_base_table_kernel<C><<<1, 32, 0, st>>>(kc, xyzz);
    fixed_base_affine_kernel<C><<<8192 / kEcThreads, kEcThreads, 0, st>>>(kc, xyzz, aff);
    s = cuda_st(cudaGetLastError());
    if (s == NTT_OK) s = cuda_st(cudaStreamSynchronize(st));
  }
  cudaFree(xyzz);
  if (s != NTT_OK) {
    if (aff) cudaFree(aff);
    return s;
  }
  g_fb_tables[{dev, curve}] = aff;
  *out = aff;
  return NTT_OK;
}

template <class C>
ntt_status fixed_base(int dev, int sms, int curve, const uint4 *ts, uint64_t n, uint4 *out, cudaStream_t st) {
  const EcConst<typename C::T> kc = make_const<C>();
  uint4 *table = nullptr;
  MSM_TRY(fixed_base_table<C>(dev, curve, kc, st, &table));
  fixed_base_points_kernel<C><<<grid_for(n, kEcThreads, sms, 16), kEcThreads, 0, st>>>(kc, table, ts, n, out);
  return cuda_st(cudaGetLastError());
}

bool curve_valid(int curve) { return curve == MSM_CURVE_BN254_G1 || curve == MSM_CURVE_BLS12_381_G1; }

}  // namespace

extern "C" {

ntt_status msm_point_bytes(msm_curve curve, uint32_t *bytes) {
  if (!bytes || !curve_valid((int)curve)) return NTT_ERR_INVALID_ARG;
  *bytes = 2 * curve_elem_bytes((int)curve);
  return NTT_OK;
}

ntt_status msm_plan_create(msm_plan *out, msm_curve curve, uint64_t max_n, uint32_t window_bits) {
  if (!out) return NTT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!curve_valid((int)curve)) return NTT_ERR_INVALID_ARG;
  if (max_n > MSM_MAX_POINTS) return NTT_ERR_UNSUPPORTED;
  if (window_bits > 22) return NTT_ERR_UNSUPPORTED;
  const uint32_t sbits = curve_scalar_bits((int)curve);
  const uint32_t c = window_bits ? window_bits : default_window(std::max<uint64_t>(max_n, 1), sbits);
  // sorted entries are counted in 32 bits (with room for one segment past
  // the end); point indices stay below 2^31, bit 31 carries the digit sign
  if (max_n * num_windows(c, sbits) >= (1ull << 32) - 256) return NTT_ERR_UNSUPPORTED;
  int dev = 0, sms = 0;
  MSM_TRY(check_device(&dev, &sms));
  msm_plan p = new (std::nothrow) msm_plan_s();
  if (!p) return NTT_ERR_OOM;
  p->device = dev;
  p->sms = sms;
  p->curve = (int)curve;
  p->elem_bytes = curve_elem_bytes((int)curve);
  p->max_n = max_n;
  p->c = c;
  p->K = num_windows(c, sbits);
  p->S = segment_length(max_n, p->K, sms);
  p->nb = (uint64_t)p->K << (c - 1);
  const uint64_t entries = max_n * p->K;
  p->max_segments = (entries + p->S - 1) / p->S + 1;
  p->num_tiles = (uint32_t)((p->nb + kScanTile - 1) / kScanTile);
  if (p->curve == MSM_CURVE_BLS12_381_G1) p->k381 = make_const<CurveBls381>();
  else p->k254 = make_const<CurveBn254>();
  const uint64_t pb = 2ull * p->elem_bytes, xb = 4ull * p->elem_bytes;  // affine and XYZZ point bytes
  uint64_t &tb = p->device_bytes;
  ntt_status s = NTT_OK;
  if (s == NTT_OK) s = alloc(&p->pts_m, max_n * pb, &tb);
  if (s == NTT_OK) s = alloc(&p->counts, p->nb * 4, &tb);
  if (s == NTT_OK) s = alloc(&p->offsets, (p->nb + 1) * 4, &tb);
  if (s == NTT_OK) s = alloc(&p->cursor, p->nb * 4, &tb);
  if (s == NTT_OK) s = alloc(&p->tile_sums, (uint64_t)p->num_tiles * 4, &tb);
  if (s == NTT_OK) s = alloc(&p->tot, sizeof(MsmTotals), &tb);
  if (s == NTT_OK) s = alloc(&p->sorted, entries * 4, &tb);
  if (s == NTT_OK) s = alloc(&p->seg_ends, p->max_segments * sizeof(uint2), &tb);
  if (s == NTT_OK) s = alloc(&p->bucket_sum, p->nb * xb, &tb);
  if (s == NTT_OK) s = alloc(&p->pieces, 2 * p->max_segments * xb, &tb);
  if (s == NTT_OK) s = alloc(&p->heap_w, p->nb * xb, &tb);
  if (s == NTT_OK) s = alloc(&p->heap_b, p->nb * xb, &tb);
  if (s == NTT_OK) s = cuda_st(cudaMemset(p->tot, 0, sizeof(MsmTotals)));
  if (s != NTT_OK) {
    free_plan(p);
    return s;
  }
  *out = p;
  return NTT_OK;
}

ntt_status msm_plan_info(msm_plan plan, msm_plan_desc *out) {
  if (!plan || !out) return NTT_ERR_INVALID_ARG;
  out->max_n = plan->max_n;
  out->window_bits = plan->c;
  out->num_windows = plan->K;
  out->segment_length = plan->S;
  out->reserved = 0;
  out->device_bytes = plan->device_bytes;
  return NTT_OK;
}

ntt_status msm_plan_destroy(msm_plan plan) {
  if (!plan) return NTT_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  free_plan(plan);
  return NTT_OK;
}

ntt_status msm_execute(msm_plan p, const void *d_scalars, const void *d_points, uint64_t n, void *d_result,
                       ntt_stream stream) {
  gb300ntt::NvtxRange range("msm_execute");
  if (!p || !d_result || ((uintptr_t)d_result % 16)) return NTT_ERR_INVALID_ARG;
  if (n > p->max_n) return NTT_ERR_INVALID_ARG;
  const uintptr_t pa = p->curve == MSM_CURVE_BLS12_381_G1 ? 16 : 32;  // one 128- or 256-bit access
  if ((uintptr_t)d_result % pa) return NTT_ERR_INVALID_ARG;
  if (n > 0 && (!d_scalars || !d_points || ((uintptr_t)d_scalars % 32) || ((uintptr_t)d_points % pa)))
    return NTT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const uint4 *sc = (const uint4 *)d_scalars;
  const uint4 *pt = (const uint4 *)d_points;
  if (p->curve == MSM_CURVE_BLS12_381_G1)
    return enqueue_msm<CurveBls381>(p, sc, pt, n, 0, p->K, (uint4 *)d_result, st);
  return enqueue_msm<CurveBn254>(p, sc, pt, n, 0, p->K, (uint4 *)d_result, st);
}

ntt_status msm_execute_windows(msm_plan p, const void *d_scalars, const void *d_points, uint64_t n,
                               uint32_t window_begin, uint32_t window_end, void *d_result, ntt_stream stream) {
  if (!p || window_begin > window_end || window_end > p->K) return NTT_ERR_INVALID_ARG;
  if (window_begin == 0 && window_end == p->K) return msm_execute(p, d_scalars, d_points, n, d_result, stream);
  // the same argument checks as msm_execute
  if (!d_result || n > p->max_n) return NTT_ERR_INVALID_ARG;
  const uintptr_t pa = p->curve == MSM_CURVE_BLS12_381_G1 ? 16 : 32;
  if ((uintptr_t)d_result % pa) return NTT_ERR_INVALID_ARG;
  if (n > 0 && (!d_scalars || !d_points || ((uintptr_t)d_scalars % 32) || ((uintptr_t)d_points % pa)))
    return NTT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const uint4 *sc = (const uint4 *)d_scalars;
  const uint4 *pt = (const uint4 *)d_points;
  if (p->curve == MSM_CURVE_BLS12_381_G1)
    return enqueue_msm<CurveBls381>(p, sc, pt, n, window_begin, window_end, (uint4 *)d_result, st);
  return enqueue_msm<CurveBn254>(p, sc, pt, n, window_begin, window_end, (uint4 *)d_result, st);
}

ntt_status msm_plan_set_bases(msm_plan p, const void *d_points, uint64_t n, ntt_stream stream) {
  if (!p || n > p->max_n) return NTT_ERR_INVALID_ARG;
  const uintptr_t pa = p->curve == MSM_CURVE_BLS12_381_G1 ? 16 : 32;
  if (n > 0 && (!d_points || ((uintptr_t)d_points % pa))) return NTT_ERR_INVALID_ARG;
  if (p->K > kMaxBaseWindows || (uint64_t)p->K * p->max_n >= (1ull << 31)) return NTT_ERR_UNSUPPORTED;
  if (!p->bases) {
    const uint64_t bytes = (uint64_t)p->K * std::max<uint64_t>(p->max_n, 1) * 2 * p->elem_bytes;
    MSM_TRY(cuda_st(cudaMalloc((void **)&p->bases, bytes)));
    p->device_bytes += bytes;
  }
  cudaStream_t st = (cudaStream_t)stream;
  p->bases_n = 0;
  if (n > 0) {
    const uint4 *pt = (const uint4 *)d_points;
    if (p->curve == MSM_CURVE_BLS12_381_G1)
      msm_bases_kernel<CurveBls381><<<grid_for(n, kEcThreads, p->sms, 8), kEcThreads, 0, st>>>(
          pt, n, p->c, p->K, p->max_n, p->k381, p->bases, p->tot);
    else
      msm_bases_kernel<CurveBn254><<<grid_for(n, kEcThreads, p->sms, 8), kEcThreads, 0, st>>>(
          pt, n, p->c, p->K, p->max_n, p->k254, p->bases, p->tot);
    MSM_TRY(cuda_st(cudaGetLastError()));
  }
  p->bases_n = n;
  return NTT_OK;
}

ntt_status msm_execute_bases(msm_plan p, const void *d_scalars, uint64_t n, void *d_result, ntt_stream stream) {
  if (!p || !d_result || n > p->bases_n || (n == 0 && !p->bases)) return NTT_ERR_INVALID_ARG;
  const uintptr_t pa = p->curve == MSM_CURVE_BLS12_381_G1 ? 16 : 32;
  if (((uintptr_t)d_result % pa) || (n > 0 && (!d_scalars || ((uintptr_t)d_scalars % 32))))
    return NTT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const uint4 *sc = (const uint4 *)d_scalars;
  if (p->curve == MSM_CURVE_BLS12_381_G1)
    return enqueue_msm<CurveBls381>(p, sc, nullptr, n, 0, p->K, (uint4 *)d_result, st, true);
  return enqueue_msm<CurveBn254>(p, sc, nullptr, n, 0, p->K, (uint4 *)d_result, st, true);
}

ntt_status msm_poll_error(msm_plan p, uint32_t *flags) {
  if (!p || !flags) return NTT_ERR_INVALID_ARG;
  // the calls may run on non-blocking streams: wait for all of them
  MSM_TRY(cuda_st(cudaDeviceSynchronize()));
  MsmTotals t;
  MSM_TRY(cuda_st(cudaMemcpy(&t, p->tot, sizeof(t), cudaMemcpyDeviceToHost)));
  *flags = t.err;
  const uint32_t zero = 0;
  MSM_TRY(cuda_st(cudaMemcpy(&p->tot->err, &zero, sizeof(zero), cudaMemcpyHostToDevice)));
  return NTT_OK;
}

ntt_status msm_fixed_base(msm_curve curve, const void *d_scalars, uint64_t n, void *d_points, ntt_stream stream) {
  if (!curve_valid((int)curve)) return NTT_ERR_INVALID_ARG;
  if (n == 0) return NTT_OK;
  const uintptr_t pa = curve == MSM_CURVE_BLS12_381_G1 ? 16 : 32;
  if (!d_scalars || !d_points || ((uintptr_t)d_scalars % 32) || ((uintptr_t)d_points % pa))
    return NTT_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  MSM_TRY(check_device(&dev, &sms));
  cudaStream_t st = (cudaStream_t)stream;
  const uint4 *ts = (const uint4 *)d_scalars;
  if (curve == MSM_CURVE_BLS12_381_G1)
    return fixed_base<CurveBls381>(dev, sms, (int)curve, ts, n, (uint4 *)d_points, st);
  return fixed_base<CurveBn254>(dev, sms, (int)curve, ts, n, (uint4 *)d_points, st);
}

}  // extern "C"
