// msm.cu -- multi-scalar multiplication on BN254 G1 by the paper's
// Layout-Stationary Pippenger (MORPH, Algorithm 2), GB300 form.
//
//   MSM = sum_{n<N} S_n P_n, S_n < r (254 bits), P_n affine points.
//
// Each scalar is cut into K = ceil(254 / c) unsigned c-bit digits; window k
// keeps 2^c buckets.  The four phases of Algorithm 2 map to kernels:
//
//   Bucketize    msm_count_kernel      digit histogram (one counter per bucket,
//                                      atomics in L2; digit 0 is skipped)
//                scan_*_kernel         exclusive scan -> bucket offsets, plus
//                                      a scan of ceil(count / S) -> segments
//                msm_scatter_kernel    point index n into its bucket's slot
//                                      (the argsort of the digits, as a
//                                      counting sort)
//   BA           msm_accumulate_kernel one thread per segment of at most S
//                                      points of one bucket (bucket += affine
//                                      point, XYZZ madd); then
//                msm_combine_kernel    a pairwise tree over a bucket's
//                                      segments, so no bucket is ever summed
//                                      by one thread alone (a skewed or
//                                      constant scalar set stays parallel)
//   BR           msm_reduce_level_kernel  the tree of Algorithm 2, one launch
//                                      per level s = c-1 .. 0, all windows at
//                                      once: W_b = W_2b + W_2b+1 + B_2b+1,
//                                      B_b = 2 (B_2b + B_2b+1)
//   WM           msm_merge_kernel      Horner over the windows, top one first
//                                      (MSM = 2^c MSM + W_k), then the affine
//                                      standard-form result.
//
// The paper streams the sorted points straight into bucket accumulation on
// the TPU; here the sort moves 4-byte point indices and the accumulation
// gathers the 64-byte points by index (a point is read once per window from
// HBM; the accumulation is bound by the integer multiply pipe, not by these
// reads).  Points are converted to Montgomery form once per call
// (msm_prepare_kernel), which also checks that every point lies on the curve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <map>
#include <mutex>
#include <new>

#include "../../include/msm_gb300.h"
#include "ec_bn254.cuh"
#include "host_field.h"

namespace gb300ntt {
namespace {

constexpr uint32_t kScalarBits = 254;
constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;
constexpr int kEcThreads = 128;

struct EcConst {
  uint32_t one[8];  // 2^256 mod q (Montgomery 1)
  uint32_t r2[8];   // 2^512 mod q (to Montgomery form)
  uint32_t b3[8];   // 3 * 2^256 mod q (curve constant b, Montgomery)
};

struct MsmTotals {
  uint32_t entries;   // points placed in buckets (digit != 0)
  uint32_t segments;  // accumulation segments
  uint32_t max_seg;   // most segments of one bucket
  uint32_t err;       // MSM_ERR_* bits
};

// ----------------------------------------------------------- small helpers

__device__ __forceinline__ void load_point_xyzz(PointXyzz &p, const uint4 *base, uint64_t i) {
  fe_load_global(p.X, base, 4 * i + 0);
  fe_load_global(p.Y, base, 4 * i + 1);
  fe_load_global(p.ZZ, base, 4 * i + 2);
  fe_load_global(p.ZZZ, base, 4 * i + 3);
}

__device__ __forceinline__ void store_point_xyzz(uint4 *base, uint64_t i, const PointXyzz &p) {
  fe_store_global(base, 4 * i + 0, p.X);
  fe_store_global(base, 4 * i + 1, p.Y);
  fe_store_global(base, 4 * i + 2, p.ZZ);
  fe_store_global(base, 4 * i + 3, p.ZZZ);
}

// c-bit digit of window k of the scalar s (8 little-endian words); c <= 24
__device__ __forceinline__ uint32_t window_digit(const uint32_t s[8], uint32_t k, uint32_t c) {
  const uint32_t bit = k * c, w = bit >> 5, sh = bit & 31u;
  if (w >= 8) return 0u;
  uint64_t v = s[w];
  if (w + 1 < 8) v |= (uint64_t)s[w + 1] << 32;
  return (uint32_t)(v >> sh) & ((1u << c) - 1u);
}

__device__ __forceinline__ bool scalar_is_canonical(const uint32_t s[8]) {
  const uint32_t r[8] = {0xf0000001u, 0x43e1f593u, 0x79b97091u, 0x2833e848u,
                         0x8181585du, 0xb85045b6u, 0xe131a029u, 0x30644e72u};
#pragma unroll
  for (int j = 7; j >= 0; --j)
    if (s[j] != r[j]) return s[j] < r[j];
  return false;
}

// ---------------------------------------------------------------- kernels

// Points to Montgomery form (x R, y R); (0, 0) stays the point at infinity.
// Flags points that are not canonical or not on y^2 = x^3 + 3 (and treats
// them as O so that the arithmetic below never sees a value >= q).
__global__ void __launch_bounds__(kEcThreads) msm_prepare_kernel(const uint4 *pts, uint64_t n, EcConst k,
                                                                 uint4 *pts_m, MsmTotals *tot) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x[8], y[8];
    fe_load_global(x, pts, 2 * i);
    fe_load_global(y, pts, 2 * i + 1);
    if (fe_is_zero(x) && fe_is_zero(y)) {
      fe_store_global(pts_m, 2 * i, x);
      fe_store_global(pts_m, 2 * i + 1, y);
      continue;
    }
    bool ok = fq_is_canonical(x) && fq_is_canonical(y);
    if (ok) {
      mont_mul<Fq>(x, x, k.r2);
      mont_mul<Fq>(y, y, k.r2);
      uint32_t l[8], r[8];
      mont_mul<Fq>(l, y, y);
      mont_mul<Fq>(r, x, x);
      mont_mul<Fq>(r, r, x);
      add_mod<Fq>(r, r, k.b3);
      ok = fe_equal(l, r);
    }
    if (!ok) {
      atomicOr(&tot->err, (uint32_t)MSM_ERR_POINT);
      fe_zero(x);
      fe_zero(y);
    }
    fe_store_global(pts_m, 2 * i, x);
    fe_store_global(pts_m, 2 * i + 1, y);
  }
}

// Bucketize, pass 1: one counter per (window, digit).
__global__ void __launch_bounds__(256) msm_count_kernel(const uint4 *scalars, uint64_t n, uint32_t c, uint32_t K,
                                                        uint32_t *counts, MsmTotals *tot) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t s[8];
    fe_load_global(s, scalars, i);
    if (!scalar_is_canonical(s)) atomicOr(&tot->err, (uint32_t)MSM_ERR_SCALAR);
    for (uint32_t k = 0; k < K; ++k) {
      const uint32_t d = window_digit(s, k, c);
      if (d) atomicAdd(&counts[((uint64_t)k << c) + d], 1u);
    }
  }
}

__device__ __forceinline__ uint32_t segs_of(uint32_t count, uint32_t S) { return (count + S - 1) / S; }

__device__ __forceinline__ uint2 add2(uint2 a, uint2 b) { return make_uint2(a.x + b.x, a.y + b.y); }

// Inclusive scan of a uint2 across a warp.
__device__ __forceinline__ uint2 warp_scan2(uint2 v) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(0xffffffffu, v.x, o);
    const uint32_t b = __shfl_up_sync(0xffffffffu, v.y, o);
    if (lane >= (uint32_t)o) {
      v.x += a;
      v.y += b;
    }
  }
  return v;
}

// Exclusive scan of v over the CTA (blockDim.x = kScanThreads); *total gets
// the CTA's sum.
__device__ __forceinline__ uint2 block_excl_scan2(uint2 v, uint2 *total) {
  __shared__ uint2 warp_sums[kScanThreads / 32];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint2 inc = warp_scan2(v);
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint2 w = lane < kScanThreads / 32 ? warp_sums[lane] : make_uint2(0, 0);
    const uint2 wi = warp_scan2(w);
    if (lane < kScanThreads / 32) warp_sums[lane] = make_uint2(wi.x - w.x, wi.y - w.y);
    if (lane == kScanThreads / 32 - 1) *total = wi;
  }
  __syncthreads();
  const uint2 base = warp_sums[warp];
  __syncthreads();
  return make_uint2(base.x + inc.x - v.x, base.y + inc.y - v.y);
}

// Scan pass 1: per-tile sums of (count, segments) and the largest segment
// count of a bucket.
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t *counts, uint64_t nb, uint32_t S,
                                                                   uint2 *tile_sums, MsmTotals *tot) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanPer;
  uint2 v = make_uint2(0, 0);
  uint32_t mx = 0;
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    if (base + j < nb) {
      const uint32_t cnt = counts[base + j];
      const uint32_t g = segs_of(cnt, S);
      v.x += cnt;
      v.y += g;
      mx = max(mx, g);
    }
  }
  __shared__ uint2 total;
  block_excl_scan2(v, &total);
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31u) == 0 && mx) atomicMax(&tot->max_seg, mx);
  __syncthreads();
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Scan pass 2 (one CTA): exclusive scan of the tile sums in place; the
// grand totals go to tot and to the final entries offsets[nb], seg_off[nb].
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(uint2 *tile_sums, uint32_t num_tiles, uint64_t nb,
                                                                  uint32_t *offsets, uint32_t *seg_off,
                                                                  MsmTotals *tot) {
  __shared__ uint2 chunk_total;
  uint2 carry = make_uint2(0, 0);
  for (uint32_t b0 = 0; b0 < num_tiles; b0 += kScanThreads) {
    const uint32_t i = b0 + threadIdx.x;
    const uint2 v = i < num_tiles ? tile_sums[i] : make_uint2(0, 0);
    const uint2 ex = block_excl_scan2(v, &chunk_total);
    if (i < num_tiles) tile_sums[i] = add2(carry, ex);
    __syncthreads();
    carry = add2(carry, chunk_total);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    tot->entries = carry.x;
    tot->segments = carry.y;
    offsets[nb] = carry.x;
    seg_off[nb] = carry.y;
  }
}

// Scan pass 3: bucket offsets (also copied to the scatter cursors) and
// segment offsets.
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t *counts, uint64_t nb, uint32_t S,
                                                                  const uint2 *tile_sums, uint32_t *offsets,
                                                                  uint32_t *cursor, uint32_t *seg_off) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanPer;
  uint32_t cnt[kScanPer];
  uint2 v = make_uint2(0, 0);
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    cnt[j] = base + j < nb ? counts[base + j] : 0u;
    v.x += cnt[j];
    v.y += segs_of(cnt[j], S);
  }
  __shared__ uint2 total;
  uint2 run = add2(block_excl_scan2(v, &total), tile_sums[blockIdx.x]);
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    if (base + j < nb) {
      offsets[base + j] = run.x;
      cursor[base + j] = run.x;
      seg_off[base + j] = run.y;
    }
    run.x += cnt[j];
    run.y += segs_of(cnt[j], S);
  }
}

// Bucketize, pass 2: each point index into the next free slot of its bucket.
__global__ void __launch_bounds__(256) msm_scatter_kernel(const uint4 *scalars, uint64_t n, uint32_t c, uint32_t K,
                                                          uint32_t *cursor, uint32_t *sorted) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t s[8];
    fe_load_global(s, scalars, i);
    for (uint32_t k = 0; k < K; ++k) {
      const uint32_t d = window_digit(s, k, c);
      if (d) sorted[atomicAdd(&cursor[((uint64_t)k << c) + d], 1u)] = (uint32_t)i;
    }
  }
}

// Largest b with seg_off[b] <= s (seg_off non-decreasing, seg_off[0] = 0).
__device__ __forceinline__ uint32_t bucket_of_segment(const uint32_t *seg_off, uint64_t nb, uint32_t s) {
  uint64_t lo = 0, hi = nb;  // seg_off[lo] <= s < seg_off[hi]
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (__ldg(seg_off + mid) <= s) lo = mid;
    else hi = mid;
  }
  return (uint32_t)lo;
}

// BA: segment s of bucket b sums at most S consecutive sorted points.
__global__ void __launch_bounds__(kEcThreads, 4)
    msm_accumulate_kernel(const uint4 *pts_m, const uint32_t *sorted, const uint32_t *offsets,
                          const uint32_t *seg_off, uint64_t nb, uint32_t S, EcConst k, const MsmTotals *tot,
                          uint32_t *seg_bucket, uint4 *partial) {
  const uint32_t num_segs = tot->segments;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < num_segs; s += gridDim.x * blockDim.x) {
    const uint32_t b = bucket_of_segment(seg_off, nb, s);
    const uint32_t i = s - seg_off[b];
    const uint32_t begin = offsets[b] + i * S;
    const uint32_t end = min(begin + S, offsets[b + 1]);
    PointXyzz acc;
    xyzz_set_inf(acc);
    for (uint32_t e = begin; e < end; ++e) {
      const uint32_t idx = __ldg(sorted + e);
      uint32_t x[8], y[8];
      fe_load_global(x, pts_m, 2 * (uint64_t)idx);
      fe_load_global(y, pts_m, 2 * (uint64_t)idx + 1);
      if (fe_is_zero(x) && fe_is_zero(y)) continue;  // point at infinity
      xyzz_madd(acc, x, y, k.one);
    }
    seg_bucket[s] = b;
    store_point_xyzz(partial, s, acc);
  }
}

// BA, combine round r: segment i (local index within its bucket) with i a
// multiple of 2^(r+1) adds segment i + 2^r; after ceil(log2(max_seg)) rounds
// a bucket's sum is in its first segment.
__global__ void __launch_bounds__(kEcThreads, 4)
    msm_combine_kernel(const uint32_t *seg_off, const uint32_t *seg_bucket, const MsmTotals *tot, uint32_t r,
                       uint4 *partial) {
  if ((1u << r) >= tot->max_seg) return;
  const uint32_t num_segs = tot->segments;
  const uint32_t step = 1u << r;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < num_segs; s += gridDim.x * blockDim.x) {
    const uint32_t b = seg_bucket[s];
    const uint32_t i = s - seg_off[b];
    const uint32_t m = seg_off[b + 1] - seg_off[b];
    if ((i & (2 * step - 1)) != 0 || i + step >= m) continue;
    PointXyzz a, q;
    load_point_xyzz(a, partial, s);
    load_point_xyzz(q, partial, s + step);
    xyzz_add(a, q);
    store_point_xyzz(partial, s, a);
  }
}

// Bucket B_{k,j} (leaf of the reduction tree): the first segment's sum, or O.
__device__ __forceinline__ void load_bucket(PointXyzz &p, const uint4 *partial, const uint32_t *counts,
                                            const uint32_t *seg_off, uint64_t b) {
  if (counts[b] == 0) xyzz_set_inf(p);
  else load_point_xyzz(p, partial, seg_off[b]);
}

// BR, level s of the tree (all windows): node (k, b), b < 2^s, from its two
// children.  Level s of window k is stored at heap index 2^s + b.
__global__ void __launch_bounds__(kEcThreads, 4)
    msm_reduce_level_kernel(uint32_t s, uint32_t c, uint32_t K, const uint4 *partial, const uint32_t *counts,
                            const uint32_t *seg_off, uint4 *heap_w, uint4 *heap_b) {
  const uint64_t per = 1ull << s, total = per * K;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = t >> s, b = t & (per - 1);
    const uint64_t heap0 = k << c;  // window k's heap
    const uint64_t node = heap0 + per + b;
    PointXyzz a, br;
    // W first (at most two points live at a time)
    if (s + 1 == c) {
      const uint64_t leaf = (k << c) + 2 * b;
      load_bucket(br, partial, counts, seg_off, leaf + 1);
      store_point_xyzz(heap_w, node, br);  // W_L = W_R = O at the leaves: W = B_R
      if (s == 0) continue;
      load_bucket(a, partial, counts, seg_off, leaf);
    } else {
      const uint64_t child = heap0 + 2 * per + 2 * b;
      load_point_xyzz(a, heap_w, child);
      load_point_xyzz(br, heap_w, child + 1);
      xyzz_add(a, br);
      load_point_xyzz(br, heap_b, child + 1);
      xyzz_add(a, br);
      store_point_xyzz(heap_w, node, a);
      if (s == 0) continue;  // the root's B is not needed
      load_point_xyzz(a, heap_b, child);
    }
    xyzz_add(a, br);
    xyzz_dbl(a, a);
    store_point_xyzz(heap_b, node, a);
  }
}

// WM: MSM = sum_k 2^(k c) W_k by Horner, then affine standard form.
__global__ void msm_merge_kernel(uint32_t c, uint32_t K, const uint4 *heap_w, EcConst kc, uint4 *result) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  PointXyzz acc;
  xyzz_set_inf(acc);
  for (int k = (int)K - 1; k >= 0; --k) {
    if (!xyzz_is_inf(acc))
      for (uint32_t j = 0; j < c; ++j) xyzz_dbl(acc, acc);
    PointXyzz w;
    load_point_xyzz(w, heap_w, ((uint64_t)k << c) + 1);
    xyzz_add(acc, w);
  }
  uint32_t x[8], y[8];
  xyzz_to_affine_std(x, y, acc, kc.one);
  fe_store_global(result, 0, x);
  fe_store_global(result, 1, y);
}

// ------------------------------------------------- fixed-base generation

// Comb table T[w][d] = d 2^(8 w) G (w < 32, d < 256), XYZZ, one thread per w.
__global__ void fixed_base_table_kernel(EcConst kc, uint4 *table_xyzz) {
  const uint32_t w = threadIdx.x;
  if (blockIdx.x != 0 || w >= 32) return;
  // G = (1, 2) in Montgomery form
  uint32_t gx[8], gy[8];
  fe_copy(gx, kc.one);
  add_mod<Fq>(gy, kc.one, kc.one);
  PointXyzz base;
  fe_copy(base.X, gx);
  fe_copy(base.Y, gy);
  fe_copy(base.ZZ, kc.one);
  fe_copy(base.ZZZ, kc.one);
  for (uint32_t j = 0; j < 8 * w; ++j) xyzz_dbl(base, base);
  PointXyzz acc;
  xyzz_set_inf(acc);
  store_point_xyzz(table_xyzz, 256 * w, acc);
  for (uint32_t d = 1; d < 256; ++d) {
    xyzz_add(acc, base);
    store_point_xyzz(table_xyzz, 256 * w + d, acc);
  }
}

// Table entries to affine Montgomery form ((0, 0) for O).
__global__ void __launch_bounds__(kEcThreads) fixed_base_affine_kernel(EcConst kc, const uint4 *table_xyzz,
                                                                       uint4 *table_aff) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 32 * 256) return;
  PointXyzz p;
  load_point_xyzz(p, table_xyzz, i);
  uint32_t x[8], y[8];
  if (xyzz_is_inf(p)) {
    fe_zero(x);
    fe_zero(y);
  } else {
    uint32_t t[8], inv[8], zi[8];
    mont_mul<Fq>(t, p.ZZ, p.ZZZ);
    fq_inverse(inv, t, kc.one);
    mont_mul<Fq>(zi, inv, p.ZZZ);
    mont_mul<Fq>(x, p.X, zi);
    mont_mul<Fq>(zi, inv, p.ZZ);
    mont_mul<Fq>(y, p.Y, zi);
  }
  fe_store_global(table_aff, 2 * i, x);
  fe_store_global(table_aff, 2 * i + 1, y);
}

// P_n = t_n G = sum_w T[w][byte w of t_n], affine standard form.
__global__ void __launch_bounds__(kEcThreads) fixed_base_points_kernel(EcConst kc, const uint4 *table_aff,
                                                                       const uint4 *ts, uint64_t n, uint4 *out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t t[8];
    fe_load_global(t, ts, i);
    PointXyzz acc;
    xyzz_set_inf(acc);
    for (uint32_t w = 0; w < 32; ++w) {
      const uint32_t d = (t[w >> 2] >> (8 * (w & 3))) & 0xffu;
      if (!d) continue;
      uint32_t x[8], y[8];
      fe_load_global(x, table_aff, 2 * (256 * w + d));
      fe_load_global(y, table_aff, 2 * (256 * w + d) + 1);
      xyzz_madd(acc, x, y, kc.one);
    }
    uint32_t x[8], y[8];
    xyzz_to_affine_std(x, y, acc, kc.one);
    fe_store_global(out, 2 * i, x);
    fe_store_global(out, 2 * i + 1, y);
  }
}

// ------------------------------------------------------------------ host

void to_words(uint32_t out[8], const U256 &v) {
  for (int j = 0; j < 4; ++j) {
    out[2 * j] = (uint32_t)v.w[j];
    out[2 * j + 1] = (uint32_t)(v.w[j] >> 32);
  }
}

EcConst make_const() {
  const HostField F(U256{{0x3c208c16d87cfd47ULL, 0x97816a916871ca8dULL, 0xb85045b68181585dULL,
                          0x30644e72e131a029ULL}},
                    3, 1);
  EcConst k;
  const U256 one = F.to_mont(u256(1));
  to_words(k.one, one);
  to_words(k.r2, F.to_mont(one));
  to_words(k.b3, F.to_mont(u256(3)));
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

// Window size minimising the modelled multiply count: K (10 n + 26 2^c)
// (one 10-product madd per point and window, about 26 products per bucket
// in the reduction tree), capped so that the tree stays small.
uint32_t default_window(uint64_t n) {
  uint32_t best = 4;
  double best_cost = 1e300;
  for (uint32_t c = 4; c <= 20; ++c) {
    const double K = (double)((kScalarBits + c - 1) / c);
    const double cost = K * (10.0 * (double)n + 26.0 * (double)(1u << c));
    if (cost < best_cost) {
      best_cost = cost;
      best = c;
    }
  }
  return best;
}

uint32_t segment_length(uint64_t max_n, uint32_t K, int sms) {
  // enough segments to fill the GPU several times over, at most 256 points each
  const uint64_t entries = max_n * K;
  const uint64_t want = (uint64_t)sms * 512 * 4;
  uint64_t S = entries / want;
  S = std::max<uint64_t>(16, std::min<uint64_t>(256, S));
  return (uint32_t)S;
}

}  // namespace
}  // namespace gb300ntt

using namespace gb300ntt;

struct msm_plan_s {
  int device = 0;
  int sms = 0;
  uint64_t max_n = 0;
  uint32_t c = 0, K = 0, S = 0;
  uint64_t nb = 0;            // K 2^c buckets
  uint64_t max_segments = 0;
  uint32_t num_tiles = 0;
  EcConst k;
  uint4 *pts_m = nullptr;     // max_n x 64 B
  uint32_t *counts = nullptr, *offsets = nullptr, *cursor = nullptr, *seg_off = nullptr;
  uint2 *tile_sums = nullptr;
  MsmTotals *tot = nullptr;
  uint32_t *sorted = nullptr, *seg_bucket = nullptr;
  uint4 *partial = nullptr;   // max_segments x 128 B
  uint4 *heap_w = nullptr, *heap_b = nullptr;  // K 2^c x 128 B each
  uint64_t device_bytes = 0;
};

namespace {

void free_plan(msm_plan p) {
  void *bufs[] = {p->pts_m, p->counts, p->offsets, p->cursor, p->seg_off, p->tile_sums, p->tot,
                  p->sorted, p->seg_bucket, p->partial, p->heap_w, p->heap_b};
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

std::mutex g_fb_mutex;
std::map<int, uint4 *> g_fb_tables;  // device -> affine comb table (8192 x 64 B)

ntt_status fixed_base_table(int dev, const EcConst &kc, cudaStream_t st, uint4 **out) {
  std::lock_guard<std::mutex> lock(g_fb_mutex);
  auto it = g_fb_tables.find(dev);
  if (it != g_fb_tables.end()) {
    *out = it->second;
    return NTT_OK;
  }
  uint4 *xyzz = nullptr, *aff = nullptr;
  MSM_TRY(cuda_st(cudaMalloc((void **)&xyzz, 8192ull * 128)));
  ntt_status s = cuda_st(cudaMalloc((void **)&aff, 8192ull * 64));
  if (s == NTT_OK) {
    fixed_base_table_kernel<<<1, 32, 0, st>>>(kc, xyzz);
    fixed_base_affine_kernel<<<8192 / kEcThreads, kEcThreads, 0, st>>>(kc, xyzz, aff);
    s = cuda_st(cudaGetLastError());
    if (s == NTT_OK) s = cuda_st(cudaStreamSynchronize(st));
  }
  cudaFree(xyzz);
  if (s != NTT_OK) {
    if (aff) cudaFree(aff);
    return s;
  }
  g_fb_tables[dev] = aff;
  *out = aff;
  return NTT_OK;
}

}  // namespace

extern "C" {

ntt_status msm_plan_create(msm_plan *out, msm_curve curve, uint64_t max_n, uint32_t window_bits) {
  if (!out) return NTT_ERR_INVALID_ARG;
  *out = nullptr;
  if (curve != MSM_CURVE_BN254_G1) return NTT_ERR_INVALID_ARG;
  if (max_n > MSM_MAX_POINTS) return NTT_ERR_UNSUPPORTED;
  if (window_bits > 22) return NTT_ERR_UNSUPPORTED;
  {
    const uint32_t c = window_bits ? window_bits : default_window(std::max<uint64_t>(max_n, 1));
    if (max_n * ((kScalarBits + c - 1) / c) >= (1ull << 32)) return NTT_ERR_UNSUPPORTED;
  }
  int dev = 0, sms = 0;
  MSM_TRY(check_device(&dev, &sms));
  msm_plan p = new (std::nothrow) msm_plan_s();
  if (!p) return NTT_ERR_OOM;
  p->device = dev;
  p->sms = sms;
  p->max_n = max_n;
  p->c = window_bits ? window_bits : default_window(std::max<uint64_t>(max_n, 1));
  p->K = (kScalarBits + p->c - 1) / p->c;
  p->S = segment_length(max_n, p->K, sms);
  p->nb = (uint64_t)p->K << p->c;
  const uint64_t entries = max_n * p->K;
  p->max_segments = entries / p->S + std::min<uint64_t>(p->nb, entries) + 1;
  p->num_tiles = (uint32_t)((p->nb + kScanTile - 1) / kScanTile);
  p->k = make_const();
  uint64_t &tb = p->device_bytes;
  ntt_status s = NTT_OK;
  if (s == NTT_OK) s = alloc(&p->pts_m, max_n * 64, &tb);
  if (s == NTT_OK) s = alloc(&p->counts, p->nb * 4, &tb);
  if (s == NTT_OK) s = alloc(&p->offsets, (p->nb + 1) * 4, &tb);
  if (s == NTT_OK) s = alloc(&p->cursor, p->nb * 4, &tb);
  if (s == NTT_OK) s = alloc(&p->seg_off, (p->nb + 1) * 4, &tb);
  if (s == NTT_OK) s = alloc(&p->tile_sums, (uint64_t)p->num_tiles * sizeof(uint2), &tb);
  if (s == NTT_OK) s = alloc(&p->tot, sizeof(MsmTotals), &tb);
  if (s == NTT_OK) s = alloc(&p->sorted, entries * 4, &tb);
  if (s == NTT_OK) s = alloc(&p->seg_bucket, p->max_segments * 4, &tb);
  if (s == NTT_OK) s = alloc(&p->partial, p->max_segments * 128, &tb);
  if (s == NTT_OK) s = alloc(&p->heap_w, p->nb * 128, &tb);
  if (s == NTT_OK) s = alloc(&p->heap_b, p->nb * 128, &tb);
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
  if (!p || !d_result || ((uintptr_t)d_result % 32)) return NTT_ERR_INVALID_ARG;
  if (n > p->max_n) return NTT_ERR_INVALID_ARG;
  if (n > 0 && (!d_scalars || !d_points || ((uintptr_t)d_scalars % 32) || ((uintptr_t)d_points % 32)))
    return NTT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const uint4 *sc = (const uint4 *)d_scalars;
  const uint4 *pt = (const uint4 *)d_points;
  const int sms = p->sms;
  MSM_TRY(cuda_st(cudaMemsetAsync(p->counts, 0, p->nb * 4, st)));
  // keep the error bits (read by msm_poll_error), reset the rest
  MSM_TRY(cuda_st(cudaMemsetAsync(p->tot, 0, offsetof(MsmTotals, err), st)));
  if (n > 0) {
    msm_prepare_kernel<<<grid_for(n, kEcThreads, sms, 16), kEcThreads, 0, st>>>(pt, n, p->k, p->pts_m, p->tot);
    msm_count_kernel<<<grid_for(n, 256, sms, 8), 256, 0, st>>>(sc, n, p->c, p->K, p->counts, p->tot);
  }
  scan_reduce_kernel<<<p->num_tiles, kScanThreads, 0, st>>>(p->counts, p->nb, p->S, p->tile_sums, p->tot);
  scan_tiles_kernel<<<1, kScanThreads, 0, st>>>(p->tile_sums, p->num_tiles, p->nb, p->offsets, p->seg_off, p->tot);
  scan_apply_kernel<<<p->num_tiles, kScanThreads, 0, st>>>(p->counts, p->nb, p->S, p->tile_sums, p->offsets,
                                                           p->cursor, p->seg_off);
  if (n > 0) {
    msm_scatter_kernel<<<grid_for(n, 256, sms, 8), 256, 0, st>>>(sc, n, p->c, p->K, p->cursor, p->sorted);
    const uint64_t segs_bound = n * p->K / p->S + std::min<uint64_t>(p->nb, n * p->K) + 1;
    const int g = grid_for(segs_bound, kEcThreads, sms, 4);
    msm_accumulate_kernel<<<g, kEcThreads, 0, st>>>(p->pts_m, p->sorted, p->offsets, p->seg_off, p->nb, p->S,
                                                    p->k, p->tot, p->seg_bucket, p->partial);
    // a bucket holds at most n points, so at most ceil(n / S) segments
    const uint64_t max_m = (n + p->S - 1) / p->S;
    for (uint32_t r = 0; (1ull << r) < max_m; ++r)
      msm_combine_kernel<<<g, kEcThreads, 0, st>>>(p->seg_off, p->seg_bucket, p->tot, r, p->partial);
  }
  for (int s = (int)p->c - 1; s >= 0; --s) {
    const uint64_t work = ((uint64_t)p->K) << s;
    msm_reduce_level_kernel<<<grid_for(work, kEcThreads, sms, 4), kEcThreads, 0, st>>>(
        (uint32_t)s, p->c, p->K, p->partial, p->counts, p->seg_off, p->heap_w, p->heap_b);
  }
  msm_merge_kernel<<<1, 32, 0, st>>>(p->c, p->K, p->heap_w, p->k, (uint4 *)d_result);
  return cuda_st(cudaGetLastError());
}

ntt_status msm_poll_error(msm_plan p, uint32_t *flags) {
  if (!p || !flags) return NTT_ERR_INVALID_ARG;
  MsmTotals t;
  MSM_TRY(cuda_st(cudaMemcpy(&t, p->tot, sizeof(t), cudaMemcpyDeviceToHost)));
  *flags = t.err;
  const uint32_t zero = 0;
  MSM_TRY(cuda_st(cudaMemcpy(&p->tot->err, &zero, sizeof(zero), cudaMemcpyHostToDevice)));
  return NTT_OK;
}

ntt_status msm_fixed_base(msm_curve curve, const void *d_scalars, uint64_t n, void *d_points, ntt_stream stream) {
  if (curve != MSM_CURVE_BN254_G1) return NTT_ERR_INVALID_ARG;
  if (n == 0) return NTT_OK;
  if (!d_scalars || !d_points || ((uintptr_t)d_scalars % 32) || ((uintptr_t)d_points % 32))
    return NTT_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  MSM_TRY(check_device(&dev, &sms));
  const EcConst kc = make_const();
  cudaStream_t st = (cudaStream_t)stream;
  uint4 *table = nullptr;
  MSM_TRY(fixed_base_table(dev, kc, st, &table));
  fixed_base_points_kernel<<<grid_for(n, kEcThreads, sms, 16), kEcThreads, 0, st>>>(
      kc, table, (const uint4 *)d_scalars, n, (uint4 *)d_points);
  return cuda_st(cudaGetLastError());
}

}  // extern "C"
