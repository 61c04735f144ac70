// ntt_launch.h -- host-side launchers of the per-field kernels.
//
// Each field's kernels are instantiated in translation units of their own
// (kernels_<field>*.cu, one per kernel family) so that they compile in
// parallel; the plan code dispatches on the field id.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ntt_matrix.cuh"
#include "ntt_pass.cuh"

namespace gb300ntt {

// One element as eight 32-bit limbs (kernel-argument form).
struct Fe32 {
  uint32_t w[8];
};

// base^(2^b) for b < 32, Montgomery form: the square-and-multiply ladder
// used by the table generators.
struct Pow2Table {
  Fe32 v[32];
};

// One segment of a batched launch: all tiles of one pass of one job.
// Segments are ordered by pass level, so a segment only ever depends on an
// earlier one (deadlock-free with any number of resident CTAs).
struct BatchSeg {
  PassArgs a;
  uint32_t logs;        // log2 of the pass's sub-transform size
  uint32_t mode;        // PassMode
  uint32_t first_item;  // index of the segment's first tile in the item space
  uint32_t num_tiles;
  int32_t dep_seg;      // segment that must be complete first, or -1
  uint32_t dep_tiles;   // number of tiles of dep_seg
};

// Multipliers of the pointwise quotient, passed by value (no device table):
// z_j * 2^512 mod M for j < len, len a power of two <= kMaxQuotientZ.
constexpr int kMaxQuotientZ = 64;
struct QuotientZ {
  Fe32 z[kMaxQuotientZ];
  uint32_t len;
};

struct BatchLaunch {
  const BatchSeg *segs;   // device array, sorted by first_item
  uint32_t num_segs;
  uint32_t total_items;
  uint32_t *head;         // device: next item to claim (zeroed before launch)
  uint32_t *done;         // device: completed tiles per segment (zeroed)
  uint32_t *err;          // device: first error code (NTT_ERR_TIMEOUT)
  uint64_t wait_ns;       // bound of every dependency wait
  uint32_t grid;          // CTAs (a multiple of the SM count)
};

struct FieldLaunchers {
  cudaError_t (*prepare)();
  // one pass; tl = log2 of the tile (10 or 11), logs <= tl; fused selects the
  // fused tile where one exists (tl = 10, logs >= 4), else the staged one
  cudaError_t (*pass)(int logs, int mode, int tl, bool fused, const PassArgs &a, uint64_t tiles, cudaStream_t st);
  // out[n * Mp + q] = init * fac[n] * base^(n*q)    (fac may be null)
  cudaError_t (*gen_2d)(uint4 *out, uint32_t log_s, uint32_t log_mp, const Pow2Table &pw, const uint4 *fac,
                        Fe32 init, cudaStream_t st);
  // out[i] = init * base^i, i < count
  cudaError_t (*gen_1d)(uint4 *out, uint64_t count, const Pow2Table &pw, Fe32 init, cudaStream_t st);
  // out[i] = a[i] * b[i] * 2^-256 (element-wise Montgomery product; tests)
  cudaError_t (*mul_vec)(uint4 *out, const uint4 *a, const uint4 *b, uint64_t count, cudaStream_t st);
  // persistent batched kernel over the items of `b`
  cudaError_t (*batch)(const BatchLaunch &b, cudaStream_t st);
  // out[i] = a[i] * (b[i] 2^-256)^reps; variant 0 per-thread chains, 1 warp-cooperative
  cudaError_t (*mul_rep)(uint4 *out, const uint4 *a, const uint4 *b, uint64_t count, uint32_t reps, int variant,
                         cudaStream_t st);
  // one matrix-form pass (logs <= 3), `grid` persistent CTAs
  cudaError_t (*matrix_pass)(int logs, int mode, const MatrixPassArgs &ma, const CUtensorMap &in_map, uint32_t grid,
                             cudaStream_t st);
  // out[i] = (a[i] b[i] - c[i]) z[i mod z_len] (z given as z 2^512 mod M)
  cudaError_t (*quotient)(uint4 *out, const uint4 *a, const uint4 *b, const uint4 *c, const QuotientZ &z,
                          uint64_t count, cudaStream_t st);
};

namespace bls12_381 {
const FieldLaunchers &launchers();
}
namespace bn254 {
const FieldLaunchers &launchers();
}

inline const FieldLaunchers &launchers(int field) {
  return field == 0 ? bls12_381::launchers() : bn254::launchers();
}

}  // namespace gb300ntt
