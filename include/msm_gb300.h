/*
 * msm_gb300.h -- C ABI of the multi-scalar multiplication (MSM) of the
 * GB300 (sm_103a) library.
 *
 * The operation (MORPH, Sec. 2.3.1, the MSM definition; computed by the
 * paper's Layout-Stationary Pippenger, Algorithm 2): for N scalars S_n and
 * N points P_n of an elliptic-curve group,
 *
 *     MSM = sum_{n<N} S_n P_n.
 *
 * The result is a group element, so it is exact and unique.
 *
 * Curves:
 *   MSM_CURVE_BN254_G1      y^2 = x^3 + 3 over F_q,
 *     q = 0x30644e72e131a029b85045b68181585d97816a916871ca8d3c208c16d87cfd47,
 *     prime order r = the BN254 scalar field (ntt_gb300.h's NTT_FIELD_BN254_FR),
 *     generator (1, 2);
 *   MSM_CURVE_BLS12_381_G1  y^2 = x^3 + 4 over the 381-bit F_q,
 *     q = 0x1a0111ea397fe69a4b1ba7b6434bacd764774b84f38512bf6730d2a0f6b0f6241eabfffeb153ffffb9feffffffffaaab,
 *     points of the subgroup of prime order r = the BLS12-381 scalar field
 *     (NTT_FIELD_BLS12_381_FR), its standard generator.
 *
 * Data layout (device buffers):
 *   scalars  N x 32 bytes: four little-endian uint64 limbs, canonical in [0, r),
 *            32-byte aligned;
 *   points   N x (2 E) bytes, E = 32 (BN254) or 48 (BLS12-381) = msm_point_bytes / 2:
 *            affine x then y, each E / 8 little-endian uint64 limbs, standard
 *            (not Montgomery) form, canonical in [0, q); the point at
 *            infinity is encoded as x = y = 0 (not a curve point); aligned
 *            to 32 bytes (BN254) or 16 bytes (BLS12-381);
 *   result   one point, same encoding and alignment.
 *
 * Points are taken to lie in the prime-order group: BN254 G1 is the whole
 * curve; on BLS12-381 the caller supplies subgroup points (a point on the
 * curve but outside the subgroup is not detected).
 *
 * Ownership: the caller owns scalars, points and result.  A plan owns its
 * device scratch (a Montgomery copy of the points, the bucket index arrays,
 * segment sums and the reduction tree), allocated by msm_plan_create on the
 * current device and freed by msm_plan_destroy; msm_plan_info reports its
 * size.
 *
 * Streams: msm_execute only enqueues work on `stream` and returns.  The
 * scratch is shared by every call on a plan, so calls on one plan must be
 * ordered (one stream, or one plan per stream).
 *
 * Errors: NTT_ERR_INVALID_ARG for a NULL plan or buffer, a misaligned
 * buffer, an unknown curve or n > max_n; NTT_ERR_UNSUPPORTED for max_n above
 * MSM_MAX_POINTS, window_bits outside [1, 22] (0 = automatic), or a plan whose
 * bucket index count (max_n x windows) would not fit 32 bits;
 * NTT_ERR_OOM / NTT_ERR_CUDA / NTT_ERR_NO_DEVICE as in ntt_gb300.h.  Input
 * checks run on the device: a point that is not canonical or not on the
 * curve sets MSM_ERR_POINT and is treated as the point at infinity; a scalar
 * >= r sets MSM_ERR_SCALAR (the result stays exact for scalars below 2^254
 * and is unspecified above).  msm_poll_error reads and clears these bits
 * (it synchronises with the device).
 */
#ifndef MSM_GB300_H
#define MSM_GB300_H

#include "ntt_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum msm_curve {
    MSM_CURVE_BN254_G1 = 0,
    MSM_CURVE_BLS12_381_G1 = 1
} msm_curve;

#define MSM_MAX_POINTS (1ull << 28)
#define MSM_ERR_POINT 1u  /* a point not canonical or not on the curve */
#define MSM_ERR_SCALAR 2u /* a scalar >= r */

typedef struct msm_plan_s *msm_plan;

typedef struct msm_plan_desc {
    uint64_t max_n;          /* largest n accepted by msm_execute */
    uint32_t window_bits;    /* c: signed digits of c bits, 2^(c-1) buckets per window */
    uint32_t num_windows;    /* K = ceil((S + 1) / c), S = 254 (BN254) or 255 (BLS12-381) scalar bits */
    uint32_t segment_length; /* points summed by one thread before the tree */
    uint32_t reserved;
    uint64_t device_bytes;   /* scratch owned by the plan */
} msm_plan_desc;

/* Bytes of one affine point of `curve` (64 or 96). */
ntt_status msm_point_bytes(msm_curve curve, uint32_t *bytes);

/* Plan for up to max_n points.  window_bits = 0 picks c from max_n; for
 * window_bits = 1 every window holds one bucket. */
ntt_status msm_plan_create(msm_plan *out, msm_curve curve, uint64_t max_n, uint32_t window_bits);
ntt_status msm_plan_info(msm_plan plan, msm_plan_desc *out);
/* Synchronises the device, then frees the plan's scratch. */
ntt_status msm_plan_destroy(msm_plan plan);

/* result = sum_{n < count} scalars[n] points[n]; count may be 0 (result = O). */
ntt_status msm_execute(msm_plan plan, const void *d_scalars, const void *d_points, uint64_t count,
                       void *d_result, ntt_stream stream);
ntt_status msm_poll_error(msm_plan plan, uint32_t *flags);

/* Part of the MSM over the windows [window_begin, window_end) of the plan's
 * signed-digit decomposition (0 <= begin <= end <= num_windows):
 *     result = sum_{begin <= k < end} 2^(k c) W_k,
 * W_k the window's bucket sum (Algorithm 2's window sums, already scaled by
 * their weight).  The parts over a split of [0, num_windows) add up to the
 * MSM (msm_execute with all-ones scalars adds points), which is how the MSM
 * shards across GPUs: each GPU takes a range of windows, one gathers and
 * adds the parts.  An empty range gives the point at infinity.  Same
 * arguments, layout and errors as msm_execute otherwise. */
ntt_status msm_execute_windows(msm_plan plan, const void *d_scalars, const void *d_points, uint64_t count,
                               uint32_t window_begin, uint32_t window_end, void *d_result, ntt_stream stream);

/* Precomputed bases, for points reused across calls (a prover's fixed
 * setup points): msm_plan_set_bases checks and converts points[0..count)
 * once and stores, for every window k, the copies 2^(k c) P_n (affine), so
 * that msm_execute_bases(scalars) computes sum_n S_n P_n with one bucket set
 * for all windows: one reduction tree instead of K, and no window merge.
 * Same result as msm_execute.  Scratch: K x max_n extra points (counted in
 * device_bytes); NTT_ERR_UNSUPPORTED when the plan has more than 32 windows
 * (window_bits below 8 or 9) or K x max_n >= 2^31.  Invalid points set
 * MSM_ERR_POINT and count as the point at infinity.  msm_execute_bases
 * accepts count <= the count last set (NTT_ERR_INVALID_ARG otherwise, or
 * before any set); both calls enqueue on `stream`. */
ntt_status msm_plan_set_bases(msm_plan plan, const void *d_points, uint64_t count, ntt_stream stream);
ntt_status msm_execute_bases(msm_plan plan, const void *d_scalars, uint64_t count, void *d_result,
                             ntt_stream stream);

/* Fixed-base generation of inputs: points[n] = scalars[n] G (affine, standard
 * form; a zero scalar gives the point at infinity), any scalars < 2^256.
 * The first call per device and curve builds and keeps a comb table of 8192
 * multiples of G (512 or 768 KiB; it synchronises `stream` once). */
ntt_status msm_fixed_base(msm_curve curve, const void *d_scalars, uint64_t count, void *d_points,
                          ntt_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* MSM_GB300_H */
