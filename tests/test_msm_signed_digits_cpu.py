"""The GPU MSM's digit scheme, checked on the CPU against the oracle's group law.

The kernels cut each scalar into K = ceil((S + 1) / c) signed c-bit digits
(v = raw window value + carry; v > 2^(c-1) becomes v - 2^c with a carry into
the next window), put a point with digit d into bucket |d| - 1 (negated when
d < 0), and run Algorithm 2's reduction tree with its leaves started at
W_j = B_j, so that the root holds sum_j (j + 1) B_j.  This restates that
scheme in Python from its definition and checks the facts it relies on:
the digits reconstruct every scalar below 2^S, their magnitudes stay in
[0, 2^(c-1)], no carry is left over when K c >= S + 1, and the offset tree
gives the weighted sum.  Together they give the MSM definition (checked
against ``oracle.msm_oracle.msm``).
"""

from __future__ import annotations

import random

import pytest

import ntt_synth
from oracle import limbs_to_ints
from oracle import msm_oracle as mo


def signed_digits(s: int, c: int, K: int):
    """The kernels' recoding: list of (magnitude, negative), and the final carry."""
    out, carry = [], 0
    for k in range(K):
        v = ((s >> (k * c)) & ((1 << c) - 1)) + carry
        neg = v > (1 << (c - 1))
        carry = 1 if neg else 0
        out.append(((1 << c) - v if neg else v, neg))
    return out, carry


def offset_tree(buckets, curve):
    """Algorithm 2's tree with the leaves started at W_j = B_j."""
    B = list(buckets)
    W = list(buckets)
    n = len(B)
    while n > 1:
        W = [curve.add(curve.add(W[2 * b], W[2 * b + 1]), B[2 * b + 1]) for b in range(n // 2)]
        B = [curve.double(curve.add(B[2 * b], B[2 * b + 1])) for b in range(n // 2)]
        n //= 2
    return W[0]


@pytest.mark.parametrize("bits", [254, 255])
def test_recoding_reconstructs_and_bounds(bits):
    rng = random.Random(bits)
    scalars = [rng.getrandbits(bits) for _ in range(300)] + [0, 1, (1 << bits) - 1, (1 << (bits - 1))]
    for c in (1, 2, 5, 8, 13, 16, 17, 20, 22):
        K = -(-(bits + 1) // c)
        for s in scalars:
            digits, carry = signed_digits(s, c, K)
            assert carry == 0, (c, s)
            assert all(0 <= m <= (1 << (c - 1)) for m, _ in digits)
            assert sum((-m if neg else m) << (k * c) for k, (m, neg) in enumerate(digits)) == s


def test_one_window_short_leaves_a_carry():
    # the reason for K c >= S + 1: with K = ceil(S / c) windows a top-heavy
    # scalar can end with a carry that no window holds
    c, bits = 8, 256
    s = (1 << bits) - 1
    _, carry = signed_digits(s, c, bits // c)
    assert carry == 1


@pytest.mark.parametrize("lb", [0, 1, 2, 3, 4])
def test_offset_tree_is_weighted_sum(lb):
    curve = mo.BN254_G1
    pts = mo.fixed_base_points(limbs_to_ints(ntt_synth.uniform_elements("bn254_fr", 1 << lb, 90 + lb)))
    rng = random.Random(lb)
    buckets = [P if rng.random() > 0.25 else None for P in pts]
    expect = None
    for j, Bj in enumerate(buckets):
        expect = curve.add(expect, mo.scalar_mul(curve, j + 1, Bj))
    assert offset_tree(buckets, curve) == expect


def test_signed_bucket_msm_matches_definition():
    """Bucketize by |d| - 1 with signs, offset trees per window, Horner merge:
    the definition's result, on both curves."""
    for name, (curve, bits, _) in mo.CURVES.items():
        field = "bn254_fr" if name == "bn254_g1" else "bls12_381_fr"
        n = 24
        ss = limbs_to_ints(ntt_synth.uniform_elements(field, n, 95))
        pts = mo.fixed_base_points(limbs_to_ints(ntt_synth.uniform_elements(field, n, 96)), curve)
        for c in (3, 6):
            K = -(-(bits + 1) // c)
            windows = []
            for k in range(K):
                buckets = [None] * (1 << (c - 1))
                for s, P in zip(ss, pts):
                    m, neg = signed_digits(s, c, K)[0][k]
                    if m:
                        buckets[m - 1] = curve.add(buckets[m - 1], curve.neg(P) if neg else P)
                windows.append(offset_tree(buckets, curve))
            assert mo.window_merge(windows, c, curve) == mo.msm(ss, pts, curve), (name, c)


def test_mutant_leaf_start_is_caught():
    # leaves started at O (the unsigned form) lose the +1 of every weight
    curve = mo.BN254_G1
    pts = mo.fixed_base_points(limbs_to_ints(ntt_synth.uniform_elements("bn254_fr", 8, 99)))
    expect = None
    for j, Bj in enumerate(pts):
        expect = curve.add(expect, mo.scalar_mul(curve, j + 1, Bj))
    assert mo.bucket_reduce_tree(pts) != expect
    assert offset_tree(pts, curve) == expect
