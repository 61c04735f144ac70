"""Pins of the MSM oracle (CPU only) to facts outside itself.

  * the group law on tiny curves, by brute force: every point enumerated,
    closure, identity, inverses, commutativity, associativity, Lagrange
    (#E * P = O), repeated addition = double-and-add, and the closed-form
    count #E = q + 1 of y^2 = x^3 + b when q = 2 mod 3 (x -> x^3 is then a
    bijection of F_q, so every y gives exactly one x);
  * BN254 G1: the generator (1, 2) on the curve, r G = O for the published
    group order r, and 2G = (-23/16, -11/64) worked by hand from the tangent
    rule in rationals (slope 3 x^2 / (2 y) = 3/4);
  * the MSM definition against the closed form sum S_n (t_n G) =
    (sum S_n t_n mod r) G;
  * Algorithm 2 (LS-PPG) against the definition, over window sizes, lengths
    and the degenerate inputs (zero scalars, r - 1, repeated points, P and
    -P, points at infinity), and its tree-form bucket reduction against
    sum_j j B_j;
  * planted mistakes (made in a copy of the oracle, here on the CPU) that
    each pin must catch.
"""

from __future__ import annotations

import itertools
import random

import pytest

import ntt_synth
from oracle import msm_oracle as mo

pytestmark = pytest.mark.timeout(600)


def _all_points(curve: mo.Curve):
    q = curve.q
    sq = {}
    for y in range(q):
        sq.setdefault(y * y % q, []).append(y)
    pts = []
    for x in range(q):
        for y in sq.get((x * x * x + curve.b) % q, []):
            pts.append((x, y))
    return pts


@pytest.mark.parametrize("q,b", [(11, 1), (11, 3), (17, 3), (101, 3), (103, 3), (103, 5), (107, 2)])
def test_tiny_curve_group_law(q, b):
    curve = mo.Curve(q, b)
    pts = _all_points(curve)
    order = len(pts) + 1
    # Hasse bound
    assert (order - (q + 1)) ** 2 <= 4 * q
    if q % 3 == 2:
        assert order == q + 1
    allp = pts + [None]
    rng = random.Random(q * 31 + b)
    for P in allp:
        assert curve.add(P, None) == P and curve.add(None, P) == P
        assert curve.add(P, curve.neg(P)) is None
        assert mo.scalar_mul(curve, order, P) is None  # Lagrange
        # repeated addition equals double-and-add
        acc = None
        for k in range(1, min(order, 40) + 1):
            acc = curve.add(acc, P)
            assert mo.scalar_mul(curve, k, P) == acc
    pairs = list(itertools.product(allp, allp))
    if len(pairs) > 4000:
        pairs = rng.sample(pairs, 4000)
    for P, Q in pairs:
        R = curve.add(P, Q)
        assert curve.on_curve(R)
        assert R == curve.add(Q, P)
    triples = list(itertools.product(allp, repeat=3))
    if len(triples) > 6000:
        triples = rng.sample(triples, 6000)
    for P, Q, R in triples:
        assert curve.add(curve.add(P, Q), R) == curve.add(P, curve.add(Q, R))


def test_bn254_generator_and_order():
    c = mo.BN254_G1
    G = mo.BN254_G
    assert c.on_curve(G)
    assert 2 * 2 == 1 + 3
    assert mo.scalar_mul(c, mo.BN254_R, G) is None
    assert mo.scalar_mul(c, mo.BN254_R - 1, G) == c.neg(G)
    assert mo.scalar_mul(c, mo.BN254_R + 5, G) == mo.scalar_mul(c, 5, G)
    q = mo.BN254_Q
    two_g = ((-23) * pow(16, -1, q) % q, (-11) * pow(64, -1, q) % q)
    assert c.double(G) == two_g
    assert mo.scalar_mul(c, 2, G) == two_g
    assert c.on_curve(two_g)


def _scalars(n, seed):
    return [int(v) for v in _ints(ntt_synth.uniform_elements("bn254_fr", n, seed))]


def _ints(words):
    return [sum(int(row[j]) << (64 * j) for j in range(4)) for row in words]


def test_fixed_base_points():
    ts = _scalars(6, 11) + [0, 1, mo.BN254_R - 1]
    pts = mo.fixed_base_points(ts)
    for t, P in zip(ts, pts):
        assert P == mo.scalar_mul(mo.BN254_G1, t, mo.BN254_G)
        assert mo.BN254_G1.on_curve(P)


def test_msm_closed_form():
    n = 24
    ts = _scalars(n, 21)
    ss = _scalars(n, 22)
    pts = mo.fixed_base_points(ts)
    expect = mo.scalar_mul(mo.BN254_G1, sum(s * t for s, t in zip(ss, ts)) % mo.BN254_R, mo.BN254_G)
    assert mo.msm(ss, pts) == expect
    assert mo.msm([], []) is None


def _edge_inputs():
    ts = _scalars(12, 31)
    pts = mo.fixed_base_points(ts)
    c = mo.BN254_G1
    r = mo.BN254_R
    cases = {
        "random": (_scalars(12, 32), pts),
        "zero_scalars": ([0] * 12, pts),
        "r_minus_one": ([r - 1] * 3, pts[:3]),
        "repeated_point": ([5, 5, 7, 5], [pts[0]] * 4),
        "cancelling": ([9, 9, 4], [pts[1], c.neg(pts[1]), pts[2]]),
        "infinity_points": ([3, 8, 1], [None, pts[3], None]),
        "single": ([123456789], [pts[4]]),
        "empty": ([], []),
        "top_bits": ([(1 << 253) + 1, (1 << 253) - 1], pts[5:7]),
    }
    return cases


@pytest.mark.parametrize("c", [1, 2, 3, 4, 7, 8])
def test_ls_ppg_matches_definition(c):
    for name, (ss, pts) in _edge_inputs().items():
        assert mo.msm_ls_ppg(ss, pts, c) == mo.msm(ss, pts), (name, c)


def test_ls_ppg_ragged_window_and_length():
    # c not dividing 254 leaves a short top window; lengths not a power of two
    ss = _scalars(37, 41)
    pts = mo.fixed_base_points(_scalars(37, 42))
    expect = mo.msm(ss, pts)
    for c in (5, 6, 10, 13):
        assert mo.num_windows(254, c) == -(-254 // c)
        assert mo.msm_ls_ppg(ss, pts, c) == expect


@pytest.mark.parametrize("c", [1, 2, 3, 5, 6])
def test_bucket_reduce_tree_is_weighted_sum(c):
    pts = mo.fixed_base_points(_scalars(1 << c, 50 + c))
    rng = random.Random(c)
    buckets = [P if rng.random() > 0.2 else None for P in pts]
    buckets[0] = None
    assert mo.bucket_reduce_tree(buckets) == mo.bucket_reduce_direct(buckets)


def test_window_digits_cover_the_scalar():
    for s in _scalars(20, 60) + [mo.BN254_R - 1, 0, 1]:
        for c in (1, 4, 13, 16, 20):
            K = mo.num_windows(254, c)
            assert sum(mo.window_digit(s, k, c) << (k * c) for k in range(K)) == s


# -------------------------------------------------------- planted mistakes

class _WrongTangent(mo.Curve):
    """Doubling slope 2 x^2 / (2 y) instead of 3 x^2 / (2 y)."""

    def add(self, P, Q):
        if P is not None and Q is not None and P == Q and P[1] != 0:
            q = self.q
            lam = 2 * P[0] * P[0] * pow(2 * P[1], -1, q) % q
            x3 = (lam * lam - 2 * P[0]) % q
            return (x3, (lam * (P[0] - x3) - P[1]) % q)
        return super().add(P, Q)


class _WrongChordSign(mo.Curve):
    """y3 = lambda (x3 - x1) - y1: the sign of the chord term flipped."""

    def add(self, P, Q):
        if P is None or Q is None or P[0] == Q[0]:
            return super().add(P, Q)
        q = self.q
        lam = (Q[1] - P[1]) * pow(Q[0] - P[0], -1, q) % q
        x3 = (lam * lam - P[0] - Q[0]) % q
        return (x3, (lam * (x3 - P[0]) - P[1]) % q)


def test_mutant_group_laws_are_caught():
    for cls in (_WrongTangent, _WrongChordSign):
        bad = cls(mo.BN254_Q, mo.BN254_B, mo.BN254_R, mo.BN254_G)
        assert mo.scalar_mul(bad, mo.BN254_R, mo.BN254_G) is not None, cls.__name__
        tiny = cls(101, 3)
        pts = _all_points(tiny)
        failed = any(mo.scalar_mul(tiny, len(pts) + 1, P) is not None for P in pts) or any(
            not tiny.on_curve(tiny.add(P, Q)) for P, Q in itertools.product(pts[:20], pts[:20]))
        assert failed, cls.__name__


def test_mutant_msm_and_ppg_are_caught(monkeypatch):
    n = 10
    ts = _scalars(n, 71)
    ss = _scalars(n, 72)
    pts = mo.fixed_base_points(ts)
    curve = mo.BN254_G1
    closed = mo.scalar_mul(curve, sum(s * t for s, t in zip(ss, ts)) % mo.BN254_R, mo.BN254_G)

    # a dropped term in the definition
    assert mo.msm(ss[:-1], pts[:-1]) != closed
    # an off-by-one window index in the digits
    assert sum(mo.window_digit(ss[0], k + 1, 8) << (k * 8) for k in range(32)) != ss[0]

    # the tree reduction without the B_R term of the W update
    def tree_without_br(buckets, curve=curve):
        B = list(buckets)
        W = [None] * len(B)
        for s in range(len(B).bit_length() - 2, -1, -1):
            W = [curve.add(W[2 * b], W[2 * b + 1]) for b in range(1 << s)]
            B = [curve.double(curve.add(B[2 * b], B[2 * b + 1])) for b in range(1 << s)]
        return W[0]

    monkeypatch.setattr(mo, "bucket_reduce_tree", tree_without_br)
    assert mo.msm_ls_ppg(ss, pts, 4) != closed
    monkeypatch.undo()

    # window merging with one doubling too few per window
    def merge_short(window_sums, c, curve=curve):
        acc = None
        for W in reversed(window_sums):
            for _ in range(c - 1):
                acc = curve.double(acc)
            acc = curve.add(acc, W)
        return acc

    monkeypatch.setattr(mo, "window_merge", merge_short)
    assert mo.msm_ls_ppg(ss, pts, 4) != closed
    monkeypatch.undo()
    assert mo.msm_ls_ppg(ss, pts, 4) == closed


# ------------------------------------------------------------ BLS12-381 G1

def test_bls12_381_generator_and_order():
    c = mo.BLS12_381_G1
    G = mo.BLS12_381_G
    assert c.on_curve(G)
    assert mo.scalar_mul(c, mo.BLS12_381_R, G) is None  # G has order r (r prime, G != O)
    assert mo.scalar_mul(c, mo.BLS12_381_R - 1, G) == c.neg(G)
    assert mo.BLS12_381_Q.bit_length() == 381 and mo.BLS12_381_Q % 4 == 3
    # the subgroup order is the scalar field of the transforms
    assert mo.BLS12_381_R == ntt_synth.MODULI["bls12_381_fr"]


def test_bls12_381_msm_closed_form_and_ls_ppg():
    c = mo.BLS12_381_G1
    n = 12
    ts = [int(v) for v in _ints(ntt_synth.uniform_elements("bls12_381_fr", n, 81))]
    ss = [int(v) for v in _ints(ntt_synth.uniform_elements("bls12_381_fr", n, 82))]
    pts = mo.fixed_base_points(ts, c)
    for t, P in zip(ts[:3], pts[:3]):
        assert P == mo.scalar_mul(c, t, mo.BLS12_381_G)
    expect = mo.scalar_mul(c, sum(s * t for s, t in zip(ss, ts)) % mo.BLS12_381_R, mo.BLS12_381_G)
    assert mo.msm(ss, pts, c) == expect
    for w in (3, 8):
        assert mo.msm_ls_ppg(ss, pts, w, c, mo.BLS12_381_SCALAR_BITS) == expect
    # top scalar bit 254 set: the 255-bit windows must cover it
    big = [(1 << 254) + 3, mo.BLS12_381_R - 1]
    assert mo.msm_ls_ppg(big, pts[:2], 8, c, 255) == mo.msm(big, pts[:2], c)


def test_point_words_round_trip():
    c = mo.BLS12_381_G1
    pts = [mo.BLS12_381_G, None, c.double(mo.BLS12_381_G)]
    w = mo.points_to_words(pts, limbs=6)
    assert w.shape == (3, 12)
    assert mo.words_to_points(w, limbs=6) == pts
