"""Pins of the RNS lazy-multiplication oracle (oracle/rns_oracle.py).

What fixes the result independently of the oracle's own steps:
  * big-integer arithmetic: the reconstructed output R satisfies
    R == x y (mod M) and 0 <= R < L (the lazy bound), for random inputs, the
    extreme inputs L - 1 and 0, and along long chains of products;
  * the quotient estimates k and k2 equal the exact CRT quotients
    (sum_i xi_i (Q/q_i) - c) / Q and (sum_j eta_j (P/p_j) - R) / P, computed
    by big-integer division;
  * the bases: every modulus a prime below 2^31 (checked by sympy), the two
    bases disjoint, Q > 4 L^2 and P > 2^20 L;
  * planted mistakes in a copy of the oracle (a dropped CRT factor, k read at
    the wrong scale, a wrong correction sign, a byte-merge shift error, E1 without the
    P-side factor) each break one of the pins.
"""

from __future__ import annotations

import random

import pytest
import sympy

from oracle import rns_oracle as R

FIELDS = ["bls12_381_fr", "bn254_fr"]


@pytest.fixture(scope="module", params=FIELDS)
def basis(request):
    b = R.rns_basis(request.param)
    return b, R.tables(b)


def check_product(b, tabs, x, y, impl=R.rns_mul_lazy):
    r = impl(b, R.to_rns(x, b.q), R.to_rns(y, b.q), tabs)
    v = R.from_rns(r, b.q)
    return v % b.modulus == x * y % b.modulus and 0 <= v < b.L


def test_bases_are_prime_disjoint_and_large_enough(basis):
    b, _ = basis
    assert all(sympy.isprime(m) and m < 2**31 for m in b.q + b.p)
    assert not set(b.q) & set(b.p)
    assert b.Q > 4 * b.L * b.L
    assert b.P > (b.L << 20)
    assert b.L == (sum(b.q) + len(b.q)) * b.modulus


def test_products_are_congruent_and_within_the_lazy_bound(basis):
    b, tabs = basis
    rng = random.Random(11)
    cases = [(0, 0), (1, 1), (b.L - 1, b.L - 1), (b.L - 1, 1), (b.modulus - 1, b.modulus - 1)]
    cases += [(rng.randrange(b.L), rng.randrange(b.L)) for _ in range(200)]
    for x, y in cases:
        assert check_product(b, tabs, x, y), (x, y)


def test_quotient_estimates_are_exact(basis):
    b, tabs = basis
    rng = random.Random(12)
    Q, P = b.Q, b.P
    for _ in range(100):
        x, y = rng.randrange(b.L), rng.randrange(b.L)
        tr = {}
        r = R.rns_mul_lazy(b, R.to_rns(x, b.q), R.to_rns(y, b.q), tabs, tr)
        c = x * y
        k_exact, rem = divmod(sum(xi * (Q // qi) for xi, qi in zip(tr["xi"], b.q)) - c, Q)
        assert rem == 0 and tr["k"] == k_exact
        Rv = R.from_rns(r, b.q)
        k2_exact, rem2 = divmod(sum(e * (P // pj) for e, pj in zip(tr["eta"], b.p)) - Rv, P)
        assert rem2 == 0 and tr["k2"] == k2_exact


def test_chains_of_products_stay_exact(basis):
    b, tabs = basis
    rng = random.Random(13)
    x = rng.randrange(b.modulus)
    y = rng.randrange(b.modulus)
    r = R.to_rns(x, b.q)
    yr = R.to_rns(y, b.q)
    want = x
    for _ in range(300):
        r = R.rns_mul_lazy(b, r, yr, tabs)
        want = want * y % b.modulus
        v = R.from_rns(r, b.q)
        assert v < b.L and v % b.modulus == want


# ------------------------------------------------------- planted mistakes


def _mutant(change):
    def impl(b, x, y, tabs):
        t = dict(tabs)
        return change(b, x, y, t)
    return impl


def _no_crt_factor(b, x, y, t):
    t["q_hat_inv"] = [1] * len(b.q)
    return R.rns_mul_lazy(b, x, y, t)


def _k_wrong_scale(b, x, y, t):       # quotient estimate read at 2^(u-1)
    saved = R.U_SHIFT
    try:
        R.U_SHIFT = saved - 1
        return R.rns_mul_lazy(b, x, y, t)
    finally:
        R.U_SHIFT = saved


def _wrong_correction_sign(b, x, y, t):
    t["g"] = [(-gj) % pj for gj, pj in zip(t["g"], b.p)]
    return R.rns_mul_lazy(b, x, y, t)


def _merge_shift(b, x, y, t):
    saved = R.byte_merge
    try:
        R.byte_merge = lambda parts: sum(int(v) << (7 * h) for h, v in enumerate(parts))
        return R.rns_mul_lazy(b, x, y, t)
    finally:
        R.byte_merge = saved


def _e1_without_p_factor(b, x, y, t):
    M, Q = b.modulus, b.Q
    E1 = [[[R.byte_decompose((((Q // qi) % M) << (8 * bb)) % pj) for pj in b.p] for bb in range(4)] for qi in b.q]
    t["E1"] = E1
    return R.rns_mul_lazy(b, x, y, t)


MUTANTS = {
    "no_crt_factor": _no_crt_factor,
    "k_wrong_scale": _k_wrong_scale,
    "wrong_correction_sign": _wrong_correction_sign,
    "byte_merge_shift": _merge_shift,
    "e1_without_p_factor": _e1_without_p_factor,
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    b = R.rns_basis("bn254_fr")
    tabs = R.tables(b)
    impl = _mutant(MUTANTS[name])
    rng = random.Random(14)
    caught = any(not check_product(b, tabs, rng.randrange(b.L), rng.randrange(b.L), impl) for _ in range(20))
    assert caught, name
