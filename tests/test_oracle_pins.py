"""Pins that tie the CPU oracle to something other than itself.

Each pin is a fact the mathematics or an independent library fixes:
  * field constants: primality, 2-adicity, generator order (sympy), and the
    public curve definitions stored in tests/golden/fields.json;
  * the root of unity: omega^N = 1 and omega^(N/2) = -1;
  * sympy.discrete.transforms.ntt (an independent library NTT that uses the
    same smallest primitive root, 7 / 5) on small sizes;
  * brute force: the literal O(N^2) definition on tiny sizes;
  * closed forms for special vectors (delta_0, ones, delta_1);
  * the convolution theorem against a schoolbook polynomial product;
  * coset outputs against Horner evaluation at s * omega^k;
  * the coset inverse against the evaluations of monomials z^m on the coset
    (it must return the unit vector e_m) and the literal definition;
  * the pointwise quotient through a whole prover step: with
    C = A B - (X^n - 1) Q built by schoolbook polynomial arithmetic, coset
    transforms, the quotient by the vanishing polynomial and the coset
    inverse must give back Q exactly;
  * the inverse round trip and linearity;
  * the Python oracle against the independent C oracle.
The mutation tests at the end plant plausible mistakes in a copy of the
oracle and check that at least one pin fails for each.
"""

from __future__ import annotations

import json
import os
import random
import types

import numpy as np
import pytest
import sympy
from sympy.discrete.transforms import intt as sympy_intt
from sympy.discrete.transforms import ntt as sympy_ntt

import oracle
from oracle import ntt_oracle as O
from ntt_synth import uniform_elements, words64_of

HERE = os.path.dirname(os.path.abspath(__file__))
FIELDS = [O.BLS12_381_FR, O.BN254_FR]
FIELD_IDS = [f.name for f in FIELDS]
WIDE = [O.W377, O.W753]
ALL_FIELDS = FIELDS + WIDE
ALL_IDS = [f.name for f in ALL_FIELDS]


def rand_vec(field, n, seed):
    return O.limbs_to_ints(uniform_elements(field.name, n, seed), words64_of(field.name))


# ------------------------------------------------------------- field data


@pytest.mark.parametrize("field", FIELDS, ids=FIELD_IDS)
def test_field_constants_match_golden(field):
    with open(os.path.join(HERE, "golden", "fields.json")) as fh:
        g = json.load(fh)[field.name]
    assert field.modulus == int(g["modulus"], 16)
    assert field.modulus.bit_length() == g["bits"]
    assert field.generator == g["generator"]
    assert field.two_adicity == g["two_adicity"]
    assert O.default_coset_shift(field) == g["coset_shift"]


@pytest.mark.parametrize("field", FIELDS, ids=FIELD_IDS)
def test_field_is_prime_with_stated_two_adicity_and_generator(field):
    r = field.modulus
    assert sympy.isprime(r)
    k = field.two_adicity
    assert (r - 1) % (1 << k) == 0 and (r - 1) % (1 << (k + 1)) != 0
    assert sympy.is_primitive_root(field.generator, r)


@pytest.mark.parametrize("field", FIELDS, ids=FIELD_IDS)
def test_root_of_unity_has_exact_order(field):
    r = field.modulus
    for log_n in (1, 2, 5, 12, 20, 24, field.two_adicity):
        n = 1 << log_n
        w = O.root_of_unity(field, n)
        assert pow(w, n, r) == 1
        assert pow(w, n // 2, r) == r - 1
    with pytest.raises(ValueError):
        O.root_of_unity(field, 1 << (field.two_adicity + 1))


# ------------------------------------------------------------------ pins
# Each takes an object with ntt / intt / coset_ntt / dft_direct so that the
# mutation tests below can run the same checks against a broken copy.


def pin_sympy(impl, field, sizes=(2, 4, 8, 16, 32, 64)):
    for n in sizes:
        x = rand_vec(field, n, 1000 + n)
        if impl.ntt(field, x) != sympy_ntt(x, field.modulus):
            return False
        X = rand_vec(field, n, 2000 + n)
        if impl.intt(field, X) != sympy_intt(X, field.modulus):
            return False
    return True


def pin_brute_force(impl, field, sizes=(2, 4, 8, 16)):
    # The definition computed as a matrix-vector product with explicitly
    # built powers omega^(k*n) (pow with the exponent k*n, no recurrence).
    r = field.modulus
    for n in sizes:
        w = pow(field.generator, (r - 1) // n, r)
        x = rand_vec(field, n, 3000 + n)
        want = [sum(x[j] * pow(w, j * k, r) for j in range(n)) % r for k in range(n)]
        if impl.ntt(field, x) != want:
            return False
    return True


def pin_special_vectors(impl, field, n=64):
    r = field.modulus
    w = pow(field.generator, (r - 1) // n, r)
    delta0 = [1] + [0] * (n - 1)
    ones = [1] * n
    delta1 = [0, 1] + [0] * (n - 2)
    if impl.ntt(field, delta0) != [1] * n:
        return False
    if impl.ntt(field, ones) != [n % r] + [0] * (n - 1):
        return False
    if impl.ntt(field, delta1) != [pow(w, k, r) for k in range(n)]:
        return False
    # inverse of the delta_1 spectrum's conjugate: intt(ones) = delta_0
    if impl.intt(field, ones) != delta0:
        return False
    return True


def pin_convolution(impl, field, n=64):
    r = field.modulus
    a = rand_vec(field, n // 2, 4000) + [0] * (n // 2)
    b = rand_vec(field, n // 2, 4001) + [0] * (n // 2)
    # schoolbook polynomial product (degree < n, so cyclic == linear)
    prod = [0] * n
    for i in range(n // 2):
        for j in range(n // 2):
            prod[i + j] = (prod[i + j] + a[i] * b[j]) % r
    A = impl.ntt(field, a)
    B = impl.ntt(field, b)
    C = [u * v % r for u, v in zip(A, B)]
    return impl.intt(field, C) == prod


def pin_coset_horner(impl, field, n=128):
    r = field.modulus
    s = field.generator
    w = pow(field.generator, (r - 1) // n, r)
    x = rand_vec(field, n, 5000)
    X = impl.coset_ntt(field, x, s)
    for k in (0, 1, 2, n // 2 - 1, n // 2, n - 1, 37 % n):
        z = s * pow(w, k, r) % r
        acc = 0
        for c in reversed(x):
            acc = (acc * z + c) % r
        if X[k] != acc:
            return False
    return True


def pin_roundtrip_linearity(impl, field, n=256):
    r = field.modulus
    x = rand_vec(field, n, 6000)
    y = rand_vec(field, n, 6001)
    if impl.intt(field, impl.ntt(field, x)) != x:
        return False
    c = 0x1234567890ABCDEF1234567890ABCDEF % r
    lhs = impl.ntt(field, [(u + c * v) % r for u, v in zip(x, y)])
    X = impl.ntt(field, x)
    Y = impl.ntt(field, y)
    return lhs == [(u + c * v) % r for u, v in zip(X, Y)]


def pin_coset_inverse(impl, field, n=64):
    # interpolation from the coset {s omega^k}: the evaluations of z^m there
    # are the coefficient vector e_m; small sizes against the literal
    # definition x_n = s^-n N^-1 sum_k X_k omega^-nk; and it undoes coset_ntt
    r = field.modulus
    s = field.generator
    w = pow(field.generator, (r - 1) // n, r)
    for m in (0, 1, 5, n - 1):
        X = [pow(s * pow(w, k, r) % r, m, r) for k in range(n)]
        if impl.coset_intt(field, X, s) != [1 if j == m else 0 for j in range(n)]:
            return False
    for nn in (2, 4, 16):
        ww = pow(field.generator, (r - 1) // nn, r)
        X = rand_vec(field, nn, 5500 + nn)
        ninv = pow(nn, r - 2, r)
        sinv = pow(s, r - 2, r)
        # omega^-jk = omega^((nn - jk mod nn) mod nn)
        want = [pow(sinv, j, r) * ninv * sum(X[k] * pow(ww, (nn - j * k % nn) % nn, r) for k in range(nn)) % r
                for j in range(nn)]
        if impl.coset_intt(field, X, s) != want:
            return False
    x = rand_vec(field, n, 5600)
    return impl.coset_intt(field, impl.coset_ntt(field, x, s), s) == x


def _poly_mul(a, b, r):
    out = [0] * (len(a) + len(b) - 1)
    for i, u in enumerate(a):
        for j, v in enumerate(b):
            out[i + j] = (out[i + j] + u * v) % r
    return out


def pin_quotient_pipeline(impl, field, n=16, blowup=4):
    # A, B, Q of degree < n; C = A B - (X^n - 1) Q, so (A B - C) / (X^n - 1)
    # = Q exactly.  On the coset s<omega_m> (m = blowup n) the vanishing
    # polynomial X^n - 1 takes the values s^n omega_blowup^j - 1, j = k mod blowup.
    r = field.modulus
    m = blowup * n
    s = field.generator
    A = rand_vec(field, n, 5700)
    B = rand_vec(field, n, 5701)
    Q = rand_vec(field, n, 5702)
    AB = _poly_mul(A, B, r)                         # degree 2n - 2
    ZQ = [0] * n + Q                                # X^n Q
    C = [(AB[i] if i < len(AB) else 0) - (ZQ[i] if i < len(ZQ) else 0) + (Q[i] if i < n else 0)
         for i in range(2 * n)]
    C = [v % r for v in C]
    pad = lambda v: list(v) + [0] * (m - len(v))    # noqa: E731
    a, b, c = (impl.coset_ntt(field, pad(v), s) for v in (A, B, C))
    w_b = pow(field.generator, (r - 1) // blowup, r)
    sn = pow(s, n, r)
    z = [pow((sn * pow(w_b, j, r) - 1) % r, r - 2, r) for j in range(blowup)]
    t = impl.quotient_pointwise(field, a, b, c, z)
    return impl.coset_intt(field, t, s) == pad(Q)


ALL_PINS = [pin_sympy, pin_brute_force, pin_special_vectors, pin_convolution,
            pin_coset_horner, pin_roundtrip_linearity, pin_coset_inverse, pin_quotient_pipeline]


@pytest.mark.parametrize("field", ALL_FIELDS, ids=ALL_IDS)
@pytest.mark.parametrize("pin", ALL_PINS, ids=[p.__name__ for p in ALL_PINS])
def test_oracle_pin(pin, field):
    if pin is pin_sympy and field in WIDE:
        pytest.skip("sympy's NTT needs a factorisation of p - 1 (a 345/721-bit cofactor here)")
    assert pin(O, field)


@pytest.mark.parametrize("field", WIDE, ids=[f.name for f in WIDE])
def test_wide_field_follows_its_rule(field):
    # the smallest prime c 2^32 + 1 (c odd) above floor(pi 2^(b-2)), b its bit
    # length; the generator is the smallest quadratic non-residue
    import mpmath

    p = field.modulus
    b = p.bit_length()
    mpmath.mp.prec = b + 64
    start = int(mpmath.floor(mpmath.pi * mpmath.mpf(2) ** (b - 2)))
    assert p > start and (p - 1) % (1 << 32) == 0 and ((p - 1) >> 32) % 2 == 1
    assert sympy.isprime(p)
    c = (start >> 32) + 1
    c += (c + 1) % 2
    while (c << 32) + 1 < p:
        assert not sympy.isprime((c << 32) + 1)
        c += 2
    g = field.generator
    assert all(pow(a, (p - 1) // 2, p) == 1 for a in range(2, g))
    assert pow(g, (p - 1) // 2, p) == p - 1
    w = O.root_of_unity(field, 1 << 32)
    assert pow(w, 1 << 31, p) == p - 1 and pow(w, 1 << 32, p) == 1


@pytest.mark.parametrize("field", WIDE, ids=[f.name for f in WIDE])
def test_wide_direct_definition_equals_radix2(field):
    for n in (1 << k for k in range(1, 6)):
        x = rand_vec(field, n, 7100 + n)
        assert O.dft_direct(field, x) == O.ntt(field, x)


@pytest.mark.parametrize("field", FIELDS, ids=FIELD_IDS)
def test_direct_definition_equals_radix2(field):
    for n in (1 << k for k in range(1, 8)):
        x = rand_vec(field, n, 7000 + n)
        assert O.dft_direct(field, x) == O.ntt(field, x)


# ---------------------------------------------------------- the C oracle


@pytest.mark.parametrize("field", FIELDS, ids=FIELD_IDS)
@pytest.mark.parametrize("kind", ["forward", "inverse", "coset", "coset_inverse"])
def test_c_oracle_matches_python_oracle(field, kind):
    for log_n in list(range(1, 11)) + [12]:
        n = 1 << log_n
        x = uniform_elements(field.name, n, 8000 + log_n)
        want = O.transform(field, kind, O.limbs_to_ints(x))
        got = oracle.c_transform(field, kind, x)
        assert O.limbs_to_ints(got) == want, (kind, log_n)


@pytest.mark.parametrize("field", FIELDS, ids=FIELD_IDS)
def test_c_oracle_custom_coset_shift(field):
    x = uniform_elements(field.name, 256, 8100)
    s = 0xABCDEF0123456789 % field.modulus
    got = oracle.c_transform(field, "coset", x, shift=s)
    assert O.limbs_to_ints(got) == O.coset_ntt(field, O.limbs_to_ints(x), s)


@pytest.mark.parametrize("field", FIELDS, ids=FIELD_IDS)
def test_c_oracle_root_and_eval(field):
    r = field.modulus
    for log_n in (1, 12, 20, 24, field.two_adicity):
        assert oracle.c_root(field, log_n) == O.root_of_unity(field, 1 << log_n)
    x = uniform_elements(field.name, 1000, 8200)
    z = 0x1111222233334444555566667777 % r
    assert oracle.c_eval(field, x, z) == O.horner(field, O.limbs_to_ints(x), z)


@pytest.mark.parametrize("field", FIELDS, ids=FIELD_IDS)
def test_c_oracle_invariants_at_2_16(field):
    r = field.modulus
    log_n = 16
    n = 1 << log_n
    w = O.root_of_unity(field, n)
    delta1 = np.zeros((n, 4), dtype=np.uint64)
    delta1[1, 0] = 1
    got = O.limbs_to_ints(oracle.c_transform(field, "forward", delta1))
    p = 1
    for k in range(n):
        assert got[k] == p
        p = p * w % r
    x = uniform_elements(field.name, n, 8300)
    X = oracle.c_transform(field, "forward", x)
    assert np.array_equal(oracle.c_transform(field, "inverse", X), x)
    # spot outputs by Horner evaluation at omega^k
    xi = O.limbs_to_ints(x)
    Xi = O.limbs_to_ints(X)
    rng = random.Random(5)
    for k in [0, 1, n - 1] + [rng.randrange(n) for _ in range(3)]:
        assert Xi[k] == O.horner(field, xi, pow(w, k, r))


def test_c_oracle_rejects_bad_arguments():
    lib = oracle.c_oracle()
    x = np.zeros((4, 4), dtype=np.uint64)
    y = np.zeros_like(x)
    p = oracle._ptr
    assert lib.oracle_ntt(2, 0, 2, None, p(x), p(y)) == 1
    assert lib.oracle_ntt(0, 0, 0, None, p(x), p(y)) == 2
    assert lib.oracle_ntt(1, 0, 29, None, p(x), p(y)) == 2
    assert lib.oracle_ntt(0, 7, 2, None, p(x), p(y)) == 3
    bad = O.ints_to_limbs([O.BLS12_381_FR.modulus] * 4)
    assert lib.oracle_ntt(0, 0, 2, None, p(bad), p(y)) == 5


# ------------------------------------------------------- planted mistakes


def _mutant(**overrides):
    ns = types.SimpleNamespace(ntt=O.ntt, intt=O.intt, coset_ntt=O.coset_ntt, coset_intt=O.coset_intt,
                               quotient_pointwise=O.quotient_pointwise, dft_direct=O.dft_direct)
    for k, v in overrides.items():
        setattr(ns, k, v)
    return ns


def _ntt_wrong_root(field, x):          # omega^2 instead of omega
    r = field.modulus
    w = O.root_of_unity(field, len(x))
    return O.ntt_with_root(field, x, w * w % r)


def _ntt_no_bitreverse(field, x):       # bit-reversal step dropped
    saved = O._bit_reverse_permute
    try:
        O._bit_reverse_permute = lambda a: list(a)
        return O.ntt(field, x)
    finally:
        O._bit_reverse_permute = saved


def _ntt_swapped_butterfly(field, x):   # (u - v, u + v): outputs of a butterfly swapped
    r = field.modulus
    n = len(x)
    a = O._bit_reverse_permute([v % r for v in x])
    w0 = O.root_of_unity(field, n)
    length = 2
    while length <= n:
        wl = pow(w0, n // length, r)
        half = length // 2
        for s in range(0, n, length):
            w = 1
            for j in range(half):
                u, v = a[s + j], a[s + j + half] * w % r
                a[s + j], a[s + j + half] = (u - v) % r, (u + v) % r
                w = w * wl % r
        length *= 2
    return a


def _intt_no_scale(field, X):           # N^-1 factor dropped
    n = len(X)
    return O.ntt_with_root(field, X, O.inverse(field, O.root_of_unity(field, n)))


def _intt_conjugate_missing(field, X):  # inverse uses omega instead of omega^-1
    n = len(X)
    ninv = O.inverse(field, n)
    return [v * ninv % field.modulus for v in O.ntt(field, X)]


def _coset_off_by_one(field, x, s=None):  # x_n s^(n+1)
    s = field.generator if s is None else s
    r = field.modulus
    return O.ntt(field, [v * pow(s, i + 1, r) % r for i, v in enumerate(x)])


def _coset_inverse_wrong_sign(field, X, s=None):  # x_n s^(+n) instead of s^(-n)
    s = field.generator if s is None else s
    r = field.modulus
    return [v * pow(s, i, r) % r for i, v in enumerate(O.intt(field, X))]


def _coset_inverse_unscaled(field, X, s=None):  # N^-1 dropped
    n = len(X)
    r = field.modulus
    return [v * n % r for v in O.coset_intt(field, X, s)]


def _quotient_shifted_z(field, a, b, c, z):  # z index off by one
    r = field.modulus
    return [(x * y - w) * z[(i + 1) % len(z)] % r for i, (x, y, w) in enumerate(zip(a, b, c))]


def _quotient_sign(field, a, b, c, z):        # (a b + c) instead of (a b - c)
    r = field.modulus
    return [(x * y + w) * z[i % len(z)] % r for i, (x, y, w) in enumerate(zip(a, b, c))]


def _ntt_transposed_output(field, x):   # output index bit-reversed (a transposed four-step)
    X = O.ntt(field, x)
    return O._bit_reverse_permute(X)


MUTANTS = {
    "wrong_root": _mutant(ntt=_ntt_wrong_root),
    "no_bit_reverse": _mutant(ntt=_ntt_no_bitreverse),
    "swapped_butterfly": _mutant(ntt=_ntt_swapped_butterfly),
    "inverse_unscaled": _mutant(intt=_intt_no_scale),
    "inverse_wrong_root": _mutant(intt=_intt_conjugate_missing),
    "coset_off_by_one": _mutant(coset_ntt=_coset_off_by_one),
    "output_bit_reversed": _mutant(ntt=_ntt_transposed_output),
    "coset_inverse_wrong_sign": _mutant(coset_intt=_coset_inverse_wrong_sign),
    "coset_inverse_unscaled": _mutant(coset_intt=_coset_inverse_unscaled),
    "quotient_shifted_z": _mutant(quotient_pointwise=_quotient_shifted_z),
    "quotient_sign": _mutant(quotient_pointwise=_quotient_sign),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    impl = MUTANTS[name]
    field = O.BN254_FR
    failed = [p.__name__ for p in ALL_PINS if not p(impl, field)]
    assert failed, f"no pin caught the planted mistake {name}"


def test_c_oracle_all_cores_mode_equals_serial():
    """The C oracle's OpenMP mode (the all-cores CPU baseline) splits each
    stage's butterflies into runs that start their twiddle by exponentiation;
    it must give the serial loop's bytes for every kind and size, including
    sizes whose stages have fewer butterflies than runs."""
    from ntt_synth import uniform_elements

    try:
        for field in ("bls12_381_fr", "bn254_fr"):
            for log_n in (1, 3, 12, 14):
                x = uniform_elements(field, 1 << log_n, 7700 + log_n)
                for kind in ("forward", "inverse", "coset", "coset_inverse"):
                    oracle.c_set_threads(1)
                    serial = oracle.c_transform(field, kind, x)
                    oracle.c_set_threads(4)
                    assert np.array_equal(oracle.c_transform(field, kind, x), serial), (field, log_n, kind)
    finally:
        oracle.c_set_threads(1)
