"""Plain, slow CPU oracle for the 255-bit number-theoretic transform.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link
or execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` use it.  It shares no code with
the CUDA library (``paper_2604_17808_gb300``): it has its own copy of the field
moduli, its own arithmetic (Python big integers) and its own transform.

What it computes (MORPH, Sec. 2.3.1, the NTT definition):

    X_k = sum_{n=0}^{N-1} x_n * omega_N^{k n}  mod M,   k in [0, N)

with omega_N a primitive N-th root of unity of the prime field F_M.  The paper
states the forward transform only; the inverse and the coset transform are the
standard companions that a prover's evaluation/interpolation step uses:

    inverse:        x_n = N^{-1} * sum_k X_k * omega_N^{-k n}
    coset:          X_k = sum_n x_n * (s * omega_N^k)^n = forward(x_n * s^n)
    coset inverse:  x_n = s^{-n} * inverse(X)_n, so coset_inverse(coset(x)) = x
                    (interpolation from a coset, the step after a prover's
                    pointwise work on the coset evaluations)

Readings of points the paper leaves open:
  * omega_N = g^((M-1)/N) with g the field's multiplicative generator (7 for
    BLS12-381 Fr, 5 for BN254 Fr).  The paper names neither field; the
    workload's fields and generators are the public curve definitions.
  * Coset shift s: the generator g (5 for BN254, 7 for BLS12-381) unless the
    caller passes another.
  * Elements are canonical integers in [0, M), natural order in and out.

Two evaluations of the definition are provided:
  * ``dft_direct``: the definition written out, O(N^2); used for tiny N.
  * ``ntt``: the textbook iterative radix-2 Cooley-Tukey evaluation (bit
    reversal, then log2 N butterfly stages; the paper's "butterfly NTT",
    Sec. 2.3.3 and Fig. 5a), which reaches exactly the same integers.

The pins that tie this module to something other than itself live in
``tests/test_oracle_pins.py`` (a library NTT, closed forms, invariants,
brute force on tiny inputs and the convolution theorem).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Field:
    name: str
    modulus: int          # the prime M (the curve's scalar-field order r)
    generator: int        # multiplicative generator g of F_M^*
    two_adicity: int      # largest k with 2^k | M - 1


# Scalar fields of the two curves the workload names.
BLS12_381_FR = Field(
    "bls12_381_fr",
    0x73EDA753299D7D483339D80809A1D80553BDA402FFFE5BFEFFFFFFFF00000001,
    7,
    32,
)
BN254_FR = Field(
    "bn254_fr",
    0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001,
    5,
    28,
)
# Wider fields for the paper's 377- and 753-bit rows (Sec. 4.3.1, Tab. 3
# evaluates those precisions without naming the moduli).  Reading: the
# smallest prime p = c 2^32 + 1, c odd, above floor(pi 2^(b-2)) (pseudo-random
# high bits, 2-adicity exactly 32), generator = the smallest quadratic
# non-residue, so g^((p-1)/N) is a primitive N-th root for N | 2^32.  The
# pins recompute the rule with sympy/mpmath.
W377 = Field(
    "w377",
    0x1921FB54442D18469898CC51701B839A252049C1114CF98E804177D4C76273644A29410F31C6809BBDF2BD500000001,
    7,
    32,
)
W753 = Field(
    "w753",
    0x1921FB54442D18469898CC51701B839A252049C1114CF98E804177D4C76273644A29410F31C6809BBDF2A33679A748636605614DBE4BE286E9FC26ADADAA3848BC90B6AECC4BCFD8DE89885D34C6FDAD617FEB96DE80D6FDBDCD300000001,
    11,
    32,
)
FIELDS = {f.name: f for f in (BLS12_381_FR, BN254_FR, W377, W753)}
# Index order used by the C ABI and by the C oracle (which covers the first two).
FIELD_BY_INDEX = (BLS12_381_FR, BN254_FR, W377, W753)


def limbs_of_field(field) -> int:
    """32-bit limbs of an element: 8 (<= 256 bits), 12 (377), 24 (753)."""
    bits = get_field(field).modulus.bit_length()
    return 8 if bits <= 256 else 12 if bits <= 384 else 24


def get_field(field) -> Field:
    if isinstance(field, Field):
        return field
    if isinstance(field, int):
        return FIELD_BY_INDEX[field]
    return FIELDS[field]


# ---------------------------------------------------------------- basics


def root_of_unity(field, n: int) -> int:
    """omega_n = g^((M-1)/n) mod M, a primitive n-th root of unity (n | 2^adicity)."""
    f = get_field(field)
    if n < 1 or n & (n - 1) or n.bit_length() - 1 > f.two_adicity:
        raise ValueError(f"no radix-2 root of unity of order {n} in {f.name}")
    return pow(f.generator, (f.modulus - 1) // n, f.modulus)


def inverse(field, a: int) -> int:
    f = get_field(field)
    return pow(a, f.modulus - 2, f.modulus)


def default_coset_shift(field) -> int:
    return get_field(field).generator


def _log2_exact(n: int) -> int:
    if n < 1 or n & (n - 1):
        raise ValueError(f"length {n} is not a power of two")
    return n.bit_length() - 1


# ------------------------------------------------------- the definition


def dft_direct(field, x, omega: int | None = None) -> list[int]:
    """X_k = sum_n x_n omega^{kn} mod M, written out literally (O(N^2))."""
    f = get_field(field)
    n = len(x)
    w = root_of_unity(f, n) if omega is None else omega
    out = []
    for k in range(n):
        wk = pow(w, k, f.modulus)
        acc = 0
        term = 1
        for j in range(n):
            acc += x[j] * term
            term = term * wk % f.modulus
        out.append(acc % f.modulus)
    return out


# --------------------------------------------- radix-2 butterfly evaluation


def _bit_reverse_permute(a: list[int]) -> list[int]:
    n = len(a)
    bits = _log2_exact(n)
    out = [0] * n
    for i in range(n):
        r = int(format(i, f"0{bits}b")[::-1], 2) if bits else 0
        out[r] = a[i]
    return out


def ntt_with_root(field, x, omega: int) -> list[int]:
    """Iterative radix-2 Cooley-Tukey: bit-reverse, then log2 N stages.

    Stage with block length L combines pairs (u, v) of the two half blocks as
    (u + w v, u - w v) with w running over the powers of omega^(N/L).
    """
    f = get_field(field)
    m = f.modulus
    n = len(x)
    _log2_exact(n)
    a = _bit_reverse_permute([int(v) % m for v in x])
    length = 2
    while length <= n:
        w_len = pow(omega, n // length, m)
        half = length // 2
        for start in range(0, n, length):
            w = 1
            for j in range(half):
                u = a[start + j]
                v = a[start + j + half] * w % m
                a[start + j] = (u + v) % m
                a[start + j + half] = (u - v) % m
                w = w * w_len % m
        length *= 2
    return a


def ntt(field, x) -> list[int]:
    """Forward transform X_k = sum_n x_n omega_N^{kn}."""
    return ntt_with_root(field, x, root_of_unity(field, len(x)))


def intt(field, X) -> list[int]:
    """Inverse transform x_n = N^{-1} sum_k X_k omega_N^{-kn}."""
    f = get_field(field)
    n = len(X)
    w_inv = inverse(f, root_of_unity(f, n))
    y = ntt_with_root(f, X, w_inv)
    n_inv = inverse(f, n % f.modulus)
    return [v * n_inv % f.modulus for v in y]


def coset_ntt(field, x, shift: int | None = None) -> list[int]:
    """Coset transform X_k = sum_n x_n (s omega_N^k)^n = forward(x_n s^n)."""
    f = get_field(field)
    s = default_coset_shift(f) if shift is None else shift % f.modulus
    scaled = []
    p = 1
    for v in x:
        scaled.append(int(v) * p % f.modulus)
        p = p * s % f.modulus
    return ntt(f, scaled)


def coset_intt(field, X, shift: int | None = None) -> list[int]:
    """Coset inverse x_n = s^{-n} N^{-1} sum_k X_k omega_N^{-kn}."""
    f = get_field(field)
    s = default_coset_shift(f) if shift is None else shift % f.modulus
    s_inv = inverse(f, s)
    y = intt(f, X)
    out = []
    p = 1
    for v in y:
        out.append(v * p % f.modulus)
        p = p * s_inv % f.modulus
    return out


def quotient_pointwise(field, a, b, c, z) -> list[int]:
    """out_i = (a_i b_i - c_i) z_(i mod len(z)) mod M, element by element.

    The prover step between the coset transforms and the coset inverse (with
    z the inverse of the vanishing polynomial on the coset points); not part
    of the paper, whose workload is the transform itself.
    """
    m = get_field(field).modulus
    L = len(z)
    return [(int(x) * int(y) - int(w)) * int(z[i % L]) % m for i, (x, y, w) in enumerate(zip(a, b, c))]


def horner(field, coeffs, z: int) -> int:
    """Evaluate sum_n coeffs[n] z^n mod M by Horner's rule."""
    f = get_field(field)
    acc = 0
    for c in reversed(list(coeffs)):
        acc = (acc * z + int(c)) % f.modulus
    return acc


def transform(field, kind: str, x, shift: int | None = None) -> list[int]:
    """kind in {'forward', 'inverse', 'coset', 'coset_inverse'}."""
    if kind == "forward":
        return ntt(field, x)
    if kind == "inverse":
        return intt(field, x)
    if kind == "coset":
        return coset_ntt(field, x, shift)
    if kind == "coset_inverse":
        return coset_intt(field, x, shift)
    raise ValueError(kind)


# ------------------------------------------------------- limb conversions


def limbs_to_ints(a: np.ndarray, words64: int = 4) -> list[int]:
    """[n, words64] uint64 little-endian limbs -> list of Python ints."""
    a = np.ascontiguousarray(a, dtype=np.uint64).reshape(-1, words64)
    out = []
    for row in a.tolist():
        v = 0
        for i, w in enumerate(row):
            v |= w << (64 * i)
        out.append(v)
    return out


def ints_to_limbs(v, words64: int = 4) -> np.ndarray:
    """list of ints in [0, 2^(64 words64)) -> [n, words64] uint64 limbs."""
    mask = (1 << 64) - 1
    rows = [[(x >> (64 * i)) & mask for i in range(words64)] for x in v]
    return np.array(rows, dtype=np.uint64).reshape(-1, words64)
