"""Seeded synthetic inputs for the 255-bit NTT workloads.

This module is shared by the tests, the benchmark and the oracle's checks.  It
holds no transform arithmetic: only a counter-free SplitMix64 stream and
rejection sampling of field elements, so the oracle and the CUDA path see the
same bytes without sharing any of the method's code.

Recipe (uniform field elements "from seed"):
  * SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
    generators", OOPSLA 2014) seeded with ``seed``; successive outputs are
    grouped four at a time as little-endian 64-bit limbs of a candidate;
  * the top limb is masked to the modulus's bit length (255 bits for
    BLS12-381 Fr, 254 for BN254 Fr);
  * candidates >= r are rejected (acceptance ~0.91 and ~0.76), accepted ones
    are kept in order.

Workload seeds: configuration i (1-based) uses ``CONFIG_SEED_BASE + i``; job j
of a batched or served workload uses that seed plus j.
"""

from __future__ import annotations

import numpy as np

# Scalar-field moduli of the two curves (public curve definitions).
MODULI = {
    "bls12_381_fr": 0x73EDA753299D7D483339D80809A1D80553BDA402FFFE5BFEFFFFFFFF00000001,
    "bn254_fr": 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001,
    # 377- and 753-bit NTT-friendly primes (c 2^32 + 1 above pi 2^(b-2))
    "w377": 0x1921FB54442D18469898CC51701B839A252049C1114CF98E804177D4C76273644A29410F31C6809BBDF2BD500000001,
    "w753": 0x1921FB54442D18469898CC51701B839A252049C1114CF98E804177D4C76273644A29410F31C6809BBDF2A33679A748636605614DBE4BE286E9FC26ADADAA3848BC90B6AECC4BCFD8DE89885D34C6FDAD617FEB96DE80D6FDBDCD300000001,
}
FIELD_NAMES = ("bls12_381_fr", "bn254_fr", "w377", "w753")


def words64_of(field) -> int:
    """64-bit words of one element in memory: 4, 6 (377 bits) or 12 (753 bits)."""
    bits = MODULI[_field_name(field)].bit_length()
    return 4 if bits <= 256 else 6 if bits <= 384 else 12

CONFIG_SEED_BASE = 0x5EED0000

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of SplitMix64 seeded with ``seed``.

    State after k steps is seed + k * golden (mod 2^64), so any window of the
    stream is computed directly and vectorised.
    """
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _field_name(field) -> str:
    if isinstance(field, int):
        return FIELD_NAMES[field]
    return str(getattr(field, "name", field))


def uniform_elements(field, n: int, seed: int) -> np.ndarray:
    """n field elements uniform in [0, r), shape [n, W] uint64 little-endian
    (W = 4 for the 256-bit fields, 6 and 12 for the wide ones)."""
    r = MODULI[_field_name(field)]
    bits = r.bit_length()
    W = words64_of(field)
    top_mask = np.uint64((1 << (bits - 64 * (W - 1))) - 1)
    r_limbs = [np.uint64((r >> (64 * i)) & 0xFFFFFFFFFFFFFFFF) for i in range(W)]
    out = np.empty((n, W), dtype=np.uint64)
    have = 0
    pos = 0
    while have < n:
        want = max(1024, int((n - have) * 1.4) + 64)
        c = splitmix64(seed, W * want, start=pos).reshape(want, W)
        pos += W * want
        c[:, W - 1] &= top_mask
        # lexicographic c < r from the top limb down
        lt = np.zeros(want, dtype=bool)
        eq = np.ones(want, dtype=bool)
        for i in range(W - 1, -1, -1):
            lt |= eq & (c[:, i] < r_limbs[i])
            eq &= c[:, i] == r_limbs[i]
        acc = c[lt]
        take = min(n - have, acc.shape[0])
        out[have:have + take] = acc[:take]
        have += take
    return out


def config_seed(config_index: int, job: int = 0) -> int:
    """Seed of configuration ``config_index`` (1-based), job ``job``."""
    return CONFIG_SEED_BASE + config_index + job


def batch_sizes(count: int, log_min: int, log_max: int, seed: int) -> list[int]:
    """log2 sizes uniform over the integers [log_min, log_max], seeded."""
    span = log_max - log_min + 1
    z = splitmix64(seed ^ 0xB47C4, count)
    return [log_min + int(v % np.uint64(span)) for v in z]
