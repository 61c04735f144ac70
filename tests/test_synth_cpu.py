"""The seeded input generators (ntt_synth) every test, the benchmark and the
oracle's checks draw from: SplitMix64 against its published output
sequences, windows of the stream against the sequential stream, uniform
field elements in [0, r) by masking and rejection, and the batched
workload's size mix."""

from __future__ import annotations

import numpy as np
import pytest

import ntt_synth as S


def test_splitmix64_published_sequences():
    # seed 0: the first outputs of the reference generator (Steele, Lea and
    # Flood's SplitMix64 as published with xoshiro's seeding code)
    assert [int(v) for v in S.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # seed 1234567: the sequence the usual published test vector lists
    assert [int(v) for v in S.splitmix64(1234567, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
        16408922859458223821]


def test_splitmix64_windows_are_the_stream():
    whole = S.splitmix64(0xABCDEF, 1000)
    for start, count in ((0, 1), (1, 7), (500, 500), (999, 1)):
        assert np.array_equal(S.splitmix64(0xABCDEF, count, start=start), whole[start:start + count])
    # seeds are taken mod 2^64
    assert np.array_equal(S.splitmix64(5 + (1 << 64), 10), S.splitmix64(5, 10))


@pytest.mark.parametrize("field", S.FIELD_NAMES)
def test_uniform_elements_are_canonical_and_seeded(field):
    r = S.MODULI[field]
    W = S.words64_of(field)
    n = 3000
    x = S.uniform_elements(field, n, 77)
    assert x.shape == (n, W) and x.dtype == np.uint64
    vals = [sum(int(v) << (64 * i) for i, v in enumerate(row)) for row in x]
    assert all(0 <= v < r for v in vals)
    # the top bit of the modulus is reached (masking keeps the full range)
    assert max(vals).bit_length() == r.bit_length()
    assert len(set(vals)) == n
    assert np.array_equal(S.uniform_elements(field, n, 77), x)
    assert not np.array_equal(S.uniform_elements(field, n, 78), x)
    # a prefix of a longer draw is the shorter draw
    assert np.array_equal(S.uniform_elements(field, 2 * n, 77)[:n], x)


def test_uniform_elements_follow_the_recipe():
    # candidates are four consecutive outputs (little-endian limbs), the top
    # limb masked to the modulus's bit length, candidates >= r skipped
    field = "bn254_fr"
    r = S.MODULI[field]
    raw = S.splitmix64(9, 4 * 64).reshape(64, 4)
    want = []
    for c in raw:
        v = sum(int(w) << (64 * i) for i, w in enumerate(c)) & ((1 << r.bit_length()) - 1)
        if v < r:
            want.append(v)
    got = S.uniform_elements(field, len(want), 9)
    assert [sum(int(w) << (64 * i) for i, w in enumerate(row)) for row in got] == want
    # acceptance of BN254's 254-bit mask is r / 2^254, about 0.76
    assert 0.6 < len(want) / 64 < 0.95


def test_batch_sizes_cover_the_range_uniformly():
    sizes = S.batch_sizes(64, 14, 22, S.config_seed(4))
    assert len(sizes) == 64 and set(sizes) <= set(range(14, 23))
    assert S.batch_sizes(64, 14, 22, S.config_seed(4)) == sizes
    many = S.batch_sizes(90000, 14, 22, 1)
    counts = np.bincount(many, minlength=23)[14:]
    assert counts.min() > 9000 and counts.max() < 11000


def test_config_seeds():
    assert S.config_seed(1) == 0x5EED0001 and S.config_seed(4, 3) == 0x5EED0007
