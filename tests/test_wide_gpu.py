"""GPU parity of the 377- and 753-bit transforms (ntt_wide_transform) with
the Python oracle: every size from 2^1 to 2^13 (one and two passes, ragged
splits) in all four kinds (forward, inverse, coset, coset inverse) element
by element, the coset kinds also with caller-chosen shifts; in place; and
at 2^16 and 2^20 the exact round trips plus outputs the oracle evaluates
one by one (Horner at omega^k and at s omega^k; the coset inverse at
omega^-n, scaled by s^-n N^-1).  The bar is bit-exact."""

from __future__ import annotations

import random

import numpy as np
import pytest

from oracle import ntt_oracle as O
from ntt_synth import uniform_elements, words64_of

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_17808_gb300 import _native as N  # noqa: E402

FIELDS = ["w377", "w753"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    N.load(build_if_missing=True)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def ints(a, field):
    return O.limbs_to_ints(a, words64_of(field))


@pytest.mark.parametrize("field", FIELDS)
def test_element_bytes(field):
    assert N.ntt_field_element_bytes(field) == 8 * words64_of(field)
    assert N.ntt_field_element_bytes("bls12_381_fr") == 32


@pytest.mark.parametrize("field", FIELDS)
def test_all_small_sizes_match_oracle(field):
    f = O.get_field(field)
    for log_n in range(1, 14):
        x = uniform_elements(field, 1 << log_n, 64000 + log_n)
        d_x = dev(x)
        d_y = torch.empty_like(d_x)
        N.ntt_wide_transform(field, "forward", log_n, d_x, d_y)
        assert ints(host(d_y), field) == O.ntt(f, ints(x, field)), ("forward", log_n)
        N.ntt_wide_transform(field, "inverse", log_n, d_x, d_y)
        assert ints(host(d_y), field) == O.intt(f, ints(x, field)), ("inverse", log_n)


@pytest.mark.parametrize("field", FIELDS)
def test_coset_kinds_all_small_sizes_match_oracle(field):
    f = O.get_field(field)
    for log_n in range(1, 14):
        x = uniform_elements(field, 1 << log_n, 64300 + log_n)
        d_x = dev(x)
        d_y = torch.empty_like(d_x)
        N.ntt_wide_transform(field, "coset", log_n, d_x, d_y)
        assert ints(host(d_y), field) == O.coset_ntt(f, ints(x, field)), ("coset", log_n)
        N.ntt_wide_transform(field, "coset_inverse", log_n, d_x, d_y)
        assert ints(host(d_y), field) == O.coset_intt(f, ints(x, field)), ("coset_inverse", log_n)
        # the plain kinds of the same size still agree after the coset tables exist
        N.ntt_wide_transform(field, "forward", log_n, d_x, d_y)
        assert ints(host(d_y), field) == O.ntt(f, ints(x, field)), ("forward after coset", log_n)


@pytest.mark.parametrize("field", FIELDS)
def test_in_place_round_trip(field):
    log_n = 14
    x = uniform_elements(field, 1 << log_n, 64100)
    d = dev(x)
    N.ntt_wide_transform(field, "forward", log_n, d, d)
    N.ntt_wide_transform(field, "inverse", log_n, d, d)
    assert np.array_equal(host(d), x)
    f = O.get_field(field)
    N.ntt_wide_transform(field, "coset", log_n, d, d)
    assert ints(host(d), field) == O.coset_ntt(f, ints(x, field))
    N.ntt_wide_transform(field, "coset_inverse", log_n, d, d)
    assert np.array_equal(host(d), x)


@pytest.mark.parametrize("field", FIELDS)
@pytest.mark.parametrize("log_n", [16, 20])
def test_large_sizes_round_trip_and_sampled_outputs(field, log_n):
    f = O.get_field(field)
    n = 1 << log_n
    x = uniform_elements(field, n, 64200 + log_n)
    d_x = dev(x)
    d_y = torch.empty_like(d_x)
    d_z = torch.empty_like(d_x)
    N.ntt_wide_transform(field, "forward", log_n, d_x, d_y)
    N.ntt_wide_transform(field, "inverse", log_n, d_y, d_z)
    assert torch.equal(d_z, d_x)
    w = O.root_of_unity(f, n)
    xs = ints(x, field)
    rng = random.Random(log_n)
    ks = [0, 1, n - 1, rng.randrange(n)]
    got = ints(host(d_y)[ks], field)
    for k, v in zip(ks, got):
        assert v == O.horner(f, xs, pow(w, k, f.modulus)), k
    # coset kinds: X_k = x(s omega^k); the coset inverse of x gives
    # s^-m N^-1 x(omega^-m) at position m, and the pair is the identity
    M = f.modulus
    s = O.default_coset_shift(f)
    N.ntt_wide_transform(field, "coset", log_n, d_x, d_y)
    N.ntt_wide_transform(field, "coset_inverse", log_n, d_y, d_z)
    assert torch.equal(d_z, d_x)
    got = ints(host(d_y)[ks], field)
    for k, v in zip(ks, got):
        assert v == O.horner(f, xs, s * pow(w, k, M) % M), ("coset", k)
    N.ntt_wide_transform(field, "coset_inverse", log_n, d_x, d_y)
    got = ints(host(d_y)[ks], field)
    n_inv, s_inv, w_inv = O.inverse(f, n), O.inverse(f, s), O.inverse(f, w)
    for m, v in zip(ks, got):
        want = O.horner(f, xs, pow(w_inv, m, M)) * n_inv % M * pow(s_inv, m, M) % M
        assert v == want, ("coset_inverse", m)


@pytest.mark.parametrize("field", FIELDS)
def test_custom_coset_shift_matches_oracle(field):
    f = O.get_field(field)
    M = f.modulus
    rng = random.Random(64400)
    shifts = [3, rng.randrange(2, M)]
    for log_n in (5, 12, 14):
        x = uniform_elements(field, 1 << log_n, 64400 + log_n)
        xs = ints(x, field)
        d_x = dev(x)
        d_y = torch.empty_like(d_x)
        for s in shifts + [shifts[0]]:   # a change of shift, and back
            N.ntt_wide_transform(field, "coset", log_n, d_x, d_y, shift=s)
            assert ints(host(d_y), field) == O.coset_ntt(f, xs, s), ("coset", log_n, s)
            N.ntt_wide_transform(field, "coset_inverse", log_n, d_x, d_y, shift=s)
            assert ints(host(d_y), field) == O.coset_intt(f, xs, s), ("coset_inverse", log_n, s)
        # the default call goes back to the generator
        N.ntt_wide_transform(field, "coset", log_n, d_x, d_y)
        assert ints(host(d_y), field) == O.coset_ntt(f, xs), ("coset, generator", log_n)
        # an explicit shift equal to the generator is the default transform
        N.ntt_wide_transform(field, "coset_inverse", log_n, d_x, d_y, shift=f.generator)
        assert ints(host(d_y), field) == O.coset_intt(f, xs), ("coset_inverse, generator", log_n)
    x = torch.zeros((32, 2 * (6 if field == "w377" else 12)), dtype=torch.int64, device="cuda")
    for bad in (0, M, M + 1):
        with pytest.raises(N.NttError) as e:
            N.ntt_wide_transform(field, "coset", 5, x, x, shift=bad)
        assert e.value.status == 1


def test_wide_argument_errors():
    x = torch.zeros((64, 12), dtype=torch.int64, device="cuda")
    with pytest.raises(N.NttError) as e:
        N.ntt_wide_transform("w753", 4, 6, x, x)
    assert e.value.status == 1
    with pytest.raises(N.NttError):
        N.ntt_wide_transform("w753", "forward", 25, x, x)
    with pytest.raises(N.NttError):
        N.ntt_wide_transform("bls12_381_fr", "forward", 6, x, x)
    with pytest.raises(N.NttError):
        N.ntt_wide_transform("w377", "forward", 6, x.data_ptr() + 8, x)
