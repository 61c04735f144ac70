"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Bar: bit-exact.  All arithmetic is exact modular arithmetic with canonical
outputs, so the result is unique and the tolerance is zero.

Sizes: every log_n from 1 to 18 for both fields and all four kinds (one,
two and three passes, ragged pass splits, tiles that are only partly
filled), the full sizes of the workloads (2^12, 2^20 BLS12-381 forward and
inverse, 2^24 BN254 coset, 2^24 BLS12-381 forward) against stored oracle
digests, live oracle runs and sampled outputs the oracle evaluates one by
one (Horner at s * omega^k).
"""

from __future__ import annotations

import hashlib
import json
import os
import random

import numpy as np
import pytest

import oracle
from oracle import ntt_oracle as O
from ntt_synth import config_seed, uniform_elements

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_17808_gb300 import _native as N  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
FIELDS = ["bls12_381_fr", "bn254_fr"]
KINDS = ["forward", "inverse", "coset", "coset_inverse"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    N.load(build_if_missing=True)


def dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def host(t) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(a.astype("<u8").tobytes()).hexdigest()


def golden():
    with open(os.path.join(HERE, "golden", "oracle_digests.json")) as fh:
        return json.load(fh)


def gpu_transform(field, kind, x, log_n=None, plan=None, inplace=False):
    own = plan is None
    if own:
        plan = N.ntt_plan_create(field, log_n, coset=kind in ("coset", "coset_inverse"))
    try:
        d_in = dev(x)
        d_out = d_in if inplace else torch.empty_like(d_in)
        N.ntt_execute(plan, kind, d_in, d_out)
        return host(d_out)
    finally:
        if own:
            N.ntt_plan_destroy(plan)


# ------------------------------------------------------------ field level


@pytest.mark.parametrize("field", FIELDS)
def test_field_mont_mul_edge_operands(field):
    f = O.get_field(field)
    p = f.modulus
    edge = [0, 1, 2, 3, p - 1, p - 2, (p - 1) // 2, (p + 1) // 2, 2**32 - 1, 2**32, 2**64 - 1, 2**128 + 1,
            2**192 - 1, 2**254 % p, (2**255 - 1) % p, 7, 5]
    rng = random.Random(11)
    edge += [rng.randrange(p) for _ in range(15)]
    a = [x for x in edge for _ in edge]
    b = [y for _ in edge for y in edge]
    rinv = pow(2**256, -1, p)
    d_a, d_b = dev(O.ints_to_limbs(a)), dev(O.ints_to_limbs(b))
    d_c = torch.empty_like(d_a)
    N.ntt_field_mont_mul(field, d_a, d_b, d_c, len(a))
    got = O.limbs_to_ints(host(d_c))
    want = [x * y * rinv % p for x, y in zip(a, b)]
    assert got == want


@pytest.mark.parametrize("field", FIELDS)
def test_field_mont_mul_variants_agree_with_python(field):
    # per-thread carry chains (0) and 8-lane warp-shuffle carries (1)
    f = O.get_field(field)
    p = f.modulus
    rng = random.Random(12)
    a = [0, 1, p - 1, p - 2, 2**32 - 1, 2**224 + 5, (p + 1) // 2] + [rng.randrange(p) for _ in range(249)]
    b = [p - 1, 1, p - 1, 2**64 + 1, 0, 3, (p - 1) // 2] + [rng.randrange(p) for _ in range(249)]
    rinv = pow(2**256, -1, p)
    d_a, d_b = dev(O.ints_to_limbs(a)), dev(O.ints_to_limbs(b))
    for reps in (1, 2, 7):
        want = [x * pow(y * rinv % p, reps, p) % p for x, y in zip(a, b)]
        for variant in (0, 1):
            d_c = torch.empty_like(d_a)
            N.ntt_field_mont_mul_rep(field, d_a, d_b, d_c, len(a), reps, variant)
            assert O.limbs_to_ints(host(d_c)) == want, (reps, variant)


# ------------------------------------------------------ all small sizes


@pytest.mark.parametrize("field", FIELDS)
@pytest.mark.parametrize("kind", KINDS)
def test_small_and_medium_sizes_match_oracle(field, kind):
    for log_n in range(1, 19):
        x = uniform_elements(field, 1 << log_n, 9000 + log_n)
        want = oracle.c_transform(field, kind, x)
        got = gpu_transform(field, kind, x, log_n)
        assert np.array_equal(got, want), (field, kind, log_n)


@pytest.mark.parametrize("field", FIELDS)
@pytest.mark.parametrize("log_n", [3, 8, 9, 16, 17])
def test_in_place_matches_oracle(field, log_n):
    x = uniform_elements(field, 1 << log_n, 9100 + log_n)
    plan = N.ntt_plan_create(field, log_n, coset=True)
    try:
        for kind in KINDS:
            want = oracle.c_transform(field, kind, x)
            assert np.array_equal(gpu_transform(field, kind, x, plan=plan, inplace=True), want), (kind, log_n)
    finally:
        N.ntt_plan_destroy(plan)


@pytest.mark.parametrize("field", FIELDS)
def test_special_vectors(field):
    log_n = 14
    n = 1 << log_n
    f = O.get_field(field)
    w = O.root_of_unity(f, n)
    delta1 = np.zeros((n, 4), dtype=np.uint64)
    delta1[1, 0] = 1
    got = O.limbs_to_ints(gpu_transform(field, "forward", delta1, log_n))
    pw = 1
    for k in range(n):
        assert got[k] == pw
        pw = pw * w % f.modulus
    ones = O.ints_to_limbs([1] * n)
    got = O.limbs_to_ints(gpu_transform(field, "forward", ones, log_n))
    assert got[0] == n and not any(got[1:])
    zeros = np.zeros((n, 4), dtype=np.uint64)
    assert not gpu_transform(field, "inverse", zeros, log_n).any()
    top = O.ints_to_limbs([f.modulus - 1] * n)  # all p - 1: every add/sub wraps
    assert np.array_equal(gpu_transform(field, "forward", top, log_n), oracle.c_transform(field, "forward", top))


@pytest.mark.parametrize("field", FIELDS)
def test_custom_coset_shift(field):
    f = O.get_field(field)
    log_n = 12
    x = uniform_elements(field, 1 << log_n, 9200)
    s = 0x1234567890ABCDEF1234567890ABCDEF % f.modulus
    plan = N.ntt_plan_create(field, log_n, coset=True)
    try:
        N.ntt_plan_set_coset_shift(plan, s)
        got = gpu_transform(field, "coset", x, plan=plan)
        back = gpu_transform(field, "coset_inverse", x, plan=plan)
    finally:
        N.ntt_plan_destroy(plan)
    assert np.array_equal(got, oracle.c_transform(field, "coset", x, shift=s))
    assert np.array_equal(back, oracle.c_transform(field, "coset_inverse", x, shift=s))


# ------------------------------------------------------------ tables


@pytest.mark.parametrize("field", FIELDS)
def test_device_twiddle_tables_match_oracle_roots(field):
    f = O.get_field(field)
    p = f.modulus
    log_n = 20
    plan = N.ntt_plan_create(field, log_n, coset=True)
    try:
        desc = N.ntt_plan_describe(plan)
        logs = desc["pass_log"]
        assert sum(logs) == log_n
        w_n = O.root_of_unity(f, 1 << log_n)
        for j, ls in enumerate(logs):
            S = 1 << ls
            for kind, sign in (("forward", 1), ("inverse", -1)):
                buf = np.zeros((S // 2, 4), dtype=np.uint64)
                N.ntt_plan_read_table(plan, kind, j, 0, 0, S // 2, buf)
                w_s = pow(O.root_of_unity(f, S), sign, p)
                assert O.limbs_to_ints(buf) == [pow(w_s, i, p) for i in range(S // 2)]
        # inter-pass table of pass 1: omega_M^(n q), row-major [n][q]
        log_mp = logs[0]
        log_m = logs[0] + logs[1]
        w_m = O.root_of_unity(f, 1 << log_m)
        count = 1 << log_m
        buf = np.zeros((count, 4), dtype=np.uint64)
        N.ntt_plan_read_table(plan, "forward", 1, 1, 0, count, buf)
        got = O.limbs_to_ints(buf)
        for idx in list(range(0, count, 37)) + [count - 1]:
            n, q = idx >> log_mp, idx & ((1 << log_mp) - 1)
            assert got[idx] == pow(w_m, n * q, p)
        # coset pass-0 multipliers: s^(n N / S_0)
        S0 = 1 << logs[0]
        buf = np.zeros((S0, 4), dtype=np.uint64)
        N.ntt_plan_read_table(plan, "coset", 0, 1, 0, S0, buf)
        s = O.default_coset_shift(f)
        step = pow(s, (1 << log_n) // S0, p)
        assert O.limbs_to_ints(buf) == [pow(step, i, p) for i in range(S0)]
        # coset inverse output multipliers of the last pass: s^-n
        count = 1 << log_n
        buf = np.zeros((count, 4), dtype=np.uint64)
        N.ntt_plan_read_table(plan, "coset_inverse", len(logs) - 1, 2, 0, count, buf)
        got = O.limbs_to_ints(buf)
        s_inv = pow(s, p - 2, p)
        for n in list(range(0, count, 4099)) + [1, count - 1]:
            assert got[n] == pow(s_inv, n, p)
    finally:
        N.ntt_plan_destroy(plan)


# ------------------------------------------------------- workload sizes


def _golden_case(config, kind, field=None):
    for c in golden()["single"]:
        if c["config"] == config and c["kind"] == kind and (field is None or c["field"] == field):
            return c
    raise KeyError((config, kind, field))


@pytest.mark.parametrize("kind", ["forward", "inverse"])
def test_bls12_381_2_12_matches_oracle_and_digest(kind):
    field, log_n = "bls12_381_fr", 12
    x = uniform_elements(field, 1 << log_n, config_seed(1))
    g = _golden_case(1, kind)
    assert digest(x) == g["input_sha256"]
    got = gpu_transform(field, kind, x, log_n)
    assert digest(got) == g["output_sha256"]
    assert np.array_equal(got, oracle.c_transform(field, kind, x))


@pytest.mark.parametrize("kind", ["forward", "inverse"])
def test_bls12_381_2_20_matches_oracle_and_digest(kind):
    field, log_n = "bls12_381_fr", 20
    x = uniform_elements(field, 1 << log_n, config_seed(2))
    g = _golden_case(2, kind)
    assert digest(x) == g["input_sha256"]
    got = gpu_transform(field, kind, x, log_n)
    assert digest(got) == g["output_sha256"]
    assert np.array_equal(got, oracle.c_transform(field, kind, x))


def _horner_spot_checks(field, x, got, kind, shift=None, samples=3, seed=0):
    f = O.get_field(field)
    p = f.modulus
    n = x.shape[0]
    w = O.root_of_unity(f, n)
    s = (O.default_coset_shift(f) if shift is None else shift) if kind == "coset" else 1
    rng = random.Random(seed)
    ks = [0, n - 1] + [rng.randrange(n) for _ in range(samples)]
    out = O.limbs_to_ints(got[ks])
    for k, v in zip(ks, out):
        z = s * pow(w, k, p) % p
        assert v == oracle.c_eval(field, x, z), k


def test_bn254_2_24_coset_matches_digest_and_sampled_outputs():
    field, log_n = "bn254_fr", 24
    x = uniform_elements(field, 1 << log_n, config_seed(3))
    g = _golden_case(3, "coset")
    assert digest(x) == g["input_sha256"]
    plan = N.ntt_plan_create(field, log_n, coset=True)
    try:
        got = gpu_transform(field, "coset", x, plan=plan)
        back = gpu_transform(field, "coset_inverse", got, plan=plan)
    finally:
        N.ntt_plan_destroy(plan)
    assert digest(got) == g["output_sha256"]
    assert np.array_equal(back, x)   # the coset inverse undoes the coset transform
    _horner_spot_checks(field, x, got, "coset", samples=2, seed=3)


def test_bls12_381_2_24_forward_and_inverse_match_oracle_digests():
    """The 2^24-point BLS12-381 transform, compared in full: forward and
    inverse outputs against the stored C-oracle digests, the round trip, and
    sampled outputs evaluated one by one (Horner at omega^k)."""
    field, log_n = "bls12_381_fr", 24
    x = uniform_elements(field, 1 << log_n, config_seed(3, 100))
    gf = _golden_case(3, "forward", field)
    gi = _golden_case(3, "inverse", field)
    assert digest(x) == gf["input_sha256"] == gi["input_sha256"]
    plan = N.ntt_plan_create(field, log_n)
    try:
        d_x = dev(x)
        d_y = torch.empty_like(d_x)
        d_z = torch.empty_like(d_x)
        N.ntt_forward(plan, d_x, d_y)
        N.ntt_inverse(plan, d_y, d_z)
        y = host(d_y)
        assert torch.equal(d_z, d_x)
        N.ntt_inverse(plan, d_x, d_z)
        z = host(d_z)
    finally:
        N.ntt_plan_destroy(plan)
    assert digest(y) == gf["output_sha256"]
    assert digest(z) == gi["output_sha256"]
    _horner_spot_checks(field, x, y, "forward", samples=2, seed=4)


def test_maximum_size_2_28_round_trip_and_sampled_outputs():
    # 2^28 points (BN254 Fr's 2-adicity, the largest size the library takes):
    # 8 GiB per vector.  Checked by the round trip and by sampled outputs the
    # oracle evaluates one by one (a full oracle transform of this size takes
    # minutes on one core and is not stored).
    field, log_n = "bn254_fr", 28
    n = 1 << log_n
    x = uniform_elements(field, n, 0x5EED0100)
    plan = N.ntt_plan_create(field, log_n)
    try:
        d_x = dev(x)
        d_y = torch.empty_like(d_x)
        N.ntt_forward(plan, d_x, d_y)
        N.ntt_inverse(plan, d_y, d_y)  # in place
        torch.cuda.synchronize()
        assert torch.equal(d_y, d_x)
        N.ntt_forward(plan, d_x, d_y)
        f = O.get_field(field)
        w = O.root_of_unity(f, n)
        ks = [1, n - 1, 0x1234567]
        got = O.limbs_to_ints(d_y[ks].cpu().numpy().view(np.uint64))
        for k, v in zip(ks, got):
            assert v == oracle.c_eval(field, x, pow(w, k, f.modulus)), k
    finally:
        N.ntt_plan_destroy(plan)


# ------------------------------------------------------------ boundary


def test_transform_host_round_trip():
    field, log_n = "bls12_381_fr", 16
    x = uniform_elements(field, 1 << log_n, 9300)
    plan = N.ntt_plan_create(field, log_n)
    try:
        h_in = torch.from_numpy(x.view(np.int64)).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        d_work = torch.empty(h_in.shape, dtype=torch.int64, device="cuda")
        N.ntt_transform_host(plan, "forward", h_in, h_out, d_work)
        want = oracle.c_transform(field, "forward", x)
        assert np.array_equal(h_out.numpy().view(np.uint64), want)
        # asynchronous form on a side stream
        h_out2 = torch.zeros_like(h_in).pin_memory()
        s = torch.cuda.Stream()
        N.ntt_transform_host_async(plan, "forward", h_in, h_out2, d_work, s)
        s.synchronize()
        assert np.array_equal(h_out2.numpy().view(np.uint64), want)
    finally:
        N.ntt_plan_destroy(plan)


def test_argument_errors_are_reported():
    plan = N.ntt_plan_create("bn254_fr", 10)
    try:
        buf = torch.zeros((1 << 10, 4), dtype=torch.int64, device="cuda")
        with pytest.raises(N.NttError) as e:
            N.ntt_coset_forward(plan, buf, buf)  # plan built without coset tables
        assert e.value.status == 1
        with pytest.raises(N.NttError):
            N.ntt_coset_inverse(plan, buf, buf)
        lib = N.load()
        assert lib.ntt_forward(plan, None, buf.data_ptr(), None) == 1
        assert lib.ntt_forward(plan, buf.data_ptr() + 8, buf.data_ptr(), None) == 1  # misaligned
        # 16-byte but not 32-byte aligned: every element moves as one 256-bit
        # access, so buffers must be 32-byte aligned
        assert lib.ntt_forward(plan, buf.data_ptr() + 16, buf.data_ptr(), None) == 1
        assert lib.ntt_execute(plan, 9, buf.data_ptr(), buf.data_ptr(), None) == 1
        assert lib.ntt_plan_set_coset_shift(plan, None) == 1
        assert N.ntt_plan_poll_error(plan) == 0
    finally:
        N.ntt_plan_destroy(plan)
