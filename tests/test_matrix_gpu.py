"""GPU parity of the matrix-form path (every pass a tcgen05 tensor-core
product of signed-byte digits with a precomputed byte matrix, then ByteMerge
and Montgomery reduction) against the oracle, and path equivalence with the
butterfly path (byte-identical outputs)."""

from __future__ import annotations

import hashlib
import json
import os

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def matrix_plan(field, log_n, coset=True):
    plan = N.ntt_plan_create(field, log_n, coset=coset)
    N.ntt_plan_set_path(plan, "matrix")
    return plan


@pytest.mark.parametrize("field", FIELDS)
def test_matrix_path_all_small_sizes_and_kinds(field):
    for log_n in range(1, 15):
        plan = matrix_plan(field, log_n)
        try:
            desc = N.ntt_plan_describe(plan)
            assert desc["path"] == 2 and desc["launches_per_transform"] == -(-log_n // 3)
            # the described split is the matrix path's own: passes of <= 2^3 points
            assert len(desc["pass_log"]) == desc["num_passes"] == -(-log_n // 3)
            assert sum(desc["pass_log"]) == log_n and max(desc["pass_log"]) <= 3
            for kind in KINDS:
                x = uniform_elements(field, 1 << log_n, 40000 + log_n)
                d_x = dev(x)
                d_y = torch.empty_like(d_x)
                N.ntt_execute(plan, kind, d_x, d_y)
                assert np.array_equal(host(d_y), oracle.c_transform(field, kind, x)), (field, kind, log_n)
            assert N.ntt_plan_poll_error(plan) == 0
        finally:
            N.ntt_plan_destroy(plan)


@pytest.mark.parametrize("field", FIELDS)
def test_matrix_path_adversarial_inputs(field):
    # all p-1 and alternating maximal / zero limbs: the signed digits hit
    # their extremes and every ByteMerge carry path is exercised
    f = O.get_field(field)
    log_n = 12
    n = 1 << log_n
    vals = [f.modulus - 1] * (n // 2) + [(f.modulus - 1) if i % 3 else 0 for i in range(n // 2)]
    x = O.ints_to_limbs(vals)
    plan = matrix_plan(field, log_n)
    try:
        for kind in KINDS:
            d_x = dev(x)
            d_y = torch.empty_like(d_x)
            N.ntt_execute(plan, kind, d_x, d_y)
            assert np.array_equal(host(d_y), oracle.c_transform(field, kind, x)), kind
    finally:
        N.ntt_plan_destroy(plan)


# Folded passes: pass j >= 1 (not the last) is folded when each q has at
# least 2^11 rows, i.e. log_n >= (points of passes 0..j, log2) + 11.  With
# passes of 2^3 points: 2^17 and 2^18 fold pass 1, 2^20 passes 1-2, 2^24
# passes 1-3.
FOLDED = {17: 1, 18: 1, 20: 2, 24: 3}


@pytest.mark.parametrize("field", FIELDS)
@pytest.mark.parametrize("log_n", [17, 18, 20])
def test_matrix_folded_passes_all_kinds(field, log_n):
    # every kind, element by element against the oracle, at sizes whose
    # early passes carry their factors in per-q matrices E_q (four CTAs of
    # a group on neighbouring q; pass 0 and the folded passes before the
    # last one end in Barrett)
    plan = matrix_plan(field, log_n)
    try:
        desc = N.ntt_plan_describe(plan)
        assert desc["matrix_folded_passes"] == FOLDED[log_n]
        x = uniform_elements(field, 1 << log_n, 47000 + log_n)
        d_x = dev(x)
        for kind in KINDS:
            d_y = torch.empty_like(d_x)
            N.ntt_execute(plan, kind, d_x, d_y)
            assert np.array_equal(host(d_y), oracle.c_transform(field, kind, x)), (field, log_n, kind)
        assert N.ntt_plan_poll_error(plan) == 0
    finally:
        N.ntt_plan_destroy(plan)


@pytest.mark.parametrize("field", FIELDS)
@pytest.mark.parametrize("log_n", [21, 22])
def test_matrix_folded_coset_kinds_larger(field, log_n):
    # passes of 2^3 and (2^22) 2^2 points, two folded; the coset forward
    # (coset powers in the pass-0 matrix, coset inverse's s^-n in the last
    # epilogue) element by element against the oracle (its all-cores mode,
    # which the CPU tests pin to the serial loop)
    plan = matrix_plan(field, log_n)
    threads = oracle.c_set_threads(0)
    try:
        desc = N.ntt_plan_describe(plan)
        assert desc["matrix_folded_passes"] == 2 and sum(desc["pass_log"]) == log_n
        x = uniform_elements(field, 1 << log_n, 47200 + log_n)
        d_x = dev(x)
        for kind in ("coset", "coset_inverse"):
            d_y = torch.empty_like(d_x)
            N.ntt_execute(plan, kind, d_x, d_y)
            assert np.array_equal(host(d_y), oracle.c_transform(field, kind, x)), (field, log_n, kind, threads)
        assert N.ntt_plan_poll_error(plan) == 0
    finally:
        oracle.c_set_threads(1)
        N.ntt_plan_destroy(plan)


def test_matrix_path_2_26_four_folded_passes():
    # 2^26 (2 GiB per vector): passes 1-4 folded (pass 4 with 4096 matrices
    # E_q); the forward output equals the butterfly path's byte for byte and
    # the inverse gives the input back
    field, log_n = "bls12_381_fr", 26
    plan = N.ntt_plan_create(field, log_n, coset=False)
    try:
        x = torch.from_numpy(np.tile(uniform_elements(field, 1 << 20, 47300), (1 << 6, 1)).view(np.int64)).cuda()
        yb = torch.empty_like(x)
        N.ntt_execute(plan, "forward", x, yb)
        N.ntt_plan_set_path(plan, "matrix")
        assert N.ntt_plan_describe(plan)["matrix_folded_passes"] == 4
        ym = torch.empty_like(x)
        N.ntt_execute(plan, "forward", x, ym)
        assert torch.equal(ym, yb)
        del yb
        N.ntt_execute(plan, "inverse", ym, ym)
        assert torch.equal(ym, x)
        assert N.ntt_plan_poll_error(plan) == 0
    finally:
        N.ntt_plan_destroy(plan)


def test_matrix_folded_custom_shift_in_place():
    # a new coset shift rebuilds the folded coset matrices; in-place calls
    # run the folded passes on the plan's scratch
    field, log_n = "bls12_381_fr", 17
    f = O.get_field(field)
    s = 0x1234567890ABCDEF1357 % f.modulus
    x = uniform_elements(field, 1 << log_n, 47100)
    plan = matrix_plan(field, log_n)
    try:
        assert N.ntt_plan_describe(plan)["matrix_folded_passes"] == 1
        N.ntt_plan_set_coset_shift(plan, s)
        for kind in ("coset", "coset_inverse", "forward"):
            d = dev(x)
            N.ntt_execute(plan, kind, d, d)
            assert np.array_equal(host(d), oracle.c_transform(field, kind, x, shift=s)), kind
        assert N.ntt_plan_poll_error(plan) == 0
    finally:
        N.ntt_plan_destroy(plan)


@pytest.mark.parametrize("kind", ["forward", "inverse"])
def test_matrix_equals_butterfly_and_oracle_at_2_20(kind):
    field, log_n = "bls12_381_fr", 20
    x = uniform_elements(field, 1 << log_n, config_seed(2))
    with open(os.path.join(HERE, "golden", "oracle_digests.json")) as fh:
        want = [c for c in json.load(fh)["single"] if c["config"] == 2 and c["kind"] == kind][0]["output_sha256"]
    plan = N.ntt_plan_create(field, log_n)
    try:
        d_x = dev(x)
        d_b = torch.empty_like(d_x)
        d_m = torch.empty_like(d_x)
        N.ntt_execute(plan, kind, d_x, d_b)
        N.ntt_plan_set_path(plan, "matrix")
        N.ntt_execute(plan, kind, d_x, d_m)
        assert torch.equal(d_b, d_m)
        got = host(d_m)
        assert hashlib.sha256(got.astype("<u8").tobytes()).hexdigest() == want
        assert N.ntt_plan_poll_error(plan) == 0
    finally:
        N.ntt_plan_destroy(plan)


def test_matrix_path_bn254_2_24_coset_matches_oracle_digest():
    # the BN254 2^24 coset workload (shift 5) on the tensor-core path: eight
    # passes of 8-point sub-transforms; stored oracle digest of the output
    field, log_n = "bn254_fr", 24
    x = uniform_elements(field, 1 << log_n, config_seed(3))
    with open(os.path.join(HERE, "golden", "oracle_digests.json")) as fh:
        want = [c for c in json.load(fh)["single"] if c["config"] == 3 and c["kind"] == "coset"][0]
    assert hashlib.sha256(x.astype("<u8").tobytes()).hexdigest() == want["input_sha256"]
    plan = matrix_plan(field, log_n)
    try:
        d_x = dev(x)
        d_y = torch.empty_like(d_x)
        N.ntt_execute(plan, "coset", d_x, d_y)
        got = host(d_y)
        assert N.ntt_plan_poll_error(plan) == 0
    finally:
        N.ntt_plan_destroy(plan)
    assert hashlib.sha256(got.astype("<u8").tobytes()).hexdigest() == want["output_sha256"]


@pytest.mark.parametrize("path", ["butterfly", "matrix"])
def test_bn254_2_24_coset_inverse_matches_oracle_digest(path):
    # the coset inverse of the BN254 2^24 workload vector (s^-n applied to the
    # last pass's outputs; on the matrix path by the last epilogue's
    # Montgomery product), whole output against the stored oracle digest
    field, log_n = "bn254_fr", 24
    x = uniform_elements(field, 1 << log_n, config_seed(3))
    with open(os.path.join(HERE, "golden", "oracle_digests.json")) as fh:
        want = [c for c in json.load(fh)["single"]
                if c["config"] == 3 and c["kind"] == "coset_inverse" and c["field"] == field][0]
    assert hashlib.sha256(x.astype("<u8").tobytes()).hexdigest() == want["input_sha256"]
    plan = N.ntt_plan_create(field, log_n, coset=True)
    try:
        N.ntt_plan_set_path(plan, path)
        d_x = dev(x)
        d_y = torch.empty_like(d_x)
        N.ntt_execute(plan, "coset_inverse", d_x, d_y)
        got = host(d_y)
        assert N.ntt_plan_poll_error(plan) == 0
    finally:
        N.ntt_plan_destroy(plan)
    assert hashlib.sha256(got.astype("<u8").tobytes()).hexdigest() == want["output_sha256"]


@pytest.mark.parametrize("kind", ["forward", "inverse"])
def test_matrix_path_bls12_381_2_24_matches_oracle_digest(kind):
    # the 2^24-point BLS12-381 transform on the tensor-core path, whole output
    # against the stored oracle digest
    field, log_n = "bls12_381_fr", 24
    x = uniform_elements(field, 1 << log_n, config_seed(3, 100))
    with open(os.path.join(HERE, "golden", "oracle_digests.json")) as fh:
        want = [c for c in json.load(fh)["single"]
                if c["config"] == 3 and c["kind"] == kind and c["field"] == field][0]
    assert hashlib.sha256(x.astype("<u8").tobytes()).hexdigest() == want["input_sha256"]
    plan = matrix_plan(field, log_n, coset=False)
    try:
        assert N.ntt_plan_describe(plan)["matrix_folded_passes"] == FOLDED[24]
        d_x = dev(x)
        d_y = torch.empty_like(d_x)
        N.ntt_execute(plan, kind, d_x, d_y)
        got = host(d_y)
        assert N.ntt_plan_poll_error(plan) == 0
    finally:
        N.ntt_plan_destroy(plan)
    assert hashlib.sha256(got.astype("<u8").tobytes()).hexdigest() == want["output_sha256"]


def test_matrix_path_in_place_and_custom_shift():
    field, log_n = "bn254_fr", 13
    f = O.get_field(field)
    s = 0xDEADBEEF12345678 % f.modulus
    x = uniform_elements(field, 1 << log_n, 41000)
    plan = matrix_plan(field, log_n)
    try:
        N.ntt_plan_set_coset_shift(plan, s)
        d = dev(x)
        N.ntt_execute(plan, "coset", d, d)
        assert np.array_equal(host(d), oracle.c_transform(field, "coset", x, shift=s))
        d = dev(x)
        N.ntt_execute(plan, "coset_inverse", d, d)
        assert np.array_equal(host(d), oracle.c_transform(field, "coset_inverse", x, shift=s))
    finally:
        N.ntt_plan_destroy(plan)
