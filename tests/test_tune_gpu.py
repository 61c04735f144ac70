"""GPU tests of the autotuner: a tuned plan still computes the exact
transform (all kinds, custom coset shift kept), the choice is remembered for
later plans of the same (field, size) and written to NTT_TUNE_CACHE."""

from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from oracle import ntt_oracle as O
from ntt_synth import uniform_elements

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_17808_gb300 import _native as N  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def test_autotune_keeps_results_exact_and_remembers_the_choice(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("NTT_TUNE_CACHE", str(cache))
    N.load(build_if_missing=True)
    field, log_n = "bls12_381_fr", 15
    f = O.get_field(field)
    s = 0x123456789 % f.modulus
    x = uniform_elements(field, 1 << log_n, 60000)
    plan = N.ntt_plan_create(field, log_n, coset=True)
    try:
        N.ntt_plan_set_coset_shift(plan, s)
        res = N.ntt_plan_autotune(plan, reps=2)
        assert res["candidates"] >= 4
        assert res["best_ms"] > 0 and res["best_ms"] <= res["default_ms"] * 1.5
        desc = N.ntt_plan_describe(plan)
        if res["path"] == "butterfly":
            assert desc["pass_log"] == res["pass_log"]
        # every table is rebuilt for the chosen split (the coset ones with the
        # custom shift): all four kinds stay exact
        for kind in ("forward", "inverse", "coset", "coset_inverse"):
            d_x = dev(x)
            d_y = torch.empty_like(d_x)
            N.ntt_execute(plan, kind, d_x, d_y)
            want = oracle.c_transform(field, kind, x, shift=s if kind.startswith("coset") else None)
            assert np.array_equal(host(d_y), want), kind
        assert N.ntt_plan_poll_error(plan) == 0
    finally:
        N.ntt_plan_destroy(plan)
    assert cache.exists() and f"|0|{log_n} " in cache.read_text()
    # a new plan of the same field and size starts from the tuned choice
    plan2 = N.ntt_plan_create(field, log_n)
    try:
        d2 = N.ntt_plan_describe(plan2)
        assert d2["path"] == {"butterfly": 1, "matrix": 2}[res["path"]]
        if res["path"] == "butterfly":
            assert d2["pass_log"] == res["pass_log"]
        d_x = dev(x)
        d_y = torch.empty_like(d_x)
        N.ntt_forward(plan2, d_x, d_y)
        assert np.array_equal(host(d_y), oracle.c_transform(field, "forward", x))
    finally:
        N.ntt_plan_destroy(plan2)


@pytest.mark.parametrize("field,log_n,split,tile", [
    ("bls12_381_fr", 13, [13 - 11, 11], 11), ("bn254_fr", 16, [4, 4, 4, 4], 10),
    ("bls12_381_fr", 17, [1, 5, 11], 10), ("bn254_fr", 15, [3, 3, 3, 3, 3], 11),
    ("bls12_381_fr", 11, [11], 11), ("bn254_fr", 12, [1] * 12, 10)])
def test_explicit_pass_split_is_exact(field, log_n, split, tile):
    """ntt_plan_set_passes: any split (here up to NTT_MAX_PASSES passes, either
    tile shape) gives the same, exact transform for all four kinds."""
    N.load(build_if_missing=True)
    x = uniform_elements(field, 1 << log_n, 60100 + log_n)
    plan = N.ntt_plan_create(field, log_n, coset=True)
    try:
        N.ntt_plan_set_passes(plan, split, tile)
        d = N.ntt_plan_describe(plan)
        assert d["pass_log"] == split and d["launches_per_transform"] == len(split)
        for kind in ("forward", "inverse", "coset", "coset_inverse"):
            d_x = dev(x)
            d_y = torch.empty_like(d_x)
            N.ntt_execute(plan, kind, d_x, d_y)
            assert np.array_equal(host(d_y), oracle.c_transform(field, kind, x)), kind
        # in place (the plan's scratch carries the passes before the last)
        d_x = dev(x)
        N.ntt_execute(plan, "forward", d_x, d_x)
        assert np.array_equal(host(d_x), oracle.c_transform(field, "forward", x))
    finally:
        N.ntt_plan_destroy(plan)


def test_explicit_pass_split_rejects_bad_splits():
    N.load(build_if_missing=True)
    plan = N.ntt_plan_create("bls12_381_fr", 14)
    try:
        for split, tile in (([7, 6], 10), ([12, 2], 11), ([7, 7], 9), ([1] * 14, 10), ([], 10)):
            with pytest.raises(N.NttError):
                N.ntt_plan_set_passes(plan, split, tile)
    finally:
        N.ntt_plan_destroy(plan)
