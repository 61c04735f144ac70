"""The NTT_DEBUG build: bounds checks in the butterfly pass kernels.

compute-sanitizer is not available for these tests, so a debug build of the
library checks every vector and table index of the pass kernels (single and
batched) against the extent the plan recorded for it; an index out of range
is reported as NTT_ERR_BOUNDS through ntt_plan_poll_error and the access is
skipped (the context stays usable).  These tests build that library, check
that it computes the same bytes as the oracle with no check firing, and make
one check fire on purpose with a host-side hook that halves the recorded
extent of the next transform: the kernels then see in-range indices as out
of range, skip those accesses and report -- no access outside a buffer is
ever made.
"""

from __future__ import annotations

import ctypes

import numpy as np
import pytest

from ntt_synth import uniform_elements

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2604_17808_gb300 import _native as N  # noqa: E402

NTT_ERR_UNSUPPORTED = 2
NTT_ERR_BOUNDS = 8


@pytest.fixture(scope="module")
def dbg():
    return N.load_debug()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def plan_of(lib, field, log_n, coset=True):
    h = ctypes.c_void_p()
    rc = lib.ntt_plan_create(ctypes.byref(h), N.FIELD[field], log_n, 1 if coset else 0)
    assert rc == 0, N.ntt_status_string(rc)
    return h.value


def poll(lib, plan):
    code = ctypes.c_uint32(99)
    assert lib.ntt_plan_poll_error(plan, ctypes.byref(code)) == 0
    return code.value


def test_release_build_has_no_debug_hooks():
    lib = N.load(build_if_missing=True)
    assert lib.ntt_build_is_debug() == 0
    plan = N.ntt_plan_create("bn254_fr", 10)
    try:
        assert lib.ntt_debug_shrink_next_extent(plan) == NTT_ERR_UNSUPPORTED
    finally:
        N.ntt_plan_destroy(plan)


@pytest.mark.parametrize("field", ["bls12_381_fr", "bn254_fr"])
def test_debug_build_is_exact_and_quiet(dbg, field):
    assert dbg.ntt_build_is_debug() == 1
    for log_n in (1, 3, 9, 12, 17):
        plan = plan_of(dbg, field, log_n)
        try:
            x = uniform_elements(field, 1 << log_n, 64000 + log_n)
            for kind in ("forward", "inverse", "coset", "coset_inverse"):
                d_x = dev(x)
                d_y = torch.empty_like(d_x)
                assert dbg.ntt_execute(plan, N.KIND[kind], d_x.data_ptr(), d_y.data_ptr(), None) == 0
                assert np.array_equal(host(d_y), oracle.c_transform(field, kind, x)), (log_n, kind)
            assert poll(dbg, plan) == 0
        finally:
            dbg.ntt_plan_destroy(plan)


def test_debug_build_batch_is_exact_and_quiet(dbg):
    specs = [("bls12_381_fr", 14), ("bn254_fr", 11), ("bls12_381_fr", 5)]
    plans = [plan_of(dbg, f, ln, coset=False) for f, ln in specs]
    try:
        xs = [uniform_elements(f, 1 << ln, 65000 + i) for i, (f, ln) in enumerate(specs)]
        ins = [dev(x) for x in xs]
        outs = [torch.empty_like(t) for t in ins]
        arr = (N.Job * len(specs))()
        for i, (p, a, b) in enumerate(zip(plans, ins, outs)):
            arr[i] = N.Job(p, N.KIND["forward"], a.data_ptr(), b.data_ptr())
        assert dbg.ntt_batch_submit(arr, len(specs), None) == 0
        for (f, _), x, y in zip(specs, xs, outs):
            assert np.array_equal(host(y), oracle.c_transform(f, "forward", x))
        assert all(poll(dbg, p) == 0 for p in plans)
    finally:
        dbg.ntt_batch_cache_clear()
        for p in plans:
            dbg.ntt_plan_destroy(p)


@pytest.mark.parametrize("log_n", [10, 16])
def test_debug_bounds_check_fires_and_context_survives(dbg, log_n):
    field = "bls12_381_fr"
    plan = plan_of(dbg, field, log_n)
    try:
        x = uniform_elements(field, 1 << log_n, 66000 + log_n)
        d_x = dev(x)
        d_y = torch.zeros_like(d_x)
        assert poll(dbg, plan) == 0
        assert dbg.ntt_debug_shrink_next_extent(plan) == 0
        assert dbg.ntt_execute(plan, N.KIND["forward"], d_x.data_ptr(), d_y.data_ptr(), None) == 0
        assert poll(dbg, plan) == NTT_ERR_BOUNDS
        assert poll(dbg, plan) == 0   # cleared by the read
        # the context is intact: the next transform is exact and quiet
        assert dbg.ntt_execute(plan, N.KIND["forward"], d_x.data_ptr(), d_y.data_ptr(), None) == 0
        assert np.array_equal(host(d_y), oracle.c_transform(field, "forward", x))
        assert poll(dbg, plan) == 0
    finally:
        dbg.ntt_plan_destroy(plan)
