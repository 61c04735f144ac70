"""The allocation-free batched entry point (ntt_batch_submit_static).

Callers that cannot allocate device memory while they submit work -- a
service that reserved all its memory up front, or a submitter on a latency
path where cudaMalloc's implicit synchronisation would stall other streams --
use this entry point: it runs the same batched kernel with its work-item
table and counters in a fixed array the library keeps in device memory.

These tests call it through the C ABI and check its outputs against the
regular entry point (ntt_batch_submit) and against the CPU oracle, on two
calls in a row with different data; the bar is bit-exact, like every other
parity test here.  Further cases: plans split into five and six passes, an
empty job list, a call without a status pointer (errors then reach
ntt_batch_poll_error), and a forced device-wait timeout (host-side stall
hook, 5 ms wait limit) after which the next call runs normally.  The file is
named so that pytest collects it last.
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
NTT_ERR_TIMEOUT = 5


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint64)


def job_array(jobs):
    arr = (N.Job * max(1, len(jobs)))()
    for i, (plan, kind, x, y) in enumerate(jobs):
        arr[i] = N.Job(plan, N.KIND[kind], x.data_ptr(), y.data_ptr())
    return arr


def submit_static(lib, jobs, status):
    ptr = ctypes.c_void_p(status.data_ptr()) if status is not None else None
    return lib.ntt_batch_submit_static(job_array(jobs), len(jobs), ptr, None)


def test_static_batch_matches_regular_batch_and_oracle_on_two_calls():
    lib = N.load(build_if_missing=True)
    specs = [("bls12_381_fr", 14, "forward"), ("bls12_381_fr", 17, "inverse"), ("bn254_fr", 12, "coset"),
             ("bn254_fr", 20, "forward"), ("bls12_381_fr", 9, "coset"), ("bn254_fr", 16, "inverse")]
    plans = {(f, ln): N.ntt_plan_create(f, ln, coset=True) for f, ln, _ in specs}
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    try:
        for call in range(2):
            hx = [uniform_elements(f, 1 << ln, 50000 + 100 * call + i) for i, (f, ln, _) in enumerate(specs)]
            ins = [dev(x) for x in hx]
            ref = [torch.empty_like(x) for x in ins]
            got = [torch.full_like(x, -1) for x in ins]
            N.ntt_batch_submit([(plans[(f, ln)], k, x, y) for (f, ln, k), x, y in zip(specs, ins, ref)])
            rc = submit_static(lib, [(plans[(f, ln)], k, x, y) for (f, ln, k), x, y in zip(specs, ins, got)],
                               status)
            assert rc == 0, N.ntt_status_string(rc)
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            for i, (r, g) in enumerate(zip(ref, got)):
                assert torch.equal(r, g), (call, specs[i])
            for i, ((f, ln, k), x, g) in enumerate(zip(specs, hx, got)):
                assert np.array_equal(host(g), oracle.c_transform(f, k, x)), (call, specs[i])
        # beyond the maximum: a clear error, nothing launched
        too_many = (N.Job * 65)()
        assert lib.ntt_batch_submit_static(too_many, 65, None, None) == NTT_ERR_UNSUPPORTED
    finally:
        N.ntt_batch_cache_clear()
        for p in plans.values():
            N.ntt_plan_destroy(p)


def test_static_batch_with_five_and_six_pass_plans():
    """Plans split into more passes than the default (set by the caller, as
    the autotuner may), bit-exact with the regular batch and the oracle."""
    lib = N.load(build_if_missing=True)
    cases = [("bls12_381_fr", 20, [4, 4, 4, 4, 4], "forward"), ("bn254_fr", 18, [3, 3, 3, 3, 3, 3], "inverse"),
             ("bls12_381_fr", 12, [2, 2, 2, 2, 2, 2], "coset")]
    plans = []
    status = torch.full((1,), 777, dtype=torch.int32, device="cuda")
    try:
        for f, ln, split, _ in cases:
            p = N.ntt_plan_create(f, ln, coset=True)
            N.ntt_plan_set_passes(p, split, 10)
            assert N.ntt_plan_describe(p)["pass_log"] == split
            plans.append(p)
        hx = [uniform_elements(f, 1 << ln, 61000 + i) for i, (f, ln, _, _) in enumerate(cases)]
        ins = [dev(x) for x in hx]
        ref = [torch.empty_like(x) for x in ins]
        got = [torch.full_like(x, -1) for x in ins]
        N.ntt_batch_submit([(p, k, x, y) for p, (_, _, _, k), x, y in zip(plans, cases, ins, ref)])
        rc = submit_static(lib, [(p, k, x, y) for p, (_, _, _, k), x, y in zip(plans, cases, ins, got)], status)
        assert rc == 0, N.ntt_status_string(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        for (f, ln, split, k), x, r, g in zip(cases, hx, ref, got):
            assert torch.equal(r, g), (f, ln, split)
            assert np.array_equal(host(g), oracle.c_transform(f, k, x)), (f, ln, split)
    finally:
        N.ntt_batch_cache_clear()
        for p in plans:
            N.ntt_plan_destroy(p)


def test_static_batch_empty_list_and_null_status():
    lib = N.load(build_if_missing=True)
    status = torch.full((1,), 999, dtype=torch.int32, device="cuda")
    assert lib.ntt_batch_submit_static(None, 0, ctypes.c_void_p(status.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0   # cleared, nothing launched
    plan = N.ntt_plan_create("bn254_fr", 15, coset=True)
    try:
        hx = uniform_elements("bn254_fr", 1 << 15, 62000)
        x = dev(hx)
        y = torch.full_like(x, -1)
        assert N.ntt_batch_poll_error() == 0
        rc = submit_static(lib, [(plan, "coset_inverse", x, y)], None)
        assert rc == 0, N.ntt_status_string(rc)
        assert N.ntt_batch_poll_error() == 0
        assert np.array_equal(host(y), oracle.c_transform("bn254_fr", "coset_inverse", hx))
    finally:
        N.ntt_batch_cache_clear()
        N.ntt_plan_destroy(plan)


def test_static_batch_forced_timeout_then_normal_call():
    """A host-side hook makes one device wait unsatisfiable; with a 5 ms wait
    limit the kernel gives up and reports NTT_ERR_TIMEOUT, through the status
    pointer or (without one) through ntt_batch_poll_error.  No GPU fault is
    involved.  The next call with the hook off runs normally."""
    lib = N.load(build_if_missing=True)
    plan = N.ntt_plan_create("bls12_381_fr", 16)
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    try:
        hx = uniform_elements("bls12_381_fr", 1 << 16, 63000)
        x = dev(hx)
        y = torch.empty_like(x)
        N.ntt_batch_set_wait_limit(5_000_000)
        N.ntt_batch_debug_stall(True)
        assert submit_static(lib, [(plan, "forward", x, y)], status) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == NTT_ERR_TIMEOUT
        assert submit_static(lib, [(plan, "forward", x, y)], None) == 0
        assert N.ntt_batch_poll_error() == NTT_ERR_TIMEOUT
        assert N.ntt_batch_poll_error() == 0   # cleared by the read
    finally:
        N.ntt_batch_debug_stall(False)
        N.ntt_batch_set_wait_limit(2_000_000_000)
    try:
        y = torch.full_like(x, -1)
        assert submit_static(lib, [(plan, "forward", x, y)], status) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert np.array_equal(host(y), oracle.c_transform("bls12_381_fr", "forward", hx))
    finally:
        N.ntt_batch_cache_clear()
        N.ntt_plan_destroy(plan)
