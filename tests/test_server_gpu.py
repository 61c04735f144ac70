"""GPU tests of the serving runtime (continuous batching under a memory
budget): every result is bit-identical to the same transform run alone, with
requests of mixed fields, kinds and sizes submitted while earlier ones are
on the GPU, and admission respects the budget."""

from __future__ import annotations

import random
import time

import numpy as np
import pytest

import oracle
from ntt_synth import uniform_elements

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_17808_gb300 import _native as N  # noqa: E402

FIELDS = ["bls12_381_fr", "bn254_fr"]
KINDS = ["forward", "inverse", "coset", "coset_inverse"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    N.load(build_if_missing=True)


def pinned(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).pin_memory()


def test_results_in_the_mix_equal_results_alone():
    server = N.ntt_server_create(min_log_n=8, max_log_n=18, max_inflight=3, max_batch_jobs=8)
    rng = random.Random(42)
    reqs = []
    try:
        for i in range(60):
            field = rng.choice(FIELDS)
            kind = rng.choice(KINDS)
            log_n = rng.randint(8, 18)
            x = uniform_elements(field, 1 << log_n, 20000 + i)
            h_in = pinned(x)
            h_out = torch.empty_like(h_in).pin_memory()
            t = N.ntt_server_submit(server, field, kind, log_n, h_in, h_out)
            reqs.append((t, field, kind, log_n, x, h_in, h_out))
            if i % 7 == 3:
                time.sleep(0.002)  # let earlier requests reach the GPU first
        for t, *_ in reqs:
            N.ntt_server_wait(server, t, 60.0)
        stats = N.ntt_server_get_stats(server)
        assert stats["completed"] == len(reqs)
        assert stats["batches"] >= 2
        for t, field, kind, log_n, x, h_in, h_out in reqs:
            got = h_out.numpy().view(np.uint64)
            assert np.array_equal(got, oracle.c_transform(field, kind, x)), (field, kind, log_n)
            arrive, admit, finish = N.ntt_server_request_times(server, t)
            assert 0 <= arrive <= admit <= finish
        # the same request alone through the plain path is identical
        t, field, kind, log_n, x, h_in, h_out = reqs[5]
        plan = N.ntt_plan_create(field, log_n, coset=True)
        try:
            d_x = torch.from_numpy(x.view(np.int64)).cuda()
            d_y = torch.empty_like(d_x)
            N.ntt_execute(plan, kind, d_x, d_y)
            torch.cuda.synchronize()
            assert np.array_equal(d_y.cpu().numpy().view(np.uint64), h_out.numpy().view(np.uint64))
        finally:
            N.ntt_plan_destroy(plan)
    finally:
        N.ntt_server_destroy(server)


def test_admission_respects_the_memory_budget():
    # budget: resident tables + room for about two 2^16 requests at a time
    probe = N.ntt_server_create(min_log_n=10, max_log_n=16, max_inflight=2)
    resident = N.ntt_server_get_stats(probe)["resident_bytes"]
    N.ntt_server_destroy(probe)
    budget = resident + 4 * (32 << 16) + (32 << 16)
    server = N.ntt_server_create(memory_budget_bytes=budget, min_log_n=10, max_log_n=16, max_inflight=2)
    try:
        reqs = []
        for i in range(12):
            x = uniform_elements("bn254_fr", 1 << 16, 30000 + i)
            h_in = pinned(x)
            h_out = torch.empty_like(h_in).pin_memory()
            reqs.append((N.ntt_server_submit(server, "bn254_fr", "forward", 16, h_in, h_out), x, h_in, h_out))
        for t, *_ in reqs:
            N.ntt_server_wait(server, t, 60.0)
        stats = N.ntt_server_get_stats(server)
        assert stats["peak_device_bytes"] <= budget
        for t, x, h_in, h_out in reqs:
            assert np.array_equal(h_out.numpy().view(np.uint64), oracle.c_transform("bn254_fr", "forward", x))
    finally:
        N.ntt_server_destroy(server)


def test_server_rejects_bad_requests():
    server = N.ntt_server_create(min_log_n=10, max_log_n=12, max_inflight=1)
    try:
        h = pinned(np.zeros((1 << 10, 4), dtype=np.uint64))
        with pytest.raises(N.NttError) as e:
            N.ntt_server_submit(server, "bls12_381_fr", "forward", 14, h, h)
        assert e.value.status == 2
        with pytest.raises(N.NttError):
            N.ntt_server_submit(server, "bls12_381_fr", 7, 10, h, h)
        with pytest.raises(N.NttError):
            N.ntt_server_wait(server, 12345, 0.1)
    finally:
        N.ntt_server_destroy(server)
    with pytest.raises(N.NttError) as e:
        N.ntt_server_create(memory_budget_bytes=1 << 20, min_log_n=10, max_log_n=12)
    assert e.value.status == 6  # NTT_ERR_BUDGET
