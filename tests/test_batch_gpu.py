"""GPU parity of the batched path (one persistent launch per field, replayed
from a CUDA graph) against the oracle and against single transforms.

Bit-exact: every job's output must equal its oracle result and its result
when run alone.  The bounded-wait failure path is forced from the host
(ntt_batch_debug_stall makes one device wait unsatisfiable; the wait limit
is set to a few milliseconds): no GPU fault is involved.
"""

from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from ntt_synth import batch_sizes, config_seed, uniform_elements

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_17808_gb300 import _native as N  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    N.load(build_if_missing=True)
    yield
    N.ntt_batch_cache_clear()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def digest(a) -> str:
    return hashlib.sha256(a.astype("<u8").tobytes()).hexdigest()


def test_batched_workload_matches_oracle_digests_and_single_runs():
    with open(os.path.join(HERE, "golden", "oracle_digests.json")) as fh:
        g = json.load(fh)["batched"]
    sizes = batch_sizes(64, 14, 22, config_seed(4))
    assert sizes == [j["log_n"] for j in g["jobs"]]
    plans = {ln: N.ntt_plan_create("bls12_381_fr", ln) for ln in sorted(set(sizes))}
    try:
        ins, outs, jobs = [], [], []
        for j, ln in enumerate(sizes):
            x = dev(uniform_elements("bls12_381_fr", 1 << ln, config_seed(4, j)))
            y = torch.empty_like(x)
            ins.append(x)
            outs.append(y)
            jobs.append((plans[ln], "forward", x, y))
        N.ntt_batch_submit(jobs)
        got = [host(y) for y in outs]
        for j, job in enumerate(g["jobs"]):
            assert digest(got[j]) == job["output_sha256"], j
        # replay from the cached graph gives the same bytes
        for y in outs:
            y.zero_()
        N.ntt_batch_submit(jobs)
        for j, y in enumerate(outs):
            assert np.array_equal(host(y), got[j]), j
        assert N.ntt_batch_poll_error() == 0
        # each job alone (one launch per pass) equals its batched result
        for j in (0, 7, 63):
            y = torch.empty_like(ins[j])
            N.ntt_forward(plans[sizes[j]], ins[j], y)
            assert np.array_equal(host(y), got[j])
    finally:
        N.ntt_batch_cache_clear()
        for p in plans.values():
            N.ntt_plan_destroy(p)


def test_batched_mixed_fields_kinds_and_sizes_match_oracle():
    specs = []
    for i, ln in enumerate([1, 2, 5, 9, 11, 12, 13, 16, 17, 20]):
        for field in ("bls12_381_fr", "bn254_fr"):
            kind = ("forward", "inverse", "coset", "coset_inverse")[(i + len(field)) % 4]
            specs.append((field, ln, kind))
    plans = {}
    jobs, cases = [], []
    try:
        for k, (field, ln, kind) in enumerate(specs):
            key = (field, ln)
            if key not in plans:
                plans[key] = N.ntt_plan_create(field, ln, coset=True)
            x = uniform_elements(field, 1 << ln, 5000 + k)
            d_x = dev(x)
            d_y = torch.empty_like(d_x)
            jobs.append((plans[key], kind, d_x, d_y))
            cases.append((field, kind, x, d_y))
        N.ntt_batch_submit(jobs)
        for field, kind, x, d_y in cases:
            assert np.array_equal(host(d_y), oracle.c_transform(field, kind, x)), (field, kind, x.shape[0])
        assert N.ntt_batch_poll_error() == 0
    finally:
        N.ntt_batch_cache_clear()
        for p in plans.values():
            N.ntt_plan_destroy(p)


def test_batch_rejects_in_place_and_bad_kinds():
    plan = N.ntt_plan_create("bn254_fr", 12)
    try:
        x = torch.zeros((1 << 12, 4), dtype=torch.int64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(N.NttError) as e:
            N.ntt_batch_submit([(plan, "forward", x, x)])
        assert e.value.status == 1
        with pytest.raises(N.NttError):
            N.ntt_batch_submit([(plan, "coset", x, y)])  # no coset tables
        with pytest.raises(N.NttError):
            N.ntt_batch_submit([(plan, "coset_inverse", x, y)])
        with pytest.raises(N.NttError):
            N.ntt_batch_submit([(plan, 4, x, y)])   # unknown kind
        N.ntt_batch_submit([])
    finally:
        N.ntt_plan_destroy(plan)


def test_bounded_wait_times_out_and_reports():
    plan = N.ntt_plan_create("bls12_381_fr", 16)
    try:
        x = dev(uniform_elements("bls12_381_fr", 1 << 16, 77))
        y = torch.empty_like(x)
        N.ntt_batch_set_wait_limit(5_000_000)        # 5 ms
        N.ntt_batch_debug_stall(True)
        N.ntt_batch_submit([(plan, "forward", x, y)])
        assert N.ntt_batch_poll_error() == 5         # NTT_ERR_TIMEOUT
        assert N.ntt_batch_poll_error() == 0         # cleared on read
        N.ntt_batch_debug_stall(False)
        N.ntt_batch_set_wait_limit(2_000_000_000)
        N.ntt_batch_submit([(plan, "forward", x, y)])
        assert N.ntt_batch_poll_error() == 0
        assert np.array_equal(host(y), oracle.c_transform("bls12_381_fr", "forward", host(x)))
    finally:
        N.ntt_batch_debug_stall(False)
        N.ntt_batch_set_wait_limit(2_000_000_000)
        N.ntt_plan_destroy(plan)


def test_batch_autotune_keeps_results_and_runs_matrix_plans():
    """ntt_batch_autotune picks a policy (persistent kernel, or the larger jobs
    as ordinary transforms on parallel graph branches); whatever it picks,
    every output must stay bit-exact with the oracle digests, and lists with
    the same signature (other buffers) follow the policy.  Jobs whose plan is
    on the matrix path run inside the batch's graph as ordinary transforms."""
    with open(os.path.join(HERE, "golden", "oracle_digests.json")) as fh:
        g = json.load(fh)["batched"]
    sizes = batch_sizes(64, 14, 22, config_seed(4))
    plans = {ln: N.ntt_plan_create("bls12_381_fr", ln) for ln in sorted(set(sizes))}
    try:
        N.ntt_plan_set_path(plans[20], "matrix")   # one size on the tensor-core path
        ins, outs, jobs = [], [], []
        for j, ln in enumerate(sizes):
            x = dev(uniform_elements("bls12_381_fr", 1 << ln, config_seed(4, j)))
            y = torch.empty_like(x)
            ins.append(x)
            outs.append(y)
            jobs.append((plans[ln], "forward", x, y))
        res = N.ntt_batch_autotune(jobs, reps=1)
        assert res["candidates"] >= 2 and res["best_ms"] > 0
        assert res["best_ms"] <= min(res["persistent_ms"], res["loop_ms"]) * 1.05 + 0.05
        for y in outs:
            y.zero_()
        N.ntt_batch_submit(jobs)
        for j, job in enumerate(g["jobs"]):
            assert digest(host(outs[j])) == job["output_sha256"], j
        # same signature, other output buffers: the tuned policy applies
        outs2 = [torch.empty_like(x) for x in ins]
        N.ntt_batch_submit([(plans[ln], "forward", x, y) for ln, x, y in zip(sizes, ins, outs2)])
        for j, job in enumerate(g["jobs"]):
            assert digest(host(outs2[j])) == job["output_sha256"], j
        assert N.ntt_batch_poll_error() == 0
        assert N.ntt_plan_poll_error(plans[20]) == 0
    finally:
        N.ntt_batch_cache_clear()
        for p in plans.values():
            N.ntt_plan_destroy(p)
