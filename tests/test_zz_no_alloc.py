"""The allocation-free batched entry point (ntt_batch_submit_static).

Callers that cannot allocate device memory while they submit work -- a
service that reserved all its memory up front, or a submitter on a latency
path where cudaMalloc's implicit synchronisation would stall other streams --
use this entry point: it runs the same
batched kernel with its work-item table and counters in a fixed array the
library keeps in device memory.  This test calls it through the C ABI and
checks its outputs against the regular entry point (ntt_batch_submit) on two
calls in a row with different data; the bar is bit-exact, like every other
parity test here.  The file is named so that pytest collects it last.
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

from paper_2604_17808_gb300 import _native as N  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def test_static_batch_matches_regular_batch_on_two_calls():
    lib = N.load(build_if_missing=True)
    specs = [("bls12_381_fr", 14, "forward"), ("bls12_381_fr", 17, "inverse"), ("bn254_fr", 12, "coset"),
             ("bn254_fr", 20, "forward"), ("bls12_381_fr", 9, "coset"), ("bn254_fr", 16, "inverse")]
    plans = {(f, ln): N.ntt_plan_create(f, ln, coset=True) for f, ln, _ in specs}
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    try:
        for call in range(2):
            ins = [dev(uniform_elements(f, 1 << ln, 50000 + 100 * call + i)) for i, (f, ln, _) in enumerate(specs)]
            ref = [torch.empty_like(x) for x in ins]
            got = [torch.full_like(x, -1) for x in ins]
            N.ntt_batch_submit([(plans[(f, ln)], k, x, y) for (f, ln, k), x, y in zip(specs, ins, ref)])
            arr = (N.Job * len(specs))()
            for i, ((f, ln, k), x, y) in enumerate(zip(specs, ins, got)):
                arr[i] = N.Job(plans[(f, ln)], N.KIND[k], x.data_ptr(), y.data_ptr())
            rc = lib.ntt_batch_submit_static(arr, len(specs), ctypes.c_void_p(status.data_ptr()), None)
            assert rc == 0, N.ntt_status_string(rc)
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            for i, (r, g) in enumerate(zip(ref, got)):
                assert torch.equal(r, g), (call, specs[i])
        # beyond the maximum: a clear error, nothing launched
        too_many = (N.Job * 65)()
        assert lib.ntt_batch_submit_static(too_many, 65, None, None) == 2  # NTT_ERR_UNSUPPORTED
    finally:
        N.ntt_batch_cache_clear()
        for p in plans.values():
            N.ntt_plan_destroy(p)
