"""Window-range parts of the MSM on the GPU (the per-rank work of the
window-sharded MSM): the parts over a split of the windows must add up to the
whole MSM, for both curves, and that MSM must equal the oracle's closed form.
"""

from __future__ import annotations

import numpy as np
import pytest

import ntt_synth
from oracle import limbs_to_ints
from oracle import msm_oracle as mo

torch = pytest.importorskip("torch")

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]

CASES = {"bn254_g1": ("bn254_fr", 4), "bls12_381_g1": ("bls12_381_fr", 6)}


@pytest.fixture(scope="module")
def pkg():
    import paper_2604_17808_gb300 as p

    p._native.load(build_if_missing=True)
    return p


def _dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to("cuda")


@pytest.mark.parametrize("curve_name", list(CASES))
def test_window_parts_add_up_to_the_msm(pkg, curve_name):
    from paper_2604_17808_gb300.msm_shard import sharded_msm, sum_points, window_range

    field, limbs = CASES[curve_name]
    curve, _, _ = mo.CURVES[curve_name]
    n = 1500
    sw = ntt_synth.uniform_elements(field, n, 0x5B00)
    ts = limbs_to_ints(ntt_synth.uniform_elements(field, n, 0x5B01))
    pts = mo.fixed_base_points(ts, curve)
    d_s = _dev(sw)
    d_p = _dev(mo.points_to_words(pts, limbs=limbs))
    closed = mo.scalar_mul(curve, sum(s * t for s, t in zip(limbs_to_ints(sw), ts)) % curve.order,
                           curve.generator)
    with pkg.MsmPlan(n, 8, curve=curve_name) as plan:
        K = plan.info()["num_windows"]
        full = plan.execute(d_s, d_p).clone()
        for world in (2, 3, 5):
            parts = torch.stack([plan.execute_windows(d_s, d_p, *window_range(K, r, world)).clone()
                                 for r in range(world)])
            total = sum_points(parts, curve_name)
            torch.cuda.synchronize()
            assert torch.equal(total, full), world
        empty = plan.execute_windows(d_s, d_p, 5, 5)
        torch.cuda.synchronize()
        assert mo.words_to_points(empty.cpu().numpy().view(np.uint64), limbs=limbs)[0] is None
        # without a process group the sharded call is the whole MSM on this GPU
        single = sharded_msm(plan, d_s, d_p)
        torch.cuda.synchronize()
        assert torch.equal(single, full)
        with pytest.raises(pkg.NttError):
            plan.execute_windows(d_s, d_p, 3, 2)
        with pytest.raises(pkg.NttError):
            plan.execute_windows(d_s, d_p, 0, K + 1)
        assert plan.poll_error() == 0
    assert mo.words_to_points(full.cpu().numpy().view(np.uint64), limbs=limbs)[0] == closed
