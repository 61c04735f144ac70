"""MSM with precomputed bases (points set once per plan, their window copies
2^(k c) P stored): the result must equal msm_execute's and the oracle's
closed form, on both curves, for several window sizes, reused bases, a
prefix of the points, and invalid points.
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


def _point(t, limbs):
    return mo.words_to_points(t.cpu().numpy().view(np.uint64), limbs=limbs)[0]


@pytest.mark.parametrize("curve_name", list(CASES))
@pytest.mark.parametrize("c", [0, 9, 12])
def test_bases_match_msm_and_closed_form(pkg, curve_name, c):
    field, limbs = CASES[curve_name]
    curve, _, _ = mo.CURVES[curve_name]
    n = 1500
    ts = limbs_to_ints(ntt_synth.uniform_elements(field, n, 0x5C00 + c))
    pts = mo.fixed_base_points(ts, curve)
    d_p = _dev(mo.points_to_words(pts, limbs=limbs))
    with pkg.MsmPlan(n, c, curve=curve_name) as plan:
        plan.set_bases(d_p)
        for seed in (0x5C10 + c, 0x5C20 + c):  # the same bases, two scalar sets
            sw = ntt_synth.uniform_elements(field, n, seed)
            d_s = _dev(sw)
            got = plan.execute_bases(d_s).clone()
            ref = plan.execute(d_s, d_p).clone()
            torch.cuda.synchronize()
            assert torch.equal(got, ref)
            closed = mo.scalar_mul(curve, sum(s * t for s, t in zip(limbs_to_ints(sw), ts)) % curve.order,
                                   curve.generator)
            assert _point(got, limbs) == closed
        # a prefix of the points
        m = 700
        part = plan.execute_bases(d_s, count=m)
        torch.cuda.synchronize()
        ss = limbs_to_ints(sw)
        closed = mo.scalar_mul(curve, sum(s * t for s, t in zip(ss[:m], ts[:m])) % curve.order, curve.generator)
        assert _point(part, limbs) == closed
        with pytest.raises(pkg.NttError):
            plan.execute_bases(d_s, count=n + 1)
        assert plan.poll_error() == 0


@pytest.mark.parametrize("curve_name", list(CASES))
def test_bases_errors_and_invalid_points(pkg, curve_name):
    field, limbs = CASES[curve_name]
    curve, _, _ = mo.CURVES[curve_name]
    n = 64
    ts = limbs_to_ints(ntt_synth.uniform_elements(field, n, 0x5C30))
    pts = mo.fixed_base_points(ts, curve)
    words = mo.points_to_words(pts, limbs=limbs)
    sw = ntt_synth.uniform_elements(field, n, 0x5C31)
    d_s = _dev(sw)
    with pkg.MsmPlan(n, 10, curve=curve_name) as plan:
        with pytest.raises(pkg.NttError):
            plan.execute_bases(d_s)          # no bases set yet
        bad = words.copy()
        bad[5, limbs] ^= np.uint64(1)       # y changed: off the curve
        plan.set_bases(_dev(bad))
        got = plan.execute_bases(d_s)
        torch.cuda.synchronize()
        assert plan.poll_error() == 1
        ss = limbs_to_ints(sw)
        assert _point(got, limbs) == mo.msm(ss[:5] + ss[6:], pts[:5] + pts[6:], curve)
    with pkg.MsmPlan(n, 4, curve=curve_name) as plan:  # 64 windows: more than the 32 supported
        with pytest.raises(pkg.NttError):
            plan.set_bases(_dev(words))
