"""Multi-scalar multiplication on BN254 G1 (Algorithm 2 on the GPU) against
the CPU oracle: the result point must be identical.

Inputs are seeded: scalars uniform in [0, r) (``ntt_synth``), points
P_n = t_n G for seeded t_n, so the expected value also has the closed form
(sum_n S_n t_n mod r) G.  Small cases take their points from the oracle; the
full-size case (2^24 points, the benchmark's workload and launch
configuration) takes them from the library's fixed-base generator, checks a
sample of them against the oracle, and checks the MSM against the closed
form.
"""

from __future__ import annotations

import numpy as np
import pytest

import ntt_synth
from oracle import limbs_to_ints
from oracle import msm_oracle as mo

torch = pytest.importorskip("torch")

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]

R = mo.BN254_R
Q = mo.BN254_Q
G = mo.BN254_G
CURVE = mo.BN254_G1


@pytest.fixture(scope="module")
def msm():
    import paper_2604_17808_gb300 as pkg

    pkg._native.load(build_if_missing=True)
    return pkg


def _dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to("cuda")


def _scalar_words(values) -> np.ndarray:
    out = np.zeros((len(values), 4), dtype=np.uint64)
    for i, v in enumerate(values):
        for j in range(4):
            out[i, j] = (int(v) >> (64 * j)) & 0xFFFFFFFFFFFFFFFF
    return out


def _run(pkg, scalars: np.ndarray, points: np.ndarray, window_bits: int = 0, max_n: int | None = None,
         plan=None):
    n = scalars.shape[0]
    s = _dev(scalars if n else np.zeros((1, 4), np.uint64))
    p = _dev(points if n else np.zeros((1, 8), np.uint64))
    own = plan is None
    if own:
        plan = pkg.MsmPlan(max(max_n or n, 1), window_bits)
    try:
        out = plan.execute(s, p, count=n)
        torch.cuda.synchronize()
        err = plan.poll_error()
    finally:
        if own:
            plan.close()
    return mo.words_to_points(out.cpu().numpy().view(np.uint64))[0], err


def _closed_form(ss, ts):
    return mo.scalar_mul(CURVE, sum(int(s) * int(t) for s, t in zip(ss, ts)) % R, G)


def _inputs(n, seed):
    sw = ntt_synth.uniform_elements("bn254_fr", n, seed)
    tw = ntt_synth.uniform_elements("bn254_fr", n, seed + 1)
    ss = limbs_to_ints(sw)
    ts = limbs_to_ints(tw)
    pts = mo.fixed_base_points(ts)
    return sw, ss, ts, pts


@pytest.mark.parametrize("c", [0, 1, 3, 8, 13, 16])
def test_msm_matches_oracle(msm, c):
    sw, ss, ts, pts = _inputs(1000, 0x3510 + c)
    got, err = _run(msm, sw, mo.points_to_words(pts), window_bits=c)
    assert err == 0
    assert got == _closed_form(ss, ts)


@pytest.mark.parametrize("c", [2, 5, 20])
def test_msm_windows_and_segment_boundaries(msm, c):
    # small windows put many points in each bucket (buckets cross many
    # accumulation segments); c = 20 leaves most buckets empty
    sw, ss, ts, pts = _inputs(2500, 0x3580 + c)
    got, err = _run(msm, sw, mo.points_to_words(pts), window_bits=c)
    assert err == 0
    assert got == _closed_form(ss, ts)


def test_msm_matches_ls_ppg_oracle_directly(msm):
    sw, ss, ts, pts = _inputs(150, 0x3520)
    got, _ = _run(msm, sw, mo.points_to_words(pts), window_bits=5)
    assert got == mo.msm_ls_ppg(ss, pts, 5)
    assert got == mo.msm(ss, pts)


def test_msm_ragged_lengths_and_plan_reuse(msm):
    sw, ss, ts, pts = _inputs(4099, 0x3530)
    words = mo.points_to_words(pts)
    plan = msm.MsmPlan(5000)
    try:
        for n in (1, 2, 31, 257, 4099, 0, 17):
            got, err = _run(msm, sw[:n], words[:n], plan=plan)
            assert err == 0
            assert got == (_closed_form(ss[:n], ts[:n]) if n else None), n
        info = plan.info()
        assert info["max_n"] == 5000 and info["num_windows"] == -(-255 // info["window_bits"])  # signed digits
    finally:
        plan.close()


def test_msm_degenerate_inputs(msm):
    _, ss, ts, pts = _inputs(64, 0x3540)
    neg = CURVE.neg
    cases = {
        "zero_scalars": ([0] * 64, pts),
        "r_minus_one": ([R - 1] * 5, pts[:5]),
        "repeated_point_equal_scalars": ([77] * 9, [pts[0]] * 9),
        "cancelling": ([5, 5, 5, 9], [pts[1], neg(pts[1]), pts[1], pts[2]]),
        "infinity_points": ([3, 8, 1, 4], [None, pts[3], None, pts[4]]),
        "one_hot_low_window": ([1] * 40, pts[:40]),
        "top_bits": ([(1 << 253) + 1, (1 << 253) - 1], pts[5:7]),
    }
    for name, (scal, points) in cases.items():
        got, err = _run(msm, _scalar_words(scal), mo.points_to_words(points))
        assert err == 0, name
        assert got == mo.msm(scal, points), name


@pytest.mark.parametrize("c", [8, 16])
def test_msm_constant_scalars_spread_over_segments(msm, c):
    # every point in the same bucket of every window: the bucket is summed by
    # many segments and the pairwise combine tree (c = 16 sorts through the
    # two-level bucketize, c = 8 through the one-level one)
    n = 3000
    ts = limbs_to_ints(ntt_synth.uniform_elements("bn254_fr", n, 0x3550))
    pts = mo.fixed_base_points(ts)
    s = 0x1234_5678_9ABC_DEF0_0FED_CBA9_8765_4321
    got, err = _run(msm, _scalar_words([s] * n), mo.points_to_words(pts), window_bits=c)
    assert err == 0
    assert got == mo.scalar_mul(CURVE, s * (sum(ts) % R) % R, G)


def test_msm_input_checks(msm):
    _, ss, ts, pts = _inputs(6, 0x3560)
    words = mo.points_to_words(pts)
    bad = words.copy()
    bad[2, 4] ^= np.uint64(1)  # y changed: off the curve
    got, err = _run(msm, _scalar_words(ss), bad, window_bits=8)
    assert err == 1
    assert got == mo.msm(ss[:2] + ss[3:], pts[:2] + pts[3:])
    big = words.copy()
    big[1, :4] = _scalar_words([Q + 1])[0]  # x >= q
    got, err = _run(msm, _scalar_words(ss), big, window_bits=8)
    assert err == 1
    assert got == mo.msm([ss[0]] + ss[2:], [pts[0]] + pts[2:])
    # scalars >= r are flagged; below 2^254 the result is still exact
    got, err = _run(msm, _scalar_words([R + 5, 7]), words[:2], window_bits=8)
    assert err == 2
    assert got == mo.msm([5, 7], pts[:2])
    _, err = _run(msm, _scalar_words([(1 << 256) - 1]), words[:1], window_bits=8)
    assert err == 2


def test_fixed_base_generator(msm):
    ts = limbs_to_ints(ntt_synth.uniform_elements("bn254_fr", 200, 0x3570)) + [0, 1, 2, R - 1, R, (1 << 256) - 1]
    out = msm.fixed_base_points(_dev(_scalar_words(ts)))
    torch.cuda.synchronize()
    got = mo.words_to_points(out.cpu().numpy().view(np.uint64))
    assert got == mo.fixed_base_points(ts)
    assert got[-6] is None and got[-5] == G


def test_msm_full_size_closed_form(msm):
    """2^24 points (the benchmark's workload, automatic window): points from
    the fixed-base generator, 32 of them checked against the oracle; the MSM
    against (sum S_n t_n mod r) G."""
    n = 1 << 24
    sw = ntt_synth.uniform_elements("bn254_fr", n, ntt_synth.config_seed(6))
    tw = ntt_synth.uniform_elements("bn254_fr", n, ntt_synth.config_seed(6, 1))
    d_t = _dev(tw)
    pts = msm.fixed_base_points(d_t)
    del d_t
    rng = np.random.default_rng(7)
    idx = np.concatenate([[0, n - 1], rng.integers(0, n, 30)])
    sample = mo.words_to_points(pts[torch.from_numpy(idx).to("cuda")].cpu().numpy().view(np.uint64))
    assert sample == mo.fixed_base_points(limbs_to_ints(tw[idx]))
    plan = msm.MsmPlan(n)
    try:
        d_s = _dev(sw)
        out = plan.execute(d_s, pts)
        torch.cuda.synchronize()
        assert plan.poll_error() == 0
        got = mo.words_to_points(out.cpu().numpy().view(np.uint64))[0]
        # the same MSM from precomputed bases
        plan.set_bases(pts)
        out_b = plan.execute_bases(d_s)
        torch.cuda.synchronize()
        assert torch.equal(out_b, out) and plan.poll_error() == 0
    finally:
        plan.close()
    acc = 0
    ss = sw.view(np.uint8).reshape(n, 32)
    tt = tw.view(np.uint8).reshape(n, 32)
    for i in range(n):
        acc += int.from_bytes(ss[i].tobytes(), "little") * int.from_bytes(tt[i].tobytes(), "little")
    assert got == mo.scalar_mul(CURVE, acc % R, G)
