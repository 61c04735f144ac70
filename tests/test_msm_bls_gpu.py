"""Multi-scalar multiplication on BLS12-381 G1 (Algorithm 2 on the GPU, 381-bit
base field) against the CPU oracle: the result point must be identical.

Inputs are seeded: scalars uniform in [0, r) of BLS12-381 Fr, points
P_n = t_n G for seeded t_n, so the expected value also has the closed form
(sum_n S_n t_n mod r) G.  Small cases take their points from the oracle; the
2^22- and 2^24-point cases (the benchmark's sizes and launch configuration,
automatic window) take them from the library's fixed-base generator, check a
sample of them against the oracle, and check the MSM against the closed
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

CURVE_NAME = "bls12_381_g1"
C = mo.BLS12_381_G1
R = mo.BLS12_381_R
Q = mo.BLS12_381_Q
G = mo.BLS12_381_G
LIMBS = 6


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


def _pw(points):
    return mo.points_to_words(points, limbs=LIMBS)


def _run(pkg, scalars: np.ndarray, points: np.ndarray, window_bits: int = 0):
    n = scalars.shape[0]
    s = _dev(scalars if n else np.zeros((1, 4), np.uint64))
    p = _dev(points if n else np.zeros((1, 2 * LIMBS), np.uint64))
    plan = pkg.MsmPlan(max(n, 1), window_bits, curve=CURVE_NAME)
    try:
        out = plan.execute(s, p, count=n)
        torch.cuda.synchronize()
        err = plan.poll_error()
    finally:
        plan.close()
    return mo.words_to_points(out.cpu().numpy().view(np.uint64), limbs=LIMBS)[0], err


def _closed_form(ss, ts):
    return mo.scalar_mul(C, sum(int(s) * int(t) for s, t in zip(ss, ts)) % R, G)


def _inputs(n, seed):
    sw = ntt_synth.uniform_elements("bls12_381_fr", n, seed)
    ss = limbs_to_ints(sw)
    ts = limbs_to_ints(ntt_synth.uniform_elements("bls12_381_fr", n, seed + 1))
    return sw, ss, ts, mo.fixed_base_points(ts, C)


def test_point_bytes(msm):
    assert msm.msm_point_bytes("bls12_381_g1") == 96
    assert msm.msm_point_bytes("bn254_g1") == 64


@pytest.mark.parametrize("c", [0, 1, 5, 13, 16])
def test_bls_msm_matches_oracle(msm, c):
    sw, ss, ts, pts = _inputs(600, 0x4510 + c)
    got, err = _run(msm, sw, _pw(pts), window_bits=c)
    assert err == 0
    assert got == _closed_form(ss, ts)


def test_bls_msm_matches_ls_ppg_oracle_directly(msm):
    sw, ss, ts, pts = _inputs(80, 0x4520)
    got, _ = _run(msm, sw, _pw(pts), window_bits=6)
    assert got == mo.msm_ls_ppg(ss, pts, 6, C, mo.BLS12_381_SCALAR_BITS)


def test_bls_msm_degenerate_inputs(msm):
    _, ss, ts, pts = _inputs(40, 0x4540)
    cases = {
        "zero_scalars": ([0] * 40, pts),
        "r_minus_one": ([R - 1] * 5, pts[:5]),
        "repeated_point_equal_scalars": ([77] * 9, [pts[0]] * 9),
        "cancelling": ([5, 5, 5, 9], [pts[1], C.neg(pts[1]), pts[1], pts[2]]),
        "infinity_points": ([3, 8, 1, 4], [None, pts[3], None, pts[4]]),
        "top_bit_254": ([(1 << 254) + 1, (1 << 254) - 1], pts[5:7]),
        "single": ([123456789], [pts[8]]),
    }
    for name, (scal, points) in cases.items():
        got, err = _run(msm, _scalar_words(scal), _pw(points))
        assert err == 0, name
        assert got == mo.msm(scal, points, C), name


def test_bls_msm_constant_scalars(msm):
    n = 2000
    ts = limbs_to_ints(ntt_synth.uniform_elements("bls12_381_fr", n, 0x4550))
    pts = mo.fixed_base_points(ts, C)
    s = 0x1234_5678_9ABC_DEF0_0FED_CBA9_8765_4321_0000_1111
    got, err = _run(msm, _scalar_words([s] * n), _pw(pts), window_bits=12)
    assert err == 0
    assert got == mo.scalar_mul(C, s * (sum(ts) % R) % R, G)


def test_bls_msm_input_checks(msm):
    _, ss, ts, pts = _inputs(5, 0x4560)
    words = _pw(pts)
    bad = words.copy()
    bad[2, LIMBS] ^= np.uint64(1)  # y changed: off the curve
    got, err = _run(msm, _scalar_words(ss), bad, window_bits=8)
    assert err == 1
    assert got == mo.msm(ss[:2] + ss[3:], pts[:2] + pts[3:], C)
    big = words.copy()
    big[1, :LIMBS] = mo.points_to_words([(Q + 1, 0)], limbs=LIMBS)[0, :LIMBS]  # x >= q
    got, err = _run(msm, _scalar_words(ss), big, window_bits=8)
    assert err == 1
    assert got == mo.msm([ss[0]] + ss[2:], [pts[0]] + pts[2:], C)
    got, err = _run(msm, _scalar_words([R + 5, 7]), words[:2], window_bits=8)
    assert err == 2
    assert got == mo.msm([5, 7], pts[:2], C)


def test_bls_fixed_base_generator(msm):
    ts = limbs_to_ints(ntt_synth.uniform_elements("bls12_381_fr", 120, 0x4570)) + [0, 1, 2, R - 1, R]
    out = msm.fixed_base_points(_dev(_scalar_words(ts)), curve=CURVE_NAME)
    torch.cuda.synchronize()
    got = mo.words_to_points(out.cpu().numpy().view(np.uint64), limbs=LIMBS)
    assert got == mo.fixed_base_points(ts, C)
    assert got[-5] is None and got[-4] == G and got[-1] is None


@pytest.mark.parametrize("log_n", [22, 24])
def test_bls_msm_full_size_closed_form(msm, log_n):
    """2^22 and 2^24 points (the benchmark's sizes), automatic window: points
    from the fixed-base generator, 24 of them checked against the oracle; the
    MSM against the closed form."""
    n = 1 << log_n
    sw = ntt_synth.uniform_elements("bls12_381_fr", n, ntt_synth.config_seed(7))
    tw = ntt_synth.uniform_elements("bls12_381_fr", n, ntt_synth.config_seed(7, 1))
    d_t = _dev(tw)
    pts = msm.fixed_base_points(d_t, curve=CURVE_NAME)
    del d_t
    rng = np.random.default_rng(9)
    idx = np.concatenate([[0, n - 1], rng.integers(0, n, 22)])
    sample = mo.words_to_points(pts[torch.from_numpy(idx).to("cuda")].cpu().numpy().view(np.uint64), limbs=LIMBS)
    assert sample == mo.fixed_base_points(limbs_to_ints(tw[idx]), C)
    plan = msm.MsmPlan(n, curve=CURVE_NAME)
    try:
        d_s = _dev(sw)
        out = plan.execute(d_s, pts)
        torch.cuda.synchronize()
        assert plan.poll_error() == 0
        got = mo.words_to_points(out.cpu().numpy().view(np.uint64), limbs=LIMBS)[0]
        # the same MSM from precomputed bases
        plan.set_bases(pts)
        out_b = plan.execute_bases(d_s)
        torch.cuda.synchronize()
        assert torch.equal(out_b, out) and plan.poll_error() == 0
    finally:
        plan.close()
    ss = sw.view(np.uint8).reshape(n, 32)
    tt = tw.view(np.uint8).reshape(n, 32)
    acc = 0
    for i in range(n):
        acc += int.from_bytes(ss[i].tobytes(), "little") * int.from_bytes(tt[i].tobytes(), "little")
    assert got == mo.scalar_mul(C, acc % R, G)
