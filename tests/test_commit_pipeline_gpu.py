"""The prover's two kernels together: a KZG-style polynomial commitment on
BLS12-381, computed entirely on the GPU.

Evaluations e_k of a polynomial f on the 2^m-th roots of unity are
interpolated by the inverse NTT into coefficients c_i (the transform's
output layout is the MSM's scalar layout, so nothing leaves the device), and
the commitment is the MSM sum_i c_i P_i over setup points P_i = tau^i G.
Closed form: sum_i c_i tau^i G = f(tau) G, with f(tau) evaluated by the
oracle (its own inverse transform, then Horner at tau).
"""

from __future__ import annotations

import numpy as np
import pytest

import ntt_synth
import oracle
from oracle import limbs_to_ints
from oracle import msm_oracle as mo

torch = pytest.importorskip("torch")

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]

FIELD = "bls12_381_fr"
CURVE = "bls12_381_g1"
R = mo.BLS12_381_R
TAU = 0x1D2C3B4A59687766554433221100FFEEDDCCBBAA99887766554433221100  # a fixed setup secret < r


@pytest.fixture(scope="module")
def pkg():
    import paper_2604_17808_gb300 as p

    p._native.load(build_if_missing=True)
    return p


def _dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to("cuda")


def _powers(n: int) -> np.ndarray:
    out = np.zeros((n, 4), dtype=np.uint64)
    t = 1
    for i in range(n):
        for j in range(4):
            out[i, j] = (t >> (64 * j)) & 0xFFFFFFFFFFFFFFFF
        t = t * TAU % R
    return out


@pytest.mark.parametrize("log_n", [12, 20])
def test_kzg_commitment_pipeline(pkg, log_n):
    n = 1 << log_n
    evals = ntt_synth.uniform_elements(FIELD, n, ntt_synth.config_seed(8, log_n))
    d_e = _dev(evals)
    d_c = torch.empty_like(d_e)
    srs = pkg.fixed_base_points(_dev(_powers(n)), curve=CURVE)  # P_i = tau^i G
    with pkg.Plan(FIELD, log_n) as plan, pkg.MsmPlan(n, curve=CURVE) as msm:
        plan.inverse(d_e, out=d_c)                  # coefficients, on the device
        com = msm.execute(d_c, srs)                 # sum_i c_i P_i
        msm.set_bases(srs)
        com_b = msm.execute_bases(d_c)
        torch.cuda.synchronize()
        assert msm.poll_error() == 0
    coeffs = oracle.c_transform(FIELD, "inverse", evals)
    assert np.array_equal(d_c.cpu().numpy().view(np.uint64), coeffs)
    f_tau = oracle.c_eval(FIELD, coeffs, TAU)
    expect = mo.scalar_mul(mo.BLS12_381_G1, f_tau, mo.BLS12_381_G)
    got = mo.words_to_points(com.cpu().numpy().view(np.uint64), limbs=6)[0]
    assert got == expect
    assert torch.equal(com_b, com)
