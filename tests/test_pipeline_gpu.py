"""GPU tests of a prover's quotient step built from the library's calls:
coset transforms of A, B, C on a 4x larger coset, the fused pointwise
quotient (a b - c) / Z_H, and the coset inverse.  With C = A B - Z_H Q the
result is Q exactly (Z_H = X^n - 1 divides A B - C), which pins the whole
chain to a closed form; the pointwise kernel is also compared with the
oracle element by element, including a ragged length and extreme values.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import ntt_oracle as O
from ntt_synth import uniform_elements

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_17808_gb300 import _native as N  # noqa: E402

FIELDS = ["bls12_381_fr", "bn254_fr"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    N.load(build_if_missing=True)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("field", FIELDS)
@pytest.mark.parametrize("z_len", [1, 4, 64])
def test_pointwise_quotient_matches_oracle(field, z_len):
    f = O.get_field(field)
    count = 10007                                   # ragged: not a multiple of any block size
    a = uniform_elements(field, count, 61000)
    b = uniform_elements(field, count, 61001)
    c = uniform_elements(field, count, 61002)
    edge = O.ints_to_limbs([0, 1, f.modulus - 1, f.modulus - 2])
    a[:4], b[:4], c[:4] = edge, edge[::-1], edge   # every sub wraps or not
    z = O.limbs_to_ints(uniform_elements(field, z_len, 61003))
    z[0] = f.modulus - 1
    d_a, d_b, d_c = dev(a), dev(b), dev(c)
    d_o = torch.empty_like(d_a)
    N.ntt_pointwise_quotient(field, d_a, d_b, d_c, z, d_o, count)
    want = O.quotient_pointwise(f, O.limbs_to_ints(a), O.limbs_to_ints(b), O.limbs_to_ints(c), z)
    assert O.limbs_to_ints(host(d_o)) == want
    # out may alias an input
    N.ntt_pointwise_quotient(field, d_a, d_b, d_c, z, d_a, count)
    assert O.limbs_to_ints(host(d_a)) == want


@pytest.mark.parametrize("field", FIELDS)
def test_prover_quotient_step_recovers_q(field):
    f = O.get_field(field)
    r = f.modulus
    log_n, blowup = 12, 4
    n, m = 1 << log_n, blowup << log_n
    A = uniform_elements(field, n, 62000)
    B = uniform_elements(field, n, 62001)
    Q = uniform_elements(field, n, 62002)
    # C = A B - (X^n - 1) Q on the CPU: A B through the oracle's convolution
    pad2 = lambda v: np.vstack([v, np.zeros_like(v)])          # noqa: E731
    FA = O.limbs_to_ints(oracle.c_transform(field, "forward", pad2(A)))
    FB = O.limbs_to_ints(oracle.c_transform(field, "forward", pad2(B)))
    AB = O.limbs_to_ints(oracle.c_transform(field, "inverse", O.ints_to_limbs([u * v % r for u, v in zip(FA, FB)])))
    q = O.limbs_to_ints(Q)
    C = [(AB[i] + (q[i] if i < n else 0) - (q[i - n] if i >= n else 0)) % r for i in range(2 * n)]
    padm = lambda v: np.vstack([v, np.zeros((m - v.shape[0], 4), dtype=np.uint64)])  # noqa: E731
    s = O.default_coset_shift(f)
    w_b = O.root_of_unity(f, blowup)
    z = [pow((pow(s, n, r) * pow(w_b, j, r) - 1) % r, r - 2, r) for j in range(blowup)]
    plan = N.ntt_plan_create(field, log_n + 2, coset=True)
    try:
        d = {}
        for name, v in (("a", A), ("b", B), ("c", O.ints_to_limbs(C))):
            d[name] = dev(padm(v))
            N.ntt_coset_forward(plan, d[name], d[name])
        t = torch.empty_like(d["a"])
        N.ntt_pointwise_quotient(field, d["a"], d["b"], d["c"], z, t, m)
        N.ntt_coset_inverse(plan, t, t)
        got = host(t)
        assert N.ntt_plan_poll_error(plan) == 0
    finally:
        N.ntt_plan_destroy(plan)
    assert np.array_equal(got[:n], Q)
    assert not got[n:].any()


def test_pointwise_quotient_rejects_bad_arguments():
    x = torch.zeros((64, 4), dtype=torch.int64, device="cuda")
    for z in ([1, 2, 3], [1] * 128, [O.BN254_FR.modulus]):
        with pytest.raises(N.NttError) as e:
            N.ntt_pointwise_quotient("bn254_fr", x, x, x, z, x, 64)
        assert e.value.status == 1
    lib = N.load()
    with pytest.raises(N.NttError):
        N.ntt_pointwise_quotient("bn254_fr", x.data_ptr() + 16, x, x, [1], x, 8)
    N.ntt_pointwise_quotient("bn254_fr", x, x, x, [1], x, 0)   # empty: nothing to do
    assert lib is not None
