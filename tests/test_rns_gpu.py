"""GPU parity of the RNS lazy multiplication (tcgen05 byte products) with
its oracle, and the library's residue bases against the oracle's.

The bar is bit-exact: the algorithm fixes every residue of every output
(the quotient estimates are exact), so the CUDA path and oracle/rns_oracle
must agree word for word; the outputs are also checked to be congruent to
x y^reps modulo M and below the lazy bound L.
"""

from __future__ import annotations

import random

import numpy as np
import pytest

from oracle import rns_oracle as R

torch = pytest.importorskip("torch")

from paper_2604_17808_gb300 import _native as N  # noqa: E402

FIELDS = ["bls12_381_fr", "bn254_fr"]


@pytest.fixture(scope="module")
def lib():
    return N.load(build_if_missing=True)


@pytest.mark.parametrize("field", FIELDS)
def test_library_bases_equal_the_oracle_bases(lib, field):
    # host-only computation in the library: runs without a GPU
    got = N.ntt_rns_basis_get(field)
    b = R.rns_basis(field)
    assert got["q"] == list(b.q) and got["p"] == list(b.p)
    assert got["words_per_element"] == 20 and got["shift"] == R.U_SHIFT


def words(vals, b):
    out = np.zeros((len(vals), 20), dtype=np.uint32)
    for e, v in enumerate(vals):
        out[e, : len(b.q)] = R.to_rns(v, b.q)
    return out


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


@pytest.mark.gpu
@pytest.mark.parametrize("field", FIELDS)
@pytest.mark.parametrize("reps", [1, 3])
def test_rns_mul_matches_oracle(lib, field, reps):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    b = R.rns_basis(field)
    tabs = R.tables(b)
    rng = random.Random(70 + reps)
    count = 1000                                   # 7 full tiles of 128 and a ragged one
    xs = [rng.randrange(b.L) for _ in range(count)]
    ys = [rng.randrange(b.L) for _ in range(count)]
    xs[:4] = [0, b.L - 1, b.modulus - 1, 1]
    ys[:4] = [b.L - 1, b.L - 1, b.modulus - 1, 1]
    hx, hy = words(xs, b), words(ys, b)
    d_x, d_y = dev(hx), dev(hy)
    d_o = torch.empty_like(d_x)
    N.ntt_rns_mul(field, d_x, d_y, d_o, count, reps)
    torch.cuda.synchronize()
    got = d_o.cpu().numpy().view(np.uint32)
    assert N.ntt_rns_poll_error(field) == 0
    I = len(b.q)
    for e in range(count):
        r = [int(v) for v in hx[e, :I]]
        yr = [int(v) for v in hy[e, :I]]
        for _ in range(reps):
            r = R.rns_mul_lazy(b, r, yr, tabs)
        assert [int(v) for v in got[e, :I]] == r, e
        assert not got[e, I:].any()
        v = R.from_rns(r, b.q)
        assert v < b.L and v % b.modulus == xs[e] * pow(ys[e], reps, b.modulus) % b.modulus


@pytest.mark.gpu
def test_rns_mul_argument_errors(lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x = torch.zeros((8, 20), dtype=torch.int32, device="cuda")
    with pytest.raises(N.NttError):
        N.ntt_rns_mul("bn254_fr", x, x, x, 8, 0)                 # reps = 0
    with pytest.raises(N.NttError):
        N.ntt_rns_mul("bn254_fr", x.data_ptr() + 4, x, x, 4, 1)  # misaligned
    N.ntt_rns_mul("bn254_fr", x, x, x, 0, 1)                     # empty
