"""The C-ABI library loads and exports every function include/ntt_gb300.h
declares; argument checks that need no GPU behave as documented."""

from __future__ import annotations

import ctypes

import pytest

from paper_2604_17808_gb300 import _build, _native


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _native.load()


def test_header_declares_the_boundary():
    names = _native.declared_functions()
    for required in ("ntt_plan_create", "ntt_plan_set_path", "ntt_plan_set_coset_shift", "ntt_plan_destroy",
                     "ntt_forward", "ntt_inverse", "ntt_coset_forward", "ntt_coset_inverse", "ntt_batch_submit",
                     "ntt_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = _native.declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), f"{name} declared in the header but not exported"
        assert name in _native._SIGS, f"{name} has no Python binding"


def test_status_strings_and_version(lib):
    for code, name in _native.STATUS_NAMES.items():
        assert _native.ntt_status_string(code) == name
    assert _native.ntt_status_string(99) == "NTT_ERR_UNKNOWN"
    assert _native.ntt_version() >= 100


def test_plan_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.ntt_plan_create(None, 0, 12, 0) == 1
    assert lib.ntt_plan_create(ctypes.byref(h), 5, 12, 0) == 1
    assert lib.ntt_plan_create(ctypes.byref(h), 0, 0, 0) == 2
    assert lib.ntt_plan_create(ctypes.byref(h), 0, 29, 0) == 2
    assert lib.ntt_plan_create(ctypes.byref(h), 1, 29, 0) == 2  # BN254 2-adicity is 28
    assert lib.ntt_plan_create(ctypes.byref(h), 2, 12, 0) == 1  # the wide fields use ntt_wide_transform
    b = ctypes.c_uint32(0)
    assert lib.ntt_field_element_bytes(3, ctypes.byref(b)) == 0 and b.value == 96
    assert lib.ntt_field_element_bytes(4, ctypes.byref(b)) == 1
    assert h.value is None


def test_wide_transform_rejects_bad_arguments_without_touching_the_gpu(lib):
    buf = (ctypes.c_uint64 * 64)()
    p = ctypes.addressof(buf)
    assert lib.ntt_wide_transform(0, 0, 4, p, p, None) == 1    # a 256-bit field: use the plans
    assert lib.ntt_wide_transform(2, 4, 4, p, p, None) == 1    # no such kind
    assert lib.ntt_wide_transform(3, 0, 0, p, p, None) == 2    # sizes 2^1 .. 2^24
    assert lib.ntt_wide_transform(3, 3, 25, p, p, None) == 2
    assert lib.ntt_wide_transform(2, 2, 4, None, p, None) == 1
    assert lib.ntt_wide_transform(2, 2, 4, p + 8, p, None) == 1  # 16-byte alignment


def test_wide_shift_is_checked_without_touching_the_gpu(lib):
    buf = (ctypes.c_uint64 * 64)()
    p = ctypes.addressof(buf)
    W = ctypes.c_uint32 * 24
    p377 = 0x1921FB54442D18469898CC51701B839A252049C1114CF98E804177D4C76273644A29410F31C6809BBDF2BD500000001
    words = lambda v: W(*[(v >> (32 * i)) & 0xFFFFFFFF for i in range(24)])  # noqa: E731
    assert lib.ntt_wide_transform_shift(2, 2, 4, None, p, p, None) == 1             # no shift
    assert lib.ntt_wide_transform_shift(2, 2, 4, words(0), p, p, None) == 1         # s = 0
    assert lib.ntt_wide_transform_shift(2, 3, 4, words(p377), p, p, None) == 1      # s = p
    assert lib.ntt_wide_transform_shift(2, 3, 4, words(p377 + 5), p, p, None) == 1  # s > p
    assert lib.ntt_wide_transform_shift(2, 0, 4, words(3), p, p, None) == 1         # not a coset kind
    assert lib.ntt_wide_transform_shift(0, 2, 4, words(3), p, p, None) == 1         # a 256-bit field
    assert lib.ntt_wide_transform_shift(3, 2, 0, words(3), p, p, None) == 2


def test_null_plan_calls_are_rejected(lib):
    assert lib.ntt_forward(None, None, None, None) == 1
    assert lib.ntt_execute(None, 0, None, None, None) == 1
    assert lib.ntt_plan_destroy(None) == 0
    assert lib.ntt_batch_submit(None, 0, None) == 0
    assert lib.ntt_field_mont_mul(3, None, None, None, 1, None) == 1


def test_no_gpu_is_reported_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.ntt_plan_create(ctypes.byref(h), 0, 12, 0) == 7  # NTT_ERR_NO_DEVICE
    with pytest.raises(_native.NttError):
        _native.ntt_plan_create("bls12_381_fr", 12)


def test_msm_arguments_are_checked_without_touching_the_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.msm_plan_create(None, 0, 16, 0) == 1
    assert lib.msm_plan_create(ctypes.byref(h), 2, 16, 0) == 1          # unknown curve
    b = ctypes.c_uint32(0)
    assert lib.msm_point_bytes(0, ctypes.byref(b)) == 0 and b.value == 64
    assert lib.msm_point_bytes(1, ctypes.byref(b)) == 0 and b.value == 96
    assert lib.msm_point_bytes(2, ctypes.byref(b)) == 1
    assert lib.msm_plan_create(ctypes.byref(h), 0, (1 << 28) + 1, 0) == 2  # above MSM_MAX_POINTS
    assert lib.msm_plan_create(ctypes.byref(h), 0, 16, 23) == 2         # window too wide
    assert lib.msm_plan_create(ctypes.byref(h), 0, 1 << 25, 1) == 2     # 254 windows x 2^25 > 2^32 indices
    assert h.value is None
    assert lib.msm_execute(None, None, None, 0, None, None) == 1
    assert lib.msm_plan_destroy(None) == 1
    assert lib.msm_plan_info(None, None) == 1
    assert lib.msm_poll_error(None, None) == 1
    assert lib.msm_execute_windows(None, None, None, 0, 0, 0, None, None) == 1
    assert lib.msm_plan_set_bases(None, None, 0, None) == 1
    assert lib.msm_execute_bases(None, None, 0, None, None) == 1
    assert lib.msm_fixed_base(3, None, 4, None, None) == 1
    assert lib.msm_fixed_base(1, None, 4, None, None) == 1
    assert lib.msm_fixed_base(0, None, 0, None, None) == 0              # nothing to do
    assert lib.msm_fixed_base(0, None, 4, None, None) == 1


def test_msm_no_gpu_is_reported_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.msm_plan_create(ctypes.byref(h), 0, 1024, 0) == 7  # NTT_ERR_NO_DEVICE
