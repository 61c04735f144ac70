"""GB300 (sm_103a) 255-bit number-theoretic transform library.

The compute path is libntt_gb300.so (hand-written CUDA, C ABI in
include/ntt_gb300.h); this package is its thin Python binding:

  * ``_native``  -- ctypes wrappers named like the C calls;
  * ``_build``   -- the nvcc build of the library;
  * ``Plan``     -- a small owner object over a plan handle for torch users;
  * ``MsmPlan``  -- the same for the multi-scalar multiplication on BN254 G1
                    or BLS12-381 G1 (C ABI in include/msm_gb300.h);
  * ``msm_shard`` -- the MSM with its windows shared out over ranks.

Importing the package does not load CUDA; the first call does, and raises if
the library has not been built.
"""

from __future__ import annotations

from . import _build, _native  # noqa: F401
from ._native import (  # noqa: F401
    FIELD,
    KIND,
    CURVE,
    PATH,
    NttError,
    msm_execute,
    msm_execute_bases,
    msm_execute_windows,
    msm_fixed_base,
    msm_plan_create,
    msm_point_bytes,
    msm_plan_destroy,
    msm_plan_info,
    msm_plan_set_bases,
    msm_poll_error,
    ntt_batch_submit,
    ntt_coset_forward,
    ntt_coset_inverse,
    ntt_execute,
    ntt_field_mont_mul,
    ntt_forward,
    ntt_inverse,
    ntt_plan_create,
    ntt_plan_describe,
    ntt_plan_destroy,
    ntt_plan_poll_error,
    ntt_plan_read_table,
    ntt_plan_set_coset_shift,
    ntt_plan_set_path,
    ntt_pointwise_quotient,
    ntt_status_string,
    ntt_transform_host,
    ntt_version,
)


class Plan:
    """Owns one ntt_plan handle; buffers are torch int64 tensors of shape [N, 4]."""

    def __init__(self, field, log_n: int, coset: bool = False, path: str | None = None):
        self.field = field
        self.log_n = int(log_n)
        self.n = 1 << self.log_n
        self.handle = ntt_plan_create(field, self.log_n, coset)
        if path is not None:
            ntt_plan_set_path(self.handle, path)

    def run(self, kind, x, out=None, stream=None):
        if out is None:
            out = x.new_empty(x.shape)
        ntt_execute(self.handle, kind, x, out, stream)
        return out

    def forward(self, x, out=None, stream=None):
        return self.run("forward", x, out, stream)

    def inverse(self, x, out=None, stream=None):
        return self.run("inverse", x, out, stream)

    def coset_forward(self, x, out=None, stream=None):
        return self.run("coset", x, out, stream)

    def coset_inverse(self, x, out=None, stream=None):
        return self.run("coset_inverse", x, out, stream)

    def describe(self) -> dict:
        return ntt_plan_describe(self.handle)

    def close(self) -> None:
        if self.handle:
            ntt_plan_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MsmPlan:
    """Owns one msm_plan handle.  Scalars: torch int64 [n, 4]; points:
    [n, 2 w] with w = 4 (BN254) or 6 (BLS12-381) 64-bit limbs per coordinate
    (affine x limbs then y limbs, standard form, (0, 0) = infinity); the
    result is one point, [2 w]."""

    def __init__(self, max_n: int, window_bits: int = 0, curve: str = "bn254_g1"):
        self.curve = curve
        self.max_n = int(max_n)
        self.point_words = msm_point_bytes(curve) // 8
        self.handle = msm_plan_create(curve, self.max_n, window_bits)

    def info(self) -> dict:
        return msm_plan_info(self.handle)

    def execute(self, scalars, points, out=None, count: int | None = None, stream=None):
        n = scalars.shape[0] if count is None else int(count)
        if out is None:
            out = scalars.new_empty((self.point_words,))
        msm_execute(self.handle, scalars, points, n, out, stream)
        return out

    def execute_windows(self, scalars, points, window_begin: int, window_end: int, out=None,
                        count: int | None = None, stream=None):
        """sum over windows [begin, end) of 2^(k c) W_k (see msm_execute_windows)."""
        n = scalars.shape[0] if count is None else int(count)
        if out is None:
            out = scalars.new_empty((self.point_words,))
        msm_execute_windows(self.handle, scalars, points, n, window_begin, window_end, out, stream)
        return out

    def set_bases(self, points, count: int | None = None, stream=None) -> None:
        """Precompute the window copies of fixed points (msm_plan_set_bases)."""
        msm_plan_set_bases(self.handle, points, points.shape[0] if count is None else int(count), stream)

    def execute_bases(self, scalars, out=None, count: int | None = None, stream=None):
        """sum_n scalars[n] P_n over the points given to set_bases."""
        n = scalars.shape[0] if count is None else int(count)
        if out is None:
            out = scalars.new_empty((self.point_words,))
        msm_execute_bases(self.handle, scalars, n, out, stream)
        return out

    def poll_error(self) -> int:
        return msm_poll_error(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            msm_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fixed_base_points(scalars, out=None, stream=None, curve: str = "bn254_g1"):
    """points[n] = scalars[n] G on the curve's generator (input generation for MSM)."""
    if out is None:
        out = scalars.new_empty((scalars.shape[0], msm_point_bytes(curve) // 8))
    msm_fixed_base(curve, scalars, scalars.shape[0], out, stream)
    return out
