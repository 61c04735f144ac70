"""ctypes binding of libntt_gb300.so (the C ABI declared in include/ntt_gb300.h).

Argument marshalling only: every step of a transform runs in the library's
CUDA kernels.  Buffers may be given as integers (raw device / host addresses)
or as objects with ``data_ptr()`` (torch tensors); streams as integers (a
cudaStream_t value), objects with ``cuda_stream`` (torch.cuda.Stream) or None
(legacy default stream).  The library must have been built (``_build.build``);
loading fails loudly otherwise -- there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
import re

from . import _build

NTT_OK = 0
STATUS_NAMES = {
    0: "NTT_OK", 1: "NTT_ERR_INVALID_ARG", 2: "NTT_ERR_UNSUPPORTED", 3: "NTT_ERR_OOM",
    4: "NTT_ERR_CUDA", 5: "NTT_ERR_TIMEOUT", 6: "NTT_ERR_BUDGET", 7: "NTT_ERR_NO_DEVICE", 8: "NTT_ERR_BOUNDS",
}
FIELD = {"bls12_381_fr": 0, "bn254_fr": 1, "w377": 2, "w753": 3}
KIND = {"forward": 0, "inverse": 1, "coset": 2, "coset_inverse": 3}
PATH = {"auto": 0, "butterfly": 1, "matrix": 2}
HEADER = os.path.join(_build.ROOT, "include", "ntt_gb300.h")
HEADERS = (HEADER, os.path.join(_build.ROOT, "include", "msm_gb300.h"))
CURVE = {"bn254_g1": 0, "bls12_381_g1": 1}
MAX_PASSES = 12  # NTT_MAX_PASSES


class NttError(RuntimeError):
    def __init__(self, status: int, call: str):
        self.status = status
        super().__init__(f"{call} failed: {STATUS_NAMES.get(status, status)}")


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("field", ctypes.c_uint32), ("log_n", ctypes.c_uint32), ("num_passes", ctypes.c_uint32),
        ("pass_log", ctypes.c_uint32 * MAX_PASSES), ("launches_per_transform", ctypes.c_uint32),
        ("path", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64),
        ("matrix_folded_passes", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
    ]


class ServerConfig(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_uint64), ("min_log_n", ctypes.c_uint32),
                ("max_log_n", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32),
                ("max_batch_jobs", ctypes.c_uint32), ("max_batch_elements", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("queued", ctypes.c_uint64), ("resident_bytes", ctypes.c_uint64),
                ("peak_device_bytes", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64)]


class TuneResult(ctypes.Structure):
    _fields_ = [("path", ctypes.c_uint32), ("num_passes", ctypes.c_uint32),
                ("pass_log", ctypes.c_uint32 * MAX_PASSES), ("tile_log", ctypes.c_uint32 * MAX_PASSES),
                ("candidates", ctypes.c_uint32), ("best_ms", ctypes.c_double),
                ("default_ms", ctypes.c_double)]


class BatchTuneResult(ctypes.Structure):
    _fields_ = [("split_log", ctypes.c_uint32), ("branches", ctypes.c_uint32), ("candidates", ctypes.c_uint32),
                ("best_ms", ctypes.c_double), ("persistent_ms", ctypes.c_double), ("loop_ms", ctypes.c_double)]


class MsmPlanDesc(ctypes.Structure):
    _fields_ = [("max_n", ctypes.c_uint64), ("window_bits", ctypes.c_uint32), ("num_windows", ctypes.c_uint32),
                ("segment_length", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64)]


class Job(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("kind", ctypes.c_int32), ("in_", ctypes.c_void_p),
                ("out", ctypes.c_void_p)]


_lib = None

_VP = ctypes.c_void_p
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_SIGS = {
    "ntt_plan_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _U32, ctypes.c_int]),
    "ntt_plan_set_path": (ctypes.c_int, [_VP, ctypes.c_int]),
    "ntt_plan_set_coset_shift": (ctypes.c_int, [_VP, ctypes.POINTER(_U64)]),
    "ntt_plan_destroy": (ctypes.c_int, [_VP]),
    "ntt_forward": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ntt_inverse": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ntt_coset_forward": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ntt_coset_inverse": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ntt_execute": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    "ntt_transform_host": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "ntt_transform_host_async": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "ntt_plan_describe": (ctypes.c_int, [_VP, ctypes.POINTER(PlanDesc)]),
    "ntt_plan_read_table": (ctypes.c_int, [_VP, ctypes.c_int, _U32, _U32, _U64, _U64, _VP]),
    "ntt_batch_submit": (ctypes.c_int, [ctypes.POINTER(Job), ctypes.c_size_t, _VP]),
    "ntt_batch_autotune": (ctypes.c_int, [ctypes.POINTER(Job), ctypes.c_size_t, _U32, ctypes.POINTER(BatchTuneResult)]),
    "ntt_plan_autotune": (ctypes.c_int, [_VP, _U32, ctypes.POINTER(TuneResult)]),
    "ntt_plan_set_passes": (ctypes.c_int, [_VP, _U32, ctypes.POINTER(_U32), _U32]),
    "ntt_plan_poll_error": (ctypes.c_int, [_VP, ctypes.POINTER(_U32)]),
    "ntt_build_is_debug": (ctypes.c_int, []),
    "ntt_debug_shrink_next_extent": (ctypes.c_int, [_VP]),
    "ntt_batch_submit_static": (ctypes.c_int, [ctypes.POINTER(Job), ctypes.c_size_t, _VP, _VP]),
    "ntt_batch_poll_error": (ctypes.c_int, [ctypes.POINTER(_U32)]),
    "ntt_batch_set_wait_limit": (ctypes.c_int, [_U64]),
    "ntt_batch_debug_stall": (ctypes.c_int, [ctypes.c_int]),
    "ntt_batch_cache_clear": (ctypes.c_int, []),
    "ntt_field_mont_mul": (ctypes.c_int, [ctypes.c_int, _VP, _VP, _VP, _U64, _VP]),
    "ntt_rns_basis_get": (ctypes.c_int, [ctypes.c_int, _VP]),
    "ntt_wide_transform": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _U32, _VP, _VP, _VP]),
    "ntt_wide_transform_shift": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _U32, ctypes.POINTER(_U32), _VP, _VP,
                                                _VP]),
    "ntt_field_element_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_U32)]),
    "ntt_rns_mul": (ctypes.c_int, [ctypes.c_int, _VP, _VP, _VP, _U64, _U32, _VP]),
    "ntt_rns_poll_error": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_U32)]),
    "ntt_pointwise_quotient": (ctypes.c_int, [ctypes.c_int, _VP, _VP, _VP, ctypes.POINTER(_U64), _U32, _VP, _U64,
                                              _VP]),
    "ntt_field_mont_mul_rep": (ctypes.c_int, [ctypes.c_int, _VP, _VP, _VP, _U64, _U32, ctypes.c_int, _VP]),
    "ntt_plan_enable_timing": (ctypes.c_int, [_VP, ctypes.c_int]),
    "ntt_plan_read_timing": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_U64)]),
    "ntt_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_VP)]),
    "ntt_server_submit": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _U32, _VP, _VP, ctypes.POINTER(_U64)]),
    "ntt_server_query": (ctypes.c_int, [_VP, _U64, ctypes.POINTER(ctypes.c_int)]),
    "ntt_server_wait": (ctypes.c_int, [_VP, _U64, ctypes.c_double]),
    "ntt_server_request_times": (ctypes.c_int, [_VP, _U64, ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "ntt_server_release": (ctypes.c_int, [_VP, _U64]),
    "ntt_server_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ServerStats)]),
    "ntt_server_destroy": (ctypes.c_int, [_VP]),
    "msm_point_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_U32)]),
    "msm_plan_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _U64, _U32]),
    "msm_plan_info": (ctypes.c_int, [_VP, ctypes.POINTER(MsmPlanDesc)]),
    "msm_plan_destroy": (ctypes.c_int, [_VP]),
    "msm_execute": (ctypes.c_int, [_VP, _VP, _VP, _U64, _VP, _VP]),
    "msm_poll_error": (ctypes.c_int, [_VP, ctypes.POINTER(_U32)]),
    "msm_execute_windows": (ctypes.c_int, [_VP, _VP, _VP, _U64, _U32, _U32, _VP, _VP]),
    "msm_plan_set_bases": (ctypes.c_int, [_VP, _VP, _U64, _VP]),
    "msm_execute_bases": (ctypes.c_int, [_VP, _VP, _U64, _VP, _VP]),
    "msm_fixed_base": (ctypes.c_int, [ctypes.c_int, _VP, _U64, _VP, _VP]),
    "ntt_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ntt_version": (_U32, []),
}


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libntt_gb300.so; raise if it is not built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: build the CUDA library first (__graft_entry__.build())")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def load_debug() -> ctypes.CDLL:
    """Build if needed and load the NTT_DEBUG library (bounds-checked pass
    kernels) as a separate handle with the same signatures; plans made with
    it must be used with it only."""
    lib = ctypes.CDLL(_build.build_debug())
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def declared_functions() -> list[str]:
    """Names of the functions the headers under include/ declare."""
    names: set[str] = set()
    for header in HEADERS:
        text = open(header).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*((?:ntt|msm)_[a-z0-9_]+)\s*\(",
                                text, flags=re.M))
    return sorted(names)


def _ptr(x) -> int | None:
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "__array_interface__"):
        return int(x.__array_interface__["data"][0])
    return int(x)


def _stream(s) -> int | None:
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    return int(s)


def _check(status: int, call: str) -> None:
    if status != NTT_OK:
        raise NttError(status, call)


def _field(f) -> int:
    return FIELD[f] if isinstance(f, str) else int(f)


def _kind(k) -> int:
    return KIND[k] if isinstance(k, str) else int(k)


# ----------------------------------------------------------- the C ABI calls


def ntt_plan_create(field, log_n: int, coset: bool = False) -> int:
    h = _VP()
    _check(load().ntt_plan_create(ctypes.byref(h), _field(field), int(log_n), 1 if coset else 0), "ntt_plan_create")
    return int(h.value)


def ntt_plan_set_path(plan: int, path) -> None:
    p = PATH[path] if isinstance(path, str) else int(path)
    _check(load().ntt_plan_set_path(plan, p), "ntt_plan_set_path")


def ntt_plan_set_coset_shift(plan: int, shift: int) -> None:
    arr = (_U64 * 4)(*[(shift >> (64 * i)) & (2**64 - 1) for i in range(4)])
    _check(load().ntt_plan_set_coset_shift(plan, arr), "ntt_plan_set_coset_shift")


def ntt_plan_destroy(plan: int) -> None:
    _check(load().ntt_plan_destroy(plan), "ntt_plan_destroy")


def ntt_forward(plan: int, d_in, d_out, stream=None) -> None:
    _check(load().ntt_forward(plan, _ptr(d_in), _ptr(d_out), _stream(stream)), "ntt_forward")


def ntt_inverse(plan: int, d_in, d_out, stream=None) -> None:
    _check(load().ntt_inverse(plan, _ptr(d_in), _ptr(d_out), _stream(stream)), "ntt_inverse")


def ntt_coset_forward(plan: int, d_in, d_out, stream=None) -> None:
    _check(load().ntt_coset_forward(plan, _ptr(d_in), _ptr(d_out), _stream(stream)), "ntt_coset_forward")


def ntt_coset_inverse(plan: int, d_in, d_out, stream=None) -> None:
    _check(load().ntt_coset_inverse(plan, _ptr(d_in), _ptr(d_out), _stream(stream)), "ntt_coset_inverse")


def ntt_execute(plan: int, kind, d_in, d_out, stream=None) -> None:
    _check(load().ntt_execute(plan, _kind(kind), _ptr(d_in), _ptr(d_out), _stream(stream)), "ntt_execute")


def ntt_transform_host(plan: int, kind, h_in, h_out, d_work, stream=None) -> None:
    _check(load().ntt_transform_host(plan, _kind(kind), _ptr(h_in), _ptr(h_out), _ptr(d_work), _stream(stream)),
           "ntt_transform_host")


def ntt_transform_host_async(plan: int, kind, h_in, h_out, d_work, stream=None) -> None:
    _check(load().ntt_transform_host_async(plan, _kind(kind), _ptr(h_in), _ptr(h_out), _ptr(d_work),
                                           _stream(stream)), "ntt_transform_host_async")


def ntt_plan_describe(plan: int) -> dict:
    d = PlanDesc()
    _check(load().ntt_plan_describe(plan, ctypes.byref(d)), "ntt_plan_describe")
    return {"field": d.field, "log_n": d.log_n, "num_passes": d.num_passes,
            "pass_log": list(d.pass_log)[: d.num_passes], "launches_per_transform": d.launches_per_transform,
            "path": d.path, "device_bytes": d.device_bytes, "matrix_folded_passes": d.matrix_folded_passes}


def ntt_plan_read_table(plan: int, kind, pass_index: int, table: int, first: int, count: int, h_out) -> None:
    _check(load().ntt_plan_read_table(plan, _kind(kind), pass_index, table, first, count, _ptr(h_out)),
           "ntt_plan_read_table")


def ntt_plan_autotune(plan: int, reps: int = 3) -> dict:
    r = TuneResult()
    _check(load().ntt_plan_autotune(plan, int(reps), ctypes.byref(r)), "ntt_plan_autotune")
    n = r.num_passes
    return {"path": ["auto", "butterfly", "matrix"][r.path], "num_passes": n,
            "pass_log": list(r.pass_log)[:n], "tile_log": list(r.tile_log)[:n],
            "candidates": r.candidates, "best_ms": r.best_ms, "default_ms": r.default_ms}


def ntt_plan_set_passes(plan: int, pass_log: list[int], tile_log: int = 10) -> None:
    """Rebuild the plan's butterfly path for an explicit pass split."""
    arr = (_U32 * len(pass_log))(*pass_log)
    _check(load().ntt_plan_set_passes(plan, len(pass_log), arr, int(tile_log)), "ntt_plan_set_passes")


def ntt_batch_submit(jobs, stream=None) -> None:
    """jobs: iterable of (plan, kind, d_in, d_out)."""
    jobs = list(jobs)
    arr = (Job * max(1, len(jobs)))()
    for i, (plan, kind, d_in, d_out) in enumerate(jobs):
        arr[i] = Job(plan, _kind(kind), _ptr(d_in), _ptr(d_out))
    _check(load().ntt_batch_submit(arr, len(jobs), _stream(stream)), "ntt_batch_submit")


def ntt_batch_autotune(jobs, reps: int = 3) -> dict:
    """jobs: iterable of (plan, kind, d_in, d_out); returns the chosen policy and its timings."""
    jobs = list(jobs)
    arr = (Job * max(1, len(jobs)))()
    for i, (plan, kind, x, y) in enumerate(jobs):
        arr[i] = Job(plan, _kind(kind), _ptr(x), _ptr(y))
    r = BatchTuneResult()
    _check(load().ntt_batch_autotune(arr, len(jobs), int(reps), ctypes.byref(r)), "ntt_batch_autotune")
    return {"split_log": r.split_log, "branches": r.branches, "candidates": r.candidates, "best_ms": r.best_ms,
            "persistent_ms": r.persistent_ms, "loop_ms": r.loop_ms}


def ntt_batch_submit_static(jobs, d_status=None, stream=None) -> None:
    """jobs: iterable of (plan, kind, d_in, d_out); d_status: device uint32 or None."""
    jobs = list(jobs)
    arr = (Job * max(1, len(jobs)))()
    for i, (plan, kind, d_in, d_out) in enumerate(jobs):
        arr[i] = Job(plan, _kind(kind), _ptr(d_in), _ptr(d_out))
    _check(load().ntt_batch_submit_static(arr, len(jobs), _ptr(d_status), _stream(stream)), "ntt_batch_submit_static")


def ntt_batch_poll_error() -> int:
    code = _U32()
    _check(load().ntt_batch_poll_error(ctypes.byref(code)), "ntt_batch_poll_error")
    return int(code.value)


def ntt_batch_set_wait_limit(ns: int) -> None:
    _check(load().ntt_batch_set_wait_limit(int(ns)), "ntt_batch_set_wait_limit")


def ntt_batch_debug_stall(enable: bool) -> None:
    _check(load().ntt_batch_debug_stall(1 if enable else 0), "ntt_batch_debug_stall")


def ntt_batch_cache_clear() -> None:
    _check(load().ntt_batch_cache_clear(), "ntt_batch_cache_clear")


def ntt_plan_poll_error(plan: int) -> int:
    code = _U32()
    _check(load().ntt_plan_poll_error(plan, ctypes.byref(code)), "ntt_plan_poll_error")
    return int(code.value)


def ntt_field_mont_mul(field, d_a, d_b, d_out, count: int, stream=None) -> None:
    _check(load().ntt_field_mont_mul(_field(field), _ptr(d_a), _ptr(d_b), _ptr(d_out), int(count), _stream(stream)),
           "ntt_field_mont_mul")


def ntt_pointwise_quotient(field, d_a, d_b, d_c, z_values, d_out, count: int, stream=None) -> None:
    """out[i] = (a[i] b[i] - c[i]) z[i mod len(z)]; z_values: Python ints (host)."""
    z = [int(v) for v in z_values]
    arr = (_U64 * (4 * max(1, len(z))))()
    for j, v in enumerate(z):
        for k in range(4):
            arr[4 * j + k] = (v >> (64 * k)) & 0xFFFFFFFFFFFFFFFF
    _check(load().ntt_pointwise_quotient(_field(field), _ptr(d_a), _ptr(d_b), _ptr(d_c), arr, len(z), _ptr(d_out),
                                         int(count), _stream(stream)), "ntt_pointwise_quotient")


def ntt_wide_transform(field, kind, log_n: int, d_in, d_out, stream=None, shift: int | None = None) -> None:
    """377/753-bit transform; ``shift`` (an int, coset kinds only) replaces
    the generator as the coset shift."""
    if shift is None:
        _check(load().ntt_wide_transform(_field(field), _kind(kind), int(log_n), _ptr(d_in), _ptr(d_out),
                                         _stream(stream)), "ntt_wide_transform")
        return
    words = 12 if _field(field) == FIELD["w377"] else 24
    s = int(shift)
    if s < 0 or s >= 1 << (32 * words):
        raise ValueError("shift does not fit the field's words")
    arr = (_U32 * 24)(*[(s >> (32 * i)) & 0xFFFFFFFF for i in range(24)])
    _check(load().ntt_wide_transform_shift(_field(field), _kind(kind), int(log_n), arr, _ptr(d_in), _ptr(d_out),
                                           _stream(stream)), "ntt_wide_transform_shift")


def ntt_field_element_bytes(field) -> int:
    b = _U32(0)
    _check(load().ntt_field_element_bytes(_field(field), ctypes.byref(b)), "ntt_field_element_bytes")
    return int(b.value)


class RnsBasis(ctypes.Structure):
    _fields_ = [("num_q", _U32), ("num_p", _U32), ("words_per_element", _U32), ("shift", _U32),
                ("q", _U32 * 24), ("p", _U32 * 16)]


def ntt_rns_basis_get(field) -> dict:
    b = RnsBasis()
    _check(load().ntt_rns_basis_get(_field(field), ctypes.byref(b)), "ntt_rns_basis_get")
    return {"q": list(b.q[: b.num_q]), "p": list(b.p[: b.num_p]), "words_per_element": b.words_per_element,
            "shift": b.shift}


def ntt_rns_mul(field, d_x, d_y, d_out, count: int, reps: int = 1, stream=None) -> None:
    _check(load().ntt_rns_mul(_field(field), _ptr(d_x), _ptr(d_y), _ptr(d_out), int(count), int(reps),
                              _stream(stream)), "ntt_rns_mul")


def ntt_rns_poll_error(field) -> int:
    code = _U32(0)
    _check(load().ntt_rns_poll_error(_field(field), ctypes.byref(code)), "ntt_rns_poll_error")
    return int(code.value)


def ntt_plan_enable_timing(plan: int, enable: bool = True) -> None:
    _check(load().ntt_plan_enable_timing(plan, 1 if enable else 0), "ntt_plan_enable_timing")


def ntt_plan_read_timing(plan: int) -> tuple[list[float], list[int]]:
    """(summed ms per pass, launches per pass) since the last read."""
    ms = (ctypes.c_double * MAX_PASSES)()
    cnt = (_U64 * MAX_PASSES)()
    _check(load().ntt_plan_read_timing(plan, ms, cnt), "ntt_plan_read_timing")
    return list(ms), list(cnt)


def ntt_server_create(memory_budget_bytes: int = 0, min_log_n: int = 0, max_log_n: int = 0,
                      max_inflight: int = 0, max_batch_jobs: int = 0, max_batch_elements: int = 0) -> int:
    cfg = ServerConfig(memory_budget_bytes, min_log_n, max_log_n, max_inflight, max_batch_jobs, max_batch_elements)
    h = _VP()
    _check(load().ntt_server_create(ctypes.byref(cfg), ctypes.byref(h)), "ntt_server_create")
    return int(h.value)


def ntt_server_submit(server: int, field, kind, log_n: int, h_in, h_out) -> int:
    t = _U64()
    _check(load().ntt_server_submit(server, _field(field), _kind(kind), int(log_n), _ptr(h_in), _ptr(h_out),
                                    ctypes.byref(t)), "ntt_server_submit")
    return int(t.value)


def ntt_server_query(server: int, ticket: int) -> bool:
    d = ctypes.c_int()
    _check(load().ntt_server_query(server, ticket, ctypes.byref(d)), "ntt_server_query")
    return bool(d.value)


def ntt_server_wait(server: int, ticket: int, timeout_s: float = 0.0) -> None:
    _check(load().ntt_server_wait(server, ticket, float(timeout_s)), "ntt_server_wait")


def ntt_server_request_times(server: int, ticket: int) -> tuple[float, float, float]:
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().ntt_server_request_times(server, ticket, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "ntt_server_request_times")
    return a.value, b.value, c.value


def ntt_server_release(server: int, ticket: int) -> None:
    _check(load().ntt_server_release(server, ticket), "ntt_server_release")


def ntt_server_get_stats(server: int) -> dict:
    st = ServerStats()
    _check(load().ntt_server_get_stats(server, ctypes.byref(st)), "ntt_server_get_stats")
    return {k: int(getattr(st, k)) for k, _ in ServerStats._fields_}


def ntt_server_destroy(server: int) -> None:
    _check(load().ntt_server_destroy(server), "ntt_server_destroy")


def ntt_field_mont_mul_rep(field, d_a, d_b, d_out, count: int, reps: int, variant: int, stream=None) -> None:
    _check(load().ntt_field_mont_mul_rep(_field(field), _ptr(d_a), _ptr(d_b), _ptr(d_out), int(count), int(reps),
                                         int(variant), _stream(stream)), "ntt_field_mont_mul_rep")


def _curve(c) -> int:
    return CURVE[c] if isinstance(c, str) else int(c)


def msm_point_bytes(curve) -> int:
    b = _U32(0)
    _check(load().msm_point_bytes(_curve(curve), ctypes.byref(b)), "msm_point_bytes")
    return int(b.value)


def msm_plan_create(curve, max_n: int, window_bits: int = 0) -> int:
    h = _VP()
    _check(load().msm_plan_create(ctypes.byref(h), _curve(curve), int(max_n), int(window_bits)), "msm_plan_create")
    return int(h.value)


def msm_plan_info(plan: int) -> dict:
    d = MsmPlanDesc()
    _check(load().msm_plan_info(plan, ctypes.byref(d)), "msm_plan_info")
    return {"max_n": d.max_n, "window_bits": d.window_bits, "num_windows": d.num_windows,
            "segment_length": d.segment_length, "device_bytes": d.device_bytes}


def msm_plan_destroy(plan: int) -> None:
    _check(load().msm_plan_destroy(plan), "msm_plan_destroy")


def msm_execute(plan: int, d_scalars, d_points, count: int, d_result, stream=None) -> None:
    _check(load().msm_execute(plan, _ptr(d_scalars), _ptr(d_points), int(count), _ptr(d_result), _stream(stream)),
           "msm_execute")


def msm_execute_windows(plan: int, d_scalars, d_points, count: int, window_begin: int, window_end: int,
                        d_result, stream=None) -> None:
    _check(load().msm_execute_windows(plan, _ptr(d_scalars), _ptr(d_points), int(count), int(window_begin),
                                      int(window_end), _ptr(d_result), _stream(stream)), "msm_execute_windows")


def msm_plan_set_bases(plan: int, d_points, count: int, stream=None) -> None:
    _check(load().msm_plan_set_bases(plan, _ptr(d_points), int(count), _stream(stream)), "msm_plan_set_bases")


def msm_execute_bases(plan: int, d_scalars, count: int, d_result, stream=None) -> None:
    _check(load().msm_execute_bases(plan, _ptr(d_scalars), int(count), _ptr(d_result), _stream(stream)),
           "msm_execute_bases")


def msm_poll_error(plan: int) -> int:
    flags = _U32(0)
    _check(load().msm_poll_error(plan, ctypes.byref(flags)), "msm_poll_error")
    return int(flags.value)


def msm_fixed_base(curve, d_scalars, count: int, d_points, stream=None) -> None:
    _check(load().msm_fixed_base(_curve(curve), _ptr(d_scalars), int(count), _ptr(d_points), _stream(stream)),
           "msm_fixed_base")


def ntt_status_string(status: int) -> str:
    return load().ntt_status_string(int(status)).decode()


def ntt_version() -> int:
    return int(load().ntt_version())
