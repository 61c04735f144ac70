"""CPU oracle for the 255-bit NTT (forward, inverse, coset, coset inverse).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  The
product library (``paper_2604_17808_gb300``) never imports it, and it never
imports the product library.

Two independent implementations of the same definition (MORPH Sec. 2.3.1):
  * ``ntt_oracle`` -- Python big integers (the definition written out, plus a
    textbook radix-2 evaluation of it);
  * ``ntt_oracle.c`` -- plain C, 4 x 64-bit limbs, HAC 14.36 Montgomery, used
    where Python is too slow (2^20 and 2^24 elements), loaded by ``c_oracle()``.

Companions: ``rns_oracle`` (the paper's RNS lazy modular multiplication) and
``msm_oracle`` (multi-scalar multiplication on BN254 G1: the definition and
the paper's Layout-Stationary Pippenger).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import ntt_oracle
from .ntt_oracle import (  # noqa: F401  (re-exported)
    BLS12_381_FR,
    BN254_FR,
    FIELD_BY_INDEX,
    FIELDS,
    coset_intt,
    coset_ntt,
    dft_direct,
    get_field,
    horner,
    ints_to_limbs,
    intt,
    limbs_to_ints,
    ntt,
    quotient_pointwise,
    root_of_unity,
    transform,
)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ntt_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_ntt.so")
_lock = threading.Lock()
_lib = None

KIND = {"forward": 0, "inverse": 1, "coset": 2, "coset_inverse": 3}


def build_c_oracle(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no -march, portable to Arm;
    OpenMP for its optional all-cores mode, without it if gcc lacks it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC]
    if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def c_oracle():
    """Load (building if needed) the C oracle; returns the ctypes CDLL."""
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_c_oracle())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.oracle_ntt.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint, u64p, u64p, u64p]
            lib.oracle_ntt.restype = ctypes.c_int
            lib.oracle_eval.argtypes = [ctypes.c_int, ctypes.c_uint64, u64p, u64p, u64p]
            lib.oracle_eval.restype = ctypes.c_int
            lib.oracle_root.argtypes = [ctypes.c_int, ctypes.c_uint, u64p]
            lib.oracle_root.restype = ctypes.c_int
            lib.oracle_mul.argtypes = [ctypes.c_int, u64p, u64p, u64p]
            lib.oracle_mul.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def c_set_threads(k: int) -> int:
    """Threads of the C oracle's butterfly stages from now on (1 = serial,
    0 = all cores); returns the count in use (1 without OpenMP)."""
    return int(c_oracle().oracle_set_threads(int(k)))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _field_index(field) -> int:
    return FIELD_BY_INDEX.index(get_field(field))


def c_transform(field, kind: str, x: np.ndarray, shift: int | None = None) -> np.ndarray:
    """C oracle: transform of x ([n, 4] uint64 limbs, n a power of two)."""
    x = np.ascontiguousarray(x, dtype=np.uint64).reshape(-1, 4)
    n = x.shape[0]
    log_n = n.bit_length() - 1
    if n != 1 << log_n:
        raise ValueError("length must be a power of two")
    out = np.empty_like(x)
    sp = None
    if shift is not None:
        sa = ints_to_limbs([shift % get_field(field).modulus])
        sp = _ptr(sa)
    rc = c_oracle().oracle_ntt(_field_index(field), KIND[kind], log_n, sp, _ptr(x), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_ntt failed with code {rc}")
    return out


def c_eval(field, coeffs: np.ndarray, z: int) -> int:
    """C oracle: sum_i coeffs[i] z^i (Horner) for one point z."""
    coeffs = np.ascontiguousarray(coeffs, dtype=np.uint64).reshape(-1, 4)
    za = ints_to_limbs([z % get_field(field).modulus])
    out = np.zeros((1, 4), dtype=np.uint64)
    rc = c_oracle().oracle_eval(_field_index(field), coeffs.shape[0], _ptr(coeffs), _ptr(za), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_eval failed with code {rc}")
    return limbs_to_ints(out)[0]


def c_root(field, log_n: int) -> int:
    out = np.zeros((1, 4), dtype=np.uint64)
    rc = c_oracle().oracle_root(_field_index(field), log_n, _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_root failed with code {rc}")
    return limbs_to_ints(out)[0]
