"""Build the CUDA library libntt_gb300.so in-tree with nvcc for sm_103a.

Each translation unit is compiled in its own nvcc process (in parallel), then
linked with ``nvcc -shared``.  Output: ``paper_2604_17808_gb300/_lib/``.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
OBJ_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libntt_gb300.so"
LIB_PATH = os.path.join(OUT_DIR, LIB_NAME)
# Debug build (NTT_DEBUG): bounds checks in the butterfly pass kernels.  Only
# the translation units that hold them (and the plan code with the debug
# hooks) are compiled again; the rest are the release objects.
DEBUG_LIB_PATH = os.path.join(OUT_DIR, "libntt_gb300_debug.so")
DEBUG_OBJ_DIR = os.path.join(HERE, "_build_debug")
DEBUG_UNITS = ("ntt_plan.cu", "kernels_bls12_381_pass10.cu", "kernels_bls12_381_pass11.cu",
               "kernels_bls12_381_batch.cu", "kernels_bn254_pass10.cu", "kernels_bn254_pass11.cu",
               "kernels_bn254_batch.cu")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE, "-I", CSRC]


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return [f for f in files if os.path.isfile(f)] + [os.path.abspath(__file__)]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libntt_gb300.so")


def is_stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile (if stale or forced) and return the path of libntt_gb300.so."""
    if not force and not is_stale():
        return LIB_PATH
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(OBJ_DIR, exist_ok=True)
    cc = nvcc()
    srcs = sources()

    def compile_one(src: str) -> str:
        obj = os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    workers = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def build_debug(force: bool = False, jobs: int | None = None) -> str:
    """Build (after the release build) and return the path of the NTT_DEBUG library."""
    build()
    deps_t = max(os.path.getmtime(f) for f in _deps())
    if not force and os.path.exists(DEBUG_LIB_PATH) and os.path.getmtime(DEBUG_LIB_PATH) > deps_t:
        return DEBUG_LIB_PATH
    os.makedirs(DEBUG_OBJ_DIR, exist_ok=True)
    cc = nvcc()

    def compile_one(unit: str) -> str:
        obj = os.path.join(DEBUG_OBJ_DIR, unit[:-3] + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, "-DNTT_DEBUG", "-c", os.path.join(CSRC, unit), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {unit} (NTT_DEBUG):\n{r.stdout}\n{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(DEBUG_UNITS), os.cpu_count() or 4)) as ex:
        dbg_objs = list(ex.map(compile_one, DEBUG_UNITS))
    rel_objs = [os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + ".o") for src in sources()
                if os.path.basename(src) not in DEBUG_UNITS]
    tmp = DEBUG_LIB_PATH + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *rel_objs, *dbg_objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed (NTT_DEBUG):\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, DEBUG_LIB_PATH)
    return DEBUG_LIB_PATH


if __name__ == "__main__":
    import sys

    if "--debug" in sys.argv:
        print(build_debug(force="--force" in sys.argv))
    else:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
