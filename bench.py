#!/usr/bin/env python
"""Throughput benchmark of the GB300 255-bit NTT library.

Workload (one step): forward NTT then inverse NTT of one vector of 2^20
BLS12-381 Fr elements (uniform from seed, standard form, natural order), on
the butterfly path, inputs resident in HBM.  Steps rotate over 8 distinct
input vectors (768 MiB of inputs, outputs and round trips), so no step finds
its data in the 129 MB L2.

Metric: NTT field elements transformed per second (each transform of N
elements counts N), whole job over all ranks.

Printed as ONE JSON line on rank 0, with
  * roofline: the dominant kernel (the pass kernel with the largest device
    time) against the 32-bit integer multiply-add (IMAD) pipe:
    algorithmic IMAD per launch = modmuls of the pass * 272 (one 8-limb CIOS
    Montgomery product, lo and hi multiplies counted), modmuls of a pass =
    (N/2) log2 S (radix-2 butterflies) + N (the pass's per-element multiplier
    when it has one); peak = 152 SMs * 64 IMAD/clk * 2.07 GHz;
  * e2e: the same metric through ntt_transform_host (pinned host buffers,
    host-to-device and device-to-host copies inside the timed region);
  * cpu_baseline: the C oracle on this host's cores on a bounded sample of
    the same workload: single-threaded (the value) and with each stage's
    butterflies over every core (all_cores, plus one 2^24 transform), with
    the host's core count;
  * secondary: the 2^24-point BLS12-381 forward NTT (elements/s and IMAD
    roofline fraction of the whole transform), 2^28, the BN254 2^24 coset
    transform on both paths, the wider fields, the batched workload (64
    forward NTTs of 2^14..2^22 points) as one persistent launch vs one
    transform per call, the multiply alone, a prover's quotient step, and
    the serving sweep (five offered rates, sampled results compared with
    the same transform run alone); the MSM and commitment legs run only
    with --leg;
  * clocks: nvidia-smi samples taken during the timed region.

``--impl reference`` times the oracle instead (rank 0 only), the baseline
the comparison of the two arms uses.
"""

from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from ntt_synth import MODULI as MODULI_R, config_seed, uniform_elements  # noqa: E402

METRIC = "255-bit NTT field elements/s (BLS12-381 Fr, n=2^20, forward+inverse, butterfly path)"
UNIT = "elements/s"
IMAD_PER_MODMUL = 272
SMS = 152
IMAD_PER_CLK_PER_SM = 64
SM_MAX_MHZ = 2070.0
FIELD = "bls12_381_fr"
LOG_N = 20
ROTATE = 8
SERVING_RATES = (100, 300, 1000, 3000, 5000)  # offered jobs/s of the serving sweep
L2_NOTE = "inputs larger than L2: 8 rotating 2^20 vectors (in, out, round trip: 768 MiB)"


def peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except OSError:
        return {}


def imad_peak_tops() -> float:
    """Tera IMAD/s: SMs x IMAD lanes per clock x maximum SM clock."""
    mhz = peaks().get("sm_max_mhz", SM_MAX_MHZ)
    return SMS * IMAD_PER_CLK_PER_SM * mhz * 1e6 / 1e12


KERNEL_SOURCES = ("paper_2604_17808_gb300/csrc/fp256.cuh", "paper_2604_17808_gb300/csrc/ntt_pass.cuh",
                  "paper_2604_17808_gb300/csrc/ntt_kernels.inl")
PROFILE_2_20 = os.path.join(ROOT, "profiles", "ntt_pass_kernel_bls12_381_2_20.md")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_tag: str) -> int | None:
    """DRAM bytes per launch of `kernel_tag` from the committed ncu summary,
    if it was captured from the current kernel sources (else None)."""
    try:
        text = open(PROFILE_2_20).read()
    except OSError:
        return None
    src = None
    traffic = None
    for line in text.splitlines():
        if line.startswith("source_sha256:"):
            src = line.split(":", 1)[1].strip()
        if line.startswith(f"traffic_bytes_per_launch[{kernel_tag}]:"):
            traffic = int(line.split(":", 1)[1].strip())
    return traffic if src == kernel_source_hash() else None


def pass_modmuls(log_n: int, pass_log: list[int], j: int, has_multiplier: bool) -> int:
    n = 1 << log_n
    return (n // 2) * pass_log[j] + (n if has_multiplier else 0)


def transform_modmuls(log_n: int) -> int:
    """Algorithmic modmuls of one transform: (N/2) log2 N butterflies + 2N."""
    n = 1 << log_n
    return (n // 2) * log_n + 2 * n


# ----------------------------------------------------------------- clocks


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.close()
        rows = []
        with open(self.tmp.name) as fh:
            for r in csv.reader(fh):
                if len(r) >= 9:
                    rows.append([c.strip() for c in r])
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------ distributed


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world: int, backend: str):
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(backend=backend)


def dist_max(value: float, world: int, device) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ----------------------------------------------------------- our arm


def to_dev(torch, a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def timed_loop(torch, N, plan, bufs, steps: int, stream) -> float:
    """Time `steps` forward+inverse steps with CUDA events on `stream`; ms."""
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(steps):
        x, y, z = bufs[i % len(bufs)]
        N.ntt_forward(plan, x, y, stream)
        N.ntt_inverse(plan, y, z, stream)
    stop.record(stream)
    stop.synchronize()
    return start.elapsed_time(stop)


def step_times(torch, N, plan, bufs, steps: int, stream) -> list[float]:
    """The same steps once more with a CUDA event pair around each one (on
    `stream`): per-step times in ms, for the median."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i, (a, b) in enumerate(evs):
        x, y, z = bufs[i % len(bufs)]
        a.record(stream)
        N.ntt_forward(plan, x, y, stream)
        N.ntt_inverse(plan, y, z, stream)
        b.record(stream)
    evs[-1][1].synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def timed_loop_streams(torch, N, plan, bufs, steps: int, stream, nstreams: int) -> float:
    """The same steps with consecutive (independent) steps alternating over
    `nstreams` streams, so that one step's last pass overlaps the next step's
    first; CUDA events on `stream`, the other streams joined before the stop
    event.  ms for all steps."""
    others = [torch.cuda.Stream() for _ in range(nstreams - 1)]
    streams = [stream] + others
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for s in others:
        s.wait_event(start)
    for i in range(steps):
        s = streams[i % nstreams]
        x, y, z = bufs[i % len(bufs)]
        N.ntt_forward(plan, x, y, s)
        N.ntt_inverse(plan, y, z, s)
    for s in others:
        ev = torch.cuda.Event()
        ev.record(s)
        stream.wait_event(ev)
    stop.record(stream)
    stop.synchronize()
    return start.elapsed_time(stop)


def golden_digest(kind: str) -> str | None:
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_digests.json")) as fh:
            for c in json.load(fh)["single"]:
                if c["config"] == 2 and c["kind"] == kind:
                    return c["output_sha256"]
    except OSError:
        return None
    return None


def measure_2_24(torch, N, stream, steps: int) -> dict:
    log_n = 24
    plan = N.ntt_plan_create(FIELD, log_n)
    try:
        desc = N.ntt_plan_describe(plan)
        xs = [to_dev(torch, uniform_elements(FIELD, 1 << log_n, config_seed(3, 200 + r))) for r in range(2)]
        ys = [torch.empty_like(x) for x in xs]
        for i in range(2):
            N.ntt_forward(plan, xs[i], ys[i], stream)
        torch.cuda.synchronize()
        N.ntt_plan_enable_timing(plan, True)
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for i in range(steps):
            N.ntt_forward(plan, xs[i % 2], ys[i % 2], stream)
        stop.record(stream)
        stop.synchronize()
        ms = start.elapsed_time(stop) / steps
        pass_ms, pass_cnt = N.ntt_plan_read_timing(plan)
        N.ntt_plan_enable_timing(plan, False)
        peak = imad_peak_tops()
        alg = transform_modmuls(log_n) * IMAD_PER_MODMUL
        per_pass = []
        for j, ls in enumerate(desc["pass_log"]):
            avg = pass_ms[j] / max(1, pass_cnt[j])
            mm = pass_modmuls(log_n, desc["pass_log"], j, j >= 1)
            per_pass.append({"pass": j, "log_s": ls, "avg_ms": round(avg, 4),
                             "frac": round(mm * IMAD_PER_MODMUL / (avg * 1e-3) / 1e12 / peak, 4)})
        # the same transform on the matrix (tensor-core) path, outputs compared
        N.ntt_plan_set_path(plan, "matrix")
        ym = torch.empty_like(ys[0])
        N.ntt_forward(plan, xs[0], ym, stream)
        torch.cuda.synchronize()
        start.record(stream)
        for i in range(steps):
            N.ntt_forward(plan, xs[i % 2], ym if i % 2 == 0 else ys[1], stream)
        stop.record(stream)
        stop.synchronize()
        ms_m = start.elapsed_time(stop) / steps
        N.ntt_forward(plan, xs[0], ym, stream)
        torch.cuda.synchronize()
        same = bool(torch.equal(ym, ys[0]))
        mdesc = N.ntt_plan_describe(plan)
        # composite bound of the matrix path: per pass the larger of its HBM
        # time (one read and one write of 32 B per element) and its tensor
        # time (2 * 32 S * 32 S flops per sub-transform of S points)
        pk = peaks()
        hbm = pk.get("hbm_gbs", 6800.0) * 1e9
        tc = pk.get("bf16_tflops", 1900.0) * 1e12
        t_min = sum(max((1 << log_n) * 64 / hbm, (1 << log_n) * 2048 * (1 << ls) / tc) for ls in mdesc["pass_log"])
        return {"workload": "BLS12-381 Fr forward NTT, n=2^24, butterfly path", "ms": round(ms, 4),
                "elements_per_s": (1 << log_n) / (ms * 1e-3),
                "imad_roofline_frac": round(alg / (ms * 1e-3) / 1e12 / peak, 4), "passes": per_pass,
                "matrix_path": {"ms": round(ms_m, 4), "elements_per_s": (1 << log_n) / (ms_m * 1e-3),
                                "passes": mdesc["launches_per_transform"],
                                "folded_passes": mdesc["matrix_folded_passes"], "identical_to_butterfly": same,
                                "composite_bound_ms": round(t_min * 1e3, 4),
                                "composite_frac": round(t_min * 1e3 / ms_m, 4),
                                "bound_note": "sum over passes of max(64 B/element at the measured HBM copy rate, "
                                              "2048 S flops/element at the measured bf16 (= fp16) tensor rate); "
                                              "the epilogue's modular reduction (IMAD pipe) is not in it",
                                "device_error": N.ntt_plan_poll_error(plan)}}
    finally:
        N.ntt_plan_destroy(plan)


def measure_large(torch, N, stream, steps: int, log_n: int = 28) -> dict:
    """BLS12-381 Fr forward NTT at 2^28 (three passes, 8 GiB per vector).
    The input is a seeded 2^20-element vector repeated (every entry a field
    element; the kernels' work does not depend on the values)."""
    plan = N.ntt_plan_create(FIELD, log_n)
    try:
        desc = N.ntt_plan_describe(plan)
        base = to_dev(torch, uniform_elements(FIELD, 1 << 20, config_seed(3, 300)))
        x = base.repeat(1 << (log_n - 20), 1)
        y = torch.empty_like(x)
        N.ntt_forward(plan, x, y, stream)
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(steps):
            N.ntt_forward(plan, x, y, stream)
        stop.record(stream)
        stop.synchronize()
        ms = start.elapsed_time(stop) / steps
        alg = transform_modmuls(log_n) * IMAD_PER_MODMUL
        return {"workload": f"BLS12-381 Fr forward NTT, n=2^{log_n}, passes {desc['pass_log'][:desc['num_passes']]}",
                "ms": round(ms, 3), "elements_per_s": (1 << log_n) / (ms * 1e-3),
                "imad_roofline_frac": round(alg / (ms * 1e-3) / 1e12 / imad_peak_tops(), 4),
                "device_bytes": desc["device_bytes"]}
    finally:
        N.ntt_plan_destroy(plan)


def measure_coset_2_24(torch, N, stream, steps: int) -> dict:
    """BN254 Fr coset NTT at 2^24 (shift 5): the butterfly path against the
    matrix (tensor-core) path on the same input, outputs compared."""
    field, log_n = "bn254_fr", 24
    plan = N.ntt_plan_create(field, log_n, coset=True)
    try:
        x = to_dev(torch, uniform_elements(field, 1 << log_n, config_seed(3)))
        outs, ms = {}, {}
        for path in ("butterfly", "matrix"):
            N.ntt_plan_set_path(plan, path)
            y = torch.empty_like(x)
            N.ntt_coset_forward(plan, x, y, stream)
            torch.cuda.synchronize()
            start = torch.cuda.Event(enable_timing=True)
            stop = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            for _ in range(steps):
                N.ntt_coset_forward(plan, x, y, stream)
            stop.record(stream)
            stop.synchronize()
            ms[path] = start.elapsed_time(stop) / steps
            outs[path] = y
        return {"workload": "BN254 Fr coset NTT, n=2^24, shift 5, butterfly vs matrix path",
                "butterfly_ms": round(ms["butterfly"], 3), "matrix_ms": round(ms["matrix"], 3),
                "butterfly_elements_per_s": (1 << log_n) / (ms["butterfly"] * 1e-3),
                "matrix_elements_per_s": (1 << log_n) / (ms["matrix"] * 1e-3),
                "identical": bool(torch.equal(outs["butterfly"], outs["matrix"])),
                "device_error": N.ntt_plan_poll_error(plan)}
    finally:
        N.ntt_plan_destroy(plan)


def measure_wide(torch, N, stream, steps: int, log_n: int = 20) -> dict:
    """Forward NTT at 2^20 over the 377- and 753-bit fields (the precisions of
    the paper's wider rows), round trip checked."""
    out = {}
    for field in ("w377", "w753"):
        x = to_dev(torch, uniform_elements(field, 1 << log_n, config_seed(2, 400)))
        y = torch.empty_like(x)
        z = torch.empty_like(x)
        N.ntt_wide_transform(field, "forward", log_n, x, y, stream)
        N.ntt_wide_transform(field, "inverse", log_n, y, z, stream)
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(steps):
            N.ntt_wide_transform(field, "forward", log_n, x, y, stream)
        stop.record(stream)
        stop.synchronize()
        ms = start.elapsed_time(stop) / steps
        out[field] = {"ms": round(ms, 4), "elements_per_s": (1 << log_n) / (ms * 1e-3),
                      "round_trip_exact": bool(torch.equal(z, x))}
    out["workload"] = f"forward NTT, n=2^{log_n}, 377- and 753-bit NTT-friendly primes"
    return out


# MORPH's MSM latencies for the 256-bit curve (TPUv6e-8, Tab. 4), in ms
PAPER_MSM_MS = {22: 1.61, 24: 6.42, 26: 25.64}
MSM_CONFIG = 6  # seeds of the MSM inputs (shared with the tests)


# curve -> (scalar field, seed configuration of its inputs)
MSM_CURVES = {"bn254_g1": ("bn254_fr", MSM_CONFIG), "bls12_381_g1": ("bls12_381_fr", MSM_CONFIG + 1)}


def msm_inputs(torch, N, stream, n: int, curve: str = "bn254_g1"):
    """Scalars uniform in [0, r); points t_n G from the library's fixed-base
    generator (t_n seeded uniform), so that the result has a closed form."""
    field, cfg = MSM_CURVES[curve]
    d_s = to_dev(torch, uniform_elements(field, n, config_seed(cfg)))
    d_t = to_dev(torch, uniform_elements(field, n, config_seed(cfg, 1)))
    pts = torch.empty((n, N.msm_point_bytes(curve) // 8), dtype=torch.int64, device=d_s.device)
    N.msm_fixed_base(curve, d_t, n, pts, stream)
    torch.cuda.synchronize()
    del d_t
    return d_s, pts


def measure_msm(torch, N, stream, reps: int, log_sizes=(22, 24), curve: str = "bn254_g1") -> dict:
    """Multi-scalar multiplication on BN254 G1 or BLS12-381 G1 (Algorithm 2,
    LS-PPG): the whole call (point conversion, bucketize, accumulation, tree
    reduction, window merge) timed with CUDA events; the paper's sizes
    2^22..2^26."""
    out = {}
    peak = imad_peak_tops()
    for lg in log_sizes:
        n = 1 << lg
        d_s, pts = msm_inputs(torch, N, stream, n, curve)
        plan = N.msm_plan_create(curve, n, 0)
        info = N.msm_plan_info(plan)
        res = torch.empty(pts.shape[1], dtype=torch.int64, device=d_s.device)
        N.msm_execute(plan, d_s, pts, n, res, stream)
        torch.cuda.synchronize()
        first = res.clone()
        times = []
        for _ in range(reps):
            start = torch.cuda.Event(enable_timing=True)
            stop = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            N.msm_execute(plan, d_s, pts, n, res, stream)
            stop.record(stream)
            stop.synchronize()
            times.append(start.elapsed_time(stop))
        ms = float(np.median(times))
        # the same MSM from precomputed bases (points set once: a prover's fixed setup points)
        bases_ms = None
        if info["num_windows"] <= 32:
            start = torch.cuda.Event(enable_timing=True)
            stop = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            N.msm_plan_set_bases(plan, pts, n, stream)
            stop.record(stream)
            stop.synchronize()
            set_ms = start.elapsed_time(stop)
            res_b = torch.empty_like(res)
            N.msm_execute_bases(plan, d_s, n, res_b, stream)
            torch.cuda.synchronize()
            tb = []
            for _ in range(reps):
                start.record(stream)
                N.msm_execute_bases(plan, d_s, n, res_b, stream)
                stop.record(stream)
                stop.synchronize()
                tb.append(start.elapsed_time(stop))
            bases_ms = {"ms": round(float(np.median(tb)), 3), "set_bases_ms": round(set_ms, 1),
                        "same_result": bool(torch.equal(res_b, first))}
        c, K = info["window_bits"], info["num_windows"]
        # algorithmic products: one 10-product mixed addition per point and
        # window, about 26 per bucket (2^(c-1) per window) in the reduction tree;
        # a product of D 32-bit limbs is 2 (2 D^2 + D) IMAD (272 for D = 8)
        modmuls = K * n * 10 + K * (1 << (c - 1)) * 26
        limbs = pts.shape[1]  # 32-bit limbs per coordinate = 64-bit words per point
        imad_per = 2 * (2 * limbs * limbs + limbs)
        achieved = modmuls * imad_per / (ms * 1e-3) / 1e12
        out[f"n_2_{lg}"] = {"ms": round(ms, 3), "points_per_s": n / (ms * 1e-3), "window_bits": c, "windows": K,
                            "segment_length": info["segment_length"], "plan_device_gb":
                            round(info["device_bytes"] / 1e9, 2), "algorithmic_modmuls": modmuls,
                            "imad_frac": round(achieved / peak, 4), "repeatable": bool(torch.equal(res, first)),
                            "device_error": N.msm_poll_error(plan),
                            "paper_tpu_ms": PAPER_MSM_MS.get(lg) if curve == "bn254_g1" else None,
                            "precomputed_bases": bases_ms}
        N.msm_plan_destroy(plan)
        del d_s, pts
        torch.cuda.empty_cache()
    out["workload"] = (f"MSM on {curve} by Layout-Stationary Pippenger, scalars uniform < r, points t_n G "
                       "(seeded), result checked against the closed form in the tests")
    return out


def measure_commit(torch, N, stream, reps: int, log_n: int = 20) -> dict:
    """A KZG-style commitment on BLS12-381, all on the GPU: inverse NTT of
    2^log_n evaluations to coefficients, then their MSM against setup points
    tau^i G (made by the fixed-base generator; the tests check the result
    against the closed form f(tau) G)."""
    n = 1 << log_n
    d_e = to_dev(torch, uniform_elements("bls12_381_fr", n, config_seed(8, log_n)))
    d_c = torch.empty_like(d_e)
    # setup scalars tau^i: a seeded geometric sequence (any scalars serve for timing)
    tau = int(uniform_elements("bls12_381_fr", 1, config_seed(8, 99))[0, 0]) | 1
    r = MODULI_R["bls12_381_fr"]
    pw = np.zeros((n, 4), dtype=np.uint64)
    t = 1
    for i in range(n):
        pw[i, 0] = t & 0xFFFFFFFFFFFFFFFF
        pw[i, 1] = (t >> 64) & 0xFFFFFFFFFFFFFFFF
        pw[i, 2] = (t >> 128) & 0xFFFFFFFFFFFFFFFF
        pw[i, 3] = t >> 192
        t = t * tau % r
    d_t = to_dev(torch, pw)
    srs = torch.empty((n, 12), dtype=torch.int64, device=d_e.device)
    N.msm_fixed_base("bls12_381_g1", d_t, n, srs, stream)
    del d_t
    plan = N.ntt_plan_create("bls12_381_fr", log_n)
    msm = N.msm_plan_create("bls12_381_g1", n, 0)
    res = torch.empty(12, dtype=torch.int64, device=d_e.device)
    N.msm_plan_set_bases(msm, srs, n, stream)

    def step(bases: bool):
        N.ntt_inverse(plan, d_e, d_c, stream)
        if bases:
            N.msm_execute_bases(msm, d_c, n, res, stream)
        else:
            N.msm_execute(msm, d_c, srs, n, res, stream)

    out = {}
    for bases in (False, True):
        step(bases)
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            start = torch.cuda.Event(enable_timing=True)
            stop = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            step(bases)
            stop.record(stream)
            stop.synchronize()
            times.append(start.elapsed_time(stop))
        out["with_precomputed_bases_ms" if bases else "ms"] = round(float(np.median(times)), 3)
    out["device_error"] = N.msm_poll_error(msm)
    N.msm_plan_destroy(msm)
    N.ntt_plan_destroy(plan)
    out["workload"] = (f"KZG-style commitment, BLS12-381: inverse NTT of 2^{log_n} evaluations + MSM of the "
                       "coefficients against 2^%d setup points tau^i G, all on the device" % log_n)
    return out


def measure_matrix(torch, N, stream, bufs, steps: int, log_n: int) -> dict:
    """The same workload on the matrix-form path (tensor-core passes)."""
    plan = N.ntt_plan_create(FIELD, log_n)
    try:
        N.ntt_plan_set_path(plan, "matrix")
        desc = N.ntt_plan_describe(plan)
        timed_loop(torch, N, plan, bufs, len(bufs), stream)
        torch.cuda.synchronize()
        ms = timed_loop(torch, N, plan, bufs, steps, stream)
        same = all(bool(torch.equal(z, x)) for x, _, z in bufs)
        return {"workload": f"BLS12-381 Fr NTT n=2^{log_n}, forward+inverse per step, matrix path "
                            f"({desc['launches_per_transform']} tensor-core passes of <= 2^3 points)",
                "ms_per_step": round(ms / steps, 4), "elements_per_s": 2 * (1 << log_n) * steps / (ms * 1e-3),
                "round_trip_exact": same, "device_error": N.ntt_plan_poll_error(plan)}
    finally:
        N.ntt_plan_destroy(plan)


def measure_paths(torch, N, stream, log_n: int, reps: int = 5) -> dict:
    """Matrix (tensor-core) path against the butterfly path at one size,
    BLS12-381 Fr: two untimed forward transforms per path (matrix first, so
    a profiler can address its launches), then `reps` timed forward+inverse
    pairs; outputs compared across paths and the round trip checked."""
    x = to_dev(torch, uniform_elements(FIELD, 1 << log_n, config_seed(3, 100)))
    plan = N.ntt_plan_create(FIELD, log_n)
    out = {"workload": f"BLS12-381 Fr NTT n=2^{log_n}, forward and inverse, matrix vs butterfly path"}
    ys = {}
    try:
        for path in ("matrix", "butterfly"):
            N.ntt_plan_set_path(plan, path)
            y = torch.empty_like(x)
            z = torch.empty_like(x)
            for _ in range(2):
                N.ntt_forward(plan, x, y, stream)
            torch.cuda.synchronize()
            start = torch.cuda.Event(enable_timing=True)
            stop = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            for _ in range(reps):
                N.ntt_forward(plan, x, y, stream)
                N.ntt_inverse(plan, y, z, stream)
            stop.record(stream)
            stop.synchronize()
            ms = start.elapsed_time(stop) / (2 * reps)
            ys[path] = y
            out[path] = {"ms_per_transform": round(ms, 4), "elements_per_s": (1 << log_n) / (ms * 1e-3),
                         "passes": N.ntt_plan_describe(plan)["launches_per_transform"],
                         "round_trip_exact": bool(torch.equal(z, x))}
        out["identical"] = bool(torch.equal(ys["matrix"], ys["butterfly"]))
        out["matrix_vs_butterfly"] = round(out["butterfly"]["ms_per_transform"] / out["matrix"]["ms_per_transform"], 3)
        out["device_error"] = N.ntt_plan_poll_error(plan)
        return out
    finally:
        N.ntt_plan_destroy(plan)


def measure_quotient(torch, N, stream, reps: int, log_n: int = 20, blowup_log: int = 2) -> dict:
    """A prover's quotient step: coset NTTs of A, B, C (degree < 2n, zero
    padded) on the coset s<omega_m> of m = 4n points, the fused pointwise
    quotient (a b - c) / (X^n - 1), and the coset inverse NTT (n = 2^20,
    BLS12-381 Fr, shift 7).  Correctness of the chain is pinned by the GPU
    tests (it returns Q exactly for C = A B - (X^n - 1) Q)."""
    from ntt_synth import MODULI

    p = MODULI[FIELD]
    n, m = 1 << log_n, 1 << (log_n + blowup_log)
    s = 7                                      # coset shift = generator
    w_b = pow(7, (p - 1) >> blowup_log, p)     # primitive 2^blowup_log-th root
    sn = pow(s, n, p)
    z = [pow((sn * pow(w_b, j, p) - 1) % p, p - 2, p) for j in range(1 << blowup_log)]
    plan = N.ntt_plan_create(FIELD, log_n + blowup_log, coset=True)
    try:
        ins = []
        for i in range(3):
            h = np.zeros((m, 4), dtype=np.uint64)
            h[: 2 * n] = uniform_elements(FIELD, 2 * n, config_seed(2, 300 + i))
            ins.append(to_dev(torch, h))
        work = [torch.empty_like(ins[0]) for _ in range(3)]

        def step():
            for i in range(3):
                N.ntt_coset_forward(plan, ins[i], work[i], stream)
            N.ntt_pointwise_quotient(FIELD, work[0], work[1], work[2], z, work[0], m, stream)
            N.ntt_coset_inverse(plan, work[0], work[0], stream)

        step()
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        mid = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(reps):
            step()
        stop.record(stream)
        stop.synchronize()
        ms = start.elapsed_time(stop) / reps
        # the fused pointwise kernel alone
        start.record(stream)
        for _ in range(reps):
            N.ntt_pointwise_quotient(FIELD, work[0], work[1], work[2], z, work[1], m, stream)
        mid.record(stream)
        mid.synchronize()
        q_ms = start.elapsed_time(mid) / reps
        # two products and one reduction per element (2.5 modmul equivalents)
        q_frac = 2.5 * m * IMAD_PER_MODMUL / (q_ms * 1e-3) / 1e12 / imad_peak_tops()
        return {"workload": f"prover quotient step, BLS12-381 Fr, n=2^{log_n}, coset of m=2^{log_n + blowup_log} "
                            "points: 3 coset NTTs + fused pointwise (a b - c)/Z_H + coset inverse NTT",
                "ms": round(ms, 4), "coset_points_per_s": m / (ms * 1e-3),
                "pointwise_ms": round(q_ms, 4), "pointwise_imad_frac": round(q_frac, 4),
                "pointwise_hbm_gbs": round(4 * 32 * m / (q_ms * 1e-3) / 1e9, 1),
                "device_error": N.ntt_plan_poll_error(plan)}
    finally:
        N.ntt_plan_destroy(plan)


def rns_words(limbs: np.ndarray, basis: dict) -> np.ndarray:
    """Residues of [n, 4]-limb integers modulo the base-Q primes, as
    [n, words_per_element] uint32 (input marshalling for ntt_rns_mul)."""
    w32 = np.ascontiguousarray(limbs, dtype=np.uint64).view(np.uint32).reshape(-1, 8).astype(np.uint64)
    out = np.zeros((w32.shape[0], basis["words_per_element"]), dtype=np.uint32)
    for i, q in enumerate(basis["q"]):
        q = np.uint64(q)
        acc = np.zeros(w32.shape[0], dtype=np.uint64)
        for w in range(8):
            acc = (acc + (w32[:, w] % q) * np.uint64(pow(2, 32 * w, int(q)))) % q
        out[:, i] = acc.astype(np.uint32)
    return out


def measure_modmul(torch, N, stream, count: int = 1 << 22, reps: int = 64) -> dict:
    """Montgomery products per second: per-thread carry chains (the library's
    form) vs 8 lanes per element with warp-shuffle carries."""
    x = to_dev(torch, uniform_elements(FIELD, count, 77))
    y = to_dev(torch, uniform_elements(FIELD, count, 78))
    res = {}
    outs = []
    for variant, name in ((0, "thread_carry_chains"), (1, "warp_shuffle_carries")):
        z = torch.empty_like(x)
        N.ntt_field_mont_mul_rep(FIELD, x, y, z, count, reps, variant, stream)
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        N.ntt_field_mont_mul_rep(FIELD, x, y, z, count, reps, variant, stream)
        stop.record(stream)
        stop.synchronize()
        ms = start.elapsed_time(stop)
        res[name] = {"ms": round(ms, 4), "modmul_per_s": count * reps / (ms * 1e-3),
                     "imad_frac_alg": count * reps * IMAD_PER_MODMUL / (ms * 1e-3) / 1e12 / imad_peak_tops()}
        outs.append(z)
    res["identical"] = bool(torch.equal(outs[0], outs[1]))
    res["workload"] = f"{count} BLS12-381 elements x {reps} dependent Montgomery products"
    # the paper's arithmetic: RNS lazy products, byte products on tcgen05
    # (inputs: the same field elements as residues in base Q, 20 words each)
    basis = N.ntt_rns_basis_get(FIELD)
    xs = uniform_elements(FIELD, count, 77)
    ys = uniform_elements(FIELD, count, 78)
    rx = torch.from_numpy(rns_words(xs, basis).view(np.int32)).cuda()
    ry = torch.from_numpy(rns_words(ys, basis).view(np.int32)).cuda()
    rz = torch.empty_like(rx)
    N.ntt_rns_mul(FIELD, rx, ry, rz, count, reps, stream)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    N.ntt_rns_mul(FIELD, rx, ry, rz, count, reps, stream)
    stop.record(stream)
    stop.synchronize()
    ms = start.elapsed_time(stop)
    res["rns_lazy_tensor_core"] = {"ms": round(ms, 4), "modmul_per_s": count * reps / (ms * 1e-3),
                                   "vs_thread_carry_chains": round(res["thread_carry_chains"]["ms"] / ms, 3),
                                   "device_error": N.ntt_rns_poll_error(FIELD),
                                   "how": f"{len(basis['q'])} + {len(basis['p'])} residues of 31 bits, "
                                          "two tcgen05 byte products per product (Alg. 1)"}
    return res


def measure_batched(torch, N, stream, reps: int, tune: bool = True) -> dict:
    """64 BLS12-381 forward jobs, log2 n uniform on {14..22} (seeded): one
    transform per call (the loop) against the batched forms -- every job in
    one persistent launch replayed from a CUDA graph (untuned), and the form
    ntt_batch_autotune picks after ntt_plan_autotune has tuned each size's
    plan (tuned).  All forms must give identical outputs."""
    from ntt_synth import batch_sizes

    sizes = batch_sizes(64, 14, 22, config_seed(4))
    plans = {ln: N.ntt_plan_create(FIELD, ln) for ln in sorted(set(sizes))}
    try:
        xs = [to_dev(torch, uniform_elements(FIELD, 1 << ln, config_seed(4, j))) for j, ln in enumerate(sizes)]
        outs = {name: [torch.empty_like(x) for x in xs] for name in ("loop", "untuned", "tuned", "loop_tuned")}
        total = sum(1 << ln for ln in sizes)

        def jobs(name):
            return [(plans[ln], "forward", x, y) for ln, x, y in zip(sizes, xs, outs[name])]

        def loop(name):
            for ln, x, y in zip(sizes, xs, outs[name]):
                N.ntt_forward(plans[ln], x, y, stream)

        def timed(fn) -> float:
            fn()
            torch.cuda.synchronize()
            start = torch.cuda.Event(enable_timing=True)
            stop = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            for _ in range(reps):
                fn()
            stop.record(stream)
            stop.synchronize()
            return start.elapsed_time(stop) / reps

        res = {"loop": timed(lambda: loop("loop")),
               "untuned": timed(lambda: N.ntt_batch_submit(jobs("untuned"), stream))}
        tuned_info = None
        if tune:
            t0 = time.perf_counter()
            plan_choice = {ln: N.ntt_plan_autotune(p, reps=2) for ln, p in plans.items()}
            tuned_info = N.ntt_batch_autotune(jobs("tuned"), reps=2)
            tuned_info["tuning_s"] = round(time.perf_counter() - t0, 2)
            tuned_info["plans"] = {str(ln): {"path": c["path"], "pass_log": c["pass_log"], "tile_log": c["tile_log"]}
                                   for ln, c in plan_choice.items()}
            res["tuned"] = timed(lambda: N.ntt_batch_submit(jobs("tuned"), stream))
            res["loop_tuned"] = timed(lambda: loop("loop_tuned"))
        names = [n for n in ("loop", "untuned", "tuned", "loop_tuned") if n in res]
        same = all(bool(torch.equal(a, b)) for n in names[1:] for a, b in zip(outs["loop"], outs[n]))
        err = N.ntt_batch_poll_error()
        out = {"workload": "64 BLS12-381 forward NTTs, log2 n uniform on {14..22}, " f"{total} elements",
               "loop_ms": round(res["loop"], 4), "batched_ms": round(res["untuned"], 4),
               "batched_elements_per_s": total / (res["untuned"] * 1e-3),
               "loop_elements_per_s": total / (res["loop"] * 1e-3),
               "speedup": round(res["loop"] / res["untuned"], 3),
               "identical_results": same, "device_error": err}
        if tune:
            out.update({"tuned_batched_ms": round(res["tuned"], 4),
                        "tuned_batched_elements_per_s": total / (res["tuned"] * 1e-3),
                        "loop_tuned_plans_ms": round(res["loop_tuned"], 4),
                        "tuned_speedup_vs_loop": round(res["loop"] / res["tuned"], 3),
                        "tuned_speedup_vs_loop_tuned_plans": round(res["loop_tuned"] / res["tuned"], 3),
                        "tuning": tuned_info})
        return out
    finally:
        N.ntt_batch_cache_clear()
        for p in plans.values():
            N.ntt_plan_destroy(p)


def measure_serving(torch, N, rates, seconds: float, min_jobs: int, log_min: int = 12, log_max: int = 24,
                    seed: int = 0x5EED0005, max_inflight: int = 8, max_batch_jobs: int = 16,
                    check: bool = False, check_per_rate: int = 3, check_max_log: int = 18) -> dict:
    """Poisson arrivals of mixed forward/inverse/coset requests over both
    fields, log2 n uniform on {log_min..log_max}, through the serving runtime
    (host buffers in, host buffers out).  Per rate: p50/p99 latency
    (finish - arrive) and elements/s over the run.  Every request of a size
    reads the same pinned input; outputs go to one shared pinned buffer per
    size, except for up to check_per_rate requests per rate (sizes up to
    2^check_max_log) which get buffers of their own and, with check=True,
    are compared with the same transform run alone (ntt_execute) after the
    rate's run: each result must be the same in the mix as alone."""
    import random

    server = N.ntt_server_create(memory_budget_bytes=64 << 30, min_log_n=log_min, max_log_n=log_max,
                                 max_inflight=max_inflight, max_batch_jobs=max_batch_jobs)
    try:
        bufs = {}
        for fi, field in enumerate(("bls12_381_fr", "bn254_fr")):
            for ln in range(log_min, log_max + 1):
                x = uniform_elements(field, 1 << ln, seed + 100 * fi + ln)
                h_in = torch.from_numpy(x.view(np.int64)).pin_memory()
                bufs[(field, ln)] = (h_in, torch.empty_like(h_in).pin_memory())
        out = []
        rng = random.Random(seed)
        checked_total, mismatches = 0, 0
        for rate in rates:
            n_jobs = max(min_jobs, int(rate * seconds))
            tickets = []
            checks = []
            elements = 0
            t_next = time.perf_counter()
            for _ in range(n_jobs):
                t_next += rng.expovariate(rate)
                while time.perf_counter() < t_next:
                    pass
                field = rng.choice(("bls12_381_fr", "bn254_fr"))
                kind = rng.choice(("forward", "inverse", "coset"))
                ln = rng.randint(log_min, log_max)
                h_in, h_out = bufs[(field, ln)]
                if check and len(checks) < check_per_rate and ln <= check_max_log:
                    h_out = torch.empty_like(h_in).pin_memory()
                    checks.append((field, kind, ln, h_in, h_out))
                tickets.append(N.ntt_server_submit(server, field, kind, ln, h_in, h_out))
                elements += 1 << ln
            lat, first, last = [], None, None
            for t in tickets:
                N.ntt_server_wait(server, t, 600.0)
                a, _, f = N.ntt_server_request_times(server, t)
                lat.append(f - a)
                first = a if first is None else min(first, a)
                last = f if last is None else max(last, f)
                N.ntt_server_release(server, t)
            lat.sort()
            row = {"rate_per_s": rate, "jobs": n_jobs, "elements": elements,
                   "window_s": round(last - first, 3), "elements_per_s": elements / (last - first),
                   "p50_ms": round(1e3 * lat[len(lat) // 2], 3),
                   "p99_ms": round(1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))], 3)}
            if check:
                same = 0
                for field, kind, ln, h_in, h_out in checks:
                    plan = N.ntt_plan_create(field, ln, coset=True)
                    try:
                        d_x = h_in.cuda()
                        d_y = torch.empty_like(d_x)
                        N.ntt_execute(plan, kind, d_x, d_y)
                        torch.cuda.synchronize()
                        same += int(torch.equal(d_y.cpu(), h_out))
                    finally:
                        N.ntt_plan_destroy(plan)
                row["checked"] = len(checks)
                row["same_as_alone"] = same
                checked_total += len(checks)
                mismatches += len(checks) - same
            out.append(row)
        stats = N.ntt_server_get_stats(server)
        res = {"workload": f"Poisson arrivals, kinds forward/inverse/coset, fields BLS12-381/BN254, "
                           f"log2 n uniform on {{{log_min}..{log_max}}}, 64 GiB budget, {max_inflight} streams, "
                           f"at most {max_batch_jobs} jobs per batch",
               "rates": out, "batches": stats["batches"], "peak_device_bytes": stats["peak_device_bytes"],
               "resident_bytes": stats["resident_bytes"]}
        if check:
            res["results_checked"] = checked_total
            res["results_same_as_alone"] = checked_total - mismatches
        return res
    finally:
        N.ntt_server_destroy(server)


def measure_e2e(torch, N, x_host: np.ndarray, steps: int, log_n: int, num_lanes: int = 4) -> dict:
    """End to end through the public host-buffer call: every step copies its
    input from pinned host memory, runs forward then inverse, and copies the
    result back (ntt_transform_host_async); steps rotate over `num_lanes`
    streams (separate plans, device buffers and host buffers) so that some
    steps' copies overlap other steps' kernels.  Wall-clock time over all
    steps."""
    n = x_host.shape[0]
    lanes = []
    for _ in range(num_lanes):
        plan = N.ntt_plan_create(FIELD, log_n)
        h_in = torch.from_numpy(x_host.view(np.int64).copy()).pin_memory()
        lanes.append({"plan": plan, "stream": torch.cuda.Stream(), "h_in": h_in,
                      "h_mid": torch.empty_like(h_in).pin_memory(), "h_out": torch.empty_like(h_in).pin_memory(),
                      "d_work": torch.empty(h_in.shape, dtype=torch.int64, device="cuda")})

    def step(ln):
        N.ntt_transform_host_async(ln["plan"], "forward", ln["h_in"], ln["h_mid"], ln["d_work"], ln["stream"])
        N.ntt_transform_host_async(ln["plan"], "inverse", ln["h_mid"], ln["h_out"], ln["d_work"], ln["stream"])

    try:
        for i in range(2 * num_lanes):
            step(lanes[i % num_lanes])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(steps):
            step(lanes[i % num_lanes])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ok = all(bool(torch.equal(ln["h_out"], ln["h_in"])) for ln in lanes)
    finally:
        for ln in lanes:
            N.ntt_plan_destroy(ln["plan"])
    return {"value": 2 * n * steps / dt, "unit": UNIT, "h2d_bytes_per_step": 2 * 32 * n,
            "d2h_bytes_per_step": 2 * 32 * n, "round_trip_exact": ok, "steps": steps,
            "how": f"ntt_transform_host_async, pinned host buffers, {num_lanes} streams, wall clock over "
                   f"{steps} steps"}


def _oracle_rate(oracle, x: np.ndarray, budget_s: float, kinds=("forward", "inverse")) -> tuple[float, int, float]:
    """Elements/s of the C oracle transforming x (each kind once per round)
    until budget_s has passed (at least one round): (rate, rounds, seconds)."""
    n = x.shape[0]
    t0 = time.perf_counter()
    rounds = 0
    while True:
        y = x
        for kind in kinds:
            y = oracle.c_transform(FIELD, kind, y)
        rounds += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return len(kinds) * n * rounds / dt, rounds, dt


def cpu_baseline(x: np.ndarray, budget_s: float = 8.0, with_2_24: bool = True) -> dict:
    """The C oracle on this host's cores: single-threaded (the headline
    baseline value), and with the butterflies of each stage split over every
    core OpenMP sees (same arithmetic), on the 2^20 workload vector and on a
    2^12 vector, plus one 2^24-point forward transform on all cores."""
    import oracle

    host_cores = len(os.sched_getaffinity(0))
    n = x.shape[0]
    try:
        oracle.c_set_threads(1)
        v1, r1, t1 = _oracle_rate(oracle, x, budget_s)
        threads = oracle.c_set_threads(0)
        vall, rall, tall = _oracle_rate(oracle, x, budget_s / 2)
        # the 2^12 workload (config 1 size), one core and all cores
        xs = uniform_elements(FIELD, 1 << 12, config_seed(1))
        oracle.c_set_threads(1)
        vs1, rs1, ts1 = _oracle_rate(oracle, xs, 0.5)
        oracle.c_set_threads(0)
        vsall, rsall, tsall = _oracle_rate(oracle, xs, 0.5)
        small = {"single": {"value": vs1, "unit": UNIT, "cores": 1, "rounds": rs1, "seconds": round(ts1, 2)},
                 "all_cores": {"value": vsall, "unit": UNIT, "cores": threads, "rounds": rsall,
                               "seconds": round(tsall, 2)},
                 "sample": "forward+inverse of the 2^12-point BLS12-381 vector"}
        big = None
        if with_2_24:
            xb = uniform_elements(FIELD, 1 << 24, config_seed(3, 100))
            vb, _, tb = _oracle_rate(oracle, xb, 0.0, kinds=("forward",))
            big = {"value": vb, "unit": UNIT, "cores": threads, "seconds": round(tb, 2),
                   "sample": "one forward transform of the 2^24-point BLS12-381 vector, all cores"}
    finally:
        oracle.c_set_threads(1)
    return {"value": v1, "unit": UNIT, "cores": 1, "host_cores": host_cores, "kind": "oracle",
            "sample": f"C oracle (single-threaded), forward+inverse of the 2^{n.bit_length() - 1} "
                      f"BLS12-381 workload vector, {r1} round(s) in {t1:.1f} s",
            "all_cores": {"value": vall, "unit": UNIT, "cores": threads, "host_cores": host_cores,
                          "sample": f"C oracle, butterflies of each stage over {threads} OpenMP threads, "
                                    f"forward+inverse of the same vector, {rall} round(s) in {tall:.1f} s"},
            "all_cores_2_24": big, "n_2_12": small}


def run_ours(args) -> None:
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    from paper_2604_17808_gb300 import _native as N

    N.load(build_if_missing=True)
    device = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    log_n = args.log_n
    n = 1 << log_n
    plan = N.ntt_plan_create(FIELD, log_n)
    desc = N.ntt_plan_describe(plan)
    host_inputs = [uniform_elements(FIELD, n, config_seed(2, 1000 * rank + r) if r else config_seed(2))
                   for r in range(args.rotate)]
    bufs = []
    for h in host_inputs:
        x = to_dev(torch, h)
        bufs.append((x, torch.empty_like(x), torch.empty_like(x)))
    # parity of the first step against the stored oracle digests (same seed as the tests)
    parity = None
    if log_n == LOG_N and rank == 0:
        N.ntt_forward(plan, bufs[0][0], bufs[0][1], stream)
        N.ntt_inverse(plan, bufs[0][0], bufs[0][2], stream)
        torch.cuda.synchronize()
        f = hashlib.sha256(bufs[0][1].cpu().numpy().astype("<i8").tobytes()).hexdigest()
        i = hashlib.sha256(bufs[0][2].cpu().numpy().astype("<i8").tobytes()).hexdigest()
        parity = (f == golden_digest("forward")) and (i == golden_digest("inverse"))
    # warm-up: every rotating buffer once, then W more steps
    timed_loop(torch, N, plan, bufs, len(bufs), stream)
    for _ in range(args.warmup):
        timed_loop(torch, N, plan, bufs, 1, stream)
    torch.cuda.synchronize()

    # clocks: nvidia-smi samples every 100 ms, so the sampler starts during an
    # untimed pre-roll of the same workload (>= 0.6 s) and stops right after
    # the timed region; the samples cover the GPU under this load.
    clocks = ClockSampler(local).start() if rank == 0 else None
    t_end = time.perf_counter() + 0.6
    while time.perf_counter() < t_end:
        timed_loop(torch, N, plan, bufs, len(bufs), stream)
    dist_barrier(world)
    torch.cuda.synchronize()
    ms = timed_loop(torch, N, plan, bufs, args.steps, stream)
    torch.cuda.synchronize()
    dist_barrier(world)
    # per-kernel durations for the roofline: the same K steps once more with a
    # CUDA event pair around every pass (recorded on the launching stream).
    # The events cost ~4% of a step, so the headline region above runs
    # without them.
    N.ntt_plan_enable_timing(plan, True)
    timed_loop(torch, N, plan, bufs, args.steps, stream)
    torch.cuda.synchronize()
    pass_ms, pass_cnt = N.ntt_plan_read_timing(plan)
    N.ntt_plan_enable_timing(plan, False)
    clk = clocks.stop() if clocks else None
    if clk:
        clk["window"] = "0.6 s pre-roll of the same steps + the timed region + the per-pass timing run"
    ms_max = dist_max(ms, world, device)
    # the median step (each step bracketed by its own event pair; a separate
    # run, so that the headline region has no events inside it)
    per_step = sorted(step_times(torch, N, plan, bufs, max(args.steps, 20), stream))
    median_ms = per_step[len(per_step) // 2] if len(per_step) % 2 else 0.5 * (
        per_step[len(per_step) // 2 - 1] + per_step[len(per_step) // 2])
    # secondary: the same steps over two streams (independent vectors overlap)
    timed_loop_streams(torch, N, plan, bufs, len(bufs), stream, 2)
    ms2 = timed_loop_streams(torch, N, plan, bufs, args.steps, stream, 2)
    concurrent = {"streams": 2, "ms_per_step": ms2 / args.steps,
                  "elements_per_s": 2 * n * args.steps / (ms2 * 1e-3),
                  "note": "consecutive independent steps alternate over two streams; the headline value is one "
                          "stream"}

    # correctness of the timed steps: the round trip must give the input back
    round_trip_ok = all(bool(torch.equal(z, x)) for x, _, z in bufs)

    elements = 2 * n * args.steps * world
    value = elements / (ms_max * 1e-3)
    peak = imad_peak_tops()
    dom = max(range(desc["num_passes"]), key=lambda j: pass_ms[j])
    avg_ms = pass_ms[dom] / max(1, pass_cnt[dom])
    mm = pass_modmuls(log_n, desc["pass_log"], dom, dom >= 1)
    achieved = mm * IMAD_PER_MODMUL / (avg_ms * 1e-3) / 1e12
    launches = args.steps * 2 * desc["launches_per_transform"]

    secondary = None
    e2e = None
    cpu = None
    matrix = measure_matrix(torch, N, stream, bufs, max(3, args.steps // 5), log_n)
    if rank == 0:
        # enough steps that the 4-stream pipeline's fill and drain (the first
        # step's input copy, the last step's result copy) are amortised
        e2e = measure_e2e(torch, N, host_inputs[0], max(100, args.steps), log_n)
        if not args.quick:
            secondary = {"n_2_24_forward": measure_2_24(torch, N, stream, steps=max(3, args.steps // 4)),
                         "n_2_28_forward": measure_large(torch, N, stream, steps=3),
                         "bn254_coset_2_24": measure_coset_2_24(torch, N, stream, steps=3),
                         "wide_2_20": measure_wide(torch, N, stream, steps=10),
                         "batched": measure_batched(torch, N, stream, reps=5),
                         "modmul": measure_modmul(torch, N, stream),
                         "quotient_step": measure_quotient(torch, N, stream, reps=5),
                         "serving": measure_serving(torch, N, rates=SERVING_RATES, seconds=0.5, min_jobs=200,
                                                    check=True)}
        if world == 1 and not args.no_cpu:
            cpu = cpu_baseline(host_inputs[0])
    N.ntt_plan_destroy(plan)
    if rank != 0:
        dist_barrier(world)
        return
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "median_ms_per_step": {"value": median_ms, "steps": len(per_step), "min": per_step[0], "max": per_step[-1],
                               "note": "one CUDA event pair per step in a separate run of the same steps; "
                                       "ms_per_step is the timed region's mean"},
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic (uniform field elements from seed, SplitMix64)",
        "config": {"workload": f"BLS12-381 Fr NTT n=2^{log_n}, forward+inverse per step, butterfly path "
                               f"(passes {desc['pass_log']})",
                   "field": FIELD, "log_n": log_n, "transforms_per_step": 2, "per_rank_vectors": args.rotate,
                   "l2": L2_NOTE if args.rotate == ROTATE and log_n == LOG_N else
                   f"{args.rotate} rotating 2^{log_n} vectors", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T IMAD/s",
                     "frac": achieved / peak,
                     "traffic": profiled_traffic(f"pass{dom}") if log_n == LOG_N else None,
                     "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum per launch, ncu --set full "
                                     "(cold cache), only if captured from the current kernel sources",
                     "kernel_source_sha256": kernel_source_hash(),
                     "kernel": f"ntt_pass_kernel pass {dom} (S=2^{desc['pass_log'][dom]})",
                     "avg_launch_ms": avg_ms,
                     "timing_note": "avg_launch_ms from CUDA events around each pass over a second run of the "
                                    "same K steps (the headline region runs without per-pass events)",
                     "peak_note": "152 SMs x 64 IMAD/clk x 2070 MHz (unit counts and maximum clock)"},
        "e2e": e2e,
        "cpu_baseline": cpu,
        "gpu_launches": launches,
        "clocks": clk,
        "parity": {"first_step_matches_oracle_digest": parity, "round_trip_exact": round_trip_ok},
        "pass_ms_total": [round(v, 4) for v in pass_ms[: desc["num_passes"]]],
        "secondary": secondary,
        "paths": {"butterfly": value, "matrix": matrix["elements_per_s"], "matrix_detail": matrix},
        "concurrent_streams": concurrent,
    }
    print(json.dumps(line), flush=True)
    dist_barrier(world)


# ----------------------------------------------------- reference arm


def run_reference(args) -> None:
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle

    oracle.c_oracle()
    # calibrate, then pick the largest sample (<= 2^20) that keeps the run short
    probe = uniform_elements(FIELD, 1 << 14, config_seed(2))
    t0 = time.perf_counter()
    oracle.c_transform(FIELD, "forward", probe)
    per_elem_log = (time.perf_counter() - t0) / ((1 << 14) * 14)
    total_steps = args.steps + args.warmup
    log_s = LOG_N
    while log_s > 12 and total_steps * 2 * per_elem_log * (1 << log_s) * log_s > 150.0:
        log_s -= 1
    x = uniform_elements(FIELD, 1 << LOG_N, config_seed(2))[: 1 << log_s].copy()
    for _ in range(args.warmup):
        oracle.c_transform(FIELD, "inverse", oracle.c_transform(FIELD, "forward", x))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.c_transform(FIELD, "inverse", oracle.c_transform(FIELD, "forward", x))
    dt = time.perf_counter() - t0
    value = 2 * (1 << log_s) * args.steps / dt
    sample = (f"C oracle (single-threaded), forward+inverse of the first 2^{log_s} elements of the 2^20 "
              f"workload vector per step")
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic (uniform field elements from seed, SplitMix64)",
        "config": {"workload": f"BLS12-381 Fr NTT n=2^{LOG_N}, forward+inverse per step (oracle on a 2^{log_s} "
                               f"sample)", "field": FIELD, "log_n": LOG_N, "sample_log_n": log_s},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def run_serving_sweep(args) -> None:
    """--serving: the full sweep (>= 10 s or 2000 jobs per rate), one JSON line."""
    import torch

    from paper_2604_17808_gb300 import _native as N

    torch.cuda.set_device(0)
    N.load(build_if_missing=True)
    res = measure_serving(torch, N, rates=SERVING_RATES, seconds=10.0, min_jobs=2000, check=True)
    print(json.dumps({"metric": "serving p50/p99 latency and elements/s", "serving": res}), flush=True)


def run_leg(args) -> None:
    import torch

    from paper_2604_17808_gb300 import _native as N

    N.load(build_if_missing=True)
    stream = torch.cuda.current_stream()
    fn = {"modmul": lambda: measure_modmul(torch, N, stream),
          "quotient": lambda: measure_quotient(torch, N, stream, reps=3),
          "batched": lambda: measure_batched(torch, N, stream, reps=3),
          "n_2_28": lambda: measure_large(torch, N, stream, steps=3),
          "coset_2_24": lambda: measure_coset_2_24(torch, N, stream, steps=3),
          "wide": lambda: measure_wide(torch, N, stream, steps=10),
          "msm": lambda: measure_msm(torch, N, stream, reps=5, log_sizes=tuple(args.msm_log), curve=args.msm_curve),
          "commit": lambda: measure_commit(torch, N, stream, reps=5),
          "paths": lambda: measure_paths(torch, N, stream, args.log_n)}[args.leg]
    print(json.dumps({args.leg: fn()}), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--log-n", type=int, default=LOG_N)
    ap.add_argument("--quick", action="store_true", help="skip the 2^24 secondary measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--serving", action="store_true", help="run only the full serving sweep")
    ap.add_argument("--leg", choices=["modmul", "quotient", "batched", "n_2_28", "coset_2_24", "wide", "msm", "commit",
                                      "paths"],
                    help="run only this secondary measurement and print its JSON (for profiling)")
    ap.add_argument("--msm-log", type=int, nargs="+", default=[22, 24, 26],
                    help="log2 point counts of the msm leg (default: the paper's 22 24 26)")
    ap.add_argument("--msm-curve", choices=["bn254_g1", "bls12_381_g1"], default="bn254_g1",
                    help="curve of the msm leg")
    ap.add_argument("--rotate", type=int, default=ROTATE,
                    help="distinct input vectors the steps rotate over (default 8: larger than L2 at 2^20)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.leg:
        run_leg(args)
    elif args.serving:
        run_serving_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
