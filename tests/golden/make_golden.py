"""Write tests/golden/oracle_digests.json from the CPU oracle alone.

Every stored value here comes from ``oracle`` (the C oracle, cross-checked
against the Python oracle by tests/test_oracle_pins.py) applied to the seeded
inputs of ``ntt_synth``.  Nothing is taken from the CUDA library.

Digest = SHA-256 of the output as little-endian uint64 limbs, [n, 4] row-major.

    python tests/golden/make_golden.py            # all workloads (~4 min)
"""

from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from ntt_synth import batch_sizes, config_seed, uniform_elements  # noqa: E402


def digest(a) -> str:
    return hashlib.sha256(a.astype("<u8").tobytes()).hexdigest()


def main() -> None:
    out = {
        "_comment": "SHA-256 of C-oracle outputs (little-endian uint64 limbs) on the seeded inputs of ntt_synth; written by tests/golden/make_golden.py.",
        "single": [],
        "batched": {},
    }
    cases = [
        # (configuration index, field, log_n, kinds, seed)
        (1, "bls12_381_fr", 12, ["forward", "inverse"], config_seed(1)),
        (2, "bls12_381_fr", 20, ["forward", "inverse"], config_seed(2)),
        (3, "bn254_fr", 24, ["coset", "coset_inverse"], config_seed(3)),
        # the 2^24-point BLS12-381 transform (the size the 2^24 measurements use)
        (3, "bls12_381_fr", 24, ["forward", "inverse"], config_seed(3, 100)),
    ]
    for cfg, field, log_n, kinds, seed in cases:
        x = uniform_elements(field, 1 << log_n, seed)
        for kind in kinds:
            t = time.time()
            y = oracle.c_transform(field, kind, x)
            out["single"].append({
                "config": cfg, "field": field, "log_n": log_n, "kind": kind,
                "seed": seed, "input_sha256": digest(x), "output_sha256": digest(y),
                "first_output_hex": [hex(int(v)) for v in y[0]],
            })
            print(cfg, field, log_n, kind, f"{time.time() - t:.1f}s", flush=True)
    # batched workload: 64 forward BLS12-381 jobs, log2 n uniform on {14..22}
    cfg = 4
    sizes = batch_sizes(64, 14, 22, config_seed(cfg))
    jobs = []
    for j, log_n in enumerate(sizes):
        x = uniform_elements("bls12_381_fr", 1 << log_n, config_seed(cfg, j))
        y = oracle.c_transform("bls12_381_fr", "forward", x)
        jobs.append({"job": j, "log_n": log_n, "seed": config_seed(cfg, j), "output_sha256": digest(y)})
    out["batched"] = {"config": cfg, "field": "bls12_381_fr", "kind": "forward",
                      "total_elements": sum(1 << s for s in sizes), "jobs": jobs}
    print("batched total elements", out["batched"]["total_elements"], flush=True)
    with open(os.path.join(HERE, "oracle_digests.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
