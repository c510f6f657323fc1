"""Writes tests/golden/pair640x480_oracle.json from the oracle alone.

Inputs: the seeded 640x480 planted-shift pair (paper_2007_06483_gb300.synth).
Stored: the input's SHA-256, and the oracle's shifts, per-level errors,
per-level shifts and per-level medians.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2007_06483_gb300 import synth  # noqa: E402


def main():
    spec = synth.PAIR_640
    imgs = synth.make_stack(spec).numpy()
    res = oracle.align_stack(imgs, spec.levels, spec.noise_tol, spec.ref)
    out = {
        "workload": spec.name,
        "levels": spec.levels,
        "noise_tol": spec.noise_tol,
        "ref": spec.ref,
        "input_sha256": hashlib.sha256(imgs.tobytes()).hexdigest(),
        "shifts": res["shifts"].tolist(),
        "level_errs": res["level_errs"].tolist(),
        "level_shifts": res["level_shifts"].tolist(),
        "medians": [oracle.pyramid_maps(imgs[e], spec.levels, spec.noise_tol)["median"].tolist()
                    for e in range(spec.n)],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pair640x480_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
