"""Write the stored oracle results under tests/golden/.

Every value written here comes from the CPU oracle (``oracle``) applied to
inputs from the seeded generator (``lbdd_inputs``); nothing is taken from
the CUDA path.  The paper prints no numeric worked example (its Figures 1
and 2 are not reproducible from the text), so these files pin the oracle's
own canonical results for regression and for GPU parity at sizes where
re-running the oracle inside a test would take too long.

Usage:  python tests/golden/make_golden.py tiny [city [rounds]]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import lbdd_inputs  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def run(name: str, rounds: int = -1) -> dict:
    inst = lbdd_inputs.make_named(name)
    t0 = time.time()
    res = oracle.asral(inst.cm, inst.cap, inst.pen, mode=oracle.MODE_HEAP, max_rounds=rounds)
    secs = time.time() - t0
    if res.rc != oracle.OK:
        raise SystemExit(f"oracle failed: {res.rc}")
    out = {
        "workload": name,
        "n": inst.n,
        "k": inst.k,
        "seed": inst.recipe.seed,
        "rounds": res.stats["rounds"],
        "cm_sha256": digest(inst.cm),
        "delta": res.delta,
        "assign_sha256": digest(res.assign.astype(np.int32)),
        "load_sha256": digest(res.load.astype(np.int64)),
        "stats": res.stats,
        "oracle_seconds": round(secs, 2),
        "oracle_mode": "heap",
        "source": "oracle.asral (CPU), written by tests/golden/make_golden.py",
    }
    suffix = "" if rounds < 0 else f"_r{rounds}"
    path = os.path.join(HERE, f"{name}{suffix}_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(path, out["delta"], f"{secs:.1f}s")
    return out


if __name__ == "__main__":
    args = sys.argv[1:] or ["tiny"]
    name = args[0]
    rounds = int(args[1]) if len(args) > 1 else -1
    run(name, rounds)
