"""Write the stored oracle results under tests/golden/.

Every value written here comes from the CPU oracle (``oracle``) applied to
inputs from the seeded generator (``lbdd_inputs``); nothing is taken from
the CUDA path.  The paper prints no numeric worked example (its Figures 1
and 2 are not reproducible from the text), so these files pin the oracle's
own canonical results for regression and for GPU parity at sizes where
re-running the oracle inside a test would take too long.

Usage:  python tests/golden/make_golden.py tiny | city [rounds] | large|wide [rounds] [--table]
        | batch [count [procs]]

A prefix of the large or wide instance is written only if it applies at least one
refinement (moves > 0), so that its parity test covers the applied paths;
``--table`` also stores digests of the oracle's best-transfer table for the
prefix's allotment.
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


def run(name: str, rounds: int = -1, table: bool = False) -> dict:
    inst = lbdd_inputs.make_named(name)
    t0 = time.time()
    res = oracle.asral(inst.cm, inst.cap, inst.pen, mode=oracle.MODE_HEAP, max_rounds=rounds)
    secs = time.time() - t0
    if res.rc != oracle.OK:
        raise SystemExit(f"oracle failed: {res.rc}")
    if name in ("large", "wide") and rounds >= 0 and res.stats["moves"] == 0:
        raise SystemExit(f"the first {rounds} rounds apply no refinement; take a longer prefix")
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
    if table:
        tc, td = oracle.best_transfer(inst.cm, res.assign)
        out["table_tc_sha256"] = digest(np.where(tc >= oracle.INF, 2**31 - 1, tc).astype(np.int32))
        out["table_td_sha256"] = digest(td.astype(np.int32))
    suffix = "" if rounds < 0 else f"_r{rounds}"
    path = os.path.join(HERE, f"{name}{suffix}_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(path, out["delta"], f"{secs:.1f}s")
    return out


def _batch_one(i: int) -> dict:
    inst = lbdd_inputs.make(lbdd_inputs.batch_recipe(i))
    t0 = time.time()
    res = oracle.asral(inst.cm, inst.cap, inst.pen, mode=oracle.MODE_HEAP)
    if res.rc != oracle.OK:
        raise RuntimeError(f"oracle failed on instance {i}: {res.rc}")
    return {"i": i, "n": inst.n, "k": inst.k, "seed": inst.recipe.seed, "delta": res.delta,
            "assign_sha256": digest(res.assign.astype(np.int32)),
            "oracle_seconds": round(time.time() - t0, 2)}


def run_batch(count: int = 256, procs: int = 4) -> None:
    """Oracle results of the batched mix (instance i: lbdd_inputs.batch_recipe(i)),
    one process per instance at a time; written when all are done."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    # largest first, so that the long ones do not end up last
    order = sorted(range(count), key=lambda i: -lbdd_inputs.batch_recipe(i).n *
                   lbdd_inputs.batch_recipe(i).k)
    with ctx.Pool(procs) as pool:
        rows = []
        for r in pool.imap_unordered(_batch_one, order):
            rows.append(r)
            print(f"{len(rows)}/{count} instance {r['i']} n={r['n']} k={r['k']} "
                  f"{r['oracle_seconds']}s", flush=True)
    rows.sort(key=lambda r: r["i"])
    path = os.path.join(HERE, f"batch{count}_oracle.json")
    with open(path, "w") as f:
        json.dump({"workload": f"batched mix, instances 0..{count - 1} of "
                               "lbdd_inputs.batch_recipe", "oracle_mode": "heap",
                   "source": "oracle.asral (CPU), written by tests/golden/make_golden.py",
                   "instances": rows}, f, indent=0)
        f.write("\n")
    print(path)


if __name__ == "__main__":
    args = sys.argv[1:] or ["tiny"]
    name = args[0]
    if name == "batch":
        run_batch(int(args[1]) if len(args) > 1 else 256, int(args[2]) if len(args) > 2 else 4)
    else:
        table = "--table" in args
        args = [a for a in args if a != "--table"]
        rounds = int(args[1]) if len(args) > 1 else -1
        run(name, rounds, table)
