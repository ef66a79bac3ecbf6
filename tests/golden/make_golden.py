"""Writes the stored expected values under tests/golden/ by calling the CPU
oracle only (``oracle/``); nothing here touches the CUDA path.

    python tests/golden/make_golden.py reach_rmat [--procs 8]
    python tests/golden/make_golden.py sg_dag

``reach_rmat``: REACH on R-MAT scale 16 with 2**19 edges (seed 3).  The full
oracle would hold ~1.1e9 tuples in std::set, so it is evaluated on disjoint
blocks of target columns: the recursive REACH rule keeps the ``to`` column of
its Reach atom, so Reach restricted to a target block T is the fixpoint of the
program seeded with Edge tuples ending in T (``oracle.reach_targets``), and
its delta at iteration k is delta_k restricted to V x T.  Sizes, delta counts
and fingerprints of the blocks add up to those of the whole relation.

``sg_dag``: SG (both rules with x != y) on the random DAG of 20,000 nodes and
40,000 edges (seed 1), evaluated in one piece; ``--literal`` takes the filter
on the first rule only.

``cspa``: the ten-rule points-to program on the skewed Assign/Dereference
inputs divided by ``--div`` (windows of ``--window`` ids, seed 2), evaluated
in one piece.  Beside the sizes, delta counts and fingerprints it stores the
whole sorted relations (``cspa_d<div>_w<window>.npz``: per IDB relation the
codes (c0 << 32) | c1 ascending, as uint64), so the GPU tests compare every
tuple and its position.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2311_02206_gb300 import workloads  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _block(args):
    lo, hi = args
    s, d = workloads.config_reach_rmat()
    r = oracle.reach_targets(s, d, np.arange(lo, hi, dtype=np.uint32))
    c0, c1 = r.relations["Reach"]
    return lo, r.size("Reach"), r.delta_counts["Reach"], oracle.fingerprint(c0, c1)


def reach_rmat(procs: int, block: int):
    t0 = time.time()
    n = 1 << 16
    jobs = [(lo, min(n, lo + block)) for lo in range(0, n, block)]
    total, counts, fp = 0, [], 0
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        for i, (lo, size, dc, f) in enumerate(pool.imap_unordered(_block, jobs)):
            total += size
            fp = (fp + f) % (1 << 64)
            if len(dc) > len(counts):
                counts += [0] * (len(dc) - len(counts))
            for k, c in enumerate(dc):
                counts[k] += c
            print(f"block {i + 1}/{len(jobs)} lo={lo} size={size} t={time.time() - t0:.0f}s", flush=True)
    s, d, draws = workloads.rmat_graph(16, 1 << 19, 3, return_draws=True)
    out = {
        "workload": "REACH on R-MAT scale 16, 2**19 distinct edges, (a,b,c,d)=(.57,.19,.19,.05), seed 3",
        "edges": int(len(s)),
        "raw_draws": int(draws),
        "reach_size": int(total),
        "delta_counts": counts,
        "fingerprint": str(fp),
        "oracle_cpu_seconds_total": round(time.time() - t0, 1),
        "procs": procs,
        "method": "oracle.reach_targets over disjoint target blocks of %d columns" % block,
    }
    with open(os.path.join(HERE, "reach_rmat_s16.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


def sg_dag(literal: bool):
    t0 = time.time()
    s, d = workloads.config_sg_dag()
    r = oracle.seminaive(*(oracle.SG_LITERAL if literal else oracle.SG), {"Edge": (s, d)})
    c0, c1 = r.relations["SG"]
    out = {
        "workload": ("SG (x != y on rule 1 only)" if literal else "SG (x != y on both rules)")
                    + " on a random DAG, n=20,000, m=40,000, gaps in [1,256], seed 1",
        "sg_size": int(r.size("SG")),
        "delta_counts": r.delta_counts["SG"],
        "fingerprint": str(oracle.fingerprint(c0, c1)),
        "oracle_cpu_seconds": round(time.time() - t0, 1),
    }
    with open(os.path.join(HERE, "sg_literal_dag_20k.json" if literal else "sg_dag_20k.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


def cspa(div: int, window: int):
    t0 = time.time()
    edb = workloads.config_cspa(div, window)
    r = oracle.seminaive(*oracle.CSPA, edb)
    out = {
        "workload": "points-to program, Assign %d / Dereference %d over %d ids, Zipf 1.1, 80%% in windows of %d, seed 2"
                    % (len(edb["Assign"][0]), len(edb["Dereference"][0]), 300_000 // div, window),
        "div": div,
        "window": window,
        "iterations": r.iterations,
        "oracle_cpu_seconds": None,
    }
    arrays = {}
    for name in ("ValueFlow", "MemoryAlias", "ValueAlias"):
        c0, c1 = r.relations[name]
        out[name] = {"size": int(r.size(name)), "delta_counts": r.delta_counts[name],
                     "fingerprint": str(oracle.fingerprint(c0, c1))}
        arrays[name] = (c0.astype(np.uint64) << np.uint64(32)) | c1.astype(np.uint64)
    np.savez_compressed(os.path.join(HERE, "cspa_d%d_w%d.npz" % (div, window)), **arrays)
    out["oracle_cpu_seconds"] = round(time.time() - t0, 1)
    with open(os.path.join(HERE, "cspa_d%d_w%d.json" % (div, window)), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["reach_rmat", "sg_dag", "cspa"])
    ap.add_argument("--literal", action="store_true", help="sg_dag: filter on rule 1 only")
    ap.add_argument("--div", type=int, default=250)
    ap.add_argument("--window", type=int, default=128)
    ap.add_argument("--procs", type=int, default=os.cpu_count())
    ap.add_argument("--block", type=int, default=256)
    a = ap.parse_args()
    if a.which == "reach_rmat":
        reach_rmat(a.procs, a.block)
    elif a.which == "cspa":
        cspa(a.div, a.window)
    else:
        sg_dag(a.literal)
