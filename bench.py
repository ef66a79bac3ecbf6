"""Benchmark of the semi-naive fixpoint hot path on one GB300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hisa|reference]
                    [--workload rmat16|rmat13|er1000|sg20k|sg20k-literal|cspa|batch5]

Workload (default): REACH, Reach(f,t) <- Edge(f,t); Reach(f,t) <- Edge(f,m),
Reach(m,t), on an R-MAT graph of scale 16 (65,536 nodes) with 2**19 distinct
edges ((a,b,c,d) = (.57,.19,.19,.05), seed 3); |Reach| = 1,159,535,104 in 8
productive iterations.  One step is one whole run of the hot path: load the
EDB from device-resident columns, encode/sort/dedup/index it, and iterate
join -> sort/dedup -> set difference -> merge -> device termination test until
the fixpoint.

Metric: fixpoint derived tuples/s = |Reach| / step time, from CUDA events on
the engine's stream around each step (L2 flushed by a 512 MiB write between
steps, outside the events).  Beside it: the dominant kernel's achieved HBM
bandwidth against the measured copy peak, the CPU oracle timed on a bounded
sample of the same workload, and the end-to-end number through the C-ABI with
host buffers.  With N > 1 (torchrun) every rank runs an independent replica
(the path does not shard across GPUs in this build): weak scaling, value =
tuples of all ranks / slowest rank's time.

Other workloads (same line format, metric = all IDB tuples at the fixpoint per
second): sg20k (SG with x != y on both rules on the 20,000-node DAG; the
literal variant filters rule 1 only), cspa (the ten-rule points-to program on
the skewed Assign/Dereference inputs divided by 250, windows of 128 ids; the
undivided inputs derive more than a GPU holds), batch5 (many independent REACH
instances, one-by-one vs served).
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fixpoint derived tuples/s"
UNIT = "tuples/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["hisa", "reference"], default="hisa")
    ap.add_argument("--instances", type=int, default=4096, help="batch5: number of instances")
    ap.add_argument("--budget-gb", type=float, default=60.0,
                    help="batch5: serving admission budget (estimates; device memory in use peaked near 2.4x it)")
    ap.add_argument("--workload", choices=["rmat16", "rmat15", "rmat13", "er1000", "sg20k", "sg20k-literal", "cspa",
                                           "batch5"],
                    default="rmat16",
                    help="rmat16: the benchmark workload; rmat15/rmat13: smaller R-MAT graphs for profiler captures")
    ap.add_argument("--single-full", action="store_true",
                    help="keep full as one sorted array (without HISA_FLAG_LOG_FULL)")
    ap.add_argument("--no-dense", action="store_true",
                    help="sort raw join results instead of the grouped bitmap join (HISA_FLAG_NO_DENSE)")
    ap.add_argument("--load-factor", type=float, default=0.0, help="hash-index load factor (0: the library default)")
    ap.add_argument("--e2e-steps", type=int, default=10,
                    help="end-to-end steps timed (every one is reported)")
    ap.add_argument("--partitioned", action="store_true",
                    help="REACH hash-partitioned over the ranks (one all-to-all per iteration; strong scaling)")
    ap.add_argument("--no-sub", action="store_true",
                    help="rmat16: skip the compact sg20k / cspa / batch5 records of the default line")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--micro", choices=["sort", "merge", "join"], default=None,
                    help="sort/merge microbenchmark on random tuples (the shapes of the paper's Table 6)")
    ap.add_argument("--tuples", type=int, default=100_000_000)
    ap.add_argument("--key-bits", type=int, default=64, help="64: 2-arity tuples of uint32; 32: packed 16+16")
    return ap.parse_args()


def _workload(name):
    from paper_2311_02206_gb300 import workloads
    if name == "rmat16":
        s, d = workloads.config_reach_rmat()
        desc = ("REACH (2 rules) on R-MAT scale 16: 65,536 nodes, 2^19 distinct edges, "
                "(a,b,c,d)=(.57,.19,.19,.05), no self-loops, seed 3")
        return s, d, desc, 65536
    if name == "rmat15":
        s, d = workloads.rmat_graph(15, 1 << 18, 3)
        return s, d, "REACH (2 rules) on R-MAT scale 15: 32,768 nodes, 2^18 distinct edges, seed 3", 1 << 15
    if name == "rmat13":
        s, d = workloads.rmat_graph(13, 1 << 16, 3)
        return s, d, "REACH (2 rules) on R-MAT scale 13: 8,192 nodes, 2^16 distinct edges, seed 3", 1 << 13
    s, d = workloads.config_reach_er()
    return s, d, "REACH (2 rules) on Erdos-Renyi n=1,000, m=3,000, seed 0", 1000


def _program_workload(name):
    """(program, EDB columns, description, CPU-sample function) of the
    non-REACH workloads.  The CPU sample runs the oracle as it stands."""
    from paper_2311_02206_gb300 import programs, workloads
    if name.startswith("sg20k"):
        prog = programs.SG_LITERAL if name.endswith("literal") else programs.SG
        s, d = workloads.config_sg_dag()
        desc = ("SG (%s) on a random DAG: 20,000 nodes, 40,000 distinct edges u<v, v-u in [1,256], seed 1"
                % ("x != y on rule 1 only" if name.endswith("literal") else "x != y on both rules"))

        def sample(nodes=3000):
            # edges point to larger ids, so every derivation of SG(x, y) with
            # x, y < N uses nodes < N only: SG of the induced subgraph on
            # [0, N) is exactly SG restricted to [0, N)^2
            import oracle
            keep = (s < nodes) & (d < nodes)
            t0 = time.perf_counter()
            r = oracle.seminaive(*prog, {"Edge": (s[keep], d[keep])})
            el = time.perf_counter() - t0
            n = r.size("SG")
            return n, el, f"SG restricted to nodes [0, {nodes}) of 20,000 (the induced subgraph; exact)"
        return prog, {"Edge": (s, d)}, desc, sample
    if name == "cspa":
        edb = workloads.config_cspa()
        desc = ("ten-rule points-to program (ValueFlow/MemoryAlias/ValueAlias) on Assign %d / Dereference %d "
                "pairs over 1,200 ids (the 400k/200k/300k inputs divided by 250), Zipf 1.1, 80%% of pairs in "
                "aligned windows of 128 ids, seed 2" % (len(edb["Assign"][0]), len(edb["Dereference"][0])))

        def sample():
            import oracle
            small = workloads.config_cspa(1000, 32)
            t0 = time.perf_counter()
            r = oracle.seminaive(*oracle.CSPA, small)
            el = time.perf_counter() - t0
            n = sum(r.size(k) for k in ("ValueFlow", "MemoryAlias", "ValueAlias"))
            return n, el, "the same program and generator divided by 1,000 (windows of 32 ids)"
        return programs.CSPA, edb, desc, sample
    raise ValueError(name)


# ---- distributed plumbing -------------------------------------------------------------------

def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _init_pg(world):
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce_over_ranks(x, world, op):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"   # gloo (the CPU tests) reduces host tensors
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def _max_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce_over_ranks(x, world, dist.ReduceOp.MAX)


def _sum_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce_over_ranks(x, world, dist.ReduceOp.SUM)


# ---- clocks ---------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples (every 200 ms) of this GPU while the timed region runs."""
    Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.rows = []
        self.proc = None

    def __enter__(self):
        self.started = threading.Event()
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi's start-up (driver and NVML initialisation) stalls the
            # GPU's work for up to seconds: the timed region starts only after
            # its first sample
            self.started.wait(timeout=30)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 10 and (not self.uuid or self.uuid in f[1]):
                self.rows.append(f)
                self.started.set()
        self.started.set()

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in self.rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[6 + i].strip() == "Active"})
        pw = [float(r[4]) for r in self.rows if r[4].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


# ---- roofline helpers -------------------------------------------------------------------------

def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


KERNEL_SOURCES = {   # the sources a kernel's counters depend on
    "radix_pass": ["radix.cuh", "common.cuh"],
    "setop_diff_merge": ["setops.cuh", "common.cuh"],
    "join_write": ["join.cuh", "common.cuh"],
    "join_count": ["join.cuh", "common.cuh"],
    "join_dense_mark": ["dense.cuh", "join.cuh", "common.cuh"],
    "join_dense_pull": ["dense.cuh", "join.cuh", "common.cuh"],
    "join_dense_emit": ["dense.cuh", "join.cuh", "common.cuh"],
    "setop_diff_probe": ["setops.cuh", "common.cuh"],
    "bit_join": ["bitjoin.cuh", "common.cuh"],
    "matrix_diff": ["matrix.cuh", "setops.cuh", "common.cuh"],
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, "paper_2311_02206_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# ---- CPU oracle baseline ----------------------------------------------------------------------

def host_description():
    """CPU model, logical CPUs and RAM of the machine the CPU baseline ran on."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":", 1)[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    ram_gb = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemTotal:"):
                ram_gb = round(int(line.split()[1]) / (1 << 20), 1)
                break
    except (OSError, ValueError, IndexError):
        pass
    return {"cpu_model": model or platform.processor() or "unknown", "arch": platform.machine(),
            "nproc": os.cpu_count(), "ram_gb": ram_gb}


def cpu_baseline(s, d, nodes, targets=64, seed=7):
    """The oracle as it stands (single-threaded std::set semi-naive), on REACH
    restricted to `targets` random target columns: exactly Reach on V x T."""
    import numpy as np
    import oracle
    T = np.random.default_rng(seed).choice(nodes, min(targets, nodes), replace=False).astype(np.uint32)
    t0 = time.perf_counter()
    r = oracle.reach_targets(s, d, T)
    el = time.perf_counter() - t0
    n = r.size("Reach")
    return {"value": n / el, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_description(),
            "sample": f"REACH restricted to {len(T)} of {nodes} target columns "
                      f"({n} tuples, {el:.1f} s; the recursive rule keeps the target column, so "
                      f"this is exactly Reach on V x T)"}


# ---- the GPU arm --------------------------------------------------------------------------------

def _profile_lines(kernel, workload):
    """Machine-readable lines of the committed ncu summary of `kernel` on
    `workload` (profiles/<kernel>_<workload>.md), if it was taken on the
    current sources: {'traffic': DRAM bytes per launch, 'limiter': text}."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    out = {}
    try:
        for line in open(path):
            if line.startswith("traffic_bytes_per_launch:"):
                parts = line.split()
                if parts[3] != kernel_source_hash(kernel):
                    return {}
                out["traffic"] = float(parts[1])
            elif line.startswith("limiter:"):
                out["limiter"] = line.split(":", 1)[1].strip()
    except (OSError, IndexError, ValueError):
        return {}
    return out


def _path_description(kstats):
    """Which evaluation the engine chose, from the kernels that ran."""
    if "bit_join" in kstats:
        return ("full and delta as bit matrices over (first, second column): per tuple (x, y) of the inner "
                "relation delta's row y ORed into row x, AND-NOT full, ORed into full (bitjoin.cuh)")
    if "join_dense_mark" in kstats:
        full = "a bit matrix" if "matrix_merge" in kstats else "sorted levels"
        return f"grouped bitmap join (push/pull per group), full as {full}"
    return "sort of raw join results, set difference and merge of sorted arrays"


def _timed_steps(ctx, dev_edb, steps, warmup, flush, kstats=None):
    """`warmup` untimed steps, then `steps` steps timed with CUDA events on the
    engine's stream (L2 flushed between steps, outside the events).  A step
    reloads the EDB from device columns and runs to the fixpoint."""
    import torch
    stream = torch.cuda.current_stream()

    def step():
        ctx.reset_edb()
        for k, (c0, c1) in dev_edb.items():
            ctx.load_tuples(k, c0, c1)
        return ctx.run()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ms, launches, st = [], 0, None
    for k in range(steps):
        flush.fill_(k)
        ev0.record(stream)
        st = step()
        ev1.record(stream)
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
        launches += st.kernel_launches
        if kstats is not None:
            for e in ctx.kernel_stats():
                acc = kstats.setdefault(e["name"], {"launches": 0, "ms": 0.0, "bytes": 0.0})
                acc["launches"] += e["launches"]
                acc["ms"] += e["ms"]
                acc["bytes"] += e["bytes"]
    return ms, launches, st


def _e2e(prog, edb, sizes, extra, load_factor, steps, local, world):
    """The metric end to end through the C-ABI with page-locked host buffers:
    each step copies the EDB in, runs to the fixpoint on the device (CUDA-graph
    while loop) and reads every IDB relation back in lexicographic order.
    Host timers around each part of each step explain the total."""
    import numpy as np
    import torch
    from paper_2311_02206_gb300 import hisa

    def pinned(x):
        return torch.from_numpy(x.view(np.int32)).pin_memory().numpy().view(np.uint32)

    idb_names = list(sizes)
    host_edb = {k: (pinned(c0), pinned(c1)) for k, (c0, c1) in edb.items()}
    outs = {k: (torch.empty(max(sizes[k], 1), dtype=torch.int32).pin_memory().numpy().view(np.uint32),
                torch.empty(max(sizes[k], 1), dtype=torch.int32).pin_memory().numpy().view(np.uint32))
            for k in idb_names}
    edb_bytes = sum(c0.nbytes + c1.nbytes for c0, c1 in edb.values())
    n_all = sum(sizes.values())
    ectx = hisa.Context(device=local, flags=hisa.FLAG_GRAPH | extra, load_factor=load_factor)
    ectx.program(*prog)

    def estep():
        t0 = time.perf_counter()
        ectx.reset_edb()
        for k, (c0, c1) in host_edb.items():
            ectx.load_tuples(k, c0, c1)
        ectx.run()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        got = sum(len(ectx.read_relation(k, out=outs[k])[0]) for k in idb_names)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return got, (t1 - t0) * 1e3, (t2 - t1) * 1e3

    estep()   # first use: buffers grow and caching-allocator blocks are created
    estep()
    torch.cuda.synchronize()
    tot, run_ms, read_ms = [], [], []
    t0 = time.perf_counter()
    for _ in range(steps):
        got, r, rd = estep()
        tot.append(round(r + rd, 2))
        run_ms.append(round(r, 2))
        read_ms.append(round(rd, 2))
        assert got == n_all
    et = time.perf_counter() - t0
    ectx.close()
    ev = _sum_over_ranks(float(n_all) * steps, world) / _max_over_ranks(et, world)
    return {"value": ev, "unit": UNIT, "h2d_bytes_per_step": int(edb_bytes), "d2h_bytes_per_step": int(8 * n_all),
            "steps": steps, "step_ms": tot, "load_run_ms": run_ms, "read_ms": read_ms,
            "loop": "CUDA graph while node (device-side termination test)"}


def _roofline(kstats, workload):
    peak, peak_kind = _peaks()
    dname, dk = max(kstats.items(), key=lambda kv: kv[1]["ms"])
    launches = max(dk["launches"], 1)
    per_launch_bytes = dk["bytes"] / launches
    avg_ms = dk["ms"] / launches
    achieved = dk["bytes"] / (dk["ms"] / 1e3) / 1e9 if dk["ms"] > 0 else 0.0
    prof = _profile_lines(dname, workload)
    traffic = prof.get("traffic")
    dram = traffic / (avg_ms / 1e3) / 1e9 if traffic and avg_ms > 0 else None
    kernel_ms_total = sum(v["ms"] for v in kstats.values())
    return {"bound": "hbm", "kernel": dname, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": peak_kind,
            "traffic": traffic, "algorithmic_bytes_per_launch": per_launch_bytes, "avg_launch_ms": avg_ms,
            "algorithmic_frac": round(achieved / peak, 4),
            "dram_achieved": round(dram, 1) if dram else None,
            "dram_frac": round(dram / peak, 4) if dram else None,
            "limiter": prof.get("limiter"),
            "note": ("achieved/frac: algorithmic bytes (what the step must move) per launch / launch time; "
                     "dram_achieved/dram_frac: ncu DRAM bytes per launch (traffic, committed profile of the "
                     "same sources) / launch time; limiter: what ncu shows bounds the kernel"),
            "share_of_kernel_time": round(dk["ms"] / kernel_ms_total, 4) if kernel_ms_total else None,
            "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                            "GBps": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 and v["bytes"] else None}
                        for k, v in sorted(kstats.items(), key=lambda kv: -kv[1]["ms"])}}


def _sub_program(name, local, flush, cpu, steps=5, warmup=3):
    """A compact record of a further workload: tuples/s of the device-resident
    fixpoint (CUDA-graph while loop, the production path), the kernel shares
    of one host-driven run with per-kernel events, the end-to-end number and
    the oracle on a bounded sample."""
    import numpy as np
    import torch
    from paper_2311_02206_gb300 import hisa
    prog, edb, desc, sample = _program_workload(name)
    idb_names = [k for k, v in prog[0].items() if v == "idb"]
    dev_edb = {k: (torch.from_numpy(c0.view(np.int32)).cuda(), torch.from_numpy(c1.view(np.int32)).cuda())
               for k, (c0, c1) in edb.items()}
    ctx = hisa.Context(device=local, flags=hisa.FLAG_GRAPH | hisa.FLAG_LOG_FULL)
    ctx.program(*prog)
    ms, launches, st = _timed_steps(ctx, dev_edb, steps, warmup, flush)
    sizes = {k: ctx.relation_size(k) for k in idb_names}
    ctx.close()
    kstats = {}
    kctx = hisa.Context(device=local, flags=hisa.FLAG_PHASE_TIMES | hisa.FLAG_LOG_FULL)
    kctx.program(*prog)
    _timed_steps(kctx, dev_edb, 1, 1, flush, kstats)
    kctx.close()
    torch.cuda.empty_cache()
    n_all = sum(sizes.values())
    tot_ms = sum(v["ms"] for v in kstats.values())
    top = [{"kernel": k, "ms_per_run": round(v["ms"], 3), "share": round(v["ms"] / tot_ms, 4)}
           for k, v in sorted(kstats.items(), key=lambda kv: -kv[1]["ms"])[:4]]
    rec = {"workload": desc, "value": n_all * steps / (sum(ms) / 1e3), "unit": UNIT,
           "ms_per_step": sum(ms) / steps, "step_ms": [round(x, 3) for x in ms], "steps": steps, "warmup": warmup,
           "idb_tuples": sizes, "iterations": st.iterations, "gpu_launches": launches,
           "loop": "CUDA graph while node", "kernels_host_driven_run": top,
           "e2e": _e2e(prog, edb, sizes, hisa.FLAG_LOG_FULL, 0.0, 3, local, 1)}
    torch.cuda.empty_cache()
    if cpu:
        n_s, el, what = sample()
        rec["cpu_baseline"] = {"value": n_s / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"{what}: {n_s} tuples in {el:.1f} s"}
    return rec


def run_hisa(a):
    import numpy as np
    import torch

    from paper_2311_02206_gb300 import build, hisa, programs

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    _init_pg(world)
    build.build()
    reach = a.workload in ("rmat16", "rmat15", "rmat13", "er1000")
    if reach:
        s, d, desc, nodes = _workload(a.workload)
        prog, edb, sample = programs.REACH, {"Edge": (s, d)}, None
    else:
        prog, edb, desc, sample = _program_workload(a.workload)
    idb_names = [k for k, v in prog[0].items() if v == "idb"]
    dev_edb = {k: (torch.from_numpy(c0.view(np.int32)).cuda(), torch.from_numpy(c1.view(np.int32)).cuda())
               for k, (c0, c1) in edb.items()}
    flush = torch.empty(512 << 18, dtype=torch.int32, device="cuda")   # 512 MiB > 129 MB L2

    extra = (0 if a.single_full else hisa.FLAG_LOG_FULL) | (hisa.FLAG_NO_DENSE if a.no_dense else 0)
    ctx = hisa.Context(device=local, flags=hisa.FLAG_PHASE_TIMES | extra, load_factor=a.load_factor)
    ctx.program(*prog)
    uuid = str(torch.cuda.get_device_properties(local).uuid) if hasattr(
        torch.cuda.get_device_properties(local), "uuid") else ""
    kstats = {}
    for _ in range(a.warmup):          # warm-up outside the clock sampling
        ctx.reset_edb()
        for k, (c0, c1) in dev_edb.items():
            ctx.load_tuples(k, c0, c1)
        ctx.run()
    _barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    gc.disable()   # no collector pause between a step's host-driven iterations
    torch.cuda.nvtx.range_push("timed")   # profilers can keep to the timed steps (ncu --nvtx-include timed/)
    with ClockSampler(uuid) as clk:
        ms, launches, st = _timed_steps(ctx, dev_edb, a.steps, 0, flush, kstats)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    gc.enable()
    _barrier(world)
    wall = time.perf_counter() - wall0
    sizes = {k: ctx.relation_size(k) for k in idb_names}
    n_reach = sum(sizes.values())
    iters = st.iterations
    total_s = sum(ms) / 1e3
    slowest = _max_over_ranks(total_s, world)
    tuples_all = _sum_over_ranks(float(n_reach) * a.steps, world)
    value = tuples_all / slowest
    roofline = _roofline(kstats, a.workload)
    ctx.close()   # release its buffers before the end-to-end context allocates its own
    torch.cuda.empty_cache()

    e2e = None
    if not a.no_e2e:
        e2e = _e2e(prog, edb, sizes, extra, a.load_factor, a.e2e_steps, local, world)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        if reach:
            cpu = cpu_baseline(s, d, nodes)
        else:
            n_s, el, what = sample()
            cpu = {"value": n_s / el, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_description(),
                   "sample": f"{what}: {n_s} tuples in {el:.1f} s"}

    # the other workloads, compactly, on the default run at N = 1
    subs = None
    if world == 1 and a.workload == "rmat16" and not a.no_sub:
        subs = {}
        for name in ("sg20k", "cspa"):
            subs[name] = _sub_program(name, local, flush, cpu=not a.no_cpu_baseline)
        del flush
        torch.cuda.empty_cache()
        subs["batch5"] = batch5_record(a, cpu=not a.no_cpu_baseline)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": total_s * 1e3 / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": desc, "idb_tuples": sizes, "iterations": iters,
                   "edb_tuples": {k: int(len(c0)) for k, (c0, c1) in edb.items()},
                   "tuples_joined_last_step": int(st.tuples_joined),
                   "l2": "flushed by a 512 MiB write between steps (outside the timed events)",
                   "loop": "host-driven, CUDA events around every kernel",
                   "path": _path_description(kstats),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "step_ms": [round(x, 3) for x in ms], "wall_s_timed_region": round(wall, 3)},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if subs is not None:
        line["workloads"] = subs
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_partitioned(a):
    """REACH hash-partitioned over the ranks (paper_2311_02206_gb300.partitioned):
    rank r loads the r-th share of the edge list; every iteration joins locally,
    sends each new tuple to the owner of its first column (NCCL all-to-all),
    and the owners deduplicate, difference and merge; an all-reduce of |delta|
    ends the loop.  value = |Reach| / the slowest rank's time (strong scaling:
    the workload is fixed, N GPUs share it).  At N = 1 the exchange is local."""
    import numpy as np
    import torch

    from paper_2311_02206_gb300 import build, partitioned

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    _init_pg(world)
    build.build()
    s, d, desc, _nodes = _workload(a.workload)
    lo, hi = rank * len(s) // world, (rank + 1) * len(s) // world
    edges = [(torch.from_numpy(s[lo:hi].view(np.int32).copy()).cuda(),
              torch.from_numpy(d[lo:hi].view(np.int32).copy()).cuda())]
    ops = partitioned.CudaPartOps()
    ex = partitioned.TorchExchange() if world > 1 else partitioned.LocalExchange(1)
    flush = torch.empty(512 << 18, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        full, b, counts = partitioned.reach_partitioned(edges, ops, ex)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    uuid = str(torch.cuda.get_device_properties(local).uuid) if hasattr(
        torch.cuda.get_device_properties(local), "uuid") else ""
    ms = []
    _barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clk:
        for k in range(a.steps):
            flush.fill_(k)
            _barrier(world)
            ev0.record(stream)
            full, b, counts = partitioned.reach_partitioned(edges, ops, ex)
            ev1.record(stream)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
    _barrier(world)
    mine = sum(int(f.numel()) for f in full)
    total = int(_sum_over_ranks(float(mine), world))
    slowest = _max_over_ranks(sum(ms) / 1e3, world)
    line = {
        "metric": METRIC, "value": total * a.steps / slowest, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": slowest * 1e3 / a.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": desc + ", hash-partitioned over the GPUs by the first column",
                   "idb_tuples": {"Reach": total}, "iterations": len(counts),
                   "l2": "flushed by a 512 MiB write between steps (outside the timed events)",
                   "loop": "host-driven; per iteration: join, hash partition, all-to-all, sort + unique, "
                           "difference + merge, all-reduce of |delta|",
                   "parallelism": f"hash partition over {world} GPU(s)",
                   "step_ms": [round(x, 3) for x in ms]},
        "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---- the reference arm: the CPU oracle as it stands ---------------------------------------------

def run_reference(a):
    import numpy as np
    import oracle

    world, rank, _ = _dist()
    if rank != 0:
        return
    if a.workload not in ("rmat16", "rmat15", "rmat13", "er1000"):
        return run_reference_program(a)
    s, d, desc, nodes = _workload(a.workload)
    rng = np.random.default_rng(11)
    per_step_targets = 16 if a.workload == "rmat16" else nodes
    oracle.build()

    def step():
        T = rng.choice(nodes, per_step_targets, replace=False).astype(np.uint32)
        t0 = time.perf_counter()
        r = oracle.reach_targets(s, d, T) if per_step_targets < nodes else oracle.reach(s, d)
        return r.size("Reach"), time.perf_counter() - t0

    for _ in range(a.warmup):
        step()
    tot_n, tot_t = 0, 0.0
    for _ in range(a.steps):
        n, t = step()
        tot_n += n
        tot_t += t
    value = tot_n / tot_t
    sample = (f"each step: REACH restricted to {per_step_targets} random target columns of {nodes} "
              f"(exact Reach on V x T)") if per_step_targets < nodes else "each step: the whole workload"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": tot_t * 1e3 / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_program(a):
    """The oracle on the bounded sample of a non-REACH workload, every step."""
    import oracle
    world, _, _ = _dist()
    oracle.build()
    _prog, _edb, desc, sample = _program_workload(a.workload)
    for _ in range(a.warmup):
        sample()
    tot_n, tot_t, what = 0, 0.0, ""
    for _ in range(a.steps):
        n, t, what = sample()
        tot_n += n
        tot_t += t
    value = tot_n / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": tot_t * 1e3 / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "each step: " + what},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- batched / served REACH (many independent instances) ------------------------------------------

def batch5_record(a, cpu=True):
    """Independent REACH instances (n log-uniform in [64, 8192], mean out-degree
    uniform in [1.5, 4], ER edges, seed 4) served three ways on one GPU:
    one by one (a run per instance), and through the serving loop with Poisson
    arrivals at 0.5x and 2x the one-by-one service rate (continuous batching:
    admission at iteration boundaries by free slots and memory budget,
    retirement on convergence), and all at once.  Latency = arrival -> result
    on the host.  Every served instance is compared with its one-by-one run;
    the CPU leg runs the oracle on instances drawn at random and compares
    those with the one-by-one results too."""
    import numpy as np
    import torch

    from paper_2311_02206_gb300 import build, hisa, programs, workloads

    build.build()
    specs = workloads.batch_instances(a.instances, 4)
    graphs = [workloads.er_graph(n, m, sd) for n, m, sd in specs]
    nmax = max(n for n, _, _ in specs)
    rng_pick = np.random.default_rng(12)
    order = rng_pick.permutation(len(graphs))
    cpu_pick = [int(i) for i in order if specs[i][0] <= 2048][:24]
    cpu_keep = set(cpu_pick)
    kept = {}

    def dev_fp(c0, c1):
        """Order-independent hash of a relation held in two int32 CUDA tensors,
        left on the device (compared after the timed loops: no sync per instance)."""
        x = ((c0.to(torch.int64) & 0xFFFFFFFF) << 32) | (c1.to(torch.int64) & 0xFFFFFFFF)
        x = x * -7046029254386353131          # 0x9E3779B97F4A7C15 as int64 (wrapping)
        x = x ^ ((x >> 29) & ((1 << 35) - 1))
        x = x * -4658895280553007687          # 0xBF58476D1CE4E5B9 as int64
        return x.sum()

    # the autotuner picks the knobs of each mode on a fixed sample of instances
    from paper_2311_02206_gb300 import autotune
    tune_rng = np.random.default_rng(21)
    samp_one = [int(i) for i in tune_rng.choice(len(graphs), min(256, len(graphs)), replace=False)]
    samp_srv = [int(i) for i in tune_rng.choice(len(graphs), min(512, len(graphs)), replace=False)]
    bmax = max(1, int(nmax).bit_length())
    islots = 1
    while islots < min(len(graphs), 4096):
        islots *= 2

    def trial_one(cfg):
        c = hisa.Context(flags=hisa.FLAG_GRAPH, **cfg)
        c.program(*programs.REACH)
        t0 = time.perf_counter()
        for i in samp_one:
            c.reset_edb()
            c.load_tuples("Edge", *graphs[i])
            c.run()
            c.read_relation("Reach", device=True)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        c.close()
        return el

    def trial_served(cfg):
        c = hisa.Context(**cfg)
        c.program(*programs.REACH)
        c.serve_open(islots, nmax, budget_bytes=int(a.budget_gb * (1 << 30)))
        t0 = time.perf_counter()
        tk = {c.serve_submit("Edge", *graphs[i]): i for i in samp_srv}
        while tk:
            if c.serve_step(1)["retired"]:
                for t in c.serve_retired():
                    c.serve_result(t, "Reach", device=True)
                    c.serve_release(t)
                    del tk[t]
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        c.close()
        torch.cuda.empty_cache()
        return el

    nedb = sum(len(g[0]) for g in graphs) // max(1, len(graphs))
    tuned_one = autotune.tune(trial_one, autotune.shape_key("reach", bmax, 0, nedb, "one_by_one"),
                              autotune.knob_candidates(False, False), rounds=1)
    tuned_srv = autotune.tune(trial_served, autotune.shape_key("reach", bmax, islots.bit_length(), nedb, "served"),
                              autotune.knob_candidates(2 * bmax + islots.bit_length() > 32, True), rounds=1)
    torch.cuda.empty_cache()

    # one by one
    ctx = hisa.Context(flags=hisa.FLAG_GRAPH, **tuned_one["config"])
    ctx.program(*programs.REACH)
    alone = {}
    lat1 = []
    for i in range(min(3, len(graphs))):   # warm-up
        ctx.reset_edb()
        ctx.load_tuples("Edge", *graphs[i])
        ctx.run()
    t_all = time.perf_counter()
    for i, (s, d) in enumerate(graphs):
        t0 = time.perf_counter()
        ctx.reset_edb()
        ctx.load_tuples("Edge", s, d)
        ctx.run()
        c0, c1 = ctx.read_relation("Reach", device=True)
        torch.cuda.synchronize()
        lat1.append(time.perf_counter() - t0)
        alone[i] = (c0.numel(), ctx.delta_counts("Reach"), dev_fp(c0, c1))
        if i in cpu_keep:
            kept[i] = (c0.cpu().numpy().view(np.uint32), c1.cpu().numpy().view(np.uint32), alone[i][1])
    t1 = time.perf_counter() - t_all
    ctx.close()
    torch.cuda.empty_cache()
    rate1 = len(graphs) / t1
    tuples = sum(v[0] for v in alone.values())

    fp_alone = torch.stack([alone[i][2] for i in range(len(graphs))])

    def served(lam, seed):
        rng = np.random.default_rng(seed)
        arrivals = np.cumsum(rng.exponential(1.0 / lam, len(graphs))) if lam else np.zeros(len(graphs))
        sctx = hisa.Context(**tuned_srv["config"])
        sctx.program(*programs.REACH)
        slots = 1
        while slots < min(len(graphs), 4096):
            slots *= 2
        sctx.serve_open(slots, nmax, budget_bytes=int(a.budget_gb * (1 << 30)))
        tickets, lat, done, fps = {}, {}, set(), {}
        nxt = 0
        start = time.perf_counter()
        while len(done) < len(graphs):
            now = time.perf_counter() - start
            while nxt < len(graphs) and arrivals[nxt] <= now:
                tickets[sctx.serve_submit("Edge", *graphs[nxt])] = nxt
                nxt += 1
            st = sctx.serve_step(1)
            if st["retired"]:
                tnow = time.perf_counter() - start
                for t in sctx.serve_retired():
                    i = tickets[t]
                    if i not in done:
                        done.add(i)
                        lat[i] = tnow - arrivals[i]
                        c0, c1, dc = sctx.serve_result(t, "Reach", device=True)
                        if c0.numel() != alone[i][0] or dc != alone[i][1]:
                            raise RuntimeError(f"instance {i} differs between served and one-by-one runs")
                        fps[i] = dev_fp(c0, c1)
                        sctx.serve_release(t)
                        del tickets[t]
            elif st["active"] == 0 and st["pending"] == 0 and nxt < len(graphs):
                time.sleep(max(0.0, min(0.01, arrivals[nxt] - (time.perf_counter() - start))))
        wall = time.perf_counter() - start
        if not bool((torch.stack([fps[i] for i in range(len(graphs))]) == fp_alone).all()):
            raise RuntimeError("an instance's tuples differ between served and one-by-one runs")
        sctx.close()
        torch.cuda.empty_cache()
        v = np.array([lat[i] for i in range(len(graphs))])
        return {"lambda_per_s": lam, "p50_ms": float(np.percentile(v, 50) * 1e3),
                "p99_ms": float(np.percentile(v, 99) * 1e3), "instances_per_s": len(graphs) / wall,
                "tuples_per_s": tuples / wall, "wall_s": wall}

    res = {
        "metric": "batched p50/p99 latency and throughput vs one-by-one", "unit": "ms / instances/s",
        "config": {"workload": f"{len(graphs)} independent REACH instances, n log-uniform in [64, 8192], "
                               "mean out-degree uniform in [1.5, 4], ER edges, seed 4, Poisson arrivals",
                   "sum_reach_tuples": tuples, "budget_gb": a.budget_gb},
        "one_by_one": {"instances_per_s": rate1, "tuples_per_s": tuples / t1,
                       "p50_ms": float(np.percentile(lat1, 50) * 1e3), "p99_ms": float(np.percentile(lat1, 99) * 1e3),
                       "note": "latency of a run started on an idle GPU (no queueing); results read into device memory"},
        "served_all_at_once": served(0, 1),
        "served_0.5x": served(0.5 * rate1, 2),
        "served_2x": served(2.0 * rate1, 3),
        "exact": "every served instance equals its one-by-one run (size, delta counts, device hash of the tuples)",
        "autotune": {"one_by_one": {k: tuned_one[k] for k in ("config", "trials", "seconds", "cached")},
                     "served": {k: tuned_srv[k] for k in ("config", "trials", "seconds", "cached")},
                     "sample": f"{len(samp_one)} instances one by one, {len(samp_srv)} served all at once",
                     "knobs": "radix_items (sort tile), load_factor (hashed run index), dense_unit (join work "
                              "split), pull_ratio (push/pull switch point)"},
    }
    res["served_2x_vs_one_by_one"] = res["served_2x"]["instances_per_s"] / rate1
    if cpu:
        import oracle
        budget_s, n_done, n_tup, el, mism = 15.0, 0, 0, 0.0, 0
        for i in cpu_pick:
            if el > budget_s:
                break
            t0 = time.perf_counter()
            r = oracle.reach(*graphs[i])
            el += time.perf_counter() - t0
            w0, w1 = r.relations["Reach"]
            g0, g1, gdc = kept[i]
            if not (np.array_equal(w0, g0) and np.array_equal(w1, g1) and gdc == r.delta_counts["Reach"]):
                mism += 1
            n_done += 1
            n_tup += len(w0)
        res["cpu_baseline"] = {"value": n_done / el, "unit": "instances/s", "tuples_per_s": n_tup / el, "cores": 1,
                               "kind": "oracle", "sample": f"{n_done} instances of at most 2,048 nodes drawn at "
                                                           f"random ({n_tup} tuples, {el:.1f} s)",
                               "oracle_equal_one_by_one": f"{n_done - mism} of {n_done}"}
        if mism:
            raise RuntimeError(f"{mism} sampled instances differ from the oracle")
    return res


def run_batch5(a):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(batch5_record(a, cpu=not a.no_cpu_baseline)), flush=True)


# ---- sort / merge microbenchmark ----------------------------------------------------------------

def run_micro(a):
    """Sort (LSD radix + unique) or difference/merge of N random 2-arity tuples,
    timed alone with CUDA events; algorithmic bytes: each radix pass reads and
    writes every code, the merge reads both inputs and writes both outputs."""
    import torch
    from paper_2311_02206_gb300 import build, hisa

    build.build()
    g = torch.Generator(device="cuda").manual_seed(5)
    n = a.tuples
    wide = a.key_bits > 32
    dt = torch.int64 if wide else torch.int32
    kb = 8 if wide else 4
    hi = (1 << 62) if wide else (1 << 31)
    keys = torch.randint(0, hi, (n,), generator=g, device="cuda", dtype=torch.int64)
    if wide:
        keys = keys * 4 + torch.randint(0, 4, (n,), generator=g, device="cuda", dtype=torch.int64)
    else:
        keys = (keys * 2 + torch.randint(0, 2, (n,), generator=g, device="cuda", dtype=torch.int64)).to(torch.int32)
    flush = torch.empty(512 << 18, dtype=torch.int32, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.micro == "join":
        # Algorithm 3 as in REACH: outer (m, t) codes probe the R-MAT 16 edge index
        # on m (codes (m, f)); results (f, t).  About 8 results per outer tuple.
        import numpy as np
        from paper_2311_02206_gb300 import workloads
        es, ed = workloads.config_reach_rmat()
        inner_np = np.unique((ed.astype(np.uint64) << np.uint64(16)) | es.astype(np.uint64)).astype(np.uint32)
        inner = torch.from_numpy(inner_np.view(np.int32)).cuda()
        m = ed[torch.randint(0, len(ed), (n,), generator=torch.Generator().manual_seed(3)).numpy()]
        t = torch.randint(0, 1 << 16, (n,), generator=torch.Generator().manual_seed(4)).numpy().astype(np.uint32)
        outer_np = np.sort((m.astype(np.uint32) << np.uint32(16)) | t)
        outer = torch.from_numpy(outer_np.view(np.int32)).cuda()

        def op():
            return hisa.join_codes(outer, inner, 16, 0, 3, 1)
        res = op()
        alg = 2 * 4 * res.numel() + 12 * n
    elif a.micro == "sort":
        def op():
            return hisa.sort_codes(keys, a.key_bits)
        passes = (a.key_bits + 7) // 8
        alg = passes * 2 * kb * n
    else:
        full = hisa.sort_unique_codes(keys, a.key_bits)
        fresh = hisa.sort_codes(keys[: n // 10].roll(1) ^ 1 if not wide else keys[: n // 10] ^ 1, a.key_bits)
        def op():
            return hisa.difference_merge(full, fresh)
        d, f = op()
        alg = kb * (full.numel() + fresh.numel() + f.numel() + d.numel())
    for _ in range(a.warmup):
        op()
    ms = []
    for k in range(a.steps):
        flush.fill_(k)
        ev0.record()
        op()
        ev1.record()
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    t = statistics.median(ms)
    peak, kind = _peaks()
    print(json.dumps({"micro": a.micro, "tuples": n, "key_bits": a.key_bits, "ms_median": t,
                      "ms": [round(x, 3) for x in ms], "algorithmic_GBps": alg / (t / 1e3) / 1e9,
                      "frac_of_hbm_peak": alg / (t / 1e3) / 1e9 / peak, "peak_source": kind,
                      "note": "call includes scratch allocation and the size read-back"}), flush=True)


if __name__ == "__main__":
    args = _args()
    if args.micro:
        run_micro(args)
    elif args.workload == "batch5" and args.impl == "hisa":
        run_batch5(args)
    elif args.partitioned and args.impl == "hisa":
        run_partitioned(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_hisa(args)
