#!/usr/bin/env python
"""Star-forest Bcast/Reduce benchmark on GB300 (one JSON line on rank 0).

Workload (default): the unstructured SpMV-style scatter of Sec. IV.A -- 2^24 roots of a random
geometric 3-D graph (expected degree 14) split into 256 simulated ranks by coordinate
bisection; leaves are each rank's owned entries followed by its ghost columns; fp64 units of
bs = 1.  One step is the SpMV communication pair: lvec = Bcast_REPLACE(x) and
y = y + Reduce_SUM(lvec) (deterministic fold), both through the C ABI.

value = algorithmic bytes of the step / device time (CUDA events on the launching stream,
L2 flushed between steps by writing a 256 MiB buffer outside the timed events).
Algorithmic bytes: Bcast reads each connected root once, writes every leaf, plus 4 bytes per
index word the two-sided plan needs; Reduce reads every leaf, reads and writes each connected
root once, plus the same index words.

--impl reference times the oracle (plain C, single-threaded) on the host cores instead.
Multi-GPU (torchrun): every rank runs an independent replica (the simulated ranks already
live in one GPU's memory; nothing crosses GPUs), value = all replicas' bytes / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SF Bcast/Reduce effective HBM GB/s (% of peak); batched vs per-SF launch time"
# the kernels and the plan layout they read: DRAM traffic from a capture holds while these are unchanged
KERNEL_SOURCES = ["paper_2102_13018_gb300/csrc/sf_kernels.cuh", "paper_2102_13018_gb300/csrc/sf_plan.h",
                  "paper_2102_13018_gb300/csrc/sf_setup.cpp"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--npoints", type=int, default=1 << 24)
    ap.add_argument("--levels", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-pingpong", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--only", default="all", choices=["all", "halo", "autograd", "batched"],
                    help="run one extra section alone (halo exchange, autograd or the batch) and print it")
    ap.add_argument("--batch-forests", type=int, default=512)
    return ap.parse_args()


def workload_config(args, forest):
    return {
        "workload": f"spmv_scatter: random geometric 3-D graph, {args.npoints} roots (degree 14), "
                    f"{2 ** args.levels} simulated ranks by coordinate bisection, leaves = owned + "
                    f"{forest.meta['ghosts']} ghost columns, fp64 bs=1; step = Bcast REPLACE + Reduce SUM "
                    f"(deterministic)",
        "roots": int(forest.nroots.sum()),
        "leaves": int(forest.nedges),
        "ranks": int(forest.nranks),
        "l2": "flushed between steps (256 MiB write outside the timed events)",
        "parallelism": "replicas (one independent forest per GPU)",
    }


def algorithmic_bytes(info, unit_bytes=8):
    idx_words = info["edges_one_indexed"] + 2 * info["edges_two_indexed"]
    bcast = unit_bytes * info["connected_roots"] + unit_bytes * info["nedges"] + 4 * idx_words
    reduce = unit_bytes * info["nedges"] + 2 * unit_bytes * info["connected_roots"] + 4 * idx_words
    return bcast, reduce


def op_bytes(info, kind, op, unit_bytes):
    """Algorithmic bytes of one operation: Bcast reads each connected root once and writes every
    leaf (and reads it for an op other than REPLACE); Reduce reads every leaf and reads and
    writes each connected root; FetchAndOp adds the leafupdate writes; plus the index words."""
    idx = 4 * (info["edges_one_indexed"] + 2 * info["edges_two_indexed"])
    U, E, C = unit_bytes, info["nedges"], info["connected_roots"]
    if kind == "bcast":
        return U * C + U * E * (1 if op == "REPLACE" else 2) + idx
    if kind == "reduce":
        return U * E + 2 * U * C + idx
    return U * E + 2 * U * C + U * E + idx


def time_op(fn, stream, flush=None, reps=30, warm=3):
    """Median CUDA-event time (ms) of fn() on `stream`, each call alone (after an L2 flush if
    a flush buffer is given)."""
    import torch
    ts = []
    for i in range(reps + warm):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warm:
            ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        fields = {}
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                k, v = line.split(":", 1)
                fields.setdefault(k.strip().lower(), v.strip())
        return fields.get("model name") or f"implementer {fields.get('cpu implementer')} part {fields.get('cpu part')}"
    except OSError:
        return "unknown"


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (burst copy, MEASURED_PEAKS.json)"
    return 6800.0, "fallback 6.8 TB/s"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the kernel
    source is unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get(kernel)
    if not ent or ent.get("source_sha") != kernel_source_sha():
        return None
    return ent.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        dev = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
        if dev.isdigit():
            rows = [r for r in rows if r[0] == dev] or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def build_forest(args):
    import sfgen
    return sfgen.cfg3_spmv(args.npoints, args.levels)


def oracle_step_time(forest, x, lvec, y, reps=1):
    import oracle
    t0 = time.perf_counter()
    for _ in range(reps):
        lv = oracle.bcast(forest, "fp64", 1, x, lvec, "REPLACE")
        oracle.reduce(forest, "fp64", 1, lv, y, "SUM")
    return (time.perf_counter() - t0) / reps


def sample_forest(forest, keep):
    """The forest restricted to the leaves of leaf ranks 0..keep-1 (all roots kept)."""
    import numpy as np
    import sfgen
    P = forest.nranks
    nl = np.array([forest.nleaves[q] if q < keep else 0 for q in range(P)])
    il = [forest.ilocal[q] if q < keep else None for q in range(P)]
    rr = [forest.iremote_rank[q] if q < keep else np.zeros(0, np.int32) for q in range(P)]
    ri = [forest.iremote_index[q] if q < keep else np.zeros(0, np.int64) for q in range(P)]
    return sfgen.Forest(P, forest.nroots, nl, il, rr, ri, name=forest.name + f"_first{keep}", meta=forest.meta)


def run_reference(args):
    import numpy as np
    import oracle
    import sfgen
    forest = build_forest(args)
    # bound the whole run to about two minutes of oracle time
    budget = 120.0 / (args.steps + args.warmup)
    ro, lo = oracle.layout(forest)
    x = sfgen.data("fp64", int(ro[-1]), 3, 1)
    y = sfgen.data("fp64", int(ro[-1]), 3, 2)
    probe = sample_forest(forest, max(1, forest.nranks // 16))
    t_probe = oracle_step_time(probe, x, np.zeros(int(oracle.layout(probe)[1][-1])), y)
    est_full = t_probe * forest.nedges / max(probe.nedges, 1)
    keep = forest.nranks if est_full <= budget else max(1, int(forest.nranks * budget / est_full))
    sample = forest if keep == forest.nranks else sample_forest(forest, keep)
    lvec = np.zeros(int(oracle.layout(sample)[1][-1]))
    info = host_info(sample)
    bb, rb = algorithmic_bytes(info)
    for _ in range(args.warmup):
        oracle_step_time(sample, x, lvec, y)
    times = [oracle_step_time(sample, x, lvec, y) for _ in range(args.steps)]
    total = sum(times)
    value = (bb + rb) * args.steps / total / 1e9
    what = ("the full workload" if keep == forest.nranks else
            f"the leaves of the first {keep} of {forest.nranks} ranks ({sample.nedges} of {forest.nedges} edges)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, forest),
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value, "unit": "GB/s",
                             "sample": what + ", one Bcast REPLACE + one Reduce SUM per step"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_batched(args, stream, flush):
    """512 uneven forests (Zipf in-degree, mixed dtype / bs / op), each doing one Bcast and one
    Reduce: one library call per forest and operation vs one batched run (variant-grouped
    launches) vs the batched run replayed as one CUDA graph -- first with every Reduce
    deterministic and the default launch shapes, then with every forest tuned on its own
    (sf_autotune: Bcast path x vector width x tile size, Reduce mode x vector width x tile size;
    a Reduce the tuner sends to atomics is no longer bit-reproducible)."""
    import collections
    import numpy as np
    import torch
    import sfgen
    from paper_2102_13018_gb300 import Batch, StarForest
    tdt = {"fp32": torch.float32, "fp64": torch.float64, "int64": torch.int64}
    forests = sfgen.cfg4_batched(nforests=args.batch_forests)
    items, nbytes, edges = [], 0, 0
    for i, f in enumerate(forests):
        sf = StarForest.from_forest(f).setup().set_mode("deterministic")
        dt, bs = tdt[f.meta["dtype"]], f.meta["bs"]
        r = (torch.rand(sf.nroots_total * bs, device="cuda") * 100).to(dt)
        l = (torch.rand(sf.leaf_extent * bs, device="cuda") * 100).to(dt)
        r2, l2 = r.clone(), l.clone()
        info = sf.info()
        ub = bs * r.element_size()
        idx = 4 * (info["edges_one_indexed"] + 2 * info["edges_two_indexed"])
        nbytes += ub * info["connected_roots"] + ub * info["nedges"] + idx      # Bcast
        nbytes += ub * info["nedges"] + 2 * ub * info["connected_roots"] + idx  # Reduce
        edges += info["nedges"]
        items.append((sf, f.meta["op"], r, l, r2, l2, bs))
    ops = [("bcast", sf, op, r, l, bs) for sf, op, r, l, r2, l2, bs in items] + ["barrier"] + \
          [("reduce", sf, op, l2, r2, bs) for sf, op, r, l, r2, l2, bs in items]

    def per_forest():
        for sf, op, r, l, r2, l2, bs in items:
            sf.bcast(r, l, op, bs=bs, stream=stream)
        for sf, op, r, l, r2, l2, bs in items:
            sf.reduce(l2, r2, op, bs=bs, stream=stream)

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    def measure():
        batch = Batch().set_ops(ops)
        t_per = timed(per_forest)
        t_batch = timed(lambda: batch.run(use_graph=False, stream=stream))
        t_graph = timed(lambda: batch.run(use_graph=True, stream=stream))
        return {"per_forest_ms": t_per, "batched_ms": t_batch, "graph_ms": t_graph,
                "launches_batched": batch.launches(), "per_forest_gbs": nbytes / (t_per * 1e-3) / 1e9,
                "batched_gbs": nbytes / (t_batch * 1e-3) / 1e9, "graph_gbs": nbytes / (t_graph * 1e-3) / 1e9,
                "speedup_graph_vs_per_forest": t_per / t_graph}

    det = measure()
    t0 = time.perf_counter()
    for sf, op, r, l, r2, l2, bs in items:
        sf.set_mode("auto").set_path("auto")
        sf.autotune("bcast", r, l, op, bs=bs, stream=stream)
        sf.autotune("reduce", l2, r2, op, bs=bs, stream=stream)
    tune_s = time.perf_counter() - t0
    tuned = measure()
    choices = collections.Counter()
    for sf, *_ in items:
        t = sf.tuning()
        choices[f"{t['path']}/{t['mode']}/vec{t['vector_bytes']}/tile{t['tile_edges']}"] += 1
    tuned.update({"tuning_s": tune_s, "choices": dict(choices.most_common())})
    return {"workload": f"{len(items)} forests, nleaves log-uniform in [1e2,1e6], Zipf(1.1) in-degree, "
                        f"fp32/fp64/int64, bs in {{1,2,3,8}}, op in {{SUM,MAX,REPLACE}}; Bcast then Reduce each",
            "edges": int(edges), "algorithmic_bytes": int(nbytes), "launches_per_forest_path": 2 * len(items),
            "deterministic": det, "tuned": tuned,
            # the headline figures: the deterministic batch (results bit-identical to the oracle)
            "per_forest_ms": det["per_forest_ms"], "graph_ms": det["graph_ms"], "graph_gbs": det["graph_gbs"]}


def run_tiny(stream):
    """The plain tiny forest (4 ranks x 4096 roots, 16384 uniform leaves): every operation of
    the workload in int32 and fp64, bs = 1, each call timed alone.  Its 0.3 MB sit in L2, so
    these are launch- and L2-bound times (us) and L2-resident GB/s, not HBM figures."""
    import torch
    import sfgen
    from paper_2102_13018_gb300 import StarForest
    f = sfgen.cfg1_plain_tiny()
    sf = StarForest.from_forest(f).setup().set_mode("deterministic")
    info = sf.info()
    out = {"workload": "plain_tiny: 4 ranks x 4096 roots, 16384 leaves uniform over all roots, bs=1",
           "l2": "resident (no flush)"}
    for dt, tdt, w in (("int32", torch.int32, 4), ("fp64", torch.float64, 8)):
        x = (torch.rand(sf.nroots_total, device="cuda") * 1000).to(tdt)
        lv = (torch.rand(sf.leaf_extent, device="cuda") * 1000).to(tdt)
        upd = torch.zeros_like(lv)
        cases = [("bcast_replace", "bcast", "REPLACE", lambda: sf.bcast(x, lv, "REPLACE", stream=stream)),
                 ("bcast_sum", "bcast", "SUM", lambda: sf.bcast(x, lv, "SUM", stream=stream)),
                 ("reduce_sum", "reduce", "SUM", lambda: sf.reduce(lv, x, "SUM", stream=stream)),
                 ("reduce_max", "reduce", "MAX", lambda: sf.reduce(lv, x, "MAX", stream=stream)),
                 ("fetch_and_op_sum", "fetch", "SUM", lambda: sf.fetch_and_op(x, lv, upd, "SUM", stream=stream))]
        for label, kind, op, fn in cases:
            ms = time_op(fn, stream, None, reps=200, warm=10)
            nb = op_bytes(info, kind, op, w)
            out[f"{label}_{dt}"] = {"us": ms * 1e3, "bytes": nb, "l2_gbs": nb / (ms * 1e-3) / 1e9}
    return out


def abi_call_cost(sf, x, lv, n=20000):
    """Host time per Begin+End pair of the 1 KB ping-pong Bcast: straight through ctypes with the
    arguments built once (the C ABI's own cost plus the kernel launch it enqueues), and through
    the Python StarForest wrapper (argument marshalling added).  The kernel is a ~2 us copy, so
    the loop is bound by the host."""
    import ctypes
    import torch
    lib = sf._lib
    args = (sf._h, sf._unit(x, sf.nroots_total, None), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(lv.data_ptr()),
            0, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    begin, end = lib.sf_bcast_begin, lib.sf_bcast_end
    for _ in range(1000):
        begin(*args)
        end(*args)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n):
        begin(*args)
        end(*args)
    t_abi = (time.perf_counter() - t0) / n
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n):
        sf.bcast(x, lv, "REPLACE")
    t_py = (time.perf_counter() - t0) / n
    torch.cuda.synchronize()
    return {"ctypes_prebuilt_us": t_abi * 1e6, "python_wrapper_us": t_py * 1e6,
            "what": "host time per Bcast Begin+End (one kernel launch), 1 KB forest"}


def run_pingpong(stream):
    """Sec. VI.A ping-pong on one GPU: n fp64 roots on rank 0 connected consecutively to n leaves
    on rank 1; one round trip is Bcast REPLACE then Reduce REPLACE (the roots come back
    unchanged).  Median round-trip latency per message size, launched one call at a time and
    replayed as a CUDA graph.  The paper's Table I (Summit V100s, CUDA-aware MPI, two GPUs) is
    context only: here nothing leaves the GPU."""
    import torch
    import sfgen
    from paper_2102_13018_gb300 import StarForest
    out = {}
    for nbytes in (1 << 10, 1 << 12, 1 << 14, 1 << 16, 1 << 18, 1 << 20, 1 << 22):
        n = nbytes // 8
        sf = StarForest.from_forest(sfgen.pingpong(n)).setup().set_mode("deterministic")
        x = torch.rand(n, dtype=torch.float64, device="cuda")
        lv = torch.zeros(n, dtype=torch.float64, device="cuda")

        def trip():
            sf.bcast(x, lv, "REPLACE")
            sf.reduce(lv, x, "REPLACE")

        for _ in range(20):
            trip()
        torch.cuda.synchronize()
        reps = 200
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            trip()
        e1.record()
        torch.cuda.synchronize()
        plain_us = e0.elapsed_time(e1) * 1e3 / reps
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            trip()
        torch.cuda.current_stream().wait_stream(s)
        with torch.cuda.graph(g):
            for _ in range(10):
                trip()
        for _ in range(5):
            g.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps // 10):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        graph_us = e0.elapsed_time(e1) * 1e3 / reps
        out[f"{nbytes // 1024}K"] = {"plain_us": plain_us, "graph_us": graph_us}
        if nbytes == 1 << 10:
            out["abi_call_cost_1K"] = abi_call_cost(sf, x, lv)
    return {"what": "round trip Bcast REPLACE + Reduce REPLACE, contiguous 2-rank forest, fp64, one GPU",
            "paper_table1_sf_dd_us": {"1K": 22.8, "4K": 23.0, "16K": 22.9, "64K": 23.5, "256K": 27.7,
                                      "1024K": 46.3, "4096K": 111.8},
            "sizes": out}


def run_autograd(flush, peak):
    """Differentiable message passing on the power-law graph (2^20 roots, 2^23 leaves, bs = 64),
    through the library's autograd functions, fp32 and bf16: Bcast, Reduce SUM and Reduce MAX,
    each forward + backward, against the same computation in plain PyTorch (index_select /
    index_add_ / scatter_reduce: atomic, not reproducible).  Algorithmic bytes (U = 64 x element
    size, E leaves, C connected roots, NR roots, 4 bytes per index):
      Bcast fwd U(C + E) + 4E, bwd (Reduce SUM from zero) U(E + NR) + 4E;
      Reduce SUM fwd U(E + NR) + 4E, bwd (Bcast) U(C + E) + 4E;
      Reduce MAX fwd U(E + NR) + 4E + 256 NR (argmax), bwd U(NR + E) + 256 NR."""
    import numpy as np
    import torch
    import sfgen
    from paper_2102_13018_gb300 import StarForest
    from paper_2102_13018_gb300 import autograd as sfa
    f = sfgen.cfg5_powerlaw()
    sf = StarForest.from_forest(f).setup().set_mode("deterministic")
    per = int(f.nroots[0])
    idx = torch.from_numpy(np.concatenate([f.iremote_rank[q].astype(np.int64) * per + f.iremote_index[q]
                                           for q in range(f.nranks)])).cuda()
    info = sf.info()
    E, C, NR, bs = info["nedges"], info["connected_roots"], sf.nroots_total, 64
    out = {}
    for name, dt in (("fp32", torch.float32), ("bf16", torch.bfloat16)):
        U = bs * torch.tensor([], dtype=dt).element_size()
        x = torch.rand(NR, bs, device="cuda").to(dt).requires_grad_(True)
        y = torch.rand(sf.leaf_extent, bs, device="cuda").to(dt).requires_grad_(True)
        gl = torch.rand(sf.leaf_extent, bs, device="cuda").to(dt)
        gr = torch.rand(NR, bs, device="cuda").to(dt)
        bytes_ = {"bcast": U * (C + E) + 4 * E + U * (E + NR) + 4 * E,
                  "reduce_sum": U * (E + NR) + 4 * E + U * (C + E) + 4 * E,
                  "reduce_max": U * (E + NR) + 4 * E + 4 * bs * NR + U * (NR + E) + 4 * bs * NR}

        def run(fn, t):
            t.grad = None
            fn()

        cases = {
            "bcast": (lambda: run(lambda: sfa.bcast(sf, x).backward(gl), x),
                      lambda: run(lambda: torch.index_select(x, 0, idx).backward(gl), x)),
            "reduce_sum": (lambda: run(lambda: sfa.reduce(sf, y, "SUM").backward(gr), y),
                           lambda: run(lambda: torch.zeros(NR, bs, device="cuda", dtype=dt)
                                       .index_add(0, idx, y).backward(gr), y)),
            "reduce_max": (lambda: run(lambda: sfa.reduce(sf, y, "MAX").backward(gr), y),
                           lambda: run(lambda: torch.zeros(NR, bs, device="cuda", dtype=dt).scatter_reduce(
                               0, idx[:, None].expand(-1, bs), y, "amax", include_self=False).backward(gr), y)),
        }
        res = {}
        for label, (ours, plain) in cases.items():
            r = {}
            for who, fn in (("sf_autograd", ours), ("torch", plain)):
                ms = time_op(fn, torch.cuda.current_stream(), flush, reps=10, warm=3)
                gbs = bytes_[label] / (ms * 1e-3) / 1e9
                r[who] = {"ms": ms, "gbs": gbs, "frac": gbs / peak}
            r["bytes"] = bytes_[label]
            res[label] = r
        out[name] = res
    return {"workload": "power-law message passing: 2^20 roots, 2^23 leaves (Chung-Lu, exponent 2.2), "
                        "bs=64; forward + backward of Bcast, Reduce SUM and Reduce MAX", **out}


def run_e2e(sf, x_h, y_h, lvec, stream, step_bytes, world, Ke):
    """End to end with x and y in pinned host memory, two ways, each step copying its x and y in
    (H2D) and its result y out (D2H) inside the timed region:
      pipelined (the reported value): independent steps y_k = y + Reduce(Bcast x) through
        sf.bcast / sf.reduce on device buffers, double-buffered over four streams (x in, y in,
        kernels, y out), so step k's D2H, step k+1's kernels and step k+2's H2D overlap;
      serial: sf_*_with_memtype on the host buffers, the host waiting for y after every step."""
    import torch
    nr = sf.nroots_total
    xh = torch.from_numpy(x_h).pin_memory()
    yh = torch.from_numpy(y_h).pin_memory()
    yo = [torch.empty_like(yh).pin_memory() for _ in range(2)]
    h2d, d2h = 8 * nr + 8 * nr, 8 * nr
    # serial, through the memtype calls
    for _ in range(2):
        sf.bcast_memtype(xh, lvec, "REPLACE", stream=stream)
        sf.reduce_memtype(lvec, yh, "SUM", stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(Ke):
        sf.bcast_memtype(xh, lvec, "REPLACE", stream=stream)
        sf.reduce_memtype(lvec, yh, "SUM", stream=stream)
        stream.synchronize()
    e1.record(stream)
    torch.cuda.synchronize()
    serial_ms = e0.elapsed_time(e1) / Ke
    # pipelined (x and y copied in on two streams, each on its own copy engine)
    s_in, s_in2, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    xd = [torch.empty(nr, dtype=torch.float64, device="cuda") for _ in range(2)]
    yd = [torch.empty(nr, dtype=torch.float64, device="cuda") for _ in range(2)]
    lv = [lvec, torch.empty_like(lvec)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_in2 = [torch.cuda.Event() for _ in range(2)]
    ev_c = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def steps(n, t0=None):
        for k in range(n):
            b = k & 1
            if k >= 2:
                for si in (s_in, s_in2):
                    si.wait_event(ev_c[b])     # step k-2's kernels are done with xd[b], yd[b]
                    si.wait_event(ev_out[b])   # and its y has left yd[b]
            if k == 0 and t0 is not None:
                t0.record(s_in)
                s_in2.wait_event(t0)
            with torch.cuda.stream(s_in):
                xd[b].copy_(xh, non_blocking=True)
            with torch.cuda.stream(s_in2):
                yd[b].copy_(yh, non_blocking=True)
            ev_in[b].record(s_in)
            ev_in2[b].record(s_in2)
            stream.wait_event(ev_in[b])
            stream.wait_event(ev_in2[b])
            if k >= 2:
                stream.wait_event(ev_out[b])
            sf.bcast(xd[b], lv[b], "REPLACE", stream=stream)
            sf.reduce(lv[b], yd[b], "SUM", stream=stream)
            ev_c[b].record(stream)
            s_out.wait_event(ev_c[b])
            if k >= 2:
                s_out.wait_event(ev_out[b])
            with torch.cuda.stream(s_out):
                yo[b].copy_(yd[b], non_blocking=True)
            ev_out[b].record(s_out)

    steps(3)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps(Ke, p0)
    p1.record(s_out)
    torch.cuda.synchronize()
    pipe_ms = p0.elapsed_time(p1) / Ke
    # the last step's result against the same step run serially on the device
    ref = yh.cuda()
    sf.bcast(xh.cuda(), lvec, "REPLACE", stream=stream)
    sf.reduce(lvec, ref, "SUM", stream=stream)
    torch.cuda.synchronize()
    same = bool(torch.equal(ref.cpu(), yo[(Ke - 1) & 1]))
    return {"value": world * step_bytes / (pipe_ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": pipe_ms,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": Ke, "result_bit_identical": same,
            "what": "pinned host x, y in and y out every step; steps pipelined over four streams "
                    "(x and y H2D, kernels, D2H overlap); sf.bcast + sf.reduce on device buffers",
            "serial_memtype": {"ms_per_step": serial_ms,
                               "value": world * step_bytes / (serial_ms * 1e-3) / 1e9,
                               "what": "sf_*_with_memtype on the host buffers, host waits for y every step"}}


def run_halo(flush, peak):
    """3-D halo exchange, 256^3 fp64 grid in 4x4x4 ranks, 27-point ghosts (about 1.2M ghost
    leaves): Bcast REPLACE (ghost update) and Reduce SUM (ghost accumulate) at bs = 1 and 5.
    Each call is timed alone with CUDA events after an L2 flush; bytes are algorithmic (roots
    read once, leaves written / read once, roots read and written for Reduce)."""
    import torch
    import sfgen
    from paper_2102_13018_gb300 import StarForest
    f = sfgen.cfg2_halo()
    sf = StarForest.from_forest(f).setup()
    info = sf.info()
    out = {"workload": "halo_27pt: 256^3 fp64 grid, 4x4x4 simulated ranks, width-1 ghost layers",
           "ghost_leaves": info["nedges"], "pattern_edges": info["edges_both_pattern"],
           "ts_tile_edges": info["ts_tile_edges"], "rm_tile_edges": info["rm_tile_edges"]}
    for bs in (1, 5):
        x = torch.rand(sf.nroots_total * bs, dtype=torch.float64, device="cuda")
        lv = torch.zeros(sf.leaf_extent * bs, dtype=torch.float64, device="cuda")
        ub = 8 * bs
        for label, mode, nbytes in (
                ("bcast_replace", None, ub * info["connected_roots"] + ub * info["nedges"]),
                ("reduce_sum_atomic", "atomic", ub * info["nedges"] + 2 * ub * info["connected_roots"]),
                ("reduce_sum_deterministic", "deterministic", ub * info["nedges"] + 2 * ub * info["connected_roots"])):
            if mode:
                sf.set_mode(mode)
                fn = lambda: sf.reduce(lv, x, "SUM", bs=bs)    # noqa: E731
            else:
                fn = lambda: sf.bcast(x, lv, "REPLACE", bs=bs)  # noqa: E731
            ev = []
            for i in range(33):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                if i >= 3:
                    ev.append((e0, e1))
            torch.cuda.synchronize()
            us = statistics.median(a.elapsed_time(b) for a, b in ev) * 1e3
            gbs = nbytes / (us * 1e-6) / 1e9
            out[f"{label}_bs{bs}"] = {"us": us, "gbs": gbs, "frac": gbs / peak}
    return out


def run_fp32_step(sf, info, x, y, stream, flush, peak, steps):
    """The benchmark step in fp32 on the same forest (bs = 1, 4-byte units): Bcast REPLACE then
    the deterministic Reduce SUM, each op timed with CUDA events, L2 flushed between steps."""
    import torch
    x32, y32 = x.float(), y.float()
    l32 = torch.zeros(sf.leaf_extent, dtype=torch.float32, device="cuda")
    for _ in range(3):
        flush.zero_()
        sf.bcast(x32, l32, "REPLACE", stream=stream)
        sf.reduce(l32, y32, "SUM", stream=stream)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        sf.bcast(x32, l32, "REPLACE", stream=stream)
        ev[i][1].record(stream)
        sf.reduce(l32, y32, "SUM", stream=stream)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    b = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    r = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    bb, rb = algorithmic_bytes(info, 4)
    return {"dtype": "f32", "steps": steps, "ms_per_step": b + r, "gbs": (bb + rb) / ((b + r) * 1e-3) / 1e9,
            "frac": (bb + rb) / ((b + r) * 1e-3) / 1e9 / peak, "bcast_ms": b, "reduce_ms": r,
            "bcast_frac": bb / (b * 1e-3) / 1e9 / peak, "reduce_frac": rb / (r * 1e-3) / 1e9 / peak}


def cpu_parallel_baseline(forest, x_h, y_h, step_bytes):
    """The step on all host cores (OpenMP, oracle/sf_cpu_parallel.c): a baseline, not a path of
    the library."""
    import numpy as np
    import oracle
    try:
        cp = oracle.CpuParallel(forest)
    except RuntimeError as e:
        return {"kind": "openmp", "unavailable": str(e)}
    lv = np.zeros(int(oracle.layout(forest)[1][-1]))
    y = y_h.copy()
    cp.bcast_replace(x_h, lv)
    cp.reduce_sum(lv, y)
    t0 = time.perf_counter()
    reps = 0
    while time.perf_counter() - t0 < 10.0 and reps < 50:
        cp.bcast_replace(x_h, lv)
        cp.reduce_sum(lv, y)
        reps += 1
    secs = (time.perf_counter() - t0) / reps
    return {"value": step_bytes / secs / 1e9, "unit": "GB/s", "cores": cp.threads, "kind": "openmp",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(), "ms_per_step": secs * 1e3,
            "sample": f"the full workload, {reps} steps of one Bcast REPLACE + one deterministic Reduce SUM"}


def sum_error_statement(sf, forest, stream):
    """Reduce SUM on the full workload against the oracle's fp64 reference (Neumaier-compensated
    r0 + sum of the leaves): the largest absolute and relative (to |r0| + sum |y|) error, and the
    largest error over the bound tol x in-degree x (|r0| + sum |y|), atomic and deterministic."""
    import numpy as np
    import torch
    import oracle
    import sfgen
    tol = {"fp32": 1e-6, "fp64": 1e-13}
    deg = np.maximum(oracle.in_degree(forest), 1).astype(np.float64)
    ro, lo = oracle.layout(forest)
    out = {}
    for dt in ("fp64", "fp32"):
        leaf = sfgen.data(dt, int(lo[-1]), 5, 1)
        root = sfgen.data(dt, int(ro[-1]), 5, 2)
        ref, absum = oracle.sum_reference(forest, dt, 1, leaf, root)
        lt = torch.from_numpy(leaf).cuda()
        for mode in ("atomic", "deterministic"):
            sf.set_mode(mode)
            r = torch.from_numpy(root).cuda()
            sf.reduce(lt, r, "SUM", stream=stream)
            err = np.abs(r.cpu().numpy().astype(np.float64) - ref)
            out[f"{dt}_{mode}"] = {"max_abs": float(err.max()),
                                   "max_rel": float((err / np.maximum(absum, 1e-300)).max()),
                                   "max_over_bound": float((err / (tol[dt] * deg * np.maximum(absum, 1e-300))).max()),
                                   "tol": tol[dt]}
    sf.set_mode("deterministic")
    return {"what": "Reduce SUM of uniform [-1,1) data, full workload, vs the oracle's fp64 compensated sum; "
                    "bound = tol x in-degree x (|r0| + sum |y|)", **out}


def max_over_ranks(local_ms: float, world: int, device: str = "cpu") -> float:
    """Slowest rank's timed total (every rank runs an independent replica)."""
    import torch
    if world <= 1:
        return float(local_ms)
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(bytes_per_step: int, steps: int, max_ms: float, world: int) -> float:
    """Whole-job GB/s: all replicas' algorithmic bytes over the slowest rank's time."""
    return world * bytes_per_step * steps / (max_ms * 1e-3) / 1e9


def host_info(forest):
    """Plan statistics from the library's host setup pass (no GPU needed)."""
    from paper_2102_13018_gb300 import StarForest
    return StarForest.from_forest(forest).analyze().info()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import sfgen
    from paper_2102_13018_gb300 import StarForest, launch_count

    if args.only != "all":
        # one extra section alone (for profiling it); prints its own JSON object
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        if args.only == "halo":
            res = run_halo(flush, measured_peak()[0])
        elif args.only == "batched":
            res = run_batched(args, torch.cuda.current_stream(), flush)
        else:
            res = run_autograd(flush, measured_peak()[0])
        if rank == 0:
            print(json.dumps({"section": args.only, **res}))
        return

    forest = build_forest(args)
    t0 = time.perf_counter()
    sf = StarForest.from_forest(forest).setup()
    setup_s = time.perf_counter() - t0
    sf.set_mode("deterministic").set_path("fused")
    info = sf.info()
    nr, nl = sf.nroots_total, sf.leaf_extent
    x_h = sfgen.data("fp64", nr, 3, 1)
    y_h = sfgen.data("fp64", nr, 3, 2)
    x = torch.from_numpy(x_h).cuda()
    y = torch.from_numpy(y_h).cuda()
    lvec = torch.zeros(nl, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        sf.bcast(x, lvec, "REPLACE", stream=stream)
        sf.reduce(lvec, y, "SUM", stream=stream)

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    clocks = ClockSampler()
    clocks.start()
    time.sleep(0.2)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = launch_count()
    wall0 = time.perf_counter()
    for i in range(K):
        flush.zero_()
        e = ev[i]
        e[0].record(stream)
        sf.bcast_begin(x, lvec, "REPLACE", stream=stream)
        sf.bcast_end(x, lvec, "REPLACE", stream=stream)
        e[1].record(stream)
        sf.reduce_begin(lvec, y, "SUM", stream=stream)
        sf.reduce_end(lvec, y, "SUM", stream=stream)
        e[2].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    launches = launch_count() - n0
    clk = clocks.stop()
    bcast_ms = [ev[i][0].elapsed_time(ev[i][1]) for i in range(K)]
    reduce_ms = [ev[i][1].elapsed_time(ev[i][2]) for i in range(K)]
    total_ms = sum(bcast_ms) + sum(reduce_ms)
    max_ms = max_over_ranks(total_ms, world, "cuda")
    bb, rb = algorithmic_bytes(info)
    value = job_value(bb + rb, K, max_ms, world)
    peak, peak_src = measured_peak()
    b_avg, r_avg = statistics.mean(bcast_ms), statistics.mean(reduce_ms)
    # the deterministic Reduce is one launch of its plan's kernel (a diagonal plan that leaves
    # roots out adds a root-major launch for them)
    plan = sf.tuning()["reduce_plan"]
    rk = {"root_major": "rm_kernel", "diagonal": "dg_kernel", "diagonal_staged": "dg_bulk_kernel"}[plan]
    dom = (rk, rb, r_avg) if r_avg >= b_avg else ("ts_kernel", bb, b_avg)
    achieved = dom[1] / (dom[2] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom[0] + (" (Reduce SUM, deterministic)" if dom[0] != "ts_kernel"
                                                    else " (Bcast REPLACE, fused)"),
                "achieved": achieved, "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                "frac": achieved / peak, "traffic": committed_traffic(dom[0]),
                "algorithmic_bytes_per_launch": dom[1]}
    ops = {"bcast_ms": b_avg, "reduce_ms": r_avg, "bcast_gbs": bb / (b_avg * 1e-3) / 1e9,
           "reduce_gbs": rb / (r_avg * 1e-3) / 1e9, "bcast_frac": bb / (b_avg * 1e-3) / 1e9 / peak,
           "reduce_frac": rb / (r_avg * 1e-3) / 1e9 / peak, "bcast_bytes": bb, "reduce_bytes": rb,
           "setup_s": setup_s, "host_wall_s": wall}

    # the other data paths on the same forest, timed the same way (not part of the step)
    variants = {}
    if not args.no_variants:
        for path in ("fused", "three_phase", "root_major"):
            sf.set_path(path)
            ms = time_op(lambda: sf.bcast(x, lvec, "REPLACE", stream=stream), stream, flush)
            variants[f"bcast_{path}"] = {"ms": ms, "gbs": bb / (ms * 1e-3) / 1e9}
        sf.set_path("fused")
        for mode in ("deterministic", "atomic"):
            sf.set_mode(mode)
            ms = time_op(lambda: sf.reduce(lvec, y, "SUM", stream=stream), stream, flush)
            variants[f"reduce_sum_{mode}"] = {"ms": ms, "gbs": rb / (ms * 1e-3) / 1e9}
        sf.set_mode("deterministic")
        if info["dg_chunks"] > 0:
            for p in ("diagonal", "diagonal_staged"):
                sf.set_reduce_plan(p)
                ms = time_op(lambda: sf.reduce(lvec, y, "SUM", stream=stream), stream, flush)
                variants[f"reduce_sum_deterministic_{p}"] = {"ms": ms, "gbs": rb / (ms * 1e-3) / 1e9}
            sf.set_reduce_plan("auto")
        ms = time_op(lambda: sf._lib.sf_reduce_noalloc(sf._h, sf._unit(y, sf.nroots_total, None),
                                                      sf._ptr(lvec), sf._ptr(y), 1, sf._stream(stream)), stream, flush)
        variants["reduce_sum_noalloc"] = {"ms": ms, "gbs": rb / (ms * 1e-3) / 1e9}
        # FetchAndOp SUM on the same forest: each root's leaves fetch its running sum
        fb = op_bytes(info, "fetch", "SUM", 8)
        upd = torch.zeros(nl, dtype=torch.float64, device="cuda")
        for mode in ("deterministic", "atomic"):
            sf.set_mode(mode)
            ms = time_op(lambda: sf.fetch_and_op(y, lvec, upd, "SUM", stream=stream), stream, flush)
            variants[f"fetch_and_op_sum_{mode}"] = {"ms": ms, "bytes": fb, "gbs": fb / (ms * 1e-3) / 1e9}
        sf.set_mode("deterministic")
        variants["fp32"] = run_fp32_step(sf, info, x, y, stream, flush, peak, max(3, min(K, 50)))

    # end to end through the public API with the data in pinned host memory: every step copies
    # its x and y in, runs Bcast + Reduce, and copies its y out
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(sf, x_h, y_h, lvec, stream, bb + rb, world, max(3, min(K, 50)))

    pingpong = None
    if not args.no_pingpong:
        pingpong = run_pingpong(stream)

    autograd = halo = tiny = None
    if not args.no_extras:
        autograd = run_autograd(flush, peak)
        halo = run_halo(flush, peak)
        tiny = run_tiny(stream)

    batched = None
    if not args.no_batched:
        batched = run_batched(args, stream, flush)

    cpu = cpu_all = sum_error = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        lv0 = np.zeros(nl)
        secs = oracle_step_time(forest, x_h, lv0, y_h, reps=1)
        reps = max(1, min(10, int(20.0 / max(secs, 1e-3))))
        secs = oracle_step_time(forest, x_h, lv0, y_h, reps=reps) if reps > 1 else secs
        cpu = {"value": (bb + rb) / secs / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "cpu_model": cpu_model(), "nproc": os.cpu_count(),
               "sample": f"the full workload, {reps} step(s) of one Bcast REPLACE + one Reduce SUM"}
        cpu_all = cpu_parallel_baseline(forest, x_h, y_h, bb + rb)
        sum_error = sum_error_statement(sf, forest, stream)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": max_ms / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args, forest),
                "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
                "sum_error_vs_fp64_reference": sum_error, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "ops": ops, "variants": variants, "batched": batched,
                "pingpong": pingpong, "autograd": autograd, "halo": halo, "plain_tiny": tiny,
                "plan": {k: info[k] for k in ("nedges", "connected_roots", "multi_roots", "multi_edges",
                                              "edges_both_pattern", "edges_one_indexed", "edges_two_indexed",
                                              "rm_masked_edges", "rm_pairs", "rm_chunks", "dg_chunks", "dg_roots",
                                              "dg_extra_leaves", "dg_list_roots", "dg_rest_roots",
                                              "device_plan_bytes")}}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
