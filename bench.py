#!/usr/bin/env python3
"""Benchmark of the stabilizer-frame hot path on the QFT workload.

One step = one QFT on n = 20 qubits from a seeded random computational basis
state (controlled-R_k applied as branches of the frame, a coalesce after each),
then the measurement probabilities of qubit 0 (with its cofactoring) and one
basis amplitude: every row of the hot path (Clifford update, branching,
coalescing, measurement, amplitude) runs in every step.

Metric: frame-element updates per second (one gate applied to one input
element; measurement and the amplitude query count one update per element),
whole job.  `value` replays the step from device-resident gate lists through a
captured CUDA graph (measurement and amplitude outside the graph, they read
results back); `e2e` runs the same step through the public C ABI with host
gate arrays, host->device copies and result reads inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Two more measurements ride on the same JSON line (rank 0): "batched", the
Steane fault-injection campaign (4096 variants in one persistent launch, shape
picked by the library's autotuner) against the one-circuit path, and
"served", a seeded Poisson stream of random Clifford+T circuits through the
continuous-batching server against the same stream one at a time, with
p50/p99 latency.  "multiframe": the Cuccaro adder on the equal superposition
(Toffolis by cofactors) as one frame and as a multiframe (Sec. IV), with the
largest amplitude difference between the two on sampled basis states.

Multi-GPU: one process per GPU (torchrun), each rank simulates its own QFT
instance (different seed); no data-path collective ("weak" scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1712_03554_gb300 import circuits as c  # noqa: E402

N_QUBITS = 20
MAX_ELEMS = 1 << 21
DROP_EPS = 1e-12
METRIC = "frame-elem updates/s"
UNIT = "updates/s"
WORKLOAD = ("QFT n=20 on a seeded random basis state (controlled-R_k as frame branches, "
            "coalesce after each) + measure qubit 0 + one amplitude")


# ---------------------------------------------------------------------------
def build_plan(n: int, seed: int):
    """The step as a list of ops with consecutive Clifford gates grouped."""
    x, ops = c.qft_random_input(n, seed)
    plan, pending = [], []
    i = 0
    while i < len(ops):
        op = ops[i]
        i += 1
        if op[0] == "C":
            pending.append((op[1], op[2], op[3]))
            continue
        if pending:
            plan.append(("C", list(pending)))
            pending = []
        if op[0] == "N" and i < len(ops) and ops[i][0] == "K":
            plan.append(("NK",) + tuple(op[1:]))  # branch + merge in one call
            i += 1
        else:
            plan.append(op)
    if pending:
        plan.append(("C", list(pending)))
    y = int(c.rng_for(seed + 101).integers(0, 1 << n))
    return x, plan, y


def bytes_model(W: int, n: int = N_QUBITS):
    """Algorithmic bytes of each kernel class as a function of the element counts
    it sees (kin elements read, kout elements written).  The merge table of
    insert/compact is scratch and not counted; single-CTA tableau kernels move
    the tableau (4 n x W words in and out)."""
    e = 8 * W + 16  # one element: phase vector + FP64 complex amplitude
    tab = 2 * 4 * n * W * 8
    return {
        "clifford": lambda kin, kout: tab + n * W * 8,
        "measure_prep": lambda kin, kout: tab,
        "amp_prep": lambda kin, kout: tab // 2,
        "affine": lambda kin, kout: 2 * 8 * W * kin,
        "branch": lambda kin, kout: e * kin + e * kout,
        "branch_merge": lambda kin, kout: e * kin + e * kout,
        "cofactor": lambda kin, kout: e * kin + e * kout,
        "index": lambda kin, kout: 8 * W * kin,
        "insert": lambda kin, kout: e * kin,
        "compact": lambda kin, kout: e * kout,
        "filter": lambda kin, kout: e * kin + e * kout,
        "prob": lambda kin, kout: 24 * kin,
        "amplitude": lambda kin, kout: e * kin,
        "reduce": lambda kin, kout: 0,
        "segment": lambda kin, kout: kin,  # recorded as the summed bytes of the ops it runs
        "gprog": lambda kin, kout: kin,    # the same for the grid program
    }


def plan_records(sfm, plan):
    """sf_op records of a plan made of Clifford batches and merged diagonal gates
    (one record per gate), and the record index at which each plan entry starts."""
    recs, starts = [], []
    for op in plan:
        starts.append(len(recs))
        if op[0] == "C":
            recs += [(g[0], g[1], g[2], 0, 0.0) for g in op[1]]
        elif op[0] == "NK":
            recs.append((sfm.OP_DIAG + op[1], op[2], op[3], 0, float(op[4])))
        else:
            break
    starts.append(len(recs))
    return np.array(recs, dtype=sfm.SF_OP_DTYPE), starts


def choose_program_prefix(sfm, torch, n, plan, y, stream, candidates=(256, 512, 1024, 2048, 4096), grid=True):
    """The single-CTA program (sf_apply_program) runs the first plan entries while
    the frame is small, the rest runs in the grid program (sf_apply_program_grid;
    with grid=False, per op); pick the single-CTA frame limit by timing the eager
    step for each candidate (and without it).  Returns (max_frame, plan entries,
    records, the device records of the whole plan, their number)."""
    recs, starts = plan_records(sfm, plan)
    d_all = torch.from_numpy(recs.view(np.uint8).copy()).cuda()
    consumed = torch.zeros(1, dtype=torch.int64, device="cuda")
    fr = sfm.Frame(n, MAX_ELEMS, stream=stream)

    def run(mf, p, m):
        with torch.cuda.stream(stream):
            fr.reset()
            if m:
                fr.apply_program_device(d_all.data_ptr(), m, DROP_EPS, 0, 0, mf)
            if grid:
                if len(recs) > m:
                    fr.apply_program_grid_device(d_all.data_ptr() + recs.itemsize * m, len(recs) - m, DROP_EPS)
            else:
                for op in plan[p:]:
                    if op[0] == "C":
                        fr.apply_clifford(op[1])
                    elif op[0] == "NK":
                        fr.apply_nonclifford_coalesce(op[1], op[2], op[3], op[4], DROP_EPS)
        fr.measure(0, -1)
        fr.amplitude(y)

    best = None
    for mf in (0,) + tuple(candidates):
        p = m = 0
        if mf:
            with torch.cuda.stream(stream):
                fr.reset()
                fr.apply_program_device(d_all.data_ptr(), len(recs), DROP_EPS, consumed.data_ptr(), 0, mf)
            fr.sync()
            m = int(consumed.item())
            p = max(i for i in range(len(starts)) if starts[i] <= m)
            m = starts[p]
        run(mf, p, m)
        ts = []
        for _ in range(7):
            t0 = time.perf_counter()
            run(mf, p, m)
            ts.append(time.perf_counter() - t0)
        t = statistics.median(ts)
        if best is None or t < best[0]:
            best = (t, mf, p, m)
    fr.close()
    _, mf, p, m = best
    return mf, p, m, d_all, len(recs)


def instrumented_pass(sfm, n, plan, y):
    """Run the step once eagerly with a sync after every op to record the
    element counts each kernel class sees (the circuit is deterministic)."""
    f = sfm.Frame(n, MAX_ELEMS)
    W = 1 << max(0, math.ceil(math.log2(max(1, (n + 63) // 64))))
    rec = {k: [] for k in bytes_model(W, n)}
    updates = 0
    coal_elems = 0
    k = 1
    peak = 1
    indexed = True  # the index of the current frame is valid (see sf_api.cu)
    ops_rec = []  # (plan index, class, kin, kout) of every launch of the captured part
    for pi, op in enumerate(plan):
        if op[0] == "C":
            f.apply_clifford(op[1])
            updates += len(op[1]) * k
            rec["affine"].append((k, k))
            rec["clifford"].append((k, k))
            ops_rec += [(pi, "affine", k, k), (pi, "clifford", k, k)]
            indexed = False
        elif op[0] == "NK":
            f.apply_nonclifford_coalesce(op[1], op[2], op[3], op[4], DROP_EPS)
            kout = f.size()
            updates += k
            coal_elems += k
            if not indexed:
                rec["index"].append((k, k))
                ops_rec.append((pi, "index", k, k))
            rec["branch_merge"].append((k, kout))
            ops_rec.append((pi, "branch_merge", k, kout))
            indexed = True
            k = kout
        elif op[0] == "N":
            f.apply_nonclifford(op[1], op[2], op[3], op[4])
            kout = f.size()
            updates += k
            rec["branch"].append((k, kout))
            k = kout
            indexed = False
        elif op[0] == "K":
            kin = k
            k = f.coalesce(DROP_EPS, sync=True)
            coal_elems += kin
            rec["insert"].append((kin, k))
            rec["compact"].append((kin, k))
            indexed = True
        peak = max(peak, k)
    # the captured (graph) part ends here; the tail is measured eagerly
    graph_rec = {cls: list(v) for cls, v in rec.items()}
    k_before = [1]  # frame size before each plan entry
    kk = 1
    for pi, op in enumerate(plan):
        k_before.append(kk)
        for (pj, cls, a, b) in ops_rec:
            if pj == pi and cls == "branch_merge":
                kk = b
    k_before = k_before[1:]
    # measurement of qubit 0 (cofactor + coalesce + probabilities)
    kin = k
    f.measure(0, -1)
    km = f.size()
    updates += kin
    if not indexed:
        rec["index"].append((kin, kin))
    rec["cofactor"].append((kin, km))
    coal_elems += 2 * kin
    rec["prob"].append((km, km))
    f.amplitude(y)
    updates += km
    rec["amplitude"].append((km, km))
    peak = max(peak, 2 * kin)
    f.close()
    return updates, coal_elems, rec, graph_rec, peak, W, ops_rec, k_before


def measured_peak_gbs():
    for path in (os.path.join(ROOT, "MEASURED_PEAKS.json"),):
        try:
            with open(path) as fh:
                return float(json.load(fh)["hbm_gbs"]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


# the file that defines each timed kernel class; its hash (with every header it
# includes) decides whether an ncu traffic figure still describes the kernel
KERNEL_SOURCE = {"segment": "sf_campaign.cu", "gprog": "sf_gprog.cu", "clifford": "sf_tableau_warp.cu",
                 "measure_prep": "sf_tableau_warp.cu", "reset": "sf_tableau.cu", "amp_prep": "sf_tableau.cu"}


def kernel_sources_hash(cls: str) -> str:
    """sha256 (16 hex digits) of the source file defining kernel class `cls`
    and of the headers it includes, transitively (csrc/ and include/)."""
    import re
    dirs = [os.path.join(ROOT, "paper_1712_03554_gb300", "csrc"), os.path.join(ROOT, "include")]
    todo, seen = [KERNEL_SOURCE.get(cls, "sf_frame.cu")], []
    while todo:
        fn = todo.pop(0)
        if fn in seen:
            continue
        for d in dirs:
            path = os.path.join(d, fn)
            if os.path.exists(path):
                seen.append(fn)
                with open(path, encoding="utf-8") as fh:
                    todo += re.findall(r'^#include "([^"]+)"', fh.read(), re.M)
                break
    h = hashlib.sha256()
    for fn in sorted(seen):
        for d in dirs:
            path = os.path.join(d, fn)
            if os.path.exists(path):
                with open(path, "rb") as fh:
                    h.update(fn.encode() + b"\0" + fh.read())
                break
    return h.hexdigest()[:16]


def ncu_traffic(cls: str):
    """DRAM bytes per launch of `cls` from the committed ncu summary, or None if
    absent or taken on different sources of that kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
        if t.get("sources", {}).get(cls) != kernel_sources_hash(cls):
            return None
        v = t.get("bytes_per_launch", {}).get(cls)
        return float(v) if v is not None else None
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as fh:
                for ln in fh:
                    p = [v.strip() for v in ln.split(",")]
                    if len(p) >= 9 and p[1].replace(".", "").isdigit():
                        rows.append(p)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# ---------------------------------------------------------------------------
def oracle_step(n, plan, y):
    import oracle
    f = oracle.FrameOracle(n)
    for op in plan:
        if op[0] == "C":
            f.apply_clifford(op[1])
        elif op[0] in ("N", "NK"):
            f.apply_nonclifford(op[1], op[2], op[3], op[4])
            if op[0] == "NK":
                f.coalesce(DROP_EPS)
        elif op[0] == "K":
            f.coalesce(DROP_EPS)
    f.measure(0, -1)
    return f.amplitude(y)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or "unknown"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _time_oracle(n, plan, y, threads, budget_s, max_reps):
    import oracle
    prev = oracle.set_threads(threads)
    try:
        times = []
        t_all = time.perf_counter()
        while len(times) < max_reps and (time.perf_counter() - t_all) < budget_s:
            t0 = time.perf_counter()
            oracle_step(n, plan, y)
            times.append(time.perf_counter() - t0)
        return statistics.median(times), len(times)
    finally:
        oracle.set_threads(prev)


def cpu_baseline(n, plan, y, updates, budget_s=12.0, max_reps=4):
    """The C oracle on full steps of the same workload, on this host's cores:
    its per-element loops split into one range per core (Sec. V), and
    sequentially on one core."""
    cores = host_cores()
    per_mt, reps_mt = _time_oracle(n, plan, y, cores, budget_s, max_reps)
    per_1, reps_1 = _time_oracle(n, plan, y, 1, budget_s, max_reps)
    return {"value": updates / per_mt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps_mt} full steps of the same workload, median {per_mt:.3f} s/step, on the C oracle "
                      f"with its per-element loops split into {cores} ranges on {cores} threads "
                      f"(the paper's Sec. V element-range parallelisation; sort and elimination stay sequential)",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "single_thread": {"value": updates / per_1, "unit": UNIT, "cores": 1,
                              "sample": f"{reps_1} full steps, median {per_1:.3f} s/step, sequential"}}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    x, plan, y = build_plan(N_QUBITS, args.seed)
    # updates of the workload, counted from the oracle's own frame sizes
    import oracle
    f = oracle.FrameOracle(N_QUBITS)
    updates, k = 0, 1
    for op in plan:
        if op[0] == "C":
            f.apply_clifford(op[1])
            updates += len(op[1]) * k
        elif op[0] in ("N", "NK"):
            f.apply_nonclifford(op[1], op[2], op[3], op[4])
            updates += k
            k = f.size()
            if op[0] == "NK":
                k = f.coalesce(DROP_EPS)
        elif op[0] == "K":
            k = f.coalesce(DROP_EPS)
    updates += f.size()
    f.measure(0, -1)
    updates += f.size()
    del f
    cores = host_cores()
    oracle.set_threads(cores)  # Sec. V: one element range per host core
    for _ in range(args.warmup):
        oracle_step(N_QUBITS, plan, y)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(N_QUBITS, plan, y)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    val = updates / dt
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n_qubits": N_QUBITS, "seed": args.seed},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"each step is the full workload on the C oracle, its per-element loops "
                                      f"split into {cores} ranges on {cores} threads (Sec. V)",
                            "cpu_model": cpu_model(), "nproc": os.cpu_count()},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Batched campaign: the Steane [[7,1,3]] fault-injection workload, every
# variant in one persistent launch, against the one-circuit library path.
CAMPAIGN_WORKLOAD = ("Steane [[7,1,3]] encode + 3 flagged syndrome rounds + logical T by magic-state "
                     "injection on 49 qubits; per variant 1-3 Pauli errors, 0-12 coherent T/T-dagger "
                     "faults, 200-2000 ops, seeded draws for 42 measurements")


def campaign_leg(sfm, torch, n_variants: int, plain_sample: int = 16):
    t0 = time.perf_counter()
    circuits = c.steane_campaign(n_variants, seed=0)
    recs, offs = sfm.encode_program(circuits)
    prep_s = time.perf_counter() - t0
    eng = sfm.Campaign(c.STEANE_N, 4096)
    nc = len(circuits)
    ops = torch.from_numpy(recs.view(np.uint8).copy()).cuda()
    off = torch.from_numpy(offs.view(np.int64).copy()).cuda()
    out = eng.outputs(nc)
    eng.autotune(ops, off, nc, reps=2)
    threads, smem_index, ctas = eng.shape()
    eng.launch(ops, off, nc, DROP_EPS, out)
    torch.cuda.synchronize()
    ms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        eng.launch(ops, off, nc, DROP_EPS, out)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    status = out["status"].cpu().numpy()
    # both coalescing strategies in the chosen shape (the autotuner searched them all)
    sorted_chosen = eng.coalesce_sorted()
    strat_ms = {}
    for srt in (False, True):
        eng.set_coalesce(srt)
        eng.launch(ops, off, nc, DROP_EPS, out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        eng.launch(ops, off, nc, DROP_EPS, out)
        e1.record()
        torch.cuda.synchronize()
        strat_ms["sort" if srt else "hash"] = e0.elapsed_time(e1)
    eng.set_coalesce(sorted_chosen)
    # end to end: program from pinned host memory, results back to the host
    h_ops = torch.from_numpy(recs.view(np.uint8).copy()).pin_memory()
    h_off = torch.from_numpy(offs.view(np.int64).copy()).pin_memory()
    h_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
    e2e = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ops.copy_(h_ops, non_blocking=True)
        off.copy_(h_off, non_blocking=True)
        eng.launch(ops, off, nc, DROP_EPS, out)
        for k in out:
            h_out[k].copy_(out[k], non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        e2e.append(e0.elapsed_time(e1))
    eng.close()
    # the plain path: one circuit at a time through the one-circuit library calls
    t0 = time.perf_counter()
    for ops_v in circuits[:plain_sample]:
        f = sfm.Frame(c.STEANE_N, 4096)
        c.run(f, ops_v)
        f.sync()
        f.close()
    plain_s = time.perf_counter() - t0
    med = statistics.median(ms)
    return {"workload": CAMPAIGN_WORKLOAD, "circuits": nc, "ops": int(len(recs)),
            "circuits_per_s": nc / (med * 1e-3), "ops_per_s": len(recs) / (med * 1e-3), "ms": med,
            "e2e_circuits_per_s": nc / (statistics.median(e2e) * 1e-3),
            "e2e_h2d_bytes": int(recs.nbytes + offs.nbytes),
            "shape": {"threads_per_circuit": threads, "index_in_shared_memory": smem_index, "ctas": ctas,
                      "coalescing": "sort" if sorted_chosen else "hash", "chosen_by": "sf_campaign_autotune",
                      "ms_by_coalescing_in_this_shape": strat_ms},
            "plain_circuits_per_s": plain_sample / plain_s,
            "plain_sample": f"first {plain_sample} variants, one at a time through sf_create/sf_apply_*/sf_measure",
            "speedup_vs_plain": (nc / (med * 1e-3)) / (plain_sample / plain_s),
            "circuits_failed": int((status != 0).sum()), "host_prep_s": prep_s}


# Serving: a seeded Poisson stream of random Clifford+T circuits admitted by
# HBM footprint (continuous batching) against the same stream one at a time.
SERVING_WORKLOAD = ("Poisson stream of random Clifford+T circuits, n uniform in {16,64,256,1024}, "
                    "1e3-1e5 Clifford gates (log-uniform), 0-20 T gates, frames up to 2^20 elements, "
                    "then 8 measurements with seeded draws; amplitudes of 4 basis states returned")


def _run_stream(sfm, stream, recs, slots, budget):
    """Submit the requests at their arrival times; circuits/s over the span from
    the first submission to the last completion, latency = completion -
    submission."""
    srv = sfm.Server(budget, slots)
    t0 = srv.clock()
    ids = []
    for r, rc in zip(stream, recs):
        while srv.clock() - t0 < r["arrival"]:
            time.sleep(0.0002)
        ids.append(srv.submit(r["n"], rc, r["max_elems"], r["probes"]))
    srv.wait(900.0)
    res = {x["id"]: x for x in srv.poll()}
    srv.close()
    out = [res[i] for i in ids]
    lat = np.array([x["t_done"] - x["t_submit"] for x in out])
    span = max(x["t_done"] for x in out) - min(x["t_submit"] for x in out)
    return out, {"circuits_per_s": len(out) / span, "p50_latency_s": float(np.percentile(lat, 50)),
                 "p99_latency_s": float(np.percentile(lat, 99)), "span_s": span,
                 "failed": int(sum(x["status"] != 0 for x in out))}


def serving_leg(sfm, n_requests: int, slots: int, budget_gb: int = 96, fractions=(0.5, 0.8, 1.2),
                cap_sample: int = 12):
    """The capacities of the plain path (cap_sample requests queued at once,
    one at a time) and of the server (the same burst over `slots` slots), then
    the same seeded stream at arrival rates fraction x plain capacity, served
    and one at a time."""
    budget = budget_gb << 30
    burst = c.serving_stream(cap_sample, 1e9, seed=1)  # every request arrives at once
    burst_recs = [sfm.encode_program([r["ops"]])[0] for r in burst]
    _, cap_stats = _run_stream(sfm, burst, burst_recs, 1, budget)
    _, scap_stats = _run_stream(sfm, burst, burst_recs, slots, budget)
    capacity = cap_stats["circuits_per_s"]
    sweep = []
    all_same, max_diff = True, 0.0
    gates = 0
    for fr in fractions:
        lam = fr * capacity
        stream = c.serving_stream(n_requests, lam, seed=0)
        recs = [sfm.encode_program([r["ops"]])[0] for r in stream]
        gates = sum(len(r) for r in recs)
        served, s_stats = _run_stream(sfm, stream, recs, slots, budget)
        alone, p_stats = _run_stream(sfm, stream, recs, 1, budget)
        # element order inside a frame follows CTA scheduling, so amplitude sums
        # may differ in the last bits between runs: compare within 1e-10
        diff = max((abs(x - y) for a, b in zip(served, alone) for x, y in zip(a["amps"], b["amps"])), default=0.0)
        same = all(a["status"] == b["status"] and a["k_final"] == b["k_final"] and a["outcomes"] == b["outcomes"]
                   for a, b in zip(served, alone)) and diff <= 1e-10
        all_same &= same
        max_diff = max(max_diff, diff)
        sweep.append({"load_fraction_of_plain_capacity": fr, "arrival_rate_hz": lam, "served": s_stats,
                      "plain_one_at_a_time": p_stats,
                      "speedup_circuits_per_s": s_stats["circuits_per_s"] / p_stats["circuits_per_s"],
                      "p50_latency_ratio_plain_over_served": p_stats["p50_latency_s"] / max(1e-9, s_stats["p50_latency_s"]),
                      "p99_latency_ratio_plain_over_served": p_stats["p99_latency_s"] / max(1e-9, s_stats["p99_latency_s"]),
                      "results_same_alone_and_mixed": same})
    return {"workload": SERVING_WORKLOAD, "requests_per_load_point": n_requests, "gates_total_per_load_point": int(gates),
            "max_active": slots, "hbm_budget_gb": budget_gb,
            "plain_capacity": {"circuits_per_s": capacity, "sample": f"{cap_sample} requests queued at once, "
                                                                    f"one at a time", "stats": cap_stats},
            "served_capacity": {"circuits_per_s": scap_stats["circuits_per_s"],
                                "sample": f"the same {cap_sample} requests queued at once, over {slots} slots",
                                "stats": scap_stats,
                                "over_plain_capacity": scap_stats["circuits_per_s"] / capacity},
            "sweep": sweep, "results_same_alone_and_mixed": all_same, "max_amp_diff_alone_vs_mixed": max_diff,
            "note": ("the stated stream has 2000 requests; this run takes the largest count that keeps the bench "
                     "within a few minutes (--serving-requests sets it)")}


# Multiframes (Sec. IV): the same adder state as one frame and as a list of
# frames built by COALESCE and the merge of equal matrices.
def multiframe_leg(sfm, nb: int = 6, reps: int = 3):
    try:
        ops = c.cuccaro(nb, True, toffoli="cofactor", coalesce=False)
        n = 2 * nb + 2
        f = sfm.Frame(n, 1 << min(2 * nb + 2, 24))
        ts = []
        for _ in range(reps + 1):
            f.reset()
            f.sync()
            t0 = time.perf_counter()
            c.run(f, ops)
            f.sync()
            ts.append(time.perf_counter() - t0)
        frame_ms = statistics.median(ts[1:]) * 1e3
        ts, mf = [], None
        for _ in range(reps + 1):
            if mf is not None:
                mf.close()
            mf = sfm.MultiFrame(n, 4096, 8192)
            mf.count()
            t0 = time.perf_counter()
            c.run(mf, ops)
            frames, states = mf.count()
            ts.append(time.perf_counter() - t0)
        mf_ms = statistics.median(ts[1:]) * 1e3
        ys = [int(y) for y in c.rng_for(7).integers(1 << n, size=8)]
        diff = max(abs(mf.amplitude(y) - f.amplitude(y)) for y in ys)
        out = {"workload": f"Cuccaro adder, {nb}-bit, equal superposition of both inputs, Toffolis by cofactors "
                           f"(Eq. 2), {n} qubits",
               "single_frame": {"states": f.size(), "ms": frame_ms},
               "multiframe": {"frames": frames, "states": states, "ms": mf_ms},
               "state_ratio": f.size() / max(states, 1), "time_ratio": mf_ms / frame_ms,
               "max_amp_diff_single_vs_multi": diff, "same_state": diff <= 1e-10,
               "timing": f"wall time of the whole circuit, median of {reps} after one warm-up"}
        mf.close()
        f.close()
        return out
    except Exception as e:  # the headline line must not depend on this leg
        return {"error": f"{type(e).__name__}: {e}"}


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-program", action="store_true", help="no single-CTA program for the small-frame prefix")
    ap.add_argument("--no-grid-program", action="store_true",
                    help="per-op launches after the prefix instead of the grid program")
    ap.add_argument("--no-campaign", action="store_true", help="skip the batched-campaign leg")
    ap.add_argument("--campaign-variants", type=int, default=4096)
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-multiframe", action="store_true", help="skip the multiframe leg")
    ap.add_argument("--no-streaming", action="store_true",
                    help="skip the per-kernel roofline leg of the streaming kernels at 16 words per phase vector")
    ap.add_argument("--serving-requests", type=int, default=30, help="requests per load point of the serving sweep")
    ap.add_argument("--serving-slots", type=int, default=32)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    else:
        torch.cuda.set_device(0)
    from paper_1712_03554_gb300 import sf

    seed = args.seed + rank
    n = N_QUBITS
    x, plan, y = build_plan(n, seed)
    updates, coal_elems, rec, graph_rec, peak, W, ops_rec, k_before = instrumented_pass(sf, n, plan, y)
    model = bytes_model(W, n)

    stream = torch.cuda.Stream()
    use_grid = not args.no_grid_program
    # the first plan entries run as one single-CTA program while the frame is
    # small, the rest as one grid program (or per op)
    cands = () if args.no_program else (256, 512, 1024, 2048, 4096)
    max_frame, p_pre, m_pre, d_prog, n_rec = choose_program_prefix(sf, torch, n, plan, y, stream, cands,
                                                                    grid=use_grid)
    if p_pre or use_grid:
        graph_rec = {cls: [] for cls in graph_rec}
        seg_bytes = gp_bytes = 0
        for (pi, cls, a, b) in ops_rec:
            if pi < p_pre:
                seg_bytes += model[cls](a, b)
            elif use_grid:
                gp_bytes += model[cls](a, b)
            else:
                graph_rec[cls].append((a, b))
        if p_pre:
            graph_rec["segment"] = [(seg_bytes, 0)]
        if use_grid and n_rec > m_pre:
            graph_rec["gprog"] = [(gp_bytes, 0)]
        # the single-CTA program leaves no index: the grid program, or the first
        # merged branch after it, builds one
        if p_pre and p_pre < len(plan) and (use_grid or (plan[p_pre][0] == "NK" and not any(
                pi == p_pre and cls == "index" for (pi, cls, a, b) in ops_rec))):
            kk = k_before[p_pre]
            graph_rec["index"].insert(0, (kk, kk))
    frame = sf.Frame(n, MAX_ELEMS, stream=stream)
    # device-resident gate lists for the graph path
    dev_lists = []
    for op in ([] if use_grid else plan[p_pre:]):
        if op[0] == "C":
            arr = np.array([[g[0], g[1], g[2], 0] for g in op[1]], dtype=np.uint32)
            t = torch.from_numpy(arr.view(np.int32)).cuda()
            dev_lists.append(t)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def async_part(fr):
        fr.reset()
        if m_pre:
            fr.apply_program_device(d_prog.data_ptr(), m_pre, DROP_EPS, 0, 0, max_frame)
        if use_grid:
            if n_rec > m_pre:
                fr.apply_program_grid_device(d_prog.data_ptr() + 24 * m_pre, n_rec - m_pre, DROP_EPS)
            return
        di = 0
        for op in plan[p_pre:]:
            if op[0] == "C":
                fr.apply_clifford_device(dev_lists[di].data_ptr(), dev_lists[di].shape[0])
                di += 1
            elif op[0] == "NK":
                fr.apply_nonclifford_coalesce(op[1], op[2], op[3], op[4], DROP_EPS)
            elif op[0] == "N":
                fr.apply_nonclifford(op[1], op[2], op[3], op[4])
            elif op[0] == "K":
                fr.coalesce(DROP_EPS)

    def tail(fr):
        p = fr.measure(0, -1)
        a = fr.amplitude(y)
        return p, a

    # reference result of the eager path
    with torch.cuda.stream(stream):
        async_part(frame)
    p_ref, a_ref = tail(frame)
    # the grid program counts the element bytes its passes read and write (each
    # pass once); that is its algorithmic traffic, not the per-op sum above
    gp_moved = None
    if use_grid and n_rec > m_pre:
        with torch.cuda.stream(stream):
            async_part(frame)
        gp_moved = frame.grid_program_bytes()
        tail(frame)
        graph_rec["gprog"] = [(gp_moved, 0)]

    # per-class device time of one eager step -> dominant kernel class
    per_class = {}
    for cls in sf.KERNEL_CLASSES:
        if cls in ("export", "reset", "filter"):
            continue
        frame.time_kernel(cls)
        async_part(frame)
        tail(frame)
        ms, cnt = frame.kernel_time()
        per_class[cls] = ms
    frame.time_kernel(-1)
    # the roofline is reported for the class with the largest device time in the
    # captured part of the step (where the timed event pairs live)
    graph_classes = [cls for cls in per_class if graph_rec.get(cls)] or list(per_class)
    dominant = max(graph_classes, key=per_class.get)
    # the streaming kernel with the largest time, when the dominant class is a
    # latency-bound program kernel: its roofline is reported beside (a class of
    # the eager tail is timed on the tail's launches)
    streaming = ("affine", "branch", "branch_merge", "insert", "compact", "index", "cofactor", "prob", "amplitude")
    hbm_classes = [cls for cls in streaming if per_class.get(cls, 0) > 0 and rec.get(cls)]
    second = max(hbm_classes, key=per_class.get) if dominant in ("segment", "gprog") and hbm_classes else None
    second_in_graph = second is not None and bool(graph_rec.get(second))

    # capture the asynchronous part in CUDA graphs: `graph` for the timed steps,
    # `tgraph` (the same launches with the dominant class bracketed by CUDA
    # events) for the roofline measurement
    use_graph = not args.no_graph
    graph = tgraph = tgraph2 = None
    token = 0
    if use_graph:
        try:
            frame.time_kernel(dominant)
            async_part(frame)  # warm (creates the event pairs outside capture)
            tail(frame)
            frame.time_kernel(dominant)
            tgraph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(tgraph, stream=stream):
                async_part(frame)
            frame.time_kernel(-1)  # keep the captured pairs; eager tail launches are not timed
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                async_part(frame)
            token = frame.host_state()  # replays restore the handle's host bookkeeping
            for gph in (graph, tgraph, graph):
                with torch.cuda.stream(stream):
                    gph.replay()
                frame.set_host_state(token)
                p_g, a_g = tail(frame)
                if abs(p_g[0] - p_ref[0]) > 1e-10 or abs(a_g - a_ref) > 1e-10:
                    raise RuntimeError("graph replay differs from the eager step")
        except Exception as exc:  # fall back to eager launches from the host
            print(f"# graph capture unavailable ({exc}); timing eager launches", file=sys.stderr)
            graph = tgraph = tgraph2 = None
    if graph is None:
        frame.time_kernel(dominant)

    def step(gph=None):
        if graph is not None:
            with torch.cuda.stream(stream):
                (gph or graph).replay()
            frame.set_host_state(token)
            return tail(frame)
        frame.time_kernel(dominant)
        with torch.cuda.stream(stream):
            async_part(frame)
        frame.time_kernel(-1)
        return tail(frame)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()

    launches0 = frame.kernel_launches()
    step_ms = []
    dom_ms = 0.0
    dom_launches = 0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()  # evict the frame from L2 between steps
                ev0.record(stream)
            step()
            with torch.cuda.stream(stream):
                ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            if graph is None:
                ms, cnt = frame.kernel_time()
                dom_ms += ms
                dom_launches += cnt
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
        launches_timed = frame.kernel_launches() - launches0
        # roofline of the dominant class: the same steps replayed with its event pairs
        if tgraph is not None:
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.zero_()
                step(tgraph)
                ms, cnt = frame.kernel_time()
                dom_ms += ms
                dom_launches += cnt
        sec_ms, sec_launches = 0.0, 0
        if second is not None and not second_in_graph:
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.zero_()
                frame.time_kernel(second)  # brackets this class's launches from here on
                if graph is not None:
                    with torch.cuda.stream(stream):
                        graph.replay()
                    frame.set_host_state(token)
                else:
                    with torch.cuda.stream(stream):
                        async_part(frame)
                tail(frame)
                ms, cnt = frame.kernel_time()
                sec_ms += ms
                sec_launches += cnt
            frame.time_kernel(-1)
        elif second is not None and tgraph is not None:
            # captured only now: the timing event pairs of a handle are one pool
            frame.time_kernel(second)
            async_part(frame)
            tail(frame)
            frame.time_kernel(second)
            tgraph2 = torch.cuda.CUDAGraph()
            with torch.cuda.graph(tgraph2, stream=stream):
                async_part(frame)
            frame.time_kernel(-1)
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.zero_()
                step(tgraph2)
                ms, cnt = frame.kernel_time()
                sec_ms += ms
                sec_launches += cnt
    clocks = clk.summary()
    # graph replays do not pass through the host launch counter: add the captured kernels
    launches_total = launches_timed  # launched from the host inside the timed steps
    if graph is not None and use_grid:  # reset and the program kernels
        launches_total += (1 + (1 if m_pre else 0) + (1 if n_rec > m_pre else 0)) * args.steps
    elif graph is not None:
        launches_total += graph_launch_count(plan[p_pre:], start_indexed=not m_pre,
                                             extra=1 if m_pre else 0) * args.steps  # graph replays
    ms_step = float(np.mean(step_ms))

    # e2e: the public API with host buffers -- the QFT's records from host
    # memory in one sf_run_program call (the library copies them), then the
    # measurement and the amplitude, each reading its result back
    e2e_frame = sf.Frame(n, MAX_ELEMS, stream=stream)
    h_recs = plan_records(sf, plan)[0]
    h2d = int(h_recs.nbytes) + 8 * e2e_frame.W
    d2h = 16 + 16

    def e2e_step():
        e2e_frame.reset()
        e2e_frame.run_program_records(h_recs, DROP_EPS)
        return e2e_frame.measure(0, -1), e2e_frame.amplitude(y)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            e2e_step()
        e2e_ms = []
        for _ in range(max(3, args.steps // 2)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p_e, a_e = e2e_step()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    if abs(a_e - a_ref) > 1e-10 or abs(p_e[0] - p_ref[0]) > 1e-10:
        raise RuntimeError("e2e result differs from the device path")
    e2e_ms_step = float(np.mean(e2e_ms))

    # whole-job aggregation
    tot_updates, max_ms, max_e2e = aggregate_ranks(dist, updates, ms_step, e2e_ms_step, "cuda")
    value = tot_updates / (max_ms * 1e-3)
    e2e_value = tot_updates / (max_e2e * 1e-3)

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    peak_gbs, peak_src = measured_peak_gbs()
    dom_bytes_per_step = sum(model[dominant](a, b) for a, b in graph_rec[dominant])
    dom_launch_per_step = max(1, len(graph_rec[dominant]))
    avg_launch_ms = dom_ms / max(1, dom_launches)
    bytes_per_launch = dom_bytes_per_step / dom_launch_per_step
    achieved = bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9 if avg_launch_ms > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                "frac": achieved / peak_gbs, "peak_source": peak_src, "traffic": ncu_traffic(dominant),
                "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_launch_ms * 1e3,
                "launches_timed": dom_launches}
    if dominant == "gprog" and gp_moved is not None:
        roofline["bytes_model"] = ("the grid program's own count of element bytes (8 per phase-vector word, 16 per "
                                   "amplitude) read and written by its passes, each pass once (sf_grid_program_bytes)")
        roofline["per_op_equivalent_bytes"] = gp_bytes if (p_pre or use_grid) else None
    if dominant in ("segment", "gprog"):
        roofline["note"] = ("the dominant kernel is a program kernel (the single-CTA small-frame prefix, or the "
                            "grid program that runs the rest of the circuit with grid barriers between its "
                            "passes): a serial chain of latency-bound passes whose achieved bandwidth is the "
                            "summed algorithmic bytes of its ops over its time; roofline_streaming gives the "
                            "streaming kernel with the largest time")
    roofline_streaming = None
    if second is not None and sec_launches:
        src = graph_rec if second_in_graph else rec
        b2 = sum(model[second](a, b) for a, b in src[second]) / max(1, len(src[second]))
        t2 = sec_ms / sec_launches
        a2 = b2 / (t2 * 1e-3) / 1e9
        roofline_streaming = {"bound": "hbm", "kernel": second, "achieved": a2, "peak": peak_gbs, "unit": "GB/s",
                              "frac": a2 / peak_gbs, "peak_source": peak_src, "traffic": ncu_traffic(second),
                              "algorithmic_bytes_per_launch": b2, "avg_launch_us": t2 * 1e3,
                              "launches_timed": sec_launches}
    step_share = {k: round(v / max(1e-9, sum(per_class.values())), 4) for k, v in
                  sorted(per_class.items(), key=lambda kv: -kv[1])}

    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(n, plan, y, updates)
    batched = None if args.no_campaign else campaign_leg(sf, torch, args.campaign_variants)
    served = None if (args.no_serving or args.serving_requests <= 0) else serving_leg(sf, args.serving_requests,
                                                                                       args.serving_slots)
    multiframe = None if args.no_multiframe else multiframe_leg(sf)
    streaming = None
    if not args.no_streaming:
        try:
            from paper_1712_03554_gb300 import kernel_bench
            streaming = kernel_bench.streaming_roofline(1000, 20, reps=2, peak_gbs=peak_gbs)
            streaming["peak_source"] = peak_src
            streaming["workload"] = ("n = 1000 (16 words per phase vector), 2^20 elements after 4000 random Clifford "
                                     "gates and 20 merged T gates on scrambled qubits; each per-op kernel class "
                                     "timed alone with CUDA events")
        except Exception as e:  # the headline line must not depend on this leg
            streaming = {"error": f"{type(e).__name__}: {e}"}

    out = {
        "impl": "gb300", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_qubits": n, "seed": args.seed, "max_elems": MAX_ELEMS,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "flushed between steps (512 MiB write)", "cuda_graph": graph is not None,
                   "updates_per_step": updates, "coalesce_elems_per_step": coal_elems,
                   "program_prefix": {"plan_entries": p_pre, "records": m_pre, "max_frame": max_frame,
                                      "of_plan_entries": len(plan), "chosen_by": "eager step timing sweep"},
                   "grid_program": {"records": n_rec - m_pre} if use_grid else None,
                   "coalesce_elems_per_s": coal_elems * world / (max_ms * 1e-3), "frame_peak": peak,
                   "wall_s_timed_region": wall},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": max_e2e,
                "path": "sf_reset; sf_run_program (the QFT's sf_op records from host memory, copied by the library); "
                        "sf_measure(0, -1); sf_amplitude -- results read back every step"},
        "roofline": roofline,
        "roofline_streaming": roofline_streaming,
        "kernel_time_share_eager_step": step_share,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": int(launches_total),
        "batched": batched,
        "served": served,
        "multiframe": multiframe,
        "roofline_streaming_w16": streaming,
    }
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def aggregate_ranks(dist, updates: float, ms_step: float, e2e_ms_step: float, device: str):
    """Whole-job figures of a weak-scaling run: every rank simulates its own
    instance, so the updates add up and the step time is the slowest rank's.
    dist is torch.distributed (None for one process)."""
    if dist is None:
        return float(updates), float(ms_step), float(e2e_ms_step)
    import torch
    t = torch.tensor([float(updates), ms_step, e2e_ms_step], dtype=torch.float64, device=device)
    tu = t.clone()
    dist.all_reduce(tu[:1], op=dist.ReduceOp.SUM)
    dist.all_reduce(t[1:], op=dist.ReduceOp.MAX)
    return float(tu[0]), float(t[1]), float(t[2])


def graph_launch_count(plan, start_indexed: bool = True, extra: int = 0) -> int:
    """Kernels in the captured part of a step: reset, the program kernel if any
    (extra), 2 per Clifford batch (tableau + affine), 1 per unmerged branch, 2
    per generic coalesce (insert + compact), 1 per merged branch plus an index
    build when the previous op left the frame unindexed."""
    cnt = 1 + extra
    indexed = start_indexed
    for op in plan:
        cnt += {"C": 2, "N": 1, "K": 2, "NK": 1}[op[0]]
        if op[0] == "NK" and not indexed:
            cnt += 1
        indexed = op[0] in ("NK", "K")
    return cnt


if __name__ == "__main__":
    sys.exit(main())
