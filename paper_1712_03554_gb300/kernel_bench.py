"""Per-kernel throughput of the frame kernels at a chosen frame size.

A frame of exactly 2^m distinct elements is built on n = 40 qubits (H on every
qubit, then T on qubits 0..m-1, merged after each), and each kernel class is
timed with the library's CUDA-event brackets (sf_time_kernel) on its own
stream.  GB/s use the algorithmic bytes of each kernel (phase vectors and
amplitudes read and written; index and hash tables are not counted).

  python -m paper_1712_03554_gb300.kernel_bench throughput 16 20 24
  python -m paper_1712_03554_gb300.kernel_bench latency
  python -m paper_1712_03554_gb300.kernel_bench merge-case 20   (a short run for ncu captures)
  python -m paper_1712_03554_gb300.kernel_bench qft-step [max_frame] (one eager QFT n=20 step, the bench's circuit)
  python -m paper_1712_03554_gb300.kernel_bench qft-grid          (QFT n=20: per-op vs grid program, wall per pass)
  python -m paper_1712_03554_gb300.kernel_bench qft-trace         (QFT n=20 in the grid program: time per phase)
  python -m paper_1712_03554_gb300.kernel_bench streaming 1000 20 (per-op streaming kernels, n qubits, 2^m elements)
  python -m paper_1712_03554_gb300.kernel_bench campaign-case 64 (one campaign launch, 32 threads, global index)
  python -m paper_1712_03554_gb300.kernel_bench clifford-case 1024 (one Clifford batch of 200 gates at n)
  python -m paper_1712_03554_gb300.kernel_bench clifford-rate     (tableau us per gate, n = 64 ... 1024)
  python -m paper_1712_03554_gb300.kernel_bench clifford-mix 1024 (tableau us per gate by gate mix)
  python -m paper_1712_03554_gb300.kernel_bench cuccaro 5 6 7   (adder: Toffoli by cofactors vs Clifford+7T)
  python -m paper_1712_03554_gb300.kernel_bench cuccaro-mf 4 5 6 7 (adder: one frame vs a multiframe)
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np

from . import circuits as c
from . import sf

N = 40
E = 24  # bytes of one element at W = 1: phase vector + FP64 complex amplitude


def frame_of(n: int, m: int, cap: int, stream=None):
    f = sf.Frame(n, cap, stream=stream)
    f.apply_clifford([(c.H, q, 0) for q in range(n)])
    for q in range(m):
        f.apply_nonclifford_coalesce(c.T, q, 0, 0.0, 1e-12)
    f.sync()
    return f


def timed(f, cls, fn, reps):
    f.time_kernel(cls)
    for _ in range(reps):
        fn()
    ms, cnt = f.kernel_time()
    f.time_kernel(-1)
    return ms / max(cnt, 1)


def throughput(ms_list):
    import torch
    stream = torch.cuda.Stream()
    for m in ms_list:
        k = 1 << m
        f = frame_of(N, m, 1 << (m + 2), stream)
        assert f.size() == k
        res = {"k": k}
        gates = [(c.S, m + 1, 0), (c.CNOT, m + 2, m + 3), (c.H, m + 4, 0), (c.CZ, m + 5, m + 6)]
        ms = timed(f, "affine", lambda: f.apply_clifford(gates), 5)
        res["affine_us"] = ms * 1e3
        res["affine_GBs"] = 2 * 8 * k / (ms * 1e-3) / 1e9
        res["clifford_us_4_gates"] = timed(f, "clifford", lambda: f.apply_clifford(gates), 5) * 1e3

        def tt():  # k -> 2k -> k
            f.apply_nonclifford_coalesce(c.T, m, 0, 0.0, 1e-12)
            f.apply_nonclifford_coalesce(c.TDG, m, 0, 0.0, 1e-12)
        ms = timed(f, "branch_merge", tt, 3)
        res["branch_merge_us"] = ms * 1e3
        res["branch_merge_GBs"] = E * 3 * k / (ms * 1e-3) / 1e9  # per launch: k in + 2k out, or 2k in + k out

        def br():
            f.apply_nonclifford(c.T, m, 0, 0.0)
            f.coalesce(1e-12)
            f.apply_nonclifford(c.TDG, m, 0, 0.0)
            f.coalesce(1e-12)
        ms = timed(f, "branch", br, 2)
        res["branch_us"] = ms * 1e3
        res["branch_GBs"] = (E * 1.5 * k + E * 3 * k) / (ms * 1e-3) / 1e9
        res["insert_us"] = timed(f, "insert", br, 2) * 1e3
        res["compact_us"] = timed(f, "compact", br, 2) * 1e3
        ms = timed(f, "index", lambda: (f.apply_clifford(gates),
                                        f.apply_nonclifford_coalesce(c.PHASE, m + 7, 0, 0.0, 1e-12)), 2)
        res["index_us"] = ms * 1e3
        res["index_GBs"] = 8 * k / (ms * 1e-3) / 1e9
        assert f.size() == k
        t0 = time.perf_counter()
        f.measure(m + 10, -1)
        res["measure_ms_wall"] = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        f.amplitude(12345)
        res["amplitude_ms_wall"] = (time.perf_counter() - t0) * 1e3
        print(json.dumps(res), flush=True)
        f.close()


def latency():
    import torch
    stream = torch.cuda.Stream()
    res = {}
    for m in (4, 8, 12, 16, 20):
        f = frame_of(30, m, 1 << (m + 2), stream)
        res[f"branch_merge_us_k2^{m}"] = timed(f, "branch_merge", lambda: (
            f.apply_nonclifford_coalesce(c.CPHASE, m, m + 1, 0.3, 1e-12),
            f.apply_nonclifford_coalesce(c.CPHASE, m, m + 1, -0.3, 1e-12)), 5) * 1e3
        res[f"affine_us_k2^{m}"] = timed(f, "affine", lambda: f.apply_clifford([(c.S, m + 2, 0)]), 5) * 1e3
        res[f"clifford_us_k2^{m}"] = timed(f, "clifford", lambda: f.apply_clifford([(c.S, m + 2, 0)]), 5) * 1e3
        f.close()
    print(json.dumps({k: round(v, 2) for k, v in res.items()}), flush=True)


def merge_case(m):
    """m merged T gates (launches 0..m-1 of k_branch_merge at k = 2^i), then T
    and T-dagger on a fresh qubit (launch m: 2^m -> 2^(m+1), launch m+1 back)."""
    f = frame_of(N, m, 1 << (m + 2))
    f.apply_nonclifford_coalesce(c.T, m, 0, 0.0, 1e-12)
    f.apply_nonclifford_coalesce(c.TDG, m, 0, 0.0, 1e-12)
    f.sync()
    print("k", f.size())


def qft_step(seed=0, max_frame=2048):
    """The bench's step eagerly: QFT n = 20 on a seeded random basis state, the
    small-frame prefix as one sf_apply_program launch (frame limit max_frame,
    0: none), the rest as one sf_apply_program_grid launch, then the
    probabilities of qubit 0 and one amplitude."""
    x, ops = c.qft_random_input(20, seed)
    f = frame_of(20, 0, 1 << 21)
    f.reset()
    i = f.apply_program(ops, max_frame=max_frame)[0] if max_frame else 0
    f.apply_program_grid(ops[i:])
    f.measure(0, -1)
    f.amplitude(x)
    f.sync()
    print("k", f.size())


def qft_grid(reps=5):
    """QFT n = 20 (the bench's circuit) three ways, wall time per pass after a
    warm-up (median of reps): the small-frame prefix in the single-CTA program
    and the rest per op; the prefix and the rest in the grid program; all of
    it in the grid program.  Then one frame check against the closed form."""
    import torch
    x, ops = c.qft_random_input(20, 0)
    f = frame_of(20, 0, 1 << 21)
    f.reset()
    i = f.apply_program(ops, max_frame=2048)[0]
    recs_a, _ = sf.encode_program([ops[:i]])
    recs_b, _ = sf.encode_program([ops[i:]])
    recs_all, _ = sf.encode_program([ops])
    dev = {k: torch.from_numpy(v.view(np.uint8).copy()).cuda() for k, v in
           (("a", recs_a), ("b", recs_b), ("all", recs_all))}
    n_rec = {"a": len(recs_a), "b": len(recs_b), "all": len(recs_all)}
    res = {}
    for mode in ("prefix+per-op", "prefix+grid", "grid"):
        ts = []
        for rep in range(reps + 1):
            f.reset()
            f.sync()
            t0 = time.perf_counter()
            if mode == "grid":
                f.apply_program_grid_device(dev["all"].data_ptr(), n_rec["all"])
            else:
                f.apply_program_device(dev["a"].data_ptr(), n_rec["a"], 1e-12, 0, 0, 2048)
                if mode == "prefix+grid":
                    f.apply_program_grid_device(dev["b"].data_ptr(), n_rec["b"])
                else:
                    c.run(f, ops[i:])
            f.sync()
            ts.append(time.perf_counter() - t0)
        res[mode + "_ms"] = round(sorted(ts[1:])[len(ts[1:]) // 2] * 1e3, 3)
        res[mode + "_k"] = f.size()
        y = 12345
        res[mode + "_amp_err"] = abs(f.amplitude(y) - c.qft_expected_amplitude(20, x, y))
    print(json.dumps(res), flush=True)


def _random_qubits(f, n):
    """Qubits whose Z anticommutes with some row of the handle's tableau."""
    x, _, _ = f.tableau()
    return [q for q in range(n) if ((x[:, q // 64] >> np.uint64(q % 64)) & np.uint64(1)).any()]


def streaming_roofline(n=1000, m=20, reps=3, seed=7, peak_gbs=None):
    """The per-op streaming kernels on a frame of 2^m elements over n qubits
    (n = 1000: 16 words per phase vector, 144 B per element; 2^20 elements are
    151 MB, more than L2): a scramble of 4n random H/S/CNOT gates, then T on m
    random qubits of the scrambled tableau (masks spread over all words),
    merged after each.  Each kernel class is timed with CUDA events on the
    frame's stream, L2 flushed (512 MiB write) before every timed operation;
    GB/s = algorithmic bytes (phase vectors and amplitudes read and written;
    index and slot tables are scratch) / device time.  The frame returns to
    2^m elements after each operation pair."""
    import torch
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    k = 1 << m
    f = sf.Frame(n, 4 * k, stream=stream)  # a merge may hold 2 x (2k) children before merging
    f.apply_clifford([(g[1], g[2], g[3]) for g in c.random_clifford(n, 4 * n, seed)])
    rq = _random_qubits(f, n)
    rng = c.rng_for(seed + 1)
    pick = [rq[int(i)] for i in rng.choice(len(rq), size=m + 2 + 4 * reps, replace=False)]
    for q in pick[:m]:
        f.apply_nonclifford_coalesce(c.T, q, 0, 0.0, 1e-12)
    assert f.size() == k, f.size()
    W = f.W
    e = 8 * W + 16
    qa, qb = pick[m], pick[m + 1]
    fresh = iter(pick[m + 2:])  # a random qubit for every measurement

    def timed_cls(classes, op, reps=reps):
        # one untimed pass first (first-use costs of the driver stay out), then
        # the median over the timed passes of the time per launch
        op()
        assert f.size() == k
        per = {cl: [] for cl in classes}
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush.zero_()
            for cl in classes:  # one class per pass of the op
                f.time_kernel(cl)
                with torch.cuda.stream(stream):
                    flush.zero_()
                torch.cuda.nvtx.range_push("streaming_timed")  # for profiler filters
                op()
                torch.cuda.nvtx.range_pop()
                ms, cnt = f.kernel_time()
                f.time_kernel(-1)
                kk = f.size()  # synchronises and reports a deferred device error here
                assert kk == k, (cl, kk, k)
                if cnt:
                    per[cl].append((ms / cnt, cnt))
        out = {}
        for cl, v in per.items():
            v = sorted(v)
            out[cl] = v[len(v) // 2] if v else (0.0, 0)
        return out

    rows = {}

    def add(name, cls, ms, bytes_per_launch):
        gbs = bytes_per_launch / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        rows[name] = {"kernel_class": cls, "us": ms * 1e3, "bytes_per_launch": bytes_per_launch, "GB_s": gbs}
        if peak_gbs:
            rows[name]["frac"] = gbs / peak_gbs

    t = timed_cls(["affine"], lambda: f.apply_clifford([(c.S, qa, 0)]))
    add("K2 phase update (affine, W words per element in and out)", "affine", t["affine"][0], 2 * 8 * W * k)

    def merged_pair():
        f.apply_nonclifford_coalesce(c.T, qb, 0, 0.0, 1e-12)
        f.apply_nonclifford_coalesce(c.TDG, qb, 0, 0.0, 1e-12)
    f.apply_nonclifford_coalesce(c.PHASE, qa, 0, 0.0, 1e-12)  # the index is current before timing
    t = timed_cls(["branch_merge"], merged_pair)
    add("K3+K4 branch merged through the index (k -> 2k and 2k -> k)", "branch_merge", t["branch_merge"][0],
        3 * e * k)

    def unmerged():
        f.apply_nonclifford(c.T, qb, 0, 0.0)
        f.coalesce(1e-12)
        f.apply_nonclifford_coalesce(c.TDG, qb, 0, 0.0, 1e-12)
    t = timed_cls(["branch", "insert", "compact"], unmerged)
    add("K3 branch unmerged (k in, 2k out)", "branch", t["branch"][0], 3 * e * k)
    add("K4 coalesce: insert (2k elements hashed)", "insert", t["insert"][0], 2 * e * k)
    add("K4 coalesce: compact (2k survivors written)", "compact", t["compact"][0], 2 * e * k)

    def reindex():
        f.apply_clifford([(c.S, qa, 0)])
        f.apply_nonclifford_coalesce(c.PHASE, qa, 0, 0.0, 1e-12)
    t = timed_cls(["index"], reindex)
    add("index build (phase vectors read)", "index", t["index"][0], 8 * W * k)

    def measure_pair():
        q = next(fresh)
        f.measure(q, -1)
        f.measure(q, 0)
    t = timed_cls(["cofactor", "prob", "filter"], measure_pair)
    add("K5 cofactor merge (k in, 2k out)", "cofactor", t["cofactor"][0], 3 * e * k)
    add("K5 probabilities (one word + amplitude per element)", "prob", t["prob"][0], 24 * 2 * k)
    add("K5 collapse filter (2k in, k out)", "filter", t["filter"][0], 3 * e * k)
    assert f.size() == k, f.size()
    t = timed_cls(["amplitude"], lambda: f.amplitude(12345))
    add("K6 amplitude query (every element read)", "amplitude", t["amplitude"][0], e * k)
    f.close()
    return {"n_qubits": n, "words_per_phase_vector": W, "elements": k, "bytes_per_element": e,
            "frame_bytes": e * k, "l2": "flushed (512 MiB write) before every timed operation", "kernels": rows}


PHASE_NAMES = {1: "clifford", 2: "plan", 3: "branch", 4: "in-place", 5: "merge", 6: "compact", 7: "index",
               8: "map", 10: "check"}


def qft_trace(seed=0, reps=3):
    """QFT n = 20 (the bench's circuit) as one grid program launch with per-phase
    tracing (sf_set_trace): each phase's kind, records, elements, CTA 0's own
    work, and the wait for the last CTA; summed by kind.  Times in us from the
    GPU's global timer (the last of reps launches after a warm-up)."""
    import torch
    x, ops = c.qft_random_input(20, seed)
    recs, _ = sf.encode_program([ops])
    d = torch.from_numpy(recs.view(np.uint8).copy()).cuda()
    f = sf.Frame(20, 1 << 21)
    f.set_trace(True)
    for _ in range(reps + 1):
        f.reset()
        f.apply_program_grid_device(d.data_ptr(), len(recs))
        f.sync()
    tr = f.grid_program_trace().astype(np.int64)
    rows, by_kind = [], {}
    mark_names = ("step_wait", "step_taken", "plan_end", "hull_end", "pass_start", "map_tables_end", "loop_end",
                  "prev_pass_counts_read")
    for i, rec in enumerate(tr):
        code, t0, arr0, last, who = (int(v) for v in rec[:5])
        kind = PHASE_NAMES.get(code & 15, str(code & 15))
        nrec, k = (code >> 4) & 15, code >> 8
        end = max(arr0, last)
        row = {"i": i, "kind": kind, "records_mod16": nrec, "k": k, "phase_us": (end - t0) / 1e3,
               "cta0_us": (arr0 - t0) / 1e3, "last_after_cta0_us": (last - arr0) / 1e3, "last_cta": who}
        marks = {nm: round((int(v) - t0) / 1e3, 3) for nm, v in zip(mark_names, rec[5:]) if int(v) >= t0 > 0}
        row["marks_us_from_start"] = marks
        rows.append(row)
        agg = by_kind.setdefault(kind, {"phases": 0, "us": 0.0})
        agg["phases"] += 1
        agg["us"] += row["phase_us"]
    total = (max(int(tr[-1][2]), int(tr[-1][3])) - int(tr[0][1])) / 1e3 if len(tr) else 0.0
    print(json.dumps({"phases": len(rows), "total_us": total, "by_kind": by_kind,
                      "moved_bytes": f.grid_program_bytes()}), flush=True)
    for r in rows:
        print(json.dumps(r), flush=True)
    # the planning CTAs, per step: durations of each stage (us) and the gap
    # between consecutive publications of the plan CTA
    pt = f.grid_program_plan_trace(64).astype(np.int64)
    t_ref = int(tr[0][1]) if len(tr) else 0
    prev_pub = None
    plan_rows = []
    for st, m in enumerate(pt):
        if not m.any():
            continue
        row = {"step": st,
               "tableau_us": (m[1] - m[0]) / 1e3 if m[1] and m[0] else None,
               "plan_wait_us": (m[2] - m[1]) / 1e3 if m[2] and m[1] else None,
               "plan_copy_us": (m[3] - m[2]) / 1e3 if m[3] and m[2] else None,
               "plans_us": (m[4] - m[3]) / 1e3 if m[4] and m[3] else None,
               "extents_hull_map_us": (m[5] - m[4]) / 1e3 if m[5] and m[4] else None,
               "walk_verdicts_us": (m[6] - m[5]) / 1e3 if m[6] and m[5] else None,
               "publish_us": (m[7] - m[6]) / 1e3 if m[7] and m[6] else None,
               "published_at_us": (m[7] - t_ref) / 1e3 if m[7] else None,
               "since_last_publication_us": (m[7] - prev_pub) / 1e3 if m[7] and prev_pub else None}
        if m[7]:
            prev_pub = int(m[7])
        plan_rows.append(row)
    for r in plan_rows:
        print(json.dumps({"plan": r}), flush=True)
    y = 12345
    print(json.dumps({"amp_err": abs(f.amplitude(y) - c.qft_expected_amplitude(20, x, y))}), flush=True)


def campaign_case(nv=64):
    """One launch of the campaign kernel on nv Steane variants."""
    eng = sf.Campaign(c.STEANE_N, 4096)
    eng.set_shape(32, False)
    res = eng.run(c.steane_campaign(nv, seed=0))
    print("ok", int((res["status"] != 0).sum()) == 0, "ctas", eng.ctas())


def clifford_case(n=1024, gates=200):
    """One Clifford batch of random H/S/CNOT gates on a scrambled tableau."""
    ops = c.random_clifford(n, 4000 + gates, seed=n, kinds=(c.H, c.S, c.CNOT))
    g = [(op[1], op[2], op[3]) for op in ops]
    f = sf.Frame(n, 64)
    f.apply_clifford(g[:4000])
    f.sync()
    f.apply_clifford(g[4000:])
    f.sync()
    print("r", f.tableau()[2])


def clifford_rate(ns=(64, 128, 256, 512, 1024), gates=1000):
    """Tableau cost per Clifford gate (class clifford, CUDA events): a batch of
    `gates` random H/S/CNOT gates on a tableau scrambled by 4n gates, for each n."""
    out = {}
    for n in ns:
        ops = c.random_clifford(n, 4 * n + gates, seed=n, kinds=(c.H, c.S, c.CNOT))
        g = [(op[1], op[2], op[3]) for op in ops]
        f = sf.Frame(n, 64)
        f.apply_clifford(g[:4 * n])
        f.sync()
        ms = timed(f, "clifford", lambda: f.apply_clifford(g[4 * n:]), 1)
        out[f"n{n}_us_per_gate"] = round(ms * 1e3 / gates, 2)
        f.close()
    print(json.dumps(out), flush=True)


def clifford_mix(n=1024, gates=1000):
    """Tableau cost per gate at n by gate mix (class clifford, CUDA events), on a
    tableau scrambled by 4n random H/S/CNOT gates: H only; monomial gates only
    (S, CNOT, CZ: one repair at the end of the batch); H/S/CNOT."""
    out = {"n": n, "gates": gates}
    mixes = {"h_only": (c.H,), "monomial_only": (c.S, c.CNOT, c.CZ), "h_s_cnot": (c.H, c.S, c.CNOT)}
    for name, kinds in mixes.items():
        pre = c.random_clifford(n, 4 * n, seed=n, kinds=(c.H, c.S, c.CNOT))
        ops = c.random_clifford(n, gates, seed=n + 1, kinds=kinds)
        f = sf.Frame(n, 64)
        f.apply_clifford([(op[1], op[2], op[3]) for op in pre])
        f.sync()
        g = [(op[1], op[2], op[3]) for op in ops]
        timed(f, "clifford", lambda: f.apply_clifford(g), 1)  # warm-up
        ms = timed(f, "clifford", lambda: f.apply_clifford(g), 2)
        out[f"{name}_us_per_gate"] = round(ms * 1e3 / gates, 2)
        f.close()
    print(json.dumps(out), flush=True)


def cuccaro_compare(nbs=(5, 6, 7)):
    """The Cuccaro adder on the equal superposition with every Toffoli applied
    by cofactors (Eq. 2) and as Clifford+7T: wall time of the whole circuit
    (median of 3 after a warm-up) and the final frame size."""
    for nb in nbs:
        n = 2 * nb + 2
        row = {"nbits": nb, "qubits": n}
        for how in ("cofactor", "clifford_t"):
            ops = c.cuccaro(nb, True, toffoli=how)
            f = sf.Frame(n, 1 << min(2 * nb + 4, 24))
            ts = []
            for rep in range(4):
                f.reset()
                f.sync()
                t0 = time.perf_counter()
                c.run(f, ops)
                f.sync()
                ts.append(time.perf_counter() - t0)
            row[how + "_ms"] = sorted(ts[1:])[1] * 1e3
            row[how + "_frame"] = f.size()
            f.close()
        row["speedup"] = row["clifford_t_ms"] / row["cofactor_ms"]
        print(json.dumps(row), flush=True)


def cuccaro_multiframe(nbs=(4, 5, 6, 7)):
    """The Cuccaro adder on the equal superposition, Toffolis by cofactors
    (Eq. 2), as one frame and as a multiframe (COALESCE and the merge of equal
    matrices after every Toffoli, Sec. IV): wall time of the whole circuit
    (median of 3 after a warm-up), final frames and states, kernel launches."""
    for nb in nbs:
        n = 2 * nb + 2
        ops = c.cuccaro(nb, True, toffoli="cofactor", coalesce=False)
        row = {"nbits": nb, "qubits": n}
        ts = []
        f = sf.Frame(n, 1 << min(2 * nb + 2, 24))
        for rep in range(4):
            f.reset()
            f.sync()
            l0 = f.kernel_launches()
            t0 = time.perf_counter()
            c.run(f, ops)
            f.sync()
            ts.append(time.perf_counter() - t0)
        row["frame_ms"] = sorted(ts[1:])[1] * 1e3
        row["frame_states"] = f.size()
        row["frame_launches"] = f.kernel_launches() - l0
        f.close()
        ts = []
        for rep in range(4):
            mf = sf.MultiFrame(n, max_elems=4096, max_frames=8192)
            mf.count()
            l0 = mf.kernel_launches()
            t0 = time.perf_counter()
            c.run(mf, ops)
            nf, ns = mf.count()
            ts.append(time.perf_counter() - t0)
            launches = mf.kernel_launches() - l0
            mf.close()
        row["multiframe_ms"] = sorted(ts[1:])[1] * 1e3
        row["multiframe_frames"], row["multiframe_states"] = nf, ns
        row["multiframe_launches"] = launches
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    mode = sys.argv[1] if len(sys.argv) > 1 else "throughput"
    args = [int(a) for a in sys.argv[2:]]
    if mode == "throughput":
        throughput(args or [16, 20, 24])
    elif mode == "latency":
        latency()
    elif mode == "merge-case":
        merge_case(args[0] if args else 20)
    elif mode == "qft-step":
        qft_step(max_frame=args[0] if args else 2048)
    elif mode == "qft-grid":
        qft_grid()
    elif mode == "qft-trace":
        qft_trace(args[0] if args else 0)
    elif mode == "streaming":
        import os
        peak = None
        try:
            with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                   "MEASURED_PEAKS.json")) as fh:
                peak = float(json.load(fh)["hbm_gbs"])
        except Exception:
            pass
        print(json.dumps(streaming_roofline(args[0] if args else 1000, args[1] if len(args) > 1 else 20,
                                            peak_gbs=peak)), flush=True)
    elif mode == "campaign-case":
        campaign_case(args[0] if args else 64)
    elif mode == "cuccaro":
        cuccaro_compare(args or [5, 6, 7])
    elif mode == "cuccaro-mf":
        cuccaro_multiframe(args or [4, 5, 6, 7])
    elif mode == "clifford-case":
        clifford_case(args[0] if args else 1024)
    elif mode == "clifford-rate":
        clifford_rate(tuple(args) if args else (64, 128, 256, 512, 1024))
    elif mode == "clifford-mix":
        clifford_mix(args[0] if args else 1024)
    else:
        raise SystemExit(f"unknown mode {mode}")
