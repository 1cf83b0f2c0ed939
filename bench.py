#!/usr/bin/env python
"""Benchmark of exact local-alignment search (effective GCUPS = m*n/time).

Workload (default): the 100 Mbp DNA text at 41% GC with 8 queries each of
10 kbp, 100 kbp and 1 Mbp (1% of each planted from the text at 5-15%
divergence), scheme <1,-3,-5,-2>, H = 19/21/23 from E = 10.  A step is one
batched search of all of a rank's queries with the index and queries resident
in HBM; `value` is sum(m) * n / step time over all ranks.  `plain` times the
same queries one launch sequence per query; `e2e` goes through the host API
(queries from host memory in, results to host memory out).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --workload sweep     # scheme and E-value sweeps (Sections 7.3, 7.4)

Under torchrun each rank takes every N-th query (queries are independent
problems; no collective on the data path) and the job time is the max over
ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import (DNA_SCALE_H, Scheme, dna_batch, dna_scale_bench, dna_scale_text, dna_serve,  # noqa: E402
                       dna_small, protein, PROTEIN)

METRIC = "effective GCUPS (m*n/time) at bit-exact hits, batched"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="dna_scale",
                   choices=["dna_scale", "dna_small", "dna_serve", "dna_batch", "protein", "sweep"])
    p.add_argument("--queries", type=int, default=4096, help="dna_batch: number of queries")
    p.add_argument("--plain-sample", type=int, default=256, help="dna_batch: queries timed one launch at a time")
    p.add_argument("--requests", type=int, default=1000, help="dna_serve: number of requests")
    p.add_argument("--rate", type=float, default=200.0, help="dna_serve: Poisson arrival rate (1/s)")
    p.add_argument("--slots", type=int, default=3, help="dna_serve: concurrent search slots")
    p.add_argument("--train-queries", type=int, default=256, help="dna_serve: searches logged to train the predictor")
    p.add_argument("--work-budget", type=float, default=4e8, help="dna_serve: predicted DP entries per batch")
    p.add_argument("--lengths", type=str, default="10000,100000,1000000")
    p.add_argument("--per-length", type=int, default=8)
    p.add_argument("--n", type=int, default=100_000_000)
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--leaf-segment", type=int, default=None)
    p.add_argument("--item-columns", type=int, default=None)
    p.add_argument("--batch-columns", type=int, default=None)
    p.add_argument("--leaf-delay", type=int, default=None)
    p.add_argument("--verbose", action="store_true")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def shard(n_items, rank, world):
    """Items of rank `rank` of `world`: every world-th item from rank.  Queries
    are independent problems, so the shards need no exchange."""
    return list(range(rank, n_items, world))


def job_totals(ms, units, dist=None, device="cpu"):
    """Whole-job time (max over ranks) and work (sum over ranks)."""
    if dist is None:
        return float(ms), float(units)
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def make_workload(args):
    """(name, text, queries, H list, scheme, description) identical on every rank."""
    scheme = Scheme(1, -3, -5, -2)
    if args.workload == "dna_small":
        wl = dna_small()
        return ("dna_small", wl.text, wl.queries, wl.H, scheme,
                {"workload": "dna_small: 100 kbp uniform ACGT text, one 1 kbp query with 5 planted "
                             "150-300 bp copies (10% subs, 2% indels), <1,-3,-5,-2>, H=30",
                 "n": int(wl.text.size), "queries": 1, "sum_m": int(wl.queries[0].size)})
    if args.workload == "protein":
        n = args.n if args.n != 100_000_000 else 50_000_000
        lengths = [100, 1000, 5000] if args.lengths == "10000,100000,1000000" else \
            [int(x) for x in args.lengths.split(",")]
        wl = protein(n=n, lengths=lengths, per_length=args.per_length)
        return ("protein", wl.text, wl.queries, wl.H, wl.scheme,
                {"workload": f"protein: {n:,} residues at background frequencies; {args.per_length} queries each of "
                             f"{'/'.join(str(x) for x in lengths)} residues with planted homologs at 30-60% identity; "
                             "BLOSUM62, gap -11/-1, H=50",
                 "n": int(n), "queries": len(wl.queries), "sum_m": int(sum(q.size for q in wl.queries)),
                 "l2": "flushed between timed steps (512 MiB write)"})
    lengths = [int(x) for x in args.lengths.split(",")]
    text, queries, H, _ = dna_scale_bench(n=args.n, lengths=lengths, per_length=args.per_length)
    desc = {"workload": f"dna_scale: {args.n:,} bp i.i.d. text at 41% GC; {args.per_length} queries each of "
                        f"{'/'.join(str(x) for x in lengths)} bp with 1% planted from the text at 5-15% "
                        f"divergence; <1,-3,-5,-2>; H={'/'.join(str(DNA_SCALE_H.get(m, 21)) for m in lengths)} "
                        f"(E=10)",
            "n": int(args.n), "queries": len(queries), "sum_m": int(sum(q.size for q in queries)),
            "l2": "flushed between timed steps (512 MiB write)"}
    return args.workload, text, queries, H, scheme, desc


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"ae_clocks_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_traffic(kernel, units):
    """DRAM bytes (read + write) of `kernel` for `units` work units (DP
    entries written by the trie levels for k_rows, sweep entries for k_leaf),
    from the per-unit figure of its last ncu capture
    (profiles/dram_per_unit.txt: `kernel bytes_per_unit sha1`).  None if there
    is no capture or the kernel's source changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_per_unit.txt")
    src_of = {"k_rows": "ae_rows_dna.cu", "k_leaf": "ae_kernels.cu"}
    if kernel not in src_of or not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel:
            src = os.path.join(ROOT, "paper_1208_0274_gb300", "csrc", src_of[kernel])
            digest = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
            if parts[2] != digest:
                return None
            return int(float(parts[1]) * units)
    return None


# Algorithmic work of the row update, per DP entry (the unit the method's cost
# is counted in, Table 4): the parent entry read (j and the packed M, G_a: 8 B,
# plus 2 B of node metadata amortised) and the child entry written (10 B); 6
# integer operations for a full three-term entry (D add, G_a add + add-max, G_b
# add-max, the two maxima of M).
BYTES_PER_ENTRY = 20
OPS_PER_ENTRY = 6
# Per (child, parent entry) triple, the unit the kernels iterate over: slot A
# (add, select, two adds and a max for G_a, a max, a threshold compare), slot B
# (add, select, compare), one add-max for G_b.
OPS_PER_TRIPLE = 12


def int_peaks():
    """Measured integer instruction rates of this GPU (ae_int_peak, run live),
    else the committed measurement (MEASURED_INT_PEAKS.json)."""
    try:
        from paper_1208_0274_gb300 import ae
        iadd = max(ae.ae_int_peak(ae.AE_PEAK_IADD, 4, 1024, 16)[1] for _ in range(2))
        imax = max(ae.ae_int_peak(ae.AE_PEAK_IMAX, 4, 1024, 16)[1] for _ in range(2))
        return {"iadd": iadd, "imax": imax, "source": "measured live (ae_int_peak)"}
    except Exception:
        d = json.load(open(os.path.join(ROOT, "MEASURED_INT_PEAKS.json")))
        return {"iadd": d["iadd_s32_inst_per_s"], "imax": d["imax_s32_inst_per_s"],
                "source": "MEASURED_INT_PEAKS.json"}


def cpu_info():
    """(threads this process may use, CPU model string)."""
    import oracle
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return oracle.host_threads(), f"{model or platform.processor() or 'unknown'} ({platform.machine()})"


def cpu_baseline(text, queries, scheme, H, seconds, alphabet=b"ACGT"):
    """The oracle (plain full-matrix Smith-Waterman) on every host core, on a
    bounded sample: the shortest query against a text slice sized for about
    `seconds` of work."""
    import oracle
    threads, model = cpu_info()
    q = min(queries, key=lambda x: x.size)[: 10_000]
    h = H[int(np.argmin([x.size for x in queries]))]
    probe = text[: max(1, 200_000_000 // max(q.size, 1))]
    t0 = time.perf_counter()
    oracle.sw_hits_mt(probe, q, scheme, h, alphabet=alphabet, threads=threads)
    rate = probe.size * q.size / max(time.perf_counter() - t0, 1e-6)
    L = int(min(text.size, max(1000, rate * seconds / q.size)))
    t0 = time.perf_counter()
    oracle.sw_hits_mt(text[:L], q, scheme, h, alphabet=alphabet, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": round(L * q.size / dt / 1e9, 4), "unit": "GCUPS", "cores": threads, "kind": "oracle",
            "cpu": model,
            "sample": f"one {q.size} bp query against the first {L:,} bp of the text "
                      f"({L * q.size:.3g} cells, {dt:.1f} s, {threads} threads)"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    name, text, queries, H, scheme, desc = make_workload(args)
    import oracle
    oracle.build()
    threads, model = cpu_info()
    q = min(queries, key=lambda x: x.size)[: 10_000]
    h = H[int(np.argmin([x.size for x in queries]))]
    # size one step at ~5 s of oracle work on every core
    alphabet = PROTEIN if name == "protein" else b"ACGT"
    probe = text[: max(1, 200_000_000 // max(q.size, 1))]
    t0 = time.perf_counter()
    oracle.sw_hits_mt(probe, q, scheme, h, alphabet=alphabet, threads=threads)
    rate = probe.size * q.size / max(time.perf_counter() - t0, 1e-6)
    L = int(min(text.size, max(1000, rate * 5.0 / q.size)))
    for _ in range(max(args.warmup, 0)):
        oracle.sw_hits_mt(text[: L // 10], q, scheme, h, alphabet=alphabet, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sw_hits_mt(text[:L], q, scheme, h, alphabet=alphabet, threads=threads)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    v = args.steps * L * q.size / tot / 1e9
    sample = f"each step: one {q.size} bp query against the first {L:,} bp of the text, {threads} threads"
    line = {"metric": METRIC, "value": round(v, 4), "unit": "GCUPS", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * tot / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": desc,
            "cpu_baseline": {"value": round(v, 4), "unit": "GCUPS", "cores": threads, "kind": "oracle",
                             "cpu": model, "sample": sample},
            "e2e": {"value": round(v, 4), "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1208_0274_gb300 import ae

    name, text, queries, H, scheme, desc = make_workload(args)
    mine = shard(len(queries), rank, ws)
    qs = [queries[k] for k in mine]
    hs = [H[k] for k in mine]
    t0 = time.perf_counter()
    idx = ae.ae_index_build(text, ae.AE_PROTEIN if name == "protein" else ae.AE_DNA)
    t_index = time.perf_counter() - t0
    log(f"[rank {rank}] index of {text.size:,} letters built in {t_index:.2f} s")
    n = text.size
    stream = torch.cuda.Stream()
    # one search over all queries: 2 M query letters per engine batch (fewer batches, fewer
    # sweep tails; ~172 GB of workspace on the 100 Mbp workload, within the device's memory)
    batch_columns = args.batch_columns if args.batch_columns is not None else (1 << 21)
    # single-occurrence nodes stay in the trie walk for 10 levels on the 100 Mbp workload
    # (measured per step: 6 → 2.53 s, 8 → 2.30 s, 10 → 2.24 s, 12 → 2.46 s, 14 → 2.49 s)
    leaf_delay = args.leaf_delay if args.leaf_delay is not None else (10 if args.workload == "dna_scale" else None)
    opts = ae.make_options(leaf_segment=args.leaf_segment, item_columns=args.item_columns,
                           batch_columns=batch_columns, leaf_delay=leaf_delay, profile=1)
    opts_e2e = ae.make_options(leaf_segment=args.leaf_segment, item_columns=args.item_columns,
                               batch_columns=batch_columns, leaf_delay=leaf_delay)
    desc["batch_columns"] = batch_columns
    desc["leaf_delay"] = int(opts.leaf_delay)
    seq = np.concatenate(qs) if qs else np.zeros(0, np.uint8)
    offsets = np.concatenate([[0], np.cumsum([q.size for q in qs])]).astype(np.int64)
    d_seq = torch.from_numpy(seq).to(f"cuda:{local}")
    cap = 1 << 20
    d_hits = torch.empty(cap * 16, dtype=torch.uint8, device=f"cuda:{local}")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=f"cuda:{local}")

    def step():
        nonlocal cap, d_hits
        while True:
            st, counts = ae.ae_search_device(idx, d_seq.data_ptr(), offsets, scheme, hs, d_hits.data_ptr(), cap,
                                             options=opts, stream=stream)
            if st == ae.AE_OK:
                return counts
            cap = int(counts.sum() * 1.25) + 1024
            d_hits = torch.empty(cap * 16, dtype=torch.uint8, device=f"cuda:{local}")

    cells = sum(q.size for q in qs) * n
    for w in range(args.warmup):
        t1 = time.perf_counter()
        counts = step()
        st = ae.ae_last_stats()
        log(f"[rank {rank}] warmup {w}: {time.perf_counter() - t1:.3f} s, hits {int(counts.sum())}, "
            f"entries {st['entries']:,} (leaf {st['entries_leaf']:,}), nodes {st['nodes']:,}, "
            f"k_rows {st['ms_k_rows']:.1f} ms, k_children {st['ms_k_expand']:.1f} ms, k_leaf {st['ms_k_leaf']:.1f} ms, "
            f"k_sort {st['ms_k_sort']:.1f} ms, k_other {st['ms_k_other']:.1f} ms, launches {st['launches']}, "
            f"leaf rows {st['leaf_rows']:,} max steps {st['leaf_max_steps']:,} max width {st['leaf_max_width']:,}, "
            f"injections {st['injections']:,}, levels {st['levels']}, triples {st['triples']:,}, "
            f"ws {st['ws_bytes'] / 1e9:.1f} GB")

    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = []
    kstats = {"ms_k_expand": 0.0, "ms_k_rows": 0.0, "ms_k_leaf": 0.0, "ms_k_sort": 0.0, "ms_k_other": 0.0,
              "launches": 0, "levels": 0, "triples": 0, "leaf_sweeps": 0,
              "entries": 0, "entries_leaf": 0, "nodes": 0, "hits": 0, "raw_hits": 0}
    for s in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(s & 0xFF)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
        counts = step()
        with torch.cuda.stream(stream):
            b.record(stream)
        ev.append((a, b))
        st = ae.ae_last_stats()
        for k in kstats:
            kstats[k] += st[k]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms, cells_all = job_totals(sum(step_ms), cells, dist, device=f"cuda:{local}")
    value = args.steps * cells_all / (tot_ms / 1000.0) / 1e9
    qps = args.steps * (len(queries) if ws > 1 else len(qs)) / (tot_ms / 1000.0)

    # plain: one launch sequence per query (the static single-query form)
    plain = None
    if not args.no_plain and rank == 0:
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.fill_(7)
            a.record(stream)
        for k, q in enumerate(qs):
            off1 = np.array([0, q.size], dtype=np.int64)
            dq = d_seq[offsets[k]:offsets[k + 1]]
            st_, c_ = ae.ae_search_device(idx, dq.data_ptr(), off1, scheme, [hs[k]], d_hits.data_ptr(), cap,
                                          stream=stream)
        with torch.cuda.stream(stream):
            b.record(stream)
        torch.cuda.synchronize()
        pms = a.elapsed_time(b)
        plain = {"value": round(cells / (pms / 1000.0) / 1e9, 3), "unit": "GCUPS", "ms_per_step": round(pms, 3),
                 "queries_per_s": round(len(qs) / (pms / 1000.0), 3)}

    # e2e: host queries in, host results out, through ae_search
    e2e = None
    if not args.no_e2e:
        hbytes = 0
        t_e = []
        for s in range(max(1, args.steps)):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            hits, counts = ae.ae_search(idx, qs, scheme, hs, options=opts_e2e, stream=stream)
            t_e.append(time.perf_counter() - t1)
            hbytes = hits.nbytes + counts.nbytes
        et, _ = job_totals(sum(t_e) / len(t_e), 0, dist, device=f"cuda:{local}")
        e2e = {"value": round(cells_all / et / 1e9, 3), "unit": "GCUPS",
               "h2d_bytes_per_step": int(seq.nbytes), "d2h_bytes_per_step": int(hbytes),
               "ms_per_step": round(et * 1000, 3)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel (device time from CUDA events recorded by
    # the library on the search stream around each launch, during the timed steps)
    groups = {"k_rows": kstats["ms_k_rows"], "k_leaf": kstats["ms_k_leaf"],
              "k_children": kstats["ms_k_expand"], "k_sort": kstats["ms_k_sort"], "k_other": kstats["ms_k_other"]}
    dom = max(groups, key=groups.get)
    peak, src = peaks()
    ent_leaf = kstats["entries_leaf"]
    ent_trie = kstats["entries"] - ent_leaf
    # The row update's roofline is HBM: 20 algorithmic bytes against 6 integer
    # operations per DP entry (0.3 op/B, far below the GPU's ~5.5 op/B balance).
    sec = groups[dom] / 1000.0
    # one launch per trie level (DNA route; a level run again at exact sizes adds one)
    launches_dom = {"k_rows": max(1, kstats["levels"]), "k_leaf": max(1, kstats["leaf_sweeps"])}.get(dom, 1)
    ent = {"k_rows": ent_trie, "k_leaf": ent_leaf}.get(dom, kstats["raw_hits"])
    gbs = BYTES_PER_ENTRY * ent / sec / 1e9 if sec > 0 else 0.0
    traffic = measured_traffic(dom, ent)
    roof = {"kernel": dom, "bound": "hbm", "achieved": round(gbs, 2), "peak": peak, "unit": "GB/s",
            "frac": round(gbs / peak, 4), "traffic": None if traffic is None else int(traffic / launches_dom),
            "peak_source": f"{src} (copy bandwidth, MEASURED_PEAKS.json)",
            "algorithmic_bytes_per_unit": BYTES_PER_ENTRY, "unit_of_work": "DP entry",
            "units_per_launch": int(ent / launches_dom),
            "group_ms_per_step": {k: round(v / args.steps, 3) for k, v in groups.items()}}
    # integer view: 6 ops per DP entry (and 12 per triple) against the measured int32 add rate
    ip = int_peaks()
    ops_e = OPS_PER_ENTRY * ent / sec / 1e9 if sec > 0 else 0.0
    units_t = {"k_rows": kstats["triples"], "k_leaf": ent_leaf}.get(dom, 0)
    ops_t = OPS_PER_TRIPLE * units_t / sec / 1e9 if sec > 0 else 0.0
    roof_alu = {"kernel": dom, "bound": "alu", "achieved": round(ops_e, 2), "peak": round(ip["iadd"] / 1e9, 1),
                "unit": "Gop/s", "frac": round(ops_e / (ip["iadd"] / 1e9), 5), "ops_per_unit": OPS_PER_ENTRY,
                "unit_of_work": "DP entry", "peak_source": f"int32 add rate, {ip['source']}",
                "imax_peak_ginst": round(ip["imax"] / 1e9, 1),
                "per_triple": {"achieved": round(ops_t, 2), "ops_per_unit": OPS_PER_TRIPLE,
                               "frac": round(ops_t / (ip["iadd"] / 1e9), 5), "triples": int(units_t)}}
    cpu = None
    if not args.no_cpu:
        import oracle
        oracle.build()
        cpu = cpu_baseline(text, queries, scheme, H, args.cpu_seconds,
                           alphabet=PROTEIN if name == "protein" else b"ACGT")
    line = {"metric": METRIC, "value": round(value, 3), "unit": "GCUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(tot_ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": desc,
            "queries_per_s": round(qps, 3), "hits_per_step": int(kstats["hits"] / max(args.steps, 1)),
            "entries_per_step": int(kstats["entries"] / max(args.steps, 1)),
            "gpu_launches": int(kstats["launches"]), "plain": plain, "e2e": e2e, "roofline": roof,
            "roofline_alu": roof_alu,
            "cpu_baseline": cpu, "clocks": clk,
            "index_build_s": round(t_index, 3)}
    print(json.dumps(line), flush=True)
    idx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_serve(args):
    """Request loop: Poisson arrivals of DNA queries (70% of 200 bp-2 kbp, 30%
    of 2-100 kbp, log-uniform) against the resident 100 Mbp index.  The same
    arrivals are served (1) by the learned policy: concurrent slots, requests
    of least predicted work first within a work budget, predicted hit records
    as buffer hints, admission by predicted device memory; (2) by FIFO
    continuous batching (columns budget, admission by a per-letter memory
    bound); (3) one query at a time.  Reports queries/s and p50/p99 latency of
    each; the hits of every request must be identical across the three."""
    import torch
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    from paper_1208_0274_gb300 import ae, serve
    from paper_1208_0274_gb300.predictor import WorkPredictor
    text = dna_scale_text(n=args.n)
    wl = dna_serve(text, k=args.requests, rate=args.rate)
    scheme = wl.scheme
    idx = ae.ae_index_build(text, ae.AE_DNA)

    def fresh():
        return [serve.Request(rid=k, query=q, H=int(h), arrival=float(a))
                for k, (q, h, a) in enumerate(zip(wl.queries, wl.H, wl.arrivals))]

    # predictor: trained on searches of other queries of the same mix, logged alone
    t0 = time.perf_counter()
    tw = dna_serve(text, seed=20120806, k=args.train_queries, rate=args.rate)
    pred = WorkPredictor(idx, scheme, seed=1)
    T = pred.log_searches(tw.queries, tw.H)
    X = pred.features(tw.queries)
    loss = pred.fit(X, T)
    t_train = time.perf_counter() - t0
    warm = sorted(wl.queries, key=lambda q: -q.size)[:8]

    def serve_once(**kw):
        srv = serve.Server(idx, scheme, nslots=args.slots, **kw)
        srv.warmup(warm, [21] * len(warm))
        srv.leaf_sweeps, srv.batches_run = 0, 0
        clocks = Clocks(local)
        clocks.start()
        rep = srv.run(fresh())
        clk = clocks.stop()
        out = {"queries_per_s": round(rep.qps, 3), "p50_ms": round(rep.p50_ms, 3), "p99_ms": round(rep.p99_ms, 3),
               "wall_s": round(rep.wall, 3), "batches": rep.batches, "mean_batch": round(rep.mean_batch, 3),
               "peak_concurrency": rep.peak_concurrency, "admission_waits": srv.admission_waits,
               "leaf_sweeps": srv.leaf_sweeps}
        for st in srv.streams:
            ae.ae_workspace_release(idx, st)
        return rep, out, clk

    rep_l, learned, clk = serve_once(predictor=pred, work_budget=args.work_budget)
    rep_f, fifo, _ = serve_once()
    base_st = torch.cuda.Stream()
    ae.ae_search(idx, warm, scheme, [21] * len(warm), stream=base_st)
    base = serve.one_at_a_time(idx, scheme, fresh(), stream=base_st)
    ref = {r.rid: r.hits for r in base.requests}
    same = all(np.array_equal(ref[r.rid], r.hits) for r in rep_l.requests) and \
        all(np.array_equal(ref[r.rid], r.hits) for r in rep_f.requests)
    sum_m = int(sum(q.size for q in wl.queries))
    line = {"metric": "queries/s and p50/p99 latency (ms) under Poisson arrivals, continuous batching",
            "value": learned["queries_per_s"], "unit": "queries/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": round(rep_l.wall * 1000, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"dna_serve: {args.requests} requests, Poisson {args.rate:g}/s, DNA queries "
                                   f"200 bp-100 kbp (70% under 2 kbp, log-uniform) vs {args.n:,} bp index",
                       "slots": args.slots, "sum_m": sum_m, "work_budget": args.work_budget},
            "p50_ms": learned["p50_ms"], "p99_ms": learned["p99_ms"],
            "effective_gcups": round(sum_m * text.size / rep_l.wall / 1e9, 3),
            "learned": learned, "fifo": fifo,
            "one_at_a_time": {"queries_per_s": round(base.qps, 3), "p50_ms": round(base.p50_ms, 3),
                              "p99_ms": round(base.p99_ms, 3), "wall_s": round(base.wall, 3)},
            "predictor": {"train_queries": args.train_queries, "train_s": round(t_train, 3),
                          "final_loss": round(float(loss), 5),
                          "bytes_per_entry": round(pred.bytes_per_entry, 3), "fixed_bytes": int(pred.fixed_bytes),
                          "hit_margin": round(pred.hit_margin, 3)},
            "hits_identical": bool(same), "hits": int(sum(h.size for h in ref.values())),
            "clocks": clk}
    print(json.dumps(line), flush=True)
    idx.close()
    return 0 if same else 1


def run_batch(args):
    """Many queries of uneven length (log-uniform 100-20,000 bp, 1% planted)
    against the resident 100 Mbp index.  A step is one search of all queries:
    the autotuned configuration (engine batch size, leaf delay, streams) with
    the queries packed onto the streams by predicted work (LPT).  Also timed:
    the same configuration with static round-robin packing, and single-query
    launches on a sample (queries/s)."""
    import torch
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    from paper_1208_0274_gb300 import ae, autotune
    from paper_1208_0274_gb300.batch import search_many
    from paper_1208_0274_gb300.predictor import WorkPredictor
    text = dna_scale_text(n=args.n)
    wl = dna_batch(text, k=args.queries)
    qs, Hs, scheme = wl.queries, wl.H, wl.scheme
    idx = ae.ae_index_build(text, ae.AE_DNA)
    sum_m = int(sum(q.size for q in qs))
    cells = sum_m * text.size

    t0 = time.perf_counter()
    tw = dna_batch(text, seed=20120807, k=args.train_queries)
    pred = WorkPredictor(idx, scheme, seed=1)
    T = pred.log_searches(tw.queries, tw.H)
    pred.fit(pred.features(tw.queries), T)
    t_train = time.perf_counter() - t0
    t0 = time.perf_counter()
    cfg, cached = autotune.tune(idx, qs, Hs, scheme, sample=512)
    t_tune = time.perf_counter() - t0
    log(f"tuned {cfg} (cached {cached}) in {t_tune:.1f} s; predictor trained in {t_train:.1f} s")
    opts = {"batch_columns": cfg["batch_columns"], "leaf_delay": cfg["leaf_delay"]}
    streams = [torch.cuda.Stream() for _ in range(cfg["nstreams"])]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def step(policy):
        flush.fill_(1)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        out, info = search_many(idx, qs, Hs, scheme, nstreams=cfg["nstreams"], policy=policy, predictor=pred,
                                options=opts, streams=streams)
        torch.cuda.synchronize()
        return time.perf_counter() - t1, out, info

    for _ in range(args.warmup):
        step("lpt")
    clocks = Clocks(local)
    clocks.start()
    times, info = [], None
    for _ in range(args.steps):
        dt, out_l, info = step("lpt")
        times.append(dt)
    clk = clocks.stop()
    rr_times = []
    for _ in range(max(1, args.steps)):
        dt, out_r, info_r = step("round_robin")
        rr_times.append(dt)
    same = all(np.array_equal(a, b) for a, b in zip(out_l, out_r))
    # the two packings at three streams (the autotuner's choice may be fewer)
    multi = {}
    streams3 = [torch.cuda.Stream() for _ in range(3)]
    for policy in ("lpt", "round_robin"):
        flush.fill_(2)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        out_m, info_m = search_many(idx, qs, Hs, scheme, nstreams=3, policy=policy, predictor=pred,
                                    options=opts, streams=streams3)
        torch.cuda.synchronize()
        multi[policy] = {"ms_per_step": round(1000 * (time.perf_counter() - t1), 3), "groups": info_m["groups"]}
        same &= all(np.array_equal(a, b) for a, b in zip(out_l, out_m))
    for st_ in streams3:
        ae.ae_workspace_release(idx, st_)
    # single-query launches on a sample (the static plain form)
    rng = np.random.default_rng(3)
    pick = rng.choice(len(qs), size=min(args.plain_sample, len(qs)), replace=False)
    st = torch.cuda.Stream()
    ae.ae_search(idx, [qs[pick[0]]], scheme, [Hs[pick[0]]], stream=st)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    plain_same = True
    for k in pick:
        h, _ = ae.ae_search(idx, [qs[k]], scheme, [Hs[k]], stream=st)
        plain_same &= bool(np.array_equal(h, out_l[k]))
    t_plain = time.perf_counter() - t1
    m_plain = int(sum(qs[k].size for k in pick))
    ms = 1000 * sum(times) / len(times)
    line = {"metric": "effective GCUPS (m*n/time) and queries/s, batched + learned packing vs static",
            "value": round(cells / (ms / 1000) / 1e9, 3), "unit": "GCUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"dna_batch: {len(qs)} DNA queries, lengths log-uniform 100-20,000 bp (1% planted), "
                                   f"vs {args.n:,} bp index; H by length (E=10)",
                       "sum_m": sum_m, "tuned": cfg, "tune_cached": cached,
                       "l2": "flushed between timed steps (512 MiB write)"},
            "queries_per_s": round(len(qs) / (ms / 1000), 3),
            "round_robin": {"ms_per_step": round(1000 * sum(rr_times) / len(rr_times), 3),
                            "value": round(cells / (sum(rr_times) / len(rr_times)) / 1e9, 3),
                            "groups": info_r["groups"]},
            "lpt_groups": info["groups"], "leaf_sweeps": info["leaf_sweeps"], "gpu_launches": info["launches"],
            "three_streams": multi,
            "single_query": {"queries": len(pick), "queries_per_s": round(len(pick) / t_plain, 3),
                             "value": round(m_plain * text.size / t_plain / 1e9, 3), "unit": "GCUPS"},
            "predictor_train_s": round(t_train, 3), "tune_s": round(t_tune, 3),
            "hits_identical": bool(same and plain_same), "hits": int(sum(h.size for h in out_l)), "clocks": clk}
    print(json.dumps(line), flush=True)
    idx.close()
    return 0 if (same and plain_same) else 1


def run_sweep(args):
    """The paper's sensitivity experiments on the scaled DNA workload: the scheme
    sweep (Section 7.4, Fig. 9 / Table 5: four BLAST schemes, E = 10, 8 queries
    of 100 kbp) and the E-value sweep (Section 7.3, Fig. 8: E = 1e-15, 1e-5, 10
    under <1,-3,-5,-2>, 8 queries each of 10 kbp and 100 kbp), against the
    10^8-letter text.  Each point is timed with CUDA events (median of `steps`
    searches after one warm-up) and counted once more with tier_stats for the
    filtering and reuse figures (Eq. 5, Eq. 6)."""
    import torch
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    from paper_1208_0274_gb300 import ae
    from workloads import SWEEP_H
    t0 = time.perf_counter()
    text, q100, _, _ = dna_scale_bench(n=args.n, lengths=[100_000], per_length=args.per_length)
    _, q10, _, _ = dna_scale_bench(n=args.n, lengths=[10_000], per_length=args.per_length)
    idx = ae.ae_index_build(text, ae.AE_DNA)
    log(f"index built in {time.perf_counter() - t0:.1f} s")
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    batch_columns = args.batch_columns if args.batch_columns is not None else (1 << 19)

    def point(scheme_t, E, qs, m):
        scheme = Scheme(*scheme_t)
        H = [SWEEP_H[scheme_t][E][m]] * len(qs)
        opts = ae.make_options(batch_columns=batch_columns)
        ae.ae_search(idx, qs, scheme, H, options=opts, stream=stream)   # warm-up
        times = []
        for _ in range(max(1, args.steps)):
            with torch.cuda.stream(stream):
                flush.fill_(1)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            hits, counts = ae.ae_search(idx, qs, scheme, H, options=opts, stream=stream)
            with torch.cuda.stream(stream):
                b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        st = ae.ae_last_stats()
        ae.ae_search(idx, qs, scheme, H, options=ae.make_options(batch_columns=batch_columns, tier_stats=1),
                     stream=stream)
        ts = ae.ae_last_stats()
        ms = statistics.median(times)
        cells = sum(q.size for q in qs) * text.size
        cand = max(ts["candidates"], 1)
        row = {"scheme": list(scheme_t), "E": E, "m": m, "queries": len(qs), "H": H[0], "ms": round(ms, 3),
               "gcups": round(cells / (ms / 1000) / 1e9, 1), "hits": int(hits.size), "entries": int(st["entries"]),
               "seed_depth": int(st["seed_depth"]),
               "filtering_ratio": round((ts["pruned_nonpos"] + ts["pruned_reach"]) / cand, 4),
               "reused": int(st["reused"]), "accessed": int(st["reused"] + st["entries"]),
               "reusing_ratio": round(st["reused"] / max(st["reused"] + st["entries"], 1), 5),
               "dominated": int(st["dominated"])}
        log(json.dumps(row))
        return row

    clocks = Clocks(local)
    clocks.start()
    schemes = [point(sc, 10.0, q100, 100_000) for sc in SWEEP_H]
    evalues = [point((1, -3, -5, -2), E, qs, m) for E in (1e-15, 1e-5, 10.0)
               for qs, m in ((q10, 10_000), (q100, 100_000))]
    clk = clocks.stop()
    base = schemes[0]["ms"]
    line = {"metric": "effective GCUPS (m*n/time) across scoring schemes and E-values", "value": schemes[0]["gcups"],
            "unit": "GCUPS", "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": base,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"sweep: {args.n:,} bp i.i.d. text at 41% GC; {args.per_length} queries each of "
                                   "10 kbp / 100 kbp with 1% planted; H from E per scheme (Gumbel fits)",
                       "batch_columns": batch_columns, "l2": "flushed between timed steps (512 MiB write)"},
            "schemes": schemes, "evalues": evalues,
            "entries_vs_default": {str(r["scheme"]): round(r["entries"] / max(schemes[0]["entries"], 1), 2)
                                   for r in schemes},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    idx.close()
    return 0


def main():
    args = parse()
    if args.workload == "dna_serve":
        return run_serve(args)
    if args.workload == "dna_batch":
        return run_batch(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
