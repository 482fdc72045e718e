#!/usr/bin/env python
"""Benchmark of the TCR-NET network-construction hot path on B300.

One step = one complete network build of the N = 800,000-string synthetic
repertoire (seed = rank) at l_max = 1 through the library's default method
(validate + encode, distinct-string collapse, deletion-neighbourhood join,
offsets, fill, per-row sort, int32 CSR export), with the inputs already in
device memory. `value` is candidate pairs resolved per second: the unordered
pairs whose lengths differ by at most l_max (same-length and +-1-length
buckets; every other pair is farther apart than l_max, since the distance is
at least the length difference), per build, summed over ranks (weak scaling:
every rank builds its own repertoire; there is no collective on the data
path). The deletion method never enumerates these pairs; the count is the work
an all-pairs method must resolve, so methods and the CPU baselines compare on
one unit.

The same JSON line also carries:
  all_pairs_per_s  N (N - 1) / 2 per build over the step time;
  edges_per_s      undirected edges produced per second;
  roofline         the dominant phase of the step against measured HBM bandwidth;
  roofline_step    the whole build's algorithmic bytes over the step time;
  peaks            the integer-issue microbenchmark (per-SM rates by instruction kind);
  tile             the all-pairs tile kernel (count pass) on the same workload:
                   candidate pair tests per second and its integer-issue roofline;
  query            p50/p99 latency of query batches against the resident
                   repertoire (host strings in, host neighbour lists out);
  e2e              the same metric through the public API from pinned host
                   buffers, including the upload and the read-back of the CSR;
  cpu_baseline     the CPU oracle (plain Wagner-Fischer) on a bounded row sample,
                   and the paper's own early-abort algorithm (all cores, one core).

`--impl reference` times the CPU oracle alone (there is no reference library
to install: the paper's code is not available) and prints the same metric.
`--legs cpu_full` (not run by default) times full oracle builds at 1e4 and 1e5
strings and 10,000-row samples at 8e5 for the baseline tables.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pair comparisons/s and edges/s at N=8e5 (frac of int/HBM roofline); query p50/p99"
UNIT = "pairs/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6400.0
SMS = 148
# Nominal integer issue ceiling per SM and clock: 4 schedulers x 1 warp-instruction x
# 32 lanes. The `peaks` leg measures the rates on the device (tcrnet_probe_int_issue:
# independent chains of logic, shift, add, multiply-add and popc instructions) and
# the tile roofline uses the measured ceiling when that leg runs.
INT_LANES_PER_SM = 128
# Minimal integer operations of the pair test on one 128-bit word pair (24 letters
# of 5-bit codes): same length 2 XOR + 2 field folds (3 three-input logic ops each)
# + 2 POPC + add + compare = 12; lengths L, L+1 about twice that plus the
# count-leading/trailing-zero steps = 26. Longer strings take one more word pair
# per 24 letters.
OPS_SAME_PER_WORD = 12
OPS_INDEL_PER_WORD = 26


# DRAM bytes (read + write) per build of the phase's kernels at N = 800,000,
# from one ncu capture of the current kernels (profiles/k_records_join_n800000.md,
# profiles/k_sort_fill_expand_n800000.md); absent where no capture covers the phase.
PHASE_TRAFFIC_N800000 = {
    "records": 23.824e6 + 3.853e6 + 89.421e6 + 74.904e6,              # count, partition scan, scatter
    "join": 79.972e6 + 4.089e6 + 1.242e6 + 0.019e6 + 0.015e6 + 32.100e6 + 0.040e6,  # windows, sorted, fallback, confirmation
    "list_sort": 25.039e6 + 27.430e6 + 14.242e6 + 0.350e6,            # the four sort classes
    "expand": 83.515e6 + 198.961e6,
}

LEGS = ("peaks", "tile", "query", "e2e", "insert", "analytics", "lmax2", "batched", "serving", "cpu")
EXTRA_LEGS = ("cpu_full", "n8e6")  # run only when named in --legs


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=800_000)
    ap.add_argument("--method", default="auto", choices=["auto", "deletion", "tile"])
    ap.add_argument("--tile-steps", type=int, default=2)
    ap.add_argument("--phase-steps", type=int, default=20,
                    help="profiled builds after the timed region, for the per-phase times")
    ap.add_argument("--query-batches", type=int, default=30)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="0 skips the serving leg")
    ap.add_argument("--serve-n", type=int, default=2_000_000)
    ap.add_argument("--insert-sizes", default="100,1000,10000,25000",
                    help="comma list of insert sizes of the insert leg")
    ap.add_argument("--batched-reps", type=int, default=256, help="0 skips the batched leg")
    ap.add_argument("--no-extras", action="store_true", help="skip every leg after the timed step")
    ap.add_argument("--legs", default=",".join(LEGS),
                    help="comma list of the legs run after the timed step (default: all but cpu_full)")
    return ap.parse_args()


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2032.0)), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, 2032.0, "fallback"


def workload(n, seed):
    from synthgen import generate_config2

    return generate_config2(n, seed=seed)


def workload_config(args, method):
    return {
        "workload": f"config 2: N={args.n} synthetic CDR3beta strings (V-insertion-J templates, "
                    f"insertion 0-6 aa, lengths 10-20, Zipf(1) background), l_max=1, int32 CSR",
        "n": args.n,
        "threshold": 1,
        "method": method,
        "seed": "rank",
        "inputs_resident": True,
        "l2": "flushed between timed steps (512 MB write)",
    }


# ---------------------------------------------------------------------------
# clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "25"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                mx.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# candidate pairs and the CPU legs

def candidate_pairs(lengths, threshold=1):
    """Unordered pairs whose lengths differ by at most `threshold`: the pairs an
    all-pairs method must resolve (any other pair has a larger distance)."""
    cnt = np.bincount(np.asarray(lengths, dtype=np.int64), minlength=64).astype(np.float64)
    total = float((cnt * (cnt - 1) / 2).sum())
    for d in range(1, threshold + 1):
        total += float((cnt[:-d] * cnt[d:]).sum())
    return total


def row_candidates(lengths, rows, threshold=1):
    """Candidate partners (other strings within `threshold` of its length) of each row."""
    lengths = np.asarray(lengths, dtype=np.int64)
    cnt = np.bincount(lengths, minlength=64)
    cum = np.concatenate([[0], np.cumsum(cnt)])
    L = lengths[rows]
    lo = np.clip(L - threshold, 0, 63)
    hi = np.clip(L + threshold + 1, 0, 64)
    return cum[hi] - cum[lo] - 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def sampled_rate(rep, seconds, fn, nthreads, seed=0, rows_per_call=None, min_calls=1):
    """Rows of the N-string network by `fn` (the oracle or the baseline) on seeded
    row samples for about `seconds`. Returns a dict with the rate in candidate
    pairs per second of a full build (elapsed time extrapolated from the rows
    done to all N rows; the build resolves candidate_pairs(lengths) pairs) and in
    all pairs per second."""
    import oracle

    cores = nthreads if nthreads > 0 else oracle.max_threads()
    rng = np.random.default_rng(seed)
    # eight rows per thread and call: row times vary, and with one row per
    # thread the threads idled at the end of every call (the sampled all-core
    # rates came out 2-4x below those of a 10,000-row call)
    per = rows_per_call or max(1, 8 * cores)
    lens = rep.lengths()
    cand_build = candidate_pairs(lens)
    done, calls, t0 = 0, 0, time.perf_counter()
    while True:
        rows = rng.choice(rep.n, size=per, replace=False).astype(np.int64)
        fn(rep.chars, rep.offsets, rows, max_dist=1, nthreads=cores)
        done += per
        calls += 1
        el = time.perf_counter() - t0
        if el >= seconds and calls >= min_calls:
            break
    build_s = el * rep.n / done  # extrapolated full build
    return {"value": cand_build / build_s, "unit": UNIT, "cores": cores, "rows": done, "elapsed_s": el,
            "extrapolated_build_s": build_s, "all_pairs_per_s": rep.n * (rep.n - 1) / 2 / build_s}


def oracle_rate(rep, seconds, seed=0, rows_per_call=None):
    """Oracle (plain Wagner-Fischer, all host cores) on sampled rows of the network."""
    import oracle

    return sampled_rate(rep, seconds, oracle.rows, 0, seed, rows_per_call)


def cpu_leg(rep, seconds):
    """cpu_baseline: the oracle as it stands on all host cores, plus the paper's
    own algorithm (the early-abort table with the length skip) on all cores and
    on one core, each on a bounded row sample of the same N-string network."""
    import oracle

    o = oracle_rate(rep, seconds)
    b_all = sampled_rate(rep, seconds / 2, oracle.baseline_rows, 0, seed=1)
    b_one = sampled_rate(rep, seconds / 2, oracle.baseline_rows, 1, seed=2)
    model = cpu_model()
    n = rep.n
    return {
        "value": o["value"], "unit": UNIT, "cores": o["cores"], "kind": "oracle", "cpu_model": model,
        "sample": f"{o['rows']} seeded rows of the N={n} network, each the full Wagner-Fischer scan against "
                  f"all {n} strings ({o['elapsed_s']:.1f} s); value = candidate pairs of one build over the "
                  f"build time extrapolated from the rows done ({o['extrapolated_build_s']:.0f} s)",
        "all_pairs_per_s": o["all_pairs_per_s"],
        "listing1": {
            "kind": "listing1", "value": b_all["value"], "unit": UNIT, "cores": b_all["cores"],
            "single_core": b_one["value"], "cpu_model": model,
            "extrapolated_build_s": b_all["extrapolated_build_s"],
            "single_core_extrapolated_build_s": b_one["extrapolated_build_s"],
            "sample": f"{b_all['rows']} rows on {b_all['cores']} cores ({b_all['elapsed_s']:.1f} s) and "
                      f"{b_one['rows']} rows on one core ({b_one['elapsed_s']:.1f} s) of the N={n} network",
            "algorithm": "the paper's per-pair test (Methods 'GPU-based network generation', Listing 1) "
                         "restated correctly: two-row table with the row-minimum early abort, pairs with "
                         "|length difference| > l_max skipped",
        },
    }


def cpu_full_leg():
    """Baseline tables: full oracle builds at 1e4 and 1e5 strings (all cores),
    10,000 seeded rows at 8e5 (extrapolated x80 to the full build), the same for
    the paper's early-abort algorithm, and that algorithm on one core (1,000 rows
    at 8e5, extrapolated x800)."""
    import oracle
    from synthgen import generate_config1, generate_config2

    out = {"cpu_model": cpu_model(), "cores": oracle.max_threads(), "runs": []}
    for n in (10_000, 100_000):
        rep = generate_config1(n, seed=0)
        cand = candidate_pairs(rep.lengths())
        for label, fn in (("oracle", oracle.network), ("listing1", oracle.baseline_network)):
            t = time.perf_counter()
            off, _, _ = fn(rep.chars, rep.offsets, max_dist=1)
            el = time.perf_counter() - t
            out["runs"].append({"run": f"{label}, full network", "n": n, "threads": out["cores"], "s": el,
                                "candidate_pairs_per_s": cand / el, "all_pairs_per_s": n * (n - 1) / 2 / el,
                                "nnz": int(off[-1])})
    rep = generate_config2(800_000, seed=0)
    cand = candidate_pairs(rep.lengths())
    n = rep.n
    rng = np.random.default_rng(3)
    for label, fn, rows, threads in (("oracle", oracle.rows, 10_000, 0),
                                     ("listing1", oracle.baseline_rows, 10_000, 0),
                                     ("listing1", oracle.baseline_rows, 1_000, 1)):
        ids = rng.choice(n, size=rows, replace=False).astype(np.int64)
        t = time.perf_counter()
        fn(rep.chars, rep.offsets, ids, max_dist=1, nthreads=threads)
        el = time.perf_counter() - t
        build_s = el * n / rows
        out["runs"].append({"run": f"{label}, {rows} seeded rows, extrapolated x{n // rows}", "n": n,
                            "threads": threads or out["cores"], "s": el, "extrapolated_build_s": build_s,
                            "candidate_pairs_per_s": cand / build_s, "all_pairs_per_s": n * (n - 1) / 2 / build_s})
    return out


def large_leg(tn, torch, dev, stream, flush, steps=5):
    """Config 3 (N = 8,000,000, insertion 0-9 aa, lengths 8-24, int64 CSR offsets):
    builds by the default method from device inputs, CUDA events, L2 flushed."""
    from synthgen import generate_config3

    rep = generate_config3(8_000_000, seed=0)
    chars = torch.from_numpy(rep.chars).to(dev)
    offs = torch.from_numpy(rep.offsets).to(dev)
    tn.tcrnet_build_flat(chars, offs, 1, stream=stream).free()
    ts, st = [], None
    for k in range(steps):
        flush.fill_(k & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g = tn.tcrnet_build_flat(chars, offs, 1, stream=stream)
        b.record(stream)
        b.synchronize()
        st = g.stats()
        g.free()
        ts.append(a.elapsed_time(b))
    g = tn.tcrnet_build_flat(chars, offs, 1, stream=stream, profile=True)
    ph = g.stats()["ms_phase"]
    g.free()
    ms = statistics.mean(ts)
    cand = candidate_pairs(rep.lengths())
    names = ["dedup", "records", "join", "join_fill", "unused", "list_sort", "expand"]
    return {"n": rep.n, "build_ms": ms, "build_ms_min": min(ts), "builds": steps, "nnz": st["nnz"],
            "distinct_strings": st["n_unique"], "records": st["n_records"], "fallback_partitions": st["n_fallback"],
            "candidate_pairs_per_s": cand / (ms / 1e3), "edges_per_s": st["nnz"] / 2 / (ms / 1e3),
            "edge_write_gbs": 4 * st["nnz"] / (ph[6] / 1e3) / 1e9 if ph[6] > 0 else None,
            "phases_ms": {nm: ph[i] for i, nm in enumerate(names) if nm != "unused"},
            "timing": f"CUDA events, mean of {steps} after 1 warm-up, L2 flushed; phases from one profiled build"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    rep = workload(args.n, 0)
    cores = oracle.max_threads()
    rng = np.random.default_rng(1)
    per = max(1, 4 * cores)  # four rows per thread per step (about 0.6 s; balanced across threads)
    cand_build = candidate_pairs(rep.lengths())

    def step():
        rows = rng.choice(rep.n, size=per, replace=False).astype(np.int64)
        oracle.rows(rep.chars, rep.offsets, rows, max_dist=1, nthreads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    build_s = el * rep.n / (args.steps * per)  # extrapolated full build
    value = cand_build / build_s
    sample = (f"{per} sampled rows per step (each row: the query string against all {rep.n} strings), "
              f"{args.steps} steps; value = candidate pairs of one build over the build time extrapolated "
              f"from the rows done ({build_s:.0f} s)")
    line = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
        "config": dict(workload_config(args, "cpu-oracle"), inputs_resident=False, l2="not applicable (host)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "all_pairs_per_s": rep.n * (rep.n - 1) / 2 / build_s,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# cross-rank aggregation (weak scaling: every rank builds its own repertoire)

def aggregate_ranks(ms_local, pairs_per_build, edges_per_build, world, dist_mod=None, device="cpu"):
    """Max step time over ranks and whole-job throughputs.

    value = world x pairs per build / max step time (all ranks' units over the
    slowest rank's time). With dist_mod (torch.distributed, any backend) the max
    is an all-reduce; without it the local time is used."""
    ms = float(ms_local)
    if dist_mod is not None and world > 1:
        import torch

        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * pairs_per_build / (ms / 1e3), world * edges_per_build / (ms / 1e3)


# ---------------------------------------------------------------------------
# ours

def tile_alg_ops(lengths, threshold=1):
    """Algorithmic integer operations of the all-pairs tile test over every
    candidate pair: OPS_SAME_PER_WORD per same-length pair and
    OPS_INDEL_PER_WORD per (L, L+1) pair, per 128-bit word pair of the longer
    string (24 letters each). Returns (ops, candidate pairs)."""
    cnt = np.bincount(np.asarray(lengths, dtype=np.int64), minlength=64).astype(np.float64)
    ops = 0.0
    pairs = 0.0
    for L in range(1, 49):
        nl = cnt[L]
        if nl == 0:
            continue
        words = math.ceil(L / 24)
        same = nl * (nl - 1) / 2
        ops += same * OPS_SAME_PER_WORD * words
        pairs += same
        if threshold >= 1 and cnt[L + 1] > 0:
            ind = nl * cnt[L + 1]
            ops += ind * OPS_INDEL_PER_WORD * math.ceil((L + 1) / 24)
            pairs += ind
    return ops, pairs


def peaks_leg(tn, torch, dev, stream, sms):
    """Integer-issue rates by instruction kind: each kind's microbenchmark kernel
    (2,048 threads per SM, independent chains) timed with CUDA events on the
    bench stream, median of 5 launches; rates per SM and clock at the SM clock
    sampled during the leg."""
    n_threads = sms * 2048
    out = torch.empty(n_threads, dtype=torch.int32, device=dev)
    iters = 4096
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    time.sleep(0.3)
    res = {}
    for kind in tn.PROBE_KINDS:
        tn.tcrnet_probe_int_issue(kind, 64, out, stream)  # warm-up
        ts = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ops = tn.tcrnet_probe_int_issue(kind, iters, out, stream)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts)
        res[kind] = {"ops_per_launch": float(ops) * n_threads, "ms": ms,
                     "tops": float(ops) * n_threads / (ms / 1e3) / 1e12}
    clocks = sampler.stop()
    clk = (clocks or {}).get("sm_mhz") or 2032.0
    for kind, r in res.items():
        r["lanes_per_clk_per_sm"] = r["tops"] * 1e12 / (sms * clk * 1e6)
    issue = max(r["tops"] for r in res.values())
    return {"kinds": res, "sms": sms, "sm_mhz": clk, "clocks": clocks,
            "issue_ceiling_tops": issue, "issue_ceiling_lanes_per_clk_per_sm": issue * 1e12 / (sms * clk * 1e6),
            "alu_pipe_tops": res["lop3"]["tops"],
            "method": "tcrnet_probe_int_issue: 8 independent rotating triples per thread, 4096 rounds, "
                      "CUDA events on the bench stream, median of 5"}


def serve_leg(args, tn, torch, stream):
    """Serving: resident repertoire of args.serve_n strings, open-loop Poisson
    arrivals (200/s) of queries (90%, log-uniform 1..50,000 strings) and inserts
    (10%, log-uniform 1,000..100,000 strings) for args.serve_seconds."""
    from paper_2112_06613_b300.serving import ServingEngine, latency_by_answer_size, latency_summary
    from synthgen import generate, generate_config2

    rng = np.random.default_rng(11)
    base = generate_config2(args.serve_n, seed=100)
    # queries and inserts are later draws of the same repertoire model
    qpool = generate(400_000, seed=101, template_seed=100, ins_max=6, len_lo=10, len_hi=20)
    ipool = generate(3_000_000, seed=102, template_seed=100, ins_max=6, len_lo=10, len_hi=20)
    rate = 200.0
    arrivals, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > args.serve_seconds:
            break
        if rng.random() < 0.1:
            arrivals.append((t, "insert", int(round(math.exp(rng.uniform(math.log(1e3), math.log(1e5)))))))
        else:
            arrivals.append((t, "query", int(round(math.exp(rng.uniform(0, math.log(5e4)))))))
    chars = torch.from_numpy(base.chars).to("cuda")
    offs = torch.from_numpy(base.offsets).to("cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = tn.tcrnet_build_flat(chars, offs, 1, stream=stream)
    torch.cuda.synchronize()
    plain_build_ms = 1e3 * (time.perf_counter() - t0)
    reqs = []
    ip = 0
    with ServingEngine(g, slots=4, max_batch_strings=200_000) as eng:
        start = time.perf_counter()
        for at, kind, size in arrivals:
            now = time.perf_counter() - start
            if at > now:
                time.sleep(at - now)
            if kind == "query":
                k0 = int(rng.integers(0, qpool.n - size))
                o = qpool.offsets[k0:k0 + size + 1]
                reqs.append(eng.query(qpool.chars[o[0]:o[-1]], o - o[0]))
            else:
                size = min(size, ipool.n - ip)
                o = ipool.offsets[ip:ip + size + 1]
                reqs.append(eng.insert(ipool.chars[o[0]:o[-1]], o - o[0]))
                ip += size
        for r in reqs:
            r.done.wait()
        wall = time.perf_counter() - start
    n_final, nnz_final, _ = g.info()
    g.free()
    errors = sum(r.error is not None for r in reqs)
    qs = [r for r in reqs if r.kind == "query"]
    return {
        "resident_strings_start": args.serve_n, "resident_strings_end": n_final, "nnz_end": nnz_final,
        "arrival_rate_per_s": rate, "duration_s": args.serve_seconds, "wall_s": wall,
        "requests": len(reqs), "errors": errors,
        "query": latency_summary(reqs, "query"), "insert": latency_summary(reqs, "insert"),
        "query_by_answer_size": latency_by_answer_size(reqs),
        "query_time_split": {
            "mean_queue_ms": float(np.mean([1e3 * (r.t_start - r.t_arrival) for r in qs])) if qs else None,
            "mean_call_ms": float(np.mean([1e3 * r.s_call for r in qs])) if qs else None,
            "mean_copy_ms": float(np.mean([1e3 * r.s_copy for r in qs])) if qs else None,
            "mean_split_ms": float(np.mean([1e3 * r.s_split for r in qs])) if qs else None,
            "note": "per query request: waiting for a slot, the device call (with its stream sync), the copy "
                    "of the shared batch answer to pinned host memory, the split into per-request arrays"},
        "throughput_requests_per_s": len(reqs) / wall,
        "query_strings_per_s": sum(r.n_strings for r in qs) / wall,
        "device_calls": len({r.batch_id for r in reqs}),
        "plain_build_ms_at_start": plain_build_ms,
        "engine": "4 slots (streams), queued queries merged up to 200,000 strings per call, inserts copy-on-write on low-priority streams, "
                  "admission by free HBM",
    }


def batched_leg(args, tn, torch, stream, flush, reps_steps=3):
    """Repertoires with log-uniform sizes in [1e3, 2e5]: one batched build of all of
    them against one plain build per repertoire (device inputs, CUDA events)."""
    from synthgen import generate_batched

    reps = generate_batched(args.batched_reps, seed=0)
    sizes = np.array([r.n for r in reps], dtype=np.int64)
    bounds = np.zeros(len(reps) + 1, dtype=np.int64)
    np.cumsum(sizes, out=bounds[1:])
    chars = np.concatenate([r.chars for r in reps])
    lens = np.concatenate([np.diff(r.offsets) for r in reps])
    offs = np.zeros(lens.shape[0] + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    dev = torch.device("cuda", torch.cuda.current_device())
    dc, do = torch.from_numpy(chars).to(dev), torch.from_numpy(offs).to(dev)
    per = [(torch.from_numpy(r.chars).to(dev), torch.from_numpy(r.offsets).to(dev)) for r in reps]
    pairs = float((sizes * (sizes - 1) // 2).sum())

    def timed(fn):
        out = []
        for k in range(reps_steps + 1):
            flush.fill_(3)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            extra = fn()
            b.record(stream)
            b.synchronize()
            if k > 0:
                out.append((a.elapsed_time(b), extra))
        return out

    from paper_2112_06613_b300.autotune import PartitionTuner

    tuner = PartitionTuner(trials=1)
    target = tuner.tune(dc, do, rep_offsets=bounds, stream=stream)  # untimed

    def batched():
        g = tn.tcrnet_build_batched(dc, do, bounds, 1, stream=stream, profile=False, partition_target=target)
        st = g.stats()
        g.free()
        return st

    def sequential():
        nnz, launches = 0, 0
        for c, o in per:
            g = tn.tcrnet_build_flat(c, o, 1, stream=stream)
            st = g.stats()
            nnz += st["nnz"]
            launches += st["kernel_launches"]
            g.free()
        return {"nnz": nnz, "kernel_launches": launches}

    tb = timed(batched)
    ts = timed(sequential)
    mb = statistics.mean(t for t, _ in tb)
    ms = statistics.mean(t for t, _ in ts)
    assert tb[0][1]["nnz"] == ts[0][1]["nnz"]
    return {"repertoires": len(reps), "strings": int(sizes.sum()), "size_range": "log-uniform [1e3, 2e5]",
            "pairs": pairs, "nnz": int(tb[0][1]["nnz"]),
            "batched_ms": mb, "batched_pairs_per_s": pairs / (mb / 1e3),
            "batched_kernel_launches": int(tb[0][1]["kernel_launches"]),
            "sequential_ms": ms, "sequential_pairs_per_s": pairs / (ms / 1e3),
            "sequential_kernel_launches": int(ts[0][1]["kernel_launches"]),
            "speedup": ms / mb, "timing": f"CUDA events, mean of {reps_steps} after 1 warm-up, L2 flushed",
            "partition_target": target, "autotune_ms": {str(k): v for k, v in tuner.last_timings.items()},
            "autotune": "records per partition chosen by timing the candidates once on this input (untimed)"}


def _components_device(g, keep_dev, tn):
    """tcrnet_components with a device-resident removal mask; labels stay on the device."""
    import ctypes

    nc, lc = ctypes.c_int64(), ctypes.c_int64()
    st = tn.load_library().tcrnet_components(g.handle, keep_dev.data_ptr(), None, tn.DEVICE, ctypes.byref(nc),
                                             ctypes.byref(lc))
    if st != tn.OK:
        raise tn.TcrnetError(st, "tcrnet_components")
    return None, nc.value, lc.value


def run_ours(args):
    import torch

    import paper_2112_06613_b300 as tn

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    hbm_peak, sm_max_nominal, peak_kind = load_peaks()

    rep = workload(args.n, rank)
    chars = torch.from_numpy(rep.chars).to(dev)
    offs = torch.from_numpy(rep.offsets).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def build(method=args.method, profile=True):
        return tn.tcrnet_build_flat(chars, offs, 1, method=method, stream=stream, profile=profile)

    # the clock sampler starts before the warm-up builds, so that it runs
    # through the timed region without an idle pause in front of it (a 0.3 s
    # sleep there let host and GPU fall into deeper idle states and made the
    # first ~150 timed builds up to 20% slower, measured)
    sampler = ClockSampler(local)
    sampler.start()
    warm = 0
    t_warm = time.perf_counter()
    # at least W builds, then more (untimed) until the sampler reports, so that
    # its samples cover the timed region even when that is short
    while warm < args.warmup or (sampler.proc is not None and not sampler.lines
                                 and time.perf_counter() - t_warm < 2.0):
        build().free()
        warm += 1
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        evs[k][0].record(stream)
        g = build(profile=False)
        evs[k][1].record(stream)
        stats.append(g.stats())
        g.free()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    st0 = stats[-1]
    n = args.n
    pairs_per_build = n * (n - 1) / 2
    cand_per_build = candidate_pairs(rep.lengths())
    edges = st0["nnz"] / 2
    ms, value, edges_per_s = aggregate_ranks(statistics.mean(step_ms), cand_per_build, edges, world, dist, dev)
    all_pairs_per_s = world * pairs_per_build / (ms / 1e3)
    launches = int(sum(s["kernel_launches"] for s in stats))
    # per-phase times: the same build with CUDA-event marks between its phases,
    # run after the timed region (the marks cost ~45 us per build, so the timed
    # builds run without them)
    pstats = []
    for k in range(max(args.phase_steps, 1)):
        flush.fill_(k & 0xff)
        g = build(profile=True)
        pstats.append(g.stats())
        g.free()
    torch.cuda.synchronize()

    is_tile = st0["method"] == 1
    # dominant phase of the step and its algorithmic bytes
    names = ["dedup", "records", "join", "join_fill", "unused", "list_sort", "expand"]
    phase_ms = {nm: statistics.mean(s["ms_phase"][i] for s in pstats) for i, nm in enumerate(names) if nm != "unused"}
    phase_ms["pack"] = statistics.mean(s["ms_pack"] for s in pstats)
    if is_tile:
        phase_ms = {"count_pass": statistics.mean(s["ms_count"] for s in pstats),
                    "write_pass": statistics.mean(s["ms_write"] for s in pstats),
                    "row_sort": statistics.mean(s["ms_sort"] for s in pstats)}
    dom = max(phase_ms, key=phase_ms.get)
    nnz = st0["nnz"]
    U, R, E, SD = st0["n_unique"], st0["n_records"], st0["unique_edges"], st0["closed_total"]
    # algorithmic bytes per phase (U distinct strings, R records, SD total
    # closed-list length): what each phase must read and write at least once
    phase_bytes = {} if is_tile else {
        "expand": 4 * nnz + 4 * SD + 8 * (n + 1) + 4 * n,  # write cols; read lists, offsets, ids
        "list_sort": 8 * SD + 8 * (U + 1),                # read + write lists, read offsets
        "join_fill": 8 * R + 8 * SD,                      # read records; read members, write lists
        "join": 8 * R,                                    # read records (candidates, confirmation)
        "records": 32 * U + 8 * R,                        # read strings, scatter records
        "dedup": 32 * n + 32 * U + 8 * n,                 # read codes, write distinct strings, ids
        "pack": int(rep.chars.nbytes) + 8 * (n + 1) + 33 * n,  # read chars + offsets; write codes + lengths
    }
    alg_bytes = phase_bytes.get(dom, 1)
    achieved = alg_bytes / (phase_ms[dom] / 1e3) / 1e9
    roofline_step = None
    if not is_tile:
        step_bytes = float(sum(phase_bytes.values()))
        sa = step_bytes / (ms / 1e3) / 1e9
        roofline_step = {"bound": "hbm", "achieved": sa, "peak": hbm_peak, "unit": "GB/s", "frac": sa / hbm_peak,
                         "alg_bytes_per_step": step_bytes, "ms_per_step": ms, "peak_kind": f"{peak_kind} hbm_gbs",
                         "formula": "sum over phases: pack chars+8(n+1)+33n; dedup 72n+32U; records 32U+8R; "
                                    "join 8R; fill 8R+8SD; list sort 8SD+8(U+1); expand 4nnz+4SD+8(n+1)+4n"}
    if is_tile:
        ops, _ = tile_alg_ops(rep.lengths())
        peak_ops = SMS * INT_LANES_PER_SM * sm_max_nominal * 1e6
        ach = ops / (phase_ms[dom] / 1e3)
        roofline_tile = {"bound": "alu", "kernel_phase": dom, "achieved": ach / 1e12, "peak": peak_ops / 1e12,
                         "unit": "Tops/s", "frac": ach / peak_ops, "traffic": None, "ms_per_launch": phase_ms[dom]}
    traffic = PHASE_TRAFFIC_N800000.get(dom) if (n == 800_000 and not is_tile) else None
    roofline = {"bound": "hbm", "kernel_phase": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic, "peak_kind": f"{peak_kind} hbm_gbs",
                "alg_bytes_per_launch": alg_bytes, "ms_per_launch": phase_ms[dom],
                "traffic_source": "ncu DRAM bytes of the phase's kernels, one capture (profiles/)" if traffic else None}
    if is_tile:
        roofline = roofline_tile
    # edge write: the CSR columns (4 B per directed entry) the expansion writes, over
    # the expansion phase, against the HBM peak
    edge_write = None
    if not is_tile and phase_ms.get("expand"):
        ew = 4 * nnz / (phase_ms["expand"] / 1e3) / 1e9
        edge_write = {"bound": "hbm", "kernel_phase": "expand", "achieved": ew, "peak": hbm_peak, "unit": "GB/s",
                      "frac": ew / hbm_peak, "bytes_per_launch": 4 * nnz, "ms_per_launch": phase_ms["expand"],
                      "traffic": PHASE_TRAFFIC_N800000.get("expand") if n == 800_000 else None}

    q = np.percentile(step_ms, [0, 10, 50, 90, 100])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "ms_per_step_distribution": {"min": float(q[0]), "p10": float(q[1]), "p50": float(q[2]), "p90": float(q[3]),
                                     "max": float(q[4]), "note": "this rank's CUDA-event step times; "
                                                                 "ms_per_step is their mean (max over ranks)"},
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(args, "deletion" if st0["method"] == 2 else "tile"),
        "candidate_pairs_per_build": cand_per_build, "all_pairs_per_s": all_pairs_per_s,
        "all_pairs_per_build": pairs_per_build,
        "edges_per_s": edges_per_s, "edges_per_build": edges, "nnz": nnz, "edge_write": edge_write,
        "wall_s_timed_region": wall, "phases_ms": phase_ms, "roofline": roofline, "roofline_step": roofline_step,
        "gpu_launches": launches, "clocks": clocks, "warmup_builds": warm,
    }

    legs = set(args.legs.split(",")) - {""}
    if rank == 0 and not args.no_extras:
        peaks = None
        if "peaks" in legs:
            try:
                # --- integer-issue rates of this device (the tile roofline's denominator)
                peaks = peaks_leg(tn, torch, dev, stream, torch.cuda.get_device_properties(dev).multi_processor_count)
                line["peaks"] = peaks
            except Exception as exc:  # keep the line: record the failed leg
                line.setdefault("leg_errors", {})["peaks"] = repr(exc)
        if "tile" in legs:
            try:
                # --- tile kernel: candidate pair tests per second vs the integer-issue roofline
                lens = rep.lengths()
                ops, pairs = tile_alg_ops(lens)
                tstats = []
                build(method="tile").free()
                for _ in range(args.tile_steps):
                    flush.fill_(1)
                    g = build(method="tile")
                    tstats.append(g.stats())
                    g.free()
                cnt_ms = statistics.mean(s["ms_count"] for s in tstats)
                tot_ms = statistics.mean(s["ms_total"] for s in tstats)
                cand = tstats[0]["candidate_pairs"]
                clk = (clocks or {}).get("sm_mhz") or sm_max_nominal
                nominal = SMS * INT_LANES_PER_SM * sm_max_nominal * 1e6
                ach_ops = ops / (cnt_ms / 1e3)
                if peaks:  # the measured issue ceiling of this device
                    peak_ops = peaks["issue_ceiling_tops"] * 1e12
                    basis = (f"measured by the peaks leg: fastest instruction mix, "
                             f"{peaks['issue_ceiling_lanes_per_clk_per_sm']:.1f} lanes/clk/SM at {peaks['sm_mhz']:.0f} MHz")
                else:
                    peak_ops = nominal
                    basis = f"nominal: {SMS} SMs x {INT_LANES_PER_SM} int32 issue lanes x {sm_max_nominal:.0f} MHz"
                line["tile"] = {
                    "candidate_pairs": cand, "count_pass_ms": cnt_ms, "build_ms": tot_ms,
                    "candidate_pairs_per_s": cand / (cnt_ms / 1e3),
                    "all_pairs_per_s_build": pairs_per_build / (tot_ms / 1e3),
                    "roofline": {"bound": "alu", "achieved": ach_ops / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                                 "frac": ach_ops / peak_ops, "frac_of_nominal_issue": ach_ops / nominal,
                                 "ops_per_launch": ops, "peak_basis": basis,
                                 "ops_basis": f"{OPS_SAME_PER_WORD} per same-length and {OPS_INDEL_PER_WORD} per "
                                              f"(L, L+1) candidate pair per 128-bit word pair (minimal test)",
                                 "sampled_sm_mhz": clk},
                }
            except Exception as exc:  # keep the line: record the failed leg
                line.setdefault("leg_errors", {})["tile"] = repr(exc)
        if "query" in legs:
            try:
                # --- queries against the resident repertoire (host in, host out)
                from synthgen import generate

                # queries drawn from the resident repertoire's model (same templates)
                qsrc = generate(200_000, seed=1000 + rank, template_seed=rank, ins_max=6, len_lo=10, len_hi=20)
                qstr_off = qsrc.offsets
                rng = np.random.default_rng(7)
                resident = build(profile=False)
                lat, qn = [], []
                for b in range(args.query_batches + 2):
                    m = int(round(math.exp(rng.uniform(0, math.log(50_000)))))
                    start = int(rng.integers(0, qsrc.n - m))
                    qo = (qstr_off[start:start + m + 1] - qstr_off[start]).astype(np.int64)
                    qc = qsrc.chars[qstr_off[start]:qstr_off[start + m]]
                    t = time.perf_counter()
                    r = resident.query_flat(qc, qo)
                    r.copy_csr()
                    dt = time.perf_counter() - t
                    r.free()
                    if b >= 2:
                        lat.append(dt * 1e3)
                        qn.append(m)
                resident.free()
                line["query"] = {"batches": len(lat), "batch_size": "log-uniform 1..50000", "p50_ms": float(np.percentile(lat, 50)),
                                 "p99_ms": float(np.percentile(lat, 99)), "queries_per_s": sum(qn) / (sum(lat) / 1e3),
                                 "method": "deletion index of the resident build (probe of the query strings own records)"}
            except Exception as exc:  # keep the line: record the failed leg
                line.setdefault("leg_errors", {})["query"] = repr(exc)
        if "e2e" in legs:
            try:
                # --- end to end: pinned host inputs in, CSR back in pinned host memory
                hc = torch.from_numpy(rep.chars).pin_memory()
                ho = torch.from_numpy(rep.offsets).pin_memory()
                off_h = torch.empty(n + 1, dtype=torch.int32).pin_memory()
                cols_h = torch.empty(max(nnz, 1), dtype=torch.int32).pin_memory()
                deg_h = torch.empty(n, dtype=torch.int32).pin_memory()
                e2e_ms = []
                for k in range(args.e2e_steps + 2):
                    flush.fill_(2)
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    g = tn.tcrnet_build_flat(hc, ho, 1, method=args.method, stream=stream)
                    g.copy_csr(out=(off_h, cols_h, deg_h))
                    torch.cuda.synchronize()
                    dt = time.perf_counter() - t
                    g.free()
                    if k >= 2:
                        e2e_ms.append(dt * 1e3)
                e_ms = statistics.mean(e2e_ms)
                # pipelined: three host threads, each with its own stream and pinned
                # result buffers, run their steps back to back, so one step's
                # copies overlap the others' builds (the link is full duplex);
                # whole-job throughput = all steps / wall time
                depth = 3
                bufs = [(torch.cuda.Stream(), off_h, cols_h, deg_h)] + [
                    (torch.cuda.Stream(), torch.empty(n + 1, dtype=torch.int32).pin_memory(),
                     torch.empty(max(nnz, 1), dtype=torch.int32).pin_memory(),
                     torch.empty(n, dtype=torch.int32).pin_memory()) for _ in range(depth - 1)]
                per = max(4, args.e2e_steps // depth)
                errors = []

                def e2e_worker(k, steps):
                    try:
                        st_k, o_k, c_k, d_k = bufs[k]
                        for _ in range(steps):
                            gk = tn.tcrnet_build_flat(hc, ho, 1, method=args.method, stream=st_k)
                            gk.copy_csr(out=(o_k, c_k, d_k))
                            gk.free()
                    except BaseException as exc:  # reported after the join
                        errors.append(exc)

                for k in range(depth):
                    e2e_worker(k, 1)  # warm each stream's path
                torch.cuda.synchronize()
                t = time.perf_counter()
                workers = [threading.Thread(target=e2e_worker, args=(k, per)) for k in range(depth)]
                for w in workers:
                    w.start()
                for w in workers:
                    w.join()
                torch.cuda.synchronize()
                p_ms = 1e3 * (time.perf_counter() - t) / (per * depth)
                if errors:
                    raise errors[0]
                line["e2e"] = {"value": cand_per_build / (p_ms / 1e3), "unit": UNIT, "ms_per_step": p_ms,
                               "h2d_bytes_per_step": int(rep.chars.nbytes + rep.offsets.nbytes),
                               "d2h_bytes_per_step": int(4 * (n + 1) + 4 * nnz + 4 * n),
                               "pipeline": f"{depth} host threads with their own streams and pinned buffers, "
                                           f"{per * depth} steps, each step's upload, build and CSR download included",
                               "serial_ms_per_step": e_ms, "serial_value": cand_per_build / (e_ms / 1e3)}
            except Exception as exc:  # keep the line: record the failed leg
                line.setdefault("leg_errors", {})["e2e"] = repr(exc)
        if "insert" in legs:
            try:
                # --- inserts into the resident N = 8e5 network: merged (query + network
                #     of the new strings, grown rows and index) vs rebuilt; copy-on-write
                #     (tcrnet_extend), new strings in device memory
                from synthgen import generate

                # later draws of the same repertoire model (same templates): the new
                # strings join the resident network
                ipool = generate(100_000, seed=2000 + rank, template_seed=rank, ins_max=6, len_lo=10, len_hi=20)
                ic = torch.from_numpy(ipool.chars).to(dev)
                io = torch.from_numpy(ipool.offsets).to(dev)
                ins = {}
                with build() as g:
                    for m_ins in [int(x) for x in args.insert_sizes.split(",") if x]:
                        row = {}
                        for mode, kw in (("merged", {"merge": True}), ("rebuilt", {"rebuild": True}), ("auto", {})):
                            ts = []
                            for k in range(4):
                                torch.cuda.synchronize()
                                t = time.perf_counter()
                                g2 = g.extend_flat(ic, io[:m_ins + 1], stream=stream, **kw)
                                torch.cuda.synchronize()
                                dt = 1e3 * (time.perf_counter() - t)
                                if k == 0:
                                    st2 = g2.stats()
                                g2.free()
                                if k >= 1:
                                    ts.append(dt)
                            row[f"{mode}_ms"] = statistics.median(ts)
                            if mode == "merged":
                                row["merged"] = st2["merged_inserts"] == 1
                                row["nnz_after"] = st2["nnz"]
                            if mode == "auto":
                                row["auto_merged"] = st2["merged_inserts"] == 1
                        row["speedup"] = row["rebuilt_ms"] / row["merged_ms"]
                        ins[str(m_ins)] = row
                line["insert"] = {"resident_strings": n, "sizes": ins,
                                  "timing": "host time of tcrnet_extend (copy-on-write insert) with a stream sync, median of 3 "
                                            "after 1 warm-up; new strings already in device memory; merged = "
                                            "insert_rebuild 2, rebuilt = 1, auto = 0 (the measured rule)"}
            except Exception as exc:  # keep the line: record the failed leg
                line.setdefault("leg_errors", {})["insert"] = repr(exc)
        if "analytics" in legs:
            try:
                # --- analytics on the N = 8e5 network: LCC under random node removal
                #     (normalisations of Methods "Computing LCC"), average neighbour degree
                with build() as g:
                    ps = [0.0, 0.01, 0.1, 0.3, 0.49, 0.7, 0.89, 0.95, 0.98]
                    rng = np.random.default_rng(2024)
                    curve, t_cc = [], []
                    lcc0 = None
                    for p in ps:
                        keep = (rng.random(n) >= p).astype(np.uint8)
                        kt = torch.from_numpy(keep).to(dev)
                        torch.cuda.synchronize()
                        t = time.perf_counter()
                        _, nc, lcc = _components_device(g, kt, tn)
                        t_cc.append(1e3 * (time.perf_counter() - t))
                        lcc0 = lcc if p == 0.0 else lcc0
                        norm1 = lcc / ((1 - p) * n)
                        curve.append({"p": p, "lcc": lcc, "components": nc, "lcc_norm1": norm1,
                                      "lcc_norm2": norm1 / (lcc0 / n)})
                    knn_d = torch.empty(n, dtype=torch.float64, device=dev)
                    t_knn = []
                    for _ in range(5):  # output in device memory; host time of the call
                        torch.cuda.synchronize()
                        t = time.perf_counter()
                        st = tn.load_library().tcrnet_neighbor_degree(g.handle, knn_d.data_ptr(), tn.DEVICE)
                        t_knn.append(1e3 * (time.perf_counter() - t))
                        if st != tn.OK:
                            raise tn.TcrnetError(st, "tcrnet_neighbor_degree")
                line["analytics"] = {"lcc_under_removal": curve, "components_ms_median": statistics.median(t_cc),
                                     "neighbor_degree_ms": statistics.median(t_knn),
                                     "mean_neighbor_degree": float(knn_d.mean().item()),
                                     "timing": "host time of each call, removal masks and outputs in device memory; "
                                               "deletion builds run on the graph of distinct strings"}
            except Exception as exc:  # keep the line: record the failed leg
                line.setdefault("leg_errors", {})["analytics"] = repr(exc)
        if "lmax2" in legs:
            try:
                # --- l_max = 2: the paper's assortativity setting of 4 x 8,000 sequences,
                #     and N = 1e5, by the default method (deletion candidates + exact
                #     distance) and by the all-pairs bit-parallel distance kernel
                from synthgen import generate_config1

                lm2 = {}
                peak = peaks["issue_ceiling_tops"] * 1e12 if peaks else SMS * INT_LANES_PER_SM * sm_max_nominal * 1e6
                for n2 in (32_000, 100_000):
                    r2 = generate_config1(n2, seed=7)
                    c2 = torch.from_numpy(r2.chars).to(dev)
                    o2 = torch.from_numpy(r2.offsets).to(dev)
                    row = {}
                    for label, meth in (("default", "auto"), ("all_pairs", "tile")):
                        tn.tcrnet_build_flat(c2, o2, 2, method=meth, stream=stream).free()
                        ts = []
                        for _ in range(3):
                            a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                            a2.record(stream)
                            g2 = tn.tcrnet_build_flat(c2, o2, 2, method=meth, stream=stream)
                            b2.record(stream)
                            b2.synchronize()
                            st2 = g2.stats()
                            g2.free()
                            ts.append(a2.elapsed_time(b2))
                        ms2 = statistics.median(ts)
                        entry = {"build_ms": ms2, "method": {1: "tile", 2: "deletion"}.get(st2["method"], "?"),
                                 "nnz": st2["nnz"], "all_pairs_per_s": n2 * (n2 - 1) / 2 / (ms2 / 1e3)}
                        if st2["method"] == tn.METHOD_DELETION:
                            entry["candidates_checked"] = st2["candidate_pairs"]
                            entry["variant_records"] = st2["n_records"]
                        else:
                            # per candidate pair the recurrence runs one step per letter of
                            # the row string, 17 integer operations per step (an estimate
                            # from the mean length), against the issue ceiling
                            g3 = tn.tcrnet_build_flat(c2, o2, 2, method=meth, stream=stream, profile=True)
                            st3 = g3.stats()
                            g3.free()
                            mean_len = float(np.diff(r2.offsets).mean())
                            ach = st3["candidate_pairs"] * mean_len * 17.0 / (st3["ms_count"] / 1e3)
                            entry.update({"candidate_pairs": st3["candidate_pairs"], "count_pass_ms": st3["ms_count"],
                                          "roofline": {"bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12,
                                                       "unit": "Tops/s", "frac": ach / peak,
                                                       "ops_per_pair": f"17 x mean length ({mean_len:.2f}), estimate"}})
                        row[label] = entry
                    if n2 == 100_000:
                        # queries against the l_max = 2 build: its variant-record index
                        # vs the all-pairs kernel, 1,000 strings of the resident model
                        from synthgen import generate as _gen

                        q2 = _gen(1000, seed=2024, template_seed=7, ins_max=6, len_lo=10, len_hi=20)
                        qc2 = torch.from_numpy(q2.chars).to(dev)
                        qo2 = torch.from_numpy(q2.offsets).to(dev)
                        qrow = {}
                        with tn.tcrnet_build_flat(c2, o2, 2, stream=stream) as g2:
                            for qlabel, qm in (("index", "deletion"), ("all_pairs", "tile")):
                                g2.query_flat(qc2, qo2, method=qm, stream=stream).free()
                                qts = []
                                for _ in range(5):
                                    t0 = time.perf_counter()
                                    rq = g2.query_flat(qc2, qo2, method=qm, stream=stream)
                                    qts.append((time.perf_counter() - t0) * 1e3)
                                    qn = rq.info()[1]
                                    rq.free()
                                qrow[qlabel] = {"ms": statistics.median(qts), "answers": qn}
                        qrow["timing"] = "host time of tcrnet_query_ex with its stream sync, median of 5; queries in device memory"
                        row["query_1000"] = qrow
                    lm2[str(n2)] = row
                line["lmax2"] = lm2
            except Exception as exc:  # keep the line: record the failed leg
                line.setdefault("leg_errors", {})["lmax2"] = repr(exc)
        if "batched" in legs:
            try:
                # --- batched: uneven repertoires in one pass vs one plain build each
                if args.batched_reps > 0:
                    line["batched"] = batched_leg(args, tn, torch, stream, flush)
            except Exception as exc:  # keep the line: record the failed leg
                line.setdefault("leg_errors", {})["batched"] = repr(exc)
        if "serving" in legs:
            try:
                # --- serving: resident repertoire, Poisson queries and inserts
                if args.serve_seconds > 0:
                    line["serving"] = serve_leg(args, tn, torch, stream)
            except Exception as exc:  # keep the line: record the failed leg
                line.setdefault("leg_errors", {})["serving"] = repr(exc)
        if "cpu" in legs:
            try:
                # --- CPU oracle and the paper's algorithm on bounded samples (rank 0, one GPU only)
                if world == 1 and args.cpu_seconds > 0:
                    line["cpu_baseline"] = cpu_leg(rep, args.cpu_seconds)
            except Exception as exc:  # keep the line: record the failed leg
                line.setdefault("leg_errors", {})["cpu"] = repr(exc)
        if "n8e6" in legs:
            try:
                line["n8e6"] = large_leg(tn, torch, dev, stream, flush)
            except Exception as exc:  # keep the line: record the failed leg
                line.setdefault("leg_errors", {})["n8e6"] = repr(exc)
        if "cpu_full" in legs and world == 1:
            try:
                line["cpu_full"] = cpu_full_leg()
            except Exception as exc:  # keep the line: record the failed leg
                line.setdefault("leg_errors", {})["cpu_full"] = repr(exc)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
