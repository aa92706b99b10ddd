#!/usr/bin/env python
"""Benchmark of batched range-filtered k-NN search (UNIFY / HSIG) on GB300.

Default workload (c2, SIFT1M shape, seeded synthetic stand-in): n = 1,000,000
integer-valued vectors, d = 128, uniform integer attributes in [0, 1e6), HSIG with
S = 16 segments and M = 16; a batch of 10,000 queries from the same mixture with
range fractions 0.1 / 1 / 10 / 50 / 100 % (2,000 each), k = 10, range-aware
routing. ``--config c4`` runs the precision shape instead: n = 10,000,000 unit
vectors, d = 96, ranges 1 / 10 / 50 %, FP32 against BF16 and FP8 E4M3 storage with
the FP32 re-rank of 4k candidates, at k = 10 and k = 100.

One step = one search of the whole batch through the C ABI (route, pre-filter
scan + merge, hybrid search, post-filter search, result writing). The metric is
queries per second at recall@10 >= 0.95 in every range-fraction group. The
autotuner picks the beam widths, thresholds and kernel shape on a held-out batch
(an independent query stream of the same recipe); the timed batch is scored
against its exact answers (Strategy A with FP32 storage).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--config c2|c4]
Multi-GPU (torchrun): every rank holds a replica of the index and searches its
own batch (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QPS at recall@10>=0.95 by range fraction; FP32 vs BF16/FP8 path; % HBM peak"
UNIT = "queries/s"
WORKLOADS = {
    "c1": "c1: n=10,000 d=64 N(0,1), attribute a permutation, 200 queries, ranges 1/10/50%, k=10, auto-routed",
    "c2": "c2: n=1,000,000 d=128 int-valued mixture, 10,000 queries, ranges 0.1/1/10/50/100%, k=10, auto-routed",
    "c3": "c3: n=1,000,000 d=96 unit-normalised 500-centroid mixture, 10,000 queries, range fractions log-uniform "
          "in 0.01-100% (recall grouped by decade, labelled by its lower edge), k=10, auto-routed",
    "c4": "c4: n=10,000,000 d=96 unit-normalised mixture, 10,000 queries, ranges 1/10/50%, k=10 and 100, "
          "auto-routed; FP32 vs BF16 / FP8 E4M3 storage with FP32 re-rank of 4k",
}
FALLBACK_HBM_GBS = 6800.0
TUNE_SEED_OFFSET = 1_000_003  # query stream of the held-out tuning batch
# the paper's default search parameters (Sections 5.2 and 5.7): the reference arm's
PAPER_EF, PAPER_M = 100, 16

# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum, one pass) of one
# full-size search-kernel launch, with the kernel source digest, the workload and
# the search parameters the capture ran with. A run whose digest, workload or
# parameters differ reports traffic null, beside the nearest capture's parameters.
NCU_TRAFFIC = [
    {"digest": "641a67db8b15", "workload": "c2", "bytes": 1_947_512_576 + 12_342_272,
     "params": {"ef": 16, "ef_post": 96, "m": 64, "tau_a": 50000, "tau_b": 600000, "dtype": 0, "selection": 2,
                "cand_cap": 256, "visited_cap": 1024, "warps_per_block": 4, "scan_rows": 8192, "reg_budget": 80,
                "tc_scan": 1},
     "profile": "profiles/batch_kernel_c2_1m_launches.md"},
    {"digest": "641a67db8b15", "workload": "c2", "bytes": 1_948_306_432 + 12_202_240,
     "params": {"ef": 16, "ef_post": 96, "m": 64, "tau_a": 20000, "tau_b": 600000, "dtype": 0, "selection": 2,
                "cand_cap": 256, "visited_cap": 1024, "warps_per_block": 4, "scan_rows": 8192, "reg_budget": 80,
                "tc_scan": 1},
     "profile": "profiles/batch_kernel_c2_1m_launches.md"},
    {"digest": "641a67db8b15", "workload": "c2", "bytes": 1_947_282_944 + 11_829_248,
     "params": {"ef": 16, "ef_post": 96, "m": 64, "tau_a": 20000, "tau_b": 750000, "dtype": 0, "selection": 2,
                "cand_cap": 256, "visited_cap": 1024, "warps_per_block": 4, "scan_rows": 8192, "reg_budget": 80,
                "tc_scan": 1},
     "profile": "profiles/batch_kernel_c2_1m_launches.md"},
]
TRAFFIC_KEYS = ("ef", "ef_post", "m", "tau_a", "tau_b", "dtype", "selection", "cand_cap", "visited_cap",
                "warps_per_block", "scan_rows", "reg_budget", "tc_scan")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def src_digest(*names):
    h = hashlib.sha1()
    for n in names:
        with open(os.path.join(ROOT, "paper_2412_02448_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def cache_dir():
    d = os.environ.get("UNIFY_CACHE_DIR", os.path.join(ROOT, "_cache"))
    os.makedirs(d, exist_ok=True)
    return d


def get_index(w, rank, world, barrier, gpu=False):
    """The cached index of workload w, built on rank 0 when missing: with the
    GPU-assisted builder when gpu is set, else with the host builder."""
    import hsig_build
    path = hsig_build.cached_index_path(cache_dir(), w.name, w.n, w.seed)
    if rank == 0 and not os.path.exists(path):
        t = time.time()
        if gpu:
            import paper_2412_02448_gb300 as U
            U.build_index(w.vectors, w.attrs, path, w.S, w.M, w.efc, seed=w.seed)
        else:
            hsig_build.build_index(w.vectors, w.attrs, path, w.S, w.M, w.efc, seed=w.seed)
        log(f"built index {path} in {time.time() - t:.1f} s")
    barrier()
    return path


def config_dict(name, w, world, nq):
    """The workload description shared by both arms' JSON lines."""
    return {"workload": WORKLOADS[name], "n": w.n, "d": w.d, "queries_per_step": nq,
            "k": [10, 100] if name == "c4" else 10, "S": w.S, "M": w.M, "efc": w.efc,
            "parallelism": f"replicas x{world}",
            "l2": "flushed between steps (256 MiB write); " + ("the c1 index (a few MB) fits in L2" if name == "c1"
                                                               else "the index is larger than L2")}


def fraction_groups(name, fractions):
    """The groups recall is reported by: the range fractions themselves, or for the
    log-uniform fractions of c3 their decade, labelled by its lower edge."""
    fractions = np.asarray(fractions, dtype=np.float64)
    if name != "c3":
        return fractions
    return 10.0 ** np.clip(np.floor(np.log10(fractions)), -4, 0)


def stratified_rows(fractions, per_fraction):
    """Up to per_fraction rows of every range-fraction group (all rows when per_fraction <= 0)."""
    if per_fraction <= 0:
        return np.arange(len(fractions))
    return np.sort(np.concatenate([np.flatnonzero(fractions == f)[:per_fraction] for f in np.unique(fractions)]))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def traffic_for(digest, workload, params):
    """(bytes, capture) of the ncu capture matching this kernel, workload and
    parameters, else (None, the latest capture of this kernel and workload)."""
    want = {k_: int(getattr(params, k_)) for k_ in TRAFFIC_KEYS}
    near = None
    for c in NCU_TRAFFIC:
        if c["digest"] != digest or c["workload"] != workload:
            continue
        near = c
        if all(int(c["params"].get(k_, -1)) == v for k_, v in want.items()):
            return c["bytes"], c
    return None, near


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = os.path.join(cache_dir(), f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def truth_check(w, rows, truth_ids, truth_cnt, k, per_fraction):
    """The exact answers the GPU arm scores recall against (Strategy A with FP32
    storage) compared, on a stratified sample of them, with the oracle's FP64 exact
    range-filtered k-NN (Definition 1). ``rows`` are the batch rows the truth arrays
    hold. A row matches when ids and count are equal; on real-valued data ids may
    also differ by swaps of objects whose FP64 distances lie within 2e-5 relative of
    each other (the float32 tie band). Returns the counts."""
    import oracle
    fr = w.fractions[rows]
    pick = np.sort(np.concatenate([np.flatnonzero(fr == f)[:per_fraction] for f in np.unique(fr)]))
    sel = rows[pick]
    ex_ids, ex_d, ex_c = oracle.exact_knn(w.vectors, w.attrs, w.queries[sel], w.lo[sel], w.hi[sel], k)
    equal = band = mismatch = 0
    for j, t in enumerate(pick):
        c = int(ex_c[j])
        g, e = truth_ids[t, :c], ex_ids[j, :c]
        if int(truth_cnt[t]) != c:
            mismatch += 1
        elif np.array_equal(g, e):
            equal += 1
        else:
            q = w.queries[sel[j]].astype(np.float64)
            d64 = lambda v: float(((w.vectors[v].astype(np.float64) - q) ** 2).sum())
            kth = float(ex_d[j, c - 1])
            diff = set(g.tolist()) ^ set(e.tolist())
            ok = all(abs(d64(v) - kth) <= 2e-5 * kth for v in diff)
            dg = [d64(v) for v in g]
            ok = ok and all(b >= a or a - b <= 2e-5 * a for a, b in zip(dg[:-1], dg[1:]))
            band += int(ok)
            mismatch += int(not ok)
    return {"rows": int(len(pick)), "ids_equal": equal, "tie_band_swaps": band, "mismatch": mismatch}


def cpu_baseline(path, w, params, k, budget_s, per_fraction):
    """The oracle's literal HSIG search on the host cores, on a stratified sample
    of the batch, repeated until about budget_s seconds of CPU work."""
    import oracle
    oi = oracle.OracleIndex(path)
    cores = oracle.default_threads()
    fr = np.unique(w.fractions)
    idx = np.concatenate([np.flatnonzero(w.fractions == f)[:per_fraction] for f in fr])
    kw = dict(ef=params.ef, m=params.m, ef_post=params.ef_post, strategy="auto",
              tau_a=params.tau_a, tau_b=params.tau_b, threads=cores)
    t = time.perf_counter()
    oi.search(w.queries[idx], w.lo[idx], w.hi[idx], k, **kw)
    dt = time.perf_counter() - t
    # grow the stratified sample towards the budget (at most the whole batch), then repeat passes
    per = min(len(w.lo) // len(fr), max(per_fraction, int(per_fraction * budget_s / max(dt, 1e-3))))
    idx = np.concatenate([np.flatnonzero(w.fractions == f)[:per] for f in fr])
    done, passes = 0, 0
    t = time.perf_counter()
    while True:
        oi.search(w.queries[idx], w.lo[idx], w.hi[idx], k, **kw)
        done += len(idx)
        passes += 1
        if time.perf_counter() - t >= budget_s * 0.5:
            break
    dt = time.perf_counter() - t
    # the same search on one core, on a smaller stratified sample (about 2 s)
    per1 = max(2, min(per, int(2.0 * (done / dt) / cores / len(fr))))
    idx1 = np.concatenate([np.flatnonzero(w.fractions == f)[:per1] for f in fr])
    t1 = time.perf_counter()
    oi.search(w.queries[idx1], w.lo[idx1], w.hi[idx1], k, **dict(kw, threads=1))
    dt1 = time.perf_counter() - t1
    oi.close()
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(idx)} queries stratified over the range fractions of the batch, {passes} pass(es), "
                      f"{dt:.1f} s (literal HSIG search, FP64, same ef/m/tau)",
            "one_core": {"value": len(idx1) / dt1, "unit": UNIT, "cores": 1,
                         "sample": f"{len(idx1)} queries, same strata, {dt1:.1f} s"}}


def reference_arm(args, rank, world):
    """The oracle (the CPU reference of this build: the paper's literal HSIG search,
    FP64) timed on the host cores with the paper's default parameters, on the same
    workload and batch as the GPU arm. Nothing of the CUDA library is loaded."""
    from workloads import make_workload
    import oracle
    if rank != 0:
        return
    over = {k_: v for k_, v in (("n", args.n), ("nq", args.nq)) if v}
    w = make_workload(args.config, seed=args.seed, **over)
    w.fractions = fraction_groups(args.config, w.fractions)
    path = get_index(w, 0, 1, lambda: None)
    oi = oracle.OracleIndex(path)
    cores = oracle.default_threads()
    fr = np.unique(w.fractions)
    nq = len(w.lo)
    k = 10
    kw = dict(ef=PAPER_EF, m=PAPER_M, ef_post=PAPER_EF, strategy="auto", tau_a=w.n // 100, tau_b=w.n // 2,
              threads=cores)
    # calibrate the per-query time; a step is the whole batch when the run fits about
    # two minutes, otherwise a stratified sample of it
    cal = np.concatenate([np.flatnonzero(w.fractions == f)[:8] for f in fr])
    t = time.perf_counter()
    oi.search(w.queries[cal], w.lo[cal], w.hi[cal], k, **kw)
    tq = (time.perf_counter() - t) / len(cal)
    per_step = int(np.clip(150.0 / (args.steps + args.warmup) / max(tq, 1e-6), len(fr), nq))
    per_f = max(1, per_step // len(fr))
    full = per_f * len(fr) >= nq
    rng = np.random.default_rng(args.seed)
    steps_t = []
    for s in range(args.warmup + args.steps):
        if full:
            idx = np.arange(nq)
        else:
            idx = np.concatenate([rng.choice(np.flatnonzero(w.fractions == f), per_f, replace=False) for f in fr])
        t = time.perf_counter()
        oi.search(w.queries[idx], w.lo[idx], w.hi[idx], k, **kw)
        if s >= args.warmup:
            steps_t.append((time.perf_counter() - t, len(idx)))
    tot = sum(x for x, _ in steps_t)
    nqs = sum(n_ for _, n_ in steps_t)
    value = nqs / tot
    sample = (f"the whole batch ({nq} queries) per step" if full else
              f"{per_f * len(fr)} of the batch's {nq} queries per step, stratified over the range fractions")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * tot / len(steps_t), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": config_dict(args.config, w, world, nq),
            "params": {"ef": PAPER_EF, "ef_post": PAPER_EF, "m": PAPER_M, "tau_a": w.n // 100, "tau_b": w.n // 2},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample + "; literal HSIG search, FP64, the paper's default ef, m and tau"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run(args):
    """The GPU arm: tune on the held-out batch, then time and score the batch."""
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier()
    import paper_2412_02448_gb300 as U
    from paper_2412_02448_gb300 import autotune, replicas
    from workloads import make_workload, query_batch

    name = args.config
    over = {k_: v for k_, v in (("n", args.n), ("nq", args.nq)) if v}
    w = make_workload(name, seed=args.seed, **over)
    path = get_index(w, rank, world, barrier, gpu=True)
    # the held-out tuning batch: the same recipe from an independent query stream
    tq, tlo, thi, tfr = query_batch(w, args.seed + TUNE_SEED_OFFSET)
    w.fractions, tfr = fraction_groups(name, w.fractions), fraction_groups(name, tfr)
    # weak scaling: every rank searches its own batch of the same shape
    w.queries, w.lo, w.hi, w.fractions = replicas.rank_batch(w.queries, w.lo, w.hi, w.fractions, rank, args.seed)
    ix = U.Index(path, device=local)
    dev = torch.device("cuda", local)
    nq = len(w.lo)
    ks = (10, 100) if name == "c4" else (10,)
    # scored rows: every row of the c2 batches; 200 per range fraction of the c4 batches
    # (an exact answer there scans up to 5M rows), with a wider tuning margin for the
    # smaller sample
    per_f = args.truth_per_fraction if args.truth_per_fraction >= 0 else (200 if name == "c4" else 0)
    # c4 scores recall on 200 queries per range fraction (sampling noise about 0.01):
    # its tuner keeps a wider margin
    tune_margin = args.tune_margin if args.tune_margin >= 0 else (0.02 if name == "c4" else 0.005)

    def on_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    # exact answers (Strategy A, FP32 storage) of the scored rows of both batches:
    # every row of the c2 batches, a stratified sample of the 10M-row c4 batches
    t0 = time.time()
    B = {"q": on_dev(w.queries), "lo": on_dev(w.lo), "hi": on_dev(w.hi), "fr": w.fractions}
    T = {"q": on_dev(tq), "lo": on_dev(tlo), "hi": on_dev(thi), "fr": tfr}
    for b in (B, T):
        b["rows"] = stratified_rows(b["fr"], per_f)
        rt = torch.from_numpy(b["rows"]).to(dev)
        r = ix.search(b["q"][rt], b["lo"][rt], b["hi"][rt], max(ks), strategy="pre",
                      params=U.Params.defaults(dtype=U.FP32))
        torch.cuda.synchronize()
        b["t_ids"], b["t_cnt"] = r["ids"].cpu().numpy(), r["count"].cpu().numpy()
    log(f"exact answers of {len(B['rows'])} + {len(T['rows'])} rows in {time.time() - t0:.1f} s")

    q, lo, hi = B["q"], B["lo"], B["hi"]
    base = U.Params.defaults(tau_a=w.n // 100, tau_b=w.n // 2, scan_rows=args.scan_rows, ef=args.ef,
                             ef_post=args.ef_post or args.ef, m=args.m, cand_cap=args.cand_cap,
                             visited_cap=args.visited_cap, warps_per_block=args.warps_per_block,
                             reg_budget=args.reg_budget, selection=args.selection, rerank_mult=args.rerank_mult,
                             tc_scan=args.tc_scan)
    if args.tau_a >= 0:
        base.tau_a = args.tau_a
    if args.tau_b >= 0:
        base.tau_b = args.tau_b
    route = ix.route(lo, hi, base.tau_a, base.tau_b)
    pa, pb = route["pa"].cpu().numpy().astype(np.int64), route["pb"].cpu().numpy().astype(np.int64)
    mask = route["mask"].cpu().numpy().astype(np.uint32)
    Sp = np.array([bin(int(m_)).count("1") for m_ in mask])
    Y = pb - pa
    hbm, peak_kind = peaks()
    bf16_peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16_peak = float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        pass
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    d = w.d

    def routing(params):
        a_ = Y <= params.tau_a
        b_ = (~a_) & (Y >= params.tau_b)
        return a_, b_, ~(a_ | b_)

    def algorithmic_bytes(params, counters, k):
        """Bytes the search kernel must move per launch, by strategy: a scanned row
        (its storage bytes plus the 4-byte id) per in-range row for A; per distance
        evaluation one row, and per expansion the adjacency slots read (S' chunks of
        ceil(m / S') slots for C; M slots plus the bitmap words for B); plus the FP32
        re-rank rows of the BF16/FP8 paths."""
        isA, isB, isC = routing(params)
        row = {U.FP32: 4 * d, U.BF16: 2 * d, U.FP8E4M3: d + 4}[params.dtype]
        per = np.minimum(ix.M, -(-params.m // np.maximum(Sp, 1)))
        rr = 0 if params.dtype == U.FP32 else params.rerank_mult * k * 4 * d
        return {
            "scan": float(((pb - pa) * (row + 4))[isA].sum() + rr * isA.sum()),
            "hybrid": float((counters[isC, 0] * row + counters[isC, 1] * Sp[isC] * per[isC] * 4).sum() + rr * isC.sum()),
            "post": float((counters[isB, 0] * row + counters[isB, 1] * (ix.M + (ix.S * ix.M + 31) // 32) * 4).sum()
                          + rr * isB.sum()),
        }

    def scored(ids, k):
        rec = autotune.recall_rows(ids[B["rows"]], B["t_ids"][:, :k], B["t_cnt"], k)
        return autotune.group_recall(rec, B["fr"][B["rows"]])

    def fmt_recall(gr):
        return {f"{100 * f_:g}%": round(v_, 4) for f_, v_ in gr.items()}

    def flagged(status):
        bad = (status & 3) != 0
        return int(bad.sum()), {f"{100 * f_:g}%": int(bad[w.fractions == f_].sum()) for f_ in np.unique(w.fractions)}

    def measure(params, steps, warmup, k=10):
        isA, isB, isC = routing(params)
        out = ix.search(q, lo, hi, k, strategy="auto", params=params, counters=True)
        torch.cuda.synchronize()
        gr = scored(out["ids"].cpu().numpy(), k)
        counters = out["counters"].cpu().numpy().astype(np.int64)
        status = out["status"].cpu().numpy()
        timeline = {}
        for nm, sel in (("pre", isA), ("hybrid", isC), ("post", isB)):
            if sel.any():
                st_, en_ = counters[sel, 2], counters[sel, 3]
                du = en_ - st_
                idxs = np.flatnonzero(sel)
                slow = idxs[np.argsort(du)[-3:][::-1]]
                timeline[nm] = {"queries": int(sel.sum()), "dur_us_p50": float(np.percentile(du, 50)),
                                "dur_us_p99": float(np.percentile(du, 99)), "dur_us_max": int(du.max()),
                                "last_end_us": int(en_.max()), "first_start_us": int(st_.min()),
                                "slowest": [{"frac": float(w.fractions[i_]), "Y": int(pb[i_] - pa[i_]),
                                             "segments": int(Sp[i_]), "n_exp": int(counters[i_, 1]),
                                             "n_dist": int(counters[i_, 0]),
                                             "us": int(counters[i_, 3] - counters[i_, 2]),
                                             "status": int(status[i_])} for i_ in slow]}
        out = ix.search(q, lo, hi, k, strategy="auto", params=params)
        for _ in range(warmup):
            flush.fill_(1)
            out = ix.search(q, lo, hi, k, strategy="auto", params=params, out=out)
        ix.collect_timing()
        ix.timing(True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for s_ in range(steps):
            flush.fill_(s_ & 0xFF)
            evs[s_][0].record(stream)
            out = ix.search(q, lo, hi, k, strategy="auto", params=params, out=out)
            evs[s_][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - wall0
        ix.timing(False)
        phases = ix.collect_timing()
        ms = float(np.mean([a_.elapsed_time(b_) for a_, b_ in evs]))
        ms_max = replicas.max_over_ranks(ms, world, dev)
        search_ms = phases["search"][0] / max(1, phases["search"][1])
        tc_used = phases["tcscan"][1] > 0
        parts = algorithmic_bytes(params, counters, k)
        tc_roof = None
        if tc_used:
            # the pre-filter queries ran on the tensor cores, not in the search kernel:
            # the scan leaves the search kernel's bytes and is rated by its useful work,
            # 2 d FLOP per (query, in-range row), against the format's dense peak (the
            # measured bf16 peak times the nominal ratio: tf32 1/2, E4M3 2)
            del parts["scan"]
            tc_ms = phases["tcscan"][0] / max(1, phases["tcscan"][1])
            flops = float(2.0 * d * (pb - pa)[isA].sum())
            ratio = {U.FP32: 0.5, U.BF16: 1.0, U.FP8E4M3: 2.0}[params.dtype]
            tf = flops / (tc_ms / 1000.0) / 1e12 if tc_ms > 0 else 0.0
            tc_roof = {"bound": "tensor", "kernel": "tc_scan_kernel (both passes) + tc_finish", "unit": "TFLOP/s",
                       "achieved": tf, "peak": ratio * bf16_peak if bf16_peak else None,
                       "frac": tf / (ratio * bf16_peak) if bf16_peak else None, "ms_per_step": tc_ms,
                       "useful_flops_per_step": flops,
                       "peak_source": "measured bf16_tflops x nominal format ratio" if bf16_peak else None}
        alg = sum(parts.values())
        achieved = alg / (search_ms / 1000.0) / 1e9 if search_ms > 0 else 0.0
        nflag, flag_by = flagged(status)
        return dict(ms=ms_max, value=replicas.aggregate_qps(nq, world, ms_max), out=out, wall=wall,
                    timeline=timeline, routed=(int(isA.sum()), int(isC.sum()), int(isB.sum())), recall=gr,
                    flagged=nflag, flagged_by=flag_by, tc_used=tc_used, tc_roofline=tc_roof,
                    phases={ph: (v[0] / v[1] if v[1] else 0.0) for ph, v in phases.items()},
                    achieved=achieved, alg=alg, parts=parts)

    def tuned(extra, k=10, **kw):
        b = U.Params.defaults(**{f: getattr(base, f) for f, _ in U.Params._fields_})
        for kk, v in extra.items():
            setattr(b, kk, v)
        if args.no_tune:
            return b, {}
        eval_rows = T["rows"] if per_f > 0 else None
        return autotune.tune(ix, T["q"], T["lo"], T["hi"], k, T["t_ids"][:, :k], T["t_cnt"], T["fr"],
                             target=args.target + tune_margin, base=b, log=log if rank == 0 else None,
                             eval_rows=eval_rows, **kw)

    def params_dict(p):
        return {"ef": p.ef, "ef_post": p.ef_post, "m": p.m, "rerank_mult": p.rerank_mult, "dtype": int(p.dtype),
                "tau_a": p.tau_a, "tau_b": p.tau_b, "tc_scan": p.tc_scan, "cand_cap": p.cand_cap,
                "visited_cap": p.visited_cap, "warps_per_block": p.warps_per_block, "scan_rows": p.scan_rows,
                "reg_budget": p.reg_budget, "selection": p.selection}

    def summary(r_, p_):
        return {"value": r_["value"], "ms_per_step": r_["ms"], "recall_by_fraction": fmt_recall(r_["recall"]),
                "status_flagged": r_["flagged"], "roofline_frac": r_["achieved"] / hbm,
                "achieved_gbs": r_["achieved"], "tensor_core_scan_roofline": r_["tc_roofline"],
                "routed": {"pre": r_["routed"][0], "hybrid": r_["routed"][1], "post": r_["routed"][2]},
                "phase_ms_per_step": {ph: round(v, 4) for ph, v in r_["phases"].items() if not ph.startswith("unused")},
                "params": params_dict(p_)}

    def tuned_both_scans(extra, k):
        """Tuned once with each pre-filter scan (the tensor-core run also tries larger
        tau_A, since its cheap shared scans move the best threshold up); the faster
        tuned configuration."""
        p_, rep_ = tuned(extra, k)
        if not args.no_tune:
            p_tc, rep_tc = tuned(dict(extra, tc_scan=1), k, tau_a_fracs=(0.01, 0.02, 0.05, 0.08, 0.12, 0.2))
            if rep_tc.get("ms", 1e9) < rep_.get("ms", 1e9):
                p_, rep_ = p_tc, rep_tc
        return p_, rep_

    def other_scan(p_, k):
        """The same parameters with the other pre-filter scan (tensor cores or warps)."""
        p0 = U.Params.defaults(**{f: getattr(p_, f) for f, _ in U.Params._fields_})
        p0.tc_scan = 1 - p_.tc_scan
        r0 = measure(p0, max(3, args.steps // 2), args.warmup, k)
        return ("tensor_core_scan" if p0.tc_scan else "warp_scan"), {
            "value": r0["value"], "ms_per_step": r0["ms"], "recall_by_fraction": fmt_recall(r0["recall"]),
            "phase_ms_per_step": {ph: round(v, 4) for ph, v in r0["phases"].items() if not ph.startswith("unused")}}

    def precision_line(dt, k):
        """BF16 or FP8 storage with the FP32 re-rank of 4k candidates, tuned on the
        held-out batch with each pre-filter scan, the faster kept and the other scan
        measured beside it at the same parameters."""
        p_, _ = tuned_both_scans({"dtype": dt, "rerank_mult": 4}, k)
        r_ = measure(p_, max(3, args.steps // 2), args.warmup, k)
        line_ = summary(r_, p_)
        name_, other_ = other_scan(p_, k)
        line_[name_] = other_
        return line_

    # FP32 storage at k = 10: the headline (its pre-filter queries on the warp scan or on
    # the tensor cores with tf32 operands and the FP32 re-rank of 4k candidates,
    # whichever tunes faster)
    clocks = Clocks(local)
    params, report = tuned_both_scans({}, 10)
    clocks.start()  # the measurement's warm-up and timed steps
    m32 = measure(params, args.steps, args.warmup)
    clk = clocks.stop()
    value, ms_max, out = m32["value"], m32["ms"], m32["out"]
    digest = src_digest("search.cu", "common.cuh", "warp_ops.cuh", "internal.h")
    traffic, capture = traffic_for(digest, name, params)
    roofline = {"bound": "hbm", "achieved": m32["achieved"], "peak": hbm, "unit": "GB/s",
                "frac": m32["achieved"] / hbm, "traffic": traffic,
                "traffic_frac": (traffic / (m32["phases"]["search"] / 1000.0) / 1e9 / hbm)
                if traffic and m32["phases"]["search"] > 0 else None,
                "kernel": "batch_kernel (route excluded)", "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_launch": m32["alg"], "algorithmic_bytes_by_strategy": m32["parts"],
                "tensor_core_scan": m32["tc_roofline"]}
    if traffic is None:
        roofline["traffic_capture"] = ({"bytes": capture["bytes"], "params": capture["params"],
                                        "note": "captured with other parameters"} if capture else None)
    headline_other = None
    if not args.no_extra:
        nm_, headline_other = other_scan(params, 10)
        headline_other = {"scan": nm_, **headline_other}

    # hybrid selection S1 (the m neighbours nearest to the expanded object) with the
    # same parameters, beside the tuned selection (the comparison of Section 5.6)
    other_sel = None
    if params.m <= 64 and not args.no_extra:
        ps = U.Params.defaults(**{f: getattr(params, f) for f, _ in U.Params._fields_})
        ps.selection = 3 - params.selection
        rs = measure(ps, max(3, args.steps // 2), args.warmup)
        other_sel = {"selection": f"S{ps.selection}", "value": rs["value"], "ms_per_step": rs["ms"],
                     "recall_by_fraction": fmt_recall(rs["recall"]), "status_flagged": rs["flagged"],
                     "note": "same parameters as the headline, other hybrid selection"}

    # BF16 and FP8 (per-vector scale) storage with FP32 re-rank of 4k candidates; for
    # the precision shape also every storage format at k = 100
    precision = {}
    if not args.no_precision:
        precision["bf16"] = precision_line(U.BF16, 10)
        precision["fp8e4m3"] = precision_line(U.FP8E4M3, 10)
        if 100 in ks:
            p100, _ = tuned_both_scans({}, 100)
            precision["k100"] = {"fp32": summary(measure(p100, max(3, args.steps // 2), args.warmup, 100), p100),
                                 "bf16": precision_line(U.BF16, 100),
                                 "fp8e4m3": precision_line(U.FP8E4M3, 100)}

    # tau_A / tau_B calibrated by the paper's preprocessing (Section 4.2): base objects
    # as queries with random ranges, A/B/C per range size at the recall target, the
    # turning points. Base objects as queries are easier than the batch's queries
    # (each finds itself), so the beam widths are tuned again on the held-out batch
    # under the calibrated thresholds; then timed and scored on the batch.
    tau = None
    if not args.no_extra:
        t0 = time.time()
        ta, tb, table = autotune.calibrate_tau(ix, w.vectors, (int(w.attrs.min()), int(w.attrs.max())), 10,
                                               target=args.target + tune_margin, base=params, n_sample=2048,
                                               bins=12, seed=args.seed, log=log if rank == 0 else None)
        cal_s = time.time() - t0
        pc, _ = tuned({f: getattr(params, f) for f, _ in U.Params._fields_} | {"tau_a": ta, "tau_b": tb},
                      calibrate_tau=False)
        rc = measure(pc, max(3, args.steps // 2), args.warmup)
        tau = {"method": "2048 base objects as queries, log-uniform random ranges, Strategies A/B/C per "
                         "range-size bin at the recall target, turning points (Section 4.2); beams tuned "
                         "again on the held-out batch under these thresholds",
               "tau_a": ta, "tau_b": tb, "swept": {"tau_a": params.tau_a, "tau_b": params.tau_b},
               "calibration_s": round(cal_s, 1), **summary(rc, pc),
               "bins": [{k_: (round(v, 4) if isinstance(v, float) else v) for k_, v in r_.items()} for r_ in table]}

    # the same step replayed as one CUDA graph (counter reset, route, search kernel)
    plan = ix.plan(q, lo, hi, 10, strategy="auto", params=params)
    for _ in range(args.warmup):
        flush.fill_(1)
        plan.launch()
    gevs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for s_ in range(args.steps):
        flush.fill_(s_ & 0xFF)
        gevs[s_][0].record(stream)
        plan.launch()
        gevs[s_][1].record(stream)
    torch.cuda.synchronize()
    graph_ms = float(np.mean([a_.elapsed_time(b_) for a_, b_ in gevs]))
    graph_ok = bool(torch.equal(plan.out["ids"], out["ids"]))
    plan.close()

    # end to end through the host-buffer entry point (pinned memory)
    hq = torch.from_numpy(w.queries).pin_memory()
    hlo = torch.from_numpy(w.lo).pin_memory()
    hhi = torch.from_numpy(w.hi).pin_memory()
    hout = dict(ids=torch.empty((nq, 10), dtype=torch.int64).pin_memory(),
                dist=torch.empty((nq, 10), dtype=torch.float32).pin_memory(),
                count=torch.empty(nq, dtype=torch.int32).pin_memory(),
                status=torch.empty(nq, dtype=torch.int32).pin_memory())
    for _ in range(max(3, args.warmup // 2)):
        ix.search_auto_host(hq, hlo, hhi, 10, params=params, out=hout)
    e2e_steps = max(3, args.steps // 2)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ix.search_auto_host(hq, hlo, hhi, 10, params=params, out=hout)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_value = replicas.aggregate_qps(nq, world, 1000.0 * replicas.max_over_ranks(e2e_s, world, dev))
    h2d = nq * w.d * 4 + 2 * nq * 8
    d2h = nq * 10 * (8 + 4) + nq * 4 + nq * 4

    # the CPU-baseline leg: the oracle's literal HSIG search on the host cores, and the
    # exact answers recall is scored against checked with the oracle's FP64 answers
    cpu, tcheck = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        tcheck = truth_check(w, B["rows"], B["t_ids"], B["t_cnt"], max(ks), per_fraction=8)
        cpu = cpu_baseline(path, w, params, 10, args.cpu_budget, per_fraction=20)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(name, w, world, nq),
            "params": params_dict(params),
            "tuning": {"batch": f"held-out: {len(T['fr'])} queries of the same recipe, query stream "
                                f"seed {args.seed + TUNE_SEED_OFFSET}", "target": args.target + tune_margin,
                       "scored_rows": int(len(T["rows"]))},
            "recall_by_fraction": fmt_recall(m32["recall"]),
            "recall_rows": int(len(B["rows"])),
            "status_flagged": m32["flagged"], "status_flagged_by_fraction": m32["flagged_by"],
            "truth_mismatch": tcheck["mismatch"] if tcheck else None, "truth_check": tcheck,
            "routed": {"pre": m32["routed"][0], "hybrid": m32["routed"][1], "post": m32["routed"][2]},
            "phase_ms_per_step": {ph: round(v, 4) for ph, v in m32["phases"].items() if not ph.startswith("unused")},
            "wall_s_timed_region": m32["wall"],
            "timeline_us": m32["timeline"],
            "roofline": roofline,
            "precision": precision,
            "tau": tau,
            "hybrid_selection_other": other_sel,
            "cuda_graph": {"ms_per_step": graph_ms, "value": world * nq / (graph_ms / 1000.0),
                           "same_ids_as_direct": graph_ok},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            # per step: route and search kernels, plus the tensor-core scan's eight
            # (bucket count, bucket scan, scatter, tile prep, unit plan, two passes, finish)
            "gpu_launches": (2 + (8 if m32["tc_used"] else 0)) * args.steps,
            "other_scan": headline_other,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        if report:
            line["tune"] = {"chosen_ms": report.get("ms"), "trials": len(report.get("trials", []))}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def scan_compare(args):
    """Pre-filter scans compared on the c5 shape (d = 960, ranges 0.5/2/10 %, every query
    forced to Strategy A): FP32 warp scan, BF16 warp scan and BF16 tensor-core scan (both
    BF16 paths re-rank 4k candidates in FP32). Prints its own JSON line; not part of the
    default run."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import hsig_build
    import paper_2412_02448_gb300 as U
    from paper_2412_02448_gb300 import autotune
    from workloads import make_workload
    n = args.n or 200_000
    w = make_workload("c5", seed=args.seed, n=n, nq=args.nq or 5000, efc=16)
    # the graph is not used by forced pre-filtering: a light build (efCons 16)
    path = hsig_build.cached_index_path(cache_dir(), "c5scan", w.n, w.seed)
    if not os.path.exists(path):
        t = time.time()
        hsig_build.build_index(w.vectors, w.attrs, path, w.S, w.M, w.efc, seed=w.seed)
        log(f"built index {path} in {time.time() - t:.1f} s")
    ix = U.Index(path)
    dev = torch.device("cuda", 0)
    q = torch.from_numpy(w.queries).to(dev)
    lo = torch.from_numpy(w.lo).to(dev)
    hi = torch.from_numpy(w.hi).to(dev)
    k, nq = w.k, len(w.lo)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    variants = {"fp32_warp": U.Params.defaults(),
                "bf16_warp": U.Params.defaults(dtype=U.BF16, rerank_mult=4),
                "bf16_tensor_core": U.Params.defaults(dtype=U.BF16, rerank_mult=4, tc_scan=1),
                "fp32_tensor_core": U.Params.defaults(rerank_mult=4, tc_scan=1),
                "fp8_tensor_core": U.Params.defaults(dtype=U.FP8E4M3, rerank_mult=4, tc_scan=1)}
    steps = max(3, min(args.steps, 20))
    res, rows = {}, {}
    for name, p in variants.items():
        out = ix.search(q, lo, hi, k, strategy="pre", params=p)
        for _ in range(max(3, args.warmup)):
            flush.fill_(1)
            out = ix.search(q, lo, hi, k, strategy="pre", params=p, out=out)
        ix.collect_timing()
        ix.timing(True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for s_ in range(steps):
            flush.fill_(s_ & 0xFF)
            evs[s_][0].record(stream)
            out = ix.search(q, lo, hi, k, strategy="pre", params=p, out=out)
            evs[s_][1].record(stream)
        torch.cuda.synchronize()
        ix.timing(False)
        ph = ix.collect_timing()
        ms = float(np.mean([a_.elapsed_time(b_) for a_, b_ in evs]))
        rows[name] = {kk: v.cpu().numpy() for kk, v in out.items()}
        res[name] = {"ms_per_step": ms, "value": nq / (ms / 1000.0),
                     "phase_ms_per_step": {kk: round(v[0] / max(1, v[1]), 4) for kk, v in ph.items()
                                           if not kk.startswith("unused")}}
    ref = rows["fp32_warp"]
    for name in ("bf16_warp", "bf16_tensor_core", "fp32_tensor_core", "fp8_tensor_core"):
        rec = autotune.recall_rows(rows[name]["ids"], ref["ids"], ref["count"], k)
        res[name]["recall_vs_fp32_scan"] = autotune.group_recall(rec, w.fractions)
        res[name]["recall_vs_fp32_scan"] = {f"{100 * f_:g}%": round(v_, 4) for f_, v_ in
                                            res[name]["recall_vs_fp32_scan"].items()}
    same = np.all(rows["bf16_warp"]["ids"] == rows["bf16_tensor_core"]["ids"], axis=1)
    Y = np.searchsorted(np.sort(w.attrs), w.hi, side="right") - np.searchsorted(np.sort(w.attrs), w.lo)
    # useful work of the scan: 2 d flops per (query, in-range row); the tensor-core
    # phase against the measured bf16 peak, the warp scans against HBM as bytes per row
    flops = float(2.0 * w.d * Y.sum())
    pk = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
    except OSError:
        pass
    # the operand formats' dense peaks from the measured bf16 one by the nominal ratios
    # (tf32 1/2, E4M3 2x of bf16)
    for name, ratio in (("bf16_tensor_core", 1.0), ("fp32_tensor_core", 0.5), ("fp8_tensor_core", 2.0)):
        tc_ms = res[name]["phase_ms_per_step"].get("tcscan", 0.0)
        if tc_ms > 0:
            tf = flops / (tc_ms / 1000.0) / 1e12
            res[name]["useful_tflops"] = tf
            if pk.get("bf16_tflops"):
                res[name]["tensor_frac_of_measured_peak"] = tf / (ratio * pk["bf16_tflops"])
    for name, row_bytes in (("fp32_warp", 4 * w.d + 4), ("bf16_warp", 2 * w.d + 4)):
        gbs = float(row_bytes * Y.sum()) / (res[name]["ms_per_step"] / 1000.0) / 1e9
        res[name]["row_bytes_gbs"] = gbs
        if pk.get("hbm_gbs"):
            res[name]["hbm_frac_of_measured"] = gbs / pk["hbm_gbs"]
    print(json.dumps({"mode": "scan_compare", "unit": "queries/s",
                      "workload": f"c5 shape: n={w.n} d={w.d} nonneg mixture, {nq} queries, ranges "
                                  "0.5/2/10%, k=10, every query Strategy A",
                      "mean_rows_per_query": float(Y.mean()), "useful_flops_per_step": flops, "steps": steps,
                      "l2": "flushed between steps (256 MiB write)",
                      "rows_equal_bf16_warp_vs_tensor_core": float(same.mean()), **res}), flush=True)


def build_compare(args):
    """HSIG construction of the c2 shape (int mixture, d = 128, S = 16, M = 16, efCons =
    100) at n = --n (default 200,000): the host builder on every host core against the
    GPU-assisted builds, proposals only (the searches of every batch of 64 or more
    nodes on the GPU) and proposals plus edge application on the GPU. Integer vectors
    make every float32 distance exact, so the files must be identical. Prints its own
    JSON line; not part of the default run."""
    import __graft_entry__
    __graft_entry__.build()
    import hsig_build
    import paper_2412_02448_gb300 as U
    from workloads import make_workload
    w = make_workload("c2", seed=args.seed, n=args.n or 200_000, nq=16)
    d = cache_dir()
    p_host = os.path.join(d, f"build_compare_host_{os.getpid()}.idx")
    p_gpu = {m: os.path.join(d, f"build_compare_{m}_{os.getpid()}.idx") for m in ("propose", "apply")}
    hsig_build.compile()
    res = {}
    try:
        t = time.perf_counter()
        hsig_build.build_index(w.vectors, w.attrs, p_host, w.S, w.M, w.efc, seed=w.seed)
        res["host_s"] = time.perf_counter() - t
        for m, p_ in p_gpu.items():
            t = time.perf_counter()
            U.build_index_gpu(w.vectors, w.attrs, p_, w.S, w.M, w.efc, seed=w.seed, device_apply=(m == "apply"))
            res[f"assisted_{m}_s"] = time.perf_counter() - t
        with open(p_host, "rb") as f:
            ref = f.read()
        equal = {}
        for m, p_ in p_gpu.items():
            with open(p_, "rb") as f:
                equal[m] = f.read() == ref
    finally:
        for p_ in [p_host, *p_gpu.values()]:
            if os.path.exists(p_):
                os.remove(p_)
    print(json.dumps({"mode": "build_compare", "unit": "s", "higher_is_better": False,
                      "workload": f"c2 shape: n={w.n} d={w.d} int mixture, S={w.S} M={w.M} efCons={w.efc}",
                      **{k: round(v, 2) for k, v in res.items()},
                      "speedup_propose": round(res["host_s"] / res["assisted_propose_s"], 2),
                      "speedup_apply": round(res["host_s"] / res["assisted_apply_s"], 2),
                      "host_cores": os.cpu_count(), "files_equal": equal}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="c2", choices=sorted(WORKLOADS),
                    help="c2: the default workload; c1, c3 and c4 (the 10M-row precision shape) print their own "
                         "JSON line")
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--target", type=float, default=0.95)
    ap.add_argument("--tune-margin", type=float, default=-1,
                    help="the tuner aims this far above --target on the held-out batch (default 0.005 for "
                         "c2 and the others, 0.02 for c4)")
    ap.add_argument("--truth-per-fraction", type=int, default=-1,
                    help="scored rows per range fraction (0: all; default all for c2, 200 for c4)")
    ap.add_argument("--ef", type=int, default=100, help="starting / no-tune beam width")
    ap.add_argument("--ef-post", type=int, default=0)
    ap.add_argument("--m", type=int, default=16)
    ap.add_argument("--cand-cap", type=int, default=512)
    ap.add_argument("--visited-cap", type=int, default=2048)
    ap.add_argument("--warps-per-block", type=int, default=4)
    ap.add_argument("--tau-a", type=int, default=-1)
    ap.add_argument("--tau-b", type=int, default=-1)
    ap.add_argument("--scan-rows", type=int, default=8192)
    ap.add_argument("--reg-budget", type=int, default=128)
    ap.add_argument("--selection", type=int, default=2, choices=[1, 2], help="hybrid selection S1 or S2")
    ap.add_argument("--rerank-mult", type=int, default=4)
    ap.add_argument("--tc-scan", type=int, default=0, choices=[0, 1], help="starting / no-tune pre-filter scan")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the BF16/FP8 lines")
    ap.add_argument("--no-extra", action="store_true", help="skip the S1 and tau-calibration lines")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--n", type=int, default=0, help="smaller base set (profiling captures only)")
    ap.add_argument("--nq", type=int, default=0, help="smaller batch (profiling captures only)")
    ap.add_argument("--scan-compare", action="store_true",
                    help="only compare the pre-filter scans on the c5 shape (its own JSON line)")
    ap.add_argument("--build-compare", action="store_true",
                    help="only compare host and GPU-assisted HSIG construction (its own JSON line)")
    args = ap.parse_args()
    if args.scan_compare:
        scan_compare(args)
        return
    if args.build_compare:
        build_compare(args)
        return
    if args.impl == "reference":
        reference_arm(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
        return
    run(args)


if __name__ == "__main__":
    main()
