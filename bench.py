#!/usr/bin/env python3
"""Benchmark of the GB300 vertical-bitmap Eclat hot path.

One step = the whole hot path on one synthetic database resident in HBM:
build the vertical bitmaps (item counts + bitmap build), the 1%-sample
class-cost estimate (sample build + sample mining + tally), and the mining of
every frequent itemset (pair kernel, level-2 compaction, persistent DFS),
results left in device memory.

Prints one JSON line.  `value` is the algorithmic AND+popcount throughput of
the mining in GB/s (bytes of all tidset intersections, the dense definition) over the
whole step time; `itemsets_per_s` is |F| over the same time.  `e2e` repeats the
step through the C ABI with host buffers (pinned CSR in, itemsets out).
`--impl reference` times the CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2108_05038_gb300 import synth  # noqa: E402

METRIC = "tidset AND+popc GB/s"
WORKLOAD = "large_sparse"  # the largest configuration (1M transactions, 1.25 GB of rows); --workload picks another
SAMPLE_RATE = 0.01
EST_SEED = 1
L2_FLUSH_BYTES = 512 << 20
# DRAM traffic from one ncu launch-list capture of `bench.py --workload <w> --mode once` with the metrics
# gpu__time_duration.sum, dram__bytes_read.sum and dram__bytes_write.sum (one pass; the summary under
# profiles/ gives the command and the per-kernel figures): per launch of the pair step and of the DFS
# stage, and for the whole step (build, estimate, mine).  A record is used only while the CUDA sources
# hash to the SHA-256 it was captured with; otherwise the line reports no traffic and says why.
# DRAM bytes (read + written) of one `bench.py --workload <w> --mode once` process's launches, from the ncu
# launch lists summarised in profiles/ (one-pass metrics gpu__time_duration, dram__bytes_read/write); a
# record applies only while the CUDA sources hash to the value it was captured with.  "pair": the mine's
# pair kernel; "dfs": the mine's DFS stage (projection + DFS + fallback, or the one DFS launch); "step": the
# build, estimate and mine launches (the closed/maximal flags pass of --mode once excluded).
CAPTURES = {
    "large_sparse": {"sources_sha256": "b7fa302ba7ee8f829e4355c71eb6aa41ed99fd4654012ab5e226a54ec7557371",
                     "date": "2026-12-03", "summary": "profiles/launches_large_sparse.md",
                     "kernels": {"pair": 781809664, "dfs": 1014534400}, "step": 2760817152},
    "sparse_mid": {"sources_sha256": "b7fa302ba7ee8f829e4355c71eb6aa41ed99fd4654012ab5e226a54ec7557371",
                   "date": "2026-12-03", "summary": "profiles/launches_sparse_mid.md",
                   "kernels": {"pair": 14441984, "dfs": 4328704}, "step": 48670464},
}
MAX_ITEMSETS_PER_JOB = 4_000_000  # serving: jobs whose output passes this are stopped and counted as rejected


def sources_sha256() -> str:
    """SHA-256 over the CUDA sources and the ABI header (file names and contents, in name order)."""
    import hashlib

    h = hashlib.sha256()
    base = os.path.join(ROOT, "paper_2108_05038_gb300", "csrc")
    files = sorted(f for f in os.listdir(base) if f.endswith((".cu", ".cuh")))
    for f in files + ["../../include/fim.h"]:
        h.update(f.encode())
        with open(os.path.join(base, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured(workload):
    """The DRAM-traffic record of a workload when it matches the current sources, else (None, reason)."""
    rec = CAPTURES.get(workload)
    if rec is None:
        return None, f"no ncu capture of {workload}"
    if rec["sources_sha256"] != sources_sha256():
        return None, f"the CUDA sources changed since the ncu capture of {rec['date']} ({rec['summary']})"
    return rec, f"ncu capture of {rec['date']} ({rec['summary']}), sources sha256 {rec['sources_sha256'][:12]}"


def workload_desc(w):
    if w["kind"] == "pattern":
        law = f"pattern-embedded TL={w['TL']} PL={w['PL']} npat={w['npat']} {w['popularity']} items"
    elif w["kind"] == "bernoulli":
        law = f"Bernoulli p_i={w['p_lo']}..{w['p_hi']}"
    else:
        law = f"exactly {w['k']} weighted items"
    return (f"{w['name']}: D={w['D']:,} N={w['N']:,} {law}, seed {w['seed']}, minsup {w['minsup']} "
            f"({w['rel_minsup'] * 100:.2f}%), {w['word_bits']}-bit words")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, one sample every 50 ms, each stamped with its arrival time.

    Started before the clock ramp so that it is streaming when the timed region begins; `summary`
    reports the samples that arrived during the timed region, or, when the region is shorter than
    the sampling interval, those since the ramp began (the GPU is under load throughout)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_S = 0.05

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.samples = []  # (arrival time, line)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(int(self.INTERVAL_S * 1000))],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t_load: float, t0: float, t1: float):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        inside = [ln for t, ln in self.samples if t0 <= t <= t1 + self.INTERVAL_S]
        window = "timed region"
        if not inside:
            inside = [ln for t, ln in self.samples if t_load <= t <= t1 + self.INTERVAL_S]
            window = "clock ramp + warm-up + timed region (timed region shorter than the 50 ms sampling interval)"
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in inside:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


def gather_ranks(values, dist, world: int, device: str):
    """Every rank's per-rank figures (world x k array; one row when not distributed)."""
    import torch

    per_rank = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is None or world == 1:
        return per_rank.cpu().numpy()[None, :]
    gathered = [torch.zeros_like(per_rank) for _ in range(world)]
    dist.all_gather(gathered, per_rank)
    return torch.stack(gathered).cpu().numpy()


def combine_ranks(allv):
    """Replicas (weak scaling): the job takes as long as its slowest rank; bytes and itemsets add up.
    Columns: device ms, algorithmic bytes, itemsets, end-to-end seconds."""
    return float(allv[:, 0].max()), float(allv[:, 1].sum()), float(allv[:, 2].sum()), float(allv[:, 3].max())


def run_ours(args):
    import torch

    from paper_2108_05038_gb300 import fim

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = synth.make_workload(args.workload)
    w["name"] = args.workload
    D, N, minsup, rel = w["D"], w["N"], w["minsup"], w["rel_minsup"]
    wb = w["word_bits"]
    stream = torch.cuda.current_stream()
    d_off = torch.from_numpy(w["offsets"].astype(np.int32)).cuda()
    d_items = torch.from_numpy(w["items"].astype(np.int32)).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()

    def step(collect_times=False):
        db = fim.build_vertical_db_device(d_off, d_items, D, N, wb, 0, stream=stream)
        db.estimate_class_costs(SAMPLE_RATE, rel, EST_SEED, outputs=False)
        res = db.mine(minsup, result_on_device=True, collect_times=collect_times)
        st = res.stats
        res.free()
        db.free()
        return st

    clocks = ClockSampler(local)
    clocks.start()
    # bring the SM clocks up from idle (a few hundred ms of device work) before the warm-up steps:
    # sub-millisecond steps would otherwise be timed while the clocks still ramp
    t_ramp = time.perf_counter()
    while time.perf_counter() - t_ramp < 0.3:
        flush.fill_(1)
        torch.cuda.synchronize()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms, bytes_alg, n_sets = 0.0, 0, 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = None
    wall0 = time.perf_counter()
    launches0 = fim.kernel_launches()
    step_ms = []
    for _ in range(args.steps):
        flush.fill_(1)  # write 512 MB: the 129 MB L2 holds nothing of the previous step
        e0.record(stream)
        stats = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        total_ms += step_ms[-1]
        bytes_alg += stats["bytes_algorithmic"]
        n_sets += stats["n_frequent"]
    torch.cuda.synchronize()
    launches = fim.kernel_launches() - launches0  # the library's own kernels in the timed region
    if dist:
        dist.barrier()
    t_end = time.perf_counter()
    wall = t_end - wall0
    clocks.stop()
    clk = clocks.summary(t_ramp, wall0, t_end)

    # dominant kernel: live CUDA-event timing of each launch inside the library
    pair_ms, dfs_ms, reps = [], [], max(3, args.steps)
    for _ in range(reps):
        flush.fill_(1)
        st = step(collect_times=True)
        pair_ms.append(st["ms_pair_kernel"])
        dfs_ms.append(st["ms_dfs_kernel"])
    pair_avg = sum(pair_ms) / len(pair_ms)
    dfs_avg = sum(dfs_ms) / len(dfs_ms)

    # end to end through the C ABI with host buffers (pinned CSR in, itemsets out)
    h_off = torch.from_numpy(w["offsets"]).pin_memory()
    h_items = torch.from_numpy(w["items"]).pin_memory()
    e2e_s, d2h = 0.0, 0
    for k in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        db = fim.build_vertical_db(h_off.numpy(), h_items.numpy(), N, wb, 0, stream=stream)
        db.estimate_class_costs(SAMPLE_RATE, rel, EST_SEED, outputs=False)
        res = db.mine(minsup)
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_s += t1 - t0
            d2h = res.set_offsets.nbytes + res.set_items.nbytes + res.supports.nbytes
        db.free()
    h2d = int(w["offsets"].nbytes + w["items"].nbytes)

    # max over ranks
    allv = gather_ranks([total_ms, bytes_alg, n_sets, e2e_s], dist, world, "cuda")
    max_ms, tot_bytes, tot_sets, max_e2e = combine_ranks(allv)

    out = None
    if rank == 0:
        value = tot_bytes / (max_ms * 1e-3) / 1e9
        peaks = {}
        pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(pk_path):
            peaks = json.load(open(pk_path))
        sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        num_sms = torch.cuda.get_device_properties(local).multi_processor_count
        # integer-pipe roofline of AND+POPC on word pairs: 64 LOP3 lanes/clk/SM and 32 POPC lanes/clk/SM;
        # every scheme trades two LOP3 for one POPC, and the balanced mix (1.5 LOP3 + 0.75 POPC per word)
        # reaches 42.67 words/clk/SM on both pipes
        alu_peak_gword = 128.0 / 3.0 * num_sms * sm_max_mhz * 1e6 / 1e9
        words = stats["n_pair_intersections"] * ((D + 31) // 32)  # algorithmic 32-bit word pairs
        achieved_gword = words / (pair_avg * 1e-3) / 1e9
        rec, rec_note = captured(args.workload)
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        hbm_src = "measured copy rate (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
        if dfs_avg > pair_avg:  # the DFS stage dominates: its operand bytes against the measured copy rate
            proj = stats.get("bytes_projected", 0) > 0
            alg = stats["bytes_projected"] if proj else stats["bytes_dfs_kernel"]
            dfs_gbs = alg / (dfs_avg * 1e-3) / 1e9
            roofline = {"kernel": ("k_proj_tids + k_proj_bits + k_dfs_proj (+ k_dfs_sparse on the classes left out)"
                                   if proj else "k_dfs"),
                        "bound": "hbm", "achieved": round(dfs_gbs, 1), "peak": round(hbm, 1),
                        "unit": "GB/s", "frac": round(dfs_gbs / hbm, 4),
                        "traffic": rec["kernels"]["dfs"] if rec else None, "traffic_source": rec_note,
                        "peak_source": hbm_src,
                        "note": ("algorithmic bytes of the projected DFS in its own representation (stats "
                                 "bytes_projected): each class database part built (row read, one word gathered "
                                 "per survivor and transaction, bitmaps written) and per class node its prefix and "
                                 "candidates over its region's width; the regions (tens of MB) stay in the 129 MB L2"
                                 if proj else
                                 "algorithmic bytes count every candidate row in full (the dense definition); the "
                                 "kernel reads row words only under nonzero prefix words")}
        elif stats.get("pair_kernel") in (2, 3, 4):  # level 2 on the tensor cores: the 0/1 contraction, kind::f8f6f4
            flops = 2.0 * stats["n_pair_intersections"] * D  # one multiply-add per pair and transaction
            tf = flops / (pair_avg * 1e-3) / 1e12
            peak = 2.0 * float(peaks.get("bf16_tflops", 1900.0))
            kname = {2: "k_expand_e2m1 + k_pair_mma", 3: "k_expand_e4m3 + k_pair_mma",
                     4: "k_pair_mma_fused"}[stats["pair_kernel"]]
            roofline = {"kernel": kname, "bound": "tensor", "achieved": round(tf, 1),
                        "peak": round(peak, 1), "unit": "TFLOP/s", "frac": round(tf / peak, 4),
                        "traffic": rec["kernels"]["pair"] if rec else None, "traffic_source": rec_note,
                        "peak_source": ("kind::f8f6f4 (e2m1 and e4m3 operands alike) at the fp8 dense rate = 2 x the "
                                        "measured bf16 burst (MEASURED_PEAKS.json bf16_tflops; nominal fp8:bf16 = 4.5:2.25)" if "bf16_tflops" in peaks
                                        else "fallback 1.9 PFLOP/s bf16 x 2"),
                        "note": "algorithmic flops: 2 x pairs i<j x transactions; the time includes widening "
                                "the rows to the operand form (inside the kernel when fused)"}
        else:
            roofline = {"kernel": "k_pair_counts", "bound": "alu", "achieved": round(achieved_gword, 1),
                        "peak": round(alu_peak_gword, 1), "unit": "Gword/s",
                        "frac": round(achieved_gword / alu_peak_gword, 4),
                        "traffic": rec["kernels"]["pair"] if rec else None, "traffic_source": rec_note,
                        "peak_source": "derived: (64 LOP3 + 32 POPC lanes/clk/SM) -> 42.67 word pairs/clk/SM x SMs "
                                       "x max SM clock"}
        ms_step = max_ms / args.steps
        dram = {"bytes_per_step": rec["step"] if rec else None, "source": rec_note}
        if rec:
            dram["gbs"] = round(rec["step"] / (ms_step * 1e-3) / 1e9, 1)
            dram["frac_of_hbm"] = round(dram["gbs"] / hbm, 4)
            dram["note"] = "DRAM bytes of one step's launches (ncu) over this run's ms_per_step"
        out = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(max_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {1: "u32", 2: "u32 + e2m1 (level-2 0/1 products, f32 sums)",
                      3: "u32 + e4m3 (level-2 0/1 products, f32 sums)",
                      4: "u32 + e4m3 (level-2 0/1 products widened in shared memory, f32 sums)"}.get(
                          stats.get("pair_kernel", 1), "u32"),
            "data": "synthetic",
            "config": {"workload": workload_desc(w), "sample_rate": SAMPLE_RATE,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "512 MB buffer written between timed steps"},
            "itemsets_per_s": round(tot_sets / (max_ms * 1e-3), 1),
            "n_frequent": int(stats["n_frequent"]),
            "breakdown_ms": {"pair_kernel": round(pair_avg, 4), "dfs_kernel": round(dfs_avg, 4),
                             "step": round(max_ms / args.steps, 4),
                             "step_min": round(min(step_ms), 4), "step_median": round(statistics.median(step_ms), 4),
                             "step_max": round(max(step_ms), 4)},
            "roofline": roofline,
            "dram": dram,
            "value_note": "value counts the dense-definition bytes of every intersection (a work rate: words that "
                          "the kernels skip or read from projected bitmaps count in full); dram gives the HBM "
                          "fraction of the step",
            "e2e": {"value": round(tot_bytes / max_e2e / 1e9, 2), "unit": "GB/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": round(max_e2e / args.steps * 1e3, 3)},
            "gpu_launches": int(launches),
            "clocks": clk,
            "wall_s": round(wall, 3),
        }
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(w, stats["bytes_algorithmic"], args.workload)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if out is not None and world == 1 and not args.no_legs:
        # the two systems forms, measured in the same run: one mine of the deep dense workload captured in a
        # CUDA graph and replayed, and the served request loop against the plain loop (a prefix of the
        # 2,000-request serving workload, same laws and arrival rate)
        out["legs"] = {"plan": run_plan(args, workload="dense_deep", steps=max(args.steps, 20)),
                       "serve": run_serve(args, n_requests=args.serve_requests)}
    return out


def run_plan(args, workload=None, steps=None):
    """Graph replays of one captured mine (batched mode): all prefix classes in one persistent launch."""
    import torch

    from paper_2108_05038_gb300 import fim

    torch.cuda.set_device(0)
    workload = workload or args.workload
    w = synth.make_workload(workload)
    w["name"] = workload
    args_steps = steps or args.steps
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], w["word_bits"], 0, stream=s)
    db.estimate_class_costs(SAMPLE_RATE, w["rel_minsup"], EST_SEED)
    shape, tuned_ms = db.autotune(w["minsup"])
    plan = db.plan(w["minsup"], shape=shape, result_on_device=True)
    for _ in range(args.warmup):
        plan.launch()
    res = plan.result(result_on_device=True)
    st = res.stats
    res.free()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    launches0 = fim.kernel_launches()
    for _ in range(args_steps):
        with torch.cuda.stream(s):
            flush.fill_(1)
            e0.record(s)
        plan.launch()
        e1.record(s)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    ms = total / args_steps
    launches = fim.kernel_launches() - launches0
    plan.free()
    db.free()
    return {"metric": METRIC, "value": round(st["bytes_algorithmic"] / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "n_gpus": 1, "steps": args_steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "mode": "plan (CUDA-graph replay of one mine; build and estimate once before timing)",
            "config": {"workload": workload_desc(w), "shape": shape, "autotuned_ms": round(tuned_ms, 4),
                       "l2": "512 MB buffer written before each replay"},
            "itemsets_per_s": round(st["n_frequent"] / (ms * 1e-3), 1), "n_frequent": st["n_frequent"],
            "n_classes": st["n_classes"], "n_queue_entries": st["n_queue_entries"], "gpu_launches": int(launches)}


def run_balance(args):
    """Estimator fidelity (the thesis's Exp. 1/2 on one GPU): estimated vs actual class costs, and the
    persistent DFS's time and per-CTA load imbalance under each class order."""
    import torch

    from paper_2108_05038_gb300 import fim

    torch.cuda.set_device(0)
    w = synth.make_workload(args.workload)
    w["name"] = args.workload
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], w["word_bits"], 0)
    ms = w["minsup"]

    def run(order, reps):
        best = None
        for _ in range(reps):
            flush.fill_(1)
            torch.cuda.synchronize()
            res = db.mine(ms, class_order=order, collect_times=True, result_on_device=True, class_work=True)
            st = res.stats
            cw = res.class_work.astype(np.float64)
            res.free()
            if best is None or st["ms_dfs_kernel"] < best[0]["ms_dfs_kernel"]:
                best = (st, cw)
        st, cw = best
        return {"dfs_ms": round(st["ms_dfs_kernel"], 4),
                "cta_busy_max_ms": round(st["dfs_cta_busy_max_ms"], 4),
                "cta_busy_mean_ms": round(st["dfs_cta_busy_mean_ms"], 4),
                "imbalance_max_over_mean": round(st["dfs_cta_busy_max_ms"] / max(st["dfs_cta_busy_mean_ms"], 1e-9), 3)}, cw

    def ranks(v):  # average ranks for ties
        order = np.argsort(v, kind="stable")
        r = np.empty(len(v))
        sv = v[order]
        i = 0
        while i < len(v):
            j = i
            while j + 1 < len(v) and sv[j + 1] == sv[i]:
                j += 1
            r[order[i:j + 1]] = (i + j) / 2.0
            i = j + 1
        return r

    def fidelity(est, actual):
        m = actual > 0
        e, a = est[m], actual[m] / actual[m].sum()
        pear = float(np.corrcoef(e, a)[0, 1]) if m.sum() > 1 else float("nan")
        spear = float(np.corrcoef(ranks(e), ranks(a))[0, 1]) if m.sum() > 1 else float("nan")
        k = max(1, int(0.05 * m.sum()))
        top = len(set(np.argsort(-e)[:k]) & set(np.argsort(-a)[:k])) / k
        return {"pearson": round(pear, 4), "spearman": round(spear, 4), "top5pct_overlap": round(top, 3),
                "abs_share_error_sum": round(float(np.abs(e - a).sum()), 4)}

    reps = max(3, args.steps)
    out = {"metric": "estimator fidelity and DFS load balance", "mode": "balance", "data": "synthetic", "n_gpus": 1,
           "config": {"workload": workload_desc(w), "sample_rate": SAMPLE_RATE, "reps": reps}}
    uni, actual = run("uniform", reps)
    out["uniform_order"] = uni
    out["actual_classes"] = int((actual > 0).sum())
    out["actual_top_class_share"] = round(float(actual.max() / actual.sum()), 4)
    for kind in ("itemsets", "intersections"):
        cost, _ = db.estimate_class_costs(SAMPLE_RATE, w["rel_minsup"], EST_SEED, cost=kind)
        r, _ = run("estimate", reps)
        r["fidelity"] = fidelity(np.asarray(cost, dtype=np.float64), actual)
        out[f"estimate_{kind}"] = r
    db.free()
    return out


def run_once(args):
    """One build + one mine of a workload, nothing else (for profiler captures): with --no-estimate the
    mine's kernels are the first of their kind in the process."""
    import torch

    from paper_2108_05038_gb300 import fim

    torch.cuda.set_device(0)
    w = synth.make_workload(args.workload, D=args.D)
    w["name"] = args.workload
    d_off = torch.from_numpy(w["offsets"].astype(np.int32)).cuda()
    d_items = torch.from_numpy(w["items"].astype(np.int32)).cuda()
    db = fim.build_vertical_db_device(d_off, d_items, w["D"], w["N"], w["word_bits"], 0)
    if not args.no_estimate:
        db.estimate_class_costs(SAMPLE_RATE, w["rel_minsup"], EST_SEED, outputs=False)
    res = db.mine(w["minsup"], result_on_device=True, collect_times=True)
    st = res.stats
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fl = res.flags()  # closed and maximal itemsets of the result (fim_result_flags)
    t_flags = time.perf_counter() - t0
    res.free()
    db.free()
    return {"mode": "once", "config": {"workload": workload_desc(w), "estimate": not args.no_estimate},
            "closed": int((fl & 1).sum()), "maximal": int((fl & 2).sum() // 2),
            "ms_result_flags": round(t_flags * 1e3, 3),
            "n_frequent": st["n_frequent"], "n_intersections": st["n_intersections"],
            "ms_pair_kernel": round(st["ms_pair_kernel"], 4), "ms_dfs_kernel": round(st["ms_dfs_kernel"], 4),
            "bytes_pair_kernel": st["bytes_pair_kernel"], "bytes_dfs_kernel": st["bytes_dfs_kernel"],
            "gpu_launches": fim.kernel_launches()}


def run_stream(args):
    """Streaming microbenchmark of the counting step on its own: supp({0, c}) for every item c of a
    database of 8,388,608 transactions over 4,096 items whose item 0 is in every transaction.  t({0})
    is dense (1 MiB, held in L2), so the call streams all 4,096 candidate rows (4 GiB, far above the
    129 MB L2) from HBM once.  Closed form checked on every call's output: supp({0, c}) = supp(c)."""
    import torch

    from paper_2108_05038_gb300 import fim

    torch.cuda.set_device(0)
    D, N = args.D or 8_388_608, 4096
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    lens = torch.randint(0, 9, (D,), device="cuda", generator=g, dtype=torch.int64) + 1  # item 0 + 0..8 others
    off = torch.zeros(D + 1, dtype=torch.int64, device="cuda")
    off[1:] = torch.cumsum(lens, 0)
    nnz = int(off[-1])
    items = torch.randint(1, N, (nnz,), device="cuda", generator=g, dtype=torch.int32)
    items[off[:-1]] = 0
    off = off.to(torch.int32)
    stream = torch.cuda.current_stream()
    db = fim.build_vertical_db_device(off, items, D, N, 64, 0, stream=stream)
    kept, supp = db.rows()
    info = db.info()
    row_bytes = info["words_per_row"] * 4
    alg_bytes = len(kept) * ((D + 7) // 8)  # candidate rows: the D bits each, read once

    clocks = ClockSampler(0)
    clocks.start()
    t_ramp = time.perf_counter()
    while time.perf_counter() - t_ramp < 0.3:
        db.extension_supports([0], kept)
    for _ in range(args.warmup):
        db.extension_supports([0], kept)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, bad = [], 0
    launches0 = fim.kernel_launches()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        e0.record(stream)
        got = db.extension_supports([0], kept)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        bad += int(np.count_nonzero(got != supp))
    t_end = time.perf_counter()
    launches = fim.kernel_launches() - launches0
    clocks.stop()
    clk = clocks.summary(t_ramp, wall0, t_end)
    # a two-item prefix adds the AND of two rows into scratch before the stream
    e0.record(stream)
    got2 = db.extension_supports([0, int(kept[-1])], kept)
    e1.record(stream)
    e1.synchronize()
    ms2 = e0.elapsed_time(e1)
    db.free()
    avg = sum(ms) / len(ms)
    gbs = alg_bytes / (avg * 1e-3) / 1e9
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    return {"mode": "stream", "metric": "extension-support stream GB/s", "value": round(gbs, 1), "unit": "GB/s",
            "steps": args.steps, "warmup": args.warmup, "ms_per_call": round(avg, 4),
            "ms_min": round(min(ms), 4), "ms_max": round(max(ms), 4), "higher_is_better": True, "dtype": "u32",
            "data": "synthetic, generated on the device",
            "config": {"workload": f"D={D} transactions, N={N} items, item 0 in all, 1-9 items per transaction",
                       "candidates": int(len(kept)), "row_bytes": int(row_bytes),
                       "bitmap_bytes": int(len(kept) * row_bytes),
                       "l2": "inputs (4 GiB of rows) far larger than the 129 MB L2"},
            "verified": bad == 0 and bool(np.all(got2 <= supp)),
            "two_item_prefix_ms": round(ms2, 4),
            "roofline": {"kernel": "k_extension_counts", "bound": "hbm", "achieved": round(gbs, 1),
                         "peak": round(hbm, 1), "unit": "GB/s", "frac": round(gbs / hbm, 4), "traffic": None,
                         "timing": "CUDA events around the whole call (rows H2D, kernel, counts D2H, host sync)",
                         "peak_source": "measured copy rate (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks
                         else "fallback 6.8 TB/s"},
            "gpu_launches": int(launches), "clocks": clk}


def _gen_request(r):
    off, items = synth.request_db(r)
    return off, items


def result_digest(res):
    """Order-independent digest of a host result: (itemsets, sum over itemsets of a 64-bit mix of the
    itemset's items and support).  Equal results give equal digests whatever their record order."""
    n = res.n_sets
    if n == 0:
        return (0, 0)
    so = res.set_offsets.astype(np.int64)
    it = res.set_items.astype(np.uint64)
    m = np.uint64(0xbf58476d1ce4e5b9)
    with np.errstate(over="ignore"):
        h = (it + np.uint64(0x9e3779b97f4a7c15)) * m
        h ^= h >> np.uint64(31)
        h *= np.uint64(0x94d049bb133111eb)
        per_set = np.add.reduceat(h, so[:-1]) if len(it) else np.zeros(n, dtype=np.uint64)
        per_set = (per_set ^ (res.supports.astype(np.uint64) * m)) * np.uint64(0x94d049bb133111eb)
        per_set ^= per_set >> np.uint64(29)
        return (int(n), int(per_set.sum(dtype=np.uint64)))


def serve_arm(reqs, dbs, slots):
    """Requests submitted at their arrival times to a server with `slots` slots; results collected in a
    second thread.  Returns latencies (s), per-request digests (None = rejected over the itemset limit),
    the makespan, the peak of jobs in flight and the service times."""
    import threading

    from paper_2108_05038_gb300 import fim

    srv = fim.Server(slots=slots, ctas_per_sm=1, max_itemsets=MAX_ITEMSETS_PER_JOB)
    for k in range(min(4, len(reqs))):  # warm the library (kernels loaded, pools primed)
        srv.wait(srv.submit(dbs[k][0], dbs[k][1], reqs[k]["N"], reqs[k]["minsup"], SAMPLE_RATE))[0].free()
    lat, dig, svc = [None] * len(reqs), [None] * len(reqs), [0.0] * len(reqs)
    ids = [None] * len(reqs)
    ready = threading.Semaphore(0)

    def collector():
        for k in range(len(reqs)):
            ready.acquire()
            try:
                res, l, sv = srv.wait(ids[k])
                dig[k] = result_digest(res)
                svc[k] = sv
                res.free()
            except fim.FimError as e:
                if e.status != fim.FIM_ERR_OUTPUT_OVERFLOW:
                    raise
                l = time.perf_counter() - t0 - reqs[k]["arrival_s"]
            lat[k] = l
            if (k + 1) % 100 == 0:
                print(f"slots={slots}: served {k + 1}/{len(reqs)} at {time.perf_counter() - t0:.1f} s",
                      file=sys.stderr, flush=True)

    th = threading.Thread(target=collector)
    th.start()
    t0 = time.perf_counter()
    for k, r in enumerate(reqs):
        delay = t0 + r["arrival_s"] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        ids[k] = srv.submit(dbs[k][0], dbs[k][1], r["N"], r["minsup"], SAMPLE_RATE)
        ready.release()
    th.join()
    span = time.perf_counter() - t0
    peak = srv.stats()["peak_in_flight"]
    srv.free()
    return lat, dig, span, peak, svc


def run_serve(args, n_requests=None):
    """Serving: Poisson arrivals of mining requests on their own databases; p50/p99 latency and itemsets/s of
    the continuous-batching server (`--slots` slots) against the plain one-job-at-a-time loop, which is the
    same server with one slot, so both arms run the same C++ worker code and differ only in batching."""
    import multiprocessing as mp

    reqs = synth.serving_requests(n_requests or args.requests, rate=args.rate)
    with mp.get_context("spawn").Pool(max(1, (os.cpu_count() or 4) - 2)) as pool:  # before any CUDA call
        dbs = pool.map(_gen_request, reqs, chunksize=4)
    import torch

    torch.cuda.set_device(0)

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(round(q / 100 * (len(v) - 1))))]

    def summary(lat, dig, span, peak, svc, slots):
        sets = sum(d[0] for d in dig if d is not None)
        slow = sorted(range(len(reqs)), key=lambda k: -svc[k])[:3]
        return {"slots": slots, "p50_ms": round(pct(lat, 50) * 1e3, 2), "p99_ms": round(pct(lat, 99) * 1e3, 2),
                "itemsets_per_s": round(sets / span, 1), "makespan_s": round(span, 2), "peak_in_flight": peak,
                "rejected_over_limit": sum(1 for d in dig if d is None),
                "slowest_service": [{"k": k, "D": reqs[k]["D"], "N": reqs[k]["N"], "minsup": reqs[k]["minsup"],
                                     "service_ms": round(svc[k] * 1e3, 1)} for k in slow]}

    served_raw = serve_arm(reqs, dbs, args.slots)
    plain_raw = serve_arm(reqs, dbs, 1)
    same = [a == b for a, b in zip(served_raw[1], plain_raw[1])]
    served, plain = summary(*served_raw, args.slots), summary(*plain_raw, 1)
    return {"metric": "served p50/p99 latency vs plain loop", "value": served["p99_ms"], "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "mode": "serve", "data": "synthetic",
            "config": {"requests": len(reqs), "rate_per_s": args.rate, "slots": args.slots,
                       "sample_rate": SAMPLE_RATE, "max_itemsets_per_job": MAX_ITEMSETS_PER_JOB,
                       "workload": "pattern-embedded, D log-uniform [1e4, 5e5], N uniform [100, 5000], "
                                   "TL uniform [5, 30], PL 4, npat 2N, minsup log-uniform [0.1%, 5%], "
                                   "request seed 1000+k, Poisson arrivals"},
            "served": served, "plain_loop": plain,
            "per_request_equal": all(same), "requests_differing": [k for k, x in enumerate(same) if not x][:10],
            "n_frequent_total": int(sum(d[0] for d in served_raw[1] if d is not None))}


ORACLE_MAX_D = 200_000  # larger workloads: the oracle mines a prefix sample (its full mine takes many minutes)
ORACLE_SAMPLE_D = 50_000


def oracle_sample(w):
    """The workload itself, or for large databases its first ORACLE_SAMPLE_D transactions mined at the same
    relative minsup; returns (offsets, items, D, minsup, description)."""
    if w["D"] <= ORACLE_MAX_D:
        return w["offsets"], w["items"], w["D"], w["minsup"], f"one full oracle Eclat mine of {w['name']}"
    Ds = ORACLE_SAMPLE_D
    off = w["offsets"][: Ds + 1]
    items = w["items"][: int(off[-1])]
    ms = synth.abs_minsup(w["rel_minsup"], Ds)
    return off, items, Ds, ms, (f"oracle Eclat mine of the first {Ds:,} transactions of {w['name']} at the same "
                                f"relative minsup ({ms})")


def oracle_bytes(off, items, N, D, minsup, word_bits=64):
    """Algorithmic bytes of the bitmap path for a database, computed from the oracle's own output."""
    import oracle

    so, si, sp = oracle.eclat(off, items, N, minsup)
    order = oracle.item_order(off, items, N, 0)
    item_rank = np.zeros(N, dtype=np.int64)
    item_rank[order] = np.arange(len(order))
    I, C, M = bitmap_work(so, si, item_rank)
    return (I + C + M) * ((D + word_bits - 1) // word_bits * (word_bits // 8)), len(sp)


def host_cpu():
    """The host CPU as a short string (architecture and model), for the CPU-baseline records."""
    import platform

    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key, _, val = line.partition(":")
                if key.strip() in ("model name", "CPU part") and val.strip():
                    model = val.strip()
                    break
    except OSError:
        pass
    return f"{platform.machine()} {model}".strip()


def cpu_baseline(w, bytes_alg_per_step, name):
    """The oracle as it stands, on the host, on the same workload (one full mine; a prefix sample of large
    databases): on every host core (one-item classes spread over threads) and on one core."""
    import oracle

    off, items, D, ms, desc = oracle_sample(w)
    if D != w["D"]:
        bytes_alg_per_step, _ = oracle_bytes(off, items, w["N"], D, ms, w["word_bits"])
    cores = os.cpu_count() or 1

    def median_time(fn, budget_s):  # up to 5 runs within the time budget (at least one): their median
        times = []
        while len(times) < 5 and (not times or sum(times) + times[-1] <= budget_s):
            t0 = time.perf_counter()
            out = fn()
            times.append(time.perf_counter() - t0)
        return sorted(times)[len(times) // 2], len(times), out

    dt, n_mt, (so, si, sp) = median_time(lambda: oracle.eclat_mt(off, items, w["N"], ms, cores), 5.0)
    dt1, n_1, _ = median_time(lambda: oracle.eclat(off, items, w["N"], ms), 10.0)
    return {"value": round(bytes_alg_per_step / dt / 1e9, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "cpu": host_cpu(), "sample": f"{desc} ({len(sp)} itemsets) in {dt:.2f} s on {cores} threads ({dt1:.2f} s on one); "
                      f"medians of {n_mt} and {n_1} runs; GB/s counts the bitmap path's algorithmic bytes for the "
                      f"same answer",
            "itemsets_per_s": round(len(sp) / dt, 1),
            "single_core": {"value": round(bytes_alg_per_step / dt1 / 1e9, 4), "unit": "GB/s", "cores": 1,
                            "itemsets_per_s": round(len(sp) / dt1, 1)}}


def run_reference(args):
    """--impl reference: the CPU oracle timed on the host cores, same workload and metric."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle

    w = synth.make_workload(args.workload)
    w["name"] = args.workload
    off, items, D, ms, desc = oracle_sample(w)
    bytes_alg, n_sets = oracle_bytes(off, items, w["N"], D, ms, w["word_bits"])
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.eclat_mt(off, items, w["N"], ms, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.eclat_mt(off, items, w["N"], ms, cores)
    dt = time.perf_counter() - t0
    value = bytes_alg * args.steps / dt / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload_desc(w)},
            "itemsets_per_s": round(n_sets * args.steps / dt, 1),
            "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "cpu": host_cpu(), "sample": f"{desc} per step ({n_sets} itemsets), one-item classes over {cores} "
                                       f"threads"},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def bitmap_work(so, si, item_rank):
    """Work of the bitmap Eclat for a given output, from the output alone.

    Classes are formed in row order (ascending support, ties by id).  With k_P =
    number of frequent itemsets P u {e}, e after P's last item:
    intersections I = n1(n1-1)/2 + sum_{|P|>=1} k_P(k_P-1)/2, class nodes with
    candidates C = (n1-1) + sum_{|P|>=1} (k_P-1)+, materialised prefixes
    M = #{X : |X| >= 2, k_X >= 2}.  Algorithmic bytes = (I + C + M) x row bytes."""
    groups = {}
    n1 = 0
    for k in range(len(so) - 1):
        s = tuple(sorted(int(item_rank[v]) for v in si[so[k]:so[k + 1]]))
        if len(s) == 1:
            n1 += 1
        else:
            groups[s[:-1]] = groups.get(s[:-1], 0) + 1
    I = n1 * (n1 - 1) // 2 + sum(k * (k - 1) // 2 for k in groups.values())
    C = max(n1 - 1, 0) + sum(max(k - 1, 0) for k in groups.values())
    M = sum(1 for p, k in groups.items() if len(p) >= 2 and k >= 2)
    return I, C, M


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--no-estimate", action="store_true", help="--mode once: mine without a sample estimate")
    ap.add_argument("--D", type=int, default=None, help="--mode once: the workload's laws at another D; --mode stream: transactions")
    ap.add_argument("--mode", default="step", choices=["step", "plan", "serve", "balance", "once", "stream"],
                    help="step: build+estimate+mine per step (default); plan: graph replays of one captured "
                         "mine; serve: the request loop against the plain one-job-at-a-time loop; balance: "
                         "estimated vs actual class costs and the DFS load balance per class order; once: one "
                         "build + mine (profiler captures); stream: the counting step alone over 4 GiB of "
                         "bitmap rows")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving leg of the default run (config 4 in full: about 100 s per arm)")
    ap.add_argument("--no-legs", action="store_true", help="default run: skip the plan and serving legs")
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--slots", type=int, default=4)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        out = run_reference(args)
    elif args.mode == "plan":
        out = run_plan(args)
    elif args.mode == "serve":
        out = run_serve(args)
    elif args.mode == "balance":
        out = run_balance(args)
    elif args.mode == "once":
        out = run_once(args)
    elif args.mode == "stream":
        out = run_stream(args)
    else:
        out = run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
