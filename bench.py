"""Benchmark: full-inventory Wide & Deep scoring + top-K of single requests.

Workload (default): 2,000,000 ads, d = 64 FP32 embeddings, 16 user x 16 ad
fields, 64 cross pairs, hashed 2^24 cross-weight table, K = 500 (the plain FP32
single-request path at inventory scale).  A step is one request through the
whole hot path: query expansion, the wide term via the compressed inverted list
(Algorithm 2), the streaming inner product with the fused wide add and top-K,
and the final selection.

Prints one JSON line.  `value` is ads scored per second with inputs resident in
device memory; `e2e` is the same metric through the C ABI with host buffers
(host->device copy of the request and device->host copy of the K results inside
the timed region).  Between timed steps the L2 cache is flushed by writing a
256 MiB buffer (outside the per-step events).

--impl reference times the FP64 CPU oracle on the host cores instead.
--gpus N (under torchrun): N independent replicas, one per GPU; the path has no
cross-GPU exchange, so `value` sums the replicas' throughput (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2511_22460_gb300.datagen import make_workload  # noqa: E402

WORKLOAD = "single_fp32_2m"
METRIC = "ads scored/s"
UNIT = "ads/s"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _config(w, extra=None):
    r = w.recipe
    cfg = {"workload": r.name, "n_ads": r.n_ads, "d": r.d, "emb_dtype": r.emb_dtype,
           "user_fields": r.f_u, "ad_fields": r.f_a, "cross_pairs": int(len(w.pairs)),
           "weights": "hashed 2^24 FP32" if r.weights == "hashed" else "dense per pair",
           "k": int(w.ks[0]), "n_keys": w.n_keys, "postings": w.nnz,
           "l2": "flushed between steps (256 MiB write); embedding table 512 MB > L2"}
    if extra:
        cfg.update(extra)
    return cfg


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_2511_22460_gb300 import ebr

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    st = torch.cuda.current_stream()
    w = make_workload(args.workload, seed=args.seed)
    pk, pa = w.postings()
    ix = ebr.build_index(w.n_ads, w.n_keys, pk, pa, w.emb, dtype=w.recipe.emb_dtype,
                         device=local_rank)
    del pk, pa
    cross = ebr.cross_from_workload(w, device=local_rank)
    info = ix.info()
    k = int(w.ks[0])
    nreq = w.users.shape[0]
    h_u = torch.from_numpy(w.h_u).to(dev)
    users = torch.from_numpy(w.users).to(dev)
    ids = torch.empty(k, dtype=torch.int32, device=dev)
    sc = torch.empty(k, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(i):
        b = i % nreq
        ebr.score_topk(ix, cross, [ebr.Query(h_u=h_u[b], k=k, user_vals=users[b])], ids, sc,
                       stream=st)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    ix.profile_enable(True)
    launches0 = ix.profile_read().launches
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(st)
        step(i)
        evs[i][1].record(st)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    times = [a.elapsed_time(b) for a, b in evs]
    prof = ix.profile_read()
    ix.profile_enable(False)
    total_ms = float(sum(times))
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / args.steps
    value = w.n_ads * args.steps * world / (total_ms / 1e3)

    # End to end through the C ABI with host buffers (request in, K results out).
    hk_ids = np.empty(k, np.uint32)
    hk_sc = np.empty(k, np.float32)
    h_hu = w.h_u.copy()
    h_users = w.users.copy()
    e2e_t = []
    for i in range(args.warmup + args.steps):
        b = i % nreq
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ebr.score_topk(ix, cross, [ebr.Query(h_u=h_hu[b], k=k, user_vals=h_users[b])], hk_ids,
                       hk_sc, io=ebr.IO_HOST, stream=st)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_t.append(t1 - t0)
    e2e_val = w.n_ads * len(e2e_t) / sum(e2e_t)

    peak, peak_kind = _peaks()
    scan_ms = prof.ms_scan / max(prof.calls, 1)
    emb_bytes = info.emb_bytes
    # the fused scan must read the embedding table and the window-major view of
    # the compressed lists (keys + value bytes + window offsets)
    kern_bytes = emb_bytes + info.window_view_bytes
    achieved = kern_bytes / (scan_ms / 1e3) / 1e9
    step_bytes = kern_bytes
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "scan_traffic.json")
    if os.path.exists(tr_path):
        with open(tr_path) as f:
            tr = json.load(f)
        if tr.get("workload") == args.workload and tr.get("kernel_rev") == KERNEL_REV:
            traffic = tr.get("bytes_per_launch")
    launches_per_step = (prof.launches - launches0) / max(args.steps, 1)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(w, {"replicas": world, "build_ms": round(info.build_ms, 3),
                              "window_view_ms": round(info.window_view_ms, 3),
                              "index_bytes": info.index_bytes,
                              "window_view_bytes": info.window_view_bytes}),
        "latency_us": {"p50": 1e3 * float(np.percentile(times, 50)),
                       "p99": 1e3 * float(np.percentile(times, 99))},
        "req_per_s": 1e3 / ms_step * world,
        "step_hbm_gbs": step_bytes / (ms_step / 1e3) / 1e9,
        "stage_ms": {"expand": prof.ms_expand / prof.calls, "wide": prof.ms_wide / prof.calls,
                     "scan_topk": scan_ms, "final": prof.ms_final / prof.calls},
        "roofline": {"kernel": "k_fused_window", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": traffic,
                     "algorithmic_bytes": kern_bytes,
                     "bytes_note": "embedding table + window-major view of the compressed "
                                   "lists, per launch"},
        "e2e": {"value": e2e_val, "unit": UNIT,
                "h2d_bytes_per_step": int(w.recipe.d * 4 + w.recipe.f_u * 4),
                "d2h_bytes_per_step": int(k * 8)},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "gpu_launches_per_step": launches_per_step,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, budget_s=args.cpu_budget)
    return out


KERNEL_REV = "fused-v1"


def cpu_baseline(w, budget_s=15.0):
    """FP64 oracle (expansion + postings walk + dot + full sort) on the host."""
    import oracle
    cross = oracle.Cross.from_workload(w)
    pk, pa = w.postings()
    k = int(w.ks[0])
    t_total, n = 0.0, 0
    while t_total < budget_s and n < 64:
        b = n % w.users.shape[0]
        t0 = time.perf_counter()
        s = oracle.score_query(w, b, cross, (pk, pa))
        oracle.topk(s, k)
        t_total += time.perf_counter() - t0
        n += 1
    return {"value": w.n_ads * n / t_total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d full requests of the %s workload (%d ads each), single thread" % (
                n, w.recipe.name, w.n_ads)}


def run_reference(args):
    w = make_workload(args.workload, seed=args.seed)
    import oracle
    cross = oracle.Cross.from_workload(w)
    pk, pa = w.postings()
    k = int(w.ks[0])
    for i in range(args.warmup):
        s = oracle.score_query(w, i % w.users.shape[0], cross, (pk, pa))
        oracle.topk(s, k)
    t = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        s = oracle.score_query(w, i % w.users.shape[0], cross, (pk, pa))
        oracle.topk(s, k)
        t.append(time.perf_counter() - t0)
    value = w.n_ads * len(t) / sum(t)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / len(t),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference", "config": _config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d full requests, single thread" % len(t)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out = run_gpu(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
