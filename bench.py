#!/usr/bin/env python3
"""Benchmark: correctly rounded binary32 functions over large device arrays on GB300.

Metric: Gelem/s (elements whose correctly rounded result is stored, all functions
together) and the dominant kernel's fraction of the measured HBM roofline.

Default workload ("all19_2p26"): each of the 19 binary32 functions on its own 2^26-element
array of uniform random bit patterns restricted to the function's domain plus 1% specials
(seed 0xC0DE0000 + 256*2 + func_id).  A step evaluates every array once; inputs are
256 MiB per function, larger than the 129 MB L2, so no flush is needed between steps.
The form (--form plain|df|auto) selects the evaluation tier; results are bit-identical.

Also supported: --workload precision (expf/logf/sinf/tanhf/rsqrtf at 2^28, U[-10,10]
and log-uniform sets, both forms) and --workload expf_mixed (2^20, correctness config).

`--impl reference` times the CPU oracle (the repository's correctly rounded reference
evaluator) on a bounded sample of the same workload on the host cores.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2605_15547_gb300 import workloads as W  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def load_peaks():
    try:
        with open(PEAKS_PATH) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock and throttle reasons)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- workloads

def build_workload(name: str, scale: int, only=None):
    """Returns a list of (func, host float32 array) and a config dict."""
    items = []
    if name == "all19_2p26":
        n = (1 << 26) >> scale
        for f in W.F32_FUNCS:
            if only and f not in only:
                continue
            items.append((f, W.domain_bits(f, n, W.rng_for(2, f)).view(np.float32)))
        cfg = {"workload": f"all 19 binary32 functions, 2^{26 - scale} inputs each, domain bit patterns + 1% specials",
               "elems_per_func": n}
    elif name == "precision":
        n = (1 << 28) >> scale
        for f in ("expf", "logf", "sinf", "tanhf", "rsqrtf"):
            if only and f not in only:
                continue
            rng = W.rng_for(3, f)
            if f in ("logf", "rsqrtf"):
                items.append((f, W.loguniform(-126, 127, n, rng, signed=False)))
            else:
                items.append((f, W.uniform(-10, 10, n, rng)))
        cfg = {"workload": f"expf/logf/sinf/tanhf/rsqrtf, 2^{28 - scale} inputs each (U[-10,10]; "
                           "log-uniform [2^-126,2^127] for logf/rsqrtf)", "elems_per_func": n}
    elif name == "expf_mixed":
        n = 1 << 20
        items.append(("expf", W.expf_mixed(n, W.rng_for(1, "expf"))))
        cfg = {"workload": "expf, 2^20 inputs: 90% U[-103.98,88.73] + 10% specials", "elems_per_func": n}
    else:
        raise SystemExit(f"unknown workload {name}")
    return items, cfg


def bytes_per_elem(func: str) -> int:
    return 12 if func == "sincosf" else (16 if func in ("exp2", "log") else 8)


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    items, cfg = build_workload(args.workload, args.scale, set(args.funcs.split(",")) if args.funcs else None)
    sample = args.ref_sample
    cores = os.cpu_count() or 1
    # warm-up (constants, thread pool)
    for f, x in items[:1]:
        O.eval_bits(f, x[:1024].view(np.uint32))
    times = []
    total = 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cnt = 0
        for f, x in items:
            xs = x[:sample].view(np.uint32)
            O.eval_bits(f, xs, nthreads=cores)
            cnt += xs.size
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            total += cnt
    secs = sum(times)
    value = total / secs / 1e9
    line = {
        "impl": "reference", "metric": "Gelem/s (correctly rounded results, all functions)",
        "value": value, "unit": "Gelem/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": dict(cfg, sample_per_func=sample, l2="n/a (CPU)"),
        "cpu_baseline": {"value": value, "unit": "Gelem/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {sample} inputs of each function's array"},
        "e2e": {"value": value, "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- our arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="auto", choices=["auto", "plain", "df"])
    ap.add_argument("--workload", default="all19_2p26", choices=["all19_2p26", "precision", "expf_mixed"])
    ap.add_argument("--scale", type=int, default=0, help="divide sizes by 2^scale (testing)")
    ap.add_argument("--ref-sample", type=int, default=1 << 16)
    ap.add_argument("--cpu-sample", type=int, default=1 << 15)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--funcs", default="", help="comma list to restrict the workload (testing)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2605_15547_gb300 as crm

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as g
    g.build()

    items, cfg = build_workload(args.workload, args.scale, set(args.funcs.split(",")) if args.funcs else None)
    # drop functions the library does not provide yet (reported in the config)
    avail = []
    for f, x in items:
        t = torch.from_numpy(x[:64]).to(dev)
        try:
            crm.eval(f, t, form=args.form)
            avail.append((f, x))
        except crm.CrmError:
            pass
    missing = [f for f, _ in items if f not in {a for a, _ in avail}]
    items = avail
    dx = [torch.from_numpy(x).to(dev) for _, x in items]
    dy = [torch.empty(((2,) if f == "sincosf" else ()) + (x.size,), dtype=torch.float32, device=dev)
          for f, x in items]
    funcs = [f for f, _ in items]
    n_elems = sum(x.size for _, x in items)
    stream = torch.cuda.current_stream()

    def step():
        for f, a, b in zip(funcs, dx, dy):
            crm.eval_into(f, a, b, form=args.form)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    crm.stats_reset()
    # per-call events (the main + slow kernels of each function)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in funcs]
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        for i, (f, a, b) in enumerate(zip(funcs, dx, dy)):
            ev[s][i][0].record(stream)
            crm.eval_into(f, a, b, form=args.form)
            ev[s][i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms_total = t_start.elapsed_time(t_end)
    if world > 1:
        tt = torch.tensor([ms_total], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(tt.item())
    per_func_ms = [statistics.mean(ev[s][i][0].elapsed_time(ev[s][i][1]) for s in range(args.steps))
                   for i in range(len(funcs))]
    st = crm.stats()
    value = n_elems * args.steps * world / (ms_total / 1e3) / 1e9
    peak, peak_kind = load_peaks()
    # dominant kernel = the function whose call takes the most time
    dom = int(np.argmax(per_func_ms))
    dom_bytes = items[dom][1].size * bytes_per_elem(funcs[dom])
    achieved = dom_bytes / (per_func_ms[dom] / 1e3) / 1e9
    per_func = {f: {"gelem_s": items[i][1].size / (per_func_ms[i] / 1e3) / 1e9,
                    "hbm_frac": items[i][1].size * bytes_per_elem(f) / (per_func_ms[i] / 1e3) / 1e9 / peak}
                for i, f in enumerate(funcs)}

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    try:
        hin = [torch.from_numpy(x).pin_memory() for _, x in items]
        hout = [torch.empty(tuple(b.shape), dtype=torch.float32).pin_memory() for b in dy]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps // 2)):
            for f, a, b in zip(funcs, hin, hout):
                crm.eval_host(f, a.numpy(), b.numpy().reshape(-1), form=args.form)
        t1 = time.perf_counter()
        k = max(1, args.steps // 2)
        e2e = {"value": n_elems * k / (t1 - t0) / 1e9, "unit": "Gelem/s",
               "h2d_bytes_per_step": int(sum(x.nbytes for _, x in items)),
               "d2h_bytes_per_step": int(sum(b.numel() * 4 for b in dy))}
    except Exception as exc:  # host entry point not available
        e2e = {"value": None, "unit": "Gelem/s", "error": str(exc)[:120]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        cnt = 0
        for f, x in items:
            xs = x[:args.cpu_sample].view(np.uint32)
            O.eval_bits(f, xs, nthreads=cores)
            cnt += xs.size
        dt = time.perf_counter() - t0
        cpu = {"value": cnt / dt / 1e9, "unit": "Gelem/s", "cores": cores, "kind": "oracle",
               "sample": f"first {args.cpu_sample} inputs of each function's array"}

    launches = args.steps * len(funcs) * 2
    line = {
        "metric": "Gelem/s (correctly rounded results, all functions)",
        "value": value, "unit": "Gelem/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.form == "df" else ("f64" if args.form == "plain" else "f32"),
        "data": "synthetic",
        "config": dict(cfg, form=args.form, functions=funcs, missing=missing,
                       l2="inputs larger than L2 (no flush)", parallelism=f"replicas{world}"),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": f"k_main<{funcs[dom]}>",
                     "peak_kind": peak_kind},
        "per_function": per_func,
        "hard_case_rate": st["hard_total"] / max(1, n_elems * args.steps),
        "unresolved": st["unresolved_total"],
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
