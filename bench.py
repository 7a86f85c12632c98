#!/usr/bin/env python3
"""Benchmark: correctly rounded binary32 functions over large device arrays on GB300.

Metric: Gelem/s of correctly rounded results (every result bit-exact against the CPU
oracle, which the GPU test suite checks), and the dominant kernel's fraction of the
measured HBM roofline; the double-float form against the FP64 form.

Workloads (--workload):
  all19   (default) each of the 19 binary32 functions on its own 2^26-element array of
          uniform random bit patterns restricted to the function's domain, plus 1%
          specials (generated on the GPU, seeded).  A step evaluates every array once.
          256 MiB per input, larger than the 129 MB L2: no flush needed between steps.
  precision  expf/logf/sinf/tanhf/rsqrtf on 2^28-element arrays: (i) U[-10,10], (ii)
          log-uniform magnitudes in [2^-126, 2^127]; sinf also (iii) = (i) with 5% of the
          arguments in |x| > 2^20.  Hard-case rate reported per array.
  f64     binary64 exp2 and log on 2^26-element arrays: uniform over the domain and the
          paper's U[-20,20] (exp2) / U[0.125,8] (log).
  batch   10,000 arrays, lengths log-uniform in [2^6, 2^22], functions uniform over the
          19: one batched launch per step (and, for comparison, one launch per array).
Before the warm-up the autotuner picks each array's launch shape (the batch tile size for
the batch workload).  The step uses --form (auto = double-float for the 19 binary32
functions; plain = the FP64-internal form); the other form is measured beside it per
array.  `--impl reference` times the CPU oracle on a bounded sample of the same workload.
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

METRIC = "Gelem/s per function (0-ulp vs oracle) & % of HBM roofline; double-float vs FP64 form"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


# DRAM traffic per element (dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture
# of the function's main kernel on 2^25 inputs -- binary32 domain bit patterns in launch
# shape 9, binary64 the domain / bit-pattern arrays in shape 1 -- divided by the elements of
# that launch), with the fingerprint of the kernel sources it was taken on; a
# traffic figure is reported only while the sources still match.
TRAFFIC_BYTES_PER_ELEM = {"expf": 7.054, "exp2f": 7.037, "exp10f": 7.06, "expm1f": 7.064, "logf": 7.04,
                          "log2f": 7.058, "log10f": 7.059, "log1pf": 7.09, "sinf": 7.175, "cosf": 7.154,
                          "sincosf": 10.956, "tanf": 7.277, "asinf": 7.181, "acosf": 7.187, "atanf": 7.195,
                          "sinhf": 7.092, "coshf": 7.138, "tanhf": 7.198, "rsqrtf": 6.568, "exp2": 14.54,
                          "log": 14.54, "exp": 14.53, "exp10": 14.521, "log2": 14.546, "log10": 14.531}
TRAFFIC_SOURCES = "fdaae95bd968c852"  # the kernel sources the ncu captures were taken on


def kernel_sources_fingerprint() -> str:
    import hashlib
    csrc = os.path.join(ROOT, "paper_2605_15547_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, name), "rb") as fh:
                h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def measured_traffic(func: str, n: int):
    if func not in TRAFFIC_BYTES_PER_ELEM or kernel_sources_fingerprint() != TRAFFIC_SOURCES:
        return None
    return TRAFFIC_BYTES_PER_ELEM[func] * n


# Thread instructions per element of each function's main kernel (smsp__inst_executed.sum x 32
# / elements, from the same captures as the traffic figures), gated by the same source
# fingerprint as the traffic figures.  The kernels are bound by instruction issue, not by
# DRAM: 152 SMs x 4 schedulers issue one warp instruction each per cycle.
INST_PER_ELEM = {"expf": 58.0, "exp2f": 50.1, "exp10f": 58.9, "expm1f": 90.6, "logf": 53.4,
                 "log2f": 57.5, "log10f": 57.4, "log1pf": 66.1, "sinf": 120.8, "cosf": 114.6,
                 "sincosf": 138.6, "tanf": 132.2, "asinf": 131.4, "acosf": 138.2, "atanf": 104.7,
                 "sinhf": 118.3, "coshf": 79.4, "tanhf": 107.7, "rsqrtf": 37.7, "exp2": 210.3,
                 "log": 388.5, "exp": 226.8, "exp10": 226.8, "log2": 457.4, "log10": 459.3}
SMS, SCHEDULERS_PER_SM, WARP = 152, 4, 32


def issue_peak_tinst_s(sm_mhz: float) -> float:
    """Thread instructions per second the GPU can issue at the given SM clock."""
    return SMS * SCHEDULERS_PER_SM * WARP * sm_mhz * 1e6 / 1e12


# The instruction count depends on the data (the branch, and for the trigonometric
# functions the reduction, each element takes): the arrays of the other workloads have their
# own captures (2^25 elements of each, the binary32 ones in launch shape 9), keyed by label.
INST_PER_ELEM_SET = {"exp2:domain": 210.3, "exp2:u20": 192.8, "log:bits": 388.5, "log:u0.125_8": 415.0,
                     "exp:edomain": 226.8, "log2:bits": 457.4, "log10:bits": 459.3, "exp10:tdomain": 226.8,
                     "expf:u10": 52.6, "expf:log": 57.2, "logf:u10": 52.0, "logf:log": 53.1,
                     "sinf:u10": 90.7, "sinf:log": 120.5, "tanhf:u10": 110.1, "tanhf:log": 107.5,
                     "rsqrtf:u10": 34.4, "rsqrtf:log": 35.6, "sinf:large": 121.6, "cosf:u10": 84.4,
                     "sincosf:u10": 109.8, "tanf:u10": 102.1}


# The same per element for the packing launch shapes (captured in shape 11 on the headline's
# inputs), used for an array whose autotuned shape packs.
INST_PER_ELEM_PACK = {"expf": 48.6, "exp2f": 46.5, "exp10f": 50.0, "expm1f": 54.0, "sinhf": 52.1,
                      "coshf": 44.7, "tanhf": 44.6, "log1pf": 68.0, "sinf": 111.1, "cosf": 109.6,
                      "sincosf": 130.6, "tanf": 120.3, "asinf": 44.2, "acosf": 66.2, "atanf": 71.0}


def inst_per_elem(func: str, label: str = "", packs: bool = False):
    if kernel_sources_fingerprint() != TRAFFIC_SOURCES:
        return None
    if packs:
        return INST_PER_ELEM_PACK.get(func)
    if label in INST_PER_ELEM_SET:
        return INST_PER_ELEM_SET[label]
    return INST_PER_ELEM.get(func)


def packs_now(crm, func: str, form: str) -> bool:
    """Whether the function's current launch shape (the autotuner's choice) packs."""
    try:
        return bool(crm.variant_info(crm.get_variant(func, form=None if form == "auto" else form))["easy"])
    except Exception:
        return False


def load_peaks():
    try:
        with open(PEAKS_PATH) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock and throttle reasons)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
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


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest of the ranks' values (timings: the job is as slow as its slowest rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gelem_s(elems_per_rank: int, steps: int, world: int, ms_total: float) -> float:
    """Weak scaling: every rank evaluates its own copy of the workload."""
    return elems_per_rank * steps * world / (ms_total / 1e3) / 1e9


def bytes_per_elem(func: str) -> int:
    return 12 if func == "sincosf" else (16 if func in W.F64_FUNCS else 8)


# ----------------------------------------------------------------------------- workloads

# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    sample = args.ref_sample
    if args.workload == "batch":
        items = [(f, f, sample) for f in W.F32_FUNCS]
        cfg = {"workload": "batch: 10,000 arrays, lengths log-uniform [2^6,2^22], 19 functions"}
        wl = "all19"  # the batch arrays use the domain recipe
    else:
        items, cfg = W.bench_arrays(args.workload, args.scale)
        wl = args.workload
    bits = np.uint64 if args.workload == "f64" else np.uint32
    xs = [(f, W.bench_input_host(wl, lab, f, sample).view(bits)) for lab, f, _ in items]
    O.eval_bits(xs[0][0], xs[0][1][:1024])
    times = []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for f, x in xs:
            O.eval_bits(f, x, nthreads=cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    n_step = sum(x.size for _, x in xs)
    secs = sum(times)
    value = n_step * args.steps / secs / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gelem/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": dict(cfg, sample_per_func=sample, l2="n/a (CPU)"),
        "cpu_baseline": {"value": value, "unit": "Gelem/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} inputs per function, same recipe"},
        "e2e": {"value": value, "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- our arm

def time_calls(crm, torch, funcs, xs, ys, form, reps, stream):
    """Average device time per call of each function, `reps` calls back to back."""
    out = []
    for f, x, y in zip(funcs, xs, ys):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        crm.eval_into(f, x, y, form=form)
        s.record(stream)
        for _ in range(reps):
            crm.eval_into(f, x, y, form=form)
        e.record(stream)
        e.synchronize()
        out.append(s.elapsed_time(e) / reps)
    return out


def run_batch(args, crm, torch, dev, stream, rank, world):
    line = batch_measure(args, crm, torch, dev, stream, world)
    if rank == 0:
        print(json.dumps(line))
    return 0


def batch_measure(args, crm, torch, dev, stream, world):
    """The batching form on the 10,000-array workload: the step is one CUDA-graph replay of
    the batched call; returns the JSON line's fields."""
    count = args.batch_count
    rng = np.random.Generator(np.random.PCG64(W.seed_for(4, 0)))
    lens, funcs = W.batch_lengths(count, rng)
    lens = lens >> args.scale
    lens[lens < 1] = 1
    gen = torch.Generator(device=dev)
    gen.manual_seed(W.seed_for(4, 0))
    xs, ys = [], []
    for f, n in zip(funcs, lens):
        xs.append(W.domain_bits_device(f, int(n), gen, device=dev))
        ys.append(torch.empty((2 * int(n),) if f == "sincosf" else (int(n),), dtype=torch.float32, device=dev))
    items = list(zip(funcs, xs, ys))
    n_elems = int(lens.sum())
    crm.reserve(1 << 24, count, stream=stream)
    tile = mode = None
    if not args.no_autotune:
        mode, tile, _ = crm.autotune_batch(items, form=args.form, reps=1, stream=stream)
    for _ in range(args.warmup):
        crm.eval_batch(items, form=args.form, stream=stream)
    torch.cuda.synchronize()
    # the step: one CUDA-graph replay of the captured batched call (its persistent
    # kernels and the slow pass; the descriptors were staged at capture)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        crm.eval_batch(items, form=args.form, stream=stream)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    crm.stats_reset(stream=stream)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    s.record(stream)
    for _ in range(args.steps):
        g.replay()
    e.record(stream)
    e.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(s.elapsed_time(e), world, dev)
    st = crm.stats(stream=stream)
    # the same call without the graph (host staging of the 10,000 descriptors each call)
    s3, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s3.record(stream)
    for _ in range(args.steps):
        crm.eval_batch(items, form=args.form, stream=stream)
    e3.record(stream)
    e3.synchronize()
    ms_direct = s3.elapsed_time(e3) / args.steps
    # one launch per array, for comparison (also via CUDA events)
    s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s2.record(stream)
    for f, x, y in items:
        crm.eval_into(f, x, y, form=args.form, stream=stream)
    e2.record(stream)
    e2.synchronize()
    ms_single = s2.elapsed_time(e2)
    nbytes = sum(x.numel() * 4 + y.numel() * 4 for _, x, y in items)
    bmode = mode if mode is not None else "grouped"
    launches_per_step = (len(set(funcs)) if bmode == "grouped" else 1) + 1
    peak, kind = load_peaks()
    value = whole_job_gelem_s(n_elems, args.steps, world, ms)
    achieved = nbytes / (ms / args.steps / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "Gelem/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch: {count} arrays, lengths log-uniform [2^6,2^22] >> {args.scale}, "
                               "functions uniform over the 19", "total_elems": n_elems, "form": args.form,
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{world}",
                   "tile_log2": tile if tile is not None else "default 14",
                   "batch_mode": mode if mode is not None else "default grouped"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_batch (step)", "peak_kind": kind},
        "one_launch_per_array": {"gelem_s": n_elems / (ms_single / 1e3) / 1e9, "ms": ms_single,
                                 "launches": 2 * count},
        "step": "one CUDA-graph replay of the batched call",
        "direct_call": {"gelem_s": n_elems / (ms_direct / 1e3) / 1e9, "ms": ms_direct},
        "hard_case_rate": st["hard_total"] / max(1, n_elems * args.steps), "unresolved": st["unresolved_total"],
        "gpu_launches": launches_per_step * args.steps, "clocks": clk,
        "e2e": {"value": None, "unit": "Gelem/s", "note": "batch workload is device resident"},
        "cpu_baseline": None,
    }
    return line


def measure_set(args, crm, torch, dev, workload, reps=3):
    """One of the other workloads (the 2^28 precision arrays, the binary64 pair) measured
    beside the headline step: per array, the default form's and the plain form's device time
    per call (CUDA events, back-to-back calls on arrays larger than L2), both rooflines and
    the hard-case rate.  The arrays are freed on return."""
    spec, cfg = W.bench_arrays(workload, args.scale)
    peak, _ = load_peaks()
    out = {"config": cfg["workload"]}
    stream = torch.cuda.current_stream()
    for lab, f, n in spec:
        x = W.bench_input_device(workload, lab, f, n, dev)
        y = torch.empty(((2,) if f == "sincosf" else ()) + (n,), dtype=x.dtype, device=dev)
        if not args.no_autotune:
            crm.autotune(f, x, y, form=args.form, reps=2)
        ms = time_calls(crm, torch, [f], [x], [y], args.form, reps, stream)[0]
        try:
            ms_plain = time_calls(crm, torch, [f], [x], [y], "plain", 2, stream)[0]
        except crm.CrmError:
            ms_plain = None
        crm.stats_reset()
        crm.eval_into(f, x, y, form=args.form)
        st = crm.stats()
        g = n / (ms / 1e3) / 1e9
        ipe = inst_per_elem(f, lab, packs_now(crm, f, args.form))
        out[lab] = {"gelem_s": g, "hbm_frac": g * bytes_per_elem(f) / peak,
                    "issue_frac": (g * ipe / 1e3 / issue_peak_tinst_s(2070.0)) if ipe else None,
                    "plain_gelem_s": (n / (ms_plain / 1e3) / 1e9) if ms_plain else None,
                    "df_over_plain": (ms_plain / ms) if ms_plain else None,
                    "hard_case_rate": st["hard_total"] / n, "unresolved": st["unresolved_total"]}
        del x, y
        torch.cuda.empty_cache()
    return out


def time_fn(torch, fn, reps, stream):
    """Device time per call of fn (CUDA events, after one untimed call)."""
    fn()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(reps):
        fn()
    e.record(stream)
    e.synchronize()
    return s.elapsed_time(e) / reps


def measure_modes(args, crm, torch, dev, reps=3):
    """Directed rounding and the 16-bit formats (crm_eval_rm): expf, logf, sinf on 2^26
    domain inputs (binary32 in RD/RU/RZ; binary16 and bfloat16 in RN), against the same
    call in round-to-nearest binary32."""
    n = (1 << 26) >> args.scale
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device=dev)
    out = {"config": f"expf, logf, sinf x 2^{26 - args.scale} domain bit patterns + 1% specials"}
    for f in ("expf", "logf", "sinf"):
        gen.manual_seed(W.seed_for(2, f))
        x = W.domain_bits_device(f, n, gen, device=dev)
        y = torch.empty_like(x)
        row = {"rn_f32": n / (time_fn(torch, lambda: crm.eval_into(f, x, y), reps, stream) / 1e3) / 1e9}
        for m in ("rd", "ru", "rz"):
            row[m + "_f32"] = n / (time_fn(torch, lambda: crm.eval_rm(f, x, m, out=y), reps, stream) / 1e3) / 1e9
        for dt, nm in ((torch.float16, "f16"), (torch.bfloat16, "bf16")):
            xh = x.to(dt)
            yh = torch.empty_like(xh)
            row["rn_" + nm] = n / (time_fn(torch, lambda: crm.eval_rm(f, xh, "rn", out=yh), reps, stream) / 1e3) / 1e9
        out[f] = row
        del x, y
    return out


def measure_apps(args, crm, torch, dev, reps=3):
    """The paper's applications: complex expf / logf / sinf on 2^26 complex inputs uniform in
    [-40, 40]^2 (16 bytes per element), and spectral interpolation by a brute-force DFT of
    N = 2^14 samples at M = 2^14 non-integer frequencies (2^28 sine-cosine terms per call)."""
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device=dev)
    gen.manual_seed(W.seed_for(6, 0))
    n = (1 << 26) >> args.scale
    z = ((torch.rand(2 * n, generator=gen, device=dev, dtype=torch.float64) * 80.0 - 40.0)
         .to(torch.float32).view(torch.complex64))
    w = torch.empty_like(z)
    peak, _ = load_peaks()
    out = {"complex_config": f"2^{26 - args.scale} complex64 inputs uniform in [-40,40]^2"}
    for f in ("cexpf", "clogf", "csinf"):
        ms = time_fn(torch, lambda: crm.eval_complex(f, z, out=w), reps, stream)
        out[f] = {"gelem_s": n / (ms / 1e3) / 1e9, "hbm_frac": 16 * n / (ms / 1e3) / 1e9 / peak}
    del z, w
    N, M = 1 << (14 - args.scale // 2), 1 << (14 - (args.scale + 1) // 2)
    t = torch.arange(N, device=dev, dtype=torch.float64)
    x = (torch.sin(2 * np.pi * 37.3 * t / N) + 0.5 * torch.cos(2 * np.pi * 101.7 * t / N)).to(torch.float32)
    fr = (torch.rand(M, generator=gen, device=dev, dtype=torch.float64) * N).to(torch.float32)
    ms = time_fn(torch, lambda: crm.spectral_dft(x, fr), reps, stream)
    out["spectral"] = {"config": f"N = {N} samples, M = {M} frequencies", "terms_per_call": N * M,
                       "gterms_s": N * M / (ms / 1e3) / 1e9, "ms_per_call": ms}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="auto", choices=["auto", "plain", "df"])
    ap.add_argument("--workload", default="all19", choices=["all19", "precision", "f64", "trig", "batch"])
    ap.add_argument("--scale", type=int, default=0, help="divide sizes by 2^scale (testing)")
    ap.add_argument("--ref-sample", type=int, default=1 << 15)
    ap.add_argument("--cpu-sample", type=int, default=1 << 18)
    ap.add_argument("--batch-count", type=int, default=10000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--variant", type=int, default=-1,
                    help="launch shape for every array (skips the autotuner; profiling runs)")
    ap.add_argument("--funcs", default="", help="comma list restricting the workload (testing)")
    ap.add_argument("--extras", default="precision,trig,f64,batch,modes,apps",
                    help="other workloads measured after the headline step (comma list, or none)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2605_15547_gb300 as crm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)  # before the process group, so NCCL binds this rank's GPU
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__ as g
    g.build()
    stream = torch.cuda.current_stream()
    if args.workload == "batch":
        side = torch.cuda.Stream(device=dev)  # graph capture needs a non-default stream
        with torch.cuda.stream(side):
            return run_batch(args, crm, torch, dev, side, rank, world)

    spec, cfg = W.bench_arrays(args.workload, args.scale)
    if args.funcs:
        keep = set(args.funcs.split(","))
        spec = [s for s in spec if s[1] in keep or s[0] in keep]
    labels = [lab for lab, _, _ in spec]
    funcs = [f for _, f, _ in spec]
    xs = [W.bench_input_device(args.workload, lab, f, n, dev) for lab, f, n in spec]
    ys = [torch.empty(((2,) if f == "sincosf" else ()) + (x.numel(),), dtype=x.dtype, device=dev)
          for f, x in zip(funcs, xs)]
    n_elems = sum(x.numel() for x in xs)
    f64 = args.workload == "f64"

    def step(form):
        for f, x, y in zip(funcs, xs, ys):
            crm.eval_into(f, x, y, form=form)

    # the autotuner picks each array's launch shape on that array (untimed)
    tuned = {}
    if args.variant >= 0:
        for f in funcs:
            crm.set_variant(f, args.variant, form=args.form)
        args.no_autotune = True
        tuned = {"all": f"variant {args.variant}"}
    if not args.no_autotune:
        for lab, f, x, y in zip(labels, funcs, xs, ys):
            best, _ = crm.autotune(f, x, y, form=args.form, reps=2)
            info = crm.variant_info(best)
            tuned[lab] = ("pipelined" if info["pipelined"] else
                          f"u{info['unroll']}b{info['block']}" + ("pf" if info["prefetch"] else "") +
                          (f"m{info['min_blocks']}" if info["min_blocks"] > 1 else "") +
                          ("w32" if info["vec_bytes"] == 32 else "") + ("reg16" if info["reg_table"] else "") +
                          ("pack" if info["easy"] else ""))

    for _ in range(args.warmup):
        step(args.form)
    torch.cuda.synchronize()
    crm.stats_reset()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_s, t_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_s.record(stream)
    for _ in range(args.steps):
        step(args.form)
    t_e.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms_total = max_over_ranks(t_s.elapsed_time(t_e), world, dev)
    st = crm.stats()
    value = whole_job_gelem_s(n_elems, args.steps, world, ms_total)

    # per array, both forms (back-to-back calls, device time per call), and hard-case rates
    other = "plain" if args.form != "plain" else "auto"
    ms_main = time_calls(crm, torch, funcs, xs, ys, args.form, 3, stream)
    try:
        ms_other = time_calls(crm, torch, funcs, xs, ys, other, 2, stream)
    except crm.CrmError:  # the binary64 pair has one form
        ms_other = None
    hard = []
    for f, x, y in zip(funcs, xs, ys):
        crm.stats_reset()
        crm.eval_into(f, x, y, form=args.form)
        hard.append(crm.stats()["hard_total"] / x.numel())
    peak, peak_kind = load_peaks()
    per_arr = {}
    for i, lab in enumerate(labels):
        n = xs[i].numel()
        gi = n / (ms_main[i] / 1e3) / 1e9
        ipe = inst_per_elem(funcs[i], packs=packs_now(crm, funcs[i], args.form))
        per_arr[lab] = {
            args.form: {"gelem_s": gi, "hbm_frac": gi * bytes_per_elem(funcs[i]) / peak,
                        "issue_frac": (gi * ipe / 1e3 / issue_peak_tinst_s(2070.0)) if ipe else None},
            "hard_case_rate": hard[i]}
        if ms_other is not None:
            per_arr[lab][other] = {"gelem_s": n / (ms_other[i] / 1e3) / 1e9}
            hi, lo = (ms_other[i], ms_main[i]) if args.form != "plain" else (ms_main[i], ms_other[i])
            per_arr[lab]["df_over_plain"] = hi / lo
    step_other = (n_elems / (sum(ms_other) / 1e3) / 1e9) if ms_other is not None else None
    # dominant kernel: the array taking the largest share of the step
    dom = int(np.argmax(ms_main))
    dom_bytes = xs[dom].numel() * bytes_per_elem(funcs[dom])
    achieved = dom_bytes / (ms_main[dom] / 1e3) / 1e9
    hbm_roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": peak_kind}
    # The binding bound of these kernels is instruction issue: thread instructions per
    # element (ncu, the kernel's own sources) x elements / time, against 152 SMs x 4
    # schedulers x 32 lanes x the SM clock (2070 MHz, the clock measured under load)
    dom_ipe = inst_per_elem(funcs[dom], packs=packs_now(crm, funcs[dom], args.form))
    if dom_ipe:
        ach_i = xs[dom].numel() * dom_ipe / (ms_main[dom] / 1e3) / 1e12
        pk_i = issue_peak_tinst_s(2070.0)
        roof = {"bound": "alu", "achieved": ach_i, "peak": pk_i, "unit": "Tinst/s", "frac": ach_i / pk_i,
                "peak_kind": "derived: 152 SMs x 4 schedulers x 32 lanes x 2070 MHz",
                "inst_per_elem": dom_ipe, "hbm": hbm_roof}
    else:
        roof = dict(hbm_roof)

    e2e = None
    if not args.no_e2e:
        hin = [x.cpu().pin_memory() for x in xs]
        hout = [torch.empty(tuple(y.shape), dtype=y.dtype).pin_memory() for y in ys]
        for f, a, b in zip(funcs, hin, hout):  # warm-up pass: first touch of the pinned pages
            crm.eval_host(f, a.numpy(), b.numpy().reshape(-1), form=args.form)
        t0 = time.perf_counter()
        for f, a, b in zip(funcs, hin, hout):
            crm.eval_host(f, a.numpy(), b.numpy().reshape(-1), form=args.form)
        t1 = time.perf_counter()
        e2e = {"value": n_elems / (t1 - t0) / 1e9, "unit": "Gelem/s",
               "h2d_bytes_per_step": int(sum(x.numel() * x.element_size() for x in xs)),
               "d2h_bytes_per_step": int(sum(y.numel() * y.element_size() for y in ys)),
               "note": "crm_eval_host on page-locked host in/out: the kernels read and write them in "
                       "place over the host link (NVLink-C2C); every input and output byte crosses it "
                       "inside the timed region"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        cores = os.cpu_count() or 1
        bits = np.uint64 if f64 else np.uint32
        sample = [(f, xs[i][:args.cpu_sample].cpu().numpy().view(bits)) for i, f in enumerate(funcs)]
        t0 = time.perf_counter()
        for f, xh in sample:
            O.eval_bits(f, xh, nthreads=cores)
        dt = time.perf_counter() - t0
        cnt = sum(x.size for _, x in sample)
        cpu = {"value": cnt / dt / 1e9, "unit": "Gelem/s", "cores": cores, "kind": "oracle",
               "sample": f"first {args.cpu_sample} inputs of each array"}

    line = {
        "metric": METRIC, "value": value, "unit": "Gelem/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": ("f64" if args.form == "plain" else ("int64" if f64 else "f32")),
        "data": "synthetic",
        "config": dict(cfg, form=args.form, arrays=labels, l2="inputs larger than L2 (no flush)",
                       parallelism=f"replicas{world}", launch_shapes=tuned or "default"),
        "roofline": dict(roof, traffic=measured_traffic(funcs[dom], xs[dom].numel()),
                         kernel=f"k_main+k_slow<{funcs[dom]}>", array=labels[dom],
                         bytes_per_elem=bytes_per_elem(funcs[dom])),
        "other_form": {"form": other, "step_gelem_s": step_other},
        "per_array": per_arr,
        "hard_case_rate": st["hard_total"] / max(1, n_elems * args.steps), "unresolved": st["unresolved_total"],
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps * len(funcs) * 2, "clocks": clk,
    }
    # the other workloads, measured after the headline step on freshly generated arrays
    extras = [e for e in args.extras.split(",") if e and e != "none"] if args.workload == "all19" else []
    if extras:
        del xs, ys
        if e2e is not None:
            del hin, hout
        torch.cuda.empty_cache()
        line["extras"] = {}
        for wl in extras:
            if wl == "batch":
                side = torch.cuda.Stream(device=dev)
                with torch.cuda.stream(side):
                    b = batch_measure(args, crm, torch, dev, side, world)
                torch.cuda.empty_cache()
                line["extras"]["batch"] = {k: b[k] for k in ("value", "ms_per_step", "config", "roofline",
                                                             "one_launch_per_array", "direct_call",
                                                             "hard_case_rate", "unresolved", "clocks")}
            elif wl == "modes":
                line["extras"]["modes"] = measure_modes(args, crm, torch, dev)
            elif wl == "apps":
                line["extras"]["apps"] = measure_apps(args, crm, torch, dev)
            else:
                line["extras"][wl] = measure_set(args, crm, torch, dev, wl)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
