#!/usr/bin/env python3
"""Throughput of the Fourier Poisson solve (FLUPS method) on GB300: one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

A step is one full solve (all passes of the hot path) of the workload's
synthetic right-hand side, inputs resident in HBM.  Under torchrun (N > 1)
every rank solves its own replica (weak scaling, no data-path collective).

Default workload (`unb128_f64`): fully unbounded 3D Poisson, cell-centred
128^3 FP64 (doubled to 256^3), unit cube, unit-mass Gaussian blob sigma = 0.1
centred at 0.5 + seeded 1e-3 jitter, HEJ2 kernel eps = 2h.  Other workloads:
per32_f64, unb128_f32, mixed257_f32, mixed257_f64, unb512_f32, per1024_f64.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2211_07777_gb300 import workloads as W  # noqa: E402

L2_BYTES = 129 * 1024 * 1024
PRECS = {"f32": 0, "f64": 1, "f64e": 2}
PREC_NAMES = {0: "FP32", 1: "FP64", 2: "FP64-class double-float (FP32 units)"}
DTYPES = {0: "f32", 1: "f64", 2: "f32x2"}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12   # 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz (1.26 TF)
FP32_PEAK_TFLOPS = 2 * 128 * 152 * 2.070e9 / 1e12  # 128 FP32 lanes/SM


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
def workload(name):
    """(description, n, bc, center, prec, kernel, rhs builder, L)."""
    E, O, P, U = W.EVEN, W.ODD, W.PER, W.UNB
    if name in ("unb128_f64", "unb128_f32", "unb512_f32", "unb128_f64e", "unb512_f64e"):
        n = 512 if name.startswith("unb512") else 128
        prec = PRECS[name.split("_")[1]]
        desc = f"fully unbounded {n}^3 cell-centred {PREC_NAMES[prec]} (doubled {2*n}^3), " \
               f"HEJ2 eps=2h, Gaussian blob sigma=0.1"
        return dict(desc=desc, n=(n, n, n), bc=((U, U),) * 3, center=W.CELL, prec=prec, kernel="hej2",
                    rhs=lambda: W.gaussian_blob((n, n, n), 0.1, W.blob_center(2)), L=(1.0, 1.0, 1.0))
    if name in ("per32_f64", "per1024_f64", "per32_f64e", "per1024_f64e"):
        n = 32 if name.startswith("per32") else 1024
        seed = 1 if n == 32 else 5
        prec = PRECS[name.split("_")[1]]
        desc = f"fully periodic {n}^3 cell-centred {PREC_NAMES[prec]}, spectral kernel, 4 seeded sine products"
        return dict(desc=desc, n=(n, n, n), bc=((P, P),) * 3, center=W.CELL, prec=prec, kernel="spectral",
                    rhs=lambda: W.periodic_sines((n, n, n), W.sine_modes(seed)), L=(1.0, 1.0, 1.0))
    if name in ("mixed257_f32", "mixed257_f64", "mixed257_f64e"):
        prec = PRECS[name.split("_")[1]]
        desc = "node-centred 257x256x257, x even-even (DCT-I), y periodic, z unbounded, HEJ2, " \
               f"{PREC_NAMES[prec]}, Gaussian blob sigma=0.08 + 4 seeded y-modes"
        return dict(desc=desc, n=(257, 256, 257), bc=((E, E), (P, P), (U, U)), center=W.NODE, prec=prec,
                    kernel="hej2", rhs=lambda: W.mixed_blob_modes(), L=(1.0, 1.0, 1.0), h=(1 / 256,) * 3)
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# The oracle (CPU baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_problem(wl):
    import oracle
    n = wl["n"]
    h = wl.get("h") or tuple(wl["L"][d] / (n[d] if wl["center"] == W.CELL else n[d] - 1) for d in range(3))
    return oracle.Problem(bc=wl["bc"], h=tuple(h), center=wl["center"], kernel=wl["kernel"])


def oracle_solve(wl, f):
    import oracle
    if wl["center"] == W.NODE and any(b[0] == W.PER for b in wl["bc"]):
        # periodic node direction stored without its duplicate node: append it for the oracle
        d = [i for i in range(3) if wl["bc"][i][0] == W.PER][0]
        ax = 2 - d
        full = np.concatenate([f, np.take(f, [0], axis=ax)], axis=ax)
        out = oracle.solve(full, oracle_problem(wl))
        return np.take(out, range(f.shape[ax]), axis=ax)
    return oracle.solve(f, oracle_problem(wl))


def cores_used():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def time_oracle(wl, f, budget_s=30.0, max_steps=None):
    """Run the oracle repeatedly within a time budget; (seconds per solve, solves, result)."""
    t0 = time.perf_counter()
    ref = oracle_solve(wl, f)
    times = [time.perf_counter() - t0]
    while sum(times) + times[-1] < budget_s and (max_steps is None or len(times) < max_steps):
        t0 = time.perf_counter()
        oracle_solve(wl, f)
        times.append(time.perf_counter() - t0)
    return float(np.mean(times)), len(times), ref


# ---------------------------------------------------------------------------
def traffic_record(kernel_name, workload_name):
    """ncu DRAM bytes per launch recorded under profiles/, if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(f"{kernel_name}@{workload_name}")
    except Exception:
        return None
    if not rec or rec.get("source_sha") != kernel_source_sha():
        return None
    return rec.get("dram_bytes_per_launch")


# the sources that define the compile-time pass kernels (the FFT engine, the tile loaders, the
# pass kernels and their instantiations); the host planner and the other kernels are not among them
KERNEL_SOURCES = ("fft_engine.cuh", "dfloat.cuh", "passes.cuh", "pass_common.cuh", "pass_kernels.cuh",
                  "passes_ct_f32.cu", "passes_ct_f64.cu", "passes_ct_df.cu", "passes_ct_df_large.cu")


def kernel_source_sha():
    """Digest of the pass kernels' sources: a recorded ncu figure is used only while the kernel
    code it was taken on is unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2211_07777_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fn.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


KIND_NAMES = {0: "k_fwd_real", 1: "k_inv_real", 2: "k_fwd_c2c", 3: "k_inv_c2c", 4: "k_fused_real", 5: "k_fused_c2c"}


def measured_peaks():
    if os.path.exists(PEAKS_FILE):
        try:
            pk = json.load(open(PEAKS_FILE))
            return float(pk["hbm_gbs"]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM, "fallback"


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = workload(args.workload)
    f = wl["rhs"]()
    pts = float(np.prod(wl["n"]))
    # warm-up: at most args.warmup solves within 60 s
    t_end = time.perf_counter() + 60.0
    for _ in range(max(0, args.warmup)):
        oracle_solve(wl, f)
        if time.perf_counter() > t_end:
            break
    # timed: the requested steps, bounded to about 150 s of CPU work
    times = []
    budget = 150.0
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        oracle_solve(wl, f)
        times.append(time.perf_counter() - t0)
        if sum(times) > budget:
            break
    sec = float(np.mean(times))
    val = pts / sec / 1e6
    line = {
        "impl": "reference", "metric": "Mpts/s per Poisson solve", "value": val, "unit": "Mpts/s",
        "n_gpus": args.gpus, "steps": len(times), "steps_requested": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "name": args.workload},
        "cpu_baseline": {"value": val, "unit": "Mpts/s", "cores": 1, "kind": "oracle",
                         "sample": f"{len(times)} full oracle solve(s) of the workload (NumPy pocketfft, one thread)"},
        "e2e": {"value": val, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_2211_07777_gb300 import flups as F

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = workload(args.workload)
    prec = wl["prec"]
    dt = torch.float32 if prec == 0 else torch.float64
    f_host = wl["rhs"]()
    pts = float(np.prod(wl["n"]))
    solver = F.Solver(wl["n"], wl["bc"], L=wl["L"], center=wl["center"], prec=prec, green=wl["kernel"],
                      h=wl.get("h"))
    rhs = torch.from_numpy(f_host).to(dev, dt)
    phi = torch.empty_like(rhs)
    stream = torch.cuda.current_stream(dev)
    npass = solver.info["launches"]
    pinfo = [solver.pass_info(i) for i in range(npass)]
    flush = L2Flush(torch, dev)

    # parity check of this exact launch configuration against the oracle (rank 0, modest sizes only)
    err = None
    ref = None
    if rank == 0 and pts <= 2 ** 22:
        solver.solve(phi, rhs, stream)
        torch.cuda.synchronize()
        ref = oracle_solve(wl, f_host)
        err = float(np.abs(phi.double().cpu().numpy() - ref).max() / np.abs(ref).max())

    for _ in range(args.warmup):
        flush.zero_()
        solver.solve(phi, rhs, stream)
    torch.cuda.synchronize()

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(npass + 1)] for _ in range(K)]
    for row in ev:              # torch creates the CUDA event at its first record
        for e in row:
            e.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        for k in range(K):
            flush.zero_()            # L2 flush between timed solves (outside the per-step events)
            solver.solve_events(phi, rhs, ev[k], stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
        if K > 0 and t_wall < 1.5:
            # keep sampling clocks under a comparable load for at least ~1.5 s (untimed)
            t1 = time.perf_counter()
            while time.perf_counter() - t1 < 1.5 - t_wall:
                for _ in range(20):
                    solver.solve(phi, rhs, stream)
                torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    step_ms = [ev[k][0].elapsed_time(ev[k][npass]) for k in range(K)]
    pass_ms = np.array([[ev[k][i].elapsed_time(ev[k][i + 1]) for i in range(npass)] for k in range(K)])
    total_ms, ms_per_step, value = aggregate_replicas(float(np.sum(step_ms)), pts, K, world, dist, dev)

    # the same configuration in the other arithmetic paths (FP32 vs FP64 at the stated error)
    variants = {}
    if rank == 0 and not args.no_variants and args.workload.split("_")[1] in PRECS:
        base = args.workload.rsplit("_", 1)[0]
        for tag in ("f32", "f64", "f64e"):
            name = f"{base}_{tag}"
            if name == args.workload:
                continue
            try:
                wv = workload(name)
            except SystemExit:
                continue
            variants[tag] = measure_variant(F, torch, wv, f_host, ref, flush, stream, max(5, K // 2), args.warmup)

    # e2e: public API with pinned host buffers, H2D + solve + D2H every step
    h_in = torch.from_numpy(f_host.astype(np.float32 if prec == 0 else np.float64)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    for _ in range(max(1, args.warmup)):
        solver.solve_host(h_out, h_in, stream)
    Ke = max(3, min(K, 50))
    t0 = time.perf_counter()
    for _ in range(Ke):
        solver.solve_host(h_out, h_in, stream)
    e2e_s = (time.perf_counter() - t0) / Ke
    e2e_val = world * pts / e2e_s / 1e6
    nbytes = h_in.numel() * h_in.element_size()
    host_path = "mapped" if F.flups_host_mapped(h_in) and F.flups_host_mapped(h_out) else "staged"
    # the same transfers as explicit copies around a device solve (pinned buffers, one stream)
    d_in = torch.empty(h_in.shape, dtype=h_in.dtype, device=dev)
    d_out = torch.empty_like(d_in)
    with torch.cuda.stream(stream):
        for k in range(max(1, args.warmup) + Ke):
            if k == max(1, args.warmup):
                t0 = time.perf_counter()
            d_in.copy_(h_in, non_blocking=True)
            solver.solve(d_out, d_in, stream)
            h_out.copy_(d_out, non_blocking=True)
            stream.synchronize()
    copy_val = world * pts / ((time.perf_counter() - t0) / Ke) / 1e6

    # roofline of the dominant kernel
    mean_pass = pass_ms.mean(axis=0)
    dom = int(np.argmax(mean_pass))
    kname = KIND_NAMES[pinfo[dom]["kind"]]
    hbm, hbm_src = measured_peaks()
    ach_gbs = pinfo[dom]["bytes"] / (mean_pass[dom] * 1e-3) / 1e9
    ach_tf = pinfo[dom]["flops"] / (mean_pass[dom] * 1e-3) / 1e12
    if prec == 1:
        roof = {"bound": "alu", "achieved": ach_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach_tf / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz",
                "hbm_achieved_gbs": ach_gbs, "hbm_frac": ach_gbs / hbm, "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src}
    else:
        roof = {"bound": "hbm", "achieved": ach_gbs, "peak": hbm, "unit": "GB/s", "frac": ach_gbs / hbm,
                "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else "fallback 6.8 TB/s"}
        if prec == 2:
            # double-float arithmetic on the FP32 units: FP64-equivalent rate against the native FP64 peak
            roof["fp64_equiv_tflops"] = ach_tf
            roof["fp64_equiv_over_native_fp64_peak"] = ach_tf / FP64_PEAK_TFLOPS
    roof["kernel"] = kname
    roof["traffic"] = traffic_record(kname, args.workload)
    roof["algorithmic_bytes_per_launch"] = pinfo[dom]["bytes"]
    roof["algorithmic_flops_per_launch"] = pinfo[dom]["flops"]
    roof["launch_ms"] = float(mean_pass[dom])
    model_bytes = sum(p["bytes"] for p in pinfo)
    solve_frac = model_bytes / (ms_per_step * 1e-3) / 1e9 / hbm

    line = {
        "metric": "Mpts/s per Poisson solve", "value": value, "unit": "Mpts/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[prec], "data": "synthetic",
        "config": {"workload": wl["desc"], "name": args.workload, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "max_rel_err_vs_oracle": err,
        "variants": variants,
        "passes": [{"kernel": KIND_NAMES[p["kind"]], "axis": p["axis"], "P": p["P"], "ms": float(m),
                    "gbs": p["bytes"] / (m * 1e-3) / 1e9} for p, m in zip(pinfo, mean_pass)],
        "solve_hbm_frac": solve_frac,
        "roofline": roof,
        "e2e": {"value": e2e_val, "unit": "Mpts/s", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "host_path": host_path, "explicit_copies_value": copy_val},
        "gpu_launches": K * npass,
        "clocks": clk.summary(),
    }
    # CPU baseline: the oracle on this host, rank 0, N = 1 only
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if pts <= 2 ** 22:
            sec, nsol, _ = time_oracle(wl, f_host, budget_s=20.0, max_steps=3)
            line["cpu_baseline"] = {"value": pts / sec / 1e6, "unit": "Mpts/s", "cores": 1, "kind": "oracle",
                                    "sample": f"{nsol} full oracle solve(s) of the same workload "
                                              f"(NumPy pocketfft, single thread)"}
        else:
            line["cpu_baseline"] = {"value": None, "unit": "Mpts/s", "cores": 1, "kind": "oracle",
                                    "sample": "skipped: the oracle's full extended box does not fit a bounded sample"}
    # device-side status of every solve above (0: no bounded wait gave up; checked outside timing)
    line["device_status"] = solver.check()
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_served(args):
    """Served stream: 4096 seeded requests, sizes {32..256}^3, random face conditions, 30% Biot-Savart,
    FP32/FP64 50/50; closed-loop capacity, then Poisson arrivals at 0.8x capacity."""
    import torch

    from paper_2211_07777_gb300 import flups as F
    from paper_2211_07777_gb300 import serve
    nreq = args.served_requests
    reqs = W.served_stream(nreq=nreq, seed=4)
    free, _ = torch.cuda.mem_get_info()
    budget = int(min(free * 0.6, 96 << 30))
    pool = serve.HostPool()
    for r in reqs:
        pool.input(r)
    eng = args.fp64_engine
    warm = serve.run_stream(reqs[:64], budget, nstreams=args.streams, closed_loop=True, pool=pool, fp64_engine=eng)
    cap = serve.run_stream(reqs, budget, nstreams=args.streams, closed_loop=True, pool=pool, fp64_engine=eng)
    rate = 0.8 * cap["req_per_s"]
    nominal = 1.0 / np.mean(np.diff([r.arrival_s for r in reqs]))
    with ClockSampler(0) as clk:
        run = serve.run_stream(reqs, budget, nstreams=args.streams, time_scale=nominal / rate, pool=pool,
                               fp64_engine=eng)
    n_df = sum(1 for r in reqs if serve.engine_prec(r, eng) == F.F64E)
    # FP64-class requests on the double-float path: their error against the native FP64 path
    df_errs = []
    if n_df:
        for r in [q for q in reqs if serve.engine_prec(q, eng) == F.F64E][:6]:
            outs = []
            for prec in (F.F64E, F.F64):
                creq = serve.c_request(W.Request(**{**r.__dict__, "prec": F.F64}), "df" if prec == F.F64E else "native")
                bc = [[tuple(creq.bc[(c * 3 + d) * 2:(c * 3 + d) * 2 + 2]) for d in range(3)] for c in range(3)]
                sol = F.Solver(r.n, bc if r.op == F.BIOT_SAVART else bc[0], prec=prec, op=r.op, green=r.kernel)
                rhs = torch.from_numpy(np.ascontiguousarray(W.request_rhs(r))).to("cuda", torch.float64)
                phi = torch.empty_like(rhs)
                sol.solve(phi, rhs)
                torch.cuda.synchronize()
                outs.append(phi.cpu().numpy())
                sol.close()
            df_errs.append(float(np.abs(outs[0] - outs[1]).max() / np.abs(outs[1]).max()))
    # FP32 against FP64 on sampled request classes (same input), the stated error of the FP32 path
    errs = []
    for r in [q for q in reqs if q.prec == F.F32][:8]:
        outs = []
        for prec in (F.F32, F.F64):
            rr = W.Request(**{**r.__dict__, "prec": prec})
            creq = serve.c_request(rr)
            bc = [[tuple(creq.bc[(c * 3 + d) * 2:(c * 3 + d) * 2 + 2]) for d in range(3)] for c in range(3)]
            sol = F.Solver(rr.n, bc if rr.op == 1 else bc[0], prec=prec, op=rr.op, green=rr.kernel)
            dt = torch.float32 if prec == F.F32 else torch.float64
            rhs = torch.from_numpy(np.ascontiguousarray(W.request_rhs(rr))).to("cuda", dt)
            phi = torch.empty_like(rhs)
            sol.solve(phi, rhs)
            torch.cuda.synchronize()
            outs.append(phi.double().cpu().numpy())
            sol.close()
        errs.append(float(np.abs(outs[0] - outs[1]).max() / np.abs(outs[1]).max()))
    for k in ("outputs",):
        run.pop(k, None)
    line = {
        "metric": "served throughput (Mpts/s) with p50/p99 latency", "value": run["mpts_per_s"], "unit": "Mpts/s",
        "n_gpus": 1, "steps": nreq, "warmup": 64, "ms_per_step": run["makespan_s"] * 1e3 / nreq,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"served stream: {nreq} seeded requests, sizes uniform on {{32..256}}^3, random face "
                               "conditions, 30% Biot-Savart Gaussian rings, FP32/FP64 50/50, Poisson arrivals at "
                               "0.8x measured capacity", "name": "served", "hbm_budget_bytes": budget,
                   "streams": args.streams},
        "p50_ms": run["p50_ms"], "p99_ms": run["p99_ms"], "req_per_s": run["req_per_s"],
        "fp32": run.get("fp32"), "fp64": run.get("fp64"),
        "capacity_req_per_s": cap["req_per_s"], "capacity_mpts_per_s": cap["mpts_per_s"],
        "fp32_vs_fp64_max_rel_err": max(errs) if errs else None,
        "fp64_engine": {"policy": eng, "requests_on_double_float": n_df,
                        "double_float_vs_fp64_max_rel_err": max(df_errs) if df_errs else None},
        "server": run["server"], "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


class L2Flush:
    """Between timed solves: write a buffer twice the L2 size (evicting the solve's data), then read
    another one, so that the next solve starts with no dirty lines of the flush left to write back."""

    def __init__(self, torch, dev):
        self.a = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
        self.b = torch.zeros(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
        self.sink = torch.zeros(1, dtype=torch.float32, device=dev)

    def zero_(self):
        self.a.zero_()
        self.sink += self.b.sum()


def aggregate_replicas(total_ms, pts, K, world, dist=None, device="cpu"):
    """Weak scaling over replicas: every rank solved its own problem K times in total_ms; the job
    time is the slowest rank's, and the job throughput counts every rank's points."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / K
    value = world * pts * K / (total_ms * 1e-3) / 1e6
    return total_ms, ms_per_step, value


def measure_variant(F, torch, wl, f_host, ref, flush, stream, K, warmup):
    """Time one other arithmetic path of the same workload (whole solves, CUDA events, L2 flushed)."""
    dt = torch.float32 if wl["prec"] == 0 else torch.float64
    s = F.Solver(wl["n"], wl["bc"], L=wl["L"], center=wl["center"], prec=wl["prec"], green=wl["kernel"],
                 h=wl.get("h"))
    try:
        rhs = torch.from_numpy(f_host).to(stream.device, dt)
        phi = torch.empty_like(rhs)
        s.solve(phi, rhs, stream)
        torch.cuda.synchronize()
        err = None
        if ref is not None:
            err = float(np.abs(phi.double().cpu().numpy() - ref).max() / np.abs(ref).max())
        for _ in range(warmup):
            flush.zero_()
            s.solve(phi, rhs, stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            s.solve(phi, rhs, stream)
            b.record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    finally:
        s.close()
    return {"value": float(np.prod(wl["n"])) / (ms * 1e-3) / 1e6, "unit": "Mpts/s", "ms_per_step": ms,
            "dtype": DTYPES[wl["prec"]], "max_rel_err_vs_oracle": err, "steps": K}


def run_profile(args):
    import torch

    from paper_2211_07777_gb300 import flups as F
    wl = workload(args.workload)
    dt = torch.float32 if wl["prec"] == 0 else torch.float64
    solver = F.Solver(wl["n"], wl["bc"], L=wl["L"], center=wl["center"], prec=wl["prec"], green=wl["kernel"],
                      h=wl.get("h"))
    rhs = torch.from_numpy(wl["rhs"]()).to("cuda", dt)
    phi = torch.empty_like(rhs)
    for _ in range(args.warmup + args.steps):
        solver.solve(phi, rhs)
    torch.cuda.synchronize()
    solver.close()
    print(json.dumps({"profile_run": args.workload, "solves": args.warmup + args.steps,
                      "launches_per_solve": solver.info["launches"]}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="unb128_f64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip timing the other arithmetic paths")
    ap.add_argument("--served-requests", type=int, default=4096)
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--fp64-engine", default="native", choices=["native", "df"],
                    help="served stream: FP64-class requests natively or on the double-float path (FP64 tolerance)")
    ap.add_argument("--profile", action="store_true",
                    help="only W warm-up and K solves, no checks or side measurements (for ncu captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)
    if args.workload == "served":
        return run_served(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
