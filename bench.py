#!/usr/bin/env python3
"""Throughput of the Fourier Poisson solve (FLUPS method) on GB300: one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

A step is one full solve (all passes of the hot path) of the workload's
synthetic right-hand side, inputs resident in HBM, L2 flushed between steps.
Under torchrun (N > 1) every rank solves its own replica (weak scaling, no
data-path collective).

Default workload (`unb512_f32`): fully unbounded 3D Poisson, cell-centred
512^3 FP32 (doubled to 1024^3, R2C first), unit cube, unit-mass Gaussian blob
sigma = 0.1 centred at 0.5 + seeded 1e-3 jitter, HEJ2 kernel eps = 2h -- the
largest single-solve workload.  Beside it, on rank 0: the same workload in
double-float (FP64-class) and native FP64, the fully periodic 1024^3 FP64
workload (native and double-float), the served request stream (p50/p99), the
measured FP32/FP64 FMA peaks, the oracle on the host cores (one thread on a
bounded sample, and the full workload with a multi-threaded FFT when the host
has the memory) and the error of every result against the oracle or the
closed-form solution.  Other workloads: unb128_f64, unb128_f32, unb256_f32,
per32_f64, per256_f64, per1024_f64, mixed257_f32, mixed257_f64 (and _f64e
variants), served.
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
DEFAULT_WORKLOAD = "unb512_f32"
# the single-thread oracle runs on a bounded sample: the same workload at this size at most
CPU_SAMPLE_N = 256
METRIC = "Mpts/s per Poisson solve"


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
def workload(name):
    """dict(desc, n, bc, center, prec, kernel, rhs, L[, h], check) of a named workload."""
    E, O, P, U = W.EVEN, W.ODD, W.PER, W.UNB
    fam, _, tag = name.partition("_")
    if tag not in PRECS:
        raise SystemExit(f"unknown workload {name}")
    prec = PRECS[tag]
    if fam.startswith("unb") and fam[3:].isdigit():
        n = int(fam[3:])
        c = W.blob_center(2)
        desc = f"fully unbounded {n}^3 cell-centred {PREC_NAMES[prec]} (doubled {2*n}^3), " \
               f"HEJ2 eps=2h, Gaussian blob sigma=0.1"
        return dict(desc=desc, n=(n, n, n), bc=((U, U),) * 3, center=W.CELL, prec=prec, kernel="hej2",
                    rhs=lambda: W.gaussian_blob((n, n, n), 0.1, c), L=(1.0, 1.0, 1.0),
                    check=("gaussian", 0.1, c, 2.0 / n))
    if fam.startswith("unb") and all(t.isdigit() for t in fam[3:].split("x")) and fam.count("x") == 2:
        # non-cubic unbounded box (small cases of the long transforms for profiling), h = 1/max(n)
        n = tuple(int(t) for t in fam[3:].split("x"))
        hh = 1.0 / max(n)
        Lb = tuple(v * hh for v in n)
        c = tuple(0.5 * v for v in Lb)
        desc = f"fully unbounded {n[0]}x{n[1]}x{n[2]} cell-centred {PREC_NAMES[prec]} (doubled), HEJ2 eps=2h, " \
               f"Gaussian blob sigma=0.1 L/max(n)"
        return dict(desc=desc, n=n, bc=((U, U),) * 3, center=W.CELL, prec=prec, kernel="hej2",
                    rhs=lambda: W.gaussian_blob(n, 0.1 * min(Lb), c, L=Lb), L=Lb, check=None)
    if fam.startswith("per") and fam[3:].isdigit():
        n = int(fam[3:])
        seed = 1 if n == 32 else 5
        modes = W.sine_modes(seed)
        desc = f"fully periodic {n}^3 cell-centred {PREC_NAMES[prec]}, spectral kernel, 4 seeded sine products"
        return dict(desc=desc, n=(n, n, n), bc=((P, P),) * 3, center=W.CELL, prec=prec, kernel="spectral",
                    rhs=lambda: W.periodic_sines((n, n, n), modes), L=(1.0, 1.0, 1.0),
                    rhs_device=lambda dev, dt: W.periodic_sines_torch((n, n, n), modes, dev, dt),
                    check=("sines", modes))
    if fam.startswith("per") and all(t.isdigit() for t in fam[3:].split("x")) and fam.count("x") == 2:
        # non-cubic periodic box (small cases of the long transforms for profiling), h = 1/max(n)
        n = tuple(int(t) for t in fam[3:].split("x"))
        Lb = tuple(v / max(n) for v in n)
        modes = W.sine_modes(5)
        desc = f"fully periodic {n[0]}x{n[1]}x{n[2]} cell-centred {PREC_NAMES[prec]}, spectral kernel"
        return dict(desc=desc, n=n, bc=((P, P),) * 3, center=W.CELL, prec=prec, kernel="spectral",
                    rhs=lambda: W.periodic_sines(n, modes, L=1.0), L=Lb, check=None)
    if fam == "mixed257":
        desc = "node-centred 257x256x257, x even-even (DCT-I), y periodic, z unbounded, HEJ2, " \
               f"{PREC_NAMES[prec]}, Gaussian blob sigma=0.08 + 4 seeded y-modes"
        return dict(desc=desc, n=(257, 256, 257), bc=((E, E), (P, P), (U, U)), center=W.NODE, prec=prec,
                    kernel="hej2", rhs=lambda: W.mixed_blob_modes(), L=(1.0, 1.0, 1.0), h=(1 / 256,) * 3,
                    check=None)
    raise SystemExit(f"unknown workload {name}")


def config_of(wl, name, world):
    """The `config` of both arms' lines (identical for the same workload and N)."""
    return {"workload": wl["desc"], "name": name, "l2": "flushed between timed steps (256 MB write)",
            "parallelism": f"replicas x{world}"}


def cpu_sample_name(name):
    """The bounded sample the single-thread oracle times: the same workload at <= 256^3."""
    fam, _, tag = name.partition("_")
    for pre in ("unb", "per"):
        if fam.startswith(pre) and fam[3:].isdigit() and int(fam[3:]) > CPU_SAMPLE_N:
            return f"{pre}{CPU_SAMPLE_N}_{tag}"
    return name


def rel_linf(a, b):
    return float(np.abs(a - b).max() / max(float(np.abs(b).max()), 1e-300))


# ---------------------------------------------------------------------------
# Closed-form checks (no oracle): the HEJ2-smoothed Gaussian potential of an
# unbounded blob, and the exact solution of the periodic sine products.
# ---------------------------------------------------------------------------
def closed_form_planes(wl, zidx):
    """Expected phi on the z-planes zidx, or None when the workload has no closed form."""
    chk = wl.get("check")
    n = wl["n"]
    if not chk:
        return None
    x = W.coords(n[0], 1.0, W.CELL)
    y = W.coords(n[1], 1.0, W.CELL)
    z = W.coords(n[2], 1.0, W.CELL)[np.asarray(zidx)]
    if chk[0] == "gaussian":
        # HEJ2 is Gaussian smoothing of width eps: phi = -erf(r / (sqrt2 s)) / (4 pi r), s^2 = sigma^2 + eps^2
        from scipy.special import erf
        _, sigma, c, eps = chk
        s = math.sqrt(sigma * sigma + eps * eps)
        r = np.sqrt((x[None, None, :] - c[0]) ** 2 + (y[None, :, None] - c[1]) ** 2 + (z[:, None, None] - c[2]) ** 2)
        rs = np.where(r > 0, r, 1.0)
        return np.where(r > 0, -erf(rs / (math.sqrt(2) * s)) / (4 * math.pi * rs), -1.0 / ((2 * math.pi) ** 1.5 * s))
    out = np.zeros((len(z), n[1], n[0]))
    for a, b, cc, A in chk[1]:
        out += -A / ((2 * math.pi) ** 2 * (a * a + b * b + cc * cc)) * np.sin(2 * math.pi * cc * z)[:, None, None] \
            * np.sin(2 * math.pi * b * y)[None, :, None] * np.sin(2 * math.pi * a * x)[None, None, :]
    return out


def sample_planes(n):
    return sorted({0, 1, n // 3, n // 2, n - 1})


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
# The CPU leg: the only part of the benchmark that runs the oracle (the
# cpu_baseline of the GPU line, the parity of the timed results, and the
# reference arm).
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


def host_mem_available():
    try:
        with open("/proc/meminfo") as fh:
            for ln in fh:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except Exception:
        pass
    return 0


def oracle_host_bytes(wl):
    """Peak host memory of one oracle solve (about 60 bytes per point of the extended box, measured)."""
    ext = 1
    for d in range(3):
        t = wl["bc"][d]
        ext *= wl["n"][d] * (2 if W.UNB in t else 1)
    return 60 * ext


def timed_oracle(wl, f, workers, steps=1):
    """Seconds per oracle solve (mean of `steps`) with `workers` FFT threads, and the last result."""
    import oracle
    used = oracle.set_fft_workers(workers)
    try:
        times, ref = [], None
        for _ in range(max(1, steps)):
            t0 = time.perf_counter()
            ref = oracle_solve(wl, f)
            times.append(time.perf_counter() - t0)
    finally:
        oracle.set_fft_workers(1)
    return float(np.mean(times)), used, ref


def sampled_direct_sums(wl, f, got, npts=2, seed=1):
    """Max deviation, relative to max|got|, of got at npts random points from the oracle's kernel
    summed directly over the whole grid (h^3 sum_j G(x_i - x_j) f_j: the unbounded solution's
    definition; HEJ2 workloads only)."""
    import oracle
    n = wl["n"]
    h = 1.0 / n[0]
    x = W.coords(n[0], 1.0, W.CELL)
    rng = np.random.default_rng(seed)
    scale = float(np.abs(got).max())
    worst = 0.0
    for _ in range(npts):
        i = rng.integers(0, n[0], size=3)
        r = np.sqrt((x - x[i[0]])[:, None, None] ** 2 + (x - x[i[1]])[None, :, None] ** 2
                    + (x - x[i[2]])[None, None, :] ** 2)
        val = h ** 3 * float(np.sum(oracle.green.hej2_3d(r, 2 * h) * f))
        worst = max(worst, abs(float(got[i[0], i[1], i[2]]) - val) / scale)
    return worst


def cpu_leg(name, wl, f_host, full_budget_s=240.0):
    """The oracle on this host.  (1) As it stands (NumPy FFT, one thread) on a bounded sample: one
    solve of the same workload at <= 256^3.  (2) The full workload, one solve, with the FFT on
    scipy.fft worker threads (one per core), when the host has the memory.  Returns (cpu_baseline,
    reference field of the full workload or None)."""
    cores = cores_used()
    sname = cpu_sample_name(name)
    swl = workload(sname)
    sf = f_host if sname == name else swl["rhs"]()
    sec1, _, sref = timed_oracle(swl, sf, 1)
    spts = float(np.prod(swl["n"]))
    base = {"value": spts / sec1 / 1e6, "unit": "Mpts/s", "cores": 1, "kind": "oracle",
            "sample": f"one full oracle solve of the same workload at {'x'.join(map(str, swl['n']))} "
                      f"(NumPy pocketfft, one thread, {sec1:.1f} s)"}
    ref = sref if sname == name else None
    pts = float(np.prod(wl["n"]))
    need = oracle_host_bytes(wl)
    if cores > 1 and need < 0.8 * host_mem_available():
        sec, used, fref = timed_oracle(wl, f_host, cores)
        base["multicore"] = {"value": pts / sec / 1e6, "unit": "Mpts/s", "cores": used, "kind": "oracle",
                             "sample": f"one full oracle solve of the workload at {'x'.join(map(str, wl['n']))} "
                                       f"with its FFTs on scipy.fft, workers={used} ({sec:.1f} s)"}
        ref = fref
    else:
        base["multicore"] = {"value": None, "cores": cores,
                             "sample": f"skipped: the full oracle solve needs ~{need / 2**30:.0f} GiB of host "
                                       f"memory, {host_mem_available() / 2**30:.0f} GiB available"}
    return base, ref


# ---------------------------------------------------------------------------
# GPU measurement
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
                  "passes_ct_f32.cu", "passes_ct_f64.cu", "passes_ct_df.cu", "passes_ct_df_large.cu",
                  "passes_ct_small.cu")


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


def fma_peaks(F):
    """Measured FP32 and FP64 FMA rates of this device (TFLOP/s), from the library's microbenchmark."""
    out = {}
    for prec, key, iters in ((0, "fp32_tflops", 20000), (1, "fp64_tflops", 2000)):
        best = 0.0
        for _ in range(3):
            tf, _ = F.flups_measure_fma_peak(prec, iters)
            best = max(best, tf)
        out[key] = best
    out["how"] = "flups_measure_fma_peak: 8 CTAs/SM x 256 threads x 8 independent FMA chains, CUDA events, best of 3"
    return out


def make_solver(F, wl):
    return F.Solver(wl["n"], wl["bc"], L=wl["L"], center=wl["center"], prec=wl["prec"], green=wl["kernel"],
                    h=wl.get("h"))


def timed_setup(F, torch, wl):
    """A solver of the workload and its setup time in ms: plan, twiddles and Green spectrum, host and
    device, synchronised on both sides.  The solve rates exclude it; the lines report it beside them."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = make_solver(F, wl)
    torch.cuda.synchronize()
    return s, (time.perf_counter() - t0) * 1e3


def device_rhs(torch, wl, dev, f_host=None):
    dt = torch.float32 if wl["prec"] == 0 else torch.float64
    if f_host is None and "rhs_device" in wl:
        return wl["rhs_device"](dev, dt)
    return torch.from_numpy(f_host if f_host is not None else wl["rhs"]()).to(dev, dt)


def roofline(pinfo, mean_pass, prec, peaks, workload_name):
    """Roofline of the dominant pass: HBM for FP32 and double-float, the FP64 FMA rate for FP64."""
    dom = int(np.argmax(mean_pass))
    kname = KIND_NAMES[pinfo[dom]["kind"]]
    hbm, hbm_src = measured_peaks()
    ach_gbs = pinfo[dom]["bytes"] / (mean_pass[dom] * 1e-3) / 1e9
    ach_tf = pinfo[dom]["flops"] / (mean_pass[dom] * 1e-3) / 1e12
    fp64 = peaks.get("fp64_tflops") if peaks else None
    if prec == 1 and fp64:
        roof = {"bound": "alu", "achieved": ach_tf, "peak": fp64, "unit": "TFLOP/s", "frac": ach_tf / fp64,
                "peak_source": "measured FP64 FMA rate (flups_measure_fma_peak) on this device",
                "hbm_achieved_gbs": ach_gbs, "hbm_frac": ach_gbs / hbm, "hbm_peak_gbs": hbm}
    else:
        roof = {"bound": "hbm", "achieved": ach_gbs, "peak": hbm, "unit": "GB/s", "frac": ach_gbs / hbm,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured"
                else "fallback 6.8 TB/s"}
        if prec == 2 and fp64:
            roof["fp64_equiv_tflops"] = ach_tf
            roof["fp64_equiv_over_measured_fp64_peak"] = ach_tf / fp64
    roof["kernel"] = kname
    roof["traffic"] = traffic_record(kname, workload_name)
    roof["algorithmic_bytes_per_launch"] = pinfo[dom]["bytes"]
    roof["algorithmic_flops_per_launch"] = pinfo[dom]["flops"]
    roof["launch_ms"] = float(mean_pass[dom])
    return roof


def timed_solves(torch, solver, phi, rhs, stream, flush, K, warmup, npass, clocks=None):
    """K solves after `warmup`, L2 flushed before each; per-pass CUDA events on `stream`.
    Returns (per-step ms list, per-pass ms array [K, npass])."""
    for _ in range(warmup):
        flush.zero_()
        solver.solve(phi, rhs, stream)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(npass + 1)] for _ in range(K)]
    for row in ev:              # torch creates the CUDA event at its first record
        for e in row:
            e.record(stream)
    torch.cuda.synchronize()
    for k in range(K):
        flush.zero_()            # L2 flush between timed solves (outside the per-step events)
        solver.solve_events(phi, rhs, ev[k], stream)
    torch.cuda.synchronize()
    step_ms = [ev[k][0].elapsed_time(ev[k][npass]) for k in range(K)]
    pass_ms = np.array([[ev[k][i].elapsed_time(ev[k][i + 1]) for i in range(npass)] for k in range(K)])
    return step_ms, pass_ms


def pass_records(pinfo, mean_pass):
    return [{"kernel": KIND_NAMES[p["kind"]], "axis": p["axis"], "P": p["P"], "ms": float(m),
             "gbs": p["bytes"] / (m * 1e-3) / 1e9} for p, m in zip(pinfo, mean_pass)]


def measure_variant(F, torch, name, f_host, ref, flush, stream, K, warmup, peaks):
    """Time another workload or arithmetic path (whole solves, per-pass events, L2 flushed); its
    error against `ref` (the oracle's field of the same input) or against the closed form."""
    wl = workload(name)
    s, setup_ms = timed_setup(F, torch, wl)
    try:
        rhs = device_rhs(torch, wl, stream.device, f_host)
        phi = torch.empty_like(rhs)
        s.solve(phi, rhs, stream)
        torch.cuda.synchronize()
        rec = {"dtype": DTYPES[wl["prec"]], "workload": wl["desc"], "setup_ms": setup_ms}
        if ref is not None:
            rec["max_rel_err_vs_oracle"] = rel_linf(phi.double().cpu().numpy(), ref)
        zidx = sample_planes(wl["n"][2])
        cf = closed_form_planes(wl, zidx)
        if cf is not None:
            rec["rel_err_vs_closed_form"] = rel_linf(phi[zidx].double().cpu().numpy(), cf)
            rec["closed_form_planes"] = zidx
        npass = s.info["launches"]
        pinfo = [s.pass_info(i) for i in range(npass)]
        step_ms, pass_ms = timed_solves(torch, s, phi, rhs, stream, flush, K, warmup, npass)
        ms = float(np.mean(step_ms))
        mean_pass = pass_ms.mean(axis=0)
        rec.update({"value": float(np.prod(wl["n"])) / (ms * 1e-3) / 1e6, "unit": "Mpts/s", "ms_per_step": ms,
                    "steps": K, "solve_hbm_frac": sum(p["bytes"] for p in pinfo) / (ms * 1e-3) / 1e9
                    / measured_peaks()[0], "roofline": roofline(pinfo, mean_pass, wl["prec"], peaks, name),
                    "passes": pass_records(pinfo, mean_pass), "device_status": s.check()})
        del rhs, phi
    finally:
        s.close()
        torch.cuda.empty_cache()
    return rec


SMALL_WORKLOADS = ("per32_f64", "per32_f64e", "per32_f32", "unb32_f64", "unb32_f32")


def small_record(F, torch, flush, stream, reps=200):
    """Latency of one small solve (the 32^3 configurations): the solve's five launches captured once
    in a CUDA graph; each timed replay starts with the L2 flushed (the flush outside the events);
    median over `reps` replays.  Also the eager launch of the same solve (host launches, L2 flushed)
    and the back-to-back time per solve of a graph of 32 solves (inputs L2-resident)."""
    out = {}
    stream = torch.cuda.Stream(device=stream.device)   # graphs are captured on a non-default stream
    for name in SMALL_WORKLOADS:
        wl = workload(name)
        s, setup_ms = timed_setup(F, torch, wl)
        try:
            rhs = device_rhs(torch, wl, stream.device)
            phi = torch.empty_like(rhs)
            with torch.cuda.stream(stream):
                s.solve(phi, rhs, stream)
            torch.cuda.synchronize()
            rec = {"workload": wl["desc"], "dtype": DTYPES[wl["prec"]], "setup_ms": setup_ms}
            zidx = sample_planes(wl["n"][2])
            cf = closed_form_planes(wl, zidx)
            if cf is not None:
                rec["rel_err_vs_closed_form"] = rel_linf(phi[zidx].double().cpu().numpy(), cf)
            g1, g32 = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
            with torch.cuda.graph(g1, stream=stream):
                s.solve(phi, rhs, torch.cuda.current_stream())
            with torch.cuda.graph(g32, stream=stream):
                for _ in range(32):
                    s.solve(phi, rhs, torch.cuda.current_stream())
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            evg = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            with torch.cuda.stream(stream):
                for _ in range(3):
                    g1.replay()
                    g32.replay()
                for a, b in ev:         # eager: the solve's launches from the host
                    flush.zero_()
                    a.record(stream)
                    s.solve(phi, rhs, stream)
                    b.record(stream)
                for a, b in evg:        # graph replay of one solve
                    flush.zero_()
                    a.record(stream)
                    g1.replay()
                    b.record(stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(10):
                    g32.replay()
                e1.record(stream)
            torch.cuda.synchronize()
            rec.update({
                "graph_us": float(np.median([a.elapsed_time(b) for a, b in evg]) * 1e3),
                "eager_us": float(np.median([a.elapsed_time(b) for a, b in ev]) * 1e3),
                "back_to_back_us": float(e0.elapsed_time(e1) / 320 * 1e3),
                "launches": s.info["launches"], "reps": reps, "device_status": s.check()})
            out[name] = rec
            del g1, g32, rhs, phi
        finally:
            s.close()
    return out


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


def default_variants(name):
    """The other measurements of the default line: the same workload's other arithmetic paths and,
    for the largest unbounded workload, the fully periodic 1024^3 workload (native FP64 and
    double-float)."""
    fam, _, tag = name.partition("_")
    out = [f"{fam}_{t}" for t in ("f32", "f64e", "f64") if t != tag]
    if fam == "unb512":
        out += ["per1024_f64", "per1024_f64e"]
    return out


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
    f_host = wl["rhs"]()
    pts = float(np.prod(wl["n"]))
    peaks = fma_peaks(F) if rank == 0 else {}
    solver, setup_ms = timed_setup(F, torch, wl)
    rhs = device_rhs(torch, wl, dev, f_host)
    phi = torch.empty_like(rhs)
    stream = torch.cuda.current_stream(dev)
    npass = solver.info["launches"]
    pinfo = [solver.pass_info(i) for i in range(npass)]
    flush = L2Flush(torch, dev)

    # the timed region: K solves, barrier + synchronize on both sides, clocks sampled throughout
    for _ in range(args.warmup):
        flush.zero_()
        solver.solve(phi, rhs, stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    K = args.steps
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        step_ms, pass_ms = timed_solves(torch, solver, phi, rhs, stream, flush, K, 0, npass)
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
    total_ms, ms_per_step, value = aggregate_replicas(float(np.sum(step_ms)), pts, K, world, dist, dev)
    mean_pass = pass_ms.mean(axis=0)
    hbm, _ = measured_peaks()
    model_bytes = sum(p["bytes"] for p in pinfo)
    got = phi.double().cpu().numpy() if rank == 0 else None
    zidx = sample_planes(wl["n"][2])
    cf = closed_form_planes(wl, zidx) if rank == 0 else None

    # e2e: public API with pinned host buffers, the transfers inside every step
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
    device_status = solver.check()
    solver.close()
    del rhs, phi
    torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[prec], "data": "synthetic",
        "config": config_of(wl, args.workload, world),
        "max_rel_err_vs_oracle": None,
        "passes": pass_records(pinfo, mean_pass),
        "solve_hbm_frac": model_bytes / (ms_per_step * 1e-3) / 1e9 / hbm,
        "roofline": roofline(pinfo, mean_pass, prec, peaks, args.workload),
        "e2e": {"value": e2e_val, "unit": "Mpts/s", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "host_path": host_path},
        "gpu_launches": K * npass,
        "clocks": clk.summary(),
        "device_status": device_status,
        "peaks": peaks,
        "setup_ms": setup_ms,
    }
    if cf is not None:
        line["rel_err_vs_closed_form"] = rel_linf(got[zidx], cf)
        line["closed_form_planes"] = zidx
        line["closed_form"] = ("HEJ2-smoothed Gaussian potential -erf(r/(sqrt2 s))/(4 pi r), s^2 = sigma^2 + eps^2 "
                               "(the discrete solve matches it up to the blob's truncation at the box)"
                               if wl["check"][0] == "gaussian" else "exact: -sum A sin sin sin / |k|^2")

    # CPU baseline and parity against the oracle (rank 0, N = 1 only)
    ref = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], ref = cpu_leg(args.workload, wl, f_host)
        if ref is not None:
            line["max_rel_err_vs_oracle"] = rel_linf(got, ref)
            line["oracle_check"] = "every point against the oracle's solve of the same input"
        elif wl.get("check") and wl["check"][0] == "gaussian":
            line["max_rel_err_vs_oracle"] = sampled_direct_sums(wl, f_host, got)
            line["oracle_check"] = "2 sampled points against the oracle kernel's direct sum over the grid"

    # the same configuration in the other arithmetic paths, and the periodic 1024^3 workload
    if rank == 0 and not args.no_variants:
        variants = {}
        for vname in default_variants(args.workload):
            try:
                variants[vname] = measure_variant(F, torch, vname, f_host if vname.split("_")[0] ==
                                                  args.workload.split("_")[0] else None,
                                                  ref if vname.split("_")[0] == args.workload.split("_")[0] else None,
                                                  flush, stream, max(5, K // 4), args.warmup, peaks)
            except SystemExit:
                continue
        line["variants"] = variants

    # small solves (32^3): per-solve latency of graph-replayed and eager launches
    if rank == 0 and not args.no_variants:
        line["small"] = small_record(F, torch, flush, stream)

    # the served request stream: throughput with p50/p99 latency (rank 0, N = 1)
    if rank == 0 and world == 1 and not args.no_served:
        line["served"] = served_record(args)

    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def served_record(args):
    """Served stream: `served_requests` seeded requests, sizes {32..256}^3, random face conditions,
    30% Biot-Savart, FP32/FP64 50/50; closed-loop capacity, then Poisson arrivals at 0.8x capacity."""
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
    serve.run_stream(reqs[:64], budget, nstreams=args.streams, closed_loop=True, pool=pool, fp64_engine=eng)
    cap = serve.run_stream(reqs, budget, nstreams=args.streams, closed_loop=True, pool=pool, fp64_engine=eng)
    rate = 0.8 * cap["req_per_s"]
    nominal = 1.0 / np.mean(np.diff([r.arrival_s for r in reqs]))
    with ClockSampler(0) as clk:
        run = serve.run_stream(reqs, budget, nstreams=args.streams, time_scale=nominal / rate, pool=pool,
                               fp64_engine=eng)

    def alone(r, prec, engine="native"):
        rr = W.Request(**{**r.__dict__, "prec": prec if prec != F.F64E else F.F64})
        creq = serve.c_request(rr, "df" if prec == F.F64E else engine)
        bc = [[tuple(creq.bc[(c * 3 + d) * 2:(c * 3 + d) * 2 + 2]) for d in range(3)] for c in range(3)]
        sol = F.Solver(rr.n, bc if rr.op == F.BIOT_SAVART else bc[0], prec=prec, op=rr.op, green=rr.kernel)
        dt = torch.float32 if prec == F.F32 else torch.float64
        rhs = torch.from_numpy(np.ascontiguousarray(W.request_rhs(rr))).to("cuda", dt)
        phi = torch.empty_like(rhs)
        sol.solve(phi, rhs)
        torch.cuda.synchronize()
        out = phi.double().cpu().numpy()
        sol.close()
        return out

    # FP32 against FP64 on sampled request classes (same input): the stated error of the FP32 path
    errs = [rel_linf(alone(r, F.F32), alone(r, F.F64)) for r in [q for q in reqs if q.prec == F.F32][:8]]
    n_df = sum(1 for r in reqs if serve.engine_prec(r, eng) == F.F64E)
    df_errs = [rel_linf(alone(r, F.F64E), alone(r, F.F64))
               for r in [q for q in reqs if serve.engine_prec(q, eng) == F.F64E][:6]]
    run.pop("outputs", None)
    return {
        "metric": "served throughput (Mpts/s) with p50/p99 latency", "value": run["mpts_per_s"], "unit": "Mpts/s",
        "requests": nreq, "p50_ms": run["p50_ms"], "p99_ms": run["p99_ms"], "req_per_s": run["req_per_s"],
        "completed": run["completed"], "errors": run["errors"],
        "fp32": run.get("fp32"), "fp64": run.get("fp64"),
        "capacity_req_per_s": cap["req_per_s"], "capacity_mpts_per_s": cap["mpts_per_s"],
        "fp32_vs_fp64_max_rel_err": max(errs) if errs else None,
        "fp64_engine": {"policy": eng, "requests_on_double_float": n_df,
                        "double_float_vs_fp64_max_rel_err": max(df_errs) if df_errs else None},
        "config": {"workload": f"served stream: {nreq} seeded requests, sizes uniform on {{32..256}}^3, random face "
                               "conditions, 30% Biot-Savart Gaussian rings, FP32/FP64 50/50, Poisson arrivals at "
                               "0.8x measured capacity", "hbm_budget_bytes": budget, "streams": args.streams},
        "server": run["server"], "clocks": clk.summary(),
    }


def run_served(args):
    rec = served_record(args)
    line = {"metric": rec["metric"], "value": rec["value"], "unit": rec["unit"], "n_gpus": 1,
            "steps": rec["requests"], "warmup": 64, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {**rec["config"], "name": "served"}}
    line.update({k: v for k, v in rec.items() if k not in line})
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    """The reference arm: the oracle as it stands (NumPy, one thread) on the host cores, each step a
    bounded sample of the workload (the same workload at <= 256^3), about 150 s of CPU work at most."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    wl = workload(args.workload)
    sname = cpu_sample_name(args.workload)
    swl = workload(sname)
    f = swl["rhs"]()
    pts = float(np.prod(swl["n"]))
    t_end = time.perf_counter() + 60.0
    for _ in range(max(0, args.warmup)):
        oracle_solve(swl, f)
        if time.perf_counter() > t_end:
            break
    times = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        oracle_solve(swl, f)
        times.append(time.perf_counter() - t0)
        if sum(times) > 150.0:
            break
    sec = float(np.mean(times))
    val = pts / sec / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Mpts/s",
        "n_gpus": args.gpus, "steps": len(times), "steps_requested": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": config_of(wl, args.workload, world),
        "cpu_baseline": {"value": val, "unit": "Mpts/s", "cores": 1, "kind": "oracle",
                         "sample": f"{len(times)} full oracle solve(s) of the workload at "
                                   f"{'x'.join(map(str, swl['n']))} (NumPy pocketfft, one thread)"},
        "e2e": {"value": val, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_profile(args):
    import torch

    from paper_2211_07777_gb300 import flups as F
    wl = workload(args.workload)
    solver = make_solver(F, wl)
    rhs = device_rhs(torch, wl, torch.device("cuda", 0))
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
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the other workloads and arithmetic paths")
    ap.add_argument("--no-served", action="store_true", help="skip the served request stream")
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
