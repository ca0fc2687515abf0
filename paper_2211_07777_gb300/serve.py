"""Replay a request stream against the native serving runtime (C ABI flups_server_*).

The runtime itself (admission by device memory, plan and Green caches, slots
with captured CUDA graphs, streams) is native; this module only turns the
seeded request descriptions into C requests, keeps the host buffers, drives
the open- or closed-loop arrival process and summarises latencies.
"""
from __future__ import annotations

import time
from collections import defaultdict

import numpy as np

from . import flups as F
from . import workloads as W


def swap(b):
    return {W.EVEN: W.ODD, W.ODD: W.EVEN}.get(b, b)


def vector_bc(bc):
    """Face conditions of the three vorticity components: at a symmetric face the normal
    component takes the other parity (a wall), the tangential ones keep it."""
    out = []
    for c in range(3):
        comp = []
        for d in range(3):
            l, r = bc[d]
            comp.append((swap(l), swap(r)) if c == d else (l, r))
        out.append(tuple(comp))
    return tuple(out)


def engine_prec(req: W.Request, fp64_engine: str = "native") -> int:
    """Arithmetic path for a request.  FP64-class requests run natively, or -- with
    fp64_engine="df" -- on the double-float path (FP64 tolerance on the FP32 units)."""
    if fp64_engine == "df" and req.prec == F.F64:
        return F.F64E
    return req.prec


def c_request(req: W.Request, fp64_engine: str = "native"):
    bc = vector_bc(req.bc) if req.op == F.BIOT_SAVART else req.bc
    return F.make_request(req.n, bc, center=F.CELL, prec=engine_prec(req, fp64_engine), op=req.op,
                          green=req.kernel)


def _class_key(req):
    return (req.n, req.op, req.prec)


class HostPool:
    """Pinned host buffers: one input per request class (read only), outputs reused after completion."""

    def __init__(self):
        import torch
        self.torch = torch
        self.inputs = {}
        self.free = defaultdict(list)

    def input(self, req):
        key = _class_key(req)
        if key not in self.inputs:
            f = W.request_rhs(req)
            dt = self.torch.float32 if req.prec == F.F32 else self.torch.float64
            self.inputs[key] = self.torch.from_numpy(np.ascontiguousarray(f)).to(dt).pin_memory()
        return self.inputs[key]

    def output(self, req):
        key = _class_key(req)
        if self.free[key]:
            return self.free[key].pop()
        return self.torch.empty_like(self.input(req)).pin_memory()

    def release(self, req, buf):
        self.free[_class_key(req)].append(buf)


def run_stream(reqs, budget_bytes, nstreams=8, time_scale=1.0, closed_loop=False, keep=None, pool=None,
               fp64_engine="native", per_request=False):
    """Submit reqs (sorted by arrival) and collect completions.

    time_scale multiplies the arrival times (open loop); closed_loop submits all at once.
    keep: set of request ids whose outputs are copied out and returned.
    fp64_engine: "native" or "df" (see engine_prec).
    per_request: also return 'latency_s', the latency of every completed request by id.
    Returns a summary dict (+ 'outputs' for the kept ids)."""
    pool = pool or HostPool()
    for r in reqs:
        pool.input(r)
    server = F.flups_server_create(budget_bytes, nstreams)
    inflight = {}
    lat = {}
    outputs = {}
    errors = {}
    pts = {r.rid: float(np.prod(r.n)) * (3 if r.op == F.BIOT_SAVART else 1) for r in reqs}

    def collect(done):
        for tk, l, st in done:
            r, buf = inflight.pop(tk)
            if st != 0:
                errors[r.rid] = st
            else:
                lat[r.rid] = l
                if keep is not None and r.rid in keep:
                    outputs[r.rid] = buf.clone()
            pool.release(r, buf)

    try:
        t0 = time.perf_counter()
        for r in reqs:
            if not closed_loop:
                target = t0 + r.arrival_s * time_scale
                while True:
                    collect(F.flups_server_poll(server))
                    dt = target - time.perf_counter()
                    if dt <= 0:
                        break
                    time.sleep(min(dt, 2e-4))
            out = pool.output(r)
            tk = F.flups_server_submit(server, c_request(r, fp64_engine), pool.input(r), out)
            inflight[tk] = (r, out)
            collect(F.flups_server_poll(server))
        while inflight:
            collect(F.flups_server_wait(server))
        t_end = time.perf_counter()
        stats = F.flups_server_get_stats(server)
    finally:
        F.flups_server_destroy(server)
    makespan = t_end - t0
    L = np.array([lat[r.rid] for r in reqs if r.rid in lat])
    summary = {
        "requests": len(reqs), "completed": int(L.size), "errors": len(errors), "makespan_s": makespan,
        "req_per_s": L.size / makespan, "mpts_per_s": sum(pts[i] for i in lat) / makespan / 1e6,
        "p50_ms": float(np.percentile(L, 50) * 1e3) if L.size else None,
        "p99_ms": float(np.percentile(L, 99) * 1e3) if L.size else None,
        "mean_ms": float(L.mean() * 1e3) if L.size else None,
        "server": stats,
    }
    for prec, name in ((F.F32, "fp32"), (F.F64, "fp64")):
        Lp = np.array([lat[r.rid] for r in reqs if r.rid in lat and r.prec == prec])
        if Lp.size:
            summary[name] = {"completed": int(Lp.size), "p50_ms": float(np.percentile(Lp, 50) * 1e3),
                             "p99_ms": float(np.percentile(Lp, 99) * 1e3),
                             "mpts": sum(pts[r.rid] for r in reqs if r.rid in lat and r.prec == prec) / 1e6}
    if keep is not None:
        summary["outputs"] = outputs
    if per_request:
        summary["latency_s"] = dict(lat)
    return summary
