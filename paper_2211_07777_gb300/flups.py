"""Python binding of the C ABI in include/flups_gpu.h (argument marshalling only).

Every function of the header is exposed under the same name; each raises
FlupsError on a non-zero status.  Device arrays are passed as torch CUDA
tensors (or raw integer device pointers); streams as torch.cuda.Stream or raw
handles.  The library is loaded from this package directory; if it is absent
the first call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflups_gpu.so")

EVEN, ODD, PER, UNB = 0, 1, 3, 4
CELL, NODE = 0, 1
F32, F64, F64E = 0, 1, 2
POISSON, BIOT_SAVART = 0, 1
SPECTRAL, HEJ0, HEJ2, HEJ4, HEJ6, HEJ8, HEJ10, LGF2 = 0, 1, 2, 4, 6, 8, 10, 100
DIFF_SPECTRAL, DIFF_FD2, DIFF_FD4, DIFF_FD6 = 0, 2, 4, 6
KERNELS = {"spectral": SPECTRAL, "hej0": HEJ0, "hej2": HEJ2, "hej4": HEJ4, "hej6": HEJ6, "hej8": HEJ8,
           "hej10": HEJ10, "lgf2": LGF2}

EXPORTED = (
    "flups_init_topo", "flups_topo_free", "flups_init_solver", "flups_setup", "flups_solve",
    "flups_solve_host", "flups_cleanup", "flups_solver_info", "flups_strerror", "flups_last_cuda_error",
    "flups_debug_special", "flups_solve_pass", "flups_pass_info", "flups_solve_events", "flups_solve_periodic_noalloc",
    "flups_setup_shared", "flups_cleanup_async", "flups_workspace_size", "flups_solve_ws", "flups_solver_memory",
    "flups_server_create", "flups_server_submit", "flups_server_poll", "flups_server_wait", "flups_server_pending",
    "flups_server_get_stats", "flups_server_destroy", "flups_solver_check", "flups_pass_features",
    "flups_solver_share_green", "flups_host_mapped", "flups_solver_order", "flups_workspace_status",
    "flups_debug_wait_limit", "flups_measure_fma_peak", "flups_debug_green",
)


class Request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("center", ctypes.c_int), ("prec", ctypes.c_int), ("op", ctypes.c_int),
                ("diff", ctypes.c_int), ("bc", ctypes.c_int * 18), ("h", ctypes.c_double * 3),
                ("L", ctypes.c_double * 3), ("green", ctypes.c_int), ("eps_over_h", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in ("submitted", "admitted", "completed", "rejected", "failed",
                                                   "queued_max", "plan_hits", "plan_misses", "slots_created",
                                                   "evictions", "plans_cached")] + \
               [("hbm_in_use", ctypes.c_size_t), ("hbm_peak", ctypes.c_size_t)] + \
               [("setup_seconds", ctypes.c_double), ("slot_seconds", ctypes.c_double)]


class FlupsError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = f"{where}: {_strerror(status)} ({status})"
        if status == -5:
            msg += f" [{lib().flups_last_cuda_error().decode()}]"
        super().__init__(msg)
        self.status = status


_LIB = None


def lib():
    """The loaded C library (raises if the CUDA extension has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA extension missing: {LIB_PATH} (run paper_2211_07777_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
        L.flups_init_topo.argtypes = [ip, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
        L.flups_topo_free.argtypes = [vp]
        L.flups_init_solver.argtypes = [vp, ip, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(vp)]
        L.flups_setup.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
        L.flups_solve.argtypes = [vp, vp, vp, vp]
        L.flups_solve_host.argtypes = [vp, vp, vp, vp]
        L.flups_cleanup.argtypes = [vp]
        L.flups_solver_info.argtypes = [vp, ip, ip, dp, dp]
        L.flups_strerror.argtypes = [ctypes.c_int]
        L.flups_strerror.restype = ctypes.c_char_p
        L.flups_last_cuda_error.restype = ctypes.c_char_p
        L.flups_debug_special.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.c_int, ctypes.c_double]
        L.flups_solve_pass.argtypes = [vp, ctypes.c_int, vp, vp, vp]
        L.flups_pass_info.argtypes = [vp, ctypes.c_int, ip, ip, ip, dp, dp]
        L.flups_solve_events.argtypes = [vp, vp, vp, vp, ctypes.POINTER(vp)]
        L.flups_solve_periodic_noalloc.argtypes = [vp, vp, ip, dp, vp]
        szp = ctypes.POINTER(ctypes.c_size_t)
        L.flups_setup_shared.argtypes = [vp, vp]
        L.flups_cleanup_async.argtypes = [vp, vp]
        L.flups_workspace_size.argtypes = [vp, szp]
        L.flups_solve_ws.argtypes = [vp, vp, vp, vp, vp]
        L.flups_solver_memory.argtypes = [vp, szp, szp, szp]
        L.flups_solver_check.argtypes = [vp, ip]
        L.flups_host_mapped.argtypes = [vp, ctypes.c_size_t]
        L.flups_solver_order.argtypes = [vp, ip]
        L.flups_solver_share_green.argtypes = [vp]
        L.flups_pass_features.argtypes = [vp, ctypes.c_int, ip]
        L.flups_workspace_status.argtypes = [vp, szp]
        L.flups_debug_wait_limit.argtypes = [vp, ctypes.c_int]
        L.flups_measure_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        L.flups_debug_green.argtypes = [vp, dp, dp, ctypes.c_longlong]
        llp = ctypes.POINTER(ctypes.c_longlong)
        L.flups_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(vp)]
        L.flups_server_submit.argtypes = [vp, ctypes.POINTER(Request), vp, vp, llp]
        L.flups_server_poll.argtypes = [vp, llp, dp, ip, ctypes.c_int, ip]
        L.flups_server_wait.argtypes = [vp, llp, dp, ip, ctypes.c_int, ip]
        L.flups_server_pending.argtypes = [vp, ip, ip]
        L.flups_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.flups_server_destroy.argtypes = [vp]
        for name in EXPORTED:
            if name not in ("flups_strerror", "flups_last_cuda_error"):
                getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


def _strerror(status: int) -> str:
    return lib().flups_strerror(int(status)).decode()


def _check(status: int, where: str):
    if status != 0:
        raise FlupsError(status, where)


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return s.cuda_stream


# --- the C ABI, one function each -------------------------------------------------
def flups_init_topo(n, center, ncomp, prec):
    h = ctypes.c_void_p()
    arr = (ctypes.c_int * 3)(*[int(v) for v in n])
    _check(lib().flups_init_topo(arr, int(center), int(ncomp), int(prec), ctypes.byref(h)), "flups_init_topo")
    return h


def flups_topo_free(topo):
    _check(lib().flups_topo_free(topo), "flups_topo_free")


def flups_init_solver(topo, bc, h, L, green, eps_over_h=2.0, op=POISSON, diff=DIFF_SPECTRAL):
    """bc: [comp][dir][face] nested sequence (ncomp x 3 x 2) or [dir][face] for one component."""
    flat = []
    if isinstance(bc[0][0], (list, tuple)):
        for comp in bc:
            for d in comp:
                flat.extend(int(b) for b in d)
    else:
        for d in bc:
            flat.extend(int(b) for b in d)
    arr = (ctypes.c_int * len(flat))(*flat)
    hh = (ctypes.c_double * 3)(*[float(v) for v in h])
    LL = (ctypes.c_double * 3)(*[float(v) for v in L])
    g = KERNELS[green] if isinstance(green, str) else int(green)
    s = ctypes.c_void_p()
    _check(lib().flups_init_solver(topo, arr, hh, LL, g, float(eps_over_h), int(op), int(diff), ctypes.byref(s)),
           "flups_init_solver")
    return s


def flups_setup(solver, stream=None) -> int:
    ws = ctypes.c_size_t(0)
    _check(lib().flups_setup(solver, _stream(stream), ctypes.byref(ws)), "flups_setup")
    return ws.value


def flups_solve(solver, phi, rhs, stream=None):
    _check(lib().flups_solve(solver, _ptr(phi), _ptr(rhs), _stream(stream)), "flups_solve")


def flups_solve_host(solver, phi_host, rhs_host, stream=None):
    _check(lib().flups_solve_host(solver, _ptr(phi_host), _ptr(rhs_host), _stream(stream)), "flups_solve_host")


def flups_solver_order(solver):
    """The planner's transform order: the directions (0 x, 1 y, 2 z) in the order they are transformed."""
    order = (ctypes.c_int * 3)()
    _check(lib().flups_solver_order(solver, order), "flups_solver_order")
    return tuple(order)


def flups_host_mapped(host, nbytes=None):
    """True if the host array (or nbytes from its address) is pinned memory the device addresses
    directly, i.e. flups_solve_host uses it in place."""
    if nbytes is None:
        nbytes = host.numel() * host.element_size() if hasattr(host, "element_size") else host.nbytes
    return bool(lib().flups_host_mapped(_ptr(host), nbytes))


def flups_cleanup(solver):
    _check(lib().flups_cleanup(solver), "flups_cleanup")


def flups_solver_info(solver):
    n = ctypes.c_int(0)
    order = (ctypes.c_int * 3)()
    mb = ctypes.c_double(0)
    gb = ctypes.c_double(0)
    _check(lib().flups_solver_info(solver, ctypes.byref(n), order, ctypes.byref(mb), ctypes.byref(gb)),
           "flups_solver_info")
    return {"launches": n.value, "order": list(order), "model_bytes": mb.value, "green_bytes": gb.value}


def flups_solve_pass(solver, i, phi, rhs, stream=None):
    _check(lib().flups_solve_pass(solver, int(i), _ptr(phi), _ptr(rhs), _stream(stream)), "flups_solve_pass")


def flups_solve_events(solver, phi, rhs, events, stream=None):
    """events: sequence of launches+1 torch.cuda.Event (or raw handles)."""
    hs = [e.cuda_event if hasattr(e, "cuda_event") else int(e) for e in events]
    arr = (ctypes.c_void_p * len(hs))(*hs)
    _check(lib().flups_solve_events(solver, _ptr(phi), _ptr(rhs), _stream(stream), arr), "flups_solve_events")


def flups_pass_info(solver, i):
    kind, axis, P = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    b, fl = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().flups_pass_info(solver, int(i), ctypes.byref(kind), ctypes.byref(axis), ctypes.byref(P),
                                 ctypes.byref(b), ctypes.byref(fl)), "flups_pass_info")
    return {"kind": kind.value, "axis": axis.value, "P": P.value, "bytes": b.value, "flops": fl.value}


def flups_solve_periodic_noalloc(phi, rhs, n, L, stream=None):
    """Allocation-free periodic FP64 solve (workspace in a fixed static device array)."""
    nn = (ctypes.c_int * 3)(*[int(v) for v in n])
    LL = (ctypes.c_double * 3)(*[float(v) for v in L])
    _check(lib().flups_solve_periodic_noalloc(_ptr(phi), _ptr(rhs), nn, LL, _stream(stream)),
           "flups_solve_periodic_noalloc")


def flups_setup_shared(solver, stream=None):
    _check(lib().flups_setup_shared(solver, _stream(stream)), "flups_setup_shared")


def flups_workspace_size(solver) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().flups_workspace_size(solver, ctypes.byref(b)), "flups_workspace_size")
    return b.value


def flups_workspace_status(solver) -> int:
    """Byte offset, within a workspace, of the device status word of the solve using it."""
    b = ctypes.c_size_t(0)
    _check(lib().flups_workspace_status(solver, ctypes.byref(b)), "flups_workspace_status")
    return b.value


def flups_debug_green(solver, n: int):
    """(FP64 samples, stored spectrum) of the solver's Green's function, n values each (numpy)."""
    import numpy as np
    a = np.zeros(n)
    b = np.zeros(n)
    _check(lib().flups_debug_green(solver, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(n)), "flups_debug_green")
    return a, b


def flups_debug_wait_limit(solver, mask: int):
    _check(lib().flups_debug_wait_limit(solver, int(mask)), "flups_debug_wait_limit")


def flups_measure_fma_peak(prec, iters):
    """(TFLOP/s, ms) of the FMA microbenchmark on the current device (prec F32 or F64)."""
    t, m = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().flups_measure_fma_peak(int(prec), int(iters), ctypes.byref(t), ctypes.byref(m)),
           "flups_measure_fma_peak")
    return t.value, m.value


def flups_solve_ws(solver, phi, rhs, workspace, stream=None):
    _check(lib().flups_solve_ws(solver, _ptr(phi), _ptr(rhs), _ptr(workspace), _stream(stream)), "flups_solve_ws")


def flups_solver_memory(solver):
    r, t, w = ctypes.c_size_t(0), ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(lib().flups_solver_memory(solver, ctypes.byref(r), ctypes.byref(t), ctypes.byref(w)),
           "flups_solver_memory")
    return {"resident": r.value, "transient": t.value, "workspace": w.value}


def flups_server_create(hbm_budget_bytes, nstreams=8):
    h = ctypes.c_void_p()
    _check(lib().flups_server_create(int(hbm_budget_bytes), int(nstreams), ctypes.byref(h)), "flups_server_create")
    return h


def make_request(n, bc, center=CELL, prec=F64, op=POISSON, diff=DIFF_SPECTRAL, h=None, L=(1.0, 1.0, 1.0),
                 green="spectral", eps_over_h=2.0):
    r = Request()
    r.n[:] = [int(v) for v in n]
    r.center, r.prec, r.op, r.diff = int(center), int(prec), int(op), int(diff)
    flat = []
    if isinstance(bc[0][0], (list, tuple)):
        for comp in bc:
            for d in comp:
                flat.extend(int(b) for b in d)
    else:
        for d in bc:
            flat.extend(int(b) for b in d)
    flat += [0] * (18 - len(flat))
    r.bc[:] = flat
    if h is None:
        h = [L[d] / (n[d] if center == CELL else n[d] - 1) for d in range(3)]
    r.h[:] = [float(v) for v in h]
    r.L[:] = [float(v) for v in L]
    r.green = KERNELS[green] if isinstance(green, str) else int(green)
    r.eps_over_h = float(eps_over_h)
    return r


def flups_server_submit(server, request, rhs_host, phi_host):
    t = ctypes.c_longlong(0)
    _check(lib().flups_server_submit(server, ctypes.byref(request), _ptr(rhs_host), _ptr(phi_host), ctypes.byref(t)),
           "flups_server_submit")
    return t.value


def _server_done(fn, server, maxn):
    tk = (ctypes.c_longlong * maxn)()
    lat = (ctypes.c_double * maxn)()
    st = (ctypes.c_int * maxn)()
    n = ctypes.c_int(0)
    _check(fn(server, tk, lat, st, maxn, ctypes.byref(n)), fn.__name__)
    return [(tk[i], lat[i], st[i]) for i in range(n.value)]


def flups_server_poll(server, maxn=1024):
    return _server_done(lib().flups_server_poll, server, maxn)


def flups_server_wait(server, maxn=1024):
    return _server_done(lib().flups_server_wait, server, maxn)


def flups_server_pending(server):
    q, r = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().flups_server_pending(server, ctypes.byref(q), ctypes.byref(r)), "flups_server_pending")
    return q.value, r.value


def flups_server_get_stats(server):
    st = ServerStats()
    _check(lib().flups_server_get_stats(server, ctypes.byref(st)), "flups_server_get_stats")
    return {k: getattr(st, k) for k, _ in ServerStats._fields_}


def flups_server_destroy(server):
    _check(lib().flups_server_destroy(server), "flups_server_destroy")


def flups_debug_special(which, x, y, out, n, eps):
    _check(lib().flups_debug_special(int(which), _ptr(x), _ptr(y), _ptr(out), int(n), float(eps)),
           "flups_debug_special")


# --- convenience wrapper ------------------------------------------------------------
class Solver:
    """One planned solve: Solver(n, bc, h=..., ...) then solve(phi, rhs) on CUDA tensors."""

    def __init__(self, n, bc, L=(1.0, 1.0, 1.0), center=CELL, prec=F64, green="spectral", eps_over_h=2.0,
                 op=POISSON, diff=DIFF_SPECTRAL, ncomp=None, h=None, stream=None, share_green=False):
        if ncomp is None:
            ncomp = 3 if op == BIOT_SAVART else 1
        self.n = tuple(int(v) for v in n)
        self.ncomp = ncomp
        self.prec = prec
        if h is None:
            # N = n (cell) or n - 1 (node); a node-centred periodic direction stored
            # without its duplicate node needs h given explicitly (h = L / n)
            h = [L[d] / (self.n[d] if center == CELL else self.n[d] - 1) for d in range(3)]
        self.h = tuple(h)
        self._topo = flups_init_topo(self.n, center, ncomp, prec)
        try:
            self._s = flups_init_solver(self._topo, bc, self.h, L, green, eps_over_h, op, diff)
        except Exception:
            flups_topo_free(self._topo)
            self._topo = None
            raise
        if share_green:
            _check(lib().flups_solver_share_green(self._s), "flups_solver_share_green")
        self.workspace_bytes = flups_setup(self._s, stream)
        self.info = flups_solver_info(self._s)

    def solve(self, phi, rhs, stream=None):
        flups_solve(self._s, phi, rhs, stream)

    def solve_pass(self, i, phi, rhs, stream=None):
        flups_solve_pass(self._s, i, phi, rhs, stream)

    def solve_events(self, phi, rhs, events, stream=None):
        flups_solve_events(self._s, phi, rhs, events, stream)

    def pass_info(self, i):
        return flups_pass_info(self._s, i)

    def solve_host(self, phi_host, rhs_host, stream=None):
        flups_solve_host(self._s, phi_host, rhs_host, stream)

    def features(self):
        """Per pass: dict(ct, staged_green, tma_green, pruned) (flups_pass_features)."""
        out = []
        for i in range(self.info["launches"]):
            f = ctypes.c_int(0)
            _check(lib().flups_pass_features(self._s, i, ctypes.byref(f)), "flups_pass_features")
            v = f.value
            out.append({"ct": bool(v & 1), "staged_green": bool(v & 2), "tma_green": bool(v & 4), "pruned": bool(v & 8),
                        "tma_input": bool(v & 16), "row_stages": bool(v & 32), "bulk_rows": bool(v & 64)})
        return out

    def debug_wait_limit(self, mask: int):
        """Test hook: bounded waits of the codes in mask (bit 0: code 1, bit 1: code 2) give up at once."""
        flups_debug_wait_limit(self._s, mask)

    def check(self) -> int:
        """Device-side status since the last check (0, or the code of a bounded wait that gave up)."""
        code = ctypes.c_int(0)
        _check(lib().flups_solver_check(self._s, ctypes.byref(code)), "flups_solver_check")
        return code.value

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def close(self):
        if getattr(self, "_s", None) is not None:
            flups_cleanup(self._s)
            self._s = None
        if getattr(self, "_topo", None) is not None:
            flups_topo_free(self._topo)
            self._topo = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

