"""The serving runtime: each result is the same alone and in the mix; admission
by device memory (queueing, eviction, refusal); bad requests are refused
without disturbing the others; a seeded stream replays identically."""
import numpy as np
import pytest

from paper_2211_07777_gb300 import flups as F
from paper_2211_07777_gb300 import serve
from paper_2211_07777_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _small_stream(n=24, seed=11):
    reqs = W.served_stream(nreq=n, seed=seed, sizes=(16, 24, 32))
    return reqs


def _alone(req):
    import torch
    r = serve.c_request(req)
    bc = [[tuple(r.bc[(c * 3 + d) * 2:(c * 3 + d) * 2 + 2]) for d in range(3)] for c in range(3)]
    bc = bc if req.op == F.BIOT_SAVART else bc[0]
    s = F.Solver(req.n, bc, prec=req.prec, op=req.op, green=req.kernel)
    try:
        f = W.request_rhs(req)
        dt = torch.float32 if req.prec == F.F32 else torch.float64
        rhs = torch.from_numpy(np.ascontiguousarray(f)).to("cuda", dt)
        phi = torch.empty_like(rhs)
        s.solve(phi, rhs)
        torch.cuda.synchronize()
        return phi.cpu().numpy()
    finally:
        s.close()


def test_results_alone_equal_results_in_the_mix():
    reqs = _small_stream()
    budget = 256 << 20
    out = serve.run_stream(reqs, budget, nstreams=4, closed_loop=True, keep={r.rid for r in reqs})
    assert out["completed"] == len(reqs) and out["errors"] == 0
    assert out["server"]["plan_hits"] > 0
    for r in reqs:
        ref = _alone(r)
        got = out["outputs"][r.rid].numpy()
        tol = 1e-12 if r.prec == F.F64 else 1e-5
        assert np.abs(got - ref).max() <= tol * max(np.abs(ref).max(), 1e-300), r.rid


def _oracle(req):
    """The FP64 oracle's result for a served request: oracle.solve, or oracle.biot_savart with the
    per-component face conditions the server applies (serve.vector_bc)."""
    import oracle
    f = W.request_rhs(req)
    h = tuple(1.0 / v for v in req.n)
    kernel = "hej2" if req.kernel == F.HEJ2 else "spectral"
    if req.op == F.BIOT_SAVART:
        return oracle.biot_savart(f, serve.vector_bc(req.bc), h, center=oracle.CELL, kernel=kernel)
    return oracle.solve(f, oracle.Problem(bc=req.bc, h=h, center=oracle.CELL, kernel=kernel))


def _extra_requests(rid0):
    """32^3 and 64^3 requests with unbounded, semi-unbounded and symmetric faces, both precisions,
    Poisson and Biot-Savart, arriving in the same stream."""
    E, O, P, U = F.EVEN, F.ODD, F.PER, F.UNB
    specs = [
        ((32, 32, 32), ((U, U), (E, O), (P, P)), 0, F.F64),
        ((64, 64, 64), ((O, U), (U, E), (U, U)), 0, F.F32),
        ((64, 64, 64), ((E, E), (O, O), (U, U)), 0, F.F64),
        ((32, 32, 32), ((U, U), (U, U), (E, U)), 1, F.F64),
        ((64, 64, 64), ((U, U), (U, U), (O, E)), 1, F.F32),
        ((32, 32, 32), ((P, P), (P, P), (O, O)), 1, F.F64),
    ]
    out = []
    for i, (n, bc, op, prec) in enumerate(specs):
        kernel = F.HEJ2 if any(F.UNB in b for b in bc) else F.SPECTRAL
        out.append(W.Request(rid=rid0 + i, arrival_s=0.0, n=n, bc=bc, op=op, prec=prec, kernel=kernel))
    return out


def test_served_results_match_the_oracle():
    """Every result of a mixed stream (sizes 16-64, random face conditions, Biot-Savart vortex rings,
    FP32 and FP64, solved concurrently in slots) against the FP64 oracle, element by element:
    rel. L-inf <= 1e-12 (FP64) or 1e-5 (FP32) of the whole field's max."""
    reqs = _small_stream() + _extra_requests(1000)
    out = serve.run_stream(reqs, 512 << 20, nstreams=4, closed_loop=True, keep={r.rid for r in reqs})
    assert out["completed"] == len(reqs) and out["errors"] == 0
    assert any(r.op == F.BIOT_SAVART for r in reqs) and any(r.prec == F.F32 for r in reqs)
    for r in reqs:
        ref = _oracle(r)
        got = out["outputs"][r.rid].numpy().astype(np.float64).reshape(ref.shape)
        tol = 1e-12 if r.prec == F.F64 else 1e-5
        err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
        assert err <= tol, (r.rid, r.n, r.bc, r.op, r.prec, err)


def _need(req):
    """Device bytes of one plan plus one slot for this request (host-only query)."""
    r = serve.c_request(req)
    t = F.flups_init_topo(req.n, F.CELL, 3 if req.op == F.BIOT_SAVART else 1, req.prec)
    bc = [[tuple(r.bc[(c * 3 + d) * 2:(c * 3 + d) * 2 + 2]) for d in range(3)] for c in range(3)]
    s = F.flups_init_solver(t, bc if req.op == F.BIOT_SAVART else bc[0], list(r.h), list(r.L), req.kernel, 2.0,
                            req.op)
    m = F.flups_solver_memory(s)
    F.flups_cleanup(s)
    F.flups_topo_free(t)
    io = int(np.prod(req.n)) * (4 if req.prec == F.F32 else 8)
    return m["resident"] + m["transient"] + m["workspace"] + 2 * io


def test_double_float_engine_in_the_mix_matches_native_fp64():
    """With the df policy, FP64-class Poisson requests on power-of-two grids run on the
    double-float path in the mix; each result stays within the FP64 tolerance of its native
    FP64 solve alone."""
    reqs = W.served_stream(nreq=16, seed=15, sizes=(32, 64))
    assert any(serve.engine_prec(r, "df") == F.F64E for r in reqs)
    out = serve.run_stream(reqs, 512 << 20, nstreams=4, closed_loop=True, keep={r.rid for r in reqs},
                           fp64_engine="df")
    assert out["completed"] == len(reqs) and out["errors"] == 0
    for r in reqs:
        ref = _alone(r)
        got = out["outputs"][r.rid].numpy()
        tol = 1e-12 if r.prec == F.F64 else 1e-5
        assert np.abs(got - ref).max() <= tol * max(np.abs(ref).max(), 1e-300), r.rid


def test_admission_by_memory_queues_evicts_and_refuses():
    import torch
    U, P = F.UNB, F.PER
    A = [W.Request(rid=i, arrival_s=0.0, n=(32, 32, 32), bc=((U, U),) * 3, op=0, prec=F.F64, kernel=2)
         for i in range(4)]
    B = [W.Request(rid=10 + i, arrival_s=0.0, n=(32, 32, 32), bc=((P, P), (P, P), (U, U)), op=0, prec=F.F64,
                   kernel=2) for i in range(2)]
    budget = int(1.2 * max(_need(A[0]), _need(B[0])))
    assert _need(A[0]) + _need(B[0]) > budget
    out = serve.run_stream(A + B, budget, nstreams=4, closed_loop=True, keep={r.rid for r in A + B})
    st = out["server"]
    assert out["completed"] == len(A + B) and out["errors"] == 0
    assert st["queued_max"] >= 2          # same-class requests wait for the one slot that fits
    assert st["evictions"] >= 1           # the second class needs the first one's memory
    assert st["hbm_peak"] <= budget
    for r in (A[0], A[3], B[1]):
        ref = _alone(r)
        got = out["outputs"][r.rid].numpy()
        assert np.abs(got - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1e-300)
    # a request that cannot fit even alone is refused at submission
    srv = F.flups_server_create(1 << 20, 2)
    try:
        big = W.Request(rid=0, arrival_s=0.0, n=(64, 64, 64), bc=((U, U),) * 3, op=0, prec=F.F64, kernel=2)
        x = torch.zeros(64 ** 3, dtype=torch.float64).pin_memory()
        with pytest.raises(F.FlupsError) as e:
            F.flups_server_submit(srv, serve.c_request(big), x, x)
        assert e.value.status == -4
    finally:
        F.flups_server_destroy(srv)


def test_bad_request_is_refused_without_disturbing_others():
    import torch
    reqs = _small_stream(n=6, seed=13)
    pool = serve.HostPool()
    srv = F.flups_server_create(256 << 20, 2)
    try:
        tickets = {}
        for r in reqs:
            out = pool.output(r)
            tickets[F.flups_server_submit(srv, serve.c_request(r), pool.input(r), out)] = (r, out)
            if r.rid == 2:
                bad = serve.c_request(r)
                bad.bc[0], bad.bc[1] = F.PER, F.EVEN          # periodic on one face only
                with pytest.raises(F.FlupsError) as e:
                    F.flups_server_submit(srv, bad, pool.input(r), pool.output(r))
                assert e.value.status == -2
        got = {}
        while len(got) < len(reqs):
            for tk, lat, st in F.flups_server_wait(srv):
                assert st == 0 and lat > 0
                got[tk] = tickets[tk]
        assert F.flups_server_get_stats(srv)["rejected"] == 1
        for tk, (r, out) in got.items():
            ref = _alone(r)
            tol = 1e-12 if r.prec == F.F64 else 1e-5
            assert np.abs(out.numpy() - ref).max() <= tol * max(np.abs(ref).max(), 1e-300)
    finally:
        F.flups_server_destroy(srv)


def test_seeded_stream_replays_identically():
    reqs = _small_stream(n=12, seed=14)
    keep = {r.rid for r in reqs}
    a = serve.run_stream(reqs, 128 << 20, nstreams=3, time_scale=0.5, keep=keep)
    b = serve.run_stream(reqs, 128 << 20, nstreams=3, time_scale=0.5, keep=keep)
    for rid in keep:
        assert np.array_equal(a["outputs"][rid].numpy(), b["outputs"][rid].numpy())


def test_shared_green_spectrum_outlives_the_first_solver():
    """Solvers that opt in share one stored Green spectrum when their data are the same (here x
    even-even vs odd-odd: both half-wave); releasing one leaves the other's results intact."""
    import torch
    import oracle
    U, P, E, O = F.UNB, F.PER, F.EVEN, F.ODD
    n = (32, 24, 16)
    h = tuple(1.0 / v for v in n)
    rng = np.random.default_rng(81)
    f = rng.standard_normal((n[2], n[1], n[0]))
    bcs = [((E, E), (P, P), (U, U)), ((O, O), (P, P), (U, U))]
    refs = [oracle.solve(f, oracle.Problem(bc=bc, h=h, center=oracle.CELL, kernel="hej2")) for bc in bcs]
    sols = [F.Solver(n, bc, prec=F.F64, green="hej2", share_green=True) for bc in bcs]
    rhs = torch.from_numpy(f).to("cuda", torch.float64)

    def run(s):
        phi = torch.empty_like(rhs)
        s.solve(phi, rhs)
        torch.cuda.synchronize()
        assert s.check() == 0
        return phi.cpu().numpy()

    try:
        for s, ref in zip(sols, refs):
            assert np.abs(run(s) - ref).max() <= 1e-12 * np.abs(ref).max()
        sols[0].close()
        again = F.Solver(n, bcs[0], prec=F.F64, green="hej2", share_green=True)   # a third user
        assert np.abs(run(sols[1]) - refs[1]).max() <= 1e-12 * np.abs(refs[1]).max()
        assert np.abs(run(again) - refs[0]).max() <= 1e-12 * np.abs(refs[0]).max()
        again.close()
    finally:
        for s in sols:
            s.close()
