"""Host-side logic of the served stream (no device work)."""
import numpy as np

from paper_2211_07777_gb300 import workloads as W
from paper_2211_07777_gb300 import serve


def test_stream_is_seeded_and_admissible():
    a = W.served_stream(nreq=300, seed=4)
    b = W.served_stream(nreq=300, seed=4)
    assert [(r.n, r.bc, r.op, r.prec, r.arrival_s) for r in a] == [(r.n, r.bc, r.op, r.prec, r.arrival_s) for r in b]
    for r in a:
        assert r.n[0] in W.SERVED_SIZES and r.n[0] == r.n[1] == r.n[2]
        for l, rr in r.bc:
            assert (l == W.PER) == (rr == W.PER)          # periodic only in pairs
        assert r.kernel == (2 if any(W.UNB in f for f in r.bc) else 0)
    gaps = np.diff([r.arrival_s for r in a])
    assert np.all(gaps > 0) and abs(gaps.mean() * 1000.0 - 1.0) < 0.2   # Poisson arrivals at 1 kHz
    frac_bs = np.mean([r.op == 1 for r in a])
    assert 0.2 < frac_bs < 0.4


def test_vector_bc_wall_rule_is_consistent_for_the_curl():
    """The curl of a field with wall-rule conditions has well-defined conditions: both terms of
    each component agree along every direction."""
    E, O, U, P = W.EVEN, W.ODD, W.UNB, W.PER
    sw = serve.swap
    for bc in [((U, U), (U, U), (E, O)), ((P, P), (O, U), (E, E)), ((U, E), (P, P), (O, O))]:
        f = serve.vector_bc(bc)
        for c in range(3):
            a, b = (c + 1) % 3, (c + 2) % 3
            for d in range(3):
                t1 = tuple(sw(x) for x in f[b][d]) if d == a else f[b][d]
                t2 = tuple(sw(x) for x in f[a][d]) if d == b else f[a][d]
                assert t1 == t2


def test_request_marshalling_and_fp64_engine_policy():
    """A served request becomes the C request the server plans from: the precision follows the FP64
    engine policy, Biot-Savart requests carry the wall-rule conditions of all three components, the
    spacing is L / n (cell-centred) and the kernel is the stream's."""
    from paper_2211_07777_gb300 import flups as F
    reqs = W.served_stream(nreq=200, seed=4)
    for r in reqs[:60]:
        for eng in ("native", "df"):
            c = serve.c_request(r, eng)
            want = F.F64E if (eng == "df" and r.prec == F.F64) else r.prec
            assert c.prec == want and serve.engine_prec(r, eng) == want
            assert list(c.n) == list(r.n) and c.op == r.op and c.green == r.kernel and c.center == F.CELL
            assert list(c.h) == [1.0 / r.n[d] for d in range(3)]
            bc = serve.vector_bc(r.bc) if r.op == F.BIOT_SAVART else (r.bc,)
            flat = [b for comp in bc for d in comp for b in d]
            assert list(c.bc)[:len(flat)] == flat and all(v == 0 for v in list(c.bc)[len(flat):])
