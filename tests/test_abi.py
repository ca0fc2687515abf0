"""The C ABI library builds, loads and exports every declared symbol; host-side
validation of the entry points (no device work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            names += re.findall(r"^\s*(?:int|const char\*)\s+(flups_\w+)\s*\(", txt, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2211_07777_gb300 import build as B
    B.build()
    from paper_2211_07777_gb300 import flups as F
    return F


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    L = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(lib.EXPORTED) <= set(names)


def test_strerror(lib):
    assert lib.lib().flups_strerror(0).decode() == "ok"
    assert "boundary" in lib.lib().flups_strerror(-2).decode()


def _solver(F, n, bc, center=0, green="spectral", prec=1):
    t = F.flups_init_topo(n, center, 1, prec)
    try:
        h = [1.0 / (v if center == 0 else v - 1) for v in n]
        s = F.flups_init_solver(t, bc, h, (1.0, 1.0, 1.0), green)
        F.flups_cleanup(s)
    finally:
        F.flups_topo_free(t)


def test_host_validation(lib):
    F = lib
    P, U, E, O = F.PER, F.UNB, F.EVEN, F.ODD
    _solver(F, (16, 16, 16), ((P, P), (P, P), (P, P)))
    with pytest.raises(F.FlupsError) as e:
        _solver(F, (16, 16, 16), ((P, E), (P, P), (P, P)))
    assert e.value.status == -2
    with pytest.raises(F.FlupsError) as e:
        _solver(F, (20, 16, 16), ((P, P), (P, P), (P, P)))            # 20 = 2^2 5
    assert e.value.status == -3
    with pytest.raises(F.FlupsError) as e:
        _solver(F, (16, 16, 16), ((U, U), (P, P), (P, P)), green="spectral")   # singular kernel, unbounded
    assert e.value.status == -6
    with pytest.raises(F.FlupsError) as e:
        _solver(F, (16, 16, 16), ((U, U), (E, O), (P, P)), green="lgf2")
    assert e.value.status == -6
    with pytest.raises(F.FlupsError) as e:
        _solver(F, (4096, 16, 16), ((E, O), (P, P), (P, P)))          # 4N > 4096
    assert e.value.status == -3
    with pytest.raises(F.FlupsError) as e:
        F.flups_init_topo((16, 16, 16), 2, 1, 1)
    assert e.value.status == -1
    _solver(F, (16, 16, 16), ((U, U), (U, U), (U, U)), green="hej0")
    _solver(F, (33, 33, 33), ((E, E), (O, E), (P, P)), center=1, green="lgf2")
    _solver(F, (4, 4, 4), ((P, P), (U, U), (E, O)), green="hej2")      # the smallest grid: N = 4
    _solver(F, (2048, 4, 4), ((U, U), (P, P), (P, P)), green="hej2")   # the longest transform: 2N = 4096
    _solver(F, (1024, 4, 4), ((U, E), (P, P), (P, P)), green="hej2")   # semi-unbounded: 4N = 4096


@pytest.mark.parametrize("n", [(0, 16, 16), (16, 0, 16), (-8, 16, 16), (2, 16, 16), (3, 16, 16)])
def test_empty_negative_and_too_small_grids_are_refused(lib, n):
    F = lib
    with pytest.raises(F.FlupsError) as e:
        _solver(F, n, ((F.PER, F.PER),) * 3)
    assert e.value.status in (-1, -3)


def test_solve_before_setup_is_a_state_error(lib):
    F = lib
    t = F.flups_init_topo((16, 16, 16), 0, 1, 1)
    s = F.flups_init_solver(t, ((F.PER, F.PER),) * 3, (1 / 16,) * 3, (1.0,) * 3, "spectral")
    with pytest.raises(F.FlupsError) as e:
        F.flups_solve(s, 1, 1)
    assert e.value.status == -7
    F.flups_cleanup(s)
    F.flups_topo_free(t)


_FACES = {"PER": ("PER", "PER"), "UNB": ("UNB", "UNB"), "EE": ("EVEN", "EVEN"), "EO": ("EVEN", "ODD"),
          "OE": ("ODD", "EVEN"), "OO": ("ODD", "ODD"), "EU": ("EVEN", "UNB"), "OU": ("ODD", "UNB"),
          "UE": ("UNB", "EVEN"), "UO": ("UNB", "ODD")}


def _plan_order(F, types):
    bc = tuple(tuple(getattr(F, f) for f in _FACES[t]) for t in types)
    t = F.flups_init_topo((16, 16, 16), 0, 1, F.F64)
    try:
        s = F.flups_init_solver(t, bc, (1 / 16,) * 3, (1.0,) * 3, "hej2")
        try:
            return F.flups_solver_order(s)
        finally:
            F.flups_cleanup(s)
    finally:
        F.flups_topo_free(t)


@pytest.mark.parametrize("types,want", [
    (("UNB", "EE", "PER"), (1, 2, 0)),   # symmetric, then periodic, then unbounded
    (("PER", "PER", "PER"), (0, 1, 2)),  # ties keep x, y, z
    (("UE", "OO", "UNB"), (1, 0, 2)),    # symmetric < semi-unbounded < unbounded
    (("UNB", "UNB", "EO"), (2, 0, 1)),
    (("PER", "OU", "EE"), (2, 1, 0)),
])
def test_plan_order_follows_the_cost_classes(lib, types, want):
    """Section 1: directions are transformed cheapest first — symmetric, semi-unbounded,
    periodic, unbounded — ties in x, y, z order."""
    assert _plan_order(lib, types) == want


def test_plan_order_matches_the_oracle_for_every_type_triple(lib):
    import itertools
    import oracle
    for types in itertools.product(list(_FACES), repeat=3):
        assert _plan_order(lib, types) == tuple(oracle.direction_order(types)), types
