"""The binding's ctypes structures match the C header's layout: sizes and field offsets of
flups_request and flups_server_stats, printed by a small C program compiled against
include/flups_gpu.h with the host compiler (no device work)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

REQUEST = ("n", "center", "prec", "op", "diff", "bc", "h", "L", "green", "eps_over_h")
STATS = ("submitted", "admitted", "completed", "rejected", "failed", "queued_max", "plan_hits", "plan_misses",
         "slots_created", "evictions", "plans_cached", "hbm_in_use", "hbm_peak", "setup_seconds", "slot_seconds")


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", "#include \"flups_gpu.h\"", "int main(void) {"]
    for struct, fields in (("flups_request", REQUEST), ("flups_server_stats", STATS)):
        lines.append(f'  printf("{struct} size %zu\\n", sizeof({struct}));')
        for f in fields:
            lines.append(f'  printf("{struct} {f} %zu\\n", offsetof({struct}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        struct, field, value = line.split()
        layout[(struct, field)] = int(value)
    return layout


def test_ctypes_structures_match_the_header(tmp_path):
    from paper_2211_07777_gb300 import flups as F
    layout = _c_layout(tmp_path)
    for struct, cls, fields in (("flups_request", F.Request, REQUEST), ("flups_server_stats", F.ServerStats, STATS)):
        assert ctypes.sizeof(cls) == layout[(struct, "size")], struct
        assert [name for name, _ in cls._fields_] == list(fields), struct
        for f in fields:
            assert getattr(cls, f).offset == layout[(struct, f)], (struct, f)
