"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/*.h declares; argument validation runs on the host without a GPU."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2009_14514_gb300 import build, rts, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(rts_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    declared = _declared()
    assert "rts_init" in declared and "rts_advance" in declared
    missing = declared - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    lib = C.CDLL(path)
    for name in declared:
        assert hasattr(lib, name)
    assert set(rts.EXPORTED) <= declared


def test_binding_struct_sizes_match_header():
    # the ctypes mirrors must have the C layout: compare with a tiny C probe compiled here
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "rts.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu\n", sizeof(rts_params), sizeof(rts_stats),
             offsetof(rts_params, dt_b), offsetof(rts_params, sched), offsetof(rts_stats, t_sim));
      return 0;
    }
    """
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(v) for v in subprocess.check_output([exe]).split()]
    assert vals == [C.sizeof(rts.RtsParams), C.sizeof(rts.RtsStats),
                    rts.RtsParams.dt_b.offset, rts.RtsParams.sched.offset, rts.RtsStats.t_sim.offset]


def _bad(**over):
    sc = scenes.wcsph_dam_break_8k()
    d = dict(sc.params)
    d.update(over)
    return sc, rts.make_params(d)


@pytest.mark.parametrize("over,needle", [
    (dict(block_edge=0.01), "block_edge"),
    (dict(grid_dim=[0, 4, 4]), "grid_dim"),
    (dict(n_levels=9), "n_levels"),
    (dict(level_mult=[1, 1, 4, 8]), "level_mult"),
    (dict(dt_b=0.0), "dt_b"),
    (dict(max_per_block=0), "max_per_block"),
    (dict(force_level=7), "force_level"),
    (dict(scheme=5), "scheme"),
])
def test_init_rejects_bad_parameters_on_the_host(over, needle):
    sc, P = _bad(**over)
    h = C.c_void_p()
    lib = rts.lib()
    st = lib.rts_init(C.byref(P), sc.n, sc.x.ctypes.data, sc.v.ctypes.data, sc.nb,
                      sc.xb.ctypes.data, None, C.byref(h))
    assert st == 1 and not h.value
    assert needle in lib.rts_last_error(None).decode()


def test_null_arguments_are_errors_not_crashes():
    lib = rts.lib()
    sc, P = _bad()
    assert lib.rts_init(C.byref(P), sc.n, None, None, 0, None, None, None) == 1
    h = C.c_void_p()
    assert lib.rts_init(C.byref(P), sc.n, None, None, 0, None, None, C.byref(h)) == 1
    for fn in ("rts_bin", "rts_classify_blocks", "rts_evaluate", "rts_wcsph_substep",
               "rts_pcisph_step", "rts_sync"):
        assert getattr(lib, fn)(None) == 1
    assert lib.rts_destroy(None) == 0
    assert lib.rts_last_error(None)
