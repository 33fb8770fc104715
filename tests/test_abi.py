"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/cimmino.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "cimmino.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cimmino_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("cimmino_setup", "cimmino_solve", "cimmino_free", "cimmino_aat"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1710_07769_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    import paper_1710_07769_gb300 as g
    assert sorted(g.EXPORTS) == declared()
    assert b"sm_103a" in g.load().cimmino_version()


def test_opts_defaults_without_gpu():
    import paper_1710_07769_gb300 as g
    L = g.load()
    o = g.OptsStruct()
    L.cimmino_opts_default(ctypes.byref(o))
    assert o.precision == g.FP64 and o.layout == g.SKYLINE
    assert o.max_iter == 10000 and o.refine_tol == 1e-12 and o.pivot_ratio_min == 1e-4
    assert o.multi_rhs == 1 and o.keep_aat == 0 and o.use_graph == 1 and o.refine_relax == 0
    assert o.ruiz_sweeps == 0 and o.time_proj == 0


def test_selftest_rejects_bad_limit_without_gpu():
    """The watchdog self-test validates its arguments before any CUDA call."""
    import paper_1710_07769_gb300 as g
    assert g.selftest_wait(limit_us=0)[0] == g.EINVAL
    assert g.selftest_wait(limit_us=2_000_000)[0] == g.EINVAL
