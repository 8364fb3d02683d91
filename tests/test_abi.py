"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no compute calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"EDFA_API\s+[\w\s\*]+?\b(edfa_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_core_entry_points():
    names = declared()
    for n in ("edfa_build", "edfa_setup", "edfa_apply", "edfa_solve", "edfa_free"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2009_13916_gb300 as P
    L = P.lib()
    for n in declared():
        assert hasattr(L, n), n
    assert os.path.basename(P.lib_path()) == "libedfa.so"


def test_strerror_and_defaults_without_gpu():
    import paper_2009_13916_gb300 as P
    L = P.lib()
    assert L.edfa_strerror(0) == b"ok"
    assert b"converge" in L.edfa_strerror(5)
    o = P.Options()
    L.edfa_default_options(ctypes.byref(o))
    assert o.qmode == 0 and abs(o.thresh - 0.05) < 1e-15 and o.precision == 0
