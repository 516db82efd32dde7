"""CPU-side checks of the C ABI: the library loads, exports every symbol the
header declares, and reports the geometry the oracle uses.  No GPU calls."""
import os
import re

import pytest

from oracle import oracle as O
from paper_2003_03174_b300 import build, trd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"TRD_API\s+[\w\s\*]+?\b(trd_\w+)\s*\(", text)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    L = trd.lib()
    decl = _declared()
    assert len(decl) >= 12
    missing = [n for n in decl if not hasattr(L, n)]
    assert not missing, missing
    assert set(trd.EXPORTED) <= set(decl)


def test_geometry_matches_oracle():
    g = trd.geometry()
    o = O.constants()
    for k in o:
        assert g[k] == pytest.approx(o[k], rel=0, abs=0), k


def test_version_string():
    assert "sm_103a" in trd.version()


def test_invalid_arguments_are_rejected_without_a_gpu():
    import ctypes as C
    L = trd.lib()
    assert L.trd_ctx_create(0, None) == trd.TRD_EINVAL
    assert L.trd_ctx_destroy(None) == trd.TRD_EINVAL
    assert L.trd_index_free(None) == trd.TRD_EINVAL
    assert L.trd_geometry(None, 3) == trd.TRD_EINVAL
    assert L.trd_refit(None, None, 0, None, None, 100.0, None, None) == trd.TRD_EINVAL
    h = C.c_void_p()
    rc = L.trd_ctx_create(0, C.byref(h))
    # no GPU in this container: the call must fail cleanly, never fall back
    assert rc in (trd.TRD_ECUDA, trd.TRD_OK)
    if rc == trd.TRD_OK:
        L.trd_ctx_destroy(h)
