"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(stbem_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1811_05224_gb300 import build, capi
    if not os.path.exists(capi.LIB_PATH):
        build.build()
    lib = ctypes.CDLL(capi.LIB_PATH)
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(capi.EXPORTS) <= declared
    L = capi.load()
    assert L.stbem_version().decode().startswith("stbem")
