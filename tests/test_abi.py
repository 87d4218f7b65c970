"""The C-ABI library builds for sm_103a and exports every entry point that
include/mfpoisson.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

from paper_1611_03029_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mfp_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1611_03029_gb300 import mfpoisson
    lib = mfpoisson.lib()
    for n in declared_functions():
        assert getattr(lib, n).argtypes is not None or n == "mfp_last_error"
