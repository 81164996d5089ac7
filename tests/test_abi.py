"""The C-ABI library builds, loads and exports every function that
include/*.h declares (no compute calls: no GPU is needed)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(cpt_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2510_25143_gb300 import build
    lib = ctypes.CDLL(build.build())
    names = _declared()
    assert {"cpt_compress", "cpt_decompress", "cpt_extract_trajectories", "cpt_free",
            "cpt_error_string"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_error_strings_and_version():
    from paper_2510_25143_gb300 import cpt
    L = cpt.lib()
    assert L.cpt_error_string(0) == b"ok"
    assert L.cpt_error_string(-4) == b"corrupt stream"
    assert L.cpt_version() & 0xFF == 1


def test_oracle_builds_separately():
    import oracle
    path = oracle.build()
    assert os.path.exists(path) and "oracle" in path
