"""CPU checks of the C ABI library: it builds for sm_103a, loads, and exports every
entry point that include/*.h declares (no compute call: there may be no GPU)."""
import ctypes
import glob
import os
import re

from paper_1509_05054_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(", src, flags=re.M):
            if not m.group(0).lstrip().startswith(("#", "typedef", "return")):
                names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dl_init", "dl_destroy", "dl_strerror", "omp_code", "jau_update", "dl_iterate"):
        assert required in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    lib = ctypes.CDLL(build.build())
    lib.dl_strerror.restype = ctypes.c_char_p
    assert lib.dl_strerror(0) == b"success"
    assert b"invalid" in lib.dl_strerror(-1)


def test_product_path_does_not_touch_the_oracle():
    """The package never imports, links or executes anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_1509_05054_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            txt = open(f).read()
            assert "import oracle" not in txt and "from oracle" not in txt, f
            assert "dl_oracle" not in txt and "liboracle" not in txt, f
