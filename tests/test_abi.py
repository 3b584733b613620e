"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that the headers in include/ declare (no GPU needed; no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    inc = os.path.join(ROOT, "include")
    src = "\n".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gm_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_header_symbols():
    from paper_2410_17133_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert len(syms) >= 20
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    lib.gm_version.restype = ctypes.c_char_p
    assert lib.gm_version().startswith(b"gm-gb300")


def test_binding_refuses_missing_library(tmp_path):
    import pytest
    import paper_2410_17133_gb300 as gm
    saved = gm._lib
    gm._lib = None
    try:
        with pytest.raises(ImportError):
            gm.load_library(str(tmp_path / "nope.so"))
    finally:
        gm._lib = saved


def test_binding_types_every_declared_call():
    """Every entry point the headers declare has a typed ctypes signature in
    the binding (argument marshalling only), and the binding declares nothing
    the headers do not."""
    import paper_2410_17133_gb300 as gm
    assert set(declared_symbols()) == set(gm._SIG)
