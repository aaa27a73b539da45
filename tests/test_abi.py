"""The C-ABI library builds, loads and exports every entry point declared in include/*.h
(no compute call: this runs without a GPU)."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mb_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2606_15357_gb300.nvcc_build import build
    so = build()
    import ctypes
    L = ctypes.CDLL(so)
    names = declared_functions()
    assert {"mb_index_build", "mb_seed_batch", "mb_locate"} <= names
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    import paper_2606_15357_gb300 as mb
    L = mb.lib()
    assert L.mb_strerror(0) == b"ok"
    assert L.mb_strerror(-3) == b"output buffer too small"


def test_binding_rejects_bad_arguments_on_host():
    import ctypes
    import paper_2606_15357_gb300 as mb
    L = mb.lib()
    out = ctypes.c_void_p()
    assert L.mb_index_build(None, 0, None, 0, None, ctypes.byref(out)) == -1
    assert L.mb_index_info(None, None, None, None) == -1
    assert L.mb_index_load(b"/nonexistent/path/index.mbi", None, ctypes.byref(out)) == -6
