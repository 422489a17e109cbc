"""The C-ABI library loads and exports every entry point include/*.h declares (CPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = "\n".join(ln for ln in text.splitlines() if not ln.lstrip().startswith("#"))
        text = re.sub(r"typedef[^;]*;", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\([^;{]*\)\s*;", text):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_03605_gb300 import build, pdmts
    build.build()
    return pdmts.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pd_create", "pd_set_precrack", "mts_set_time", "mts_advance", "pd_read_displacement",
                 "pd_read_damage", "pdmts_ctx_create"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2403_03605_gb300 import pdmts
    bound = {s[0] for s in pdmts.SIGNATURES}
    assert set(declared_functions()) <= bound, set(declared_functions()) - bound


def test_calls_without_gpu_fail_cleanly(lib):
    """With no device visible the context call returns an error code, not a crash."""
    import ctypes as C
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = lib.pdmts_ctx_create(C.byref(h), 0, None)
    assert rc < 0
    assert lib.pdmts_last_error()
