"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/lne.h. No compute call is made (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lne.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lne_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2302_07084_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for must in ["lne_create", "lne_destroy", "lne_last_error", "lne_embed", "lne_sparsifier_counts",
                 "lne_sparsifier_csr", "lne_rsvd", "lne_propagate"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2302_07084_gb300 import lne
    assert sorted(lne.EXPORTED) == _declared()


def test_create_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.lne_create(ctypes.byref(h), 0)
    assert rc != 0 and not h.value


def test_binding_raises_without_library(tmp_path):
    from paper_2302_07084_gb300 import lne
    saved = lne._lib
    lne._lib = None
    try:
        with pytest.raises(RuntimeError):
            lne.load_library(str(tmp_path / "missing.so"))
    finally:
        lne._lib = saved


def _header_defines():
    src = open(os.path.join(ROOT, "include", "lne.h")).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define (LNE_[A-Z0-9_]+)\s+(-?\d+)", src, re.M)}


def test_binding_constants_match_header():
    """Every option, aggregation, sketch and precision constant of the binding
    has the value the header defines (the binding passes them through)."""
    from paper_2302_07084_gb300 import lne
    h = _header_defines()
    pairs = {name[4:]: value for name, value in h.items()
             if name.startswith(("LNE_OPT_", "LNE_AGG_", "LNE_SKETCH_", "LNE_PREC_"))}
    assert len(pairs) >= 15
    for short, value in pairs.items():
        assert getattr(lne, short) == value, short
    for code, name in lne.ERRORS.items():
        assert h[name] == code, name
