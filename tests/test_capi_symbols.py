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


def test_struct_layouts_match_the_binding(tmp_path):
    """Every C ABI struct as a C99 compiler lays it out from include/lne.h
    (size and each field's offset) equals the binding's ctypes mirror."""
    import shutil
    import subprocess
    from paper_2302_07084_gb300 import lne
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = tmp_path / "abi_layout"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "cpp", "abi_layout.c"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = dict((ln.rsplit(" ", 1)[0], int(ln.rsplit(" ", 1)[1])) for ln in out if ln.strip())
    mirrors = {"lne_graph": lne._Graph, "lne_params": lne._Params, "lne_csr": lne._Csr, "lne_counts": lne._Counts,
               "lne_task": lne._Task, "lne_trace_entry": lne._TraceEntry}
    # the binding's field names where they differ from the header's
    renames = {("lne_task", "labels_dev"): "labels", ("lne_task", "train_dev"): "train",
               ("lne_task", "test_dev"): "test"}
    checked = 0
    for cname, py in mirrors.items():
        assert c_layout[f"{cname} sizeof"] == ctypes.sizeof(py), cname
        c_fields = [k.split(".", 1)[1] for k in c_layout if k.startswith(cname + ".")]
        assert len(c_fields) == len(py._fields_), cname
        for f in c_fields:
            pf = renames.get((cname, f), f)
            assert c_layout[f"{cname}.{f}"] == getattr(py, pf).offset, (cname, f)
            checked += 1
    assert checked == sum(len(py._fields_) for py in mirrors.values())
