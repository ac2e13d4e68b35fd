"""The C-ABI library builds, loads and exports every symbol include/*.h
declares; the binding covers each of them.  No compute call (no GPU here)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(qcd_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def built_lib():
    from paper_1310_7087_gb300 import build
    return build.build()


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("qcd_lattice_create", "qcd_sweep", "qcd_measure", "qcd_lattice_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(declared_functions()) <= exported


def test_binding_covers_every_declared_symbol(built_lib):
    import paper_1310_7087_gb300 as q
    assert set(declared_functions()) == set(q.SIGNATURES)
    for name in declared_functions():
        assert callable(getattr(q, name)), name


def test_build_targets_sm_103a_only():
    from paper_1310_7087_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_no_cpu_fallback_without_library(tmp_path, monkeypatch):
    import paper_1310_7087_gb300 as q
    monkeypatch.setattr(q, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(q, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        q.lib()


def test_split_lattice_argument_checks_need_no_gpu(built_lib):
    """qcd_lattice_create_split rejects nt_device outside [0, Nt] before any
    CUDA call, leaving the handle null, and says why."""
    import paper_1310_7087_gb300 as q
    q._lib = None  # bind the freshly built library
    lib = q.lib()
    for nt_device in (-1, 5):
        h = ctypes.c_void_p(1234)
        rc = lib.qcd_lattice_create_split(ctypes.byref(h), 3, 4, 4, 5.7, 0, 0, q.QCD_FIELD_LINKS,
                                          q.QCD_FP32_COMPRESSED, q.QCD_HOT, 1, None, nt_device)
        assert rc == q.QCD_ERR_INVALID_ARG
        assert not h.value
        assert b"nt_device" in lib.qcd_last_error()
