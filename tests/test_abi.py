"""The C ABI boundary, checked without a GPU: libsr builds for sm_103a and
exports every entry point include/sr.h declares; the CUDA path and the oracle
stay independent of each other."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sr_\w+)\s*\(", src,
                                 flags=re.M)))


def test_header_declares_the_four_core_calls():
    names = _declared()
    for core in ("sr_create", "sr_run_window", "sr_observables", "sr_destroy"):
        assert core in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_cs_0405053_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    import paper_cs_0405053_gb300 as sr
    lib = sr.library()
    assert lib.sr_strerror(0) == b"ok"
    assert b"converge" in lib.sr_strerror(sr.SR_NOT_CONVERGED)


def test_cuda_path_and_oracle_share_nothing():
    pkg = os.path.join(ROOT, "paper_cs_0405053_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b|sr_oracle|orc_", text), f
    text = open(os.path.join(ROOT, "oracle", "sr_oracle.c")).read()
    assert "sr_device" not in text and '#include "sr.h"' not in text
    from paper_cs_0405053_gb300 import _build
    syms = open(_build.build(), "rb").read()
    assert b"orc_philox" not in syms and b"orc_run" not in syms


def test_product_raises_without_library(tmp_path, monkeypatch):
    import paper_cs_0405053_gb300 as sr
    from paper_cs_0405053_gb300 import _build
    monkeypatch.setattr(sr, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(OSError):
        sr.library(build_if_missing=False)


def test_graph_launch_calls_reject_a_null_context_without_gpu():
    import paper_cs_0405053_gb300 as sr
    lib = sr.library()
    a, b = ctypes.c_ulonglong(7), ctypes.c_ulonglong(7)
    assert lib.sr_set_graph_launch(None, 1) == sr.SR_EINVAL
    assert lib.sr_get_graph_stats(None, ctypes.byref(a), ctypes.byref(b)) == sr.SR_EINVAL
    assert (a.value, b.value) == (7, 7)
