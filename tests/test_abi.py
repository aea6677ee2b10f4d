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


C_CALLER = r"""
#include <stdio.h>
#include "sr.h"
int main(void) {
  sr_ctx* ctx = NULL;
  sr_obs o;
  int rc = sr_create(&ctx, 64, 1.0, 0.05, 1.5, 16, 16, 1);
  if (rc != SR_OK) { printf("%s\n", sr_strerror(rc)); return 1; }
  rc = sr_run_window(ctx, 0.0, 1.0);
  if (rc == SR_OK) rc = sr_observables(ctx, &o);
  sr_destroy(ctx);
  return rc == SR_OK ? 0 : 1;
}
"""


def test_header_is_plain_c_and_links_without_gpu(tmp_path):
    """A C99 caller of the four boundary calls compiles against include/sr.h
    with every warning an error, and links against libsr (it is not run)."""
    import shutil
    import subprocess
    from paper_cs_0405053_gb300 import _build
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = _build.build()
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", os.path.dirname(lib), "-lsr"], check=True)
    assert exe.exists()
