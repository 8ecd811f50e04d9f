"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/ssa.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ssa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(ssa_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="CUDA toolkit not present")
def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_1309_5050_gb300 import _lib, build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 14, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_lib.EXPORTS) <= set(names)
    # host-only entry points are safe to call without a GPU
    lib.ssa_strerror.restype = ctypes.c_char_p
    lib.ssa_version.restype = ctypes.c_char_p
    assert lib.ssa_strerror(-3) == b"rank out of range"
    assert b"sm_103a" in lib.ssa_version()


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    """The Python face has no CPU fallback: a missing library is an error."""
    from paper_1309_5050_gb300 import _lib, build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError):
        _lib.load(build_if_missing=False)
