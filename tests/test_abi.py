"""The C-ABI library builds, loads without a GPU and exports every entry point of include/*.h."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(ntvs_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def so_path():
    from paper_1803_01112_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = _header_functions()
    for required in ("ntvs_create", "ntvs_destroy", "ntvs_load_system", "ntvs_set_params", "ntvs_set_image",
                     "ntvs_get_image", "ntvs_run", "ntvs_get_tv", "ntvs_get_stats", "ntvs_get_state",
                     "ntvs_set_state"):
        assert required in names


def test_library_exports_every_declared_symbol(so_path):
    out = subprocess.run(["nm", "-D", "--defined-only", so_path], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = _header_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    lib = ctypes.CDLL(so_path)
    for name in _header_functions():
        assert hasattr(lib, name)


def test_binding_covers_the_header(so_path):
    from paper_1803_01112_gb300 import _ffi
    import paper_1803_01112_gb300 as pkg
    assert set(_ffi.SIGNATURES) == _header_functions()
    for name in _header_functions():   # the Python binding carries the C names
        assert callable(getattr(pkg, name)), name


def test_version_and_error_text_without_gpu(so_path):
    import paper_1803_01112_gb300 as pkg
    assert "sm_103a" in pkg.ntvs_version()
    assert isinstance(pkg.ntvs_last_error(), str)


def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    from paper_1803_01112_gb300 import _ffi
    monkeypatch.setattr(_ffi, "_lib", None)
    monkeypatch.setattr(_ffi, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _ffi.lib()


def test_product_does_not_import_the_oracle():
    for path in glob.glob(os.path.join(ROOT, "paper_1803_01112_gb300", "**", "*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            src = open(path).read()
            assert "import oracle" not in src and "from oracle" not in src, path
            assert "ntvs_oracle" not in src and "orc_" not in src, path
