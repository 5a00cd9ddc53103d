"""The C-ABI library builds, loads on a machine without a GPU and exports
every function include/fdtdmor.h declares (no compute call is made)."""
import os

from paper_1406_7042_gb300 import fdtdmor as F


def test_library_exports_every_declared_symbol():
    if not os.path.exists(F.LIB_PATH):
        from paper_1406_7042_gb300 import build
        build.build()
    L = F.lib(install_allocator=False)
    names = F.declared_symbols()
    assert "fdtd_step" in names and "fdtd_grid_create" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_no_fallback_when_library_missing(tmp_path, monkeypatch):
    monkeypatch.setattr(F, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(F, "_lib", None)
    try:
        F.lib()
    except F.FdtdError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("loading a missing library must raise")


def test_checked_build_exports_every_declared_symbol():
    """The -DFDTD_CHECKED variant (synchronised launches, no graphs, index
    checks) builds on its own objects and exports the same C ABI."""
    import ctypes
    from paper_1406_7042_gb300 import build
    path = build.build(checked=True)
    assert path.endswith("libfdtdmor_checked.so") and path != F.LIB_PATH
    L = ctypes.CDLL(path)
    missing = [n for n in F.declared_symbols() if not hasattr(L, n)]
    assert not missing, missing
