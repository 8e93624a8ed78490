"""The C-ABI library builds, loads without a GPU, and exports every entry point
declared in include/*.h (no compute calls here)."""
import ctypes
import glob
import os
import re

from tests.conftest import ROOT


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(fp_[A-Za-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for n in ("fp_sim_create", "fp_set_terrain", "fp_add_pedestrians", "fp_step", "fp_read_state", "fp_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1908_05232_b300 import build
    lib_path = build.build()
    L = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1908_05232_b300._native as nat
    monkeypatch.setattr(nat._build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(nat, "_lib", None)
    try:
        nat.lib()
    except nat.FloodPedError:
        return
    raise AssertionError("expected FloodPedError")
