"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/grp.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(grp_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_entry_point():
    from paper_1807_02431_gb300 import binding, build

    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 16
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding exposes the same names
    assert all(hasattr(binding, n) or "destroy" in n or n == "grp_last_error" for n in names)
    assert set(binding.SIGNATURES) == set(names)


def test_binding_fails_loudly_without_library(tmp_path):
    import pytest

    from paper_1807_02431_gb300 import binding

    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(binding.GrpError):
            binding.load(str(tmp_path / "missing.so"))
    finally:
        binding._lib = saved
