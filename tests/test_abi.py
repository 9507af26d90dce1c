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


def test_noalloc_device_check_host_side():
    """The allocation-free branching entry point refuses a call made with a device current other
    than the one its system was created on (its tables and the per-device scratch address would
    belong to different GPUs); the check runs on the host before any launch."""
    from paper_1807_02431_gb300 import binding, build

    lib = ctypes.CDLL(build.build())
    f = lib.grp_noalloc_check_device
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_int32, ctypes.c_int32]
    lib.grp_last_error.restype = ctypes.c_char_p
    assert f(0, 0) == binding.GRP_OK and f(3, 3) == binding.GRP_OK
    assert f(1, 0) == binding.GRP_EINVAL
    msg = lib.grp_last_error().decode()
    assert "device is 0" in msg and "device 1" in msg
    assert f(0, 5) == binding.GRP_EINVAL
