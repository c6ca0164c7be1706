"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every entry point include/fsib.h declares."""
import os
import re

from paper_2302_08694_gb300 import build as fbuild
from paper_2302_08694_gb300 import fsib

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fsib.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fsib_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("fsib_create", "fsib_spread", "fsib_fluid_step", "fsib_interp", "fsib_step"):
        assert required in names


def test_library_exports_every_declared_symbol():
    fbuild.build()
    lib = fsib.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) <= set(fsib.EXPORTS)


def test_version_string():
    fbuild.build()
    assert re.match(r"^\d+\.\d+\.\d+$", fsib.version())


def test_create_calls_reject_bad_arguments_before_any_device_work():
    """fsib_create, fsib_batch_create and fsib_spread_static validate their scalar arguments
    before the first CUDA call, so each rejection below returns FSIB_EINVAL (-1) with a
    message, on a host without a GPU as on one with."""
    import ctypes

    fbuild.build()
    lib = fsib.load()
    h = ctypes.c_void_p()
    bad_create = [
        (16, 3, 0, 1.0, 1.0, 1e-3, 1e-6, "M must be"),          # no points
        (16, 3, -5, 1.0, 1.0, 1e-3, 1e-6, "M must be"),
        (7, 3, 10, 1.0, 1.0, 1e-3, 1e-6, "N must be"),          # odd N
        (2, 2, 10, 1.0, 1.0, 1e-3, 1e-6, "N must be"),          # below the smallest grid
        (1026, 2, 10, 1.0, 1.0, 1e-3, 1e-6, "N must be"),       # above the largest grid
        (16, 1, 10, 1.0, 1.0, 1e-3, 1e-6, "d must be"),
        (16, 4, 10, 1.0, 1.0, 1e-3, 1e-6, "d must be"),
        (16, 3, 10, 0.0, 1.0, 1e-3, 1e-6, "mu and dt"),         # viscosity must be positive
        (16, 3, 10, 1.0, 1.0, -1e-3, 1e-6, "mu and dt"),
        (16, 3, 10, 1.0, float("nan"), 1e-3, 1e-6, "mu and dt"),
        (16, 3, 10, 1.0, 1.0, 1e-3, 0.0, "tol must be"),        # tolerance out of range
        (16, 3, 10, 1.0, 1.0, 1e-3, 0.5, "tol must be"),
    ]
    for N, d, M, mu, rho, dt, tol, msg in bad_create:
        rc = lib.fsib_create(ctypes.byref(h), N, d, M, mu, rho, dt, tol)
        assert rc == -1, (N, d, M, mu, rho, dt, tol)
        assert h.value is None
        assert msg in lib.fsib_last_error(None).decode()
    assert lib.fsib_create(None, 16, 3, 10, 1.0, 1.0, 1e-3, 1e-6) == -1

    ints = (ctypes.c_int * 1)(16)
    dbls = (ctypes.c_double * 1)(1.0)
    b = ctypes.c_void_p()
    cast = ctypes.cast
    vp = ctypes.c_void_p
    args = [cast(ints, vp), cast(ints, vp), cast(ints, vp)] + [cast(dbls, vp)] * 4
    assert lib.fsib_batch_create(ctypes.byref(b), 0, *args, 0) == -1        # empty batch
    assert lib.fsib_batch_create(ctypes.byref(b), 1, *args, 7) == -1        # unknown precision
    assert lib.fsib_batch_create(ctypes.byref(b), 1, None, *args[1:], 0) == -1
    assert "bad batch arguments" in lib.fsib_last_error(None).decode()

    for N, d, M, tol, prec in [(16, 3, 0, 1e-6, 0), (15, 3, 8, 1e-6, 0), (16, 5, 8, 1e-6, 0),
                               (16, 3, 8, 1.0, 0), (16, 3, 8, 1e-6, 9)]:
        assert lib.fsib_spread_static(N, d, M, tol, prec, None, None, None, None, None) == -1
        assert "bad N, d, M, tol or precision" in lib.fsib_static_last_error().decode()
    assert lib.fsib_spread_static(16, 3, 8, 1e-6, 0, None, None, None, None, None) == -1
    assert "NULL array" in lib.fsib_static_last_error().decode()


def test_create_without_a_device_fails_cleanly():
    """With valid arguments and no GPU, fsib_create returns FSIB_ECUDA (-3) and a message, and
    leaves the handle NULL (what it had created is released); no CPU fallback exists."""
    import ctypes

    import torch
    if torch.cuda.is_available():
        import pytest
        pytest.skip("a GPU is present")
    fbuild.build()
    lib = fsib.load()
    h = ctypes.c_void_p()
    assert lib.fsib_create(ctypes.byref(h), 16, 3, 10, 1.0, 1.0, 1e-3, 1e-6) == -3
    assert h.value is None
    assert "no device" in lib.fsib_last_error(None).decode()
