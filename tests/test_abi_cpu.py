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
