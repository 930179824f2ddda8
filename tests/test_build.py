"""The build (CPU): the bounds-checked variant of the library compiles for
sm_103a and exports every entry point the header declares."""
import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_checked_variant_builds_and_exports_the_entry_points():
    from paper_1712_03439_gb300 import _lib, build
    path = build.build_checked()
    assert os.path.exists(path) and path != build.LIB_PATH
    lib = ctypes.CDLL(path)
    for name in _lib.EXPORTED:
        assert hasattr(lib, name), name
