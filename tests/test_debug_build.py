"""The PLQ_DEBUG build (device bounds guards) compiles and exports every entry point of
the header, like the normal build (no GPU needed)."""
import ctypes

from paper_1405_0700_gb300 import _build

from test_abi import declared


def test_debug_library_builds_and_exports_the_boundary():
    path = _build.build(debug=True)
    assert path.endswith("libplq_debug.so")
    lib = ctypes.CDLL(path)
    for name in declared():
        assert hasattr(lib, name), name
