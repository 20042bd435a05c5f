"""The C ABI library loads and exports every entry point its header declares (no GPU)."""
import ctypes
import os
import re

import pytest

from paper_1405_0700_gb300 import _build
from paper_1405_0700_gb300 import plq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^PLQ_API\s+[\w\s\*]+?\b(plq_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return plq.lib()


def test_header_declares_the_boundary():
    names = declared()
    for n in ["plq_init", "plq_gauge_upload", "plq_hopping_eo", "plq_wilson_apply", "plq_cg_solve",
              "plq_bicgstab_solve"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared():
        assert hasattr(lib, n), n
        assert n in plq.SIGNATURES, f"binding lacks {n}"


def test_binding_covers_only_declared(lib):
    assert set(plq.SIGNATURES) <= set(declared())


def test_argument_errors_without_gpu(lib):
    # validation happens before any CUDA call
    assert lib.plq_init(None, None, -1, 0) == plq.PLQ_ERR_ARG
    h = ctypes.c_void_p()
    bad = (ctypes.c_int * 4)(8, 8, 7, 8)
    assert lib.plq_init(ctypes.byref(h), ctypes.cast(bad, ctypes.c_void_p), -1, 0) == plq.PLQ_ERR_ARG
    assert "even" in plq.last_error()
    ok = (ctypes.c_int * 4)(8, 8, 8, 8)
    assert lib.plq_init(ctypes.byref(h), ctypes.cast(ok, ctypes.c_void_p), 0, 0) == plq.PLQ_ERR_ARG
    assert lib.plq_hopping_eo(None, 0, None, None, 1, 1, None) == plq.PLQ_ERR_ARG
    assert lib.plq_field_bytes(None, 1, 1) == 0
    assert lib.plq_cg_solve(None, None, None, 0.1, None, None, None) == plq.PLQ_ERR_ARG
    assert lib.plq_finalize(None) == plq.PLQ_OK
    assert lib.plq_version() >= 10000
