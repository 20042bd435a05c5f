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


def header_text():
    return "\n".join(open(os.path.join(ROOT, "include", h)).read()
                     for h in sorted(os.listdir(os.path.join(ROOT, "include"))) if h.endswith(".h"))


def strip_comments(txt):
    return re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)


C_TYPES = {"int": ctypes.c_int, "double": ctypes.c_double}


def header_structs():
    """{typedef name: [(field, ctype), ...]} for the plain structs of the header."""
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(plq_\w+)\s*;", strip_comments(header_text()), re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            typ, field = decl.rsplit(None, 1)
            fields.append((field, C_TYPES[typ.strip()]))
        out[name] = fields
    return out


@pytest.mark.parametrize("cname,cls", [("plq_solver_params", plq.SolverParams), ("plq_solve_info", plq.SolveInfo),
                                       ("plq_batch_info", plq.BatchInfo), ("plq_tune_result", plq.TuneResult)])
def test_binding_structs_match_header(cname, cls):
    """Field names, types and order of every ctypes struct equal the header's."""
    assert header_structs()[cname] == list(cls._fields_)


def test_binding_argument_counts_match_header():
    """Each declared function takes as many arguments as the binding passes."""
    txt = strip_comments(header_text())
    decls = re.findall(r"PLQ_API\s+[\w\s\*]+?\b(plq_\w+)\s*\(([^)]*)\)\s*;", txt)
    assert decls
    for name, args in decls:
        args = args.strip()
        n = 0 if args in ("", "void") else args.count(",") + 1
        assert len(plq.SIGNATURES[name][1]) == n, name


def test_host_slab_schedule(lib):
    """The time slabs of the host pipeline: they tile [0, T), each holds at least one
    time slice (so slab k's t +- 1 neighbours lie in slabs k - 1 .. k + 1), none holds
    more than max(1, T/8), the first and last hold one slice, and there are at most 64."""
    b = (ctypes.c_int * 65)()
    for T in range(2, 4098, 2):
        K = lib.plq_host_slabs(T, b)
        bounds = list(b[:K + 1])
        sizes = [bounds[k + 1] - bounds[k] for k in range(K)]
        assert 1 <= K <= 64 and bounds[0] == 0 and bounds[-1] == T, T
        assert min(sizes) >= 1 and max(sizes) <= max(1, T // 8), (T, sizes)
        assert sizes[0] == 1 and sizes[-1] == 1, (T, sizes)
    K = lib.plq_host_slabs(64, b)
    assert [b[k + 1] - b[k] for k in range(K)] == [1, 1, 2, 4, 8, 8, 8, 8, 8, 8, 4, 2, 1, 1]
    assert lib.plq_host_slabs(7, b) == 0 and lib.plq_host_slabs(0, b) == 0 and lib.plq_host_slabs(8, None) == 0


def test_every_declaration_cites_its_definition():
    """Each exported call's comment names the passage of the paper that defines the
    operation (a section or equation) or says that the paper is silent on it; the
    allocation-free Schur operator instead says that the paper has no counterpart."""
    txt = header_text()
    for m in re.finditer(r"PLQ_API\s+[\w\s\*]+?\b(plq_\w+)\s*\(", txt):
        name = m.group(1)
        before = txt[:m.start()]
        end = before.rfind("*/")
        start = before.rfind("/*", 0, end)
        assert end > 0 and start >= 0, name
        comment = before[start:end]
        if name == "plq_schur_apply_noalloc":
            assert "No counterpart in the paper" in comment
            continue
        assert re.search(r"Sec\. \d|Eq\. \(\d\)|[Pp]aper silent", comment), name
