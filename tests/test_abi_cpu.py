"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/qcd.h declares.  No compute call is made (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "qcd.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(qcd_[a-z0-9_]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def lib():
    from paper_1605_00564_gb300 import build, qcd
    build.build()
    return qcd.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("qcd_create", "qcd_load_gauge", "qcd_apply_dirac", "qcd_apply_sap", "qcd_solve",
              "qcd_nucleon_2pt", "qcd_ama_nucleon_2pt", "qcd_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1605_00564_gb300 import qcd
    names = _declared()
    assert set(names) == set(qcd.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_host_only_calls(lib):
    from paper_1605_00564_gb300 import qcd
    p = qcd.SolverParams()
    lib.qcd_default_params(ctypes.byref(p))
    assert list(p.block) == [4, 4, 4, 4] and p.ncy == 5 and p.nmr == 4 and p.nkv == 16
    # the binding's struct has the C struct's size: the library writes the last
    # field and nothing beyond the binding's size
    sz = ctypes.sizeof(qcd.SolverParams)
    buf = (ctypes.c_ubyte * (sz + 64))(*([0xAB] * (sz + 64)))
    q = qcd.SolverParams.from_buffer(buf)
    lib.qcd_default_params(ctypes.byref(q))
    assert q.graphs == 1 and q.basis_half == 0 and q.dfl_little_iters == 16
    assert all(buf[i] == 0xAB for i in range(sz, sz + 64))
    assert lib.qcd_status_string(0) == b"ok"
    assert lib.qcd_status_string(4) == b"solver did not converge"
    # argument errors are reported before any device work
    ctx = ctypes.c_void_p()
    assert lib.qcd_create(ctypes.byref(ctx), (ctypes.c_int * 4)(16, 1, 8, 8), None) == 1
    assert b"extent" in lib.qcd_last_error()


def test_library_is_sm103a():
    from paper_1605_00564_gb300 import build
    assert "compute_103a,code=sm_103a" in build.ARCH


def _c_struct_fields(header, name):
    """Field names of `typedef struct { ... } name;` in declaration order."""
    import re
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", header, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            m = re.search(r"(\w+)\s*(\[[^\]]*\])?\s*$", part.strip())
            fields.append(m.group(1))
    return fields


def test_binding_structs_match_header():
    """The ctypes structures list the C structures' fields in the same order."""
    import os
    from paper_1605_00564_gb300 import qcd
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    header = open(os.path.join(root, "include", "qcd.h")).read()
    for cname, py in (("qcd_solver_params", qcd.SolverParams), ("qcd_rhs_stats", qcd.RhsStats),
                      ("qcd_kernel_time", qcd.KernelTime)):
        assert _c_struct_fields(header, cname) == [f[0] for f in py._fields_], cname


def test_argument_errors_before_device_work(lib):
    """Entry points reject bad arguments before touching the device (runs without a GPU;
    the pointers below are never dereferenced on these paths)."""
    I4 = ctypes.c_int * 4
    buf = (ctypes.c_double * 8)()
    cases = [
        ((I4(8, 8, 8, 8), -1, None, I4(0, 0, 0, 0), buf, 0), b"null"),
        ((I4(8, 1, 8, 8), -1, buf, I4(0, 0, 0, 0), buf, 0), b"extent"),
        ((I4(8, 8, 8, 8), -1, buf, I4(0, 9, 0, 0), buf, 0), b"outside"),
        ((I4(8, 8, 8, 8), 0, buf, I4(0, 0, 0, 0), buf, 0), b"time_bc"),
        ((I4(8, 8, 8, 8), -1, buf, I4(0, 0, 0, 0), buf, 7), b"precision"),
        ((I4(512, 256, 256, 256), -1, buf, I4(0, 0, 0, 0), buf, 0), b"too large"),
    ]
    for args, msg in cases:
        assert lib.qcd_nucleon_2pt_noalloc(*args, None) == 1, msg
        assert msg in lib.qcd_last_error(), (msg, lib.qcd_last_error())
    assert lib.qcd_solve_multi(None, 1, None, None, None, None, None) == 1
    assert b"null" in lib.qcd_last_error()
    for code in range(9):
        assert lib.qcd_status_string(code)
