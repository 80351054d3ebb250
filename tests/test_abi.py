"""The C-ABI library builds, loads and exports every entry point that
include/bp.h declares; argument errors are reported without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1010_0012_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bp_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["bp_create", "bp_set_unary", "bp_set_potential", "bp_reset_messages", "bp_iterate",
                     "bp_beliefs", "bp_backward", "bp_sync", "bp_last_error", "bp_destroy",
                     "bp_iterate_dense"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_errors_without_gpu(lib):
    lib.bp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                              ctypes.POINTER(ctypes.c_void_p)]
    lib.bp_last_error.restype = ctypes.c_char_p
    lib.bp_last_error.argtypes = [ctypes.c_void_p]
    out = ctypes.c_void_p(123)
    assert lib.bp_create(0, 4, 8, 0, None, ctypes.byref(out)) == 1      # BP_ERR_ARG
    assert out.value is None
    assert b"W and H" in lib.bp_last_error(None)
    assert lib.bp_create(4, 4, 1, 0, None, ctypes.byref(out)) == 1      # M < 2
    assert lib.bp_create(4, 4, 2000, 0, None, ctypes.byref(out)) == 1   # M > 1024
    assert lib.bp_create(4, 4, 8, 7, None, ctypes.byref(out)) == 1      # dtype
    assert lib.bp_create(4, 4, 8, 0, None, None) == 1                   # out NULL
    assert lib.bp_create(1 << 16, 1 << 15, 8, 0, None, ctypes.byref(out)) == 1   # too large
    for fn in ("bp_set_unary", "bp_set_messages", "bp_get_messages"):
        getattr(lib, fn).argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        assert getattr(lib, fn)(None, None) == 1
    lib.bp_iterate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    assert lib.bp_iterate(None, 1, 0, 0) == 1
    lib.bp_destroy.argtypes = [ctypes.c_void_p]
    lib.bp_destroy(None)
    assert lib.bp_version() > 0


HANDLE_TYPES = {"bp_handle": "bp_last_error", "bp_batch": "bp_batch_last_error",
                "bp_factor_graph": "bp_fg_last_error"}


def _ctype(param):
    """ctypes type and a zero value for one C parameter declaration."""
    decl = param.strip()
    if "*" in decl or decl.split()[0] in HANDLE_TYPES:
        return ctypes.c_void_p, None
    kind = decl.rsplit(" ", 1)[0]
    if "double" in kind:
        return ctypes.c_double, 0.0
    if "float" in kind:
        return ctypes.c_float, 0.0
    if "long long" in kind or "size_t" in kind:
        return ctypes.c_longlong, 0
    return ctypes.c_int, 0


def test_every_handle_call_rejects_a_null_handle_without_a_gpu(lib):
    """Every status-returning entry point that takes a handle first returns
    BP_ERR_ARG for a NULL handle, before any other argument or the device is
    touched, and records a message naming itself where the header says
    (bp_last_error / bp_batch_last_error / bp_fg_last_error of NULL)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    decls = re.findall(r"\bbp_status\s+(bp_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", text)
    checked = 0
    for name, params in decls:
        ps = [p for p in params.split(",") if p.strip()]
        if not ps or ps[0].split()[0] not in HANDLE_TYPES:
            continue
        err = getattr(lib, HANDLE_TYPES[ps[0].split()[0]])
        err.restype = ctypes.c_char_p
        err.argtypes = [ctypes.c_void_p]
        types, vals = zip(*[_ctype(p) for p in ps])
        fn = getattr(lib, name)
        fn.argtypes = list(types)
        fn.restype = ctypes.c_int
        assert fn(*vals) == 1, name
        assert name.encode() in err(None), (name, err(None))
        checked += 1
    assert checked >= 35


def test_binding_names_match_the_abi():
    """The Python binding exposes one function per C entry point, same name."""
    import ast
    src = open(os.path.join(ROOT, "paper_1010_0012_gb300", "bp.py")).read()
    defined = {n.name for n in ast.parse(src).body if isinstance(n, ast.FunctionDef)}
    missing = [n for n in declared_functions() if n not in defined]
    assert not missing, missing


def test_no_alloc_entry_point_checks_pointers_before_touching_a_device(lib):
    """bp_iterate_dense_tc_noalloc refuses misaligned and overlapping device
    ranges on the host, before any CUDA call, so the addresses here are never
    dereferenced."""
    import numpy as np
    fn = lib.bp_iterate_dense_tc_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    lib.bp_last_error.restype = ctypes.c_char_p
    lib.bp_last_error.argtypes = [ctypes.c_void_p]
    tab = np.ones(7, dtype=np.float32)
    tp = tab.ctypes.data_as(ctypes.c_void_p)
    W, H, M = 8, 8, 64
    nbytes = 4 * W * H * M * 4
    base = 1 << 40
    assert fn(W, H, M, base, base + 2 * nbytes, base + 4 * nbytes + 4, tp, 3, 0.2, None) == 1
    assert b"aligned" in lib.bp_last_error(None)
    assert fn(W, H, M, base + 8, base + 2 * nbytes, base + 4 * nbytes, tp, 3, 0.2, None) == 1
    assert b"aligned" in lib.bp_last_error(None)
    assert fn(W, H, M, base, base + 2 * nbytes, base + 2 * nbytes + nbytes // 2, tp, 3, 0.2, None) == 1
    assert b"overlap" in lib.bp_last_error(None)
    assert fn(W, H, M, base, base + 2 * nbytes, base + 2 * nbytes, tp, 3, 0.2, None) == 1
    assert b"overlap" in lib.bp_last_error(None)
    assert fn(W, H, 32, base, base + 2 * nbytes, base + 4 * nbytes, tp, 3, 0.2, None) == 1
    assert fn(W, H, M, base, base + 2 * nbytes, base + 4 * nbytes, None, 3, 0.2, None) == 1
