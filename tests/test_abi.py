"""The C ABI library loads and exports every entry point that include/qtv.h
declares; host-side argument validation rejects bad calls before any launch.
No GPU is needed: nothing here launches a kernel."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1911_12070_gb300 as qtv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qtv.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qtv_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    qtv.build()
    return qtv.lib()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("qtv_identify", "qtv_localize", "qtv_emit_samples", "qtv_create", "qtv_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", qtv.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(qtv_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_no_internal_symbols_leak(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", qtv.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    text_syms = re.findall(r"\bT\s+(\S+)", out)
    assert all(s.startswith("qtv_") for s in text_syms), [s for s in text_syms
                                                          if not s.startswith("qtv_")][:5]


def test_version(lib):
    assert lib.qtv_version() >> 16 == 1


def test_null_handle_is_rejected_on_the_host(lib):
    g = qtv.Grid.of((8, 8, 8))
    rc = lib.qtv_identify(None, ctypes.byref(g), None, None, None, 0, None, None, None)
    assert rc == qtv.ERR_ARG
    assert b"handle" in lib.qtv_last_error_string()
    rc = lib.qtv_localize(None, ctypes.byref(g), None, None, None, 0, None, 0, 1e-3, None,
                          None, None, None)
    assert rc == qtv.ERR_ARG
    assert lib.qtv_destroy(None) == 0


def test_sample_layout_is_32_bytes():
    assert ctypes.sizeof(qtv.Sample) == 32
    assert qtv.SAMPLE_DTYPE.itemsize == 32
    assert qtv.Sample.face_id.offset == 16 and qtv.Sample.winding.offset == 24


def declared_prototypes():
    """{name: parameter count} of every QTV_API function in the header."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"QTV_API\s+[^;(]*?\b(qtv_\w+)\s*\(([^)]*)\)\s*;", src, flags=re.S):
        params = " ".join(m.group(2).split())
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header(lib):
    # every function the binding declares argtypes for takes as many
    # arguments as its prototype (a mismatch would pass garbage through ctypes)
    protos = declared_prototypes()
    assert len(protos) == len(declared_functions())
    checked = 0
    for name, n in protos.items():
        argtypes = getattr(lib, name).argtypes
        if argtypes is None:
            continue
        assert len(argtypes) == n, (name, len(argtypes), n)
        checked += 1
    assert checked >= 30


def _header_kinds():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"QTV_API\s+[^;(]*?\b(qtv_\w+)\s*\(([^)]*)\)\s*;", src, flags=re.S):
        params = " ".join(m.group(2).split())
        if params in ("", "void"):
            out[m.group(1)] = []
            continue
        kinds = []
        for p in params.split(","):
            p = p.strip()
            if "*" in p or p.startswith("qtv_handle"):
                kinds.append("ptr")
            elif re.match(r"(const\s+)?u?int64_t\b", p):
                kinds.append("i64")
            elif re.match(r"(const\s+)?(int|u?int32_t)\b", p):
                kinds.append("i32")
            elif re.match(r"(const\s+)?float\b", p):
                kinds.append("f32")
            elif re.match(r"(const\s+)?double\b", p):
                kinds.append("f64")
            else:
                kinds.append("?" + p)
        out[m.group(1)] = kinds
    return out


def _ctypes_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "contents") or \
            getattr(t, "_type_", None) is not None and isinstance(getattr(t, "_type_"), type):
        return "ptr"
    if t in (ctypes.c_uint64, ctypes.c_int64):
        return "i64"
    if t in (ctypes.c_int32, ctypes.c_uint32):
        return "i32"
    if t is ctypes.c_float:
        return "f32"
    if t is ctypes.c_double:
        return "f64"
    return "?" + repr(t)


def test_binding_argument_kinds_match_the_header(lib):
    # pointer, 64-bit, 32-bit and floating arguments in the same places
    for name, kinds in _header_kinds().items():
        argtypes = getattr(lib, name).argtypes
        if argtypes is None:
            continue
        got = [_ctypes_kind(t) for t in argtypes]
        assert got == kinds, (name, got, kinds)


def test_scan_hold_injection_is_validated_on_the_host(lib):
    assert lib.qtv_inject_scan_hold(None, 0, 0) == qtv.ERR_ARG
