"""The C-ABI library loads and exports every function include/sj.h declares
(host-only checks: no kernel is launched)."""
import ctypes
import os
import re

import paper_1902_08318_gb300 as sj
from tests.conftest import ROOT


def _declared():
    text = open(os.path.join(ROOT, "include", "sj.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sj_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sj_parse", "sj_parse_batch", "sj_parser_create", "sj_parser_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    sj.build()
    lib = sj.load()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(sj.EXPORTED) == set(_declared())


def test_host_only_calls():
    lib = sj.load()
    assert lib.sj_error_name(0) == b"SUCCESS"
    assert lib.sj_error_name(10) == b"UTF8_ERROR"
    assert lib.sj_error_name(99) == b"UNKNOWN"
    assert b"sm_103a" in lib.sj_version()
    for code, name in enumerate(sj.ERROR_NAMES):
        assert lib.sj_error_name(code).decode() == name


def test_invalid_arguments_rejected_without_a_gpu():
    lib = sj.load()
    # NULL parser / NULL outputs are rejected before any CUDA call
    assert lib.sj_parse(None, None, 0, None, None) == sj.INVALID_ARG
    assert lib.sj_parse_batch(None, None, None, 0, None, None, None, None, None) == sj.INVALID_ARG
    assert lib.sj_parser_create(None, 1, 1, 0) == sj.INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.sj_parser_create(ctypes.byref(h), 1, 1, 5000) == sj.INVALID_ARG  # depth > 4096
    assert not h.value


def test_no_cpu_fallback_in_the_product_package():
    src = open(os.path.join(ROOT, "paper_1902_08318_gb300", "__init__.py")).read()
    assert "import oracle" not in src and "from oracle" not in src


def test_server_calls_reject_invalid_arguments_without_a_gpu():
    lib = sj.load()
    assert lib.sj_server_create(None, None) == sj.INVALID_ARG
    assert lib.sj_server_poll(None, None, 0) == -sj.INVALID_ARG
    assert lib.sj_server_release(None, 0) == sj.INVALID_ARG
    assert lib.sj_server_submit(None, None, 0, None) == sj.INVALID_ARG
    assert lib.sj_server_slots(None) == 0
    assert lib.sj_parse_query(None) == -sj.INVALID_ARG
    assert lib.sj_parse_batch_async(None, None, None, 0, None) == sj.INVALID_ARG
