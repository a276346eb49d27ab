"""CPU oracle of the two-stage validating JSON parse (Langdale & Lemire).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product path (``paper_1902_08318_gb300``) never does; the two
share no code.  The C source is ``oracle/oracle.c``; this file only compiles it
with gcc and marshals arguments through ctypes.

Parity status per function (pins live in tests/test_oracle_*.py):
  utf8_valid   pinned: Table "tab:unicode" vs Python's strict utf-8 codec,
               exhaustive over 1-, 2- and 3-byte sequences; 4-byte sequences
               with every 4-byte lead, every second and third byte and the
               fourth byte's boundaries, and every lead with class
               representatives for the last two bytes.
  classify     pinned: the nibble tables printed in Sec. 3.1.2, all 256 bytes.
  stage1       pinned: the 64-byte worked example of Figs. 2-4 (every printed
               mask row) and brute-force equivalence with a literal transcription
               of the mask sequences on all short inputs over a small alphabet.
  parse        pinned: Fig. 1 -> Fig. "jsontape" (all 38 words), accept/reject
               vs Python's json on every document of <= 5 bytes over a reduced
               alphabet, numbers vs Python's float/int, invariants.
               Error categories: single defects injected into valid
               documents and ordered pairs of defects (categories fixed by
               construction); several defects at one token stay "parity
               unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SUCCESS, CAPACITY, MEMALLOC, TAPE_ERROR, DEPTH_ERROR, STRING_ERROR = 0, 1, 2, 3, 4, 5
T_ATOM_ERROR, F_ATOM_ERROR, N_ATOM_ERROR, NUMBER_ERROR, UTF8_ERROR = 6, 7, 8, 9, 10
UNCLOSED_STRING, UNESCAPED_CHARS, EMPTY, INVALID_ARG, INTERNAL = 11, 12, 13, 14, 15


class _Result(ctypes.Structure):
    _fields_ = [("error", ctypes.c_int32), ("pad_", ctypes.c_uint32),
                ("n_indices", ctypes.c_uint64), ("tape_words", ctypes.c_uint64),
                ("string_bytes", ctypes.c_uint64), ("n_tokens", ctypes.c_uint64)]


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, no SIMD flags)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    with _lock:
        if (not force and os.path.exists(_SO)
                and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.sjo_utf8_valid.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
        lib.sjo_utf8_valid_many.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_void_p]
        lib.sjo_classify.argtypes = [ctypes.c_uint8]
        lib.sjo_stage1.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                   ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
                                   ctypes.POINTER(ctypes.c_int)]
        lib.sjo_stage1_many.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_void_p, ctypes.c_void_p]
        lib.sjo_parse.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                  ctypes.c_void_p, ctypes.c_uint64,
                                  ctypes.c_void_p, ctypes.c_uint64,
                                  ctypes.c_void_p, ctypes.c_uint64,
                                  ctypes.c_void_p, ctypes.c_uint64,
                                  ctypes.POINTER(_Result)]
        lib.sjo_parse_many_errors.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                              ctypes.c_uint32, ctypes.c_void_p]
        del u8p
        _lib = lib
    return _lib


def _buf(data) -> np.ndarray:
    if isinstance(data, np.ndarray):
        return np.ascontiguousarray(data, dtype=np.uint8)
    return np.frombuffer(bytes(data), dtype=np.uint8)


def utf8_valid(data) -> bool:
    a = _buf(data)
    return bool(_load().sjo_utf8_valid(a.ctypes.data, a.size))


def utf8_valid_many(records: np.ndarray) -> np.ndarray:
    """records: (n, w) uint8 array; returns (n,) bool validity of each row."""
    r = np.ascontiguousarray(records, dtype=np.uint8)
    n, w = r.shape
    ok = np.zeros(n, dtype=np.uint8)
    _load().sjo_utf8_valid_many(r.ctypes.data, n, w, ok.ctypes.data)
    return ok.astype(bool)


def classify(c: int) -> int:
    return int(_load().sjo_classify(c))


def stage1(data):
    """Returns (indices: uint32 array, unclosed: bool)."""
    a = _buf(data)
    idx = np.zeros(max(a.size, 1), dtype=np.uint32)
    n = ctypes.c_uint64(0)
    uc = ctypes.c_int(0)
    _load().sjo_stage1(a.ctypes.data, a.size, idx.ctypes.data, idx.size,
                       ctypes.byref(n), ctypes.byref(uc))
    return idx[: n.value].copy(), bool(uc.value)


def stage1_many(records: np.ndarray):
    """records: (n, w) uint8; returns ((n, w) bool index mask, (n,) bool unclosed)."""
    r = np.ascontiguousarray(records, dtype=np.uint8)
    n, w = r.shape
    mask = np.zeros((n, w), dtype=np.uint8)
    uc = np.zeros(n, dtype=np.uint8)
    _load().sjo_stage1_many(r.ctypes.data, n, w, mask.ctypes.data, uc.ctypes.data)
    return mask.astype(bool), uc.astype(bool)


def parse(data, max_depth: int = 0, want_tokens: bool = False) -> dict:
    """Full parse.  Returns a dict with error, indices, tape, strings (and tokens)."""
    a = _buf(data)
    n = a.size
    idx = np.zeros(n + 1, dtype=np.uint32)
    tape = np.zeros(n + 4, dtype=np.uint64)
    sb = np.zeros(3 * n + 8, dtype=np.uint8)
    tok = np.zeros(n + 1, dtype=np.uint32) if want_tokens else None
    res = _Result()
    _load().sjo_parse(a.ctypes.data, n, max_depth, idx.ctypes.data, idx.size,
                      tape.ctypes.data, tape.size, sb.ctypes.data, sb.size,
                      tok.ctypes.data if tok is not None else None,
                      tok.size if tok is not None else 0, ctypes.byref(res))
    out = {
        "error": int(res.error),
        "n_indices": int(res.n_indices),
        "indices": idx[: res.n_indices].copy(),
        "tape": tape[: res.tape_words].copy(),
        "strings": sb[: res.string_bytes].copy(),
    }
    if tok is not None:
        out["tokens"] = tok[: min(res.n_tokens, tok.size)].copy()
    return out


def parse_many_errors(buf: np.ndarray, offsets: np.ndarray, max_depth: int = 0) -> np.ndarray:
    """Error code of each document buf[offsets[i]:offsets[i+1]]."""
    b = _buf(buf)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = off.size - 1
    err = np.zeros(max(n, 0), dtype=np.int32)
    _load().sjo_parse_many_errors(b.ctypes.data, off.ctypes.data, n, max_depth, err.ctypes.data)
    return err


def distinct_path_values(doc: bytes, path) -> set:
    """The tape query of Sec. 4.5 / Table "tab:userid" written out: every
    object of the document (at any depth) whose keys path[0], ..., path[-2]
    name nested objects and whose path[-1] names an integer contributes that
    integer; returns the set of them.  A plain recursive walk over Python's
    json decoder (a library routine standing for the parse)."""
    import json
    out = set()

    def at_path(o):
        for k in path[:-1]:
            if not isinstance(o, dict) or not isinstance(o.get(k), dict):
                return None
            o = o[k]
        v = o.get(path[-1]) if isinstance(o, dict) else None
        return v if isinstance(v, int) and not isinstance(v, bool) else None

    def walk(x):
        if isinstance(x, dict):
            v = at_path(x)
            if v is not None:
                out.add(v)
            for y in x.values():
                walk(y)
        elif isinstance(x, list):
            for y in x:
                walk(y)

    walk(json.loads(doc))
    return out
