"""Pins of the oracle's full parse (Sec. 3, 3.2) to the paper and to Python.

 - Fig. 1 document -> Fig. "jsontape": every printed word.
 - The paper's named valid/invalid examples (Sec. 3, Sec. 4.1).
 - Accept/reject against Python's json (strict utf-8 first) on every document
   of 1..5 symbols over a 16-symbol alphabet and 6 symbols over 10 symbols.
 - Numbers against Python's float() / int() (both exact / correctly rounded).
 - Tape + string buffer decoded back and compared with json.loads on the
   seeded workloads; structural invariants.
"""
import itertools
import json
import os
import struct
import sys

import numpy as np
import pytest

import gen
import oracle
from tests import tapeutil
from tests.conftest import GOLDEN

M56 = (1 << 56) - 1
sys.setrecursionlimit(20000)  # documents nest to depth 1024


def _tag(w):
    return chr(int(w) >> 56)


def test_fig1_tape_matches_paper():
    doc = open(os.path.join(GOLDEN, "fig1_document.json"), "rb").read()
    r = oracle.parse(doc)
    assert r["error"] == oracle.SUCCESS
    tape, sb = r["tape"], r["strings"]
    assert len(tape) == 38
    seen = set()
    for line in open(os.path.join(GOLDEN, "fig1_tape.txt"), encoding="utf-8"):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.rstrip("\n").split(" ", 2)
        i, tag = int(parts[0]), parts[1]
        seen.add(i)
        w = int(tape[i])
        assert _tag(w) == tag, (i, _tag(w), tag)
        if tag in "r{}[]":
            assert (w & M56) == int(parts[2]), i
        elif tag == '"':
            assert tapeutil.read_string(sb, w & M56).decode() == parts[2], i
        elif tag == "l":
            assert int(tape[i + 1]) == int(parts[2]), i
            seen.add(i + 1)
        else:
            assert (w & M56) == 0
    assert seen == set(range(38))
    # strings are packed in tape order: the first string starts at offset 0
    assert (int(tape[2]) & M56) == 0


@pytest.mark.parametrize("doc,code", [
    (b"012", oracle.NUMBER_ERROR), (b"1E+", oracle.NUMBER_ERROR), (b"[0e+]", oracle.NUMBER_ERROR),
    (b".1", oracle.TAPE_ERROR), (b"1e309", oracle.NUMBER_ERROR), (b"-1e309", oracle.NUMBER_ERROR),
    (b"[12 a]", oracle.TAPE_ERROR), (b'"a\nb"', oracle.UNESCAPED_CHARS),
    (b"9223372036854775807", 0), (b"9223372036854775808", oracle.NUMBER_ERROR),
    (b"-9223372036854775808", 0), (b"-9223372036854775809", oracle.NUMBER_ERROR),
    (b'"[1,2]"', 0), (b"", oracle.EMPTY), (b" \n\t\r", oracle.EMPTY), (b"[", oracle.TAPE_ERROR),
    (b"]", oracle.TAPE_ERROR), (b"[}", oracle.TAPE_ERROR), (b'{"a" 1}', oracle.TAPE_ERROR),
    (b'{"a":1,}', oracle.TAPE_ERROR), (b"[1,]", oracle.TAPE_ERROR), (b"tru", oracle.T_ATOM_ERROR),
    (b"falsey", oracle.F_ATOM_ERROR), (b"nul", oracle.N_ATOM_ERROR), (b'"abc', oracle.UNCLOSED_STRING),
    (b'"\\q"', oracle.STRING_ERROR), (b'"\\uD800"', oracle.STRING_ERROR), (b'"\\uDC00\\uD800"', oracle.STRING_ERROR),
    (b"1 2", oracle.TAPE_ERROR), (b'1"a"', oracle.NUMBER_ERROR), (b"[1\x01]", oracle.NUMBER_ERROR),
    (b"[\x01]", oracle.TAPE_ERROR), (b"\xef\xbb\xbf{}", oracle.TAPE_ERROR), (b'{"a":1,"a":2}', 0),
    (b"-0", 0), (b"-0.0", 0), (b"1e-400", 0), (b'["\x7f"]', 0),
])
def test_named_cases(doc, code):
    assert oracle.parse(doc)["error"] == code


def test_surrogate_pair_escape():
    # Sec. 3.2.2: one 4-byte code point from a \u escape pair
    r = oracle.parse(b'"\\uD834\\uDD1E"')
    assert r["error"] == 0
    assert tapeutil.read_string(r["strings"], int(r["tape"][1]) & M56) == "\U0001D11E".encode()
    assert tapeutil.read_string(r["strings"], 0) == b"\xf0\x9d\x84\x9e"


def test_nul_inside_string_kept():
    r = oracle.parse(b'["a\\u0000b"]')
    assert r["error"] == 0
    assert tapeutil.read_string(r["strings"], 0) == b"a\x00b"


def test_depth_limit():
    assert oracle.parse(b"[[[1]]]", max_depth=3)["error"] == 0
    assert oracle.parse(b"[[[1]]]", max_depth=2)["error"] == oracle.DEPTH_ERROR
    assert oracle.parse(b"[[[[", max_depth=2)["error"] == oracle.DEPTH_ERROR
    deep = b"[" * 4096 + b"]" * 4096
    assert oracle.parse(deep)["error"] == 0
    assert oracle.parse(b"[" + deep + b"]")["error"] == oracle.DEPTH_ERROR


def _python_accepts(b: bytes) -> bool:
    try:
        json.loads(b.decode("utf-8", "strict"))
        return True
    except (UnicodeDecodeError, ValueError, RecursionError):
        return False


def _enumerate(symbols, length):
    for combo in itertools.product(symbols, repeat=length):
        yield b"".join(combo)


SYM16 = [b"[", b"]", b"{", b"}", b":", b",", b'"', b"\\", b"0", b"1", b"-", b".", b"e", b"t", b" ",
         "é".encode()]
SYM10 = [b"[", b"]", b"{", b"}", b":", b",", b'"', b"0", b"1", b" "]


@pytest.mark.parametrize("symbols,length", [(SYM16, n) for n in range(1, 6)] + [(SYM10, 6)])
def test_exhaustive_tiny_documents(symbols, length):
    docs = list(_enumerate(symbols, length))
    lens = np.array([len(d) for d in docs], dtype=np.uint64)
    off = np.zeros(len(docs) + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    errs = oracle.parse_many_errors(np.frombuffer(b"".join(docs), dtype=np.uint8), off)
    for d, e in zip(docs, errs):
        assert (e == 0) == _python_accepts(d), (d, int(e))
        if e == oracle.UTF8_ERROR:
            with pytest.raises(UnicodeDecodeError):
                d.decode("utf-8")


def test_tokens_equal_stage1_indices_on_valid_tiny():
    for length in range(1, 5):
        for d in _enumerate(SYM16, length):
            r = oracle.parse(d, want_tokens=True)
            if r["error"] == 0:
                assert list(r["tokens"]) == list(r["indices"]), d


def _float_bits(s: str) -> int:
    return struct.unpack("<Q", struct.pack("<d", float(s)))[0]


HARD_NUMBERS = [
    "9007199254740993", "9007199254740993.0", "1e23", "8.98846567431158e307",
    "2.2250738585072011e-308", "2.2250738585072012e-308", "4.9e-324", "2.4703282292062327e-324",
    "2.4703282292062328e-324", "1.7976931348623157e308", "1.7976931348623158e308",
    "0.1", "0.30000000000000004", "123456789012345678901234567890e-10",
    "7.2057594037927933e16", "1." + "0" * 30 + "1", "9" * 400 + "e-400",
    "0." + "0" * 320 + "24703282292062327208828439643411068618252990130716238221279284125033775364",
    "1" + "0" * 308, "-0.0", "0e0", "1E-7", "-2.5E+10", "3.0000000000000000000000000000000001",
    "2.5000000000000000000000000000000000000000000000000000000000000001e-323",
]


def test_numbers_match_python_float():
    rng = np.random.Generator(np.random.PCG64(5))
    lexemes = list(HARD_NUMBERS)
    for _ in range(4000):
        sig = int(rng.integers(1, 20))
        digits = "".join(str(int(rng.integers(0, 10))) for _ in range(sig))
        digits = str(int(rng.integers(1, 10))) + digits[1:]
        p = int(rng.integers(1, sig + 1))
        s = digits[:p] + "." + (digits[p:] or "0")
        if rng.random() < 0.5:
            s += "e" + str(int(rng.integers(-330, 310)))
        if rng.random() < 0.5:
            s = "-" + s
        lexemes.append(s)
    for s in lexemes:
        r = oracle.parse(s.encode())
        if not any(ch in s for ch in ".eE"):  # integer form: exact int64 or error
            v = int(s)
            if -(2**63) <= v < 2**63:
                assert r["error"] == 0 and _tag(r["tape"][1]) == "l"
                assert int(r["tape"][2]) == v & ((1 << 64) - 1)
            else:
                assert r["error"] == oracle.NUMBER_ERROR
            continue
        f = float(s)
        if f in (float("inf"), float("-inf")):
            assert r["error"] == oracle.NUMBER_ERROR, s
            continue
        assert r["error"] == 0, s
        assert _tag(r["tape"][1]) == "d"
        assert int(r["tape"][2]) == _float_bits(s), s


def test_integers_match_python_int():
    rng = np.random.Generator(np.random.PCG64(6))
    vals = [0, 1, -1, 2**63 - 1, -(2**63), 10**18, -(10**18)]
    vals += [int(x) for x in rng.integers(-(2**63), 2**63 - 1, 2000, dtype=np.int64)]
    for v in vals:
        r = oracle.parse(str(v).encode())
        assert r["error"] == 0 and _tag(r["tape"][1]) == "l"
        assert int(r["tape"][2]) == v & ((1 << 64) - 1)


def _check_invariants(doc: np.ndarray):
    r = oracle.parse(doc, want_tokens=True)
    assert r["error"] == 0
    tape, sb, idx = r["tape"], r["strings"], r["indices"]
    b = doc.tobytes()
    # token starts of the descent equal the stage-1 index set
    assert np.array_equal(r["tokens"], idx)
    # counts: indices and tape words from token kinds
    first = np.frombuffer(b, dtype=np.uint8)[idx]
    n_str = int((first == ord('"')).sum())
    n_atom = int(np.isin(first, np.frombuffer(b"tfn", dtype=np.uint8)).sum())
    n_num = int(np.isin(first, np.frombuffer(b"-0123456789", dtype=np.uint8)).sum())
    n_cont = int(np.isin(first, np.frombuffer(b"{[", dtype=np.uint8)).sum())
    n_sep = int(np.isin(first, np.frombuffer(b",:", dtype=np.uint8)).sum())
    assert len(idx) == n_str + n_num + n_atom + 2 * n_cont + n_sep
    assert len(tape) == 2 + n_str + n_atom + 2 * n_num + 2 * n_cont
    # depth never negative, zero at the end
    d = np.cumsum(np.where(np.isin(first, np.frombuffer(b"{[", dtype=np.uint8)), 1,
                           np.where(np.isin(first, np.frombuffer(b"}]", dtype=np.uint8)), -1, 0)))
    assert d.min() >= 0 and d[-1] == 0
    # no index strictly inside a string: each string token's closing quote
    # (found by a plain scan that skips the byte after every backslash) lies
    # before the next index, so no index falls between its quotes
    raw = np.frombuffer(b, dtype=np.uint8)
    str_at = np.nonzero(first == ord('"'))[0]
    for k in str_at:
        p = int(idx[k]) + 1
        while raw[p] != ord('"'):
            p += 2 if raw[p] == ord("\\") else 1
        nxt = int(idx[k + 1]) if k + 1 < len(idx) else len(b)
        assert p < nxt, (int(idx[k]), p, nxt)
    # opener/closer payloads are mutually inverse
    tags = (tape >> np.uint64(56)).astype(np.uint8)
    pay = (tape & np.uint64(M56)).astype(np.int64)
    opens = np.nonzero(np.isin(tags, np.frombuffer(b"{[", dtype=np.uint8)))[0]
    # skip value words of numbers (they are raw 64-bit values)
    is_val = np.zeros(len(tape), dtype=bool)
    num = np.nonzero(np.isin(tags, np.frombuffer(b"ld", dtype=np.uint8)))[0]
    # walk once to mark value words properly
    i = 0
    while i < len(tape):
        if chr(tags[i]) in "ld":
            is_val[i + 1] = True
            i += 2
        else:
            i += 1
    opens = opens[~is_val[opens]]
    for o in opens:
        c = pay[o] - 1
        assert pay[c] == o
    # string buffer length is the sum of (5 + length)
    strs = [i for i in range(len(tape)) if not is_val[i] and chr(tags[i]) == '"']
    total = sum(5 + len(tapeutil.read_string(sb, int(pay[s]))) for s in strs)
    assert total == len(sb)
    # the whole tape decodes to what Python's json reads
    assert tapeutil.decode(tape, sb) == tapeutil.fix_lists(tapeutil.py_expected(b))
    del num


def test_config0_invariants_and_json_equality():
    _check_invariants(gen.config0(0))
    _check_invariants(gen.config0(1))


def test_config1_invariants_and_json_equality():
    _check_invariants(gen.config1(1000))


def test_config2_small_invariants_and_json_equality():
    _check_invariants(gen.config2(2000, size=3 << 20))


def test_string_heavy_invariants_and_json_equality():
    _check_invariants(gen.strings_heavy(77, 1 << 20))
