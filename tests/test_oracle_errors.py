"""Pins of the oracle's error categories that do not come from the oracle:
valid documents are written by Python's json module from random values, one
placeholder among them is replaced by a defect whose category the reading of
the paper fixes (Sec. 3, Sec. 3.1.5, Sec. 3.2.1, Sec. 3.2.2; the precedence
of several problems is the reading listed with the oracle), and the oracle
must give that category.  With two defects, the precedence decides: a UTF-8
error or an unclosed string before any token error, else the first failing
token in document order; inside one token, a grammar failure before a content
failure, and inside one string the first problem in byte order."""
import json
import random
import zlib

import pytest

import oracle

STR_MARK = "@@S@@"      # replaced inside a string's quotes
VAL_MARK = 987654321123  # replaced as a whole value


def _value(rng, depth):
    k = rng.random()
    if depth > 3 or k < 0.35:
        return rng.choice([rng.randint(-10**9, 10**9), rng.random() * 10 ** rng.randint(-5, 5),
                           "".join(rng.choice("abcxyz é漢") for _ in range(rng.randint(0, 12))),
                           True, False, None])
    if k < 0.7:
        return [_value(rng, depth + 1) for _ in range(rng.randint(0, 5))]
    return {f"k{i}{rng.randint(0, 99)}": _value(rng, depth + 1) for i in range(rng.randint(0, 5))}


def _doc_with(rng, marker):
    """A random document with `marker` at a random place (as one value)."""
    root = {"pre": _value(rng, 1), "items": [_value(rng, 2) for _ in range(rng.randint(0, 4))]}
    root["items"].insert(rng.randint(0, len(root["items"])), marker)
    root["post"] = _value(rng, 1)
    return json.dumps(root, ensure_ascii=False, indent=rng.choice([None, 2])).encode()


def _inject(rng, kind, text: bytes):
    if kind == "string":
        d = _doc_with(rng, STR_MARK)
        return d.replace(STR_MARK.encode(), text, 1)
    d = _doc_with(rng, VAL_MARK)
    return d.replace(str(VAL_MARK).encode(), text, 1)


# (where the defect goes, its text, the category the reading fixes)
SINGLE = [
    ("string", b"ab\x01cd", oracle.UNESCAPED_CHARS),
    ("string", b"ab\x1f", oracle.UNESCAPED_CHARS),
    ("string", b"ab\\qcd", oracle.STRING_ERROR),
    ("string", b"\\u12g4", oracle.STRING_ERROR),
    ("string", b"x\\ud800y", oracle.STRING_ERROR),        # lone high surrogate
    ("string", b"\\udc00", oracle.STRING_ERROR),           # lone low surrogate
    ("string", b"ab\xffcd", oracle.UTF8_ERROR),
    ("string", b"\xe0\x80\xaf", oracle.UTF8_ERROR),        # overlong
    ("string", b"\xed\xa0\x80", oracle.UTF8_ERROR),        # encoded surrogate
    ("value", b"tru", oracle.T_ATOM_ERROR),
    ("value", b"trueX", oracle.T_ATOM_ERROR),
    ("value", b"fals", oracle.F_ATOM_ERROR),
    ("value", b"nul", oracle.N_ATOM_ERROR),
    ("value", b"1.", oracle.NUMBER_ERROR),
    ("value", b"-", oracle.NUMBER_ERROR),
    ("value", b"01", oracle.NUMBER_ERROR),
    ("value", b"1e400", oracle.NUMBER_ERROR),              # overflow
    ("value", b"99999999999999999999", oracle.NUMBER_ERROR),  # beyond int64
    ("value", b"1 2", oracle.TAPE_ERROR),                   # two values, no comma
    ("value", b"[1,]", oracle.TAPE_ERROR),
    ("value", b'{"a" 1}', oracle.TAPE_ERROR),
    ("value", b"]", oracle.TAPE_ERROR),
]


@pytest.mark.parametrize("kind,text,code", SINGLE)
def test_single_defect_category(kind, text, code):
    rng = random.Random(zlib.crc32(kind.encode() + text))
    for _ in range(40):
        d = _inject(rng, kind, text)
        assert oracle.parse(d)["error"] == code, d[:200]


def test_valid_documents_are_valid():
    rng = random.Random(5)
    for _ in range(200):
        d = _doc_with(rng, 7)
        assert oracle.parse(d)["error"] == oracle.SUCCESS


def test_structure_defects():
    rng = random.Random(6)
    for _ in range(50):
        d = _doc_with(rng, 7)
        assert oracle.parse(d[:-1] if d.endswith(b"}") else d + b"]")["error"] == oracle.TAPE_ERROR
        assert oracle.parse(d + b" ]")["error"] == oracle.TAPE_ERROR
        assert oracle.parse(d + b' "x')["error"] == oracle.UNCLOSED_STRING
        assert oracle.parse(b"[" * 5000 + d + b"]" * 5000)["error"] == oracle.DEPTH_ERROR


def _two(rng, first, second):
    """A document with defect `first` early (in "pre") and `second` late."""
    d = json.dumps({"pre": [STR_MARK if first[0] == "string" else VAL_MARK],
                    "mid": _value(rng, 1),
                    "post": ["@@T@@" if second[0] == "string" else 123123123123]},
                   ensure_ascii=False).encode()
    a = STR_MARK.encode() if first[0] == "string" else str(VAL_MARK).encode()
    b = b"@@T@@" if second[0] == "string" else b"123123123123"
    return d.replace(a, first[1], 1).replace(b, second[1], 1)


@pytest.mark.parametrize("first,second,code", [
    # token errors: the first in document order
    (("value", b"tru"), ("value", b"1."), oracle.T_ATOM_ERROR),
    (("value", b"1."), ("value", b"tru"), oracle.NUMBER_ERROR),
    (("string", b"\\q"), ("value", b"nul"), oracle.STRING_ERROR),
    (("value", b"nul"), ("string", b"\\q"), oracle.N_ATOM_ERROR),
    (("string", b"a\x02"), ("string", b"\\q"), oracle.UNESCAPED_CHARS),
    (("value", b"1 2"), ("value", b"fals"), oracle.TAPE_ERROR),
    # whole-input errors before any token error, wherever they are
    (("value", b"tru"), ("string", b"\xff"), oracle.UTF8_ERROR),
    (("string", b"\\q"), ("string", b"\xc0\x80"), oracle.UTF8_ERROR),
])
def test_two_defects_precedence(first, second, code):
    rng = random.Random(9)
    for _ in range(20):
        assert oracle.parse(_two(rng, first, second))["error"] == code


def test_unclosed_string_before_token_errors():
    rng = random.Random(10)
    for _ in range(20):
        d = _two(rng, ("value", b"tru"), ("value", b"1."))
        assert oracle.parse(d + b'"')["error"] == oracle.UNCLOSED_STRING
        assert oracle.parse(d + b'"\xff')["error"] == oracle.UTF8_ERROR


# Problems inside one token, with the category the readings fix: a grammar
# failure at a token comes before a content failure of the same token, and
# inside one string the first problem in byte order decides.
SAME_TOKEN = [
    (b"[1 2.]", oracle.TAPE_ERROR),            # no comma before a bad number
    (b'{"a" tru}', oracle.TAPE_ERROR),         # no colon before a bad atom
    (b'["a" "\\q"]', oracle.TAPE_ERROR),       # no comma before a bad escape
    (b'{"a":1 "b\\q":2}', oracle.TAPE_ERROR),  # no comma before a key with a bad escape
    (b'["\\q\x01"]', oracle.STRING_ERROR),     # bad escape, then a control byte
    (b'["\x01\\q"]', oracle.UNESCAPED_CHARS),  # control byte, then a bad escape
    (b'["\\ud800\x02"]', oracle.STRING_ERROR),  # lone surrogate, then a control byte
    (b'["a\x1f\\ud800"]', oracle.UNESCAPED_CHARS),
]


@pytest.mark.parametrize("doc,code", SAME_TOKEN)
def test_problems_inside_one_token(doc, code):
    assert oracle.parse(doc)["error"] == code


@pytest.mark.parametrize("doc,code", [c for c in SAME_TOKEN if c[0].startswith(b"[")])
def test_problems_inside_one_token_in_records(doc, code):
    # the same array, as a value inside a seeded valid document, keeps its category
    rng = random.Random(zlib.crc32(doc))
    inner = doc[1:-1]  # the array's content
    for _ in range(10):
        d = _doc_with(rng, VAL_MARK).replace(str(VAL_MARK).encode(), b"[" + inner + b"]", 1)
        assert oracle.parse(d)["error"] == code, d[:200]
