"""GPU parity: the CUDA library (through its C ABI) against the oracle,
element by element: error code always; indices unless UTF8/CAPACITY/EMPTY;
tape and string buffer on success.  All integer/byte work, so bit-exact."""
import itertools
import os

import numpy as np
import pytest

import gen
import oracle
from tests import gpuutil
from tests.conftest import GOLDEN
from tests.test_oracle_parse import HARD_NUMBERS, SYM16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def parser():
    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=64 << 20, max_docs=70000)
    yield p
    p.close()


def test_paper_worked_example(parser):
    inp = None
    for line in open(os.path.join(GOLDEN, "paper_fig_masks.txt"), encoding="utf-8"):
        if line.startswith("input "):
            inp = line[len("input "):].rstrip("\n").encode()
    got = gpuutil.check_doc(parser, inp, "paper example")
    assert list(got["indices"]) == [0, 2, 13, 15, 17, 20, 21, 28, 30, 33, 35, 41, 43, 49, 50,
                                    52, 55, 56, 63]


def test_fig1_tape(parser):
    doc = open(os.path.join(GOLDEN, "fig1_document.json"), "rb").read()
    got = gpuutil.check_doc(parser, doc, "fig1")
    assert got["tape"].size == 38


NAMED = [b"012", b"1E+", b"[0e+]", b".1", b"1e309", b"-1e309", b"[12 a]", b'"a\nb"',
         b"9223372036854775807", b"9223372036854775808", b"-9223372036854775808",
         b"-9223372036854775809", b'"[1,2]"', b"", b" \n\t\r", b"[", b"]", b"[}", b'{"a" 1}',
         b'{"a":1,}', b"[1,]", b"tru", b"falsey", b"nul", b'"abc', b'"\\q"', b'"\\uD800"',
         b'"\\uDC00\\uD800"', b"1 2", b'1"a"', b"[1\x01]", b"[\x01]", b"\xef\xbb\xbf{}",
         b'{"a":1,"a":2}', b"-0", b"-0.0", b"1e-400", b'["\x7f"]', b'"\\uD834\\uDD1E"',
         b'["a\\u0000b"]', b"true", b"false", b"null", b"[true,false,null]", b"{}", b"[]",
         b"[[[]]]", b'{"a":{"b":{"c":[1,{"d":null}]}}}', b'["\xb1\x87"]', b"\xc3\xa9",
         b'"\xc3\xa9\xe2\x82\xac\xf0\x9f\x98\x80"', b"1.5e", b"-", b"--1", b"01.5", b"1.",
         b'{"a":}', b'{:1}', b'{"a"::1}', b"[,1]", b"[1,,2]", b'{"a":1 "b":2}', b"[]]",
         b'["a":1]', b'{"a",1}', b'{"a"}', b'{"a":1,"b"}']


@pytest.mark.parametrize("doc", NAMED)
def test_named_cases(parser, doc):
    gpuutil.check_doc(parser, doc)


def test_hard_numbers(parser):
    rng = np.random.Generator(np.random.PCG64(9))
    lex = list(HARD_NUMBERS)
    for _ in range(3000):
        sig = int(rng.integers(1, 25))
        digits = str(int(rng.integers(1, 10))) + "".join(str(int(rng.integers(0, 10))) for _ in range(sig - 1))
        p = int(rng.integers(1, sig + 1))
        s = digits[:p] + "." + (digits[p:] or "0")
        if rng.random() < 0.6:
            s += "e" + str(int(rng.integers(-345, 312)))
        if rng.random() < 0.5:
            s = "-" + s
        lex.append(s)
    # one document holding all of them, and each alone for exact error codes
    gpuutil.check_doc(parser, ("[" + ",".join(l for l in lex if oracle.parse(l.encode())["error"] == 0) + "]").encode(),
                      "numbers array")
    for s in lex[:400]:
        gpuutil.check_doc(parser, s.encode(), s)


def test_exhaustive_tiny_documents_batch(parser):
    docs = [b"".join(c) for n in range(1, 5) for c in itertools.product(SYM16, repeat=n)]
    buf, off = gpuutil.batch_arrays(docs)
    res, ptrs = parser.parse_batch(buf, off)
    outs = gpuutil.batch_outputs(parser, res, ptrs, int(off[-1]), len(docs))
    for i, d in enumerate(docs):
        gpuutil.compare_batch_doc(res[i], outs, oracle.parse(d), repr(d))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_config0(parser, seed):
    gpuutil.check_doc(parser, gen.config0(seed).tobytes(), f"config0 seed {seed}")


def test_config1(parser):
    gpuutil.check_doc(parser, gen.config1(1000).tobytes(), "config1")


def test_config2_small(parser):
    gpuutil.check_doc(parser, gen.config2(2000, size=8 << 20).tobytes(), "config2 8MB")


def test_strings_heavy(parser):
    gpuutil.check_doc(parser, gen.strings_heavy(5, 2 << 20).tobytes(), "strings heavy")


def test_alignment_and_ragged_tails(parser):
    import torch
    base = gen.config0(3).tobytes()[:9000]
    for cut in [1, 2, 63, 64, 65, 127, 128, 2047, 2048, 2049, 4095, 4096, 4097, 8999]:
        doc = base[:cut]
        exp = oracle.parse(doc)
        for shift in (0, 1, 3, 5, 8, 13, 15):
            dev = torch.zeros(cut + 32, dtype=torch.uint8, device="cuda")
            dev[shift: shift + cut] = torch.frombuffer(bytearray(doc), dtype=torch.uint8).cuda()
            got = gpuutil.gpu_result(parser, dev[shift: shift + cut])
            gpuutil.compare(got, exp, f"cut {cut} shift {shift}")


def test_deep_nesting(parser):
    for depth in (1, 2, 31, 32, 33, 100, 1024, 2047, 2048, 2049, 4095, 4096, 4097, 6000):
        doc = b"[" * depth + b"1" + b"]" * depth
        gpuutil.check_doc(parser, doc, f"depth {depth}")
        doc = b'{"k":' * depth + b"null" + b"}" * depth
        gpuutil.check_doc(parser, doc, f"obj depth {depth}")
    gpuutil.check_doc(parser, b"[" * 5000, "unclosed 5000")
    gpuutil.check_doc(parser, b"]" * 3000, "closers 3000")


def test_escape_runs_across_edges(parser):
    rng = np.random.Generator(np.random.PCG64(21))
    for _ in range(300):
        pre = int(rng.integers(0, 4200))
        run = int(rng.integers(1, 140))
        doc = b'["' + b"x" * pre + b"\\" * run + (b"" if run % 2 == 0 else b"\\") + b'", 1]'
        gpuutil.check_doc(parser, doc, f"pre {pre} run {run}")
        doc2 = b'["' + b"y" * pre + b"\\" * run + b'"]'  # odd runs leave the string open
        gpuutil.check_doc(parser, doc2, f"open pre {pre} run {run}")


def test_random_corruptions(parser):
    rng = np.random.Generator(np.random.PCG64(33))
    base = gen.config0(4).tobytes()[:6000] + b"}"
    alphabet = b'{}[]:,"\\ \n0123456789-.eEtfnalsru\x01\x7f\xc3\xa9\xff'
    for i in range(400):
        d = bytearray(base)
        for _ in range(int(rng.integers(1, 4))):
            op = rng.integers(0, 3)
            pos = int(rng.integers(0, len(d)))
            c = alphabet[int(rng.integers(0, len(alphabet)))]
            if op == 0:
                d[pos] = c
            elif op == 1:
                d.insert(pos, c)
            else:
                del d[pos]
        gpuutil.check_doc(parser, bytes(d), f"corruption {i}")


def test_max_depth_parameter():
    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=1 << 16, max_depth=3)
    for doc in (b"[[[1]]]", b"[[[[1]]]]", b'{"a":{"b":{"c":1}}}', b'{"a":{"b":{"c":{}}}}'):
        exp = oracle.parse(doc, max_depth=3)
        gpuutil.compare(gpuutil.gpu_result(p, doc), exp, repr(doc))
    p.close()


def test_repeated_calls_reuse_state(parser):
    docs = [gen.config0(7).tobytes(), b"[1,2", b'{"a":"b"}', gen.config1(1001).tobytes()[:50000] + b"]]}"]
    for _ in range(3):
        for d in docs:
            gpuutil.check_doc(parser, d)
