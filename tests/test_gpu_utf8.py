"""GPU UTF-8 validation (Sec. 3.1.5, Table "tab:unicode") against the oracle,
exhaustively over short sequences: every byte pair, every three-byte sequence
that starts with E0-EF, and four-byte sequences starting with F0-F7 over a
set of second/third/fourth bytes that covers every boundary of the table.
Each sequence sits inside a JSON string, once inside one 64-byte block and
once straddling a block edge (the cross-block carry), and once at the very
end of the document (truncated sequences).  Error codes are compared for
every document (one batch per family)."""
import itertools

import numpy as np
import pytest

import oracle
from tests import gpuutil

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def parser():
    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=200 << 20, max_docs=1 << 21)
    yield p
    p.close()


def _docs(seqs, pad):
    """Each sequence inside a string after `pad` filler bytes."""
    pre = b'"' + b"a" * pad
    return [pre + s + b'"' for s in seqs]


def _check(parser, docs, label):
    buf, off = gpuutil.batch_arrays(docs)
    res, _ = parser.parse_batch(buf, off)
    exp = oracle.parse_many_errors(buf, off)
    got = res["error"].astype(np.int32)
    bad = np.nonzero(got != exp)[0]
    assert bad.size == 0, (f"{label}: {bad.size} mismatches, first {docs[bad[0]]!r} "
                           f"gpu {got[bad[0]]} oracle {exp[bad[0]]}")
    return int(np.count_nonzero(exp == oracle.UTF8_ERROR))


EDGES = bytes([0x00, 0x22, 0x41, 0x5C, 0x7F, 0x80, 0x8F, 0x90, 0x9F, 0xA0, 0xBF, 0xC0, 0xC1,
               0xC2, 0xDF, 0xE0, 0xED, 0xEF, 0xF0, 0xF4, 0xF5, 0xFF])


@pytest.mark.parametrize("pad", [0, 61, 62])
def test_all_byte_pairs(parser, pad):
    seqs = [bytes([a, b]) for a in range(256) for b in range(256)]
    n_bad = _check(parser, _docs(seqs, pad), f"pairs pad {pad}")
    assert n_bad > 0


@pytest.mark.parametrize("pad", [1, 61, 62])
def test_three_byte_sequences(parser, pad):
    seqs = [bytes([a, b, c]) for a in range(0xE0, 0xF0) for b in range(256) for c in range(256)]
    _check(parser, _docs(seqs, pad), f"triples pad {pad}")


@pytest.mark.parametrize("pad", [0, 60, 61, 62])
def test_four_byte_sequences(parser, pad):
    seqs = [bytes([a, b, c, d]) for a in range(0xF0, 0xF8) for b in range(256)
            for c in EDGES for d in EDGES]
    _check(parser, _docs(seqs, pad), f"quads pad {pad}")


def test_truncated_at_document_end(parser):
    # a multi-byte lead (and part of its sequence) as the last bytes of a document,
    # after a string that closes: always invalid; ends at every offset of a block
    docs = []
    for n_fill in range(60, 70):
        for tail in (b"\xc3", b"\xe2\x82", b"\xe2", b"\xf0\x9f\x98", b"\xf0\x9f", b"\xf0"):
            docs.append(b'["' + b"a" * n_fill + b'"]' + tail)
            docs.append(b'["' + b"a" * n_fill + tail)
    _check(parser, docs, "truncated")


def test_mixed_text_blocks(parser):
    rng = np.random.Generator(np.random.PCG64(17))
    alphabet = [b"a", b"\xc3\xa9", b"\xe2\x82\xac", b"\xf0\x9f\x98\x80", b"\xed\x9f\xbf",
                b"\xee\x80\x80", b"\xf4\x8f\xbf\xbf", b"\xe0\xa0\x80", b"\xf0\x90\x80\x80"]
    wrong = [b"\xc0\x80", b"\xed\xa0\x80", b"\xf4\x90\x80\x80", b"\xe0\x9f\xbf", b"\xf0\x8f\xbf\xbf",
             b"\x80", b"\xc3", b"\xf8\x88\x80\x80\x80", b"\xe2\x82", b"\xff"]
    docs = []
    for i in range(20000):
        parts = [alphabet[int(k)] for k in rng.integers(0, len(alphabet), int(rng.integers(1, 90)))]
        if i % 3 == 0:
            parts.insert(int(rng.integers(0, len(parts) + 1)), wrong[int(rng.integers(0, len(wrong)))])
        docs.append(b'"' + b"".join(parts) + b'"')
    _check(parser, docs, "mixed")
