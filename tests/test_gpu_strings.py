"""String validation and normalisation (Sec. 3.2.2) against the oracle on
random escape-heavy strings: every escape form, bad escapes, lone and
reversed surrogates, raw control bytes, quotes and backslash runs, non-ASCII
text, strings crossing 64-byte blocks and 2 KiB tiles.  Error codes for every
document; indices, tape and string buffer for a sample."""
import numpy as np
import pytest

import oracle
from tests import gpuutil

pytestmark = pytest.mark.gpu

PIECES = [b"a", b"bc", b"xyz1", b" ", b"\xc3\xa9", b"\xe2\x82\xac", b"\xf0\x9f\x98\x80", b"\\n", b"\\t",
          b"\\\"", b"\\\\", b"\\/", b"\\b", b"\\f", b"\\r", b"\\u00e9", b"\\u0041", b"\\uffff",
          b"\\u20AC", b"\\uD834\\uDD1E", b"\\ud83d\\ude00", b"\\u0000", b"\\\\\\\"", b"\\\\\\\\"]
BAD = [b"\\q", b"\\u12", b"\\u12G4", b"\\uD800", b"\\uDC00", b"\\uD800\\u0041", b"\\uD800x",
       b"\x01", b"\x1f", b"\t", b"\\", b"\\x41", b"\\U0041"]


@pytest.fixture(scope="module")
def parser():
    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=64 << 20, max_docs=60000)
    yield p
    p.close()


def _doc(rng):
    strs = []
    for _ in range(int(rng.integers(1, 6))):
        parts = [PIECES[int(k)] for k in rng.integers(0, len(PIECES), int(rng.integers(0, 40)))]
        if rng.random() < 0.15:
            parts.insert(int(rng.integers(0, len(parts) + 1)), BAD[int(rng.integers(0, len(BAD)))])
        strs.append(b'"' + b"".join(parts) + b'"')
    pad = b" " * int(rng.integers(0, 70))
    return b"[" + pad + b",".join(strs) + b"]"


def test_random_strings_error_codes(parser):
    rng = np.random.Generator(np.random.PCG64(23))
    docs = [_doc(rng) for _ in range(50000)]
    buf, off = gpuutil.batch_arrays(docs)
    res, _ = parser.parse_batch(buf, off)
    exp = oracle.parse_many_errors(buf, off)
    bad = np.nonzero(res["error"].astype(np.int32) != exp)[0]
    assert bad.size == 0, (docs[bad[0]], int(res["error"][bad[0]]), int(exp[bad[0]]))
    assert np.count_nonzero(exp == 0) > 1000 and np.count_nonzero(exp != 0) > 1000


def test_random_strings_full_output(parser):
    rng = np.random.Generator(np.random.PCG64(29))
    for i in range(400):
        gpuutil.check_doc(parser, _doc(rng), f"doc {i}")


def test_long_escaped_strings_across_tiles(parser):
    rng = np.random.Generator(np.random.PCG64(31))
    parts = [PIECES[int(k)] for k in rng.integers(0, len(PIECES), 3000)]
    big = b'{"k": "' + b"".join(parts) + b'", "n": [' + b",".join(
        b'"' + b"".join(PIECES[int(k)] for k in rng.integers(0, len(PIECES), 50)) + b'"'
        for _ in range(400)) + b"]}"
    gpuutil.check_doc(parser, big, "long escaped strings")
