"""GPU parity on the error-category families of test_oracle_errors: documents
with one injected defect, and with two ordered defects, parsed one by one and
as one batch; error codes and, where the oracle compares them, indices are
those of the oracle.  Each runs on a parser sized to the documents (at most
2048 stage-2 tiles: numbers converted beside the tile scans, their tape
words written by the build pass) and on a 16 MiB one (numbers converted
beside the build pass, which write their own tape words and errors)."""
import random
import zlib

import numpy as np
import pytest

import oracle
from tests import gpuutil
from tests.test_oracle_errors import SINGLE, _inject, _two

pytestmark = pytest.mark.gpu

PAIRS = [(("value", b"tru"), ("value", b"1.")), (("value", b"1."), ("value", b"tru")),
         (("string", b"\\q"), ("value", b"nul")), (("string", b"a\x02"), ("string", b"\\q")),
         (("value", b"tru"), ("string", b"\xff")), (("value", b"1 2"), ("value", b"fals")),
         # a grammar error and a number error at one token: the grammar's code
         (("value", b"1 2."), ("value", b"nul"))]
BIG = 16 << 20  # a parser above 2048 stage-2 tiles


@pytest.fixture(scope="module")
def docs():
    out = []
    for kind, text, _ in SINGLE:
        rng = random.Random(zlib.crc32(kind.encode() + text) + 1)
        out += [_inject(rng, kind, text) for _ in range(6)]
    rng = random.Random(11)
    for a, b in PAIRS:
        out += [_two(rng, a, b) for _ in range(4)]
    return out


@pytest.mark.parametrize("big", [False, True])
def test_defect_documents_one_by_one(docs, big):
    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=max(max(len(d) for d in docs) + 64, BIG if big else 0))
    try:
        for i, d in enumerate(docs):
            gpuutil.check_doc(p, d, f"doc {i}")
    finally:
        p.close()


@pytest.mark.parametrize("big", [False, True])
def test_defect_documents_in_one_batch(docs, big):
    import paper_1902_08318_gb300 as sj
    buf, off = gpuutil.batch_arrays(docs)
    p = sj.Parser(max_bytes=max(int(off[-1]) + 64, BIG if big else 0), max_docs=len(docs))
    try:
        res, ptrs = p.parse_batch(buf, off)
        exp = oracle.parse_many_errors(buf, off)
        assert np.array_equal(res["error"], exp)
        outs = gpuutil.batch_outputs(p, res, ptrs, int(off[-1]), len(docs))
        for i, d in enumerate(docs):
            gpuutil.compare_batch_doc(res[i], outs, oracle.parse(d), f"doc {i}")
    finally:
        p.close()
