"""GPU parity of the batched path (sj_parse_batch): many independent documents
in one launch sequence, carries reset at every document start.  Every
document's error code is compared with the oracle; indices, tape and strings
on a sample and on every document that is not valid."""
import numpy as np
import pytest

import gen
import oracle
from tests import gpuutil

pytestmark = pytest.mark.gpu


def _check_batch(parser, buf, off, full_every=1):
    res, ptrs = parser.parse_batch(buf, off)
    n = off.size - 1
    exp_err = oracle.parse_many_errors(buf, off)
    got_err = res["error"]
    bad = np.nonzero(got_err != exp_err)[0]
    assert bad.size == 0, (f"{bad.size} documents differ, first {bad[:5]}: got "
                           f"{got_err[bad[:5]]} expected {exp_err[bad[:5]]}")
    outs = gpuutil.batch_outputs(parser, res, ptrs, int(off[-1] - off[0]), n)
    for i in range(n):
        if i % full_every == 0 or exp_err[i] != 0:
            d = buf[int(off[i]): int(off[i + 1])].tobytes()
            gpuutil.compare_batch_doc(res[i], outs, oracle.parse(d), f"doc {i}")
    return res


@pytest.fixture(scope="module")
def parser():
    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=200 << 20, max_docs=100_000)
    yield p
    p.close()


def test_config3_shaped_batch(parser):
    buf, off = gen.config3(3000, n_docs=12_000, invalid_frac=0.02)
    res = _check_batch(parser, buf, off, full_every=7)
    assert (res["error"] != 0).sum() > 100  # the defects are really there


def test_batch_with_empty_and_tiny_documents(parser):
    docs = [b"", b" ", b"1", b"[]", b"{", b'"', b"\\", b'"\\', b"[1,2]", b"  \n", b"\xff",
            b'{"a":[1,2,{"b":null}]}', b"tru", b"[" * 100 + b"]" * 100]
    docs = docs * 50
    buf, off = gpuutil.batch_arrays(docs)
    _check_batch(parser, buf, off)


def test_batch_unaligned_document_starts(parser):
    rng = np.random.Generator(np.random.PCG64(4))
    docs = []
    for i in range(400):
        d = gen.records(77 + i, int(rng.integers(50, 9000)), pretty=bool(i & 1)).tobytes()
        docs.append(d)
    buf, off = gpuutil.batch_arrays(docs)  # offsets land at arbitrary byte alignments
    assert any(int(o) % 16 for o in off[:-1])
    _check_batch(parser, buf, off)


def test_batch_equals_single_parses(parser):
    import paper_1902_08318_gb300 as sj
    docs = [gen.config0(s).tobytes() for s in range(3)] + [gen.config1(1000).tobytes()]
    buf, off = gpuutil.batch_arrays(docs)
    res, ptrs = parser.parse_batch(buf, off)
    outs = gpuutil.batch_outputs(parser, res, ptrs, int(off[-1]), len(docs))
    single = sj.Parser(max_bytes=4 << 20)
    for i, d in enumerate(docs):
        got = gpuutil.gpu_result(single, d)
        gpuutil.compare_batch_doc(res[i], outs, got, f"doc {i} batch vs single")
    single.close()


def test_large_batch_error_codes():
    """The benchmark's batch shape: 100,000 documents in one launch sequence."""
    import paper_1902_08318_gb300 as sj
    buf, off = gen.config3(3000, n_docs=100_000)
    p = sj.Parser(max_bytes=int(off[-1]) + 64, max_docs=100_000)
    res, _ = p.parse_batch(buf, off)
    exp = oracle.parse_many_errors(buf, off)
    p.close()
    assert np.array_equal(res["error"], exp)
