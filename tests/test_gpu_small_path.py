"""GPU parity on both sides of the size thresholds of the launch sequence:
parsers of at most kSubTiles (512) tiles split each tile in four for stage 2;
parsers of at most kSmallTiles (2048) stage-2 tiles scan in one thread block
and build the sparse table there, larger ones use the multi-block scans; runs of
at most kZeroCopyDocs (1024) documents (their graph bucket) take their
descriptor and offsets from pinned host memory and write their results there,
larger runs copy.  Every result is compared with the oracle."""
import numpy as np
import pytest

import gen
import oracle
from tests import gpuutil

pytestmark = pytest.mark.gpu

TILE = 2048
# max_tiles = max_bytes // 2048 + max_docs + 1 (one document)
SUB_MAX_BYTES = (512 - 2) * TILE          # 512 tiles: stage-2 tiles of 512 bytes
WHOLE_MAX_BYTES = (512 - 1) * TILE        # 513 tiles: stage-2 tiles of 2 KiB
SMALL_MAX_BYTES = (2048 - 2) * TILE - 1   # 2047 tiles: the one-block path
LARGE_MAX_BYTES = (2048 - 1) * TILE       # 2049 tiles: the multi-block path


def _docs():
    docs = [gen.config0(0).tobytes(), gen.config1(1000).tobytes(),
            gen.config2(11, size=3 << 20).tobytes(),
            b'["' + b"\\\\" * 3000 + b'", {"k": [' + b"[" * 600 + b"]" * 600 + b"]}]",
            b'{"s": "' + "é漢😀\\u00e9\\ud83d\\ude00".encode() * 2000 + b'"}',
            b"[1, 2", b'{"a": "\x01"}', b"  ", b'"' + b"x" * 9000 + b'"']
    # about the largest document the one-block parser takes (2046 tiles)
    big = gen.config2(12, size=SMALL_MAX_BYTES - 4096).tobytes()
    assert len(big) <= SMALL_MAX_BYTES
    docs.append(big)
    docs.append(gen.config2(13, size=SUB_MAX_BYTES - 4096).tobytes())  # ~the largest split
    return docs


@pytest.fixture(scope="module")
def cases():
    return [(d, oracle.parse(d)) for d in _docs()]


@pytest.mark.parametrize("max_bytes", [SUB_MAX_BYTES, WHOLE_MAX_BYTES, SMALL_MAX_BYTES,
                                       LARGE_MAX_BYTES])
def test_parsers_either_side_of_the_small_thresholds(max_bytes, cases):
    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=max_bytes)
    try:
        small = p.kernels_per_run() < 15
        assert small == (max_bytes != LARGE_MAX_BYTES)
        for i, (d, exp) in enumerate(cases):
            if len(d) > max_bytes:
                continue
            got = gpuutil.gpu_result(p, np.frombuffer(d, dtype=np.uint8))
            gpuutil.compare(got, exp, f"max_bytes {max_bytes}, doc {i} ({len(d)} bytes)")
    finally:
        p.close()


def _check_batch(parser, docs):
    buf, off = gpuutil.batch_arrays(docs)
    res, ptrs = parser.parse_batch(buf, off)
    n = len(docs)
    exp_err = oracle.parse_many_errors(buf, off)
    bad = np.nonzero(res["error"] != exp_err)[0]
    assert bad.size == 0, f"{bad.size} documents differ, first {bad[:5]}"
    outs = gpuutil.batch_outputs(parser, res, ptrs, int(off[-1]), n)
    for i in list(range(0, n, 37)) + [n - 1] + [int(k) for k in np.nonzero(exp_err)[0][:20]]:
        gpuutil.compare_batch_doc(res[i], outs, oracle.parse(docs[i]), f"doc {i} of {n}")


@pytest.mark.parametrize("small_parser", [True, False])
@pytest.mark.parametrize("n_docs", [1, 1023, 1024, 1025, 2048])
def test_batches_either_side_of_the_zero_copy_bucket(small_parser, n_docs):
    import paper_1902_08318_gb300 as sj
    rng = np.random.Generator(np.random.PCG64(n_docs))
    tiny = [b"", b"1", b"[]", b"{", b'"', b"[1,2]", b"\xff", b'{"a":[1,{"b":null}]}', b"tru"]
    docs = []
    for i in range(n_docs):
        if i % 3 == 0:
            docs.append(tiny[i % len(tiny)])
        else:
            docs.append(gen.records(500 + i, int(rng.integers(60, 1200)), pretty=bool(i & 1)).tobytes())
    total = sum(len(d) for d in docs)
    # a parser of at most 2048 tiles (one-block scans) or one of many more
    if small_parser:
        if n_docs >= 2046:
            pytest.skip("a parser for this many documents has more than 2048 tiles")
        max_docs, max_bytes = n_docs, (2047 - n_docs) * TILE
    else:
        max_docs, max_bytes = 2100, 64 << 20
    assert total <= max_bytes
    p = sj.Parser(max_bytes=max_bytes, max_docs=max_docs)
    try:
        assert (p.kernels_per_run() < 15) == (max_bytes // TILE + max_docs + 1 <= 2048)
        _check_batch(p, docs)
        _check_batch(p, docs)  # the same bucket's graph again
    finally:
        p.close()


def test_batch_on_a_parser_with_split_tiles():
    """A batch on a parser of at most 512 tiles: documents of every size up to
    a few tiles, each split in 512-byte stage-2 tiles, carries reset at every
    document."""
    import paper_1902_08318_gb300 as sj
    rng = np.random.Generator(np.random.PCG64(77))
    docs = [b"", b"[", b'"\\', b"[1,2]", b'{"a":"\\u00e9"}', b"1e400"]
    for i in range(190):
        docs.append(gen.records(900 + i, int(rng.integers(40, 5000)), pretty=bool(i & 1)).tobytes())
    p = sj.Parser(max_bytes=600 << 10, max_docs=200)  # 300 + 201 tiles
    try:
        assert sum(len(d) for d in docs) <= 600 << 10
        _check_batch(p, docs)
        _check_batch(p, docs[::-1])
    finally:
        p.close()

