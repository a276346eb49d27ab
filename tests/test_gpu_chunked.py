"""Host documents parsed while they are copied (sj_parser_set_host_chunk): a
single document in pinned host memory, longer than one chunk, is copied chunk
by chunk on a second stream; stage 1 runs on each chunk as it lands and
stage 2 on the tiles whose tokens end in landed bytes.  Every result must
equal the parse of the same bytes in device memory and the oracle's, for
chunk sizes down to one tile and for documents whose tokens, strings, escape
runs, white space and nesting straddle chunk edges."""
import numpy as np
import pytest

import gen
import oracle
from tests import gpuutil

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K = 2048  # one tile


def _long_string_doc():
    # a string of ~150 KB with escapes and non-ASCII bytes: whole chunks
    # without an index, and escapes across chunk edges
    body = (b"ab\\n\\\"c\xc3\xa9\\u00e9" + b"x" * 61 + b"\\\\") * 1500
    return b'[1, "' + body + b'", {"k": "v", "n": -1.5e-3}, "' + body[:40000] + b'"]'


def _docs():
    docs = {
        "config0": gen.config0(7).tobytes(),
        "config1": gen.config1(1007).tobytes(),
        "config2_1MiB": gen.config2(2007, size=(1 << 20) + 37).tobytes(),
        "long_string": _long_string_doc(),
        "white_space_run": b"[1," + b" " * 100_000 + b"2, " + b"\n" * 50_001 + b"3]",
        "deep": b"[" * 3000 + b'{"a": 1}' + b"]" * 3000,
        "root_string": b'"' + b"q" * 90_000 + b'"',
        "root_string_trailing_ws": b'"' + b"q" * 20_000 + b'"' + b" " * 30_000,
        "numbers_on_edges": b"[" + b",".join(b"%d.%d" % (i, i * 7) for i in range(20_000)) + b"]",
        "backslash_runs": b"[" + b",".join(b'"' + b"\\\\" * (i % 40) + b'"' for i in range(6000)) + b"]",
    }
    base = docs["config2_1MiB"]
    docs["utf8_error_late"] = base[:-100] + b"\xff" + base[-99:]
    docs["utf8_error_early"] = base[:3000] + b"\xc0\x80" + base[3002:]
    docs["unclosed_string"] = base[: len(base) // 2] + b'"' + b"z" * 100_000
    docs["tape_error_middle"] = base[: len(base) // 2].replace(b", ", b"  ", 1) + base[len(base) // 2:]
    docs["unbalanced_end"] = b"[" * 10 + b"1" + b"]" * 9 + b" " * 70_000
    return docs


@pytest.fixture(scope="module")
def parser():
    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=4 << 20, max_docs=8)
    yield p
    p.close()


def _pinned(d, shift=0):
    t = torch.empty(len(d) + shift, dtype=torch.uint8).pin_memory()
    t[shift:] = torch.frombuffer(bytearray(d), dtype=torch.uint8)
    return t[shift:]


@pytest.mark.parametrize("chunk", [K, 8 * K, 33 * K])
def test_chunked_host_input_matches_device_input_and_oracle(parser, chunk):
    docs = _docs()
    for name, d in docs.items():
        parser.set_host_chunk(0)
        ref = gpuutil.gpu_result(parser, torch.frombuffer(bytearray(d), dtype=torch.uint8).cuda())
        parser.set_host_chunk(chunk)
        got = gpuutil.gpu_result(parser, _pinned(d, shift=3))
        gpuutil.compare(got, ref, f"{name} chunk {chunk}: chunked vs device")
        gpuutil.compare(got, oracle.parse(d), f"{name} chunk {chunk}: chunked vs oracle")
    parser.set_host_chunk(512 << 20)


def test_chunked_runs_interleave_with_other_runs(parser):
    # chunked, resident, chunked again, and a batch: no state leaks between runs
    docs = _docs()
    a, b = docs["config2_1MiB"], docs["long_string"]
    parser.set_host_chunk(4 * K)
    for d in (a, b, a):
        gpuutil.compare(gpuutil.gpu_result(parser, _pinned(d)), oracle.parse(d), "chunked")
        dev = torch.frombuffer(bytearray(d), dtype=torch.uint8).cuda()
        gpuutil.compare(gpuutil.gpu_result(parser, dev), oracle.parse(d), "resident")
    small = [docs["config0"], b"[1, 2]", b"tru"]
    buf, off = gpuutil.batch_arrays(small)
    res, _ = parser.parse_batch(buf, off)
    assert [int(e) for e in res["error"]] == [oracle.parse(s)["error"] for s in small]
    parser.set_host_chunk(512 << 20)


def test_many_chunks_are_merged(parser):
    # one-tile chunks: the 64th chunk takes the rest of the document
    d = _docs()["config2_1MiB"]
    parser.set_host_chunk(K)  # 63 chunks of one tile, then 450 tiles
    gpuutil.compare(gpuutil.gpu_result(parser, _pinned(d)), oracle.parse(d), "merged chunks")
    parser.set_host_chunk(512 << 20)


def test_chunks_spanning_several_scan_blocks():
    # a tile scan covers 1024 tiles (2 MiB) per block: with a largest chunk of
    # 6 MiB the later chunks span several scan blocks, each scan starting from
    # the carry of the chunk before
    import paper_1902_08318_gb300 as sj
    d = gen.config2(2011, size=(20 << 20) + 1234).tobytes()
    p = sj.Parser(max_bytes=len(d) + 64)
    ref = gpuutil.gpu_result(p, torch.frombuffer(bytearray(d), dtype=torch.uint8).cuda())
    for chunk in (6 << 20, (3 << 20) + 2048):
        p.set_host_chunk(chunk)
        got = gpuutil.gpu_result(p, _pinned(d, shift=5))
        gpuutil.compare(got, ref, f"chunk {chunk}: chunked vs device")
    gpuutil.compare(ref, oracle.parse(d), "device vs oracle")
    p.close()
