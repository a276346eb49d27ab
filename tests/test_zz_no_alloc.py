"""The allocation-free stage-1 entry point (sj_stage1_indices_noalloc).

It is meant for callers that may not call cudaMalloc while parsing; its
scratch is a static device array shared by all calls.  Checked through the C
ABI against the indices of the ordinary entry point (sj_parse), on two calls
in a row with different documents so that state left by the first call
cannot leak into the second; against the oracle's stage 1 (indices, unclosed
string) and UTF-8 check over the families that stress its carries (escape
runs across block and tile edges, multi-byte sequences split across blocks,
strings open across many tiles, ragged tails, unaligned starts); and for
allocating nothing.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def _noalloc(lib, doc_dev, stream):
    import torch
    n = doc_dev.numel()
    idx = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    res = torch.zeros(2, dtype=torch.int32, device="cuda")
    st = lib.sj_stage1_indices_noalloc(doc_dev.data_ptr(), n, idx.data_ptr(), res.data_ptr(),
                                       stream.cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    count, flags = (int(x) for x in res.cpu())
    return idx[:count].cpu().numpy().astype(np.uint32), flags


def test_noalloc_matches_sj_parse_on_two_calls():
    import torch

    import paper_1902_08318_gb300 as sj
    lib = sj.load()
    stream = torch.cuda.current_stream()
    docs = [gen.config2(2000, size=5 << 20).tobytes(), gen.config0(5).tobytes()]
    parser = sj.Parser(max_bytes=8 << 20)
    for d in docs:
        dev = torch.frombuffer(bytearray(d), dtype=torch.uint8).cuda()
        got, flags = _noalloc(lib, dev, stream)
        ref = parser.parse(dev)
        assert ref.error == 0 and flags == 0
        exp = ref.indices().cpu().numpy()
        assert got.size == ref.n_indices
        assert np.array_equal(got, exp)
    parser.close()


def test_noalloc_reports_flags_and_rejects_oversize():
    import torch

    import paper_1902_08318_gb300 as sj
    lib = sj.load()
    stream = torch.cuda.current_stream()
    for d, want in ((b'["abc', 2), (b'["\xff"]', 1), (b"[1,2,3]", 0)):
        dev = torch.frombuffer(bytearray(d), dtype=torch.uint8).cuda()
        _, flags = _noalloc(lib, dev, stream)
        assert flags == want
    big = 65 << 20
    assert lib.sj_stage1_indices_noalloc(ctypes.c_void_p(1), big, ctypes.c_void_p(1),
                                         ctypes.c_void_p(1), None) == sj.CAPACITY


def _check_vs_oracle(lib, stream, doc: bytes, label: str, shift: int = 0):
    import torch
    t = torch.zeros(len(doc) + shift + 16, dtype=torch.uint8, device="cuda")
    if doc:
        t[shift: shift + len(doc)] = torch.frombuffer(bytearray(doc), dtype=torch.uint8).cuda()
    got, flags = _noalloc(lib, t[shift: shift + len(doc)], stream)
    exp, unclosed = oracle.stage1(doc)
    want = (0 if oracle.utf8_valid(doc) else 1) | (2 if unclosed else 0)
    assert flags == want, (label, flags, want)
    assert got.size == exp.size and np.array_equal(got, exp), (label, got.size, exp.size)


def test_noalloc_against_oracle_escape_runs_across_edges():
    import torch

    import paper_1902_08318_gb300 as sj
    lib = sj.load()
    stream = torch.cuda.current_stream()
    rng = np.random.Generator(np.random.PCG64(21))
    for _ in range(150):
        pre = int(rng.integers(0, 4200))
        run = int(rng.integers(1, 140))
        doc = b'["' + b"x" * pre + b"\\" * run + (b"" if run % 2 == 0 else b"\\") + b'", 1]'
        _check_vs_oracle(lib, stream, doc, f"pre {pre} run {run}")
        open_doc = b'["' + b"y" * pre + b"\\" * run + b'"]'  # odd runs leave the string open
        _check_vs_oracle(lib, stream, open_doc, f"open pre {pre} run {run}")


def test_noalloc_against_oracle_utf8_across_blocks():
    import torch

    import paper_1902_08318_gb300 as sj
    lib = sj.load()
    stream = torch.cuda.current_stream()
    rng = np.random.Generator(np.random.PCG64(8))
    seqs = [bytes([a, b]) for a, b in rng.integers(0, 256, size=(300, 2))]
    seqs += [bytes([0xE0 + int(a) % 16, b, c]) for a, b, c in rng.integers(0, 256, size=(300, 3))]
    seqs += [bytes([0xF0 + int(a) % 8, b, c, e]) for a, b, c, e in rng.integers(0, 256, size=(300, 4))]
    seqs += [b"\xc3\xa9", b"\xe2\x82\xac", b"\xf0\x9f\x98\x80", b"\xed\xa0\x80", b"\xc0\x80"]
    for i, sq in enumerate(seqs):
        pad = (61, 62, 63, 0)[i % 4]  # across a block edge, or inside one block
        _check_vs_oracle(lib, stream, b'"' + b"a" * pad + sq + b'"', f"seq {sq!r} pad {pad}")
    for n_fill in range(60, 68):  # truncated sequences at the document's end
        for tail in (b"\xc3", b"\xe2\x82", b"\xf0\x9f\x98"):
            _check_vs_oracle(lib, stream, b'["' + b"a" * n_fill + b'"]' + tail, f"tail {n_fill}")


def test_noalloc_against_oracle_long_strings_ragged_tails_unaligned():
    import torch

    import paper_1902_08318_gb300 as sj
    lib = sj.load()
    stream = torch.cuda.current_stream()
    base = gen.config2(2003, size=300_000).tobytes()
    for n in (2047, 2048, 2049, 4095, 4096 + 63, 4096 + 64, 4096 + 65, len(base) - 1, len(base)):
        _check_vs_oracle(lib, stream, base[:n], f"cut {n}")
    for shift in range(1, 16):
        _check_vs_oracle(lib, stream, base[:100_000], f"shift {shift}", shift=shift)
    # strings open across many tiles: the in-string state is carried where no
    # earlier tile in the look-back window has its prefix yet
    body = b"z" * 400_000
    _check_vs_oracle(lib, stream, b'["' + body + b'", "' + body + b'", [1, 2]]', "long strings")
    _check_vs_oracle(lib, stream, b'["' + body + b'\\"' + body + b'"]', "long string, escaped quote")
    _check_vs_oracle(lib, stream, b"", "empty")


def test_noalloc_allocates_no_device_memory():
    import torch

    import paper_1902_08318_gb300 as sj
    lib = sj.load()
    stream = torch.cuda.current_stream()
    doc = gen.config2(2004, size=2 << 20).tobytes()
    dev = torch.frombuffer(bytearray(doc), dtype=torch.uint8).cuda()
    idx = torch.empty(len(doc), dtype=torch.int32, device="cuda")
    res = torch.zeros(2, dtype=torch.int32, device="cuda")
    call = lambda: lib.sj_stage1_indices_noalloc(dev.data_ptr(), len(doc), idx.data_ptr(),
                                                 res.data_ptr(), stream.cuda_stream)
    assert call() == 0  # warm: the per-device set-up happens on the first call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert call() == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
