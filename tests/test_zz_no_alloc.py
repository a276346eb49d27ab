"""The allocation-free stage-1 entry point (sj_stage1_indices_noalloc).

It is meant for callers that may not call cudaMalloc while parsing; its
scratch is a static device array shared by all calls.  Checked through the C
ABI against the indices of the ordinary entry point (sj_parse), on two calls
in a row with different documents so that state left by the first call
cannot leak into the second.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import gen

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
