"""Parity on the benchmarked single document (Sec. 3 problem statement; Table
"tab:largefile" for the large-file case).

The 1 GiB config-2 document with the seed bench.py times (2000) is parsed
through the C ABI from device memory and from pinned host memory (the
end-to-end path), and its error code, every structural index, every tape word
and every string-buffer byte are compared with the oracle's, element by
element.  At this size the root array spans ~524,000 tiles, so tiles are
handed out by ticket, containers stay open across hundreds of thousands of
tiles and every carry crosses many thread blocks.
"""
import numpy as np
import pytest

import gen
import oracle
from tests.gpuutil import compare

pytestmark = pytest.mark.gpu

FULL_BYTES = 1 << 30
SEED = 2000  # bench.py's document for rank 0


@pytest.fixture(scope="module")
def full_doc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    doc = gen.config2(SEED, size=FULL_BYTES)
    exp = oracle.parse(doc)
    assert exp["error"] == oracle.SUCCESS
    return doc, exp


def _fetch(r):
    import torch
    out = {"error": r.error, "n_indices": r.n_indices}
    out["indices"] = r.indices().cpu().numpy()
    if r.error == 0:
        out["tape"] = r.tape().cpu().numpy()
        out["strings"] = r.strings().cpu().numpy()
    torch.cuda.synchronize()
    return out


def test_full_size_document_from_device(full_doc):
    import torch

    import paper_1902_08318_gb300 as sj
    doc, exp = full_doc
    p = sj.Parser(max_bytes=doc.size + 64)
    try:
        dev = torch.from_numpy(doc).cuda()
        got = _fetch(p.parse(dev))
        compare(got, exp, "config2 1 GiB (device input)")
        # the same document again on the same parser (state left by a run)
        got = _fetch(p.parse(dev))
        compare(got, exp, "config2 1 GiB (device input, second run)")
        del dev
    finally:
        p.close()


def test_full_size_document_from_pinned_host(full_doc):
    import torch

    import paper_1902_08318_gb300 as sj
    doc, exp = full_doc
    p = sj.Parser(max_bytes=doc.size + 64)
    try:
        host = torch.from_numpy(doc).pin_memory()
        got = _fetch(p.parse(host))
        compare(got, exp, "config2 1 GiB (pinned host input)")
        del host
    finally:
        p.close()
