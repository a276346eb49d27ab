"""Host input: a single document in pinned host memory is read by stage 1
over the host link, which also writes the device copy for stage 2; pageable
host memory and batches are copied first.  Every path gives the same
result as device input, and the oracle's."""
import numpy as np
import pytest

import gen
import oracle
from tests import gpuutil

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _docs():
    return [gen.config0(5).tobytes(), gen.config1(1005).tobytes(),
            gen.config2(2005, size=(1 << 20) + 37).tobytes(), b'{"a": [1, 2.5, "x\\u00e9"]}',
            b"[" + b"1," * 1000 + b"2]", b'"' + b"a" * 63 + b'"', b"7"]


@pytest.mark.parametrize("shift", [0, 1, 5, 16])
def test_pinned_host_input_matches_device_input(shift):
    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=4 << 20)
    for k, d in enumerate(_docs()):
        dev = torch.frombuffer(bytearray(d), dtype=torch.uint8).cuda()
        ref = gpuutil.gpu_result(p, dev)
        pinned = torch.empty(len(d) + shift, dtype=torch.uint8).pin_memory()
        pinned[shift:] = torch.frombuffer(bytearray(d), dtype=torch.uint8)
        got = gpuutil.gpu_result(p, pinned[shift:])
        gpuutil.compare(got, ref, f"doc {k} shift {shift}: pinned vs device")
        gpuutil.compare(got, oracle.parse(d), f"doc {k} shift {shift}: pinned vs oracle")


def test_pageable_host_input_and_invalid_document():
    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=1 << 20)
    for d in (b'{"a": [1, tru]}', b'["\xc3\x28"]', gen.config0(6).tobytes()):
        gpuutil.compare(gpuutil.gpu_result(p, np.frombuffer(d, dtype=np.uint8)), oracle.parse(d),
                        "pageable")
        pinned = torch.frombuffer(bytearray(d), dtype=torch.uint8).pin_memory()
        gpuutil.compare(gpuutil.gpu_result(p, pinned), oracle.parse(d), "pinned")
