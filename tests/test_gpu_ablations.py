"""GPU parity of the stage-1 variants used for the paper's "Effect of Specific
Optimizations" measurements (Table "tab:optimization"): every variant library
(one plain step swapped in, see csrc/s1_common.cuh) must give the oracle's
error, indices, tape and strings on the config-2 shaped 8 MiB document, the
config-1 document and stage-1 edge cases."""
import numpy as np
import pytest

import gen
import oracle
from tests.gpuutil import compare, gpu_result

pytestmark = pytest.mark.gpu


def _edge_docs():
    docs = []
    # escape runs of every length ending at every offset around a 64-byte edge
    for k in range(1, 9):
        for pad in range(56, 66):
            docs.append(b'["' + b"a" * pad + b"\\\\" * (k // 2) + (b'\\"' if k % 2 else b"") + b'", 1]')
    docs.append(b"[" + b'"' + b"\\\\" * 40 + b'"' + b"]")          # a block of backslashes
    docs.append(b'{"k": "' + "é漢😀".encode() * 300 + b'"}')       # multi-byte text across blocks
    docs.append(b'["ok", "\xe0\x80\xaf"]')                           # overlong: UTF8_ERROR
    docs.append(b'["open string ' + b"x" * 5000)                      # unclosed over tiles
    docs.append(b'[' + b" " * 4093 + b'"x"]')                          # token after a long white run
    docs.append(b'"' + b"s" * 3000 + b'"')                            # root string over two tiles
    return docs


@pytest.fixture(scope="module")
def cases():
    docs = [("config2 8 MiB", gen.config2(7, size=8 << 20).tobytes()),
            ("config1", gen.config1(1000).tobytes())]
    docs += [(f"edge {i}", d) for i, d in enumerate(_edge_docs())]
    return [(name, d, oracle.parse(d)) for name, d in docs]


@pytest.mark.parametrize("variant", sorted(__import__("paper_1902_08318_gb300").ABLATIONS))
def test_variant_matches_oracle(variant, cases):
    import paper_1902_08318_gb300 as sj
    lib = sj.load_variant(variant)
    p = sj.Parser(max_bytes=max(len(d) for _, d, _ in cases) + 64, lib=lib)
    try:
        for name, d, exp in cases:
            got = gpu_result(p, np.frombuffer(d, dtype=np.uint8))
            compare(got, exp, f"{variant}: {name}")
    finally:
        p.close()
