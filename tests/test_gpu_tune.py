"""Launch shapes and the autotuner: any shape gives the same bit-exact result
(the kernels loop over tiles), and the tuner picks shapes within the limits."""
import numpy as np
import pytest

import gen
from tests import gpuutil

pytestmark = pytest.mark.gpu


def _outputs(p, doc):
    return gpuutil.gpu_result(p, doc)


def test_every_shape_gives_the_same_result():
    import paper_1902_08318_gb300 as sj
    docs = [gen.config0(0), gen.config1(1000), gen.config2(2000, size=3 << 20)]
    p = sj.Parser(max_bytes=4 << 20)
    lim = {k: m for k, (c, m) in p.launch().items()}
    assert all(m >= 1 for m in lim.values())
    ref = [_outputs(p, d) for d in docs]
    for shape in ([1, 1, 1, 1], [lim[k] for k in sj.TUNED_KERNELS],
                  [max(1, lim[k] // 2) for k in sj.TUNED_KERNELS]):
        p.set_launch(shape)
        assert [c for c, _ in p.launch().values()] == shape
        for d, r in zip(docs, ref):
            gpuutil.compare(_outputs(p, d), r, f"shape {shape}")
    with pytest.raises(sj.SJError):
        p.set_launch([0, 1, 1, 1])
    with pytest.raises(sj.SJError):
        p.set_launch([lim["s1_blocks"] + 1, 1, 1, 1])


def test_autotune_picks_valid_shapes_and_keeps_results():
    import paper_1902_08318_gb300 as sj
    doc = gen.config2(2001, size=8 << 20)
    p = sj.Parser(max_bytes=9 << 20)
    before = _outputs(p, doc)
    rep = p.autotune(doc)
    cur = p.launch()
    for k in sj.TUNED_KERNELS:
        assert 1 <= rep[k]["blocks_per_sm"] <= cur[k][1]
        assert cur[k][0] == rep[k]["blocks_per_sm"]
        assert rep[k]["ms"] > 0
    gpuutil.compare(_outputs(p, doc), before, "after autotune")


def test_prepare_then_batches_of_every_size():
    # sj_parser_prepare captures the run of every batch-size bucket up front;
    # later batches of any size (up to max_docs) replay them
    import oracle
    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=1 << 20, max_docs=40)
    p.prepare()
    p.prepare(8)  # again, and a smaller bound: nothing to capture
    pool = [b'{"a": [1, 2.5, "x"]}', b"[true, null, -0]", b'"s\\n"', b"[1,", b"tru",
            gen.config0(7).tobytes()[:3000]]
    for n in (1, 2, 3, 17, 40):
        docs = [pool[i % len(pool)] for i in range(n)]
        buf, off = gpuutil.batch_arrays(docs)
        res, _ = p.parse_batch(buf, off)
        assert [int(e) for e in res["error"]] == [oracle.parse(d)["error"] for d in docs]
