"""Continuous-batching server (sj_server_* through the C ABI): every request's
result is the same as when its document is parsed alone, and matches the
oracle; admission follows the device-memory budget; results stay on the
device until released."""
import numpy as np
import pytest

import gen
import oracle
from tests.gpuutil import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _mix(n, seed):
    """Serving-style mix: records / number-heavy / string-heavy documents of
    log-normal sizes, a few with one defect."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.clip(np.exp(rng.normal(np.log(2048), 1.5, n)), 64, 200_000).astype(int)
    docs = []
    for i in range(n):
        s = seed * 1_000_003 + i
        u = rng.random()
        if u < 0.6:
            d = gen.records(s, int(sizes[i]), root_array=False, pretty=True).tobytes()
        elif u < 0.85:
            d = gen.geo(s, int(sizes[i])).tobytes()
        else:
            d = gen.strings_heavy(s, int(sizes[i])).tobytes()
        if rng.random() < 0.05:
            d = gen.corrupt(d, gen.DEFECTS[int(rng.integers(0, len(gen.DEFECTS)))], rng)
        docs.append(d)
    return docs


def _fetch(c):
    """Host copy of one completion's outputs (device pointers into the slot)."""
    import paper_1902_08318_gb300 as sj
    out = {"error": int(c["error"]), "n_indices": int(c["n_indices"])}
    ni = int(c["n_indices"])
    out["indices"] = (sj.Parser.view(int(c["indices"]), ni, "<u4").cpu().numpy().copy()
                      if ni else np.zeros(0, np.uint32))
    if out["error"] == 0:
        out["tape"] = sj.Parser.view(int(c["tape"]), int(c["tape_words"]), "<u8").cpu().numpy().copy()
        out["strings"] = sj.Parser.view(int(c["strings"]), int(c["string_bytes"]),
                                        "|u1").cpu().numpy().copy()
    torch.cuda.synchronize()
    return out


def _alone(parser, d):
    r = parser.parse(np.frombuffer(d, dtype=np.uint8))
    out = {"error": r.error, "n_indices": r.n_indices}
    out["indices"] = r.indices().cpu().numpy().copy() if r.n_indices else np.zeros(0, np.uint32)
    if r.error == 0:
        out["tape"] = r.tape().cpu().numpy().copy()
        out["strings"] = r.strings().cpu().numpy().copy()
    torch.cuda.synchronize()
    return out


def test_each_result_same_alone_and_in_the_mix():
    import paper_1902_08318_gb300 as sj
    docs = _mix(600, 41)
    # small batches and several slots: many batches overlap on the GPU
    srv = sj.Server(max_batch_bytes=256 << 10, max_batch_docs=64, max_slots=4, mem_budget=0)
    assert srv.slots == 4
    tickets = {}
    got = {}
    i = 0
    while len(got) < len(docs):
        # requests arrive while earlier batches are still on the GPU
        for _ in range(7):
            if i < len(docs):
                tickets[srv.submit(docs[i])] = i
                i += 1
        for c in srv.poll():
            got[tickets[int(c["ticket"])]] = _fetch(c)
            srv.release(int(c["ticket"]))
    assert srv.batches > 4
    alone = sj.Parser(max_bytes=256 << 10)
    for k, d in enumerate(docs):
        a = _alone(alone, d)
        compare(got[k], a, f"doc {k} in the mix vs alone")
        if k % 10 == 0:  # and against the oracle
            compare(got[k], oracle.parse(d), f"doc {k} vs oracle")


def test_admission_follows_the_memory_budget():
    import paper_1902_08318_gb300 as sj
    # a slot's device memory (its parsers), as the server counts it
    probe = sj.Server(max_batch_bytes=1 << 20, max_batch_docs=16, max_slots=1, mem_budget=0)
    one = probe.device_bytes
    probe.close()
    assert one >= sj.Parser(max_bytes=1 << 20, max_docs=16).device_bytes()
    srv = sj.Server(max_batch_bytes=1 << 20, max_batch_docs=16, max_slots=8,
                    mem_budget=int(2.5 * one))
    assert srv.slots == 2
    assert srv.device_bytes <= 2.5 * one
    with pytest.raises(sj.SJError):
        sj.Server(max_batch_bytes=1 << 20, max_batch_docs=16, max_slots=8, mem_budget=one // 2)


def test_results_stay_resident_until_released():
    import paper_1902_08318_gb300 as sj
    srv = sj.Server(max_batch_bytes=64 << 10, max_batch_docs=1, max_slots=2, mem_budget=0)
    docs = [b'{"a": [1, 2.5, "x"]}', b'[true, null]', b'"s"', b'{"k": {}}']
    t = [srv.submit(d) for d in docs]
    held = []
    for _ in range(10000):
        held += list(srv.poll())
        if len(held) == 2:
            break
    assert len(held) == 2  # both slots hold an unreleased result
    for _ in range(200):
        assert len(srv.poll()) == 0  # nothing else can start until a release
    first = {int(c["ticket"]): _fetch(c) for c in held}
    srv.release(int(held[0]["ticket"]))
    more = []
    for _ in range(10000):
        more += list(srv.poll())
        if more:
            break
    assert len(more) == 1
    # the still-held result is intact after another batch ran in the freed slot
    keep = int(held[1]["ticket"])
    again = _fetch(held[1])
    assert np.array_equal(again["tape"], first[keep]["tape"])
    for k, c in first.items():
        compare(c, oracle.parse(docs[t.index(k)]), f"resident {k}")


def test_replay_latencies():
    import paper_1902_08318_gb300 as sj
    docs = _mix(300, 43)
    buf = np.frombuffer(b"".join(docs), dtype=np.uint8)
    off = np.zeros(len(docs) + 1, dtype=np.uint64)
    np.cumsum([len(d) for d in docs], out=off[1:])
    arrival = np.cumsum(np.full(len(docs), 1e-4))
    srv = sj.Server(max_batch_bytes=1 << 20, max_batch_docs=256, max_slots=4, mem_budget=0)
    lat, wall = srv.replay(buf, off, arrival)
    assert np.all(lat > 0) and np.all(np.isfinite(lat))
    assert wall >= arrival[-1]
