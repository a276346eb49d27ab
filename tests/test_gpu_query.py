"""The tape query (distinct int64 values at a key path, the paper's user.id
example of Table "tab:userid") against a plain walk over the decoded
document."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _run(doc: bytes, path, max_values=1 << 16):
    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=len(doc) + 64)
    r = p.parse(np.frombuffer(doc, dtype=np.uint8))
    assert r.error == 0, r.error_name
    q = sj.Query(max_values)
    vals = q.distinct(r, path)
    got = vals.cpu().numpy().copy()
    torch.cuda.synchronize()
    assert len(got) == len(set(got.tolist())), "values must be distinct"
    return set(int(v) for v in got)


@pytest.mark.parametrize("target,users", [(631_514, 2000), (8 << 20, 50_000)])
def test_user_id_on_tweets(target, users):
    doc = gen.tweets(7, target, users).tobytes()
    exp = oracle.distinct_path_values(doc, ["user", "id"])
    assert 0 < len(exp) <= users
    assert _run(doc, ("user", "id")) == exp


def test_single_key_and_no_match():
    doc = gen.tweets(8, 200_000, 500).tobytes()
    assert _run(doc, ("id",)) == oracle.distinct_path_values(doc, ["id"])
    assert _run(doc, ("user", "nope")) == set()
    assert _run(doc, ("statuses", "id")) == set()  # statuses is an array, not an object


def test_edge_values_and_shapes():
    doc = (b'{"a":{"user":{"id":-1}},"b":[{"user":{"id":-1}},{"user":{"id":0}},'
           b'{"user":{"id":9223372036854775807}},{"user":{"id":-9223372036854775808}},'
           b'{"user":{"id":1.5}},{"user":{"id":"7"}},{"user":[{"id":3}]},{"user":{"x":{"id":4}}},'
           b'{"user":{"name":"u","id":5,"more":[1,{"id":6}]}}]}')
    exp = oracle.distinct_path_values(doc, ["user", "id"])
    assert exp == {-1, 0, 9223372036854775807, -9223372036854775808, 5}
    assert _run(doc, ("user", "id")) == exp


def test_capacity_is_reported():
    import paper_1902_08318_gb300 as sj
    doc = gen.tweets(9, 200_000, 5000).tobytes()
    with pytest.raises(sj.SJError):
        _run(doc, ("user", "id"), max_values=4)
