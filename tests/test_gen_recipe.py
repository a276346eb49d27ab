"""The synthetic inputs against the recipe they are meant to follow (the
workload configurations: sizes, value ranges, string and nesting structure,
batch size distributions, serving arrivals and mix), measured on the
generated bytes with Python's json module and plain byte counts."""
import collections
import json
import re

import numpy as np
import pytest

import gen
import oracle

STR = re.compile(rb'"((?:[^"\\]|\\.)*)"')


def _walk(x, depth, out):
    """Collect keys, scalar values and container depths (root container = 1)."""
    if isinstance(x, dict):
        out["depth"] = max(out["depth"], depth)
        for k, v in x.items():
            out["keys"].append(k)
            _walk(v, depth + 1, out)
    elif isinstance(x, list):
        out["depth"] = max(out["depth"], depth)
        for v in x:
            _walk(v, depth + 1, out)
    else:
        out["scalars"].append(x)


def _sig_digits(lexeme: bytes) -> int:
    m = re.split(rb"[eE]", lexeme)[0].lstrip(b"-").replace(b".", b"").lstrip(b"0")
    return len(m)


def test_config0_records():
    d = gen.config0(0).tobytes()
    assert len(d) >= 65536
    assert oracle.parse(d)["error"] == oracle.SUCCESS
    out = {"keys": [], "scalars": [], "depth": 0}
    _walk(json.loads(d), 1, out)
    assert isinstance(json.loads(d), dict)
    assert out["depth"] <= 6
    assert all(3 <= len(k) <= 12 and k.isascii() for k in out["keys"])
    sc = out["scalars"]
    for lit in (True, False, None):
        share = sum(1 for v in sc if v is lit) / len(sc)
        assert 0.03 < share < 0.09, (lit, share)
    ints = [v for v in sc if isinstance(v, int) and not isinstance(v, bool)]
    assert ints and all(-10**9 <= v <= 10**9 for v in ints)
    doubles = re.findall(rb"[:\[,]\s*(-?\d+\.\d+(?:[eE][-+]?\d+)?|-?\d+[eE][-+]?\d+)", d)
    sd = [_sig_digits(x) for x in doubles]
    assert min(sd) >= 1 and max(sd) <= 17
    # 5% of string characters are escape sequences: about half of the value
    # strings (0-40 characters) hold one
    vals = re.findall(rb'"((?:[^"\\]|\\.)*)"\s*[,\]\}\n]', d)
    esc = sum(1 for s in vals if b"\\" in s) / len(vals)
    assert 0.35 < esc < 0.75, esc
    assert all((len(l) - len(l.lstrip(b" "))) % 2 == 0 for l in d.split(b"\n"))


def test_config1_polygons():
    d = gen.config1(1000).tobytes()
    assert 2_500_000 <= len(d) <= 2_500_000 + 300 * 48  # within one polygon of 2.5 MB
    assert b" " not in d and b"\n" not in d
    o = json.loads(d)
    polys = o["coordinates"]
    assert all(50 <= len(p) <= 300 for p in polys)
    lon = [q[0] for p in polys for q in p]
    lat = [q[1] for p in polys for q in p]
    assert max(map(abs, lon)) <= 180 and max(map(abs, lat)) <= 90
    nums = re.findall(rb"-?\d+\.\d+(?:[eE][-+]?\d+)?", d)
    expo = [x for x in nums if b"e" in x or b"E" in x]
    assert 0.005 < len(expo) / len(nums) < 0.015
    # 15-17 significant digits (a coordinate below 1 in magnitude writes its
    # fraction's leading zeros, which are not significant)
    big = [x for x in nums if not x.lstrip(b"-").startswith(b"0.")]
    assert all(15 <= _sig_digits(x) <= 17 for x in big)


def test_config2_sample():
    d = gen.config2(2000, size=4 << 20).tobytes()
    assert oracle.parse(d)["error"] == oracle.SUCCESS
    assert d.lstrip().startswith(b"[")
    vals = re.findall(rb'"((?:[^"\\]|\\.)*)"\s*[,\]\}\n]', d)
    total = sum(len(s) for s in vals)
    nonascii = sum(sum(1 for c in s if c >= 0x80) for s in vals)
    assert 0.22 < nonascii / total < 0.32, nonascii / total  # of the bytes of string values
    leads = collections.Counter()
    for s in vals:
        for c in s:
            if 0xC0 <= c <= 0xDF:
                leads[2] += 1
            elif 0xE0 <= c <= 0xEF:
                leads[3] += 1
            elif c >= 0xF0:
                leads[4] += 1
    n = sum(leads.values())
    for k, want in ((2, 0.5), (3, 0.3), (4, 0.2)):
        assert abs(leads[k] / n - want) < 0.03, (k, leads[k] / n)
    assert re.search(rb"\\u[dD][89abAB][0-9a-fA-F]{2}\\u[dD][c-fC-F][0-9a-fA-F]{2}", d)
    depth = deepest = 0
    inside = escaped = False
    for b in d:
        if inside:
            if escaped:
                escaped = False
            elif b == 0x5C:
                escaped = True
            elif b == 0x22:
                inside = False
        elif b == 0x22:
            inside = True
        elif b in (0x5B, 0x7B):
            depth += 1
            deepest = max(deepest, depth)
        elif b in (0x5D, 0x7D):
            depth -= 1
    assert deepest >= 1024


def test_config3_batch():
    n = 300
    buf, off = gen.config3(3000, n_docs=n)
    rng = np.random.Generator(np.random.PCG64(3000))
    gen._lognormal_sizes(rng, n, 2048, 1.5, 100, 1 << 20)
    bad = rng.random(n) < 0.01
    errs = oracle.parse_many_errors(buf, off)
    assert np.array_equal(errs != 0, bad)  # every injected defect is an error, nothing else is
    sizes = gen._lognormal_sizes(np.random.Generator(np.random.PCG64(7)), 20000, 2048, 1.5, 100,
                                 1 << 20)
    assert abs(np.median(sizes) / 2048 - 1) < 0.06
    assert sizes.min() >= 100 and sizes.max() <= 1 << 20
    assert abs(np.log(sizes[(sizes > 100) & (sizes < 1 << 20)]).std() - 1.5) < 0.1


def test_config4_stream():
    n = 300
    arrival, buf, off = gen.config4(4000, n_req=n)
    rng = np.random.Generator(np.random.PCG64(4000))
    gaps = rng.exponential(1.0 / 50_000.0, n)
    assert np.allclose(arrival, np.cumsum(gaps))
    gen._lognormal_sizes(rng, n, 4096, 2.0, 64, 8 << 20)
    mix = rng.random(n)
    for i in range(n):
        head = bytes(buf[int(off[i]):int(off[i]) + 24])
        if mix[i] < 0.60:
            assert head.startswith(b"{\n"), i           # records, pretty-printed
        elif mix[i] < 0.85:
            assert head.startswith(b'{"type":"MultiPolygon"'), i
        else:
            assert head.startswith(b'["'), i            # string-heavy
    big = np.random.Generator(np.random.PCG64(11))
    g = big.exponential(1.0 / 50_000.0, 20000)
    assert abs(g.mean() * 50_000.0 - 1) < 0.03
    sizes = gen._lognormal_sizes(big, 20000, 4096, 2.0, 64, 8 << 20)
    assert abs(np.median(sizes) / 4096 - 1) < 0.08
    assert sizes.min() >= 64 and sizes.max() <= 8 << 20
    m = big.random(20000)
    assert abs((m < 0.60).mean() - 0.60) < 0.02 and abs((m >= 0.85).mean() - 0.15) < 0.02
