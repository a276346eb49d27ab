"""Seeded synthetic JSON workloads shaped like the paper's data sets.

Input generation only (no parsing arithmetic); the same documents feed the
oracle and the CUDA library.  Documents are produced by ``gen/gen.c`` (compiled
with gcc on first use) from splitmix64 streams; document sizes of the batched
and serving workloads are drawn with numpy's PCG64.

Workloads (stand-ins for the paper's files, which are not reproduced):
  config0  single ~64 KB document: root object of records nested to depth <= 6,
           keys 3-12 ASCII characters, strings 0-40 characters with 5% escapes
           (including backslash runs of 1-5), int64 in [-1e9, 1e9], doubles
           with 1-17 significant digits, true/false/null 5% each, 2-space
           pretty printing (github_events / twitter-like records).
  config1  single ~2.5 MB number-heavy document: an object wrapping an array of
           polygons of 50-300 [lon, lat] pairs with 15-17 significant digits,
           1% in exponent form, minimal white space (canada.json stand-in).
  config2  single large document (default 1 GiB): a root array of config0-style
           records, ~26% of the bytes of string values non-ASCII (2/3/4-byte
           scalars 5:3:2; keys stay ASCII),
           \\u surrogate pairs, long strings and escape runs placed on 64 B,
           2 KiB and 128 KiB edges, 1% of records nested to depth 1024.
  config3  batch of documents from the config0 generator with log-normal sizes
           (median 2 KB, sigma 1.5, clipped to [100 B, 1 MB]); 1% carry one
           defect (bad UTF-8, unbalanced bracket, unterminated string, bad
           number, control character in a string).
  config4  serving stream: Poisson arrivals, log-normal sizes (median 4 KB,
           sigma 2, clipped to [64 B, 8 MB]), 60% records / 25% number-heavy /
           15% string-heavy documents.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libsjgen.so")
_lock = threading.Lock()
_lib = None

NONASCII_P = 0.137  # per character of a string value: ~26% of their bytes non-ASCII


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "gen.c")
    with _lock:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
            return _SO
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.sjg_records.restype = ctypes.c_uint64
        lib.sjg_records.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_uint64]
        lib.sjg_geo.restype = ctypes.c_uint64
        lib.sjg_geo.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64]
        lib.sjg_tweets.restype = ctypes.c_uint64
        lib.sjg_tweets.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_void_p, ctypes.c_uint64]
        lib.sjg_strings.restype = ctypes.c_uint64
        lib.sjg_strings.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                    ctypes.c_uint64]
        _lib = lib
    return _lib


def _call(fn, target: int, *args, out: np.ndarray | None = None) -> np.ndarray:
    slack = (16 << 10) + target // 8
    while True:
        cap = target + slack
        buf = out if (out is not None and out.size >= cap) else np.empty(cap, dtype=np.uint8)
        n = fn(*args, buf.ctypes.data, cap)
        if n:
            return buf[:n]
        slack *= 4


def records(seed: int, target: int, root_array: bool = False, pretty: bool = True,
            nonascii_p: float = 0.0, deep_p: float = 0.0, deep_levels: int = 1024,
            out: np.ndarray | None = None) -> np.ndarray:
    lib = _load()
    return _call(lambda *a: lib.sjg_records(seed, target, int(root_array), int(pretty),
                                            nonascii_p, deep_p, deep_levels, *a), target, out=out)


def geo(seed: int, target: int = 2_500_000) -> np.ndarray:
    lib = _load()
    return _call(lambda *a: lib.sjg_geo(seed, target, *a), target)


def strings_heavy(seed: int, target: int) -> np.ndarray:
    lib = _load()
    return _call(lambda *a: lib.sjg_strings(seed, target, *a), target)


def tweets(seed: int, target: int = 631_514, n_users: int = 2000) -> np.ndarray:
    """Twitter-like document (statuses with nested user objects): the stand-in
    for twitter.json in the user.id query of Table "tab:userid"."""
    lib = _load()
    return _call(lambda *a: lib.sjg_tweets(seed, target, n_users, *a), target)


def config0(seed: int = 0) -> np.ndarray:
    return records(seed, 65536, root_array=False, pretty=True)


def config1(seed: int = 1000) -> np.ndarray:
    return geo(seed, 2_500_000)


def config2(seed: int = 2000, size: int = 1 << 30, out: np.ndarray | None = None) -> np.ndarray:
    return records(seed, size, root_array=True, pretty=True, nonascii_p=NONASCII_P,
                   deep_p=0.01, deep_levels=1024, out=out)


def _lognormal_sizes(rng: np.random.Generator, n: int, median: float, sigma: float,
                     lo: int, hi: int) -> np.ndarray:
    s = np.exp(np.log(median) + sigma * rng.standard_normal(n))
    return np.clip(s, lo, hi).astype(np.int64)


DEFECTS = ("utf8", "bracket", "unterminated", "number", "control")


def corrupt(doc: bytes, kind: str, rng: np.random.Generator) -> bytes:
    """Apply one defect of the given kind (the expected error is the oracle's)."""
    d = bytearray(doc)
    quotes = [i for i in range(len(d)) if d[i] == 0x22]
    if kind == "utf8":
        pos = quotes[int(rng.integers(len(quotes)))] + 1 if quotes else len(d) // 2
        d[pos:pos] = bytes([int(rng.choice([0xFF, 0xC0, 0xE2, 0x80]))])
    elif kind == "bracket":
        end = len(d.rstrip())
        del d[end - 1]
    elif kind == "unterminated":
        pos = quotes[int(rng.integers(len(quotes)))] + 1 if quotes else len(d)
        d = d[:pos] + b"abc"
    elif kind == "number":
        digits = [i for i in range(1, len(d)) if chr(d[i]).isdigit() and d[i - 1] in b" :,["]
        if digits:
            pos = digits[int(rng.integers(len(digits)))]
            d[pos:pos] = b"0" if rng.random() < 0.5 else b"-x"
        else:
            d[1:1] = b"01,"
    elif kind == "control":
        pos = quotes[int(rng.integers(len(quotes)))] + 1 if quotes else 1
        d[pos:pos] = b"\x01"
    return bytes(d)


def config3(seed: int = 3000, n_docs: int = 100_000, invalid_frac: float = 0.01):
    """Returns (buf uint8, offsets uint64[n+1]) of a concatenated batch."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = _lognormal_sizes(rng, n_docs, 2048, 1.5, 100, 1 << 20)
    bad = rng.random(n_docs) < invalid_frac
    kinds = rng.integers(0, len(DEFECTS), n_docs)
    parts = []
    for i in range(n_docs):
        doc = records(seed * 1_000_003 + i, int(sizes[i]), root_array=False, pretty=True)
        b = doc.tobytes()
        if bad[i]:
            b = corrupt(b, DEFECTS[int(kinds[i])], rng)
        parts.append(b)
    lens = np.array([len(p) for p in parts], dtype=np.uint64)
    offsets = np.zeros(n_docs + 1, dtype=np.uint64)
    np.cumsum(lens, out=offsets[1:])
    return np.frombuffer(b"".join(parts), dtype=np.uint8), offsets


def _serving_docs(args) -> tuple[bytes, list[int]]:
    """Documents [lo, hi) of a serving stream (worker of config4)."""
    seed, lo, hi, sizes, mix = args
    parts = []
    for k, i in enumerate(range(lo, hi)):
        s = seed * 1_000_003 + i
        if mix[k] < 0.60:
            doc = records(s, int(sizes[k]), root_array=False, pretty=True)
        elif mix[k] < 0.85:
            doc = geo(s, int(sizes[k]))
        else:
            doc = strings_heavy(s, int(sizes[k]))
        parts.append(doc.tobytes())
    return b"".join(parts), [len(p) for p in parts]


def config4(seed: int = 4000, n_req: int = 200_000, rate: float = 50_000.0,
            max_size: int = 8 << 20, workers: int = 1):
    """Serving stream.  Returns (arrival_s float64[n], buf uint8, offsets uint64[n+1]).
    workers > 1 generates in that many processes (same bytes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, n_req)
    arrival = np.cumsum(gaps)
    sizes = _lognormal_sizes(rng, n_req, 4096, 2.0, 64, max_size)
    mix = rng.random(n_req)
    step = max(1, -(-n_req // (8 * max(1, workers))))
    jobs = [(seed, lo, min(n_req, lo + step), sizes[lo: lo + step], mix[lo: lo + step])
            for lo in range(0, n_req, step)]
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            results = pool.map(_serving_docs, jobs)
    else:
        results = [_serving_docs(j) for j in jobs]
    lens = np.array([n for _, ls in results for n in ls], dtype=np.uint64)
    offsets = np.zeros(n_req + 1, dtype=np.uint64)
    np.cumsum(lens, out=offsets[1:])
    return arrival, np.frombuffer(b"".join(b for b, _ in results), dtype=np.uint8), offsets
