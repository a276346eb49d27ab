"""Pins of the oracle's UTF-8 check (Sec. 3.1.5, Table "tab:unicode").

The independent reference is Python's strict utf-8 codec, a library routine
implementing the same well-formedness table (RFC 3629).  Coverage: every 1-,
2- and 3-byte sequence (all 16.7 million of the latter); 4-byte sequences with
every 4-byte lead (F0-F7), every second and third byte and the fourth byte's
range boundaries, and every lead from C0 with every second byte and class
representatives for the last two; random mixed strings; the paper's rejected
example 0xb1 0x87.

Python's decoder is run over many records at once: each record is followed
by a newline (ASCII, so no sequence spans two records) and the buffer is
decoded with errors="surrogateescape", which turns every byte it cannot decode
into one code point U+DC80-U+DCFF (a code point that valid UTF-8 cannot
encode); a record is valid exactly when none of its code points is one.
"""
import os

import numpy as np

import oracle
from tests.conftest import GOLDEN

# One representative per behaviour class of a trailing byte: ASCII, the
# continuation sub-ranges that the lead-specific rules split on, and non-continuations.
REPS = np.array([0x00, 0x41, 0x7F, 0x80, 0x8F, 0x90, 0x9F, 0xA0, 0xBF, 0xC0, 0xC1, 0xC2,
                 0xDF, 0xE0, 0xED, 0xEF, 0xF0, 0xF4, 0xF5, 0xFF], dtype=np.uint8)


def _python_valid(recs: np.ndarray) -> np.ndarray:
    out = np.empty(recs.shape[0], dtype=bool)
    for i, r in enumerate(recs):
        try:
            r.tobytes().decode("utf-8", "strict")
            out[i] = True
        except UnicodeDecodeError:
            out[i] = False
    return out


def _python_valid_bulk(recs: np.ndarray) -> np.ndarray:
    """Python's strict verdict on each record, many records per decode."""
    n, w = recs.shape
    out = np.ones(n, dtype=bool)
    step = 1 << 18
    for lo in range(0, n, step):
        part = recs[lo: lo + step]
        m = part.shape[0]
        buf = np.empty((m, w + 1), dtype=np.uint8)
        buf[:, :w] = part
        buf[:, w] = 0x0A
        text = buf.tobytes().decode("utf-8", "surrogateescape")
        cp = np.frombuffer(text.encode("utf-32-le", "surrogatepass"), dtype=np.uint32)
        esc = (cp >= 0xDC80) & (cp <= 0xDCFF)
        nbytes = np.where(cp < 0x80, 1, np.where(cp < 0x800, 2, np.where(cp < 0x10000, 3, 4)))
        nbytes[esc] = 1
        start = np.cumsum(nbytes) - nbytes
        bad = np.zeros(m, dtype=bool)
        bad[start[esc] // (w + 1)] = True
        out[lo: lo + m] = ~bad
    return out


def test_bulk_reference_agrees_with_per_record_decoding():
    rng = np.random.Generator(np.random.PCG64(5))
    for w in (1, 2, 3, 4, 6):
        recs = rng.integers(0, 256, size=(3000, w), dtype=np.uint8)
        recs[::3, 0] = rng.integers(0xC2, 0xF5, size=recs[::3].shape[0], dtype=np.uint8)
        recs[::3, 1:] = rng.integers(0x80, 0xC0, size=recs[::3, 1:].shape, dtype=np.uint8)
        assert (_python_valid_bulk(recs) == _python_valid(recs)).all()


def test_all_one_and_two_byte_sequences():
    one = np.arange(256, dtype=np.uint8).reshape(-1, 1)
    assert (oracle.utf8_valid_many(one) == _python_valid(one)).all()
    two = np.indices((256, 256)).reshape(2, -1).T.astype(np.uint8)
    assert (oracle.utf8_valid_many(two) == _python_valid(two)).all()


def test_every_three_byte_sequence():
    for lead in range(256):  # 65,536 records per lead
        b, c = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
        recs = np.stack([np.full(b.size, lead), b.ravel(), c.ravel()], axis=1).astype(np.uint8)
        got = oracle.utf8_valid_many(recs)
        exp = _python_valid_bulk(recs)
        assert (got == exp).all(), (lead, recs[np.nonzero(got != exp)[0][:3]])


def test_four_byte_sequences():
    # every 4-byte lead, every second and third byte, the fourth byte's boundaries
    fourth = np.array([0x00, 0x41, 0x7F, 0x80, 0x8F, 0x90, 0x9F, 0xA0, 0xBF, 0xC0, 0xF4, 0xFF],
                      dtype=np.uint8)
    for lead in range(0xF0, 0xF8):
        b, c, d = np.meshgrid(np.arange(256), np.arange(256), fourth, indexing="ij")
        recs = np.stack([np.full(b.size, lead), b.ravel(), c.ravel(), d.ravel()],
                        axis=1).astype(np.uint8)
        assert (oracle.utf8_valid_many(recs) == _python_valid_bulk(recs)).all(), lead
    # every lead from C0, every second byte, representatives for the last two
    a, b, c, d = np.meshgrid(np.arange(0xC0, 256), np.arange(256), REPS, REPS, indexing="ij")
    recs = np.stack([a.ravel(), b.ravel(), c.ravel(), d.ravel()], axis=1).astype(np.uint8)
    assert (oracle.utf8_valid_many(recs) == _python_valid_bulk(recs)).all()


def test_random_strings():
    rng = np.random.Generator(np.random.PCG64(11))
    samples = ["aé€𝄞", "ÿ", "日本語テキスト", "߿ࠀ￿\U00010000\U0010ffff"]
    for _ in range(3000):
        s = "".join(samples[int(rng.integers(len(samples)))] for _ in range(int(rng.integers(1, 6))))
        b = bytearray(s.encode())
        if rng.random() < 0.5:
            b[int(rng.integers(len(b)))] = int(rng.integers(0x80, 256))
        if rng.random() < 0.2:
            b = b[: int(rng.integers(len(b)))]
        try:
            bytes(b).decode("utf-8")
            ok = True
        except UnicodeDecodeError:
            ok = False
        assert oracle.utf8_valid(bytes(b)) == ok, bytes(b)


def test_paper_rejected_sequence():
    # Sec. 4.1: a parser accepting 0xb1 0x87 does only partial validation
    assert not oracle.utf8_valid(b"\xb1\x87")
    assert oracle.parse(b'["\xb1\x87"]')["error"] == oracle.UTF8_ERROR


def test_cascade_example_and_lengths():
    """Sec. 3.1.5 printed example of the continuation-count steps; on valid
    strings the final value of each byte is the number of bytes left in its
    code point, so leads carry their sequence length as the oracle decodes."""
    rows = {}
    for line in open(os.path.join(GOLDEN, "utf8_cascade.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        rows[k] = [int(x) for x in v]

    def step(v, k):
        shifted = [0] * k + v[:-k]
        return [a + max(s - k, 0) for a, s in zip(v, shifted)]

    s1 = step(rows["classes"], 1)
    assert s1 == rows["step1"]
    assert step(s1, 2) == rows["step2"]
    for text in ["aé€𝄞z", "𝄞𝄞", "€a€", "߿￿\U0010ffff"]:
        b = text.encode()
        assert oracle.utf8_valid(b)
        cls = []
        for x in b:
            if x < 0x80:
                cls.append(1)
            elif x < 0xC0:
                cls.append(0)
            elif x < 0xE0:
                cls.append(2)
            elif x < 0xF0:
                cls.append(3)
            else:
                cls.append(4)
        fin = step(step(cls, 1), 2)
        remaining = []
        for ch in text:
            n = len(ch.encode())
            remaining += list(range(n, 0, -1))
        assert fin == remaining
