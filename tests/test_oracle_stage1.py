"""Pins of the oracle's stage-1 definition (Sec. 3.1) to what the paper prints.

1. The literal mask transcription (tests/masks.py) reproduces every bitmask row
   printed for the 64-byte worked example (Figs. "identifyescapedquotes",
   "identifyquoteregion", "identifypseudo").
2. The oracle's byte-at-a-time scan gives the same final index set.
3. Brute force: the oracle and the transcription agree on every input of 1..7
   bytes over an 8-symbol alphabet, and on random multi-block inputs rich in
   backslash runs and quotes (carries across 64-byte blocks).
4. The classification of Sec. 3.1.2 equals the printed nibble tables for all
   256 byte values.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from tests import masks
from tests.conftest import GOLDEN


def _load_fig():
    rows = {}
    inp = None
    for line in open(os.path.join(GOLDEN, "paper_fig_masks.txt"), encoding="utf-8"):
        if line.startswith("#") or not line.strip():
            continue
        if line.startswith("input "):
            inp = line[len("input "):].rstrip("\n").encode()
            continue
        g, name, bits = line.split()
        rows[(g, name)] = sum(1 << i for i, ch in enumerate(bits) if ch == "1")
    return inp, rows


def test_golden_input_is_64_bytes():
    inp, rows = _load_fig()
    assert len(inp) == 64
    assert len(rows) == 28


def test_escape_rows_match_paper():
    inp, rows = _load_fig()
    B = masks.byte_mask(inp, lambda c: c == 0x5C)
    assert B == rows[("escape", "B")]
    assert masks.EVEN == rows[("escape", "E")]
    assert masks.ODD == rows[("escape", "O")]
    esc = masks.escape_sequence(B)
    for name in ("S", "ES", "EC", "ECE", "OD1", "OS", "OC", "OCE", "OD2", "OD"):
        assert esc[name] == rows[("escape", name)], name


def test_quote_rows_match_paper():
    inp, rows = _load_fig()
    B = masks.byte_mask(inp, lambda c: c == 0x5C)
    Qa = masks.byte_mask(inp, lambda c: c == 0x22)
    assert Qa == rows[("quote", "Q_all")]
    OD = masks.escape_sequence(B)["OD"]
    assert OD == rows[("quote", "OD")]
    Q = Qa & ~OD & masks.M64
    assert Q == rows[("quote", "Q")]
    assert masks.prefix_xor(Q) == rows[("quote", "R")]


def test_pseudo_rows_match_paper():
    inp, rows = _load_fig()
    Q, R = rows[("pseudo", "Q")], rows[("pseudo", "R")]
    Sc = masks.byte_mask(inp, lambda c: masks.classify_table(c) & 7)
    W = masks.byte_mask(inp, lambda c: masks.classify_table(c) & 0x18)
    assert Sc == rows[("pseudo", "S_class")]
    assert W == rows[("pseudo", "W")]
    ps = masks.pseudo_sequence(Q, R, Sc, W, prev_sep=0)
    # The printed shifted row has bit 0 clear: the figure shows one block with
    # no predecessor carried in; byte 0 is '{', already structural.
    for name in ("S_outside", "S_or_Q", "P_sw", "P_shift", "P", "S_or_P", "FINAL"):
        assert ps[name] == rows[("pseudo", name)], name


def test_oracle_indices_match_paper_example():
    inp, rows = _load_fig()
    final = rows[("pseudo", "FINAL")]
    expect = [i for i in range(64) if (final >> i) & 1]
    idx, unclosed = oracle.stage1(inp)
    assert list(idx) == expect
    assert expect == [0, 2, 13, 15, 17, 20, 21, 28, 30, 33, 35, 41, 43, 49, 50, 52, 55, 56, 63]
    assert not unclosed


def test_classification_matches_nibble_tables():
    lines = [l.split() for l in open(os.path.join(GOLDEN, "vectable.txt")) if not l.startswith("#")]
    low = [int(x) for x in lines[0][1:]]
    high = [int(x) for x in lines[1][1:]]
    assert low == masks.LOW_NIBBLE and high == masks.HIGH_NIBBLE
    for c in range(256):
        assert oracle.classify(c) == (low[c & 15] & high[c >> 4]), hex(c)


ALPHABET = b'"\\,:[{a '


def _vector_single_block(recs: np.ndarray):
    """The transcription on arrays of single-block records (n, w<=64)."""
    n, w = recs.shape

    def bm(pred):
        m = np.zeros(n, dtype=np.uint64)
        for i in range(w):
            m |= pred(recs[:, i]).astype(np.uint64) << np.uint64(i)
        return m

    tab = np.array([masks.classify_table(c) for c in range(256)], dtype=np.uint8)
    B = bm(lambda c: c == 0x5C)
    Qa = bm(lambda c: c == 0x22)
    Sc = bm(lambda c: (tab[c] & 7) != 0)
    W = bm(lambda c: (tab[c] & 0x18) != 0)
    # padding bytes beyond w are white space
    pad = np.uint64(((1 << 64) - 1) ^ ((1 << w) - 1))
    W = W | pad
    esc = masks.escape_sequence(B)
    Q = Qa & ~esc["OD"]
    R = masks.prefix_xor(Q)
    ps = masks.pseudo_sequence(Q, R, Sc, W, 1)
    final = ps["FINAL"]
    out = np.zeros((n, w), dtype=bool)
    for i in range(w):
        out[:, i] = ((final >> np.uint64(i)) & np.uint64(1)) != 0
    unclosed = ((R >> np.uint64(63)) & np.uint64(1)) != 0
    return out, unclosed


@pytest.mark.parametrize("w", [1, 2, 3, 4, 5, 6, 7])
def test_bruteforce_short_inputs(w):
    alpha = np.frombuffer(ALPHABET, dtype=np.uint8)
    idx = np.indices((len(alpha),) * w).reshape(w, -1).T
    recs = alpha[idx]
    got, got_uc = oracle.stage1_many(recs)
    exp, exp_uc = _vector_single_block(recs)
    bad = np.nonzero((got != exp).any(axis=1) | (got_uc != exp_uc))[0]
    assert bad.size == 0, recs[bad[0]].tobytes()


def test_random_multiblock_inputs():
    rng = np.random.Generator(np.random.PCG64(7))
    # heavy in backslashes and quotes so that runs and strings cross edges
    pool = np.frombuffer(b'\\\\\\\\""' + ALPHABET + b"01tx\n", dtype=np.uint8)
    for _ in range(1500):
        n = int(rng.integers(60, 330))
        data = pool[rng.integers(0, len(pool), n)].tobytes()
        if rng.random() < 0.3:  # a long backslash run across a 64-byte edge
            k = int(rng.integers(1, min(n, 140)))
            s = int(rng.integers(0, n - k + 1))
            data = data[:s] + b"\\" * k + data[s + k:]
        exp, exp_uc = masks.stage1_masks(data)
        got, got_uc = oracle.stage1(data)
        assert list(got) == exp, data
        assert got_uc == exp_uc, data


def test_all_backslash_block_carries_parity():
    # 1 + 64 + 63 backslashes then a quote: the quote is escaped iff the run is odd
    for pre in range(0, 4):
        for run in (63, 64, 65, 127, 128, 129):
            data = b"a" * pre + b'"' + b"\\" * run + b'"x"'
            exp, exp_uc = masks.stage1_masks(data)
            got, got_uc = oracle.stage1(data)
            assert list(got) == exp and got_uc == exp_uc
