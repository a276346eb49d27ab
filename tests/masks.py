"""A literal transcription of the stage-1 mask sequences of Sec. 3.1.

Used only as an independent pin of the oracle's byte-at-a-time stage-1 scan:
the per-block steps follow Figs. "identifyescapedquotes", "identifyquoteregion"
and "identifypseudo" operation by operation on 64-bit integers (bit i = byte i
of the block).  The paper elides the carries between blocks (footnote in
Sec. 3.1.1); the carries used here are the reading stated in the design notes:
the parity of a backslash run reaching the end of a block, the in-string
parity, and the last bit of (S | Q | W); before byte 0 a virtual white-space
byte.
"""
from __future__ import annotations

M64 = (1 << 64) - 1
EVEN = 0x5555555555555555  # "E": bits at even offsets
ODD = 0xAAAAAAAAAAAAAAAA   # "O": bits at odd offsets

# Sec. 3.1.2 nibble tables, as printed (tests/golden/vectable.txt).
LOW_NIBBLE = [16, 0, 0, 0, 0, 0, 0, 0, 0, 8, 10, 4, 1, 12, 0, 0]
HIGH_NIBBLE = [8, 0, 17, 2, 0, 4, 0, 4, 0, 0, 0, 0, 0, 0, 0, 0]


def classify_table(c: int) -> int:
    return LOW_NIBBLE[c & 15] & HIGH_NIBBLE[c >> 4]


def byte_mask(block: bytes, pred) -> int:
    m = 0
    for i, c in enumerate(block):
        if pred(c):
            m |= 1 << i
    return m


def prefix_xor(q: int) -> int:
    """CLMUL(Q, ~0): bit i = XOR of bits 0..i (Fig. "identifyquoteregion")."""
    r = q
    for i in range(1, 64):
        r = r ^ ((q << i) & M64)
    return r


def escape_sequence(B: int, carry_odd: int = 0) -> dict:
    """Fig. "identifyescapedquotes"; with carry_odd the first run continues an
    odd-length run of the previous block (its start is treated as odd)."""
    c0 = carry_odd & 1
    S = B & ~(B << 1) & M64
    ES = S & EVEN & (M64 ^ c0)
    EC = (B + ES) & M64
    ECE = EC & ~B & M64
    OD1 = ECE & (M64 ^ EVEN)  # ECE & ~E
    OS = S & (ODD | c0)
    OC = (B + OS) & M64
    OCE = OC & ~B & M64
    OD2 = OCE & EVEN
    OD = OD1 | OD2 | (c0 & ~B & 1)
    return dict(B=B, S=S, ES=ES, EC=EC, ECE=ECE, OD1=OD1, OS=OS, OC=OC, OCE=OCE, OD2=OD2, OD=OD)


def escape_carry_out(B: int, carry_odd: int) -> int:
    if B == M64:
        return carry_odd  # 64 more backslashes keep the parity
    t = 0
    while t < 64 and (B >> (63 - t)) & 1:
        t += 1
    return t & 1


def pseudo_sequence(Q: int, R: int, S_class: int, W: int, prev_sep: int) -> dict:
    """Fig. "identifypseudo"; prev_sep is bit 63 of the previous block's S|W."""
    S1 = S_class & ~R & M64
    S2 = S1 | Q
    P0 = S2 | W
    P1 = ((P0 << 1) | (prev_sep & 1)) & M64
    P2 = P1 & ~W & ~R & M64
    S3 = S2 | P2
    final = S3 & ~(Q & ~R & M64) & M64
    return dict(S_outside=S1, S_or_Q=S2, P_sw=P0, P_shift=P1, P=P2, S_or_P=S3, FINAL=final)


def stage1_masks(data: bytes):
    """Run the three sequences over 64-byte blocks with carries.  Returns
    (sorted index list, unclosed flag)."""
    out = []
    carry_odd, in_str, prev_sep = 0, 0, 1
    for base in range(0, len(data), 64):
        blk = data[base:base + 64]
        blk = blk + b" " * (64 - len(blk))  # padding: white space, never indexed
        B = byte_mask(blk, lambda c: c == 0x5C)
        Qa = byte_mask(blk, lambda c: c == 0x22)
        Sc = byte_mask(blk, lambda c: classify_table(c) & 0x7)
        W = byte_mask(blk, lambda c: classify_table(c) & 0x18)
        esc = escape_sequence(B, carry_odd)
        Q = Qa & ~esc["OD"] & M64
        R = prefix_xor(Q) ^ (M64 if in_str else 0)
        ps = pseudo_sequence(Q, R, Sc, W, prev_sep)
        f = ps["FINAL"]
        for i in range(64):
            if (f >> i) & 1 and base + i < len(data):
                out.append(base + i)
        carry_odd = escape_carry_out(B, carry_odd)
        in_str = (R >> 63) & 1
        prev_sep = (ps["P_sw"] >> 63) & 1
    return out, bool(in_str)
