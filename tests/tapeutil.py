"""Reading a tape + string buffer back into Python values (test helper).

Layout (Sec. 3, Fig. "jsontape"): 64-bit words, tag in the top byte, 56-bit
payload.  Strings: u32 little-endian length, bytes, NUL at the payload offset.
Objects decode to lists of (key, value) pairs so that duplicate keys and their
order survive; doubles decode to their IEEE bits wrapped in Dbl so that -0.0
and bit patterns compare exactly.
"""
from __future__ import annotations

import json
import struct

import numpy as np

M56 = (1 << 56) - 1


class Dbl:
    __slots__ = ("bits",)

    def __init__(self, bits: int):
        self.bits = bits

    def __eq__(self, other):
        return isinstance(other, Dbl) and other.bits == self.bits

    def __repr__(self):
        return f"Dbl({struct.unpack('<d', struct.pack('<Q', self.bits))[0]!r})"


def read_string(strings: np.ndarray, off: int) -> bytes:
    n = int(strings[off]) | int(strings[off + 1]) << 8 | int(strings[off + 2]) << 16 | int(strings[off + 3]) << 24
    body = strings[off + 4: off + 4 + n].tobytes()
    assert int(strings[off + 4 + n]) == 0, "missing NUL terminator"
    return body


def decode(tape: np.ndarray, strings: np.ndarray):
    t = [int(x) for x in tape]
    T = len(t)
    assert t[0] >> 56 == ord("r") and (t[0] & M56) == T - 1
    assert t[T - 1] >> 56 == ord("r") and (t[T - 1] & M56) == 0

    def val(i):
        tag = chr(t[i] >> 56)
        p = t[i] & M56
        if tag == '"':
            return read_string(strings, p).decode("utf-8"), i + 1
        if tag == "l":
            v = t[i + 1]
            return (v - (1 << 64) if v >> 63 else v), i + 2
        if tag == "d":
            return Dbl(t[i + 1]), i + 2
        if tag == "t":
            return True, i + 1
        if tag == "f":
            return False, i + 1
        if tag == "n":
            return None, i + 1
        if tag in "{[":
            end = p - 1
            assert chr(t[end] >> 56) == ("}" if tag == "{" else "]")
            assert (t[end] & M56) == i
            items = []
            j = i + 1
            while j < end:
                if tag == "{":
                    k, j = val(j)
                    assert isinstance(k, str)
                    v, j = val(j)
                    items.append((k, v))
                else:
                    v, j = val(j)
                    items.append(v)
            assert j == end
            return (items if tag == "[" else ("obj", items)), end + 1
        raise AssertionError(f"bad tag {tag!r} at {i}")

    v, j = val(1)
    assert j == T - 1
    return v


def py_expected(text: bytes):
    """json.loads with the same shapes as decode(): objects as ("obj", pairs),
    floats as Dbl bits."""

    def fl(s):
        return Dbl(struct.unpack("<Q", struct.pack("<d", float(s)))[0])

    return json.loads(text.decode("utf-8"), object_pairs_hook=lambda p: ("obj", list(p)),
                      parse_float=fl)


def fix_lists(v):
    """json returns lists for arrays and our tuples for objects; normalise."""
    if isinstance(v, tuple) and len(v) == 2 and v[0] == "obj":
        return ("obj", [(k, fix_lists(x)) for k, x in v[1]])
    if isinstance(v, list):
        return [fix_lists(x) for x in v]
    return v
