"""Writes pow5_table.h: 128-bit truncated significands of 5^q, q in [-342, 308].

For each q the table holds M(q) = floor(5^q * 2^b) with b chosen so that
2^127 <= M(q) < 2^128, and the binary exponent e(q) = -b, so that
5^q = (M(q) + d) * 2^e(q) with 0 <= d < 1 (d = 0 exactly when 0 <= q <= 55).
Exact big-integer arithmetic (Python ints); run from this directory:
    python gen_pow5_table.py
"""
Q_MIN, Q_MAX = -342, 308


def entry(q: int):
    if q >= 0:
        v = 5 ** q
        L = v.bit_length()
        if L <= 128:
            m = v << (128 - L)
        else:
            m = v >> (L - 128)
        e = L - 128
    else:
        d = 5 ** (-q)
        L = d.bit_length()
        m = (1 << (127 + L)) // d
        e = -(127 + L)
    assert (1 << 127) <= m < (1 << 128), q
    return m >> 64, m & ((1 << 64) - 1), e


def main():
    lines = [
        "/* Generated by gen_pow5_table.py -- do not edit.",
        " * 5^q = (hi:lo + d) * 2^e with 0 <= d < 1, q in [SJ_POW5_QMIN, SJ_POW5_QMAX]. */",
        "#pragma once",
        "#include <stdint.h>",
        f"#define SJ_POW5_QMIN ({Q_MIN})",
        f"#define SJ_POW5_QMAX ({Q_MAX})",
        "static __device__ const uint64_t sj_pow5_hi[] = {",
    ]
    ents = [entry(q) for q in range(Q_MIN, Q_MAX + 1)]
    for i in range(0, len(ents), 3):
        lines.append("  " + ", ".join(f"0x{h:016x}ull" for h, _, _ in ents[i:i + 3]) + ",")
    lines.append("};")
    lines.append("static __device__ const uint64_t sj_pow5_lo[] = {")
    for i in range(0, len(ents), 3):
        lines.append("  " + ", ".join(f"0x{l:016x}ull" for _, l, _ in ents[i:i + 3]) + ",")
    lines.append("};")
    lines.append("static __device__ const int16_t sj_pow5_e[] = {")
    for i in range(0, len(ents), 12):
        lines.append("  " + ", ".join(str(e) for _, _, e in ents[i:i + 12]) + ",")
    lines.append("};")
    with open("pow5_table.h", "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
