// number.cuh -- JSON number validation and conversion on the device (Sec. 3.2.1).
//
// Grammar (RFC 8259 as restated in Sec. 3): -?(0|[1-9][0-9]*)(.[0-9]+)?([eE][+-]?[0-9]+)?
// followed by white space, one of ",:[]{}", or the end of the document.
// Integers (no fraction, no exponent) must lie in [-2^63, 2^63) and are kept
// exactly; everything else becomes the binary64 value nearest to the decimal
// (ties to even).  An infinite result is an error; underflow is not.
//
// Conversion of a decimal w * 10^q (w < 10^19):
//  1. Clinger's fast path when w <= 2^53 and |q| <= 22: one correctly rounded
//     IEEE multiplication or division of two exact doubles.
//  2. Otherwise w (normalised to 64 bits) times a 128-bit truncated
//     significand of 5^q (table from gen_pow5_table.py) gives a 192-bit P with
//     the true scaled value V in [P, P + w).  The rounding decision is read
//     from P whenever that whole interval falls on one side of the rounding
//     midpoint (the idea of Eisel and Lemire, "Number parsing at a gigabyte
//     per second", 2021, with an explicit interval test).
//  3. When the interval straddles the midpoint, or more than 19 significant
//     digits were given, the two nearest midpoints are compared with the exact
//     decimal using big-integer arithmetic (at most 800 significant digits are
//     kept, the rest only as a "non-zero tail" flag: a binary64 midpoint has at
//     most 767 significant decimal digits, so that flag decides exactly).
#pragma once
#include <stdint.h>

#include "pow5_table.h"
#include "sj.h"

namespace sj {

__device__ __forceinline__ bool is_digit(uint8_t c) { return (uint8_t)(c - '0') < 10; }

// White space or ",:[]{}": the bytes that may follow an atom or a number.
__device__ __forceinline__ bool is_terminator(uint8_t c) {
  return c == ' ' || c == '\n' || c == '\r' || c == '\t' || c == ',' || c == ':' || c == ']' ||
         c == '}' || c == '[' || c == '{';
}

// Eight ASCII bytes (little-endian in v) that are all decimal digits: every
// high nibble is 3 and adding 6 to every byte leaves it so (low nibble <= 9).
// The high-nibble test rules out bytes >= 0xF0, so the addition cannot carry
// from one byte into the next.  (Sec. 3.2.1 checks eight digits at once.)
__device__ __forceinline__ bool eight_digits(uint64_t v) {
  const uint64_t hi = 0xF0F0F0F0F0F0F0F0ull, threes = 0x3030303030303030ull;
  return (v & hi) == threes && ((v + 0x0606060606060606ull) & hi) == threes;
}

// Value of eight digits, first digit in the lowest byte: neighbouring digits
// are combined into 2-, then 4-, then 8-digit numbers with one multiply and
// one shift per step.
__device__ __forceinline__ uint32_t eight_digit_value(uint64_t v) {
  v -= 0x3030303030303030ull;
  v = (v * 10 + (v >> 8)) & 0x00FF00FF00FF00FFull;
  v = (v * 100 + (v >> 16)) & 0x0000FFFF0000FFFFull;
  return (uint32_t)((v * 10000 + (v >> 32)) & 0xFFFFFFFFull);
}

__device__ __forceinline__ uint64_t load8(const uint8_t *p) {
  uint64_t v = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) v |= (uint64_t)p[k] << (8 * k);
  return v;
}

// ---------------------------------------------------------------------------
// Exact comparison of a decimal with H * 2^g (big integers, rare path).
// ---------------------------------------------------------------------------
namespace bigcmp {
constexpr int LIMBS = 168;  // 5376 bits, enough for 800 digits scaled by 2^2200

struct Big {
  uint32_t v[LIMBS];
  int n;  // used limbs
};

__device__ __noinline__ void set_u64(Big &a, uint64_t x) {
  a.v[0] = (uint32_t)x;
  a.v[1] = (uint32_t)(x >> 32);
  a.n = a.v[1] ? 2 : (a.v[0] ? 1 : 0);
}

__device__ __noinline__ void mul_add_small(Big &a, uint32_t m, uint32_t add) {
  uint64_t carry = add;
  for (int i = 0; i < a.n; i++) {
    uint64_t t = (uint64_t)a.v[i] * m + carry;
    a.v[i] = (uint32_t)t;
    carry = t >> 32;
  }
  if (carry && a.n < LIMBS) a.v[a.n++] = (uint32_t)carry;
}

__device__ __noinline__ void mul_pow5(Big &a, int k) {
  while (k >= 13) { mul_add_small(a, 1220703125u, 0); k -= 13; }  // 5^13
  uint32_t m = 1;
  while (k-- > 0) m *= 5;
  if (m != 1) mul_add_small(a, m, 0);
}

__device__ __noinline__ void shl(Big &a, int bits) {
  if (a.n == 0 || bits <= 0) return;
  int limbs = bits >> 5, b = bits & 31;
  int nn = a.n + limbs + 1;
  if (nn > LIMBS) nn = LIMBS;
  for (int i = nn - 1; i >= 0; i--) {
    int src = i - limbs;
    uint32_t hi = (src >= 0 && src < a.n) ? a.v[src] : 0;
    uint32_t lo = (src - 1 >= 0 && src - 1 < a.n) ? a.v[src - 1] : 0;
    a.v[i] = b ? ((hi << b) | (lo >> (32 - b))) : hi;
  }
  a.n = nn;
  while (a.n > 0 && a.v[a.n - 1] == 0) a.n--;
}

__device__ __noinline__ int cmp(const Big &a, const Big &b) {
  if (a.n != b.n) return a.n < b.n ? -1 : 1;
  for (int i = a.n - 1; i >= 0; i--)
    if (a.v[i] != b.v[i]) return a.v[i] < b.v[i] ? -1 : 1;
  return 0;
}

// Compare the decimal lexeme [s, e) (validated; sign ignored) with H * 2^g.
__device__ __noinline__ int decimal_vs(const uint8_t *s, const uint8_t *e, uint64_t H, int g) {
  Big A, B;
  A.n = 0;
  int64_t q = 0;
  int nd = 0;
  bool sticky = false, frac = false;
  uint32_t chunk = 0, chunk_mul = 1;
  const uint8_t *p = s;
  if (p < e && *p == '-') p++;
  for (; p < e; p++) {
    uint8_t c = *p;
    if (c == '.') { frac = true; continue; }
    if (c == 'e' || c == 'E') break;
    uint32_t d = c - '0';
    if (nd == 0 && d == 0) { if (frac) q--; continue; }  // leading zeros
    if (nd < 800) {
      chunk = chunk * 10 + d;
      chunk_mul *= 10;
      nd++;
      if (frac) q--;
      if (chunk_mul == 1000000000u) { mul_add_small(A, chunk_mul, chunk); chunk = 0; chunk_mul = 1; }
    } else {
      if (d) sticky = true;
      if (!frac) q++;
    }
  }
  if (chunk_mul != 1) mul_add_small(A, chunk_mul, chunk);
  if (p < e && (*p == 'e' || *p == 'E')) {
    p++;
    bool neg = false;
    if (p < e && (*p == '+' || *p == '-')) { neg = *p == '-'; p++; }
    int64_t x = 0;
    for (; p < e && is_digit(*p); p++) if (x < 100000000) x = x * 10 + (*p - '0');
    q += neg ? -x : x;
  }
  set_u64(B, H);
  if (q >= 0) mul_pow5(A, (int)q); else mul_pow5(B, (int)-q);
  if (q >= g) shl(A, (int)(q - g)); else shl(B, (int)(g - q));
  int c = cmp(A, B);
  if (c == 0 && sticky) c = 1;
  return c;
}

}  // namespace bigcmp

__device__ const double kPow10[23] = {1e0,  1e1,  1e2,  1e3,  1e4,  1e5,  1e6,  1e7,
                                      1e8,  1e9,  1e10, 1e11, 1e12, 1e13, 1e14, 1e15,
                                      1e16, 1e17, 1e18, 1e19, 1e20, 1e21, 1e22};

// ---------------------------------------------------------------------------
// Binary64 encoding helpers.
// ---------------------------------------------------------------------------
// Encode mantissa r at unit 2^e_unit; returns false on overflow to infinity.
__device__ __forceinline__ bool encode(uint64_t r, int e_unit, bool normal, uint64_t &bits) {
  if (!normal) {  // unit 2^-1074; r <= 2^52 (2^52 is the smallest normal)
    bits = r;
    return true;
  }
  if (r >= (1ull << 53)) { r >>= 1; e_unit += 1; }
  int E = e_unit + 52;
  if (E > 1023) return false;
  bits = ((uint64_t)(E + 1023) << 52) | (r & ((1ull << 52) - 1));
  return true;
}

// Decide among m, m+1, m+2 by exact comparison with the two midpoints above m.
__device__ __noinline__ bool slow_round(const uint8_t *s, const uint8_t *e, uint64_t m, int e_unit,
                                        bool normal, uint64_t &bits) {
  uint64_t r;
  int c1 = bigcmp::decimal_vs(s, e, 2 * m + 1, e_unit - 1);
  if (c1 < 0) r = m;
  else if (c1 == 0) r = (m & 1) ? m + 1 : m;
  else if (normal && m + 1 == (1ull << 53)) r = m + 1;
  else {
    int c2 = bigcmp::decimal_vs(s, e, 2 * m + 3, e_unit - 1);
    if (c2 < 0) r = m + 1;
    else if (c2 == 0) r = ((m + 1) & 1) ? m + 2 : m + 1;
    else r = m + 2;
  }
  return encode(r, e_unit, normal, bits);
}

// w * 10^q, w != 0, w < 10^19.  `force_slow` when digits were dropped.
// Returns false on overflow to infinity.
__device__ __forceinline__ bool decimal_to_double(uint64_t w, int64_t q, bool force_slow,
                                                  const uint8_t *s, const uint8_t *e,
                                                  uint64_t &bits) {
  // 1. Clinger's fast path: both operands exact, one IEEE rounding.
  if (!force_slow && w <= (1ull << 53) && q >= -22 && q <= 22) {
    double d = (double)w;  // exact
    d = q < 0 ? __ddiv_rn(d, kPow10[-q]) : __dmul_rn(d, kPow10[q]);
    bits = (uint64_t)__double_as_longlong(d);
    return true;
  }
  if (q < SJ_POW5_QMIN) { bits = 0; return true; }  // below half the smallest subnormal
  if (q > SJ_POW5_QMAX) return false;                // at least 1e309
  // 2. 192-bit product with the truncated 5^q significand.
  int lz = __clzll((long long)w);
  uint64_t wn = w << lz;
  int qi = (int)q - SJ_POW5_QMIN;
  uint64_t mh = sj_pow5_hi[qi], ml = sj_pow5_lo[qi];
  int e5 = sj_pow5_e[qi];
  uint64_t a_lo = wn * ml, a_hi = __umul64hi(wn, ml);
  uint64_t b_lo = wn * mh, b_hi = __umul64hi(wn, mh);
  uint64_t p0 = a_lo;
  uint64_t p1 = a_hi + b_lo;
  uint64_t p2 = b_hi + (p1 < a_hi ? 1 : 0);
  int LP = (p2 >> 63) ? 191 : 190;
  int s0 = e5 + (int)q - lz;  // V = Vscaled * 2^s0, Vscaled in [P, P + wn)
  int E = LP + s0;
  bool normal = E >= -1022;
  int u = normal ? LP - 52 : -1074 - s0;  // bit of P holding the mantissa's last bit
  if (u > 192) { bits = 0; return true; }  // below half the smallest subnormal
  if (normal && E > 1023) return false;
  int sh = u - 128;  // in [10, 64]
  uint64_t lowmask = sh >= 64 ? ~0ull : ((1ull << sh) - 1);
  uint64_t m = sh >= 64 ? 0 : (p2 >> sh);
  uint64_t t2 = p2 & lowmask;                 // t = bits of P below position u
  uint64_t h2 = 1ull << (sh - 1);             // half = 2^(u-1)
  int e_unit = u + s0;
  if (force_slow) return slow_round(s, e, m, e_unit, normal, bits);
  bool exact = (q >= 0 && q <= 55);
  bool t_gt = (t2 > h2) || (t2 == h2 && (p1 | p0) != 0);
  bool t_eq = (t2 == h2) && ((p1 | p0) == 0);
  bool up;
  if (exact) {
    up = t_gt || (t_eq && (m & 1));
  } else if (t_gt || t_eq) {
    up = true;  // V > P >= midpoint
  } else {
    // t < half: does t + wn reach past the midpoint?
    uint64_t s0w = p0 + wn;
    uint64_t c0 = s0w < p0 ? 1 : 0;
    uint64_t s1w = p1 + c0;
    uint64_t c1 = (c0 && s1w == 0) ? 1 : 0;
    uint64_t s2w = t2 + c1;
    bool over = (s2w > h2) || (s2w == h2 && (s1w | s0w) != 0);
    if (over) return slow_round(s, e, m, e_unit, normal, bits);
    up = false;
  }
  return encode(m + (up ? 1 : 0), e_unit, normal, bits);
}

// Validate and convert the number starting at s (document ends at end).
// Returns SJ_SUCCESS and sets tag ('l' or 'd') and the value word, or
// SJ_NUMBER_ERROR.
__device__ __forceinline__ int parse_number(const uint8_t *s, const uint8_t *end, uint8_t &tag,
                                            uint64_t &value) {
  const uint8_t *p = s;
  bool neg = false;
  if (p < end && *p == '-') { neg = true; p++; }
  if (p >= end || !is_digit(*p)) return SJ_NUMBER_ERROR;
  uint64_t w = 0;
  int nw = 0;
  int64_t qa = 0;
  bool dropped = false;
  bool is_int = true;
  if (*p == '0') {
    p++;
  } else {
    // the first digit is 1-9, so w > 0 from here on and every digit counts
    while (nw + 8 <= 19 && p + 8 <= end) {
      const uint64_t v = load8(p);
      if (!eight_digits(v)) break;
      w = w * 100000000ull + eight_digit_value(v);
      nw += 8;
      p += 8;
    }
    while (p < end && is_digit(*p)) {
      uint32_t d = *p - '0';
      if (nw < 19) { w = w * 10 + d; nw++; }
      else { qa++; if (d) dropped = true; }
      p++;
    }
  }
  if (p < end && *p == '.') {
    is_int = false;
    p++;
    if (p >= end || !is_digit(*p)) return SJ_NUMBER_ERROR;
    while (w != 0 && nw + 8 <= 19 && p + 8 <= end) {
      const uint64_t v = load8(p);
      if (!eight_digits(v)) break;
      w = w * 100000000ull + eight_digit_value(v);
      nw += 8;
      qa -= 8;
      p += 8;
    }
    while (p < end && is_digit(*p)) {
      uint32_t d = *p - '0';
      if (nw < 19) {
        if (w == 0 && d == 0) qa--;
        else { w = w * 10 + d; nw++; qa--; }
      } else if (d) {
        dropped = true;
      }
      p++;
    }
  }
  int64_t ex = 0;
  if (p < end && (*p == 'e' || *p == 'E')) {
    is_int = false;
    p++;
    bool eneg = false;
    if (p < end && (*p == '+' || *p == '-')) { eneg = *p == '-'; p++; }
    if (p >= end || !is_digit(*p)) return SJ_NUMBER_ERROR;
    while (p < end && is_digit(*p)) {
      if (ex < 100000000) ex = ex * 10 + (*p - '0');
      p++;
    }
    if (eneg) ex = -ex;
  }
  if (p < end && !is_terminator(*p)) return SJ_NUMBER_ERROR;
  if (is_int) {
    if (qa > 0) return SJ_NUMBER_ERROR;  // 20 or more integer digits
    if (neg ? (w > (1ull << 63)) : (w > (1ull << 63) - 1)) return SJ_NUMBER_ERROR;
    tag = 'l';
    value = neg ? (uint64_t)0 - w : w;
    return SJ_SUCCESS;
  }
  tag = 'd';
  uint64_t bits;
  if (w == 0) {  // digits are counted from the first non-zero one: all zeros
    bits = 0;
  } else if (!decimal_to_double(w, qa + ex, dropped, s, p, bits)) {
    return SJ_NUMBER_ERROR;
  }
  value = bits | (neg ? (1ull << 63) : 0);
  return SJ_SUCCESS;
}

}  // namespace sj
