// strings.cuh -- string validation and normalisation on the device (Sec. 3.2.2).
//
// A string starts after its opening quote and ends at the first quote that is
// not escaped.  Raw bytes below 0x20 are errors (UNESCAPED_CHARS); escapes are
// \" \\ \/ \b \f \n \r \t and \uXXXX (hex digits in either case), where a high
// surrogate must be followed by \u and a low surrogate and the pair becomes one
// code point; any other escape, or a lone surrogate, is a STRING_ERROR.  Other
// bytes (already validated as UTF-8 by stage 1) are copied.  The first problem
// in byte order decides the code.
#pragma once
#include <stdint.h>

#include "sj.h"

namespace sj {

__device__ __forceinline__ int hex4(const uint8_t *p, const uint8_t *lim, uint32_t &v) {
  if (p + 4 > lim) return 0;
  uint32_t r = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    uint32_t c = p[k], h;
    if (c >= '0' && c <= '9') h = c - '0';
    else if ((c | 0x20) >= 'a' && (c | 0x20) <= 'f') h = (c | 0x20) - 'a' + 10;
    else return 0;
    r = (r << 4) | h;
  }
  v = r;
  return 1;
}

__device__ __forceinline__ uint32_t utf8_len(uint32_t cp) {
  return cp < 0x80 ? 1u : (cp < 0x800 ? 2u : (cp < 0x10000 ? 3u : 4u));
}

__device__ __forceinline__ void utf8_put(uint8_t *o, uint32_t cp) {
  if (cp < 0x80) { o[0] = (uint8_t)cp; }
  else if (cp < 0x800) { o[0] = (uint8_t)(0xC0 | (cp >> 6)); o[1] = (uint8_t)(0x80 | (cp & 63)); }
  else if (cp < 0x10000) {
    o[0] = (uint8_t)(0xE0 | (cp >> 12)); o[1] = (uint8_t)(0x80 | ((cp >> 6) & 63));
    o[2] = (uint8_t)(0x80 | (cp & 63));
  } else {
    o[0] = (uint8_t)(0xF0 | (cp >> 18)); o[1] = (uint8_t)(0x80 | ((cp >> 12) & 63));
    o[2] = (uint8_t)(0x80 | ((cp >> 6) & 63)); o[3] = (uint8_t)(0x80 | (cp & 63));
  }
}

// Does a 32-bit word hold a quote, a backslash or a byte below 0x20?
__device__ __forceinline__ bool special4(uint32_t x) {
  uint32_t q = x ^ 0x22222222u, b = x ^ 0x5C5C5C5Cu;
  uint32_t zq = (q - 0x01010101u) & ~q;
  uint32_t zb = (b - 0x01010101u) & ~b;
  uint32_t lt = (x - 0x20202020u) & ~x;  // bytes < 0x20 (may also flag some bytes >= 0x80)
  return ((zq | zb | lt) & 0x80808080u) != 0;
}

// Walk the string whose content starts at s (just after the opening quote);
// `lim` bounds the search.  Returns the normalised length; err is 0,
// SJ_STRING_ERROR or SJ_UNESCAPED_CHARS.  With WRITE the bytes go to out.
template <bool WRITE>
__device__ __forceinline__ uint32_t string_walk(const uint8_t *s, const uint8_t *lim, int &err,
                                                uint8_t *out) {
  uint32_t n = 0;
  const uint8_t *p = s;
  err = 0;
  for (;;) {
    // plain runs, 4 bytes at a time: aligned word loads realigned with a
    // funnel shift (a word holding a byte before `lim` lies in a page the
    // document uses)
    if (p + 4 <= lim) {
      const uintptr_t ua = (uintptr_t)p;
      const uint32_t *wp = reinterpret_cast<const uint32_t *>(ua & ~(uintptr_t)3);
      const uint32_t sh = (uint32_t)(ua & 3) * 8;
      uint32_t lo = sh ? wp[0] : 0u;  // holds byte p
      while (p + 4 <= lim) {
        uint32_t x, hi = 0;
        if (sh) {
          hi = wp[1];  // holds byte p + 3
          x = __funnelshift_r(lo, hi, sh);
        } else {
          x = wp[0];
        }
        if (special4(x)) break;
        if (WRITE) {
          out[n] = (uint8_t)x; out[n + 1] = (uint8_t)(x >> 8);
          out[n + 2] = (uint8_t)(x >> 16); out[n + 3] = (uint8_t)(x >> 24);
        }
        n += 4;
        p += 4;
        wp++;
        lo = hi;
      }
    }
    if (p >= lim) { err = SJ_STRING_ERROR; return n; }
    uint8_t c = *p;
    if (c == '"') return n;
    if (c == '\\') {
      if (p + 1 >= lim) { err = SJ_STRING_ERROR; return n; }
      uint8_t e = p[1];
      uint8_t o;
      switch (e) {
        case '"': o = '"'; break;
        case '\\': o = '\\'; break;
        case '/': o = '/'; break;
        case 'b': o = '\b'; break;
        case 'f': o = '\f'; break;
        case 'n': o = '\n'; break;
        case 'r': o = '\r'; break;
        case 't': o = '\t'; break;
        case 'u': {
          uint32_t cu;
          if (!hex4(p + 2, lim, cu)) { err = SJ_STRING_ERROR; return n; }
          p += 6;
          if (cu >= 0xDC00 && cu <= 0xDFFF) { err = SJ_STRING_ERROR; return n; }
          if (cu >= 0xD800 && cu <= 0xDBFF) {
            uint32_t lo;
            if (p + 1 >= lim || p[0] != '\\' || p[1] != 'u' || !hex4(p + 2, lim, lo) ||
                lo < 0xDC00 || lo > 0xDFFF) {
              err = SJ_STRING_ERROR;
              return n;
            }
            p += 6;
            cu = 0x10000 + ((cu - 0xD800) << 10) + (lo - 0xDC00);
          }
          if (WRITE) utf8_put(out + n, cu);
          n += utf8_len(cu);
          continue;
        }
        default: err = SJ_STRING_ERROR; return n;
      }
      if (WRITE) out[n] = o;
      n++;
      p += 2;
      continue;
    }
    if (c < 0x20) { err = SJ_UNESCAPED_CHARS; return n; }
    if (WRITE) out[n] = c;
    n++;
    p++;
  }
}

}  // namespace sj

namespace sj {

// Bytes of an 8-byte window that are a quote, a backslash or below 0x20: bit
// 7 of each byte, exact for the lowest flagged byte (a borrow can only flag
// bytes above a flagged one).
__device__ __forceinline__ uint32_t special_bits(uint32_t x) {
  const uint32_t q = x ^ 0x22222222u, b = x ^ 0x5C5C5C5Cu;
  return (((q - 0x01010101u) & ~q) | ((b - 0x01010101u) & ~b) | ((x - 0x20202020u) & ~x)) &
         0x80808080u;
}

// string_walk with the same results (length, error, output bytes), shaped for
// many strings walked side by side in one warp: every step copies the plain
// bytes of an 8-byte window up to the first special byte and then handles at
// most that one byte (end, error or one escape sequence), so lanes walking
// different strings stay in step instead of splitting between a copy loop and
// escape handling.
template <bool WRITE>
__device__ __forceinline__ uint32_t string_walk8(const uint8_t *s, const uint8_t *lim, int &err,
                                                 uint8_t *out) {
  uint32_t n = 0;
  const uint8_t *p = s;
  err = 0;
  for (;;) {
    if (p >= lim) { err = SJ_STRING_ERROR; return n; }
    // window [p, p + 8): aligned words (a word holding a byte before lim lies
    // in a page the document uses), bytes at or past lim forced to a quote
    const uintptr_t ua = (uintptr_t)p;
    const uint32_t *wp = reinterpret_cast<const uint32_t *>(ua & ~(uintptr_t)3);
    const uint32_t sh = (uint32_t)(ua & 3) * 8;
    const uint32_t w0 = wp[0];
    const uint32_t w1 = reinterpret_cast<const uint8_t *>(wp + 1) < lim ? wp[1] : 0x22222222u;
    const uint32_t w2 = reinterpret_cast<const uint8_t *>(wp + 2) < lim ? wp[2] : 0x22222222u;
    uint32_t lo = __funnelshift_r(w0, w1, sh), hi = __funnelshift_r(w1, w2, sh);
    const intptr_t avail = lim - p;
    if (avail < 8) {
      const uint64_t keep = (1ull << (8 * avail)) - 1;  // avail in [1, 7]
      const uint64_t x = (((uint64_t)hi << 32) | lo) & keep;
      const uint64_t y = x | (0x2222222222222222ull & ~keep);
      lo = (uint32_t)y;
      hi = (uint32_t)(y >> 32);
    }
    const uint32_t fl = special_bits(lo), fh = special_bits(hi);
    const uint32_t k = fl ? (uint32_t)(__ffs(fl) - 1) >> 3 : (fh ? 4u + ((uint32_t)(__ffs(fh) - 1) >> 3) : 8u);
    if (WRITE) {
#pragma unroll
      for (uint32_t i = 0; i < 8; i++)
        if (i < k) out[n + i] = (uint8_t)((i < 4 ? lo >> (8 * i) : hi >> (8 * (i - 4))) & 0xFFu);
    }
    n += k;
    p += k;
    if (k == 8) continue;
    if (p >= lim) { err = SJ_STRING_ERROR; return n; }
    const uint32_t c = (k < 4 ? lo >> (8 * k) : hi >> (8 * (k - 4))) & 0xFFu;
    if (c == '"') return n;
    if (c != '\\') { err = SJ_UNESCAPED_CHARS; return n; }  // a byte below 0x20
    if (p + 1 >= lim) { err = SJ_STRING_ERROR; return n; }
    const uint32_t e = p[1];
    if (e != 'u') {
      uint32_t o;
      switch (e) {
        case '"': o = '"'; break;
        case '\\': o = '\\'; break;
        case '/': o = '/'; break;
        case 'b': o = '\b'; break;
        case 'f': o = '\f'; break;
        case 'n': o = '\n'; break;
        case 'r': o = '\r'; break;
        case 't': o = '\t'; break;
        default: err = SJ_STRING_ERROR; return n;
      }
      if (WRITE) out[n] = (uint8_t)o;
      n++;
      p += 2;
      continue;
    }
    uint32_t cu;
    if (!hex4(p + 2, lim, cu)) { err = SJ_STRING_ERROR; return n; }
    p += 6;
    if (cu >= 0xDC00 && cu <= 0xDFFF) { err = SJ_STRING_ERROR; return n; }
    if (cu >= 0xD800 && cu <= 0xDBFF) {
      uint32_t lo2;
      if (p + 1 >= lim || p[0] != '\\' || p[1] != 'u' || !hex4(p + 2, lim, lo2) || lo2 < 0xDC00 ||
          lo2 > 0xDFFF) {
        err = SJ_STRING_ERROR;
        return n;
      }
      p += 6;
      cu = 0x10000 + ((cu - 0xD800) << 10) + (lo2 - 0xDC00);
    }
    if (WRITE) utf8_put(out + n, cu);
    n += utf8_len(cu);
  }
}

}  // namespace sj
