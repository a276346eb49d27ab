// s1_common.cuh -- building blocks of stage 1 (Sec. 3.1) shared by its kernels:
// SWAR classification of 64-byte blocks, the odd-backslash and in-string masks,
// block loading, and the UTF-8 check.
#pragma once
#include "sj_internal.cuh"

namespace sj {

// Compile-time variants for the measurements of "Effect of Specific
// Optimizations" (Table "tab:optimization"): each replaces one optimised step
// of stage 1 by its plain form and computes the same result.  None is set in
// the library; a variant build defines one of them.
//   SJ_ABL_PREFIX_XOR_LOOP    in-string mask by the definition of the
//                             carry-less product with all ones (one XOR of a
//                             shifted all-ones word per quote) instead of the
//                             shift-XOR ladder
//   SJ_ABL_QUOTE_PARITY_SHFL  quote parity of the earlier lanes by a
//                             five-step shuffle XOR scan instead of a ballot
//                             and a popcount
//   SJ_ABL_COMPARE_CLASSIFY   classification by one byte comparison per
//                             character instead of the nibble tables
//   SJ_ABL_UTF8_ALWAYS        the UTF-8 check on every block, ASCII or not
//   SJ_ABL_NAIVE_FLATTEN      each lane stores its block's indices to global
//                             memory one by one instead of staging them in
//                             shared memory for coalesced stores

// ---------------------------------------------------------------------------
// Classification (Sec. 3.1.2): two 16-entry nibble tables whose AND gives the
// class bits of a byte.  Own tables (the paper's layout, different bits):
//   bit0 ','  bit1 ':'  bit2 '[' ']' '{' '}'  bit3 '\t' '\n' '\r'  bit4 ' '
//   bit5 '"'  bit6 '\\'
// Each set is exactly the product of its low- and high-nibble sets.
// ---------------------------------------------------------------------------
constexpr uint32_t kLoA0 = 0x00200010u, kLoA1 = 0x00000000u;  // low nibble 0..7
constexpr uint32_t kLoB0 = 0x040A0800u, kLoB1 = 0x00000C41u;  // low nibble 8..15
constexpr uint32_t kHi0 = 0x02310008u, kHi1 = 0x04004400u;    // high nibble 0..7 (8..15 -> 0)

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
  return r;
}

// Four nibbles (bits 0-3 of each byte of n) packed into a 16-bit prmt selector.
__device__ __forceinline__ uint32_t nibble_selector(uint32_t n) {
  return prmt(n | (n >> 4), 0u, 0x4420u);
}

// Class byte of each of the 4 bytes of x.  A selector nibble with bit 3 set
// makes prmt replicate the sign of the chosen table byte, i.e. give 0 (all
// table bytes are < 0x80): that selects between the two halves of the
// low-nibble table and zeroes high nibbles 8..15.
__device__ __forceinline__ uint32_t classify4(uint32_t x) {
  uint32_t sl = nibble_selector(x & 0x0F0F0F0Fu);
  uint32_t sh = nibble_selector((x >> 4) & 0x0F0F0F0Fu);
  uint32_t lo = prmt(kLoA0, kLoA1, sl) | prmt(kLoB0, kLoB1, sl ^ 0x8888u);
  uint32_t hi = prmt(kHi0, kHi1, sh);
  return lo & hi;
}

// Bit 7 of each byte -> 4 contiguous bits.
__device__ __forceinline__ uint32_t movemask4(uint32_t m80) {
  return ((m80 >> 7) * 0x01020408u) >> 24;
}

struct BlockMasks {
  uint64_t bs, quote, op, ws;
  uint32_t nonascii;  // OR of all words & 0x80808080
};

// Bit 7 set in each byte of x equal to c (exact: the low seven bits are
// added without a carry into the next byte).
__device__ __forceinline__ uint32_t eq_bytes(uint32_t x, uint32_t c) {
  const uint32_t t = x ^ (c * 0x01010101u);
  return ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t | 0x7F7F7F7Fu);
}

#ifdef SJ_ABL_COMPARE_CLASSIFY
// The plain classification the paper compares with: one comparison per
// structural and white-space character, ORed together.
__device__ __forceinline__ void classify_block(const uint32_t (&w)[16], BlockMasks &m) {
  uint32_t bs[2] = {0, 0}, qu[2] = {0, 0}, op[2] = {0, 0}, ws[2] = {0, 0};
  uint32_t na = 0;
#pragma unroll
  for (int j = 0; j < 16; j++) {
    const uint32_t x = w[j];
    na |= x;
    const int h = j >> 3, s = (j & 7) * 4;
    op[h] |= movemask4(eq_bytes(x, ',') | eq_bytes(x, ':') | eq_bytes(x, '[') | eq_bytes(x, ']') |
                       eq_bytes(x, '{') | eq_bytes(x, '}')) << s;
    ws[h] |= movemask4(eq_bytes(x, ' ') | eq_bytes(x, '\t') | eq_bytes(x, '\n') |
                       eq_bytes(x, '\r')) << s;
    qu[h] |= movemask4(eq_bytes(x, '"')) << s;
    bs[h] |= movemask4(eq_bytes(x, '\\')) << s;
  }
  m.bs = ((uint64_t)bs[1] << 32) | bs[0];
  m.quote = ((uint64_t)qu[1] << 32) | qu[0];
  m.op = ((uint64_t)op[1] << 32) | op[0];
  m.ws = ((uint64_t)ws[1] << 32) | ws[0];
  m.nonascii = na & 0x80808080u;
}
#else
__device__ __forceinline__ void classify_block(const uint32_t (&w)[16], BlockMasks &m) {
  uint32_t bs[2] = {0, 0}, qu[2] = {0, 0}, op[2] = {0, 0}, ws[2] = {0, 0};
  uint32_t na = 0;
#pragma unroll
  for (int j = 0; j < 16; j++) {
    uint32_t v = classify4(w[j]);
    na |= w[j];
    const int h = j >> 3, s = (j & 7) * 4;
    op[h] |= movemask4(((v & 0x07070707u) + 0x7F7F7F7Fu) & 0x80808080u) << s;
    ws[h] |= movemask4(((v & 0x18181818u) + 0x78787878u) & 0x80808080u) << s;
    qu[h] |= movemask4((v << 2) & 0x80808080u) << s;
    bs[h] |= movemask4((v << 1) & 0x80808080u) << s;
  }
  m.bs = ((uint64_t)bs[1] << 32) | bs[0];
  m.quote = ((uint64_t)qu[1] << 32) | qu[0];
  m.op = ((uint64_t)op[1] << 32) | op[0];
  m.ws = ((uint64_t)ws[1] << 32) | ws[0];
  m.nonascii = na & 0x80808080u;
}
#endif

// Bytes below 0x20 of a block (exact per byte: with the top three bits kept,
// a byte is zero exactly when it was a control character).
__device__ __forceinline__ uint64_t ctrl_mask(const uint32_t (&w)[16]) {
  uint32_t r[2] = {0, 0};
#pragma unroll
  for (int j = 0; j < 16; j++) {
    const uint32_t t = w[j] & 0xE0E0E0E0u;
    const uint32_t z = ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t | 0x7F7F7F7Fu);
    r[j >> 3] |= movemask4(z) << ((j & 7) * 4);
  }
  return ((uint64_t)r[1] << 32) | r[0];
}

// ---------------------------------------------------------------------------
// Fig. "identifyescapedquotes": bytes that follow an odd-length backslash run,
// assuming no run is carried in.  The carried-in case differs only at the
// first non-backslash byte (see first_non_bs).
// ---------------------------------------------------------------------------
constexpr uint64_t kEven = 0x5555555555555555ull, kOdd = 0xAAAAAAAAAAAAAAAAull;

__device__ __forceinline__ uint64_t escaped_no_carry(uint64_t b) {
  uint64_t starts = b & ~(b << 1);
  uint64_t even_ends = (b + (starts & kEven)) & ~b;  // first byte after each even-start run
  uint64_t odd_ends = (b + (starts & kOdd)) & ~b;    // first byte after each odd-start run
  return (even_ends & kOdd) | (odd_ends & kEven);
}

// With an odd run carried in, the run at byte 0 has odd length where it would
// have even length without the carry, and vice versa: the escape status of
// the first non-backslash byte flips.
__device__ __forceinline__ uint64_t first_non_bs(uint64_t b) {
  uint64_t nb = ~b;
  return nb & (~nb + 1);  // lowest clear bit of b (0 when b is all ones)
}

#ifdef SJ_ABL_PREFIX_XOR_LOOP
// The carry-less product of x with an all-ones word, by its definition: every
// set bit b of x adds (XOR) the all-ones word shifted left by b.
__device__ __forceinline__ uint64_t prefix_xor(uint64_t x) {
  uint64_t r = 0;
  while (x) {
    r ^= ~0ull << (__ffsll((long long)x) - 1);
    x &= x - 1;
  }
  return r;
}
#else
__device__ __forceinline__ uint64_t prefix_xor(uint64_t x) {
  x ^= x << 1;
  x ^= x << 2;
  x ^= x << 4;
  x ^= x << 8;
  x ^= x << 16;
  x ^= x << 32;
  return x;
}
#endif

// ---------------------------------------------------------------------------
// Loading a block of a document (bytes beyond the document become spaces).
// Every loaded 16-byte chunk is 16-byte aligned and holds at least one byte of
// the document, so a load never crosses into a page the document does not use.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mask_tail(uint32_t v, int64_t valid) {
  // keep the first `valid` bytes (0..4) of v, the rest become ' '
  if (valid >= 4) return v;
  if (valid <= 0) return 0x20202020u;
  uint32_t keep = (1u << (8 * valid)) - 1;
  return (v & keep) | (0x20202020u & ~keep);
}

template <int WS>  // word shift: (address & 15) / 4
__device__ __forceinline__ void realign(const uint32_t (&c)[20], int bs8, uint32_t (&w)[16]) {
#pragma unroll
  for (int j = 0; j < 16; j++) {
    uint32_t lo = c[j + WS], hi = c[j + WS + 1];
    w[j] = bs8 ? __funnelshift_r(lo, hi, bs8) : lo;
  }
}

__device__ __forceinline__ void load_block(const uint8_t *doc, uint64_t len, uint64_t start,
                                           uint32_t (&w)[16]) {
  const uint8_t *a = doc + start;
  uintptr_t ua = (uintptr_t)a;
  if ((ua & 15) == 0 && start + 64 <= len) {
    const uint4 *p = reinterpret_cast<const uint4 *>(a);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      uint4 v = __ldg(p + k);
      w[4 * k + 0] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
    }
    return;
  }
  // General path: aligned 16-byte chunks covering [a, a+64), realigned.
  const uintptr_t doc_end = (uintptr_t)doc + len;
  const uintptr_t a0 = ua & ~(uintptr_t)15;
  uint32_t c[20];
#pragma unroll
  for (int k = 0; k < 5; k++) {
    uintptr_t ca = a0 + 16 * k;
    uint4 v = make_uint4(0x20202020u, 0x20202020u, 0x20202020u, 0x20202020u);
    if (ca < doc_end && ca + 16 > ua) v = __ldg(reinterpret_cast<const uint4 *>(ca));
    c[4 * k + 0] = v.x; c[4 * k + 1] = v.y; c[4 * k + 2] = v.z; c[4 * k + 3] = v.w;
  }
  const int sh = (int)(ua & 15);
  const int bs8 = (sh & 3) * 8;
  switch (sh >> 2) {
    case 0: realign<0>(c, bs8, w); break;
    case 1: realign<1>(c, bs8, w); break;
    case 2: realign<2>(c, bs8, w); break;
    default: realign<3>(c, bs8, w); break;
  }
  if (start + 64 > len) {
#pragma unroll
    for (int j = 0; j < 16; j++) w[j] = mask_tail(w[j], (int64_t)len - (int64_t)(start + 4 * j));
  }
}

// ---------------------------------------------------------------------------
// UTF-8 (Sec. 3.1.5, Table "tab:unicode"), one byte at a time over the
// non-ASCII words of a block.  State: continuation bytes still expected and
// the allowed range of the next one.
// ---------------------------------------------------------------------------
struct Utf8State {
  uint32_t need, lo, hi;
  bool err;
};

__device__ __forceinline__ void utf8_step(Utf8State &s, uint32_t c) {
  if (s.need) {
    if (c < s.lo || c > s.hi) s.err = true;
    s.need--;
    s.lo = 0x80;
    s.hi = 0xBF;
  } else if (c >= 0x80) {
    if (c < 0xC2) s.err = true;
    else if (c < 0xE0) s.need = 1;
    else if (c < 0xF0) { s.need = 2; s.lo = c == 0xE0 ? 0xA0 : 0x80; s.hi = c == 0xED ? 0x9F : 0xBF; }
    else if (c < 0xF5) { s.need = 3; s.lo = c == 0xF0 ? 0x90 : 0x80; s.hi = c == 0xF4 ? 0x8F : 0xBF; }
    else s.err = true;
  }
}

// Returns true if the block (with the 3 bytes before it, `prev` holding them
// in its top 3 bytes, `nprev` of them inside the document) has a UTF-8 error.
__device__ __forceinline__ bool utf8_block_error(const uint32_t (&w)[16], uint32_t prev, int nprev,
                                                 bool doc_ends_here) {
  Utf8State s{0, 0x80, 0xBF, false};
  // Rebuild the state at byte 0 from the preceding bytes; errors there belong
  // to the previous block and are ignored (a stray continuation byte resets).
  for (int k = 3 - nprev; k < 3; k++) {
    uint32_t c = (prev >> (8 * (k + 1))) & 0xFF;
    Utf8State t = s;
    utf8_step(t, c);
    if (t.err) t = Utf8State{0, 0x80, 0xBF, false};
    s = t;
  }
#pragma unroll
  for (int j = 0; j < 16; j++) {
    if ((w[j] & 0x80808080u) || s.need) {
#pragma unroll
      for (int b = 0; b < 4; b++) utf8_step(s, (w[j] >> (8 * b)) & 0xFF);
    }
  }
  if (doc_ends_here && s.need) s.err = true;
  return s.err;
}

}  // namespace sj
