// s1_common.cuh -- building blocks of stage 1 (Sec. 3.1): SWAR classification
// of 64-byte blocks, the odd-backslash and in-string masks, reading a block
// from the staged window, and the UTF-8 check.
#pragma once
#include "sj_internal.cuh"

namespace sj {

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

__device__ __forceinline__ uint64_t prefix_xor(uint64_t x) {
  x ^= x << 1;
  x ^= x << 2;
  x ^= x << 4;
  x ^= x << 8;
  x ^= x << 16;
  x ^= x << 32;
  return x;
}

// ---------------------------------------------------------------------------
// A lane's 64-byte block from the staged window (shared memory): 16 words,
// realigned with funnel shifts when the document is not 4-byte aligned;
// bytes past the document's end read as spaces.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mask_tail(uint32_t v, int64_t valid) {
  // keep the first `valid` bytes (0..4) of v, the rest become ' '
  if (valid >= 4) return v;
  if (valid <= 0) return 0x20202020u;
  uint32_t keep = (1u << (8 * valid)) - 1;
  return (v & keep) | (0x20202020u & ~keep);
}

__device__ __forceinline__ void read_block(const uint8_t *s, uint64_t blk, uint64_t len,
                                           uint32_t (&w)[16]) {
  if (blk >= len) {
#pragma unroll
    for (int j = 0; j < 16; j++) w[j] = 0x20202020u;
    return;
  }
  const uintptr_t ua = (uintptr_t)s;
  const uint32_t *wp = reinterpret_cast<const uint32_t *>(ua & ~(uintptr_t)3);
  const uint32_t sh = (uint32_t)(ua & 3u) * 8;
  if (sh == 0) {
    if ((ua & 15u) == 0) {
      const uint4 *p = reinterpret_cast<const uint4 *>(ua);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const uint4 v = p[k];
        w[4 * k] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; j++) w[j] = wp[j];
    }
  } else {
    uint32_t lo = wp[0];
#pragma unroll
    for (int j = 0; j < 16; j++) {
      const uint32_t hi = wp[j + 1];
      w[j] = __funnelshift_r(lo, hi, sh);
      lo = hi;
    }
  }
  if (blk + 64 > len) {
#pragma unroll
    for (int j = 0; j < 16; j++) w[j] = mask_tail(w[j], (int64_t)len - (int64_t)(blk + 4 * j));
  }
}

// ---------------------------------------------------------------------------
// UTF-8 check of one 64-byte block (Sec. 3.1.5, Table "tab:unicode").
// The structure of the sequences is checked on per-byte flags (bit 7 of each
// byte of a word): the continuation bytes (10xxxxxx) must be exactly the
// positions that the lead bytes before them require -- one after every
// 11xxxxxx lead, a second after 111xxxxx, a third after 1111xxxx -- including
// positions required by leads among the 3 bytes before the block (`prev`, top
// bytes; missing bytes are 0).  A word's required positions are its lead
// flags moved up by one, two and three bytes, with the flags of the word
// before shifted in.  The remaining rules of the table concern single values
// (C0, C1 and F5-FF never occur; after E0, ED, F0 and F4 the next byte has a
// narrower range) and are checked at each lead byte, read from the block's
// bytes `wb` (shared memory).  A lead whose sequence runs past the block is
// checked by the next block through its `prev`, or here when the document
// ends with the block.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool utf8_block_error_masks(const uint32_t (&w)[16], const uint8_t *wb,
                                                       uint32_t prev, bool doc_ends_here) {
  // lead flags of the word before: >= 2-, >= 3- and 4-byte leads
  uint32_t p2 = prev & (prev << 1) & 0x80808080u;
  uint32_t p3 = p2 & (prev << 2), p4 = p3 & (prev << 3);
  uint32_t bad = 0;
  uint32_t lm[2] = {0, 0};
#pragma unroll
  for (int j = 0; j < 16; j++) {
    const uint32_t x = w[j], x1 = x << 1;
    const uint32_t c = x & ~x1 & 0x80808080u;  // continuation bytes
    const uint32_t t2 = x & x1 & 0x80808080u;  // lead bytes
    const uint32_t t3 = t2 & (x << 2), t4 = t3 & (x << 3);
    const uint32_t req = __funnelshift_l(p2, t2, 8) | __funnelshift_l(p3, t3, 16) |
                         __funnelshift_l(p4, t4, 24);
    bad |= req ^ c;
    lm[j >> 3] |= movemask4(t2) << ((j & 7) * 4);
    p2 = t2;
    p3 = t3;
    p4 = t4;
  }
  if (bad) return true;
  // leads in the last bytes whose sequences run past the document's end
  if (doc_ends_here && ((p2 & 0x80000000u) | (p3 & 0x80800000u) | (p4 & 0x80808000u))) return true;
  const uint64_t L = ((uint64_t)lm[1] << 32) | lm[0];
  // value rules
  const uint32_t pb = prev >> 24;  // byte -1
  if (pb == 0xE0 || pb == 0xED || pb == 0xF0 || pb == 0xF4) {
    const uint32_t b0 = w[0] & 0xFFu;
    if ((pb == 0xE0 && b0 < 0xA0) || (pb == 0xED && b0 > 0x9F) || (pb == 0xF0 && b0 < 0x90) ||
        (pb == 0xF4 && b0 > 0x8F))
      return true;
  }
  uint64_t lead = L;
  while (lead) {
    const int i = __ffsll((long long)lead) - 1;
    lead &= lead - 1;
    const uint32_t b = wb[i];
    if (b < 0xC2 || b > 0xF4) return true;
    if (i < 63 && (b == 0xE0 || b == 0xED || b == 0xF0 || b == 0xF4)) {
      const uint32_t nb = wb[i + 1];
      if ((b == 0xE0 && nb < 0xA0) || (b == 0xED && nb > 0x9F) || (b == 0xF0 && nb < 0x90) ||
          (b == 0xF4 && nb > 0x8F))
        return true;
    }
  }
  return false;
}

}  // namespace sj
