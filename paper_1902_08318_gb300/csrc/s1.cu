// s1.cu -- stage 1 of the parser (Sec. 3.1), reduce-then-scan form.
//
// One warp takes a tile of 2 KiB: each lane owns one 64-byte block, the
// paper's unit of work, and builds its 64-bit masks with SWAR classification.
// The paper carries three facts from one block to the next (footnote of Sec.
// 3.1.1): whether an odd backslash run is pending, whether the scan is inside a
// string, and whether the previous byte separates tokens.  Between the lanes of
// a tile they travel by warp votes and shuffles.  Between tiles, two of them
// are read directly from the bytes before the tile (the backslash run, and the
// class of the previous byte); only the in-string bit needs the whole prefix
// of the document.  So stage1_blocks_kernel computes, for both values of the
// incoming in-string bit, the final structural mask of every block and the
// tile's index count; a segmented scan over tiles (scan.cu) then fixes the bit
// and the output offset of every tile, and stage1_flatten_kernel writes the
// indices.  No kernel waits on another block.
#include "s1_common.cuh"

namespace sj {

// Length of the backslash run that ends just before document position `end`
// (lanes test 32 bytes at a time going backwards).
__device__ __forceinline__ uint64_t bs_run_before(const uint8_t *doc, uint64_t end, int lane) {
  uint64_t run = 0, pos = end;
  for (;;) {
    const bool bs = pos > (uint64_t)lane && doc[pos - 1 - lane] == '\\';
    const unsigned m = __ballot_sync(0xFFFFFFFFu, bs);
    if (m != 0xFFFFFFFFu) return run + (uint64_t)(__ffs(~m) - 1);
    run += 32;
    pos -= 32;
  }
}

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
// copy `wb` in shared memory.  A lead whose sequence runs past the block is
// checked by the next block through its `prev`, or here when the document
// ends with the block.
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

// How the byte before a tile makes its first byte a token start.
enum : uint32_t { kSepNever = 0, kSepAlways = 1, kSepIfOutside = 2 };

__global__ void __launch_bounds__(32 * kS1Warps) stage1_blocks_kernel(const Job *__restrict__ job) {
  pdl_enter();
  const Job &J = *job;
  __shared__ uint32_t s_words[kS1Warps * 32][16];  // one block per thread (byte reads)
  const int lane = threadIdx.x & 31;
  uint32_t *my_words = s_words[threadIdx.x];
  uint32_t t_lo, t_hi;
  s1_range(J, t_lo, t_hi);
  TileTickets tix(J, kTicketS1, t_lo, t_hi, blockIdx.x * kS1Warps + (threadIdx.x >> 5),
                  gridDim.x * kS1Warps, lane);
  for (uint32_t t = tix.first(); t < t_hi; t = tix.next()) {
    tix.draw();
    const uint32_t d = doc_of_tile(J, t);
    const uint32_t tt = t - J.tile_first[d];
    const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
    // host input: read it over the host link here, once, and leave the device
    // copy the later kernels read (the copy overlaps this kernel's work)
    const uint8_t *doc = (J.src ? J.src : J.base) + J.doc_off[d];
    const uint64_t t0 = (uint64_t)tt * kTileBytes;
    const uint64_t blk = t0 + (uint64_t)lane * kBlockBytes;

    uint32_t w[16];
    load_block(doc, len, blk, w);
    if (J.src && blk < len) {
      uint8_t *dst = const_cast<uint8_t *>(J.base) + J.doc_off[d] + blk;
      if (blk + kBlockBytes <= len && ((uintptr_t)dst & 15) == 0) {
#pragma unroll
        for (int k = 0; k < 4; k++)
          reinterpret_cast<uint4 *>(dst)[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
      } else {
        const uint32_t nb = (uint32_t)min((uint64_t)kBlockBytes, len - blk);
#pragma unroll
        for (int k = 0; k < 16; k++)
#pragma unroll
          for (int b = 0; b < 4; b++)
            if ((uint32_t)(4 * k + b) < nb) dst[4 * k + b] = (uint8_t)(w[k] >> (8 * b));
      }
    }
    BlockMasks m;
    classify_block(w, m);

    // ---- UTF-8 (Sec. 3.1.5) --------------------------------------------------
    {
      uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, w[15], 1);
      int nprev = 3;
      if (lane == 0) {
        prev = 0;
        nprev = blk >= 3 ? 3 : (int)blk;
        for (int k = 0; k < nprev; k++) prev |= (uint32_t)doc[blk - nprev + k] << (8 * (4 - nprev + k));
      }
#ifdef SJ_ABL_UTF8_ALWAYS
      const bool need = true;
#else
      const bool need = m.nonascii != 0 || (prev & (prev << 1) & 0x80808000u);
#endif
      const bool ends_here = blk < len && blk + 64 >= len;
      if (blk < len && need) {
#pragma unroll
        for (int k = 0; k < 16; k++) my_words[k] = w[k];
        if (utf8_block_error_masks(w, reinterpret_cast<const uint8_t *>(my_words), prev, ends_here))
          atomicOr(&J.doc_flags[d], kFlagUtf8);
      }
    }

    // ---- carries read from the bytes before the tile --------------------------
    uint32_t e_in = 0, sep_rule = kSepAlways;  // byte -1 of a document: virtual white space
    if (tt > 0) {
      e_in = (uint32_t)(bs_run_before(doc, t0, lane) & 1);
      const uint8_t c = doc[t0 - 1];
      if (c == ' ' || c == '\n' || c == '\r' || c == '\t') sep_rule = kSepAlways;
      else if (c == ',' || c == ':' || c == '[' || c == ']' || c == '{' || c == '}') sep_rule = kSepIfOutside;
      else if (c == '"') sep_rule = (bs_run_before(doc, t0 - 1, lane) & 1) ? kSepNever : kSepAlways;
      else sep_rule = kSepNever;
    }

    // ---- escapes (Fig. "identifyescapedquotes") and real quotes ---------------
    const bool all_bs = (m.bs == ~0ull);
    const uint32_t tail = (uint32_t)__clzll((long long)~m.bs) & 1u;  // trailing run parity
    const unsigned nb = __ballot_sync(0xFFFFFFFFu, !all_bs);
    const unsigned tb = __ballot_sync(0xFFFFFFFFu, tail);
    const unsigned below = (1u << lane) - 1u;
    uint32_t e_lane = e_in;
    if (nb & below) e_lane = (tb >> (31 - __clz(nb & below))) & 1u;
    const uint64_t od = escaped_no_carry(m.bs) ^ (e_lane ? first_non_bs(m.bs) : 0ull);
    const uint64_t Q = m.quote & ~od;
#ifdef SJ_ABL_QUOTE_PARITY_SHFL
    const uint32_t qp = __popcll(Q) & 1u;
    uint32_t qincl = qp;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, qincl, o);
      if (lane >= o) qincl ^= u;
    }
    const uint32_t q_before = qincl ^ qp;
    const uint32_t q_tile = __shfl_sync(0xFFFFFFFFu, qincl, 31);
#else
    const unsigned pb = __ballot_sync(0xFFFFFFFFu, __popcll(Q) & 1u);
    const uint32_t q_before = __popc(pb & below) & 1u;  // real quotes in earlier lanes, mod 2
    const uint32_t q_tile = __popc(pb) & 1u;
#endif
    const uint64_t RQ = prefix_xor(Q);

    // ---- final masks (Figs. "identifyquoteregion", "identifypseudo") for both
    //      values h of the in-string bit entering the tile -----------------------
    uint64_t S[2];
    uint32_t cnt[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const uint64_t R = RQ ^ (((uint32_t)h ^ q_before) ? ~0ull : 0ull);
      const uint64_t S1 = (m.op & ~R) | Q;
      const uint64_t SW = S1 | m.ws;
      uint32_t sep_in = __shfl_up_sync(0xFFFFFFFFu, (uint32_t)(SW >> 63), 1);
      if (lane == 0) sep_in = sep_rule == kSepAlways ? 1u : (sep_rule == kSepIfOutside ? (uint32_t)(h ^ 1) : 0u);
      const uint64_t P = ((SW << 1) | sep_in) & ~m.ws & ~R;
      S[h] = (S1 | P) & ~(Q & ~R);
      uint32_t c = __popcll(S[h]);
#pragma unroll
      for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
      cnt[h] = c;
    }
    reinterpret_cast<ulonglong2 *>(J.s1_blk)[(uint64_t)t * 32 + lane] = make_ulonglong2(S[0], S[1]);
    // real quotes and string-special bytes (backslash, control) for stage 2
    J.s1_qx[(uint64_t)t * 32 + lane] = make_ulonglong2(Q, m.bs | ctrl_mask(w));
    if (lane == 0) {
      S1Agg a;
      a.qpar = q_tile;
      a.c0 = cnt[0];
      a.c1 = cnt[1];
      a.head = tt == 0;
      J.s1_rec[t] = a;
    }
  }
}

// After the tile scan: pick each block's mask for the actual in-string bit,
// and write the indices (Sec. 3.1.4) at the tile's offset, staged in shared
// memory so that the stores are coalesced.
__global__ void __launch_bounds__(32 * kS1Warps) stage1_flatten_kernel(const Job *__restrict__ job) {
  pdl_enter();
  const Job &J = *job;
  const int lane = threadIdx.x & 31;
#ifndef SJ_ABL_NAIVE_FLATTEN
  __shared__ uint16_t stage[kS1Warps][kTileBytes];  // tile-relative positions
  uint16_t *out_stage = stage[threadIdx.x >> 5];
#endif
  uint32_t t_lo, t_hi;
  s1_range(J, t_lo, t_hi);
  const uint32_t warps = gridDim.x * kS1Warps;
  const ulonglong2 *blk = reinterpret_cast<const ulonglong2 *>(J.s1_blk);
  // software pipeline: a tile's masks and prefix are loaded while the tile
  // before it is written
  uint32_t t = t_lo + blockIdx.x * kS1Warps + (threadIdx.x >> 5);
  ulonglong2 v_next = make_ulonglong2(0, 0);
  S1Pre pre_next{0, 0};
  if (t < t_hi) {
    v_next = blk[(uint64_t)t * 32 + lane];
    pre_next = J.s1_pre[t];
  }
  for (; t < t_hi; t += warps) {
    const ulonglong2 v = v_next;
    const S1Pre pre = pre_next;
    if (t + warps < t_hi) {
      v_next = blk[(uint64_t)(t + warps) * 32 + lane];
      pre_next = J.s1_pre[t + warps];
    }
    const uint32_t d = doc_of_tile(J, t);
    const uint32_t tt = t - J.tile_first[d];
    const uint32_t ntiles_d = J.tile_first[d + 1] - J.tile_first[d];
    const uint64_t S = pre.q_in ? v.y : v.x;
    const uint32_t c = __popcll(S);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += u;
    }
    const uint32_t n = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t o = incl - c;
    uint64_t s = S;
    uint32_t *dst = J.idx + idx_base(J, d) + pre.base;
    const uint32_t t0 = tt * kTileBytes;
#ifdef SJ_ABL_NAIVE_FLATTEN
    const uint32_t p0 = t0 + lane * kBlockBytes;
    while (s) {
      dst[o++] = p0 + (uint32_t)(__ffsll((long long)s) - 1);
      s &= s - 1;
    }
#else
    const uint32_t rel0 = lane * kBlockBytes;
    while (s) {
      out_stage[o++] = (uint16_t)(rel0 + (uint32_t)(__ffsll((long long)s) - 1));
      s &= s - 1;
    }
    __syncwarp();
    for (uint32_t k = lane; k < n; k += 32) dst[k] = t0 + out_stage[k];
    __syncwarp();
#endif
    // index count and first index of each stage-2 tile (the tile itself, or
    // each group of 32 >> s2_shift blocks)
    {
      const uint32_t sh = J.s2_shift, grp = 32u >> sh;
      const uint32_t end_incl = __shfl_sync(0xFFFFFFFFu, incl, lane | (int)(grp - 1));
      if ((lane & (grp - 1)) == 0) {
        const uint32_t t2 = (t << sh) + ((uint32_t)lane >> (5 - sh));
        J.tile_cnt[t2] = end_incl - (incl - c);
        J.tile_off[t2] = pre.base + incl - c;
      }
    }
    if (lane == 0) {
      if (tt == ntiles_d - 1) {
        J.doc_nidx[d] = pre.base + n;
        if (pre.q_in ^ J.s1_rec[t].qpar) atomicOr(&J.doc_flags[d], kFlagUnclosed);
      } else if (t + 1 == t_hi) {
        J.doc_nidx[d] = pre.base + n;  // the indices so far (a document arriving in chunks)
      }
    }
  }
}

}  // namespace sj
