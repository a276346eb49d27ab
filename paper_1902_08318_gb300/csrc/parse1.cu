// parse1.cu -- the first pass of a run: stage 1 (Sec. 3.1) and the scans of
// stage 2 (Sec. 3.2) in one kernel, with decoupled look-backs between tiles.
//
// One warp takes a tile of 2 KiB (its bytes copied into shared memory by one
// bulk copy) and, in order:
//   1. stage 1 per 64-byte block (one block per lane): SWAR classification,
//      UTF-8, the odd-backslash escapes and the real quotes, the in-string
//      mask by prefix XOR and the structural and pseudo-structural bits -- for
//      both values of the in-string bit entering the tile.  The escape run and
//      the separator state entering the tile are read from the bytes before
//      it; only the in-string bit needs the tiles before;
//   2. a look-back over the tiles before it (quote parity and index counts)
//      gives that bit and the tile's first index; the indices are written
//      (flatten, Sec. 3.1.4) and kept in shared memory;
//   3. the tile's tokens, 32 at a time: kinds, the depth and tape-slot scan,
//      the last opener of every level (the containers the tile leaves open),
//      the normalised length of every string (from the real-quote and
//      backslash/control masks; strings with escapes, or running past the
//      tile, are walked), and the list of number tokens;
//   4. a second look-back (depth, tape words, string-buffer bytes) gives the
//      tile's absolute depth, first tape slot and string-buffer offset.
// Tiles are taken in ticket order, so every tile a look-back waits on is held
// by a running warp: the first round by grid index (thread blocks start in
// index order), later tiles from a counter drawn when a tile is done.
#include "s1_common.cuh"
#include "strings.cuh"

namespace sj {

constexpr int kP1Warps = 4;
constexpr int kPre = 64;    // staged bytes before the tile (carries in, UTF-8)
constexpr int kPost = 64;   // staged bytes after the tile (strings' ends)
constexpr int kWin1 = ((kPre + kTileBytes + kPost + 48) + 15) & ~15;
constexpr int kOpenSmem = 512;      // levels kept in shared memory (mod 512)
constexpr int kLevelOff = kMaxTileTokens;
constexpr uint32_t kQueue = 64;

struct __align__(16) P1Smem {
  uint8_t win[kWin1];        // the staged window (bulk copy destination)
  uint64_t q[32];            // real quotes of the tile's blocks
  uint64_t x[32];            // backslash and control bytes of the tile's blocks
  uint16_t pos[kTileBytes];  // tile-relative positions of the tile's indices
  uint16_t open[kOpenSmem];  // level table
  uint32_t sq[kQueue];       // queued strings: position | (next token's position + 1) << 12
  uint64_t mbar;
};
static_assert(sizeof(P1Smem) % 16 == 0 && kWin1 % 16 == 0, "per-warp staging stays 16-byte aligned");

// ---- look-back 1: quote parity and index counts ---------------------------
// Status word of a tile: bits 35-63 the run's epoch (a word of an earlier run
// is not published), bits 33-34 the state (1: aggregate, 2: inclusive),
// bit 32 the quote parity after the tile (inclusive), bits 0-31 the payload:
// aggregate = c0 | c1 << 12 | qpar << 24 (indices when entered outside /
// inside a string, quote parity), inclusive = indices up to the tile's end.
constexpr uint32_t kEpoch1Mask = 0x1FFFFFFFu;
__device__ __forceinline__ uint64_t st1_word(uint32_t ep, uint32_t state, uint32_t q, uint32_t pay) {
  return ((uint64_t)(ep & kEpoch1Mask) << 35) | ((uint64_t)state << 33) | ((uint64_t)q << 32) | pay;
}

struct A1 {
  uint32_t qpar, c0, c1;
};
// a before b
__device__ __forceinline__ A1 a1_combine(const A1 &a, const A1 &b) {
  return A1{a.qpar ^ b.qpar, a.c0 + (a.qpar ? b.c1 : b.c0), a.c1 + (a.qpar ? b.c0 : b.c1)};
}

__device__ __forceinline__ uint64_t spin1(const Job &J, const uint64_t *p, uint32_t ep, uint32_t d) {
  uint64_t v = ld_acquire(p);
  uint32_t ns = 32;
  for (uint32_t n = 0; (uint32_t)(v >> 35) != (ep & kEpoch1Mask); n++) {
    if (n >= kSpinLimit) {  // never published: give up, mark the document
      atomicOr(&J.doc_flags[d], kFlagInternal);
      return st1_word(ep, 2, 0, 0);
    }
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
    v = ld_acquire(p);
  }
  return v;
}

// Exclusive stage-1 prefix of tile t (tiles j_min .. t-1 of its document):
// the in-string bit entering it and the number of indices before it.
__device__ void lookback1(const Job &J, uint32_t t, uint32_t j_min, uint32_t d, uint32_t ep,
                          int lane, uint32_t &q_in, uint32_t &base) {
  A1 acc{0, 0, 0};  // the tiles between the window and t, combined
  int64_t j = (int64_t)t - 1;
  for (;;) {
    const int64_t jj = j - lane;
    const bool in = jj >= (int64_t)j_min;
    const uint64_t st = in ? spin1(J, &J.st1[jj], ep, d) : 0ull;
    const uint32_t state = (uint32_t)(st >> 33) & 3u;
    const unsigned pm = __ballot_sync(0xFFFFFFFFu, in && state == 2);
    const unsigned im = __ballot_sync(0xFFFFFFFFu, in);
    const int K = pm ? __ffs(pm) - 1 : __popc(im);  // lanes [0, K) are aggregates to combine
    A1 v{0, 0, 0};
    if (lane < K) v = A1{(uint32_t)(st >> 24) & 1u, (uint32_t)st & 0xFFFu, (uint32_t)(st >> 12) & 0xFFFu};
    // ordered reduction: lane i holds tile j - i (a higher lane is an earlier tile)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      A1 u;
      u.qpar = __shfl_down_sync(0xFFFFFFFFu, v.qpar, o);
      u.c0 = __shfl_down_sync(0xFFFFFFFFu, v.c0, o);
      u.c1 = __shfl_down_sync(0xFFFFFFFFu, v.c1, o);
      if (lane + o < 32) v = a1_combine(u, v);
    }
    A1 win;
    win.qpar = __shfl_sync(0xFFFFFFFFu, v.qpar, 0);
    win.c0 = __shfl_sync(0xFFFFFFFFu, v.c0, 0);
    win.c1 = __shfl_sync(0xFFFFFFFFu, v.c1, 0);
    acc = a1_combine(win, acc);
    if (pm) {
      const uint64_t sk = __shfl_sync(0xFFFFFFFFu, st, K);
      const uint32_t q = (uint32_t)(sk >> 32) & 1u;
      q_in = q ^ acc.qpar;
      base = (uint32_t)sk + (q ? acc.c1 : acc.c0);
      return;
    }
    if (j - 32 < (int64_t)j_min) {  // reached the document's first tile
      q_in = acc.qpar;
      base = acc.c0;
      return;
    }
    j -= 32;
  }
}

// ---- look-back 2: depth, tape words, string-buffer bytes --------------------
// Flag word of a tile: epoch << 2 | state (1: agg2 holds its aggregate,
// 2: inc2 holds its inclusive prefix).  The three quantities are plain sums.
constexpr uint32_t kEpoch2Mask = 0x3FFFFFFFu;

__device__ __forceinline__ uint32_t spin2(const Job &J, const uint32_t *p, uint32_t ep, uint32_t d) {
  uint32_t v = ld_acquire(p);
  uint32_t ns = 32;
  for (uint32_t n = 0; (v >> 2) != (ep & kEpoch2Mask); n++) {
    if (n >= kSpinLimit) {
      atomicOr(&J.doc_flags[d], kFlagInternal);
      return 0u;  // read as an aggregate of zeros below
    }
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
    v = ld_acquire(p);
  }
  return v;
}

__device__ S2Incl lookback2(const Job &J, uint32_t t, uint32_t j_min, uint32_t d, uint32_t ep,
                            int lane) {
  int32_t dd = 0;
  uint32_t w = 0;
  uint64_t s = 0;
  int64_t j = (int64_t)t - 1;
  for (;;) {
    const int64_t jj = j - lane;
    const bool in = jj >= (int64_t)j_min;
    const uint32_t f = in ? spin2(J, &J.st2[jj], ep, d) : 0u;
    const bool incl = in && (f & 3u) == 2u;
    const unsigned pm = __ballot_sync(0xFFFFFFFFu, incl);
    const unsigned im = __ballot_sync(0xFFFFFFFFu, in);
    const int K = pm ? __ffs(pm) - 1 : __popc(im);
    int32_t vd = 0;
    uint32_t vw = 0;
    uint64_t vs = 0;
    if (lane < K && (f & 3u) == 1u) {
      const S2Agg a = J.agg2[jj];
      vd = a.dd;
      vw = a.w;
      vs = a.s;
    } else if (pm && lane == K) {
      const S2Incl c = J.inc2[jj];
      vd = c.d;
      vw = c.w;
      vs = c.s;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      vd += __shfl_xor_sync(0xFFFFFFFFu, vd, o);
      vw += __shfl_xor_sync(0xFFFFFFFFu, vw, o);
      vs += __shfl_xor_sync(0xFFFFFFFFu, vs, o);
    }
    dd += vd;
    w += vw;
    s += vs;
    if (pm || j - 32 < (int64_t)j_min) return S2Incl{dd, w, s};
    j -= 32;
  }
}

// ---- helpers ----------------------------------------------------------------
// Length of the backslash run ending just before document position `end`.
__device__ __forceinline__ uint64_t bs_run_before(const Window &win, uint64_t end, int lane) {
  uint64_t run = 0, pos = end;
  for (;;) {
    const bool bs = pos > (uint64_t)lane && win.at(pos - 1 - lane) == '\\';
    const unsigned m = __ballot_sync(0xFFFFFFFFu, bs);
    if (m != 0xFFFFFFFFu) return run + (uint64_t)(__ffs(~m) - 1);
    run += 32;
    pos -= 32;
  }
}

// Normalised length of a string without escapes or control bytes whose first
// content byte is at tile-relative position rel, from the tile's masks: the
// distance to the next real quote.  False when the masks cannot decide it (an
// escape or control byte first, or no quote before the tile's end).
__device__ __forceinline__ bool plain_string_len(const P1Smem &W, uint32_t rel, uint32_t &L) {
  uint32_t w = rel >> 6, b = rel & 63, acc = 0;
  while (w < 32) {
    const uint64_t q = W.q[w] >> b, x = W.x[w] >> b;
    if (q) {
      const uint32_t z = (uint32_t)__ffsll((long long)q) - 1;
      if (x & ((1ull << z) - 1)) return false;
      L = acc + z;
      return true;
    }
    if (x) return false;
    acc += 64 - b;
    b = 0;
    w++;
  }
  return false;
}

template <class T>
__device__ __forceinline__ void enqueue(T *q, uint32_t &tail, bool take, const T &e, int lane) {
  const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
  if (take) q[(tail + __popc(m & ((1u << lane) - 1u))) & (kQueue - 1)] = e;
  tail += __popc(m);
}

// How the byte before a tile makes its first byte a token start.
enum : uint32_t { kSepNever = 0, kSepAlways = 1, kSepIfOutside = 2 };

__global__ void __launch_bounds__(32 * kP1Warps) parse1_kernel(const Job *__restrict__ job) {
  const Job &J = *job;
  __shared__ P1Smem WS[kP1Warps];
  __shared__ uint8_t s_kind[256];
  const int lane = threadIdx.x & 31;
  const uint32_t wid = threadIdx.x >> 5;
  P1Smem &W = WS[wid];
  for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) s_kind[i] = token_kind((uint8_t)i);
  for (uint32_t i = lane; i < kOpenSmem; i += 32) W.open[i] = 0;
  mbar_init(&W.mbar, lane);
  __syncthreads();
  const uint32_t n_tiles = J.counters[kCtrTiles];
  const uint32_t ep = J.epoch;
  const uint32_t gw = blockIdx.x * kP1Warps + wid, nw = gridDim.x * kP1Warps;
  uint16_t *const open_g = J.open_g ? J.open_g + (uint64_t)gw * kOpenGlobal : nullptr;
  const unsigned below = (1u << lane) - 1u;
  uint32_t phase = 0;

  for (uint32_t t = gw; t < n_tiles;) {
    const uint32_t d = doc_of_tile(J, t);
    const uint32_t j_min = J.tile_first[d];
    const uint32_t tt = t - j_min;
    const uint32_t ntiles_d = J.tile_first[d + 1] - j_min;
    const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
    // the bytes are read where they are: device memory, or pinned host memory
    // (then this pass writes the device copy the later passes read)
    const uint8_t *gdoc = (J.src ? J.src : J.base) + J.doc_off[d];
    const uint64_t t0 = (uint64_t)tt * kTileBytes;
    const uint64_t p0 = t0 >= (uint64_t)kPre ? t0 - kPre : 0;
    uintptr_t a0, a1;
    window_extent(gdoc, len, p0, t0 + kTileBytes + kPost, a0, a1);
    if (J.src) {
      lane_copy(W.win, a0, a1, lane);
      __syncwarp();
    } else {
      if (lane == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_copy_start(W.win, a0, (uint32_t)(a1 - a0), &W.mbar, lane);
      if (!bulk_copy_wait(&W.mbar, phase)) atomicOr(&J.doc_flags[d], kFlagInternal);
      phase ^= 1u;
    }
    Window win;
    win.s = W.win;
    win.sbase = (int64_t)(a0 - (uintptr_t)gdoc);
    win.lo = p0;
    win.hi = min(len, (uint64_t)(a1 - (uintptr_t)gdoc));
    win.g = gdoc;

    // ---- stage 1 of this lane's block ------------------------------------------
    const uint64_t blk = t0 + (uint64_t)lane * kBlockBytes;
    const uint8_t *wb = W.win + (blk - (uint64_t)win.sbase);  // block bytes (when blk < len)
    uint32_t w[16];
    read_block(wb, blk, len, w);
    if (J.src && blk < len) {  // the device copy of the block
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

    // UTF-8 (Sec. 3.1.5)
    {
      uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, w[15], 1);
      if (lane == 0) {
        prev = 0;
        if (blk >= 3)
          for (int k = 0; k < 3; k++) prev |= (uint32_t)win.at(blk - 3 + k) << (8 * (k + 1));
      }
      const bool need = m.nonascii != 0 || (prev & (prev << 1) & 0x80808000u);
      const bool ends_here = blk < len && blk + 64 >= len;
      if (blk < len && need && utf8_block_error_masks(w, wb, prev, ends_here))
        atomicOr(&J.doc_flags[d], kFlagUtf8);
    }

    // carries read from the bytes before the tile
    uint32_t e_in = 0, sep_rule = kSepAlways;  // byte -1 of a document: virtual white space
    if (tt > 0) {
      e_in = (uint32_t)(bs_run_before(win, t0, lane) & 1);
      const uint8_t c = win.at(t0 - 1);
      if (c == ' ' || c == '\n' || c == '\r' || c == '\t') sep_rule = kSepAlways;
      else if (c == ',' || c == ':' || c == '[' || c == ']' || c == '{' || c == '}') sep_rule = kSepIfOutside;
      else if (c == '"') sep_rule = (bs_run_before(win, t0 - 1, lane) & 1) ? kSepNever : kSepAlways;
      else sep_rule = kSepNever;
    }

    // escapes (Fig. "identifyescapedquotes") and real quotes
    const bool all_bs = (m.bs == ~0ull);
    const uint32_t tail = (uint32_t)__clzll((long long)~m.bs) & 1u;  // trailing run parity
    const unsigned nbm = __ballot_sync(0xFFFFFFFFu, !all_bs);
    const unsigned tbm = __ballot_sync(0xFFFFFFFFu, tail);
    uint32_t e_lane = e_in;
    if (nbm & below) e_lane = (tbm >> (31 - __clz(nbm & below))) & 1u;
    const uint64_t od = escaped_no_carry(m.bs) ^ (e_lane ? first_non_bs(m.bs) : 0ull);
    const uint64_t Q = m.quote & ~od;
    const unsigned pb = __ballot_sync(0xFFFFFFFFu, __popcll(Q) & 1u);
    const uint32_t q_before = __popc(pb & below) & 1u;  // real quotes in earlier lanes, mod 2
    const uint64_t RQ = prefix_xor(Q);

    // final masks (Figs. "identifyquoteregion", "identifypseudo") for both
    // values h of the in-string bit entering the tile
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
    if (!J.s1_only) {
      W.q[lane] = Q;
      W.x[lane] = m.bs | ctrl_mask(w);
    }
    const uint32_t qpar = __popc(pb) & 1u;

    // ---- look-back 1 ---------------------------------------------------------
    uint32_t q_in = 0, base = 0;
    if (tt > 0) {
      if (lane == 0) st_release(&J.st1[t], st1_word(ep, 1, 0, cnt[0] | cnt[1] << 12 | qpar << 24));
      lookback1(J, t, j_min, d, ep, lane, q_in, base);
    }
    const uint32_t n = q_in ? cnt[1] : cnt[0];
    if (lane == 0) st_release(&J.st1[t], st1_word(ep, 2, q_in ^ qpar, base + n));
    const bool last_tile = tt == ntiles_d - 1;
    if (last_tile && lane == 0 && (q_in ^ qpar)) atomicOr(&J.doc_flags[d], kFlagUnclosed);

    // ---- flatten (Sec. 3.1.4): positions kept in shared memory ----------------
    const uint64_t ib = idx_base(J, d);
    {
      const uint64_t Sx = q_in ? S[1] : S[0];
      const uint32_t c = __popcll(Sx);
      uint32_t o = warp_incl_u32(c, lane) - c;
      uint64_t s = Sx;
      const uint32_t rel0 = lane * kBlockBytes;
      while (s) {
        W.pos[o++] = (uint16_t)(rel0 + (uint32_t)(__ffsll((long long)s) - 1));
        s &= s - 1;
      }
      __syncwarp();
      uint32_t *dst = J.idx + ib + base;
      const uint32_t tb = (uint32_t)t0;
      for (uint32_t k = lane; k < n; k += 32) dst[k] = tb + W.pos[k];
    }
    if (lane == 0) {
      J.tile_cnt[t] = n;
      J.tile_off[t] = base;
      if (last_tile) J.doc_nidx[d] = base + n;
    }

    if (!J.s1_only) {
      // ---- stage-2 scans of the tile's tokens -------------------------------------
      const OpenTable ot = n < (uint32_t)kOpenSmem ? OpenTable{W.open, (uint32_t)kOpenSmem - 1u, 0}
                                                   : OpenTable{open_g, 0xFFFFFFFFu, kLevelOff};
      uint32_t *slen = J.slen + ib + base;
      uint64_t *nlist = J.nlist + ib + base;
      int32_t depth = 0, mn = 0, mx = 0;
      uint32_t tape = 0, nnum = 0, shead = 0, stail = 0;
      uint64_t sb = 0;  // string-buffer bytes of this lane's strings
      // the next 32 queued strings: lengths from the masks, else a walk
      auto flush_strings = [&]() {
        const uint32_t mq = min(32u, stail - shead);
        const bool have = (uint32_t)lane < mq;
        const uint32_t e = have ? W.sq[(shead + lane) & (kQueue - 1)] : 0u;
        const uint32_t rel = (e & 0xFFFu) + 1u;  // first content byte, tile relative
        const uint32_t nx = e >> 12;             // next token's position + 1, or 0
        uint32_t L = 0, sl = 0;
        bool ok = have && plain_string_len(W, rel, L);
        if (ok) sl = L;
        if (have && !ok) {
          const uint64_t pa = t0 + rel;
          const uint64_t lim = nx ? t0 + nx - 1 : len;  // the next token, else the document's end
          int err;
          const uint8_t *sp = win.has(pa, lim) ? win.s + ((int64_t)pa - win.sbase) : gdoc + pa;
          const uint8_t *qend = sp;
          const uint32_t nn = string_walk8<false>(sp, sp + (lim - pa), err, nullptr, &qend);
          if (err) sl = kSlenErr | (uint32_t)err;
          else sl = min(nn, kSlenLen) | ((uint64_t)(qend - sp) != nn ? kSlenWalk : 0u);
          L = err ? 0u : nn;
        }
        if (have) {
          slen[shead + lane] = sl;
          sb += 5u + (uint64_t)L;
        }
        shead += mq;
        __syncwarp();
      };
      for (uint32_t b0 = 0; b0 < n; b0 += 32) {
        const uint32_t j = b0 + lane;
        const bool valid = j < n;
        const uint32_t pos = valid ? W.pos[j] : 0u;
        const uint32_t nxt = j + 1 < n ? W.pos[j + 1] + 1u : 0u;
        const uint8_t kind = valid ? s_kind[W.win[t0 + pos - (uint64_t)win.sbase]] : K_OTHER;
        const int32_t dl = depth_delta(kind);
        const uint32_t wd = tape_words_of(kind);
        const uint32_t vi = warp_incl_u32((uint32_t)(dl + 1) | (wd << 8), lane);
        const int32_t D = depth + (int32_t)(vi & 0xFFu) - (lane + 1);
        const int32_t E = D - dl;
        const uint32_t tp = tape + (vi >> 8) - wd;
        if (valid) {
          mn = min(mn, min(E, D));
          mx = max(mx, max(E, D));
        }
        // the last opener of each level of this chunk stays open for later tokens
        const bool op = valid && is_open(kind);
        const unsigned grp = __match_any_sync(0xFFFFFFFFu, op ? D : 0x7FFFFFFF);
        if (op && lane == 31 - __clz(grp))
          ot.at(D) = (uint16_t)(0x8000u | (kind == K_OPEN_OBJ ? 0x4000u : 0u) | tp);
        enqueue(W.sq, stail, valid && kind == K_STRING, pos | (nxt << 12), lane);
        {
          const bool isnum = valid && kind == K_NUMBER;
          const unsigned nb = __ballot_sync(0xFFFFFFFFu, isnum);
          if (isnum) {
            const uint32_t span = nxt ? nxt - 1u - pos : 0u;  // bytes to the next token, 0: unknown
            nlist[nnum + __popc(nb & below)] =
                (uint64_t)pos | ((uint64_t)j << 16) | ((uint64_t)tp << 32) | ((uint64_t)span << 48);
          }
          nnum += __popc(nb);
        }
        const uint32_t tot = __shfl_sync(0xFFFFFFFFu, vi, 31);
        depth += (int32_t)(tot & 0xFFu) - 32;
        tape += tot >> 8;
        __syncwarp();
        if (stail - shead >= 32) flush_strings();
      }
      while (shead != stail) flush_strings();
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        sb += __shfl_xor_sync(0xFFFFFFFFu, sb, o);
        mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
      }
      // survivors: the open container of each level in (mn, depth]
      for (int32_t lv = mn + 1 + lane; lv <= depth; lv += 32) {
        const uint16_t e = ot.at(lv);
        J.surv[ib + base + (uint32_t)(lv - mn - 1)] = ((uint32_t)(e >> 14) & 1u) << 31 | (e & 0x0FFFu);
      }
      __syncwarp();
      for (int32_t v = max(mn, -kLevelOff) + lane; v <= min(mx, kLevelOff); v += 32) ot.at(v) = 0;
      __syncwarp();

      // ---- look-back 2 -----------------------------------------------------------
      S2Incl ex{0, 0, 0};
      if (tt > 0) {
        if (lane == 0) J.agg2[t] = S2Agg{depth, mn, tape, 0u, sb};
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(&J.st2[t], (ep & kEpoch2Mask) << 2 | 1u);
        ex = lookback2(J, t, j_min, d, ep, lane);
      } else {
        __threadfence();
        __syncwarp();
      }
      if (lane == 0) {
        J.inc2[t] = S2Incl{ex.d + depth, ex.w + tape, ex.s + sb};
        __threadfence();
        st_release(&J.st2[t], (ep & kEpoch2Mask) << 2 | 2u);
        J.pre2[t] = S2Pre{ex.d, ex.d + mn, 1u + ex.w, 0u, ex.s};
        J.tile_nstr[t] = stail;
        J.tile_nnum[t] = nnum;
        if (last_tile) {  // the document's tape size, string bytes and root words
          const uint64_t T = 2ull + ex.w + tape;
          const uint64_t tape_cap = len + 3;
          if (ex.d + depth != 0) report(J, d, (uint64_t)base + n, SJ_TAPE_ERROR);
          if (T <= tape_cap) {
            uint64_t *tp = J.tape + tape_base(J, d);
            tp[0] = ((uint64_t)'r' << 56) | (T - 1);
            tp[T - 1] = (uint64_t)'r' << 56;
          }
          J.doc_tape[d] = T;
          J.doc_str[d] = ex.s + sb;
        }
      }
    }
    __syncwarp();  // every lane is done with this tile's shared memory
    // the next tile: a ticket drawn now that this one is done
    uint32_t nt = 0;
    if (lane == 0) nt = nw + atomicAdd(&J.counters[kCtrTicket1], 1u);
    t = __shfl_sync(0xFFFFFFFFu, nt, 0);
  }
}

}  // namespace sj
