// parse2.cu -- the second pass of a run (Sec. 3.2): for every tile, the
// containers open on entry, the grammar, the tape words and the string
// buffer; and the number conversions (Sec. 3.2.1) in a kernel of their own.
//
// The first pass (parse1.cu) has left, per tile, its indices, its exclusive
// prefix (depth, lowest depth, first tape slot, string-buffer offset), the
// containers it leaves open by level (survivors), the normalised length of
// each string and the list of its numbers.  Here one warp per tile:
//   - finds the container open at every level the tile starts inside: the
//     nearest earlier tile whose lowest depth is below a level holds that
//     level's container among its survivors, and one such tile serves a
//     whole range of levels.  Tiles publish a jump pointer (the nearest
//     earlier tile with a lower lowest depth) as they go; a walk takes a
//     published pointer where it finds one and otherwise steps back one tile
//     (32 tiles per warp step), so it never waits on another tile;
//   - walks its tokens 32 at a time: kinds, depth and tape-slot scan, each
//     token's enclosing container (in the tile: a search over window minima
//     of the depth plus a level table; else the frontier), the grammar check
//     against the previous two tokens and that container, the tape words of
//     containers, atoms and strings, and the string buffer (32 strings
//     assembled in shared memory and copied out with 16-byte stores).
// The first failing token of a document (smallest index; grammar before
// content at one token) gives its error code (an atomic minimum).
#include "number.cuh"
#include "sj_internal.cuh"
#include "strings.cuh"

namespace sj {

constexpr int kBWarps = 4;
constexpr int kBPost = 256;  // staged bytes after the tile: strings and atoms running past it
constexpr int kWin3 = ((kTileBytes + kBPost + 48) + 15) & ~15;
constexpr int kStrStage = 2048;  // string output of 32 strings, staged
constexpr int kOpenSmem2 = 512;
constexpr int kLevelOff2 = kMaxTileTokens;
constexpr uint32_t kQueue2 = 64;
constexpr uint32_t kFrontSmem = 64;  // frontier slots of a tile kept in shared memory

struct QEntry {
  uint32_t pos;  // tile-relative position of the opening quote
  uint32_t j;    // index of the token in the tile
  uint32_t tp;   // tape slot relative to the tile
};

struct __align__(16) BuildSmem {
  uint8_t win[kWin3];
  uint8_t sout[kStrStage];    // the string-buffer bytes of 32 strings
  QEntry sq[kQueue2];         // strings awaiting output
  uint64_t front[kFrontSmem];  // the first frontier slots of the tile
  uint16_t open[kOpenSmem2];
  uint64_t mbar;
};
static_assert(sizeof(BuildSmem) % 16 == 0 && kWin3 % 16 == 0 && kStrStage % 16 == 0,
              "per-warp staging stays 16-byte aligned");

// Grammar (Sec. 3.2, RFC 8259): which previous tokens may precede a token of
// kind k inside an object (obj) or an array.  Bit c of the row is the class
// of the previous token: its kind, or kKeyStr for a string that is an object
// key.
constexpr uint32_t kKeyStr = 12;
__device__ __forceinline__ uint16_t grammar_row(uint32_t k, bool obj) {
  const uint32_t value_end = (1u << K_NUMBER) | (1u << K_TRUE) | (1u << K_FALSE) | (1u << K_NULL) |
                             (1u << K_CLOSE_OBJ) | (1u << K_CLOSE_ARR) | (1u << K_STRING);
  const uint32_t elem = (1u << K_OPEN_ARR) | (1u << K_COMMA);  // a value starts in an array
  switch (k) {
    case K_CLOSE_OBJ: return (uint16_t)(obj ? ((1u << K_OPEN_OBJ) | value_end) : 0u);
    case K_CLOSE_ARR: return (uint16_t)(obj ? 0u : ((1u << K_OPEN_ARR) | value_end));
    case K_COMMA: return (uint16_t)value_end;
    case K_COLON: return (uint16_t)(obj ? (1u << kKeyStr) : 0u);
    case K_STRING:
      return (uint16_t)(obj ? ((1u << K_OPEN_OBJ) | (1u << K_COMMA) | (1u << K_COLON)) : elem);
    case K_OPEN_OBJ: case K_OPEN_ARR: case K_NUMBER: case K_TRUE: case K_FALSE: case K_NULL:
      return (uint16_t)(obj ? (1u << K_COLON) : elem);
    default: return 0;
  }
}

// One string's buffer entry (u32 length, its n normalised bytes from src,
// NUL) at o, byte by byte.
__device__ __forceinline__ void put_string(uint8_t *__restrict__ o, uint32_t n,
                                           const uint8_t *__restrict__ src) {
  o[0] = (uint8_t)n; o[1] = (uint8_t)(n >> 8); o[2] = (uint8_t)(n >> 16); o[3] = (uint8_t)(n >> 24);
#pragma unroll 4
  for (uint32_t i = 0; i < n; i++) o[4 + i] = src[i];
  o[4 + n] = 0;
}

// put_string within shared memory, the source with at least 3 readable bytes
// past its end: bytes until the destination is word aligned, then whole
// words (two aligned source words and a funnel shift), then the tail.
__device__ __forceinline__ void put_string_smem(uint8_t *__restrict__ o, uint32_t n,
                                                const uint8_t *__restrict__ src) {
  o[0] = (uint8_t)n; o[1] = (uint8_t)(n >> 8); o[2] = (uint8_t)(n >> 16); o[3] = (uint8_t)(n >> 24);
  uint8_t *dst = o + 4;
  uint32_t i = 0;
  while (i < n && ((uintptr_t)(dst + i) & 3u)) {
    dst[i] = src[i];
    i++;
  }
  if (i + 4 <= n) {
    const uintptr_t sa = (uintptr_t)(src + i);
    const uint32_t *sw = reinterpret_cast<const uint32_t *>(sa & ~(uintptr_t)3);
    const uint32_t sh = (uint32_t)(sa & 3u) * 8;
    uint32_t lo = sw[0];
    for (; i + 4 <= n; i += 4) {
      const uint32_t hi = sw[1];
      *reinterpret_cast<uint32_t *>(dst + i) = sh ? __funnelshift_r(lo, hi, sh) : lo;
      lo = hi;
      sw++;
    }
  }
  for (; i < n; i++) dst[i] = src[i];
  dst[n] = 0;
}

// A string with escapes, normalised into o + 4 (with its length word and
// NUL): walked in the staged window when it ends there, else in global memory.
__device__ __forceinline__ void put_walked(uint8_t *o, uint32_t n, const Window &win,
                                           uint64_t p0, uint64_t len) {
  o[0] = (uint8_t)n; o[1] = (uint8_t)(n >> 8); o[2] = (uint8_t)(n >> 16); o[3] = (uint8_t)(n >> 24);
  int err = 1;
  if (p0 >= win.lo && p0 < win.hi) {
    const uint8_t *sp = win.s + ((int64_t)p0 - win.sbase);
    string_walk8<true>(sp, sp + (win.hi - p0), err, o + 4);
  }
  if (err) string_walk8<true>(win.g + p0, win.g + len, err, o + 4);
  o[4 + n] = 0;
}

// ---- the frontier -------------------------------------------------------------
// Nearest tile c in [j_min, from] with low(c) < L, or -1.  A tile's published
// jump pointer (the nearest earlier tile with a lower `low`) skips every tile
// between when its own low is >= L.
__device__ int64_t nearest_lower(const Job &J, int64_t from, int64_t j_min, int32_t L, uint32_t ep,
                                 int lane) {
  int64_t c = from;
  while (c >= j_min) {
    const int64_t cc = c - lane;
    const bool in = cc >= j_min;
    const int32_t lw = in ? J.pre2[cc].low : 0;
    const bool hit = in && lw < L;
    bool pub = false;
    uint32_t jv = kNoTile;
    if (in && !hit) {
      const uint64_t v = ld_acquire(&J.jump[cc]);
      pub = (uint32_t)(v >> 32) == ep;
      jv = (uint32_t)v;
    }
    const unsigned hm = __ballot_sync(0xFFFFFFFFu, hit), m = hm | __ballot_sync(0xFFFFFFFFu, pub);
    if (!m) {
      c -= 32;
      continue;
    }
    const int k = __ffs(m) - 1;
    if ((hm >> k) & 1u) return c - k;
    const uint32_t jt = __shfl_sync(0xFFFFFFFFu, jv, k);
    if (jt == kNoTile) return -1;
    c = (int64_t)jt;
  }
  return -1;
}

// ---- the build pass -------------------------------------------------------------
__global__ void __launch_bounds__(32 * kBWarps) build_kernel(const Job *__restrict__ job) {
  const Job &J = *job;
  __shared__ BuildSmem WS[kBWarps];
  __shared__ uint16_t s_gram[32];
  __shared__ uint8_t s_kind[256];
  const int lane = threadIdx.x & 31;
  const uint32_t wid = threadIdx.x >> 5;
  BuildSmem &W = WS[wid];
  if (threadIdx.x < 32) s_gram[threadIdx.x] = grammar_row(threadIdx.x >> 1, threadIdx.x & 1);
  for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) s_kind[i] = token_kind((uint8_t)i);
  for (uint32_t i = lane; i < kOpenSmem2; i += 32) W.open[i] = 0;
  mbar_init(&W.mbar, lane);
  __syncthreads();
  const uint32_t n_tiles = J.counters[kCtrTiles];
  const uint32_t ep = J.epoch;
  const uint32_t max_depth = J.max_depth;
  const uint32_t gw = blockIdx.x * kBWarps + wid, nw = gridDim.x * kBWarps;
  uint16_t *const open_g = J.open_g + (uint64_t)gw * kOpenGlobal;
  uint32_t phase = 0;
  TileTickets tix(J, kCtrTicketBuild, n_tiles, gw, nw, lane);
  for (uint32_t t = tix.first(); t < n_tiles; t = tix.next()) {
    tix.draw();  // the next tile, read at the loop's end
    const uint32_t d = doc_of_tile(J, t);
    const uint32_t j_min = J.tile_first[d];
    const uint32_t tt = t - j_min;
    const uint32_t nidx = J.doc_nidx[d];
    if ((J.doc_flags[d] & kDocBad) || nidx == 0) continue;
    const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
    const uint8_t *doc = J.base + J.doc_off[d];
    const uint64_t ib = idx_base(J, d);
    uint64_t *tape = J.tape + tape_base(J, d);
    uint8_t *strs = J.strings + str_base(J, d);
    const uint64_t tape_cap = len + 3;
    const uint32_t tape_cap32 = (uint32_t)min(tape_cap, (uint64_t)0xFFFFFFFFu);
    const uint64_t str_cap = str_base(J, d + 1) - str_base(J, d);
    const uint32_t cnt = J.tile_cnt[t], off = J.tile_off[t];
    const S2Pre pre = J.pre2[t];
    const uint64_t t0 = (uint64_t)tt * kTileBytes;

    // the tile's bytes (and kBPost more), copied while the frontier is found
    uintptr_t a0, a1;
    window_extent(doc, len, t0, t0 + kTileBytes + kBPost, a0, a1);
    if (lane == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    bulk_copy_start(W.win, a0, (uint32_t)(a1 - a0), &W.mbar, lane);

    // ---- frontier: the container open at each level in [max(1, low), d_start]
    // entering the tile, deepest first: (object << 63) | its opener's tape index,
    // or ~0 when there is none (an invalid document)
    const int32_t flo = max(1, pre.low), fhi = pre.d_start;
    uint64_t *front = J.front + ib + off + t;
    int64_t from = (int64_t)t - 1;
    bool none = false;
    for (int32_t lev = fhi; lev >= flo;) {
      const int64_t c = nearest_lower(J, from, j_min, lev, ep, lane);
      if (c < 0) {
        for (int32_t L = lev - lane; L >= flo; L -= 32) {
          const uint32_t fk = (uint32_t)(fhi - L);
          if (fk < kFrontSmem) W.front[fk] = ~0ull; else front[fk] = ~0ull;
        }
        none = true;
        break;
      }
      const S2Pre cp = J.pre2[c];
      const int32_t bottom = max(flo, cp.low + 1);
      const uint32_t *sv = J.surv + ib + J.tile_off[c];
      for (int32_t L = lev - lane; L >= bottom; L -= 32) {
        const uint32_t e = sv[L - cp.low - 1];
        const uint64_t v = ((uint64_t)(e >> 31) << 63) | (cp.tape_start + (e & 0xFFFFu));
        const uint32_t fk = (uint32_t)(fhi - L);
        if (fk < kFrontSmem) W.front[fk] = v; else front[fk] = v;
      }
      lev = bottom - 1;
      from = c;
    }
    {  // this tile's jump pointer, for the walks of later tiles
      const int64_t jp = none ? -1 : nearest_lower(J, from, j_min, pre.low, ep, lane);
      if (lane == 0)
        st_release(&J.jump[t], ((uint64_t)ep << 32) | (jp < 0 ? kNoTile : (uint32_t)jp));
    }
    __syncwarp();

    // kinds of the two tokens before the tile
    uint8_t prev1 = K_OTHER, prev2 = K_OTHER;
    if (lane < 2 && off >= (uint32_t)lane + 1) {
      const uint8_t k = s_kind[doc[J.idx[ib + off - 1 - lane]]];
      if (lane == 0) prev1 = k; else prev2 = k;
    }
    prev1 = __shfl_sync(0xFFFFFFFFu, prev1, 0);
    prev2 = __shfl_sync(0xFFFFFFFFu, prev2, 1);

    if (!bulk_copy_wait(&W.mbar, phase)) atomicOr(&J.doc_flags[d], kFlagInternal);
    phase ^= 1u;
    Window win;
    win.s = W.win;
    win.sbase = (int64_t)(a0 - (uintptr_t)doc);
    win.lo = t0;
    win.hi = min(len, (uint64_t)(a1 - (uintptr_t)doc));
    win.g = doc;

    const OpenTable ot = cnt < (uint32_t)kOpenSmem2 ? OpenTable{W.open, (uint32_t)kOpenSmem2 - 1u, 0}
                                                      : OpenTable{open_g, 0xFFFFFFFFu, kLevelOff2};
    const uint32_t *slen = J.slen + ib + off;
    uint32_t shead = 0, stail = 0;
    uint64_t str_run = pre.str_start;  // buffer offset of the next queued string

    // strings (Sec. 3.2.2), 32 at a time: their entries are contiguous in the
    // buffer, so they are built in shared memory and copied out coalesced
    auto flush_strings = [&]() {
      const uint32_t m = min(32u, stail - shead);
      const bool have = (uint32_t)lane < m;
      QEntry e{0, 0, 0};
      uint32_t sl = 0;
      if (have) {
        e = W.sq[(shead + lane) & (kQueue2 - 1)];
        sl = slen[shead + lane];
      }
      const bool bad = have && (sl & kSlenErr);
      if (bad) report(J, d, (uint64_t)off + e.j, (int)(sl & 0xFFu));
      const bool is_str = have && !bad;
      const bool walk = (sl & kSlenWalk) != 0;
      const uint64_t p0 = t0 + e.pos + 1;
      uint64_t n = sl & kSlenLen;
      if (is_str && n == kSlenLen) {  // too long for the entry: measure again
        int err;
        n = string_walk<false>(doc + p0, doc + len, err, nullptr);
      }
      const uint64_t size = have ? (bad ? 5ull : 5ull + n) : 0ull;
      const uint64_t incl = warp_incl_u64(size, lane);
      const uint64_t so = str_run + incl - size;
      const uint64_t tp = (uint64_t)pre.tape_start + e.tp;
      if (is_str && tp < tape_cap) tape[tp] = ((uint64_t)'"' << 56) | so;
      const unsigned sm = __ballot_sync(0xFFFFFFFFu, is_str);
      if (sm) {
        const uint64_t so_lo = __shfl_sync(0xFFFFFFFFu, so, __ffs(sm) - 1);
        const uint64_t so_hi = __shfl_sync(0xFFFFFFFFu, so + 5 + n, 31 - __clz(sm));
        const uint32_t a = (uint32_t)((uintptr_t)(strs + so_lo) & 15u);
        const uint64_t total = a + (so_hi - so_lo);
        const bool staged = total <= (uint64_t)kStrStage && so_hi <= str_cap;
        // a string is assembled in shared memory when its source is there too
        const bool here = is_str && staged && (walk || win.has(p0, p0 + n));
        if (here) {
          uint8_t *o = W.sout + a + (so - so_lo);
          if (walk) put_walked(o, (uint32_t)n, win, p0, len);
          else put_string_smem(o, (uint32_t)n, win.s + ((int64_t)p0 - win.sbase));
        }
        __syncwarp();
        if (staged) {
          uint8_t *gb = strs + so_lo - a;  // 16-byte aligned
          const uint32_t units = (uint32_t)((total + 15) >> 4);
          for (uint32_t u = lane; u < units; u += 32) {
            const uint32_t lo = u << 4, hi = lo + 16;
            if (lo >= a && hi <= total) {
              *reinterpret_cast<uint4 *>(gb + lo) = *reinterpret_cast<const uint4 *>(W.sout + lo);
            } else {
              for (uint32_t i = max(lo, a); i < min(hi, (uint32_t)total); i++) gb[i] = W.sout[i];
            }
          }
          __syncwarp();
        }
        if (is_str && !here && so + 5 + n <= str_cap) {  // written in place
          if (walk) put_walked(strs + so, (uint32_t)n, win, p0, len);
          else put_string(strs + so, (uint32_t)n, win.ptr(p0, p0 + n));
        }
      }
      str_run += __shfl_sync(0xFFFFFFFFu, incl, 31);
      shead += m;
      __syncwarp();
    };

    // positions of the tile's tokens, one chunk loaded ahead
    const uint32_t *idxp = J.idx + ib + off;
    uint32_t pos_next = (uint32_t)lane < cnt ? idxp[lane] : 0u;
    int32_t depth = 0, mn = 0, mx = 0;
    uint32_t tape_rel = 0;
    for (uint32_t b0 = 0; b0 < cnt; b0 += 32) {
      const uint32_t j = b0 + lane;
      const bool valid = j < cnt;
      const uint32_t pos = pos_next;
      pos_next = j + 32 < cnt ? idxp[j + 32] : 0u;
      const uint8_t k = valid ? s_kind[W.win[(int64_t)pos - win.sbase]] : K_OTHER;
      // depth and tape slot: one scan over (delta + 1) | words << 8
      const int32_t dl = depth_delta(k);
      const uint32_t wd = tape_words_of(k);
      const uint32_t vi = warp_incl_u32((uint32_t)(dl + 1) | (wd << 8), lane);
      const int32_t D = depth + (int32_t)(vi & 0xFFu) - (lane + 1);
      const int32_t E = D - dl;
      const uint32_t trel = tape_rel + (vi >> 8) - wd;
      if (valid) {
        mn = min(mn, min(E, D));
        mx = max(mx, max(E, D));
      }
      // Enclosing container: depth moves by at most one per token, so it is
      // the last earlier token whose depth-before is smaller (an opener at
      // E - 1).  Found by a descent over window minima of E; when no token of
      // this chunk qualifies, the level table holds it (or, for levels the
      // tile started inside, the frontier).
      const bool op = valid && is_open(k);
      const uint16_t my = op ? (uint16_t)(0x8000u | (k == K_OPEN_OBJ ? 0x4000u : 0u) | trel) : 0;
      int32_t m1 = valid ? E : 0x7FFFFFFF, m2, m4, m8, m16, u;
      u = __shfl_up_sync(0xFFFFFFFFu, m1, 1);  m2 = lane >= 1 ? min(m1, u) : m1;
      u = __shfl_up_sync(0xFFFFFFFFu, m2, 2);  m4 = lane >= 2 ? min(m2, u) : m2;
      u = __shfl_up_sync(0xFFFFFFFFu, m4, 4);  m8 = lane >= 4 ? min(m4, u) : m4;
      u = __shfl_up_sync(0xFFFFFFFFu, m8, 8);  m16 = lane >= 8 ? min(m8, u) : m8;
      // mK at lane i: minimum of E over [i - K + 1, i] (clipped at lane 0)
      int32_t at = lane - 1;
      u = __shfl_sync(0xFFFFFFFFu, m16, max(at, 0));
      if (at >= 0 && u >= E) at -= 16;
      u = __shfl_sync(0xFFFFFFFFu, m8, max(at, 0));
      if (at >= 0 && u >= E) at -= 8;
      u = __shfl_sync(0xFFFFFFFFu, m4, max(at, 0));
      if (at >= 0 && u >= E) at -= 4;
      u = __shfl_sync(0xFFFFFFFFu, m2, max(at, 0));
      if (at >= 0 && u >= E) at -= 2;
      u = __shfl_sync(0xFFFFFFFFu, m1, max(at, 0));
      if (at >= 0 && u >= E) at -= 1;
      uint16_t parent = (uint16_t)__shfl_sync(0xFFFFFFFFu, (uint32_t)my, max(at, 0));
      if (at < 0) parent = (valid && E > -kLevelOff2 && E <= kLevelOff2) ? ot.at(E) : (uint16_t)0;
      // the last opener of each level of this chunk stays open for later tokens
      const unsigned grp = __match_any_sync(0xFFFFFFFFu, op ? D : 0x7FFFFFFF);
      if (op && lane == 31 - __clz(grp)) ot.at(D) = my;

      uint8_t p = __shfl_up_sync(0xFFFFFFFFu, k, 1);
      uint8_t pp = __shfl_up_sync(0xFFFFFFFFu, k, 2);
      if (lane == 0) { p = prev1; pp = prev2; }
      if (lane == 1) pp = prev1;
      prev2 = __shfl_sync(0xFFFFFFFFu, k, 30);
      prev1 = __shfl_sync(0xFFFFFFFFu, k, 31);
      const uint32_t g = off + j;
      const int32_t Ea = pre.d_start + E;  // absolute depth before the token
      const uint32_t tp = pre.tape_start + trel;

      // ---- grammar: the enclosing container and the previous two tokens ----
      uint8_t K = 0;
      uint32_t par_tape = 0xFFFFFFFFu;
      bool par_ok = true;
      if (Ea >= 1) {
        if (parent) {
          K = (parent & 0x4000u) ? K_OPEN_OBJ : K_OPEN_ARR;
          par_tape = pre.tape_start + (parent & 0x0FFFu);
        } else if (Ea >= flo && Ea <= fhi) {
          const uint32_t fk = (uint32_t)(fhi - Ea);
          const uint64_t ent = fk < kFrontSmem ? W.front[fk] : front[fk];
          if (ent != ~0ull) {
            K = (ent >> 63) ? K_OPEN_OBJ : K_OPEN_ARR;
            par_tape = (uint32_t)ent;
          } else {
            par_ok = false;
          }
        } else {
          par_ok = false;
        }
      }
      int code = 0;
      if (Ea <= 0) {
        if (!(g == 0 && is_value_start(k))) code = SJ_TAPE_ERROR;
      } else if (!par_ok) {
        code = SJ_TAPE_ERROR;
      } else {
        const bool obj = K == K_OPEN_OBJ;
        const uint32_t pc = (p == K_STRING && obj && pp != K_COLON) ? kKeyStr : p;
        if (!((s_gram[(k << 1) | (obj ? 1 : 0)] >> pc) & 1u)) code = SJ_TAPE_ERROR;
      }
      if (!code && is_open(k) && Ea + 1 > (int32_t)max_depth) code = SJ_DEPTH_ERROR;

      // ---- tape words of containers and atoms; strings are queued, numbers
      // are written by the numbers kernel.  Content is checked even where the
      // grammar failed: a grammar code is smaller than any content code, so
      // the minimum keeps the grammar first.
      if (valid) {
        if (is_close(k)) {
          if (!code && tp < tape_cap32 && par_tape < tape_cap32) {
            tape[tp] = ((uint64_t)(k == K_CLOSE_OBJ ? '}' : ']') << 56) | par_tape;
            tape[par_tape] = ((uint64_t)(k == K_CLOSE_OBJ ? '{' : '[') << 56) | (uint64_t)(tp + 1);
          }
        } else if (is_atom(k)) {
          // the literal and the byte after it: one 8-byte window of the staged
          // tile (two aligned words and a funnel shift), else byte by byte
          const uint32_t nlit = k == K_FALSE ? 5 : 4;
          const uint64_t lit = k == K_TRUE ? 0x65757274ull : (k == K_FALSE ? 0x65736C6166ull : 0x6C6C756Eull);
          bool ok = pos + nlit <= len;
          if (ok) {
            if (pos + 8 <= win.hi) {
              const uintptr_t ua = (uintptr_t)(win.s + ((int64_t)pos - win.sbase));
              const uint32_t *wp = reinterpret_cast<const uint32_t *>(ua & ~(uintptr_t)3);
              const uint32_t sh = (uint32_t)(ua & 3u) * 8;
              const uint64_t x = ((uint64_t)__funnelshift_r(wp[1], wp[2], sh) << 32) |
                                 __funnelshift_r(wp[0], wp[1], sh);
              ok = (x & ((1ull << (8 * nlit)) - 1)) == lit &&
                   (pos + nlit >= len || is_terminator((uint8_t)(x >> (8 * nlit))));
            } else {
              for (uint32_t i = 0; ok && i < nlit; i++) ok = win.at(pos + i) == (uint8_t)(lit >> (8 * i));
              if (ok && pos + nlit < len) ok = is_terminator(win.at(pos + nlit));
            }
          }
          if (!ok) { if (!code) code = k == K_TRUE ? SJ_T_ATOM_ERROR : (k == K_FALSE ? SJ_F_ATOM_ERROR : SJ_N_ATOM_ERROR); }
          else if (tp < tape_cap32) tape[tp] = (uint64_t)(uint8_t)lit << 56;
        }
        if (code) report(J, d, g, code);
      }
      {
        const bool isstr = valid && k == K_STRING;
        const unsigned sm = __ballot_sync(0xFFFFFFFFu, isstr);
        if (isstr) W.sq[(stail + __popc(sm & ((1u << lane) - 1u))) & (kQueue2 - 1)] =
            QEntry{pos - (uint32_t)t0, j, trel};
        stail += __popc(sm);
      }
      const uint32_t tot = __shfl_sync(0xFFFFFFFFu, vi, 31);
      depth += (int32_t)(tot & 0xFFu) - 32;
      tape_rel += tot >> 8;
      __syncwarp();
      if (stail - shead >= 32) flush_strings();
    }
    while (shead != stail) flush_strings();
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
      mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    }
    // forget this tile's levels
    for (int32_t v = max(mn, -kLevelOff2) + lane; v <= min(mx, kLevelOff2); v += 32) ot.at(v) = 0;
    __syncwarp();  // every lane is done with this tile's shared memory
  }
}

// ---------------------------------------------------------------------------
// Numbers (Sec. 3.2.1): each warp gathers the number tokens listed by the
// first pass for its tiles into a queue and converts them 32 at a time, one
// lane per number (a tile holds too few to fill a warp).  Each lane copies its
// lexeme and the byte after it (at most kNumWindow bytes, in 16-byte chunks)
// into shared memory and converts it there; longer lexemes are read in place.
// The tag ('l' or 'd') and the value go to the token's two tape words, an
// error to the document's error minimum.
constexpr int kNumWindow = 48;
constexpr int kNumThreads = 128;
struct NumEntry {
  uint32_t pos;  // document position
  uint32_t nxt;  // the next token's position, or the document's end
  uint32_t g;    // token index in the document
  uint32_t tp;   // tape slot
  uint32_t d;    // document
};
__global__ void __launch_bounds__(kNumThreads) numbers_kernel(const Job *__restrict__ job) {
  const Job &J = *job;
  __shared__ __align__(16) uint8_t win[kNumThreads][kNumWindow + 16];
  __shared__ NumEntry q[kNumThreads / 32][64];
  const int lane = threadIdx.x & 31;
  uint8_t *my = win[threadIdx.x];
  NumEntry *wq = q[threadIdx.x >> 5];
  uint32_t head = 0, tail = 0;
  auto flush = [&]() {
    const uint32_t m = min(32u, tail - head);
    if ((uint32_t)lane < m) {
      const NumEntry e = wq[(head + lane) & 63u];
      const uint64_t len = J.doc_off[e.d + 1] - J.doc_off[e.d];
      const uint8_t *doc = J.base + J.doc_off[e.d];
      const uint64_t pos = e.pos, nxt = e.nxt;
      const uint64_t wend = min(len, pos + kNumWindow);
      uint8_t tag = 0;
      uint64_t v = 0;
      int nc;
      if (nxt < wend || (nxt == len && len <= wend)) {  // lexeme and terminator fit the window
        const uintptr_t g0 = (uintptr_t)(doc + pos), a0 = g0 & ~(uintptr_t)15;
        const uintptr_t gend = (uintptr_t)(doc + wend);
        for (uintptr_t c = a0; c < gend; c += 16)
          *reinterpret_cast<uint4 *>(my + (c - a0)) = __ldg(reinterpret_cast<const uint4 *>(c));
        const uint8_t *sp = my + (g0 - a0);
        nc = parse_number(sp, sp + (wend - pos), tag, v);
      } else {
        nc = parse_number(doc + pos, doc + len, tag, v);
      }
      const uint64_t tape_cap = len + 3;
      if (nc) {
        report(J, e.d, e.g, nc);
      } else if ((uint64_t)e.tp + 1 < tape_cap) {
        uint64_t *tape = J.tape + tape_base(J, e.d);
        tape[e.tp] = (uint64_t)tag << 56;
        tape[e.tp + 1] = v;
      }
    }
    head += m;
    __syncwarp();
  };
  const uint32_t n_tiles = J.counters[kCtrTiles];
  TileTickets tix(J, kCtrTicketNum, n_tiles, blockIdx.x * (kNumThreads / 32) + (threadIdx.x >> 5),
                  gridDim.x * (kNumThreads / 32), lane);
  for (uint32_t t = tix.first(); t < n_tiles; t = tix.next()) {
    tix.draw();
    const uint32_t d = doc_of_tile(J, t);
    const uint32_t nidx = J.doc_nidx[d];
    if ((J.doc_flags[d] & kDocBad) || nidx == 0) continue;
    const uint32_t m = J.tile_nnum[t];
    if (m == 0) continue;
    const uint64_t ib = idx_base(J, d);
    const uint32_t off = J.tile_off[t];
    const uint32_t tape_start = J.pre2[t].tape_start;
    const uint32_t t0 = (t - J.tile_first[d]) * (uint32_t)kTileBytes;
    const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
    for (uint32_t k0 = 0; k0 < m; k0 += 32) {
      const uint32_t k = k0 + lane;
      const uint32_t c = min(32u, m - k0);
      if ((uint32_t)lane < c) {
        const uint64_t e = J.nlist[ib + off + k];
        const uint32_t pos = t0 + (uint32_t)(e & 0xFFFFu);
        const uint32_t j = (uint32_t)(e >> 16) & 0xFFFFu;
        const uint32_t span = (uint32_t)(e >> 48);
        const uint32_t g = off + j;
        const uint32_t nxt = span ? pos + span : (g + 1 < nidx ? J.idx[ib + g + 1] : (uint32_t)len);
        wq[(tail + lane) & 63u] = NumEntry{pos, nxt, g, tape_start + ((uint32_t)(e >> 32) & 0xFFFFu), d};
      }
      tail += c;
      __syncwarp();
      if (tail - head >= 32) flush();
    }
  }
  while (head != tail) flush();
}

}  // namespace sj
