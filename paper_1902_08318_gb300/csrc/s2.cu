// s2.cu -- stage 2 of the parser (Sec. 3.2) on sm_103a, reduce-then-scan form.
//
// The paper walks the indices with a goto state machine and a stack of open
// scopes.  Here a thread block takes the indices of one stage-1 tile (at most
// 2048) and replaces the walk with prefix sums and searches:
//   stage2_reduce_kernel  per tile: token kinds, the +1/-1 depth sum and its
//                         minimum, tape words, normalised string lengths, and
//                         the containers the tile leaves open (by level);
//   (scan.cu)             segmented scans give every tile its absolute depth,
//                         first tape slot and string-buffer offset, and the
//                         open container of every level entering it;
//   stage2_build_kernel   per tile: each token's enclosing container (in the
//                         tile, found in shared memory, or from the frontier),
//                         the grammar check against the previous two tokens
//                         and that container, and the tape words; numbers are
//                         converted and strings normalised into the buffer.
// The first failing token of a document (smallest index; grammar before
// content at one token) gives its error code (an atomic minimum).
#include "number.cuh"
#include "sj_internal.cuh"
#include "strings.cuh"

namespace sj {

constexpr uint32_t kDocBad = kFlagUtf8 | kFlagUnclosed | kFlagCapacity | kFlagInternal;

__device__ __forceinline__ void report(const Job &J, uint32_t d, uint64_t token, int code) {
  atomicMin(&J.doc_err[d], (unsigned long long)((token << 8) | (uint64_t)code));
}

// ---- one warp per tile ---------------------------------------------------
constexpr int kS2Warps = kS2Threads / 32;
constexpr int kHalo = 1024;                    // staged bytes past the tile's end
constexpr int kStageBytes = kTileBytes + kHalo;
constexpr int kLevelOff = kMaxTileTokens;      // relative levels [-2048, 2048]

// Per-warp shared state.  `open[l]` is the container currently open at
// relative level l (levels are depths after an opener, relative to the tile
// start), written by openers of this tile: 0 = none, else bit 15 set,
// bit 14 = object, bits 0-11 = the opener's tape slot relative to the tile.
struct __align__(16) WarpSmem {  // 16-byte aligned size: bytes[] of every warp takes uint4 stores
  uint8_t bytes[kStageBytes + 64];
  uint16_t open[2 * kMaxTileTokens + 1];
};
static_assert(sizeof(WarpSmem) % 16 == 0, "per-warp staging must stay 16-byte aligned");

__device__ __forceinline__ uint32_t warp_incl_u32(uint32_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}
__device__ __forceinline__ int32_t warp_incl_i32(int32_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Staged view of the document around one tile.
struct Staged {
  const uint8_t *doc;   // global
  uint64_t len;
  int64_t sbase;        // document position of bytes[0]
  uint64_t slimit;      // first document position not staged
  const uint8_t *smem;
  __device__ __forceinline__ uint8_t at(uint64_t p) const {
    return (p < slimit && (int64_t)p >= sbase) ? smem[p - sbase] : doc[p];
  }
  // pointer for reading [p, q): shared memory when staged, else global
  __device__ __forceinline__ const uint8_t *ptr(uint64_t p, uint64_t q) const {
    return (q <= slimit && (int64_t)p >= sbase) ? smem + (p - sbase) : doc + p;
  }
};

__device__ __forceinline__ Staged stage_tile(WarpSmem &W, const uint8_t *doc, uint64_t len,
                                             uint64_t t0, int lane) {
  const uintptr_t g0 = (uintptr_t)(doc + t0);
  const uintptr_t a0 = g0 & ~(uintptr_t)15;
  const uintptr_t dend = (uintptr_t)doc + len;
  const uintptr_t send = min((uintptr_t)(a0 + kStageBytes), dend);
  const uint32_t nch = (uint32_t)((send - a0 + 15) / 16);
  for (uint32_t c = lane; c < nch; c += 32)
    reinterpret_cast<uint4 *>(W.bytes)[c] = __ldg(reinterpret_cast<const uint4 *>(a0 + 16 * c));
  __syncwarp();
  Staged v;
  v.doc = doc;
  v.len = len;
  v.sbase = (int64_t)t0 - (int64_t)(g0 - a0);
  v.slimit = (uint64_t)((int64_t)t0 + (int64_t)(send - g0));
  v.smem = W.bytes;
  return v;
}

// Tokens of one tile, 32 at a time: positions, kinds, depths, tape slots and
// the enclosing container of each token (from the warp's level table, or -1
// when it was opened before the tile).
struct Chunk {
  uint32_t j;       // token index in the tile
  bool valid;
  uint32_t pos, next;
  uint8_t kind;
  int32_t E, D;     // relative depth before / after the token
  uint32_t tape;    // relative tape slot
  uint32_t sord;    // string ordinal in the tile (strings before this token)
  uint16_t parent;  // open[] entry of the enclosing container, 0 = before the tile
};

struct TileWalk {
  int32_t depth = 0, dmin = 0, dmax = 0;
  uint32_t tape = 0, nstr = 0;
  uint32_t pos_next = 0;  // first position of the next chunk

  __device__ __forceinline__ void begin(const uint32_t *idxp, uint32_t off, uint32_t cnt,
                                        uint32_t nidx, uint64_t len, int lane) {
    const uint32_t j = lane;
    pos_next = j < cnt ? idxp[off + j] : 0u;
    (void)nidx;
    (void)len;
  }

  __device__ __forceinline__ void next(Chunk &c, WarpSmem &W, const Staged &sv, const uint32_t *idxp,
                                       uint32_t off, uint32_t cnt, uint32_t nidx, uint64_t len,
                                       uint32_t base, int lane) {
    c.j = base + lane;
    c.valid = c.j < cnt;
    c.pos = pos_next;
    // prefetch the next chunk
    const uint32_t jn = base + 32 + lane;
    pos_next = jn < cnt ? idxp[off + jn] : 0u;
    uint32_t nx = __shfl_down_sync(0xFFFFFFFFu, c.pos, 1);
    const uint32_t first_next = __shfl_sync(0xFFFFFFFFu, pos_next, 0);
    if (lane == 31 || c.j + 1 == cnt) {
      const uint32_t g = off + c.j + 1;  // document index of the next token
      nx = (c.j + 1 < cnt) ? first_next : (g < nidx ? idxp[g] : (uint32_t)len);
    }
    c.next = nx;
    c.kind = c.valid ? token_kind(sv.at(c.pos)) : K_OTHER;
    const int32_t dl = c.valid ? depth_delta(c.kind) : 0;
    const int32_t di = warp_incl_i32(dl, lane);
    c.D = depth + di;
    c.E = c.D - dl;
    const uint32_t w = c.valid ? tape_words_of(c.kind) : 0u;
    const uint32_t wi = warp_incl_u32(w, lane);
    c.tape = tape + wi - w;
    const uint32_t si = __ballot_sync(0xFFFFFFFFu, c.valid && c.kind == K_STRING);
    c.sord = nstr + __popc(si & ((1u << lane) - 1u));
    // parents: the last opener of this chunk at the token's level, else the table
    const bool op = c.valid && is_open(c.kind);
    uint16_t my = op ? (uint16_t)(0x8000u | (c.kind == K_OPEN_OBJ ? 0x4000u : 0u) | c.tape) : 0;
    c.parent = 0;
    unsigned pending = __ballot_sync(0xFFFFFFFFu, c.valid);
    const unsigned below = (1u << lane) - 1u;
    while (pending) {
      const int32_t lv = __shfl_sync(0xFFFFFFFFu, c.E, __ffs(pending) - 1);
      const unsigned opl = __ballot_sync(0xFFFFFFFFu, op && c.D == lv);
      const bool mine = ((pending >> lane) & 1u) && c.E == lv;
      const unsigned m = opl & below;
      const int src = (mine && m) ? 31 - __clz(m) : lane;
      const uint16_t got = (uint16_t)__shfl_sync(0xFFFFFFFFu, (uint32_t)my, src);
      if (mine) {
        if (m) c.parent = got;
        else if (lv > -kLevelOff && lv <= kLevelOff) c.parent = W.open[lv + kLevelOff];
      }
      pending &= ~__ballot_sync(0xFFFFFFFFu, mine);
    }
    // the last opener of each level of this chunk stays open for later tokens
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, op ? c.D : 0x7FFFFFFF);
    if (op && lane == 31 - __clz(grp)) W.open[c.D + kLevelOff] = my;
    // advance
    depth += __shfl_sync(0xFFFFFFFFu, di, 31);
    tape += __shfl_sync(0xFFFFFFFFu, wi, 31);
    nstr += __popc(si);
    int32_t mn = c.valid ? min(c.E, c.D) : 0x7FFFFFFF, mx = c.valid ? max(c.E, c.D) : -0x7FFFFFFF;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
      mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    }
    dmin = min(dmin, mn);
    dmax = max(dmax, mx);
    __syncwarp();
  }

  // forget this tile's levels
  __device__ __forceinline__ void clear(WarpSmem &W, int lane) {
    for (int32_t v = max(dmin, -kLevelOff) + lane; v <= min(dmax, kLevelOff); v += 32)
      W.open[v + kLevelOff] = 0;
    __syncwarp();
  }
};

// ---------------------------------------------------------------------------
// Stage-2 reduce: per tile, the depth change and lowest depth, tape words,
// string-buffer bytes (string lengths are stored for the build pass), and the
// containers left open at each level (the survivors).
__global__ void __launch_bounds__(kS2Threads) stage2_reduce_kernel(const Job *__restrict__ job) {
  const Job &J = *job;
  __shared__ WarpSmem WS[kS2Warps];
  const int lane = threadIdx.x & 31;
  WarpSmem &W = WS[threadIdx.x >> 5];
  for (uint32_t i = lane; i < 2 * kMaxTileTokens + 1; i += 32) W.open[i] = 0;
  __syncwarp();
  const uint32_t n_tiles = J.counters[2];
  const uint32_t warps = gridDim.x * kS2Warps;
  for (uint32_t t = blockIdx.x * kS2Warps + (threadIdx.x >> 5); t < n_tiles; t += warps) {
    const uint32_t d = doc_of_tile(J, t);
    const uint32_t tt = t - J.tile_first[d];
    const uint32_t nidx = J.doc_nidx[d];
    if ((J.doc_flags[d] & kDocBad) || nidx == 0) {
      if (lane == 0) J.s2_rec[t] = S2Agg{0, 0, 0, tt == 0, 0};
      continue;
    }
    const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
    const uint8_t *doc = J.base + J.doc_off[d];
    const uint64_t ib = idx_base(J, d);
    const uint32_t *idxp = J.idx + ib;
    const uint32_t cnt = J.tile_cnt[t], off = J.tile_off[t];
    const Staged sv = stage_tile(W, doc, len, (uint64_t)tt * kTileBytes, lane);
    TileWalk tw;
    tw.begin(idxp, off, cnt, nidx, len, lane);
    uint64_t sb = 0;
    for (uint32_t base = 0; base < cnt; base += 32) {
      Chunk c;
      tw.next(c, W, sv, idxp, off, cnt, nidx, len, base, lane);
      if (c.valid && c.kind == K_STRING) {  // normalised length (Sec. 3.2.2)
        int err;
        const uint64_t p0 = (uint64_t)c.pos + 1, p1 = c.next;
        const uint8_t *sp = sv.ptr(p0, p1);
        const uint32_t n = string_walk<false>(sp, sp + (p1 - p0), err, nullptr);
        J.slen[ib + off + c.j] = err ? (0x80000000u | (uint32_t)err) : n;
        sb += 5ull + (err ? 0 : n);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) sb += __shfl_xor_sync(0xFFFFFFFFu, sb, o);
    // survivors: the open container of each level in (dmin, depth]
    const int32_t lo = tw.dmin;
    for (int32_t lv = lo + 1 + lane; lv <= tw.depth; lv += 32) {
      const uint16_t e = W.open[lv + kLevelOff];
      J.surv[ib + off + (uint32_t)(lv - lo - 1)] = ((uint32_t)(e >> 14) & 1u) << 31 | (e & 0x0FFFu);
    }
    __syncwarp();
    tw.clear(W, lane);
    if (lane == 0) J.s2_rec[t] = S2Agg{tw.depth, lo, tw.tape, tt == 0, sb};
  }
}

// ---------------------------------------------------------------------------
// Stage-2 build: grammar, tape words, numbers and strings.
__global__ void __launch_bounds__(kS2Threads) stage2_build_kernel(const Job *__restrict__ job) {
  const Job &J = *job;
  __shared__ WarpSmem WS[kS2Warps];
  const int lane = threadIdx.x & 31;
  WarpSmem &W = WS[threadIdx.x >> 5];
  for (uint32_t i = lane; i < 2 * kMaxTileTokens + 1; i += 32) W.open[i] = 0;
  __syncwarp();
  const uint32_t n_tiles = J.counters[2];
  const uint32_t max_depth = J.max_depth;
  const uint32_t warps = gridDim.x * kS2Warps;
  for (uint32_t t = blockIdx.x * kS2Warps + (threadIdx.x >> 5); t < n_tiles; t += warps) {
    const uint32_t d = doc_of_tile(J, t);
    const uint32_t j_min = J.tile_first[d];
    const uint32_t tt = t - j_min;
    const uint32_t ntiles_d = J.tile_first[d + 1] - j_min;
    const uint32_t nidx = J.doc_nidx[d];
    if ((J.doc_flags[d] & kDocBad) || nidx == 0) continue;
    const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
    const uint8_t *doc = J.base + J.doc_off[d];
    const uint64_t ib = idx_base(J, d);
    const uint32_t *idxp = J.idx + ib;
    uint64_t *tape = J.tape + tape_base(J, d);
    uint8_t *strs = J.strings + str_base(J, d);
    const uint64_t tape_cap = len + 3;
    const uint64_t str_cap = str_base(J, d + 1) - str_base(J, d);
    const uint32_t cnt = J.tile_cnt[t], off = J.tile_off[t];
    const S2Pre pre = J.s2_pre[t];
    const S2Agg agg = J.s2_rec[t];
    const uint64_t *front = J.front + ib + off + t;

    if (tt == ntiles_d - 1 && lane == 0) {  // the document's last tile closes the tape
      const int32_t d_end = pre.d_start + agg.dd;
      const uint64_t T = (uint64_t)pre.tape_start + agg.w + 1;
      if (d_end != 0) report(J, d, nidx, SJ_TAPE_ERROR);
      if (T <= tape_cap) {
        tape[0] = ((uint64_t)'r' << 56) | (T - 1);
        tape[T - 1] = (uint64_t)'r' << 56;
      }
      J.doc_tape[d] = T;
      J.doc_str[d] = pre.str_start + agg.s;
    }

    const Staged sv = stage_tile(W, doc, len, (uint64_t)tt * kTileBytes, lane);
    TileWalk tw;
    tw.begin(idxp, off, cnt, nidx, len, lane);
    // kinds of the two tokens before the tile
    uint8_t prev1 = K_OTHER, prev2 = K_OTHER;
    if (lane < 2 && off >= (uint32_t)lane + 1) {
      const uint8_t k = token_kind(doc[idxp[off - 1 - lane]]);
      if (lane == 0) prev1 = k; else prev2 = k;
    }
    prev1 = __shfl_sync(0xFFFFFFFFu, prev1, 0);
    prev2 = __shfl_sync(0xFFFFFFFFu, prev2, 1);
    uint64_t str_run = pre.str_start;
    for (uint32_t base = 0; base < cnt; base += 32) {
      Chunk c;
      tw.next(c, W, sv, idxp, off, cnt, nidx, len, base, lane);
      const uint8_t k = c.kind;
      uint8_t p = __shfl_up_sync(0xFFFFFFFFu, k, 1);
      uint8_t pp = __shfl_up_sync(0xFFFFFFFFu, k, 2);
      if (lane == 0) { p = prev1; pp = prev2; }
      if (lane == 1) pp = prev1;
      prev2 = __shfl_sync(0xFFFFFFFFu, k, 30);
      prev1 = __shfl_sync(0xFFFFFFFFu, k, 31);
      // string-buffer offsets (token order)
      uint32_t sl = 0;
      if (c.valid && k == K_STRING) sl = J.slen[ib + off + c.j];
      const uint64_t ssz = (c.valid && k == K_STRING) ? 5ull + ((sl & 0x80000000u) ? 0 : sl) : 0;
      uint64_t sinc = ssz;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(0xFFFFFFFFu, sinc, o);
        if (lane >= o) sinc += u;
      }
      const uint64_t so = str_run + sinc - ssz;
      str_run += __shfl_sync(0xFFFFFFFFu, sinc, 31);
      if (!c.valid) continue;

      const uint64_t g = (uint64_t)off + c.j;
      const int32_t E = pre.d_start + c.E;
      uint8_t K = 0;
      uint64_t par_tape = ~0ull;
      bool par_ok = true;
      if (E >= 1) {
        if (c.parent) {
          K = (c.parent & 0x4000u) ? K_OPEN_OBJ : K_OPEN_ARR;
          par_tape = (uint64_t)pre.tape_start + (c.parent & 0x0FFFu);
        } else if (E >= max(1, pre.low) && E <= pre.d_start) {
          const uint64_t ent = front[pre.d_start - E];
          if (ent != ~0ull) {
            K = (ent >> 63) ? K_OPEN_OBJ : K_OPEN_ARR;
            par_tape = ent & 0xFFFFFFFFull;
          } else {
            par_ok = false;
          }
        } else {
          par_ok = false;
        }
      }
      int code = 0;
      if (E <= 0) {
        if (!(g == 0 && is_value_start(k))) code = SJ_TAPE_ERROR;
      } else if (!par_ok) {
        code = SJ_TAPE_ERROR;
      } else {
        const bool obj = K == K_OPEN_OBJ;
        const bool value_end = p == K_NUMBER || is_atom(p) || is_close(p) ||
                               (p == K_STRING && (!obj || pp == K_COLON));
        switch (k) {
          case K_CLOSE_OBJ: if (!obj || !(p == K_OPEN_OBJ || value_end)) code = SJ_TAPE_ERROR; break;
          case K_CLOSE_ARR: if (obj || !(p == K_OPEN_ARR || value_end)) code = SJ_TAPE_ERROR; break;
          case K_COMMA: if (!value_end) code = SJ_TAPE_ERROR; break;
          case K_COLON:
            if (!(obj && p == K_STRING && (pp == K_OPEN_OBJ || pp == K_COMMA))) code = SJ_TAPE_ERROR;
            break;
          case K_STRING:
            if (obj ? !(p == K_OPEN_OBJ || p == K_COMMA || p == K_COLON)
                    : !(p == K_OPEN_ARR || p == K_COMMA))
              code = SJ_TAPE_ERROR;
            break;
          case K_OTHER: code = SJ_TAPE_ERROR; break;
          default:  // numbers, atoms, openers
            if (obj ? p != K_COLON : !(p == K_OPEN_ARR || p == K_COMMA)) code = SJ_TAPE_ERROR;
        }
      }
      if (!code && is_open(k) && E + 1 > (int32_t)max_depth) code = SJ_DEPTH_ERROR;
      const uint64_t tp = (uint64_t)pre.tape_start + c.tape;
      // Content is checked even where the grammar failed: a grammar code is
      // smaller than any content code, so the minimum keeps the grammar first.
      if (is_close(k)) {
        if (!code && tp < tape_cap && par_tape < tape_cap) {
          tape[tp] = ((uint64_t)(k == K_CLOSE_OBJ ? '}' : ']') << 56) | par_tape;
          tape[par_tape] = ((uint64_t)(k == K_CLOSE_OBJ ? '{' : '[') << 56) | (tp + 1);
        }
      } else if (is_atom(k)) {
        const char *word = k == K_TRUE ? "true" : (k == K_FALSE ? "false" : "null");
        const uint32_t n = k == K_FALSE ? 5 : 4;
        bool ok = c.pos + n <= len;
        for (uint32_t i = 0; ok && i < n; i++) ok = sv.at(c.pos + i) == (uint8_t)word[i];
        if (ok && c.pos + n < len) ok = is_terminator(sv.at(c.pos + n));
        if (!ok) { if (!code) code = k == K_TRUE ? SJ_T_ATOM_ERROR : (k == K_FALSE ? SJ_F_ATOM_ERROR : SJ_N_ATOM_ERROR); }
        else if (tp < tape_cap) tape[tp] = (uint64_t)word[0] << 56;
      } else if (k == K_NUMBER) {  // Sec. 3.2.1
        uint8_t tag;
        uint64_t v;
        int nc;
        const uint64_t p0 = c.pos, p1 = c.next;
        if (p1 < sv.slimit || (p1 == len && len <= sv.slimit)) {  // lexeme and terminator staged
          const uint8_t *sp = sv.smem + (p0 - sv.sbase);
          nc = parse_number(sp, sp + (min(len, sv.slimit) - p0), tag, v);
        } else {
          nc = parse_number(doc + p0, doc + len, tag, v);
        }
        if (nc) { if (!code) code = nc; }
        else if (tp + 1 < tape_cap) {
          tape[tp] = (uint64_t)tag << 56;
          tape[tp + 1] = v;
        }
      } else if (k == K_STRING) {  // Sec. 3.2.2
        if (sl & 0x80000000u) {
          if (!code) code = (int)(sl & 0xFF);
        } else if (tp < tape_cap && so + 5 + sl <= str_cap) {
          tape[tp] = ((uint64_t)'"' << 56) | so;
          uint8_t *o = strs + so;
          o[0] = (uint8_t)sl; o[1] = (uint8_t)(sl >> 8); o[2] = (uint8_t)(sl >> 16); o[3] = (uint8_t)(sl >> 24);
          int err;
          const uint64_t p0 = (uint64_t)c.pos + 1, p1 = c.next;
          const uint8_t *sp = sv.ptr(p0, p1);
          string_walk<true>(sp, sp + (p1 - p0), err, o + 4);
          o[4 + sl] = 0;
        }
      }
      if (code) report(J, d, g, code);
    }
    __syncwarp();
    tw.clear(W, lane);
  }
}

// ---------------------------------------------------------------------------
// Set-up: tiles per document (one block scan over the documents).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) setup_kernel(const Job *__restrict__ job) {
  const Job &J = *job;
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < J.n_docs; base += 1024) {
    const uint32_t d = base + tid;
    uint32_t nt = 0;
    if (d < J.n_docs) {
      const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
      const bool too_big = len > J.max_doc_len;
      nt = too_big ? 0u : (uint32_t)((len + kTileBytes - 1) / kTileBytes);
      J.doc_flags[d] = too_big ? kFlagCapacity : 0u;
      J.doc_nidx[d] = 0;
      J.doc_err[d] = ~0ull;
      J.doc_tape[d] = 0;
      J.doc_str[d] = 0;
    }
    uint32_t incl = nt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const uint32_t v = s_warp[lane];
      uint32_t vi = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, vi, o);
        if (lane >= o) vi += u;
      }
      s_warp[lane] = vi - v;  // exclusive
    }
    __syncthreads();
    const uint32_t excl = s_carry + s_warp[wid] + incl - nt;
    if (d < J.n_docs) J.tile_first[d] = excl;
    __syncthreads();
    if (tid == 1023) s_carry = excl + nt;
    __syncthreads();
  }
  if (tid == 0) {
    J.tile_first[J.n_docs] = s_carry;
    J.counters[2] = s_carry;
  }
}

// Per-document results (error precedence: capacity, empty, UTF-8, unclosed
// string, internal, then the first failing token).
__global__ void finalize_kernel(const Job *__restrict__ job) {
  const Job &J = *job;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t d = blockIdx.x * blockDim.x + threadIdx.x; d < J.n_docs; d += stride) {
    const uint32_t f = J.doc_flags[d];
    int err;
    if (f & kFlagCapacity) err = SJ_CAPACITY;
    else if (J.doc_nidx[d] == 0) err = SJ_EMPTY;
    else if (f & kFlagUtf8) err = SJ_UTF8_ERROR;
    else if (f & kFlagUnclosed) err = SJ_UNCLOSED_STRING;
    else if (f & kFlagInternal) err = SJ_INTERNAL;
    else if (J.doc_err[d] != ~0ull) err = (int)(J.doc_err[d] & 0xFF);
    else err = SJ_SUCCESS;
    sj_doc_result r;
    r.error = err;
    r.reserved = 0;
    r.n_indices = J.doc_nidx[d];
    r.tape_words = err == SJ_SUCCESS ? J.doc_tape[d] : 0;
    r.string_bytes = err == SJ_SUCCESS ? J.doc_str[d] : 0;
    r.indices_offset = idx_base(J, d);
    r.tape_offset = tape_base(J, d);
    r.strings_offset = str_base(J, d);
    J.results[d] = r;
  }
}

}  // namespace sj
