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
//                         and that container, and the tape words; strings
//                         are normalised into the buffer;
//   numbers_kernel        per number: conversion and its two tape words,
//                         beside the build pass.
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
constexpr int kStageBytesR = kTileBytes + 512;  // the reduce pass stages a shorter halo
constexpr int kStageBytesB = kTileBytes + 512;  // and so does the build pass
constexpr int kStageBlocksR = kStageBytesR / kBlockBytes;
constexpr int kLevelOff = kMaxTileTokens;      // relative levels [-2048, 2048]
constexpr int kOpenSmem = 512;                 // levels kept in shared memory (mod 512)
// The build pass's shared memory per warp is sized so that 7 blocks of 128
// threads fit an SM (with 72 registers a thread): one more resident block
// than with 2 KiB of string staging and 64 frontier slots, 7% faster.
constexpr int kStrStage = 1024;                // string output of 32 strings, staged (larger runs
                                               // of strings are written directly)
constexpr uint32_t kQueue = 64;                // per-warp work queues (ring buffers)
constexpr uint32_t kFrontSmem = 32;            // frontier slots of a tile kept in shared memory
constexpr uint32_t kTileHasEscapes = 0x80000000u;  // flag in tile_nnum

// A string's entry in `slen`: an error code, or its normalised length and
// whether it holds escapes (then the reduce pass has left its normalised bytes
// in the scratch buffer `unesc`, at the string's own position).
constexpr uint32_t kSlenErr = 0x80000000u, kSlenWalk = 0x40000000u, kSlenLen = 0x3FFFFFFFu;

// Token facts passed from the reduce pass to the build pass, one word per
// token: kind (4 bits), depth before the token relative to the tile (13 bits,
// biased by 4096), tape slot relative to the tile (13), and the enclosing
// container when it was opened in the tile (16: bit 15 valid, bit 14 object,
// bits 0-11 its tape slot).
__device__ __forceinline__ uint64_t pack_meta(uint32_t kind, int32_t E, uint32_t tape,
                                              uint32_t parent) {
  return (uint64_t)kind | ((uint64_t)(uint32_t)(E + 4096) << 4) | ((uint64_t)tape << 17) |
         ((uint64_t)parent << 30);
}

__device__ __forceinline__ uint32_t warp_incl_u32(uint32_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}
__device__ __forceinline__ uint64_t warp_incl_u64(uint64_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
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
  // 32-bit view for positions at or after the tile start (p >= sbase):
  // bytes[(uint32_t)p - sb32] is position p while (uint32_t)p - sb32 < sn32
  uint32_t sb32, sn32;
  __device__ __forceinline__ uint32_t rel(uint32_t p) const { return p - sb32; }
  __device__ __forceinline__ uint8_t at(uint64_t p) const {
    return (p < slimit && (int64_t)p >= sbase) ? smem[p - sbase] : doc[p];
  }
  // pointer for reading [p, q): shared memory when staged, else global
  __device__ __forceinline__ const uint8_t *ptr(uint64_t p, uint64_t q) const {
    return (q <= slimit && (int64_t)p >= sbase) ? smem + (p - sbase) : doc + p;
  }
};

// Copy n bytes from t0 on (a tile and a halo; at most STAGE) into shared
// memory in 16-byte chunks; a tile past the document's end stages nothing.
template <int STAGE = kStageBytes>
__device__ __forceinline__ Staged stage_tile(uint8_t *bytes, const uint8_t *doc, uint64_t len,
                                             uint64_t t0, int lane, uint32_t n = STAGE) {
  const uintptr_t g0 = (uintptr_t)(doc + t0);
  const uintptr_t a0 = g0 & ~(uintptr_t)15;
  const uintptr_t dend = (uintptr_t)doc + len;
  const uintptr_t send = max(min((uintptr_t)(a0 + min(n, (uint32_t)STAGE)), dend), a0);
  const uint32_t nch = (uint32_t)((send - a0 + 15) / 16);
  for (uint32_t c = lane; c < nch; c += 32)
    reinterpret_cast<uint4 *>(bytes)[c] = __ldg(reinterpret_cast<const uint4 *>(a0 + 16 * c));
  __syncwarp();
  Staged v;
  v.doc = doc;
  v.len = len;
  v.sbase = (int64_t)t0 - (int64_t)(g0 - a0);
  v.slimit = (uint64_t)((int64_t)t0 + (int64_t)(send - g0));
  v.smem = bytes;
  v.sb32 = (uint32_t)v.sbase;
  v.sn32 = (uint32_t)(send - a0);
  return v;
}

// stage_tile's copy without waiting: each lane starts asynchronous 16-byte
// copies (cp.async) into shared memory; wait_staged() completes them.
template <int STAGE = kStageBytes>
__device__ __forceinline__ Staged stage_tile_async(uint8_t *bytes, const uint8_t *doc,
                                                   uint64_t len, uint64_t t0, int lane,
                                                   uint32_t n = STAGE) {
  const uintptr_t g0 = (uintptr_t)(doc + t0);
  const uintptr_t a0 = g0 & ~(uintptr_t)15;
  const uintptr_t dend = (uintptr_t)doc + len;
  const uintptr_t send = max(min((uintptr_t)(a0 + min(n, (uint32_t)STAGE)), dend), a0);
  const uint32_t nch = (uint32_t)((send - a0 + 15) / 16);
  for (uint32_t c = lane; c < nch; c += 32) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(bytes + 16 * c);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(a0 + 16 * c) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  Staged v;
  v.doc = doc;
  v.len = len;
  v.sbase = (int64_t)t0 - (int64_t)(g0 - a0);
  v.slimit = (uint64_t)((int64_t)t0 + (int64_t)(send - g0));
  v.smem = bytes;
  v.sb32 = (uint32_t)v.sbase;
  v.sn32 = (uint32_t)(send - a0);
  return v;
}
__device__ __forceinline__ void wait_staged() {
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncwarp();
}

// Position of the token after each token of a chunk (the next index, or the
// document's end after its last token), with the next chunk prefetched.
struct Positions {
  uint32_t pos_next = 0, pos_next2 = 0;  // the next two chunks, loaded ahead
  uint32_t after = 0;  // (lane 0) the position after the tile's last token, loaded up front
  __device__ __forceinline__ void begin(const uint32_t *idxp, uint32_t off, uint32_t cnt,
                                        uint32_t nidx, uint64_t len, int lane) {
    pos_next = (uint32_t)lane < cnt ? idxp[off + lane] : 0u;
    pos_next2 = (uint32_t)lane + 32 < cnt ? idxp[off + lane + 32] : 0u;
    if (lane == 0) after = off + cnt < nidx ? idxp[off + cnt] : (uint32_t)len;
  }
  __device__ __forceinline__ void next(uint32_t &pos, uint32_t &nxt, const uint32_t *idxp,
                                       uint32_t off, uint32_t cnt, uint32_t nidx, uint64_t len,
                                       uint32_t base, int lane) {
    const uint32_t j = base + lane;
    pos = pos_next;
    pos_next = pos_next2;
    const uint32_t jn = j + 64;
    pos_next2 = jn < cnt ? idxp[off + jn] : 0u;
    uint32_t nx = __shfl_down_sync(0xFFFFFFFFu, pos, 1);
    const uint32_t first_next = __shfl_sync(0xFFFFFFFFu, pos_next, 0);
    const uint32_t aft = __shfl_sync(0xFFFFFFFFu, after, 0);
    if (lane == 31 || j + 1 == cnt) nx = (j + 1 < cnt) ? first_next : aft;
    nxt = nx;
    (void)nidx;
    (void)len;
  }
};

// Work queues.  Per-token work whose cost depends on the token (string
// lengths, numbers, string output) would leave most lanes of a chunk idle;
// instead the tokens are queued in order and taken 32 at a time.
struct QEntry {
  uint32_t pos, nxt, j, tp;  // position, next token's position, index and tape slot in the tile
  uint32_t sl;               // a string's `slen` entry
};

struct RQEntry {
  uint32_t pos, nxt, j;
};
struct RWEntry {     // a string with escapes, kept across tiles until 32 are queued
  uint64_t a;        // its first content byte, as an offset from the batch base
  uint64_t slot;     // its `slen` slot
  uint32_t n;        // bytes from there to the next token
  uint32_t tile;     // the tile whose string-buffer total it belongs to
};

template <class T>
__device__ __forceinline__ void enqueue(T *q, uint32_t &tail, bool take, const T &e, int lane) {
  const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
  if (take) q[(tail + __popc(m & ((1u << lane) - 1u))) & (kQueue - 1)] = e;
  tail += __popc(m);
}

// ---------------------------------------------------------------------------
// Stage-2 reduce: per tile, the depth change and lowest depth, tape words,
// string-buffer bytes, and the containers left open at each level (the
// survivors); per token, the facts the build pass needs (pack_meta) and the
// normalised length of each string.
// ---------------------------------------------------------------------------
struct __align__(16) ReduceSmem {  // 16-byte aligned size: bytes[] takes uint4 stores
  uint8_t bytes[kStageBytesR + 64];
  uint64_t q[kStageBlocksR];       // real quotes of the staged blocks
  uint64_t x[kStageBlocksR];       // backslash and control bytes of the staged blocks
  RQEntry sq[kQueue];              // strings awaiting their length
  RWEntry wq[kQueue];              // strings with escapes awaiting a walk
  uint16_t open[kOpenSmem];
};
static_assert(sizeof(ReduceSmem) % 16 == 0, "per-warp staging must stay 16-byte aligned");

// `open` entry of relative level l: the container currently open there, written
// by the openers of the tile (0 = none, else bit 15, bit 14 = object, bits
// 0-11 = the opener's tape slot relative to the tile).  A tile with fewer than
// 512 tokens spans fewer than 512 levels, so they fit in shared memory modulo
// 512; other tiles use the warp's table in global memory.
struct OpenTable {
  uint16_t *p;
  uint32_t mask;
  int32_t bias;
  __device__ __forceinline__ uint16_t &at(int32_t l) const { return p[(uint32_t)(l + bias) & mask]; }
};

// Normalised length of a string without escapes or control bytes, from the
// staged masks: the distance from its first content byte (document position
// p0) to the next real quote.  False when the masks cannot decide it.
__device__ __forceinline__ bool plain_string_len(const ReduceSmem &W, uint32_t t0, uint32_t p0,
                                                 uint32_t nblk, uint32_t &L) {
  const uint32_t rel = p0 - t0;
  uint32_t w = rel >> 6, b = rel & 63, acc = 0;
  while (w < nblk) {
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

// SH: the stage-2 tile is a stage-1 tile split in 2^SH (the run's s2_shift;
// one kernel for each value, so that whole tiles pay no arithmetic for it).
template <uint32_t SH>
__device__ __forceinline__ void stage2_reduce(const Job *__restrict__ job) {
  const Job &J = *job;
  __shared__ ReduceSmem WS[kS2Warps];
  __shared__ uint8_t s_kind[256];
  for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) s_kind[i] = token_kind((uint8_t)i);
  const int lane = threadIdx.x & 31;
  const uint32_t wid = threadIdx.x >> 5;
  ReduceSmem &W = WS[wid];
  for (uint32_t i = lane; i < kOpenSmem; i += 32) W.open[i] = 0;
  __syncthreads();
  uint16_t *const open_g = J.open_g + (uint64_t)(blockIdx.x * kS2Warps + wid) * kOpenGlobal;
  uint32_t t_lo, t_hi;
  s2_range(J, t_lo, t_hi);
  // Strings with escapes are walked (Sec. 3.2.2) 32 at a time, across tiles:
  // a tile holds too few of them to fill a warp.  The walk reads the staged
  // bytes while its string is in the current tile, else global memory, and
  // adds the string's buffer bytes to its own tile's total.
  uint32_t whead = 0, wtail = 0;
  uint64_t stg_lo = 1, stg_hi = 0;  // staged bytes of the current tile, as batch offsets
  auto flush_walks = [&]() {
    const uint32_t m = min(32u, wtail - whead);
    if ((uint32_t)lane < m) {
      const RWEntry e = W.wq[(whead + lane) & (kQueue - 1)];
      const uint8_t *sp = (e.a >= stg_lo && e.a + e.n <= stg_hi) ? W.bytes + (e.a - stg_lo)
                                                                 : J.base + e.a;
      int err;
      // normalised bytes are never more than the raw ones: they stay within
      // the string's own span of the scratch buffer
      const uint32_t n = string_walk8<true>(sp, sp + e.n, err, J.unesc + (e.a - J.doc_off[0]));
      uint64_t size;
      if (err) {
        J.slen[e.slot] = kSlenErr | (uint32_t)err;
        size = 5;
      } else {
        J.slen[e.slot] = kSlenWalk | min(n, kSlenLen);
        size = 5ull + n;
      }
      atomicAdd(reinterpret_cast<unsigned long long *>(&J.s2_rec[e.tile].s),
                (unsigned long long)size);
    }
    whead += m;
    __syncwarp();
  };
  TileTickets tix(J, kTicketReduce, t_lo, t_hi, blockIdx.x * kS2Warps + wid, gridDim.x * kS2Warps,
                  lane);
  for (uint32_t t = tix.first(); t < t_hi; t = tix.next()) {
    tix.draw();  // the next tile, read at the loop's end
    const uint32_t d = doc_of_tile(J, t >> SH);
    const uint32_t j_min = J.tile_first[d] << SH;
    const uint32_t tt = t - j_min;
    const uint32_t nidx = J.doc_nidx[d];
    if ((J.doc_flags[d] & kDocBad) || nidx == 0) {
      if (lane == 0) {
        J.s2_rec[t] = S2Agg{0, 0, 0, tt == 0, 0};
        J.tile_nnum[t] = 0;
      }
      continue;
    }
    if (lane == 0) J.s2_rec[t].s = 0;  // walks add to it, from this tile on
    const uint32_t ntiles_d = (J.tile_first[d + 1] << SH) - j_min;
    constexpr uint32_t tblk = 32u >> SH;  // 64-byte blocks of a stage-2 tile
    const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
    const uint8_t *doc = J.base + J.doc_off[d];
    const uint64_t ib = idx_base(J, d);
    const uint32_t *idxp = J.idx + ib;
    const uint32_t cnt = J.tile_cnt[t], off = J.tile_off[t];
    uint32_t *slen = J.slen + ib + off;
    const uint64_t t0 = (uint64_t)tt * (tblk * kBlockBytes);
    constexpr uint32_t nstage = tblk * kBlockBytes + (kStageBytesR - kTileBytes);
    // masks of the tile's blocks and of the next ones in the document
    const uint32_t nblk = min(nstage / kBlockBytes, (ntiles_d - tt) * tblk);
    for (uint32_t k = lane; k < nblk; k += 32) {
      const ulonglong2 v = J.s1_qx[(uint64_t)t * tblk + k];
      W.q[k] = v.x;
      W.x[k] = v.y;
    }
    const Staged sv = stage_tile<kStageBytesR>(W.bytes, doc, len, t0, lane, nstage);
    stg_lo = J.doc_off[d] + (uint64_t)sv.sbase;
    stg_hi = J.doc_off[d] + sv.slimit;
    const OpenTable ot = cnt < (uint32_t)kOpenSmem ? OpenTable{W.open, (uint32_t)kOpenSmem - 1u, 0}
                                                   : OpenTable{open_g, 0xFFFFFFFFu, kLevelOff};
    uint64_t sb = 0;  // string-buffer bytes of this lane's strings without escapes
    uint32_t shead = 0, stail = 0;
    uint32_t nnum = 0;  // number tokens of the tile so far, listed for numbers_kernel (index
                        // and tape slot in the tile, 16 bits each)
    const uint32_t wtail0 = wtail;  // escaped strings queued before this tile
    // strings: the next 32 queued get their length from the masks; those the
    // masks cannot decide go to the walk queue
    auto flush_strings = [&]() {
      const uint32_t m = min(32u, stail - shead);
      const bool have = (uint32_t)lane < m;
      RQEntry e{0, 0, 0};
      if (have) e = W.sq[(shead + lane) & (kQueue - 1)];
      uint32_t L = 0;
      const bool ok = have && plain_string_len(W, (uint32_t)t0, e.pos + 1, nblk, L);
      if (ok) {
        slen[e.j] = L;
        sb += 5u + L;
      }
      enqueue(W.wq, wtail, have && !ok,
              RWEntry{J.doc_off[d] + e.pos + 1, ib + off + e.j, e.nxt - (e.pos + 1), t}, lane);
      shead += m;
      __syncwarp();
    };

    Positions ps;
    ps.begin(idxp, off, cnt, nidx, len, lane);
    int32_t depth = 0, mn = 0, mx = 0;
    uint32_t tape = 0;
    for (uint32_t base = 0; base < cnt; base += 32) {
      const uint32_t j = base + lane;
      const bool valid = j < cnt;
      uint32_t pos, nxt;
      ps.next(pos, nxt, idxp, off, cnt, nidx, len, base, lane);
      const uint8_t kind = valid ? s_kind[sv.smem[sv.rel(pos)]] : K_OTHER;
      // depth and tape slot: one scan over (delta + 1) | words << 8
      const int32_t dl = depth_delta(kind);
      const uint32_t w = tape_words_of(kind);
      const uint32_t vi = warp_incl_u32((uint32_t)(dl + 1) | (w << 8), lane);
      const int32_t D = depth + (int32_t)(vi & 0xFFu) - (lane + 1);
      const int32_t E = D - dl;
      const uint32_t tp = tape + (vi >> 8) - w;
      // Enclosing container: the latest earlier opener whose depth after it
      // equals this token's depth before (depth moves by one per token, so
      // that container is still open).  Inside the chunk such an opener is
      // the token just before some token k <= i with E_k = E_i, so one match
      // on E finds it; when none qualifies, the level table holds it.
      const bool op = valid && is_open(kind);
      const uint16_t my = op ? (uint16_t)(0x8000u | (kind == K_OPEN_OBJ ? 0x4000u : 0u) | tp) : 0;
      const unsigned after_open = __ballot_sync(0xFFFFFFFFu, op) << 1;
      const unsigned same_e =
          __match_any_sync(0xFFFFFFFFu, valid ? (uint32_t)E : (0x80000000u | (uint32_t)lane));
      const unsigned cand = same_e & after_open & (0xFFFFFFFFu >> (31 - lane));
      const int hk = 31 - __clz(cand);  // -1 when no token qualifies
      uint16_t parent = (uint16_t)__shfl_sync(0xFFFFFFFFu, (uint32_t)my, max(hk - 1, 0));
      if (!cand) parent = (valid && E > -kLevelOff && E <= kLevelOff) ? ot.at(E) : (uint16_t)0;
      // the last opener of each level of this chunk stays open for later tokens
      const unsigned grp = __match_any_sync(0xFFFFFFFFu, op ? D : 0x7FFFFFFF);
      if (op && lane == 31 - __clz(grp)) ot.at(D) = my;
      if (valid) {
        J.meta[ib + off + j] = pack_meta(kind, E, tp, parent);
        mn = min(mn, min(E, D));
        mx = max(mx, max(E, D));
      }
      enqueue(W.sq, stail, valid && kind == K_STRING, RQEntry{pos, nxt, j}, lane);
      {
        const unsigned nb = __ballot_sync(0xFFFFFFFFu, valid && kind == K_NUMBER);
        if (valid && kind == K_NUMBER) J.nlist[ib + off + nnum + __popc(nb & ((1u << lane) - 1u))] = j | (tp << 16);
        nnum += __popc(nb);
      }
      const uint32_t tot = __shfl_sync(0xFFFFFFFFu, vi, 31);
      depth += (int32_t)(tot & 0xFFu) - 32;
      tape += tot >> 8;
      __syncwarp();
      if (stail - shead >= 32) {
        flush_strings();
        if (wtail - whead >= 32) flush_walks();
      }
    }
    while (shead != stail) {
      flush_strings();
      if (wtail - whead >= 32) flush_walks();
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      sb += __shfl_xor_sync(0xFFFFFFFFu, sb, o);
      mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
      mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    }
    // survivors: the open container of each level in (mn, depth]
    for (int32_t lv = mn + 1 + lane; lv <= depth; lv += 32) {
      const uint16_t e = ot.at(lv);
      J.surv[ib + off + (uint32_t)(lv - mn - 1)] = ((uint32_t)(e >> 14) & 1u) << 31 | (e & 0x0FFFu);
    }
    __syncwarp();
    // forget this tile's levels
    for (int32_t v = max(mn, -kLevelOff) + lane; v <= min(mx, kLevelOff); v += 32) ot.at(v) = 0;
    __syncwarp();
    if (lane == 0) {
      // bit 31: the tile has strings with escapes (the build pass stages its
      // scratch window ahead)
      J.tile_nnum[t] = nnum | (wtail != wtail0 ? kTileHasEscapes : 0u);
      S2Agg &a = J.s2_rec[t];
      a.dd = depth;
      a.mn = mn;
      a.w = tape;
      a.head = tt == 0;
      atomicAdd(reinterpret_cast<unsigned long long *>(&a.s), (unsigned long long)sb);
    }
  }
  while (whead != wtail) flush_walks();
}

// ---------------------------------------------------------------------------
// Numbers (Sec. 3.2.1): each warp gathers the number tokens listed by the
// reduce pass for its tiles into a queue and converts them 32 at a time, one
// lane per number (a tile holds too few to fill a warp).  Each lane copies its
// lexeme and the byte after it (at most kNumWindow bytes, in 16-byte chunks)
// into shared memory and converts it there; longer lexemes are read in place.
// numbers_kernel runs once the tile scan has given every tile its first tape
// slot, beside the build pass, and writes the number's two tape words (tag
// 'l' or 'd', value) itself, or reports its error.  On small whole runs
// (numbers_split_kernel) it runs beside the tile scan instead, where a small
// run's stage 2 leaves the GPU mostly idle, and leaves the value in `numv`
// and the tag or error in `slen` for the build pass.
constexpr int kNumWindow = 48;
constexpr int kNumThreads = 128;
struct NumEntry {
  uint64_t slot;  // the token's index slot (idx_base + index in the document)
  uint32_t d;     // its document
  uint32_t rel;   // its index in the document
  uint32_t tp;    // its tape slot in the document
};
// The queue entry of number-list entry x of tile t (document d, index base ib).
__device__ __forceinline__ NumEntry num_entry(const Job &J, uint32_t t, uint32_t d, uint64_t ib,
                                              uint32_t off, uint32_t x) {
  const uint32_t rel = off + (x & 0xFFFFu);
  return NumEntry{ib + rel, d, rel, J.s2_pre[t].tape_start + (x >> 16)};
}
// 12 resident blocks (40 registers): the kernel waits on scattered lexeme
// loads, so more warps in flight beat the few spilled registers.
// One number token: its lexeme window staged in `my` (kNumWindow + 16
// bytes of shared memory), converted; value and tag (or error) stored.
template <bool TO_TAPE>
__device__ __forceinline__ void convert_number(const Job &J, const NumEntry &e, uint8_t *my) {
      const uint64_t len = J.doc_off[e.d + 1] - J.doc_off[e.d];
      const uint8_t *doc = J.base + J.doc_off[e.d];
      const uint32_t nidx = J.doc_nidx[e.d];
      const uint64_t pos = J.idx[e.slot];
      const uint64_t nxt = e.rel + 1 < nidx ? J.idx[e.slot + 1] : len;
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
      if constexpr (TO_TAPE) {
        const uint32_t tape_cap32 = (uint32_t)min(len + 3, (uint64_t)0xFFFFFFFFu);  // >= 3
        if (nc) {
          report(J, e.d, e.rel, nc);
        } else if (e.tp < tape_cap32 - 1u) {
          uint64_t *tape = J.tape + tape_base(J, e.d);
          tape[e.tp] = (uint64_t)tag << 56;
          tape[e.tp + 1] = v;
        }
      } else if (nc) {
        J.slen[e.slot] = kSlenErr | (uint32_t)nc;
      } else {
        J.slen[e.slot] = tag;
        J.numv[e.slot] = v;
      }
}

__global__ void __launch_bounds__(kNumThreads, 12) numbers_kernel(const Job *__restrict__ job) {
  pdl_enter();
  const Job &J = *job;
  __shared__ __align__(16) uint8_t win[kNumThreads][kNumWindow + 16];
  __shared__ NumEntry q[kNumThreads / 32][64];
  const int lane = threadIdx.x & 31;
  uint8_t *my = win[threadIdx.x];
  NumEntry *wq = q[threadIdx.x >> 5];
  uint32_t head = 0, tail = 0;
  auto flush = [&]() {
    const uint32_t m = min(32u, tail - head);
    if ((uint32_t)lane < m) convert_number<true>(J, wq[(head + lane) & 63u], my);
    head += m;
    __syncwarp();
  };
  uint32_t t_lo, t_hi;
  s2_range(J, t_lo, t_hi);
  TileTickets tix(J, kTicketNumbers, t_lo, t_hi, blockIdx.x * (kNumThreads / 32) + (threadIdx.x >> 5),
                  gridDim.x * (kNumThreads / 32), lane);
  for (uint32_t t = tix.first(); t < t_hi; t = tix.next()) {
    tix.draw();
    const uint32_t d = s2_doc(J, t);
    if ((J.doc_flags[d] & kDocBad) || J.doc_nidx[d] == 0) continue;
    const uint32_t m = J.tile_nnum[t] & ~kTileHasEscapes;
    if (m == 0) continue;
    const uint64_t ib = idx_base(J, d);
    const uint32_t off = J.tile_off[t];
    for (uint32_t k0 = 0; k0 < m; k0 += 32) {
      const uint32_t k = k0 + lane;
      const uint32_t c = min(32u, m - k0);
      if ((uint32_t)lane < c) {
        wq[(tail + lane) & 63u] = num_entry(J, t, d, ib, off, J.nlist[ib + off + k]);
      }
      tail += c;
      __syncwarp();
      if (tail - head >= 32) flush();
    }
  }
  while (head != tail) flush();
}

// The same conversion for small runs, where a warp per tile leaves a
// number-heavy tile's numbers to one warp in turn: warp w of the grid takes
// group w % kNumGroups of tile w / kNumGroups -- numbers 32g to 32g + 31 of
// the tile's list, the last group all from there on -- so up to kNumGroups
// warps share a tile.
constexpr uint32_t kNumGroups = 4;
__global__ void __launch_bounds__(kNumThreads, 12) numbers_split_kernel(const Job *__restrict__ job) {
  pdl_enter();
  const Job &J = *job;
  __shared__ __align__(16) uint8_t win[kNumThreads][kNumWindow + 16];
  const int lane = threadIdx.x & 31;
  uint8_t *my = win[threadIdx.x];
  uint32_t t_lo, t_hi;
  s2_range(J, t_lo, t_hi);
  const uint32_t gw = blockIdx.x * (kNumThreads / 32) + (threadIdx.x >> 5);
  const uint32_t nw = gridDim.x * (kNumThreads / 32);
  for (uint32_t w = gw; w < (t_hi - t_lo) * kNumGroups; w += nw) {
    const uint32_t t = t_lo + w / kNumGroups, g = w % kNumGroups;
    const uint32_t d = s2_doc(J, t);
    if ((J.doc_flags[d] & kDocBad) || J.doc_nidx[d] == 0) continue;
    const uint32_t m = J.tile_nnum[t] & ~kTileHasEscapes;
    const uint32_t k0 = 32u * g, k1 = g + 1 == kNumGroups ? m : min(m, k0 + 32u);
    if (k0 >= k1) continue;
    const uint64_t ib = idx_base(J, d);
    const uint32_t off = J.tile_off[t];
    for (uint32_t k = k0 + lane; k < k1; k += 32) {
      const uint32_t x = J.nlist[ib + off + k];
      convert_number<false>(J, NumEntry{ib + off + (x & 0xFFFFu), d, off + (x & 0xFFFFu), 0u}, my);
    }
  }
}

// ---------------------------------------------------------------------------
// Stage-2 build: grammar, tape words, numbers and strings.
// ---------------------------------------------------------------------------
struct __align__(16) BuildSmem {
  uint8_t bytes[kStageBytesB + 64];
  uint8_t ubytes[kStageBytesB + 64];  // the same window of the scratch buffer (escaped strings)
  uint8_t sout[kStrStage];  // the string-buffer bytes of 32 strings, before a coalesced copy
  QEntry sq[kQueue];        // strings awaiting output
  uint64_t front[kFrontSmem];  // the first frontier slots of the tile
};
static_assert(sizeof(BuildSmem) % 16 == 0 && (kStageBytesB + 64) % 16 == 0 &&
                  kStrStage % 16 == 0,
              "per-warp staging must stay 16-byte aligned");

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

// Write one string's buffer entry (u32 length, its n normalised bytes from
// src, NUL) at o.
__device__ __forceinline__ void put_string(uint8_t *__restrict__ o, uint32_t n,
                                           const uint8_t *__restrict__ src) {
  o[0] = (uint8_t)n; o[1] = (uint8_t)(n >> 8); o[2] = (uint8_t)(n >> 16); o[3] = (uint8_t)(n >> 24);
#pragma unroll 4
  for (uint32_t i = 0; i < n; i++) o[4 + i] = src[i];
  o[4 + n] = 0;
}

// put_string for a staged entry: source and destination both in shared
// memory, the source with at least 3 readable bytes past its end.  Bytes
// until the destination is word aligned, then whole words (two aligned source
// words and a funnel shift), then the tail.
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

// NUMS: the run's numbers were left in numv and slen (small whole runs), and
// this pass writes their tape words; otherwise numbers_kernel writes them.
template <uint32_t SH, bool NUMS>
__device__ __forceinline__ void stage2_build(const Job *__restrict__ job) {
  const Job &J = *job;
  __shared__ BuildSmem WS[kS2Warps];
  __shared__ uint16_t s_gram[32];
  if (threadIdx.x < 32) s_gram[threadIdx.x] = grammar_row(threadIdx.x >> 1, threadIdx.x & 1);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  BuildSmem &W = WS[threadIdx.x >> 5];
  uint32_t t_lo, t_hi;
  s2_range(J, t_lo, t_hi);
  const uint32_t max_depth = J.max_depth;
  TileTickets tix(J, kTicketBuild, t_lo, t_hi, blockIdx.x * kS2Warps + (threadIdx.x >> 5),
                  gridDim.x * kS2Warps, lane);
  for (uint32_t t = tix.first(); t < t_hi; t = tix.next()) {
    tix.draw();  // the next tile, read at the loop's end
    const uint32_t d = doc_of_tile(J, t >> SH);
    const uint32_t j_min = J.tile_first[d] << SH;
    const uint32_t tt = t - j_min;
    const uint32_t ntiles_d = (J.tile_first[d + 1] << SH) - j_min;
    const uint32_t nidx = J.doc_nidx[d];
    if ((J.doc_flags[d] & kDocBad) || nidx == 0) continue;
    constexpr uint32_t tbytes = kTileBytes >> SH;  // bytes of a stage-2 tile
    constexpr uint32_t nstage = tbytes + (kStageBytesB - kTileBytes);
    const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
    const uint8_t *doc = J.base + J.doc_off[d];
    const uint64_t ib = idx_base(J, d);
    const uint32_t *idxp = J.idx + ib;
    uint64_t *tape = J.tape + tape_base(J, d);
    uint8_t *strs = J.strings + str_base(J, d);
    const uint64_t tape_cap = len + 3;
    // tape indices of the chunk loop in 32 bits (documents stay below 2^32 - 256 bytes)
    const uint32_t tape_cap32 = (uint32_t)min(tape_cap, (uint64_t)0xFFFFFFFFu);
    const uint64_t str_cap = str_base(J, d + 1) - str_base(J, d);
    const uint32_t cnt = J.tile_cnt[t], off = J.tile_off[t];
    const S2Pre pre = J.s2_pre[t];
    const uint64_t *front = J.front + ib + off + t;

    if (tt == ntiles_d - 1 && lane == 0) {  // the document's last tile closes the tape
      const S2Agg agg = J.s2_rec[t];
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

    // the tile's frontier slots: the container open at each level the tile
    // starts inside, deepest first (levels d_start down to max(1, low))
    const uint32_t nfront = pre.d_start >= max(1, pre.low) ? (uint32_t)(pre.d_start - max(1, pre.low) + 1) : 0u;
    for (uint32_t k = lane; k < min(nfront, kFrontSmem); k += 32) W.front[k] = front[k];
    const Staged sv = stage_tile<kStageBytesB>(W.bytes, doc, len, (uint64_t)tt * tbytes, lane, nstage);
    uint32_t shead = 0, stail = 0;
    const uint8_t *unesc = J.unesc + rel_off(J, d);
    // the scratch window, copied ahead when the tile has strings with escapes.
    // The scratch buffer has the input's alignment modulo 16, so the window
    // covers the same positions as the staged input (sv) in W.ubytes.
    const bool has_esc = (J.tile_nnum[t] & kTileHasEscapes) != 0 &&
                         (((uintptr_t)unesc ^ (uintptr_t)doc) & 15u) == 0;
    if (has_esc) stage_tile_async<kStageBytesB>(W.ubytes, unesc, len, (uint64_t)tt * tbytes, lane, nstage);
    bool us_ready = !has_esc;
    uint64_t str_run = pre.str_start;  // buffer offset of the next queued string

    // numbers (Sec. 3.2.1), 32 at a time

    // strings (Sec. 3.2.2), 32 at a time: their entries are contiguous in the
    // buffer, so they are built in shared memory and copied out coalesced
    auto flush_strings = [&]() {
      const uint32_t m = min(32u, stail - shead);
      const bool have = (uint32_t)lane < m;
      QEntry e{0, 0, 0, 0, 0};
      if (have) e = W.sq[(shead + lane) & (kQueue - 1)];
      const uint32_t sl = e.sl;
      const bool bad = have && (sl & kSlenErr);
      if (bad) report(J, d, (uint64_t)off + e.j, (int)(sl & 0xFFu));
      const bool is_str = have && !bad;
      const bool walk = (sl & kSlenWalk) != 0;
      const uint64_t p0 = (uint64_t)e.pos + 1;
      uint64_t n = sl & kSlenLen;
      if (is_str && n == kSlenLen) {  // too long for the entry: measure again
        int err;
        n = string_walk<false>(doc + p0, doc + e.nxt, err, nullptr);
      }
      const uint64_t size = have ? (bad ? 5ull : 5ull + n) : 0ull;
      const uint64_t incl = warp_incl_u64(size, lane);
      const uint64_t so = str_run + incl - size;
      const uint64_t tp = (uint64_t)pre.tape_start + e.tp;
      if (is_str && tp < tape_cap) tape[tp] = ((uint64_t)'"' << 56) | so;
      // Strings with escapes take their normalised bytes from the scratch
      // buffer of the reduce pass (same positions), staged once per tile.
      if (!us_ready && __any_sync(0xFFFFFFFFu, is_str && walk)) {
        wait_staged();
        us_ready = true;
      }
      const bool fits = !is_str || (n < kSlenLen && p0 + n <= sv.slimit && (!walk || has_esc));
      const unsigned sm = __ballot_sync(0xFFFFFFFFu, is_str);
      if (sm) {
        const bool all_fit = __all_sync(0xFFFFFFFFu, fits);
        const uint64_t so_lo = __shfl_sync(0xFFFFFFFFu, so, __ffs(sm) - 1);
        const uint64_t so_hi = __shfl_sync(0xFFFFFFFFu, so + 5 + n, 31 - __clz(sm));
        const uint32_t a = (uint32_t)((uintptr_t)(strs + so_lo) & 15u);
        const uint64_t total = a + (so_hi - so_lo);
        if (all_fit && total <= (uint64_t)kStrStage && so_hi <= str_cap) {
          if (is_str)
            put_string_smem(W.sout + a + (so - so_lo), (uint32_t)n, (walk ? W.ubytes : W.bytes) + (p0 - sv.sbase));
          __syncwarp();
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
        } else if (is_str && so + 5 + n <= str_cap) {
          put_string(strs + so, (uint32_t)n, walk ? unesc + p0 : sv.ptr(p0, p0 + n));
        }
      }
      str_run += __shfl_sync(0xFFFFFFFFu, incl, 31);
      shead += m;
      __syncwarp();
    };

    Positions ps;
    ps.begin(idxp, off, cnt, nidx, len, lane);
    // token facts and string entries are loaded one chunk ahead (the string
    // entry for every lane: a coalesced load, used only by strings)
    uint64_t meta_next = (uint32_t)lane < cnt ? J.meta[ib + off + lane] : 0ull;
    uint32_t sl_next = (uint32_t)lane < cnt ? J.slen[ib + off + lane] : 0u;
    // a number's value word, loaded one chunk ahead once the kinds are known
    uint64_t nv_next = (NUMS && (uint32_t)lane < cnt && (meta_next & 15u) == K_NUMBER)
                           ? J.numv[ib + off + lane] : 0ull;
    // kinds of the two tokens before the tile
    uint8_t prev1 = K_OTHER, prev2 = K_OTHER;
    if (lane < 2 && off >= (uint32_t)lane + 1) {
      const uint8_t k = (uint8_t)(J.meta[ib + off - 1 - lane] & 15u);
      if (lane == 0) prev1 = k; else prev2 = k;
    }
    prev1 = __shfl_sync(0xFFFFFFFFu, prev1, 0);
    prev2 = __shfl_sync(0xFFFFFFFFu, prev2, 1);
    for (uint32_t base = 0; base < cnt; base += 32) {
      const uint32_t j = base + lane;
      const bool valid = j < cnt;
      uint32_t pos, nxt;
      ps.next(pos, nxt, idxp, off, cnt, nidx, len, base, lane);
      const uint64_t meta = meta_next;
      const uint32_t sl_all = sl_next;
      const uint64_t nv = nv_next;
      meta_next = j + 32 < cnt ? J.meta[ib + off + j + 32] : 0ull;
      sl_next = j + 32 < cnt ? J.slen[ib + off + j + 32] : 0u;
      const uint8_t k = (uint8_t)(meta & 15u);
      const uint32_t sl = (valid && k == K_STRING) ? sl_all : 0u;
      const int32_t E = pre.d_start + ((int32_t)((meta >> 4) & 0x1FFFu) - 4096);
      const uint32_t trel = (uint32_t)(meta >> 17) & 0x1FFFu;
      const uint32_t tp = pre.tape_start + trel;
      const uint32_t parent = (uint32_t)(meta >> 30) & 0xFFFFu;
      uint8_t p = __shfl_up_sync(0xFFFFFFFFu, k, 1);
      uint8_t pp = __shfl_up_sync(0xFFFFFFFFu, k, 2);
      if (lane == 0) { p = prev1; pp = prev2; }
      if (lane == 1) pp = prev1;
      prev2 = __shfl_sync(0xFFFFFFFFu, k, 30);
      prev1 = __shfl_sync(0xFFFFFFFFu, k, 31);
      const uint32_t g = off + j;

      // ---- grammar: the enclosing container and the previous two tokens ----
      uint8_t K = 0;
      uint32_t par_tape = 0xFFFFFFFFu;
      bool par_ok = true;
      if (E >= 1) {
        if (parent) {
          K = (parent & 0x4000u) ? K_OPEN_OBJ : K_OPEN_ARR;
          par_tape = pre.tape_start + (parent & 0x0FFFu);
        } else if (E >= max(1, pre.low) && E <= pre.d_start) {
          const uint32_t fk = (uint32_t)(pre.d_start - E);
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
      if (E <= 0) {
        if (!(g == 0 && is_value_start(k))) code = SJ_TAPE_ERROR;
      } else if (!par_ok) {
        code = SJ_TAPE_ERROR;
      } else {
        const bool obj = K == K_OPEN_OBJ;
        const uint32_t pc = (p == K_STRING && obj && pp != K_COLON) ? kKeyStr : p;
        if (!((s_gram[(k << 1) | (obj ? 1 : 0)] >> pc) & 1u)) code = SJ_TAPE_ERROR;
      }
      if (!code && is_open(k) && E + 1 > (int32_t)max_depth) code = SJ_DEPTH_ERROR;

      // ---- tape words of closers and atoms; numbers and strings are queued.
      // Content is checked even where the grammar failed: a grammar code is
      // smaller than any content code, so the minimum keeps the grammar first.
      if (valid) {
        if (is_close(k)) {
          if (!code && tp < tape_cap32 && par_tape < tape_cap32) {
            tape[tp] = ((uint64_t)(k == K_CLOSE_OBJ ? '}' : ']') << 56) | par_tape;
            tape[par_tape] = ((uint64_t)(k == K_CLOSE_OBJ ? '{' : '[') << 56) | (uint64_t)(tp + 1);
          }
        } else if (k == K_NUMBER) {
          if constexpr (NUMS) {  // converted by numbers_split_kernel (Sec. 3.2.1)
            if (sl_all & kSlenErr) {
              if (!code) code = (int)(sl_all & 0xFFu);
            } else if (tp < tape_cap32 - 1u) {  // tape_cap32 >= 3
              tape[tp] = (uint64_t)(sl_all & 0xFFu) << 56;
              tape[tp + 1] = nv;
            }
          }  // else numbers_kernel writes the words
        } else if (is_atom(k)) {
          // the literal and the byte after it: one 8-byte window of the staged
          // tile (two aligned words and a funnel shift), else byte by byte
          const uint32_t nw = k == K_FALSE ? 5 : 4;
          const uint64_t lit = k == K_TRUE ? 0x65757274ull : (k == K_FALSE ? 0x65736C6166ull : 0x6C6C756Eull);
          bool ok = pos + nw <= len;
          if (ok) {
            if (pos + 8 <= sv.slimit) {
              const uintptr_t ua = (uintptr_t)(sv.smem + (pos - sv.sbase));
              const uint32_t *wp = reinterpret_cast<const uint32_t *>(ua & ~(uintptr_t)3);
              const uint32_t sh = (uint32_t)(ua & 3u) * 8;
              const uint64_t x = ((uint64_t)__funnelshift_r(wp[1], wp[2], sh) << 32) |
                                 __funnelshift_r(wp[0], wp[1], sh);
              ok = (x & ((1ull << (8 * nw)) - 1)) == lit &&
                   (pos + nw >= len || is_terminator((uint8_t)(x >> (8 * nw))));
            } else {
              for (uint32_t i = 0; ok && i < nw; i++) ok = sv.at(pos + i) == (uint8_t)(lit >> (8 * i));
              if (ok && pos + nw < len) ok = is_terminator(sv.at(pos + nw));
            }
          }
          if (!ok) { if (!code) code = k == K_TRUE ? SJ_T_ATOM_ERROR : (k == K_FALSE ? SJ_F_ATOM_ERROR : SJ_N_ATOM_ERROR); }
          else if (tp < tape_cap32) tape[tp] = (uint64_t)(uint8_t)lit << 56;
        }
        if (code) report(J, d, g, code);
      }
      enqueue(W.sq, stail, valid && k == K_STRING, QEntry{pos, nxt, j, trel, sl}, lane);
      if constexpr (NUMS)
        nv_next = (j + 32 < cnt && (meta_next & 15u) == K_NUMBER) ? J.numv[ib + off + j + 32] : 0ull;
      __syncwarp();
      if (stail - shead >= 32) flush_strings();
    }
    while (shead != stail) flush_strings();
    if (!us_ready) wait_staged();  // no copy may still be in flight into ubytes
    __syncwarp();  // every lane is done with this tile's staged bytes
  }
}

// ---------------------------------------------------------------------------
// Set-up: tiles per document (one block scan over the documents).
// ---------------------------------------------------------------------------
// With hjob, the run descriptor and the n_off document offsets are first
// copied from pinned host memory (hjob, hoff) into device memory (job and
// the descriptor's doc_off): a small run then needs no copy operation.
__global__ void __launch_bounds__(1024) setup_kernel(Job *job, const Job *hjob,
                                                     const uint64_t *hoff, uint32_t n_off) {
  pdl_enter();
  static_assert(sizeof(Job) % 4 == 0, "the descriptor is copied in words");
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (hjob) {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(hjob);
    uint32_t *dst = reinterpret_cast<uint32_t *>(job);
    for (uint32_t i = tid; i < sizeof(Job) / 4; i += 1024) dst[i] = src[i];
    __syncthreads();
    uint64_t *doff = const_cast<uint64_t *>(job->doc_off);
    for (uint32_t i = tid; i < n_off; i += 1024) doff[i] = hoff[i];
    __syncthreads();
  }
  const Job &J = *job;
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
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
    J.counters[4] = 0;  // both stages: all tiles
    J.counters[5] = s_carry;
    J.counters[6] = 0;
    J.counters[7] = s_carry << J.s2_shift;
    for (int k = kTicketReduce; k <= kTicketS1; k++) J.counters[k] = 0;
  }
}

// A document that arrives in chunks (one document; host input).
//   mode 0: the tiles of the next stage-1 launches are [lo1, hi1);
//   mode 1 (after stage 1 of chunk c, on the same stream): the stage-2 bound
//     that chunk allows, kept in chunk c's slot: the tile holding the last
//     index found so far -- every token of the tiles before it is followed by
//     a known index, so its bytes, and the staged bytes and masks after its
//     tile, lie in chunks that have landed and passed stage 1;
//   mode 2: the tiles of the next stage-2 launches: from where the previous
//     ones stopped to chunk c's bound, or with `last` to the document's end.
// The bound is taken in mode 1 because stage 1 of later chunks runs on
// another stream meanwhile and moves the running index count.
__global__ void chunk_range_kernel(const Job *__restrict__ job, uint32_t lo1, uint32_t hi1,
                                   int mode, uint32_t c, int last) {
  pdl_enter();
  const Job &J = *job;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (mode == 0) {
    J.counters[4] = min(lo1, J.counters[2]);
    J.counters[5] = min(hi1, J.counters[2]);
    J.counters[kTicketS1] = 0;
    if (lo1 == 0) {  // the first chunk: no stage-2 tile is done yet
      J.counters[6] = 0;
      J.counters[7] = 0;
    }
    return;
  }
  if (mode == 1) {
    uint32_t hi = 0;
    if (J.n_docs == 1 && !(J.doc_flags[0] & kDocBad)) {
      const uint32_t n = J.doc_nidx[0];
      if (n) hi = J.tile_first[0] + J.idx[idx_base(J, 0) + n - 1] / (uint32_t)kTileBytes;
    }
    J.counters[kChunkSlots + min(c, (uint32_t)kMaxChunkSlots - 1u)] = hi;
    return;
  }
  const uint32_t lo = J.counters[7];
  const uint32_t hi = last ? J.counters[2] : J.counters[kChunkSlots + min(c, (uint32_t)kMaxChunkSlots - 1u)];
  J.counters[6] = lo;
  J.counters[7] = max(hi, lo);
  J.counters[kTicketReduce] = 0;
  J.counters[kTicketBuild] = 0;
  J.counters[kTicketNumbers] = 0;
}

// Per-document results (error precedence: capacity, empty, UTF-8, unclosed
// string, internal, then the first failing token).
__global__ void finalize_kernel(const Job *__restrict__ job) {
  pdl_enter();
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

__global__ void __launch_bounds__(kS2Threads, 7) stage2_reduce_kernel(const Job *__restrict__ job) {
  pdl_enter();
  stage2_reduce<0>(job);
}
__global__ void __launch_bounds__(kS2Threads, 7) stage2_reduce_sub_kernel(const Job *__restrict__ job) {
  pdl_enter();
  stage2_reduce<kSmallShift>(job);
}
__global__ void __launch_bounds__(kS2Threads, 7) stage2_build_kernel(const Job *__restrict__ job) {
  pdl_enter();
  stage2_build<0, false>(job);
}
__global__ void __launch_bounds__(kS2Threads, 7) stage2_build_small_kernel(const Job *__restrict__ job) {
  pdl_enter();
  stage2_build<0, true>(job);
}
__global__ void __launch_bounds__(kS2Threads, 7) stage2_build_sub_kernel(const Job *__restrict__ job) {
  pdl_enter();
  stage2_build<kSmallShift, true>(job);
}

}  // namespace sj
