// sj_internal.cuh -- shared definitions of the CUDA kernels (device side).
#pragma once
#include <stdint.h>

#include "sj.h"

namespace sj {

// Stage 1 (Sec. 3.1) works on 64-byte blocks as in the paper: one block per
// lane, one warp per tile of 32 blocks.  Stage 2 (Sec. 3.2) takes the indices
// of one tile per warp.  Tiles never span documents.
constexpr int kBlockBytes = 64;
constexpr int kTileBytes = 32 * kBlockBytes;  // 2048
constexpr int kMaxTileTokens = kTileBytes;    // at most one index per byte
constexpr int kOpenGlobal = 2 * kMaxTileTokens + 1;  // relative levels [-2048, 2048] of one tile
constexpr uint32_t kMaxDepthLimit = 4096;
constexpr uint64_t kMaxDocBytes = 0xFFFFFF00ull;  // keeps positions and tape indices in u32
// Bounded waits: polls of a look-back status word (with a growing sleep of at
// most ~1 us between polls, so a wait gives up after about 16 s) and of a bulk
// copy's barrier.
constexpr uint32_t kSpinLimit = 1u << 24;

// Per-document flags written by the kernels.
constexpr uint32_t kFlagUtf8 = 1, kFlagUnclosed = 2, kFlagInternal = 4, kFlagCapacity = 8;
constexpr uint32_t kDocBad = kFlagUtf8 | kFlagUnclosed | kFlagCapacity | kFlagInternal;

constexpr uint32_t kNoTile = 0xFFFFFFFFu;

// Stage-2 tile aggregate: depth change, lowest depth reached relative to the
// tile start (<= 0, and <= dd), tape words and string-buffer bytes of its
// tokens.
struct S2Agg {
  int32_t dd, mn;
  uint32_t w, pad;
  uint64_t s;
};
// Stage-2 inclusive prefix of a tile (document relative): depth after it,
// tape words and string-buffer bytes of the tiles up to and including it.
struct S2Incl {
  int32_t d;
  uint32_t w;
  uint64_t s;
};
// Stage-2 exclusive prefix of a tile, as the build pass reads it: depth
// before the tile, its lowest depth, its first tape index and string-buffer
// offset (document relative).
struct S2Pre {
  int32_t d_start, low;
  uint32_t tape_start, pad;
  uint64_t str_start;
};

// Everything a run needs, in device memory (one copy per parser; refreshed
// by a host-to-device copy before each run so that one captured graph serves
// every call).
struct Job {
  const uint8_t *base;      // the documents (device memory)
  const uint8_t *src;       // when not null: the same bytes in pinned host memory; the
                            // first pass reads them there and writes them to `base`
  const uint64_t *doc_off;  // n_docs + 1 byte offsets into base
  uint32_t n_docs;
  uint32_t max_depth;
  uint64_t max_doc_len;
  uint32_t epoch;           // run number: tags look-back status words (never 0)
  uint32_t s1_only;         // 1: stage 1 only (indices and stage-1 flags)
  // scratch
  uint32_t *tile_first;     // n_docs + 1: first tile of each document
  uint32_t *counters;       // see kCtr*
  uint64_t *st1;            // per tile: stage-1 look-back status (see parse1.cu)
  uint32_t *st2;            // per tile: stage-2 look-back flag (epoch << 2 | state)
  S2Agg *agg2;              // per tile: stage-2 aggregate
  S2Incl *inc2;             // per tile: stage-2 inclusive prefix
  S2Pre *pre2;              // per tile: stage-2 exclusive prefix
  uint64_t *jump;           // per tile: nearest earlier tile with a lower `low` (epoch-tagged)
  uint32_t *tile_cnt;       // per tile: indices in the tile
  uint32_t *tile_off;       // per tile: document-relative offset of its first index
  uint32_t *tile_nstr;      // per tile: string tokens
  uint32_t *tile_nnum;      // per tile: number tokens
  uint32_t *surv;           // per index slot: open containers left by a tile (by level)
  uint32_t *slen;           // per index slot: the strings of a tile, listed from its first slot
  uint64_t *nlist;          // per index slot: the numbers of a tile, listed from its first slot
  uint16_t *open_g;         // per warp: level table for tiles with many tokens
  uint64_t *front;          // per index slot + tile: open container of each level entering a tile
  // outputs
  uint32_t *idx;
  uint64_t *tape;
  uint8_t *strings;
  uint32_t *doc_flags;
  uint32_t *doc_nidx;
  unsigned long long *doc_err;  // min over (token << 8 | code)
  uint64_t *doc_tape;
  uint64_t *doc_str;
  sj_doc_result *results;
};

// counters: tile tickets of the three passes and the tile count
constexpr int kCtrTicket1 = 0, kCtrTicketBuild = 1, kCtrTicketNum = 2, kCtrTiles = 3;
constexpr int kCounters = 8;

// Tiles of uneven cost: a warp takes its first tile by its index in the grid
// and each later one from a ticket counter (reset before each launch) when it
// finishes the previous, so no tail of busy warps is left.  Used by the passes
// that wait on no other tile; the next ticket is drawn when a tile starts and
// read when it ends, which hides the atomic's latency.  Usage:
//   TileTickets tt(J, kCtr..., n, warp_in_grid, warps_in_grid, lane);
//   for (uint32_t t = tt.first(); t < n; t = tt.next()) { tt.draw(); ... }
struct TileTickets {
  uint32_t *ctr;
  uint32_t past, first_t, hi, tk;
  int lane;
  __device__ TileTickets(const Job &J, int which, uint32_t hi_, uint32_t gw, uint32_t nw,
                         int lane_)
      : ctr(&J.counters[which]), past(nw), first_t(gw), hi(hi_), tk(0), lane(lane_) {}
  __device__ __forceinline__ uint32_t first() const { return first_t; }
  __device__ __forceinline__ void draw() {
    tk = past < hi && lane == 0 ? atomicAdd(ctr, 1u) : 0u;
  }
  __device__ __forceinline__ uint32_t next() const {
    return past + __shfl_sync(0xFFFFFFFFu, tk, 0);
  }
};

// Output placement: each document gets capacity proportional to its length.
__device__ __forceinline__ uint64_t rel_off(const Job &J, uint32_t d) {
  return J.doc_off[d] - J.doc_off[0];
}
__device__ __forceinline__ uint64_t idx_base(const Job &J, uint32_t d) { return rel_off(J, d); }
__device__ __forceinline__ uint64_t tape_base(const Job &J, uint32_t d) {
  return rel_off(J, d) + 3ull * d;
}
__device__ __forceinline__ uint64_t str_base(const Job &J, uint32_t d) {
  return (5ull * rel_off(J, d)) / 2 + 8ull * d;
}

// Document owning global tile t (tile_first is non-decreasing).
__device__ __forceinline__ uint32_t doc_of_tile(const Job &J, uint32_t t) {
  uint32_t lo = 0, hi = J.n_docs;  // answer in [lo, hi)
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (J.tile_first[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void report(const Job &J, uint32_t d, uint64_t token, int code) {
  atomicMin(&J.doc_err[d], (unsigned long long)((token << 8) | (uint64_t)code));
}

// ---- memory-ordering helpers for the look-backs ----------------------------
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_acquire(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(uint64_t *p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---- token kinds (first byte of an index, Sec. 3.2) ----------------------
enum : uint8_t {
  K_OTHER = 0, K_OPEN_OBJ = 1, K_OPEN_ARR = 2, K_CLOSE_OBJ = 3, K_CLOSE_ARR = 4,
  K_COMMA = 5, K_COLON = 6, K_STRING = 7, K_NUMBER = 8, K_TRUE = 9, K_FALSE = 10, K_NULL = 11
};

__device__ __forceinline__ uint8_t token_kind(uint8_t c) {
  switch (c) {
    case '{': return K_OPEN_OBJ;
    case '[': return K_OPEN_ARR;
    case '}': return K_CLOSE_OBJ;
    case ']': return K_CLOSE_ARR;
    case ',': return K_COMMA;
    case ':': return K_COLON;
    case '"': return K_STRING;
    case 't': return K_TRUE;
    case 'f': return K_FALSE;
    case 'n': return K_NULL;
    default: return (c == '-' || (uint8_t)(c - '0') < 10) ? K_NUMBER : K_OTHER;
  }
}
__device__ __forceinline__ bool is_open(uint8_t k) { return k == K_OPEN_OBJ || k == K_OPEN_ARR; }
__device__ __forceinline__ bool is_close(uint8_t k) { return k == K_CLOSE_OBJ || k == K_CLOSE_ARR; }
__device__ __forceinline__ bool is_atom(uint8_t k) { return k >= K_TRUE && k <= K_NULL; }
// A token that can start a value.
__device__ __forceinline__ bool is_value_start(uint8_t k) {
  return is_open(k) || k == K_STRING || k == K_NUMBER || is_atom(k);
}
__device__ __forceinline__ int depth_delta(uint8_t k) { return is_open(k) ? 1 : (is_close(k) ? -1 : 0); }
__device__ __forceinline__ uint32_t tape_words_of(uint8_t k) {
  return k == K_NUMBER ? 2u : ((is_open(k) || is_close(k) || k == K_STRING || is_atom(k)) ? 1u : 0u);
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

// A string's entry in `slen`: an error code, or its normalised length and
// whether it holds escapes (then the build pass walks it again to write it).
constexpr uint32_t kSlenErr = 0x80000000u, kSlenWalk = 0x40000000u, kSlenLen = 0x3FFFFFFFu;

// Level table of a warp: the container currently open at each level relative
// to the tile start (0 = none, else bit 15, bit 14 = object, bits 0-11 = the
// opener's tape slot relative to the tile).  A tile with fewer than 512
// tokens spans fewer than 512 levels, so they fit in shared memory modulo
// 512; other tiles use the warp's table in global memory (levels -2048 to
// 2048, biased).  Entries are zero between tiles.
struct OpenTable {
  uint16_t *p;
  uint32_t mask;
  int32_t bias;
  __device__ __forceinline__ uint16_t &at(int32_t l) const { return p[(uint32_t)(l + bias) & mask]; }
};

// ---- the staged window of a tile (shared memory) -----------------------------
// A warp copies the bytes around its tile into shared memory: positions
// [t0 - pre, t0 + kTileBytes + post) of the document, clipped to it, widened
// to 16-byte aligned addresses (every 16-byte chunk holds at least one byte of
// the document, so no read leaves the pages the document uses).
struct Window {
  const uint8_t *s;  // shared memory: byte of document position p is s[p - sbase]
  int64_t sbase;
  uint64_t lo, hi;   // staged document positions [lo, hi)
  const uint8_t *g;  // global copy of the document (positions outside the window)
  __device__ __forceinline__ bool has(uint64_t p, uint64_t q) const { return p >= lo && q <= hi; }
  __device__ __forceinline__ uint8_t at(uint64_t p) const {
    return (p >= lo && p < hi) ? s[(int64_t)p - sbase] : g[p];
  }
  __device__ __forceinline__ const uint8_t *ptr(uint64_t p, uint64_t q) const {
    return has(p, q) ? s + ((int64_t)p - sbase) : g + p;
  }
};

// Byte extent of the window: the aligned addresses [a0, a1) around document
// positions [p0, p1) of a document at `doc` of length len.
__device__ __forceinline__ void window_extent(const uint8_t *doc, uint64_t len, uint64_t p0,
                                              uint64_t p1, uintptr_t &a0, uintptr_t &a1) {
  if (p1 > len) p1 = len;
  a0 = (uintptr_t)(doc + p0) & ~(uintptr_t)15;
  a1 = ((uintptr_t)(doc + p1) + 15) & ~(uintptr_t)15;
}

// mbarrier-tracked bulk copy (TMA, cp.async.bulk) of [a0, a1) from global into
// shared memory, issued by lane 0.  Both ends are 16-byte aligned.
__device__ __forceinline__ void bulk_copy_start(uint8_t *dst, uintptr_t a0, uint32_t bytes,
                                                uint64_t *mbar, int lane) {
  if (lane == 0) {
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
    const uint32_t sd = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sd),
        "l"(a0), "r"(bytes), "r"(mb)
        : "memory");
  }
}

// Wait (bounded) for the copy of the current phase; false if it never came.
__device__ __forceinline__ bool bulk_copy_wait(uint64_t *mbar, uint32_t phase) {
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
  for (uint32_t n = 0; n < kSpinLimit; n++) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mb), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, int lane) {
  if (lane == 0) {
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
}

// Stage the window through 16-byte loads by the lanes (used for pinned host
// memory, which the bulk copy is not asked to read).
__device__ __forceinline__ void lane_copy(uint8_t *dst, uintptr_t a0, uintptr_t a1, int lane) {
  const uint32_t n = (uint32_t)((a1 - a0) >> 4);
  for (uint32_t c = lane; c < n; c += 32)
    reinterpret_cast<uint4 *>(dst)[c] = *reinterpret_cast<const uint4 *>(a0 + 16 * (uintptr_t)c);
}

}  // namespace sj
