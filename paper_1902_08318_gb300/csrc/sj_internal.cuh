// sj_internal.cuh -- shared definitions of the CUDA kernels (device side).
#pragma once
#include <stdint.h>

#include "sj.h"

namespace sj {

// Stage 1 (Sec. 3.1) works on 64-byte blocks as in the paper: one block per
// lane, one warp per tile of 32 blocks.  Stage 2 (Sec. 3.2) processes the
// indices of one stage-1 tile per thread block.  Tiles never span documents.
constexpr int kBlockBytes = 64;
constexpr int kTileBytes = 32 * kBlockBytes;  // 2048
constexpr int kS1Warps = 4;                   // tiles (warps) per stage-1 thread block
constexpr int kS2Threads = 128;               // threads per stage-2 thread block
constexpr int kMaxTileTokens = kTileBytes;    // at most one index per byte
constexpr int kOpenGlobal = 2 * kMaxTileTokens + 1;  // relative levels [-2048, 2048] of one tile
constexpr uint32_t kMaxDepthLimit = 4096;
constexpr uint64_t kMaxDocBytes = 0xFFFFFF00ull;  // keeps positions and tape indices in u32
// Bounded waits: polls of a look-back status word before a wait gives up
// (the waiting tile's document is then marked INTERNAL).  A test build sets a
// small limit to check that a wait which nothing ends does end.
#ifdef SJ_SPIN_LIMIT
constexpr uint32_t kSpinLimit = SJ_SPIN_LIMIT;
#else
constexpr uint32_t kSpinLimit = 1u << 24;
#endif

// Programmatic dependent launch.  The kernels of a run after the first may be
// launched with programmatic stream serialization (launch_k with pdl): the
// GPU then launches a kernel as soon as every block of the kernel ahead of it
// in the stream has exited, without waiting for that kernel's completion to
// be signalled, and the kernel's first act, pdl_enter(), waits until the
// kernel ahead has completed and its writes are visible.  The results are
// those of plain launches; what overlaps is each launch with the end of the
// kernel before.  No kernel triggers its dependents early: blocks of the next
// kernel resident and waiting beside a running kernel made the 1 GiB parse
// 3% slower.  Without the attribute the wait does nothing.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... P, typename... A>
inline void launch_k(bool pdl, void (*k)(P...), unsigned grid, unsigned block, size_t smem,
                     cudaStream_t s, A... a) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t c = {};
  c.gridDim = dim3(grid);
  c.blockDim = dim3(block);
  c.dynamicSmemBytes = smem;
  c.stream = s;
  c.attrs = at;
  c.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&c, k, a...);
}

// Per-document flags written by the kernels.
constexpr uint32_t kFlagUtf8 = 1, kFlagUnclosed = 2, kFlagInternal = 4, kFlagCapacity = 8;

// Look-back status values (top two bits of a status word).
constexpr uint32_t kStAgg = 1, kStIncl = 2;

constexpr uint32_t kNoTile = 0xFFFFFFFFu;

// Stage-1 tile aggregate (Sec. 3.1, carried in-string bit): the parity of the
// tile's real quotes and its index counts when it is entered outside (c0) or
// inside (c1) a string.  `head` marks the first tile of a document.
struct S1Agg {
  uint32_t qpar, c0, c1, head;
};
// Stage-1 tile prefix: the in-string bit entering the tile and its index offset.
struct S1Pre {
  uint32_t base, q_in;
};
// Stage-2 tile aggregate: depth change, lowest depth reached relative to the
// tile start (<= 0), tape words and string-buffer bytes of its tokens.
struct S2Agg {
  int32_t dd, mn;
  uint32_t w, head;
  uint64_t s;
};
// Stage-2 tile prefix: absolute depth before the tile, its lowest depth, its
// first tape index and string-buffer offset (document relative).
struct S2Pre {
  int32_t d_start, low;
  uint32_t tape_start, jump;  // jump: nearest earlier tile of the document with a lower `low`
  uint64_t str_start;
};
constexpr int kScanBlock = 1024;  // tiles per thread block in the tile scans
// Parsers of at most this many stage-2 tiles scan in one thread block and
// build the sparse table there; whole-document runs only.
constexpr uint32_t kSmallTiles = 2048;
// Parsers of at most kSubTiles tiles (1 MiB of input) split each stage-1
// tile in 2^kSmallShift stage-2 tiles (512 bytes) on whole-document runs, so
// that a small document keeps four times the warps busy in stage 2.
constexpr uint32_t kSmallShift = 2;
constexpr uint32_t kSubTiles = kSmallTiles >> kSmallShift;
// Runs of at most this many documents take the run descriptor and offsets
// from pinned host memory in the set-up kernel and write their results
// there (no copy operations in the run).
constexpr uint32_t kZeroCopyDocs = 1024;

// Everything a run needs, in device memory (one copy per parser; refreshed
// by a host-to-device copy before each run so that one captured graph serves
// every call).
struct Job {
  const uint8_t *base;      // 16-byte aligned buffer holding the documents
  const uint8_t *src;       // when not null: the same bytes in pinned host memory; stage 1
                            // reads them there and writes them to `base` (one document)
  const uint64_t *doc_off;  // n_docs + 1 byte offsets into base
  uint32_t n_docs;
  uint32_t max_depth;
  // Stage-2 tiles are the stage-1 tiles split in 2^s2_shift (0 or 2): small
  // whole-document runs split them so that a small document keeps more warps
  // busy in the stage-2 passes.
  uint32_t s2_shift;
  uint64_t max_doc_len;
  // scratch
  uint32_t *tile_first;     // n_docs + 1: first stage-1 tile of each document
  uint32_t *counters;       // [0] look-back ticket, [2] number of tiles, [4..7] tile ranges
  uint32_t *s1_state;       // per tile: escape/quote/separator look-back word
  uint64_t *s1_count;       // per tile: index-count look-back word
  uint32_t *tile_cnt;       // per tile: indices produced
  uint32_t *tile_off;       // per tile: document-relative offset of its first index
  uint32_t *surv;           // per index slot: open containers left by a tile (by level)
  // reduce-then-scan state
  S1Agg *s1_rec;            // per tile
  S1Pre *s1_pre;            // per tile
  uint64_t *s1_blk;         // per 64-byte block: final mask entered outside / inside a string
  S2Agg *s2_rec;            // per tile
  S2Pre *s2_pre;            // per tile
  void *scan_agg;           // per scan block (sized for S2Agg): the stage-2 tile scan
  void *scan_pre;           // per scan block
  void *scan_agg1;          // per scan block: the stage-1 tile scan (its own, so that the two
  void *scan_pre1;          // scans may run at once on different chunks)
  int32_t *spt;             // sparse table of tile `low` minima: level k at spt + k * spt_stride
  uint32_t spt_stride, spt_levels;
  ulonglong2 *s1_qx;        // per 64-byte block: real quotes, backslash|control bytes
  uint32_t *slen;           // per index slot: normalised length of the string token there
  uint64_t *meta;           // per index slot: token facts from the stage-2 reduce pass
  uint8_t *unesc;           // per input byte: normalised strings with escapes, at their position
  uint32_t *nlist;          // per index slot: the number tokens of each tile, listed from its
                            // first slot (index and tape slot in the tile, 16 bits each)
  uint64_t *numv;           // per index slot: a number's value word (small whole runs only)
  uint32_t *tile_nnum;      // per tile: number tokens
  uint16_t *open_g;         // per stage-2 reduce warp: level table for tiles with many tokens
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

// Tile ranges of the launches: stage-1 kernels work on tiles [counters[4],
// counters[5]), stage-2 kernels on [counters[6], counters[7]) (counters[8]
// to [11] are the tile tickets of four passes).  A run over
// resident input sets both to all tiles; a run over a host document that
// arrives in chunks moves them forward chunk by chunk (chunk_range_kernel).
// counters[kChunkSlots + c]: the stage-2 bound found after stage 1 of chunk c
constexpr int kChunkSlots = 16, kMaxChunkSlots = 64;
constexpr int kCounters = kChunkSlots + kMaxChunkSlots;
// tile tickets: stage-2 reduce, build and numbers; stage-1 blocks
constexpr int kTicketReduce = 8, kTicketBuild = 9, kTicketNumbers = 10, kTicketS1 = 11;

// Tiles of uneven cost: a warp takes its first tile by its index in the grid
// and each later one from a ticket counter (reset before each launch) when it
// finishes the previous, so no tail of busy warps is left.  The next ticket
// is drawn when a tile starts and read when it ends, which hides the atomic's
// latency; no ticket is drawn while no tile lies past the first round (small
// inputs never touch the counter).  Usage:
//   TileTickets tt(J, kTicket..., lo, hi, warp_in_grid, warps_in_grid, lane);
//   for (uint32_t t = tt.first(); t < hi; t = tt.next()) { tt.draw(); ... }
struct TileTickets {
  uint32_t *ctr;
  uint32_t past, first_t, hi, tk;
  int lane;
  __device__ TileTickets(const Job &J, int which, uint32_t lo, uint32_t hi_, uint32_t gw,
                         uint32_t nw, int lane_)
      : ctr(&J.counters[which]), past(lo + nw), first_t(lo + gw), hi(hi_), tk(0), lane(lane_) {}
  __device__ __forceinline__ uint32_t first() const { return first_t; }
  __device__ __forceinline__ void draw() {
    tk = past < hi && lane == 0 ? atomicAdd(ctr, 1u) : 0u;
  }
  __device__ __forceinline__ uint32_t next() const {
    return past + __shfl_sync(0xFFFFFFFFu, tk, 0);
  }
};
__device__ __forceinline__ void s1_range(const Job &J, uint32_t &lo, uint32_t &hi) {
  lo = J.counters[4];
  hi = J.counters[5];
}
__device__ __forceinline__ void s2_range(const Job &J, uint32_t &lo, uint32_t &hi) {
  lo = J.counters[6];
  hi = J.counters[7];
}

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

// Stage-2 tiles (2^s2_shift per stage-1 tile): the document owning stage-2
// tile t, and the first stage-2 tile of document d.
__device__ __forceinline__ uint32_t s2_doc(const Job &J, uint32_t t) {
  return doc_of_tile(J, t >> J.s2_shift);
}
__device__ __forceinline__ uint32_t s2_first(const Job &J, uint32_t d) {
  return J.tile_first[d] << J.s2_shift;
}

// ---- memory-ordering helpers for the decoupled look-back ----------------
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

}  // namespace sj
