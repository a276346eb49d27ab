// stage1.cu -- single-pass stage 1 (Sec. 3.1) with decoupled look-backs.
//
// This kernel serves the allocation-free entry point (noalloc.cu) for
// documents of at most 64 MiB; the main parse path uses the reduce-then-scan
// kernels of s1.cu.  Description of the single-pass scheme:
//
// One warp processes a tile of 2 KiB: each lane owns one 64-byte block, the
// paper's unit of work, and builds its 64-bit masks with SWAR classification
// of 4 bytes per 32-bit word.  The carries that the paper passes from one
// 64-byte block to the next (footnote of Sec. 3.1.1) are passed between lanes
// with warp votes and shuffles and between tiles with two decoupled
// look-backs:
//   1. (escape parity, in-string parity, last-byte separator) -- a function of
//      the incoming (escape, in-string) state, published as a 4-entry table;
//   2. the number of indices, for the output offset of the flatten step.
// UTF-8 validation (Sec. 3.1.5) runs per lane over non-ASCII words only.
#include "s1_common.cuh"

namespace sj {

// ---------------------------------------------------------------------------
// Look-back state of phase 1: a function of (escape carry e, in-string q) to
// (e', q', sep').  Table entry x = e + 2q (the state encoding) holds the
// 3-bit result e' | q' << 1 | sep' << 2.
// ---------------------------------------------------------------------------
constexpr uint32_t kIdentity = 0xFFFFFFFFu;
constexpr uint32_t kInitState = 4u;  // e = 0, q = 0, sep = 1 (virtual white space before byte 0)

__device__ __forceinline__ uint32_t apply_fn(uint32_t table, uint32_t state) {
  if (table == kIdentity) return state;
  return (table >> (3 * (state & 3))) & 7u;
}

__device__ __forceinline__ uint32_t compose_fn(uint32_t outer, uint32_t inner) {
  // (outer o inner)(x) = outer(inner(x))
  if (inner == kIdentity) return outer;
  uint32_t r = 0;
#pragma unroll
  for (int x = 0; x < 4; x++) r |= apply_fn(outer, (inner >> (3 * x)) & 7u) << (3 * x);
  return r;
}

__device__ __forceinline__ uint32_t spin_status32(const uint32_t *p, uint32_t *doc_flag) {
  uint32_t v = ld_acquire(p);
  uint32_t n = 0;
  while ((v >> 30) == 0) {
    if (++n > kSpinLimit) {
      atomicOr(doc_flag, kFlagInternal);
      return (kStIncl << 30) | kInitState;
    }
    __nanosleep(32);
    v = ld_acquire(p);
  }
  return v;
}

__device__ __forceinline__ uint64_t spin_status64(const uint64_t *p, uint32_t *doc_flag) {
  uint64_t v = ld_acquire(p);
  uint32_t n = 0;
  while ((v >> 62) == 0) {
    if (++n > kSpinLimit) {
      atomicOr(doc_flag, kFlagInternal);
      return (uint64_t)kStIncl << 62;
    }
    __nanosleep(32);
    v = ld_acquire(p);
  }
  return v;
}

// Incoming (e, q, sep) state of tile t whose predecessors are j_min .. t-1.
__device__ uint32_t lookback_state(const Job &J, uint32_t t, uint32_t j_min, uint32_t d, int lane) {
  uint32_t G = kIdentity;  // composition of the aggregates seen so far (nearest first)
  int64_t j = (int64_t)t - 1;
  for (;;) {
    int64_t jj = j - lane;
    uint32_t st = 0;
    if (jj >= (int64_t)j_min) st = spin_status32(&J.s1_state[jj], &J.doc_flags[d]);
    uint32_t flag = st >> 30;
    unsigned pmask = __ballot_sync(0xFFFFFFFFu, flag == kStIncl);
    int64_t avail = j - (int64_t)j_min + 1;  // predecessors left (>= 1)
    int K;
    uint32_t base;
    bool have_base;
    if (pmask) {
      K = __ffs(pmask) - 1;
      base = __shfl_sync(0xFFFFFFFFu, st & 7u, K);
      have_base = true;
    } else if (avail <= 32) {
      K = (int)avail;
      base = kInitState;
      have_base = true;
    } else {
      K = 32;
      base = 0;
      have_base = false;
    }
    uint32_t fn = st & 0xFFFu;
    if (have_base) {
      uint32_t s = base;
      for (int i = K - 1; i >= 0; i--) s = apply_fn(__shfl_sync(0xFFFFFFFFu, fn, i), s);
      return apply_fn(G, s);
    }
    uint32_t chain = kIdentity;  // f_0 o f_1 o ... o f_31
    for (int i = 31; i >= 0; i--) chain = compose_fn(__shfl_sync(0xFFFFFFFFu, fn, i), chain);
    G = compose_fn(G, chain);
    j -= 32;
  }
}

// Inclusive-before count (exclusive prefix) of tile t.
__device__ uint32_t lookback_count(const Job &J, uint32_t t, uint32_t j_min, uint32_t d, int lane) {
  uint32_t acc = 0;
  int64_t j = (int64_t)t - 1;
  for (;;) {
    int64_t jj = j - lane;
    uint64_t st = 0;
    if (jj >= (int64_t)j_min) st = spin_status64(&J.s1_count[jj], &J.doc_flags[d]);
    uint32_t flag = (uint32_t)(st >> 62);
    unsigned pmask = __ballot_sync(0xFFFFFFFFu, flag == kStIncl);
    int64_t avail = j - (int64_t)j_min + 1;
    int K = pmask ? __ffs(pmask) - 1 : (avail <= 32 ? (int)avail : 32);
    uint32_t v = (lane <= K && jj >= (int64_t)j_min) ? (uint32_t)st : 0u;
    if (!pmask && lane == K) v = 0;  // no base in this window
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    acc += v;
    if (pmask || avail <= 32) return acc;
    j -= 32;
  }
}

// ---------------------------------------------------------------------------
// The stage-1 kernel: persistent warps take tiles in ticket order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * kS1Warps) stage1_kernel(const Job *__restrict__ job) {
  const Job &J = *job;
  __shared__ uint32_t stage[kS1Warps][kTileBytes];  // flatten staging, per warp
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint32_t *out_stage = stage[wid];
  const uint32_t n_tiles = J.counters[2];

  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&J.counters[0], 1u);
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    if (t >= n_tiles) break;
    const uint32_t d = doc_of_tile(J, t);
    const uint32_t j_min = J.tile_first[d];
    const uint32_t tt = t - j_min;
    const uint32_t ntiles_d = J.tile_first[d + 1] - j_min;
    const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
    const uint8_t *doc = J.base + J.doc_off[d];
    const uint64_t blk = (uint64_t)tt * kTileBytes + (uint64_t)lane * kBlockBytes;

    uint32_t w[16];
    load_block(doc, len, blk, w);
    BlockMasks m;
    classify_block(w, m);

    // ---- UTF-8 ------------------------------------------------------------
    {
      uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, w[15], 1);
      int nprev = 3;
      if (lane == 0) {
        prev = 0;
        nprev = blk >= 3 ? 3 : (int)blk;
        for (int k = 0; k < nprev; k++) prev |= (uint32_t)doc[blk - nprev + k] << (8 * (4 - nprev + k));
      }
      bool need_check = m.nonascii != 0 || ((prev & 0xC0C0C000u) & ((prev << 1) & 0x80808000u));
      bool ends_here = blk < len && blk + 64 >= len;
      if (blk < len && need_check && utf8_block_error(w, prev, nprev, ends_here))
        atomicOr(&J.doc_flags[d], kFlagUtf8);
    }

    // ---- escapes and quotes under both hypotheses for the carried escape ----
    const bool all_bs = (m.bs == ~0ull);
    const uint32_t tail = (uint32_t)__clzll((long long)~m.bs) & 1u;  // trailing run parity
    const unsigned nb = __ballot_sync(0xFFFFFFFFu, !all_bs);
    const unsigned tb = __ballot_sync(0xFFFFFFFFu, tail);
    const unsigned below = (1u << lane) - 1u;
    const bool known = (nb & below) != 0;  // escape carry into this lane fixed by an earlier lane
    uint32_t e_known = 0;
    if (known) e_known = (tb >> (31 - __clz(nb & below))) & 1u;
    const uint64_t od0 = escaped_no_carry(m.bs);
    const uint64_t flip = first_non_bs(m.bs);
    const uint64_t q0 = m.quote & ~od0;                 // real quotes with no carry in
    const uint32_t flipq = (m.quote & flip) ? 1u : 0u;  // parity change with a carry in
    const uint32_t par0 = __popcll(q0) & 1u;
    // parity of this lane with e = e_known (unknown lanes: hypothesis e = 0)
    const uint32_t par_h0 = par0 ^ (e_known & flipq);
    const unsigned pb0 = __ballot_sync(0xFFFFFFFFu, par_h0);
    const int first_lane = nb ? __ffs(nb) - 1 : -1;  // the one lane whose carry is the tile's
    const uint32_t flipq_first = first_lane >= 0 ? __shfl_sync(0xFFFFFFFFu, flipq, first_lane) : 0u;
    const uint32_t qpar0 = __popc(pb0) & 1u;
    const uint32_t qpar1 = qpar0 ^ flipq_first;

    // ---- phase-1 aggregate: f(e_in, q_in) -> (e_out, q_out, sep_out) -------
    uint32_t table = 0;
    {
      const int last_nb = nb ? 31 - __clz(nb) : -1;
      const uint32_t e_fixed = last_nb >= 0 ? (tb >> last_nb) & 1u : 0u;
      // last byte of the tile (lane 31, byte 63)
      const uint32_t lastc = __shfl_sync(0xFFFFFFFFu, w[15] >> 24, 31);
      const uint64_t od_last0 = __shfl_sync(0xFFFFFFFFu, od0 >> 63, 31);
      const uint32_t flip_last = __shfl_sync(0xFFFFFFFFu, (uint32_t)(flip >> 63), 31);
      const bool lane31_known = __shfl_sync(0xFFFFFFFFu, known, 31);
      const uint32_t e31_known = __shfl_sync(0xFFFFFFFFu, e_known, 31);
#pragma unroll
      for (uint32_t x = 0; x < 4; x++) {
        const uint32_t he = x & 1, hq = x >> 1;  // x = e + 2q, the state encoding
        const uint32_t eo = last_nb >= 0 ? e_fixed : he;
        const uint32_t qo = hq ^ (he ? qpar1 : qpar0);
        const uint32_t e31 = lane31_known ? e31_known : he;
        const uint32_t esc_last = (uint32_t)od_last0 ^ (e31 & flip_last);
        uint32_t sep;
        if (lastc == ' ' || lastc == '\n' || lastc == '\r' || lastc == '\t') sep = 1;
        else if (lastc == ',' || lastc == ':' || lastc == '[' || lastc == ']' || lastc == '{' || lastc == '}')
          sep = qo ^ 1u;
        else if (lastc == '"') sep = esc_last ^ 1u;
        else sep = 0;
        table |= (eo | (qo << 1) | (sep << 2)) << (3 * x);
      }
    }
    if (lane == 0) st_release(&J.s1_state[t], (kStAgg << 30) | table);

    // ---- phase-1 look-back -------------------------------------------------
    uint32_t s_in = kInitState;
    if (tt > 0) s_in = lookback_state(J, t, j_min, d, lane);
    const uint32_t s_out = apply_fn(table, s_in);
    if (lane == 0) st_release(&J.s1_state[t], (kStIncl << 30) | s_out);
    if (tt == ntiles_d - 1 && lane == 0 && ((s_out >> 1) & 1u)) atomicOr(&J.doc_flags[d], kFlagUnclosed);

    // ---- final masks of this lane (Figs. "identifyquoteregion", "identifypseudo")
    const uint32_t e_in_tile = s_in & 1u;
    const uint32_t q_in_tile = (s_in >> 1) & 1u;
    const uint32_t e_lane = known ? e_known : e_in_tile;
    const uint64_t Q = q0 ^ ((e_lane && flipq) ? flip : 0ull);
    const uint32_t par = par0 ^ (e_lane & flipq);
    const unsigned pb = __ballot_sync(0xFFFFFFFFu, par);
    const uint32_t q_lane = q_in_tile ^ (__popc(pb & below) & 1u);
    const uint64_t R = prefix_xor(Q) ^ (q_lane ? ~0ull : 0ull);
    const uint64_t S1 = (m.op & ~R) | Q;
    const uint64_t SW = S1 | m.ws;
    uint32_t sep_in = __shfl_up_sync(0xFFFFFFFFu, (uint32_t)(SW >> 63), 1);
    if (lane == 0) sep_in = (s_in >> 2) & 1u;
    uint64_t P = ((SW << 1) | sep_in) & ~m.ws & ~R;
    const uint64_t S = (S1 | P) & ~(Q & ~R);

    // ---- counts and phase-2 look-back --------------------------------------
    const uint32_t cnt = __popcll(S);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += v;
    }
    const uint32_t tile_n = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (lane == 0) st_release(&J.s1_count[t], ((uint64_t)kStAgg << 62) | tile_n);
    uint32_t base = 0;
    if (tt > 0) base = lookback_count(J, t, j_min, d, lane);
    if (lane == 0) {
      st_release(&J.s1_count[t], ((uint64_t)kStIncl << 62) | (uint64_t)(base + tile_n));
      J.tile_cnt[t] = tile_n;
      J.tile_off[t] = base;
      if (tt == ntiles_d - 1) J.doc_nidx[d] = base + tile_n;
    }

    // ---- flatten (Sec. 3.1.4): staged in shared memory, stored coalesced ----
    {
      uint32_t o = incl - cnt;
      uint64_t s = S;
      const uint32_t pos0 = (uint32_t)blk;
      while (s) {
        out_stage[o++] = pos0 + (uint32_t)(__ffsll((long long)s) - 1);
        s &= s - 1;
      }
      __syncwarp();
      uint32_t *dst = J.idx + idx_base(J, d) + base;
      for (uint32_t k = lane; k < tile_n; k += 32) dst[k] = out_stage[k];
      __syncwarp();
    }
  }
}

}  // namespace sj
