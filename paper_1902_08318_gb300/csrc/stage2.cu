// stage2.cu -- stage 2 of the parser (Sec. 3.2) on sm_103a.
//
// The paper walks the indices with a goto state machine and a stack of
// open scopes.  Here a thread block takes the indices of one stage-1 tile
// (at most 2048) and replaces the walk with scans:
//   - depth: the +1/-1 prefix sum of the brackets;
//   - the enclosing container of every token (its "parent"): the last token
//     before it whose depth-after equals its depth-before minus one, found in
//     shared memory when it lies in the tile and otherwise in the tile
//     frontier (the open containers, by level) carried by the look-back;
//   - tape slots and string-buffer bytes: prefix sums of the per-token sizes.
// A decoupled look-back over tiles carries (depth, tape slot, string offset)
// and lets each tile reach the containers left open by earlier tiles.
// Then every token checks its grammar against its neighbours and parent,
// and writes its tape words; strings are normalised and numbers converted.
#include "number.cuh"
#include "sj_internal.cuh"
#include "strings.cuh"

namespace sj {

constexpr int kChain = 64;  // aggregates composed before waiting for an inclusive prefix

struct ChainEnt {
  uint32_t tile;
  int32_t low;          // lowest absolute depth reached in the tile
  int32_t d_end;        // absolute depth after the tile
  uint32_t tape_start;  // absolute (document) tape index of its first word
};

__device__ __forceinline__ uint32_t spin_flag(const uint32_t *p, uint32_t want_min, uint32_t *doc_flag) {
  uint32_t v = ld_acquire(p);
  uint32_t n = 0;
  while (v < want_min) {
    if (++n > kSpinLimit) {
      atomicOr(doc_flag, kFlagInternal);
      return 0;
    }
    __nanosleep(64);
    v = ld_acquire(p);
  }
  return v;
}

__device__ __forceinline__ void report(const Job &J, uint32_t d, uint64_t token, int code) {
  atomicMin(&J.doc_err[d], (unsigned long long)((token << 8) | (uint64_t)code));
}

__device__ __forceinline__ uint8_t kind_at(const Job &J, const uint32_t *idxp, const uint8_t *doc,
                                           int64_t g) {
  return g < 0 ? K_OTHER : token_kind(doc[idxp[g]]);
}

__global__ void __launch_bounds__(kS2Threads) stage2_kernel(const Job *__restrict__ job) {
  const Job &J = *job;
  __shared__ uint32_t s_pos[kMaxTileTokens + 1];
  __shared__ uint32_t s_slen[kMaxTileTokens];  // normalised string length, or 0x80000000 | error
  __shared__ int16_t s_D[kMaxTileTokens];      // depth after the token, relative to the tile
  __shared__ int16_t s_par[kMaxTileTokens];    // parent in the tile, or -1
  __shared__ uint16_t s_tape[kMaxTileTokens];  // tape slot relative to the tile
  __shared__ uint8_t s_kind[kMaxTileTokens];
  __shared__ uint32_t s_closed[kMaxTileTokens / 32];  // bit set: opener closed in the tile
  __shared__ int16_t s_chunkmin[kMaxTileTokens / 32];
  // incoming frontier, levels [lo, d_start]: tape index of the open container and its kind
  __shared__ uint32_t s_front_tape[kMaxTileTokens + 1];
  __shared__ uint8_t s_front_kind[kMaxTileTokens + 1];  // K_OPEN_OBJ, K_OPEN_ARR, or K_OTHER (none)
  __shared__ ChainEnt s_chain[kChain];
  __shared__ int32_t s_scan_d[kS2Threads], s_scan_min[kS2Threads];
  __shared__ uint32_t s_scan_w[kS2Threads];
  __shared__ uint64_t s_scan_s[kS2Threads];
  __shared__ uint32_t s_t;
  __shared__ int32_t s_min_rel, s_d_delta, s_d_start, s_front_lo;
  __shared__ uint32_t s_words, s_tape_start;
  __shared__ uint64_t s_strbytes, s_str_start;

  const int tid = threadIdx.x;
  const uint32_t n_tiles = J.counters[2];

  for (;;) {
    if (tid == 0) s_t = atomicAdd(&J.counters[1], 1u);
    __syncthreads();
    const uint32_t t = s_t;
    if (t >= n_tiles) break;
    const uint32_t d = doc_of_tile(J, t);
    const uint32_t j_min = J.tile_first[d];
    const uint32_t tt = t - j_min;
    const uint32_t ntiles_d = J.tile_first[d + 1] - j_min;
    const uint32_t flags = J.doc_flags[d];
    const uint32_t nidx = J.doc_nidx[d];
    if ((flags & (kFlagUtf8 | kFlagUnclosed | kFlagInternal | kFlagCapacity)) || nidx == 0) {
      __syncthreads();
      continue;  // every tile of this document skips; nobody waits on it
    }
    const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
    const uint8_t *doc = J.base + J.doc_off[d];
    const uint32_t *idxp = J.idx + idx_base(J, d);
    uint32_t *survp = J.surv + idx_base(J, d);
    uint64_t *tape = J.tape + tape_base(J, d);
    uint8_t *strs = J.strings + str_base(J, d);
    const uint64_t tape_cap = len + 3;
    const uint64_t str_cap = str_base(J, d + 1) - str_base(J, d);
    const uint32_t cnt = J.tile_cnt[t];
    const uint32_t off = J.tile_off[t];

    // ---- A. positions of the tile's tokens (+ the next one) ----------------
    for (uint32_t j = tid; j < cnt; j += kS2Threads) s_pos[j] = idxp[off + j];
    if (tid == 0) s_pos[cnt] = (off + cnt < nidx) ? idxp[off + cnt] : (uint32_t)len;
    for (uint32_t j = tid; j < kMaxTileTokens / 32; j += kS2Threads) s_closed[j] = 0;
    __syncthreads();

    // ---- B. per-token sizes, each thread over a contiguous range ------------
    const uint32_t per = (cnt + kS2Threads - 1) / kS2Threads;
    const uint32_t a = min(cnt, tid * per), b = min(cnt, a + per);
    int32_t dsum = 0, dmin = 0;
    uint32_t wsum = 0;
    uint64_t ssum = 0;
    for (uint32_t j = a; j < b; j++) {
      const uint32_t pos = s_pos[j];
      const uint8_t k = token_kind(doc[pos]);
      s_kind[j] = k;
      dsum += depth_delta(k);
      dmin = min(dmin, dsum);
      wsum += tape_words_of(k);
      if (k == K_STRING) {
        int err;
        uint32_t n = string_walk<false>(doc + pos + 1, doc + s_pos[j + 1], err, nullptr);
        s_slen[j] = err ? (0x80000000u | (uint32_t)err) : n;
        ssum += 5ull + (err ? 0 : n);
      }
    }
    s_scan_d[tid] = dsum;
    s_scan_min[tid] = dmin;
    s_scan_w[tid] = wsum;
    s_scan_s[tid] = ssum;
    __syncthreads();
    if (tid == 0) {  // small serial scan over the per-thread sums
      int32_t dacc = 0, mn = 0;
      uint32_t wacc = 0;
      uint64_t sacc = 0;
      for (int i = 0; i < kS2Threads; i++) {
        int32_t dv = s_scan_d[i], mv = s_scan_min[i];
        uint32_t wv = s_scan_w[i];
        uint64_t sv = s_scan_s[i];
        mn = min(mn, dacc + mv);
        s_scan_d[i] = dacc;
        s_scan_min[i] = mn;  // min depth over the tile up to the end of thread i's range
        s_scan_w[i] = wacc;
        s_scan_s[i] = sacc;
        dacc += dv;
        wacc += wv;
        sacc += sv;
      }
      s_d_delta = dacc;
      s_min_rel = mn;
      s_words = wacc;
      s_strbytes = sacc;
    }
    __syncthreads();
    const int32_t d0 = s_scan_d[tid];
    const uint32_t w0 = s_scan_w[tid];
    const int32_t pmin0 = tid > 0 ? s_scan_min[tid - 1] : 0;  // min depth before my range
    {
      int32_t r = d0;
      uint32_t wr = w0;
      for (uint32_t j = a; j < b; j++) {
        const uint8_t k = s_kind[j];
        r += depth_delta(k);
        s_D[j] = (int16_t)r;
        s_tape[j] = (uint16_t)wr;
        wr += tape_words_of(k);
      }
    }
    __syncthreads();
    for (uint32_t c = tid; c * 32 < cnt; c += kS2Threads) {
      int32_t mn = 0x7FFF;
      for (uint32_t j = c * 32; j < min(cnt, c * 32 + 32); j++) mn = min(mn, (int32_t)s_D[j]);
      s_chunkmin[c] = (int16_t)mn;
    }
    __syncthreads();

    // ---- C. parent of every token inside the tile ---------------------------
    {
      int32_t pmin = pmin0;
      for (uint32_t j = a; j < b; j++) {
        const int32_t E = j ? s_D[j - 1] : 0;  // depth before the token
        const int32_t x = E - 1;
        int32_t par = -1;
        if (x >= pmin) {
          int32_t m = (int32_t)j - 1;
          while (m >= 0) {
            if ((m & 31) == 31 && s_chunkmin[m >> 5] > x) { m -= 32; continue; }
            if (s_D[m] <= x) break;
            m--;
          }
          par = m + 1;  // m == -1: the tile start (depth 0) precedes the parent
        }
        s_par[j] = (int16_t)par;
        if (par >= 0 && is_close(s_kind[j])) atomicOr(&s_closed[par >> 5], 1u << (par & 31));
        pmin = min(pmin, (int32_t)s_D[j]);
      }
    }
    __syncthreads();

    // ---- D. publish the aggregate: sizes + containers left open ---------------
    const int32_t min_rel = s_min_rel;
    for (uint32_t j = tid; j < cnt; j += kS2Threads) {
      const uint8_t k = s_kind[j];
      if (is_open(k) && !((s_closed[j >> 5] >> (j & 31)) & 1u)) {
        const int32_t slot = s_D[j] - min_rel - 1;
        survp[off + slot] = (k == K_OPEN_OBJ ? 0x80000000u : 0u) | s_tape[j];
      }
    }
    __syncthreads();
    if (tid == 0) {
      S2Tile &me = J.s2[t];
      me.d_delta = s_d_delta;
      me.min_rel = min_rel;
      me.words = s_words;
      me.strbytes = s_strbytes;
      __threadfence();
      st_release(&J.s2_flag[t], kStAgg);
    }

    // ---- E. look-back (one thread) -------------------------------------------
    if (tid == 0) {
      int nchain = 0;
      int64_t k = (int64_t)t - 1;
      int32_t dcur = 0;
      uint32_t tcur = 1;  // tape index 0 is the root word
      uint64_t scur = 0;
      int64_t ptile = -1;  // nearest predecessor with an inclusive prefix
      while (k >= (int64_t)j_min) {
        uint32_t f = spin_flag(&J.s2_flag[k], kStAgg, &J.doc_flags[d]);
        if (f >= kStIncl || f == 0) {
          if (f == 0) break;  // gave up (INTERNAL flagged)
          const S2Tile &pk = J.s2[k];
          dcur = pk.d_start + pk.d_delta;
          tcur = pk.tape_start + pk.words;
          scur = pk.str_start + pk.strbytes;
          ptile = k;
          break;
        }
        if (nchain == kChain) {  // wait for this one to finish instead
          f = spin_flag(&J.s2_flag[k], kStIncl, &J.doc_flags[d]);
          continue;
        }
        s_chain[nchain].tile = (uint32_t)k;
        nchain++;
        k--;
      }
      // chain entries from the farthest to the nearest
      for (int i = nchain - 1; i >= 0; i--) {
        const S2Tile &pc = J.s2[s_chain[i].tile];
        s_chain[i].low = dcur + pc.min_rel;
        s_chain[i].tape_start = tcur;
        dcur += pc.d_delta;
        tcur += pc.words;
        scur += pc.strbytes;
        s_chain[i].d_end = dcur;
      }
      const int32_t d_start = dcur;
      const int32_t low = d_start + min_rel;
      // nearest earlier tile with a lower `low`
      uint32_t jump = kNoTile;
      for (int i = 0; i < nchain && jump == kNoTile; i++)
        if (s_chain[i].low < low) jump = s_chain[i].tile;
      if (jump == kNoTile) {
        int64_t c = ptile;
        while (c >= 0) {
          if (spin_flag(&J.s2_flag[c], kStIncl, &J.doc_flags[d]) == 0) break;
          const S2Tile &pc = J.s2[c];
          if (pc.d_start + pc.min_rel < low) { jump = (uint32_t)c; break; }
          c = pc.jump == kNoTile ? -1 : (int64_t)pc.jump;
        }
      }
      S2Tile &me = J.s2[t];
      me.d_start = d_start;
      me.jump = jump;
      me.tape_start = tcur;
      me.str_start = scur;
      __threadfence();
      st_release(&J.s2_flag[t], kStIncl);
      s_d_start = d_start;
      s_tape_start = tcur;
      s_str_start = scur;

      // incoming frontier: owners of levels [max(1, low), d_start], deepest first
      const int32_t lo = max(1, low);
      s_front_lo = lo;
      int ci = 0;         // position in the chain (nearest first)
      int64_t c = -1;     // current tile beyond the chain
      bool beyond = false;
      for (int32_t lev = d_start; lev >= lo; lev--) {
        uint32_t ent_tape = 0;
        uint8_t ent_kind = K_OTHER;
        for (;;) {
          int32_t clow;
          uint32_t ctile, ctape;
          if (!beyond) {
            if (ci < nchain) {
              clow = s_chain[ci].low; ctile = s_chain[ci].tile; ctape = s_chain[ci].tape_start;
            } else {
              beyond = true;
              c = ptile;
              continue;
            }
          } else {
            if (c < 0) break;
            if (spin_flag(&J.s2_flag[c], kStIncl, &J.doc_flags[d]) == 0) { c = -1; break; }
            const S2Tile &pc = J.s2[c];
            clow = pc.d_start + pc.min_rel;
            ctile = (uint32_t)c;
            ctape = pc.tape_start;
          }
          if (clow < lev) {
            const uint32_t tc_off = J.tile_off[ctile];
            const uint32_t e = survp[tc_off + (uint32_t)(lev - clow - 1)];
            ent_kind = (e >> 31) ? K_OPEN_OBJ : K_OPEN_ARR;
            ent_tape = ctape + (e & 0xFFFFu);
            break;
          }
          if (!beyond) ci++;
          else {
            const S2Tile &pc = J.s2[c];
            c = pc.jump == kNoTile ? -1 : (int64_t)pc.jump;
          }
        }
        if (lev - lo <= kMaxTileTokens) {
          s_front_tape[lev - lo] = ent_tape;
          s_front_kind[lev - lo] = ent_kind;
        }
      }
      // the document's last tile closes the tape
      if (tt == ntiles_d - 1) {
        const int32_t d_end = d_start + s_d_delta;
        const uint32_t T = tcur + s_words + 1;
        if (d_end != 0) report(J, d, nidx, SJ_TAPE_ERROR);
        if ((uint64_t)T <= tape_cap) {
          tape[0] = ((uint64_t)'r' << 56) | (uint64_t)(T - 1);
          tape[T - 1] = ((uint64_t)'r' << 56);
        }
        J.doc_tape[d] = T;
        J.doc_str[d] = scur + s_strbytes;
      }
    }
    __syncthreads();

    // ---- F. grammar, tape words, strings, numbers, atoms ----------------------
    {
      const int32_t d_start = s_d_start;
      const uint32_t tape_start = s_tape_start;
      const int32_t front_lo = s_front_lo;
      uint64_t so = s_str_start + s_scan_s[tid];
      const uint32_t max_depth = J.max_depth;
      for (uint32_t j = a; j < b; j++) {
        const uint64_t g = (uint64_t)off + j;
        const uint8_t k = s_kind[j];
        const int32_t E = d_start + (j ? s_D[j - 1] : 0);
        const uint8_t p = j >= 1 ? s_kind[j - 1] : kind_at(J, idxp, doc, (int64_t)g - 1);
        const uint8_t pp = j >= 2 ? s_kind[j - 2] : kind_at(J, idxp, doc, (int64_t)g - 2);
        // parent: in the tile, or the frontier entry of level E
        uint8_t K = 0;            // kind of the enclosing container (K_OPEN_OBJ / K_OPEN_ARR)
        uint64_t par_tape = ~0ull;
        bool par_ok = true;
        if (E >= 1) {
          const int32_t pl = s_par[j];
          if (pl >= 0) {
            K = s_kind[pl];
            par_tape = tape_start + s_tape[pl];
          } else if (E >= front_lo && E <= d_start && E - front_lo <= kMaxTileTokens &&
                     s_front_kind[E - front_lo] != K_OTHER) {
            K = s_front_kind[E - front_lo];
            par_tape = s_front_tape[E - front_lo];
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

        const uint64_t tp = (uint64_t)tape_start + s_tape[j];
        const uint32_t pos = s_pos[j];
        if (!code) {
          switch (k) {
            case K_CLOSE_OBJ:
            case K_CLOSE_ARR: {
              const uint64_t ot = par_tape;
              if (tp < tape_cap && ot < tape_cap) {
                tape[tp] = ((uint64_t)(k == K_CLOSE_OBJ ? '}' : ']') << 56) | ot;
                tape[ot] = ((uint64_t)(k == K_CLOSE_OBJ ? '{' : '[') << 56) | (tp + 1);
              }
              break;
            }
            case K_STRING: {
              const uint32_t sl = s_slen[j];
              if (sl & 0x80000000u) { code = (int)(sl & 0xFF); break; }
              if (tp < tape_cap && so + 5 + sl <= str_cap) {
                tape[tp] = ((uint64_t)'"' << 56) | so;
                uint8_t *o = strs + so;
                o[0] = (uint8_t)sl; o[1] = (uint8_t)(sl >> 8); o[2] = (uint8_t)(sl >> 16); o[3] = (uint8_t)(sl >> 24);
                int err;
                string_walk<true>(doc + pos + 1, doc + s_pos[j + 1], err, o + 4);
                o[4 + sl] = 0;
              }
              break;
            }
            case K_NUMBER: {
              uint8_t tag;
              uint64_t v;
              code = parse_number(doc + pos, doc + len, tag, v);
              if (!code && tp + 1 < tape_cap) {
                tape[tp] = (uint64_t)tag << 56;
                tape[tp + 1] = v;
              }
              break;
            }
            case K_TRUE:
            case K_FALSE:
            case K_NULL: {
              const char *word = k == K_TRUE ? "true" : (k == K_FALSE ? "false" : "null");
              const uint32_t n = k == K_FALSE ? 5 : 4;
              bool ok = pos + n <= len;
              for (uint32_t i = 0; ok && i < n; i++) ok = doc[pos + i] == (uint8_t)word[i];
              if (ok && pos + n < len) ok = is_terminator(doc[pos + n]);
              if (!ok) code = k == K_TRUE ? SJ_T_ATOM_ERROR : (k == K_FALSE ? SJ_F_ATOM_ERROR : SJ_N_ATOM_ERROR);
              else if (tp < tape_cap) tape[tp] = (uint64_t)word[0] << 56;
              break;
            }
            default: break;
          }
        }
        if (code) report(J, d, g, code);
        if (k == K_STRING) {
          const uint32_t sl = s_slen[j];
          so += 5ull + ((sl & 0x80000000u) ? 0 : sl);
        }
      }
    }
    __syncthreads();
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
      uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      uint32_t v = s_warp[lane];
      uint32_t vi = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xFFFFFFFFu, vi, o);
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

// ---------------------------------------------------------------------------
// Finalise: per-document results, then clear the look-back state for the next
// run (the status words must start at zero).
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(const Job *__restrict__ job) {
  const Job &J = *job;
  const uint32_t n_tiles = J.counters[2];
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t d = blockIdx.x * blockDim.x + threadIdx.x; d < J.n_docs; d += stride) {
    const uint32_t f = J.doc_flags[d];
    const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
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
    (void)len;
  }
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += stride) {
    J.s1_state[t] = 0;
    J.s1_count[t] = 0;
    J.s2_flag[t] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    J.counters[0] = 0;
    J.counters[1] = 0;
  }
}

}  // namespace sj
