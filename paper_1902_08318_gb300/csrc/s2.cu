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

// Exclusive scan over the threads of the block of (depth sum, tape words) and
// the running minimum of the depth, in token order (each thread owns a
// contiguous run of tokens).  Returns the block totals through the pointers.
struct DW {
  int32_t d, mn;
  uint32_t w, n;  // n: a count (strings) scanned alongside
};
__device__ __forceinline__ DW dw_combine(const DW &a, const DW &b) {
  return DW{a.d + b.d, min(a.mn, a.d + b.mn), a.w + b.w, a.n + b.n};
}
__device__ DW block_exclusive_dw(DW v, DW *s_warp, DW &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  DW x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    DW u;
    u.d = __shfl_up_sync(0xFFFFFFFFu, x.d, o);
    u.mn = __shfl_up_sync(0xFFFFFFFFu, x.mn, o);
    u.w = __shfl_up_sync(0xFFFFFFFFu, x.w, o);
    u.n = __shfl_up_sync(0xFFFFFFFFu, x.n, o);
    if (lane >= o) x = dw_combine(u, x);
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  DW pre{0, 0, 0, 0};
  for (int i = 0; i < wid; i++) pre = dw_combine(pre, s_warp[i]);
  total = DW{0, 0, 0, 0};
  for (int i = 0; i < kS2Threads / 32; i++) total = dw_combine(total, s_warp[i]);
  DW xe;  // exclusive within the warp
  xe.d = __shfl_up_sync(0xFFFFFFFFu, x.d, 1);
  xe.mn = __shfl_up_sync(0xFFFFFFFFu, x.mn, 1);
  xe.w = __shfl_up_sync(0xFFFFFFFFu, x.w, 1);
  xe.n = __shfl_up_sync(0xFFFFFFFFu, x.n, 1);
  if (lane == 0) xe = DW{0, 0, 0, 0};
  __syncthreads();
  return dw_combine(pre, xe);
}

// Shared per-tile state of both stage-2 kernels.
struct TileSmem {
  uint32_t pos[kMaxTileTokens + 1];  // token positions (+ the next token's)
  int16_t D[kMaxTileTokens];         // depth after the token, relative to the tile start
  uint16_t tape[kMaxTileTokens];     // tape slot relative to the tile
  uint8_t kind[kMaxTileTokens];
  uint16_t list[kMaxTileTokens];     // strings, then numbers (token indices)
  uint32_t closed[kMaxTileTokens / 32];
  int16_t chunkmin[kMaxTileTokens / 32];
  DW warp[kS2Threads / 32];
  uint32_t n_str, n_num;
  unsigned long long strbytes;
};

// Loads the tile's token positions and kinds and lists its strings (in token
// order) and numbers.  Then the blocked depth / tape-word scan.
__device__ void tile_tokens(const Job &J, TileSmem &S, const uint32_t *idxp, const uint8_t *doc,
                            uint64_t len, uint32_t off, uint32_t cnt, uint32_t nidx, DW &tot,
                            uint32_t &a, uint32_t &b, DW &ex) {
  const int tid = threadIdx.x;
  for (uint32_t j = tid; j < cnt; j += kS2Threads) {
    const uint32_t p = idxp[off + j];
    S.pos[j] = p;
    S.kind[j] = token_kind(doc[p]);
  }
  if (tid == 0) {
    S.pos[cnt] = (off + cnt < nidx) ? idxp[off + cnt] : (uint32_t)len;
    S.n_num = 0;
    S.strbytes = 0;
  }
  for (uint32_t j = tid; j < kMaxTileTokens / 32; j += kS2Threads) S.closed[j] = 0;
  __syncthreads();
  const uint32_t per = (cnt + kS2Threads - 1) / kS2Threads;
  a = min(cnt, tid * per);
  b = min(cnt, a + per);
  DW v{0, 0, 0, 0};
  for (uint32_t j = a; j < b; j++) {
    const uint8_t k = S.kind[j];
    v.d += depth_delta(k);
    v.mn = min(v.mn, v.d);
    v.w += tape_words_of(k);
    v.n += k == K_STRING;
  }
  ex = block_exclusive_dw(v, S.warp, tot);
  {
    int32_t r = ex.d;
    uint32_t wr = ex.w, sn = ex.n;
    for (uint32_t j = a; j < b; j++) {
      const uint8_t k = S.kind[j];
      r += depth_delta(k);
      S.D[j] = (int16_t)r;
      S.tape[j] = (uint16_t)wr;
      wr += tape_words_of(k);
      if (k == K_STRING) S.list[sn++] = (uint16_t)j;
    }
  }
  if (tid == 0) S.n_str = tot.n;
  __syncthreads();
  for (uint32_t c = tid; c * 32 < cnt; c += kS2Threads) {
    int32_t mn = 0x7FFF;
    const uint32_t e = min(cnt, c * 32 + 32);
    for (uint32_t j = c * 32; j < e; j++) mn = min(mn, (int32_t)S.D[j]);
    S.chunkmin[c] = (int16_t)mn;
  }
  __syncthreads();
}

// Parent of token j inside the tile: the token after the last one whose depth
// is at most (depth before j) - 1, or -1 if that lies before the tile.
__device__ __forceinline__ int32_t tile_parent(const TileSmem &S, uint32_t j, int32_t pmin_before) {
  const int32_t E = j ? S.D[j - 1] : 0;
  const int32_t x = E - 1;
  if (x < pmin_before) return -1;
  int32_t m = (int32_t)j - 1;
  while (m >= 0) {
    if ((m & 31) == 31 && S.chunkmin[m >> 5] > x) { m -= 32; continue; }
    if (S.D[m] <= x) break;
    m--;
  }
  return m + 1;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kS2Threads) stage2_reduce_kernel(const Job *__restrict__ job) {
  const Job &J = *job;
  __shared__ TileSmem S;
  const int tid = threadIdx.x;
  const uint32_t n_tiles = J.counters[2];
  for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const uint32_t d = doc_of_tile(J, t);
    const uint32_t tt = t - J.tile_first[d];
    const uint32_t nidx = J.doc_nidx[d];
    if ((J.doc_flags[d] & kDocBad) || nidx == 0) {
      if (tid == 0) J.s2_rec[t] = S2Agg{0, 0, 0, tt == 0, 0};
      continue;
    }
    const uint64_t len = J.doc_off[d + 1] - J.doc_off[d];
    const uint8_t *doc = J.base + J.doc_off[d];
    const uint64_t ib = idx_base(J, d);
    const uint32_t *idxp = J.idx + ib;
    const uint32_t cnt = J.tile_cnt[t], off = J.tile_off[t];
    DW tot, ex;
    uint32_t a, b;
    tile_tokens(J, S, idxp, doc, len, off, cnt, nidx, tot, a, b, ex);

    // normalised string lengths (Sec. 3.2.2), one string per thread at a time
    unsigned long long sb = 0;
    for (uint32_t i = tid; i < S.n_str; i += kS2Threads) {
      const uint32_t j = S.list[i];
      int err;
      const uint32_t n = string_walk<false>(doc + S.pos[j] + 1, doc + S.pos[j + 1], err, nullptr);
      J.slen[ib + off + j] = err ? (0x80000000u | (uint32_t)err) : n;
      sb += 5ull + (err ? 0 : n);
    }
    if (sb) atomicAdd(&S.strbytes, sb);

    // containers closed inside the tile; the others are left open (survivors)
    {
      int32_t pmin = min(0, ex.mn);
      for (uint32_t j = a; j < b; j++) {
        if (is_close(S.kind[j])) {
          const int32_t par = tile_parent(S, j, pmin);
          if (par >= 0) atomicOr(&S.closed[par >> 5], 1u << (par & 31));
        }
        pmin = min(pmin, (int32_t)S.D[j]);
      }
    }
    __syncthreads();
    const int32_t min_rel = min(0, tot.mn);
    for (uint32_t j = tid; j < cnt; j += kS2Threads) {
      const uint8_t k = S.kind[j];
      if (is_open(k) && !((S.closed[j >> 5] >> (j & 31)) & 1u)) {
        const int32_t slot = S.D[j] - min_rel - 1;
        J.surv[ib + off + slot] = (k == K_OPEN_OBJ ? 0x80000000u : 0u) | S.tape[j];
      }
    }
    if (tid == 0) J.s2_rec[t] = S2Agg{tot.d, min_rel, tot.w, tt == 0, S.strbytes};
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kS2Threads) stage2_build_kernel(const Job *__restrict__ job) {
  const Job &J = *job;
  __shared__ TileSmem S;
  __shared__ uint64_t s_soff[kMaxTileTokens / 2];  // string-buffer offset of each string (list order)
  const int tid = threadIdx.x;
  const uint32_t n_tiles = J.counters[2];
  const uint32_t max_depth = J.max_depth;
  for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
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

    if (tt == ntiles_d - 1 && tid == 0) {  // the document's last tile closes the tape
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

    DW tot, ex;
    uint32_t a, b;
    tile_tokens(J, S, idxp, doc, len, off, cnt, nidx, tot, a, b, ex);

    // string-buffer offsets of the tile's strings (token order)
    if (tid < 32) {
      uint64_t run = pre.str_start;
      for (uint32_t base = 0; base < S.n_str; base += 32) {
        const uint32_t i = base + tid;
        uint64_t v = 0;
        if (i < S.n_str) {
          const uint32_t sl = J.slen[ib + off + S.list[i]];
          v = 5ull + ((sl & 0x80000000u) ? 0 : sl);
        }
        uint64_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint64_t u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
          if (tid >= o) incl += u;
        }
        if (i < S.n_str) s_soff[i] = run + incl - v;
        run += __shfl_sync(0xFFFFFFFFu, incl, 31);
      }
    }
    __syncthreads();

    // grammar and structure words, one token per thread at a time
    {
      int32_t pmin = min(0, ex.mn);
      for (uint32_t j = a; j < b; j++) {
        const uint64_t g = (uint64_t)off + j;
        const uint8_t k = S.kind[j];
        const int32_t Erel = j ? S.D[j - 1] : 0;
        const int32_t E = pre.d_start + Erel;
        const uint8_t p = j >= 1 ? S.kind[j - 1] : (g >= 1 ? token_kind(doc[idxp[g - 1]]) : K_OTHER);
        const uint8_t pp = j >= 2 ? S.kind[j - 2] : (g >= 2 ? token_kind(doc[idxp[g - 2]]) : K_OTHER);
        uint8_t K = 0;
        uint64_t par_tape = ~0ull;
        bool par_ok = true;
        if (E >= 1) {
          const int32_t pl = tile_parent(S, j, pmin);
          if (pl >= 0) {
            K = S.kind[pl];
            par_tape = (uint64_t)pre.tape_start + S.tape[pl];
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
        pmin = min(pmin, (int32_t)S.D[j]);
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
        const uint64_t tp = (uint64_t)pre.tape_start + S.tape[j];
        const uint32_t pos = S.pos[j];
        if (!code) {
          if (is_close(k)) {
            const uint64_t ot = par_tape;
            if (tp < tape_cap && ot < tape_cap) {
              tape[tp] = ((uint64_t)(k == K_CLOSE_OBJ ? '}' : ']') << 56) | ot;
              tape[ot] = ((uint64_t)(k == K_CLOSE_OBJ ? '{' : '[') << 56) | (tp + 1);
            }
          } else if (is_atom(k)) {
            const char *word = k == K_TRUE ? "true" : (k == K_FALSE ? "false" : "null");
            const uint32_t n = k == K_FALSE ? 5 : 4;
            bool ok = pos + n <= len;
            for (uint32_t i = 0; ok && i < n; i++) ok = doc[pos + i] == (uint8_t)word[i];
            if (ok && pos + n < len) ok = is_terminator(doc[pos + n]);
            if (!ok) code = k == K_TRUE ? SJ_T_ATOM_ERROR : (k == K_FALSE ? SJ_F_ATOM_ERROR : SJ_N_ATOM_ERROR);
            else if (tp < tape_cap) tape[tp] = (uint64_t)word[0] << 56;
          } else if (k == K_NUMBER) {
            const uint32_t i = atomicAdd(&S.n_num, 1u);
            S.list[kMaxTileTokens - 1 - i] = (uint16_t)j;  // numbers fill the list from the end
          } else if (k == K_STRING) {
            const uint32_t sl = J.slen[ib + off + j];
            if (sl & 0x80000000u) code = (int)(sl & 0xFF);
          }
        }
        if (code) report(J, d, g, code);
      }
    }
    __syncthreads();

    // numbers (Sec. 3.2.1), one per thread at a time
    for (uint32_t i = tid; i < S.n_num; i += kS2Threads) {
      const uint32_t j = S.list[kMaxTileTokens - 1 - i];
      const uint64_t tp = (uint64_t)pre.tape_start + S.tape[j];
      uint8_t tag;
      uint64_t v;
      const int code = parse_number(doc + S.pos[j], doc + len, tag, v);
      if (code) report(J, d, (uint64_t)off + j, code);
      else if (tp + 1 < tape_cap) {
        tape[tp] = (uint64_t)tag << 56;
        tape[tp + 1] = v;
      }
    }
    // strings (Sec. 3.2.2): the '"' word and the (length, bytes, NUL) record
    for (uint32_t i = tid; i < S.n_str; i += kS2Threads) {
      const uint32_t j = S.list[i];
      const uint32_t sl = J.slen[ib + off + j];
      if (sl & 0x80000000u) continue;
      const uint64_t tp = (uint64_t)pre.tape_start + S.tape[j];
      const uint64_t so = s_soff[i];
      if (tp < tape_cap && so + 5 + sl <= str_cap) {
        tape[tp] = ((uint64_t)'"' << 56) | so;
        uint8_t *o = strs + so;
        o[0] = (uint8_t)sl; o[1] = (uint8_t)(sl >> 8); o[2] = (uint8_t)(sl >> 16); o[3] = (uint8_t)(sl >> 24);
        int err;
        string_walk<true>(doc + S.pos[j] + 1, doc + S.pos[j + 1], err, o + 4);
        o[4 + sl] = 0;
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
