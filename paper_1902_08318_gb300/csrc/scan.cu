// scan.cu -- the carries between tiles, as segmented scans over per-tile
// aggregates (reduce, scan of block totals, down-sweep), plus the structures
// that let a stage-2 tile find the containers left open by earlier tiles.
//
// Stage 1 carries the in-string bit and the index offset (Sec. 3.1); stage 2
// carries nesting depth, tape slot and string-buffer offset (Sec. 3.2).
// Segments restart at every document.
#include "sj_internal.cuh"

namespace sj {

// ---- monoids over tile aggregates -------------------------------------------
struct M1 {
  using T = S1Agg;
  __device__ static T identity() { return T{0, 0, 0, 0}; }
  // a before b
  __device__ static T combine(const T &a, const T &b) {
    if (b.head) return b;
    T r;
    r.qpar = a.qpar ^ b.qpar;
    r.c0 = a.c0 + (a.qpar ? b.c1 : b.c0);
    r.c1 = a.c1 + (a.qpar ? b.c0 : b.c1);
    r.head = a.head;
    return r;
  }
  __device__ static T shfl_up(const T &v, int o) {
    T r;
    r.qpar = __shfl_up_sync(0xFFFFFFFFu, v.qpar, o);
    r.c0 = __shfl_up_sync(0xFFFFFFFFu, v.c0, o);
    r.c1 = __shfl_up_sync(0xFFFFFFFFu, v.c1, o);
    r.head = __shfl_up_sync(0xFFFFFFFFu, v.head, o);
    return r;
  }
  __device__ static T load(const Job &J, uint32_t t) { return J.s1_rec[t]; }
  __device__ static T *agg(const Job &J) { return reinterpret_cast<T *>(J.scan_agg1); }
  __device__ static T *pre(const Job &J) { return reinterpret_cast<T *>(J.scan_pre1); }
  __device__ static void range(const Job &J, uint32_t &lo, uint32_t &hi) { s1_range(J, lo, hi); }
  // the exclusive prefix of tile t as stored (c1 is never read back)
  __device__ static T stored(const Job &J, uint32_t t) {
    const S1Pre p = J.s1_pre[t];
    return T{p.q_in, p.base, 0, 0};
  }
  __device__ static void store(const Job &J, uint32_t t, const T &excl, const T &) {
    J.s1_pre[t] = S1Pre{excl.c0, excl.qpar};  // documents start outside strings
  }
};

struct M2 {
  using T = S2Agg;
  __device__ static T identity() { return T{0, 0, 0, 0, 0}; }
  __device__ static T combine(const T &a, const T &b) {
    if (b.head) return b;
    T r;
    r.dd = a.dd + b.dd;
    r.mn = min(a.mn, a.dd + b.mn);
    r.w = a.w + b.w;
    r.head = a.head;
    r.s = a.s + b.s;
    return r;
  }
  __device__ static T shfl_up(const T &v, int o) {
    T r;
    r.dd = __shfl_up_sync(0xFFFFFFFFu, v.dd, o);
    r.mn = __shfl_up_sync(0xFFFFFFFFu, v.mn, o);
    r.w = __shfl_up_sync(0xFFFFFFFFu, v.w, o);
    r.head = __shfl_up_sync(0xFFFFFFFFu, v.head, o);
    r.s = __shfl_up_sync(0xFFFFFFFFu, v.s, o);
    return r;
  }
  __device__ static T load(const Job &J, uint32_t t) { return J.s2_rec[t]; }
  __device__ static T *agg(const Job &J) { return reinterpret_cast<T *>(J.scan_agg); }
  __device__ static T *pre(const Job &J) { return reinterpret_cast<T *>(J.scan_pre); }
  __device__ static void range(const Job &J, uint32_t &lo, uint32_t &hi) { s2_range(J, lo, hi); }
  // the exclusive prefix of tile t as stored (mn is never read back)
  __device__ static T stored(const Job &J, uint32_t t) {
    const S2Pre p = J.s2_pre[t];
    return T{p.d_start, 0, p.tape_start - 1u, 0, p.str_start};
  }
  __device__ static void store(const Job &J, uint32_t t, const T &excl, const T &self) {
    S2Pre p;
    p.d_start = excl.dd;
    p.low = excl.dd + self.mn;
    p.tape_start = 1u + excl.w;  // tape word 0 is the root
    p.jump = kNoTile;
    p.str_start = excl.s;
    J.s2_pre[t] = p;
  }
};

// Inclusive scan of one value per thread over a block of kScanBlock threads.
template <class M>
__device__ typename M::T block_inclusive(typename M::T v, typename M::T *s_warp,
                                         typename M::T &total) {
  using T = typename M::T;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = M::shfl_up(v, o);
    if (lane >= o) v = M::combine(u, v);
  }
  if (lane == 31) s_warp[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T x = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T u = M::shfl_up(x, o);
      if (lane >= o) x = M::combine(u, x);
    }
    s_warp[lane] = x;
  }
  __syncthreads();
  if (wid > 0) v = M::combine(s_warp[wid - 1], v);
  total = s_warp[31];
  __syncthreads();
  return v;
}

// Scan block b covers tiles [lo + b * kScanBlock, lo + (b + 1) * kScanBlock)
// of the launch's range; thread blocks loop over scan blocks, so a grid of a
// few blocks per SM serves a whole document or one chunk of it alike.
template <class M>
__global__ void __launch_bounds__(kScanBlock) scan_up_kernel(const Job *__restrict__ job) {
  pdl_enter();
  using T = typename M::T;
  const Job &J = *job;
  __shared__ T s_warp[32];
  uint32_t lo, n;
  M::range(J, lo, n);
  for (uint32_t b = blockIdx.x; lo + b * kScanBlock < n; b += gridDim.x) {
    const uint32_t t = lo + b * kScanBlock + threadIdx.x;
    T v = t < n ? M::load(J, t) : M::identity();
    T total;
    block_inclusive<M>(v, s_warp, total);
    if (threadIdx.x == 0) M::agg(J)[b] = total;
  }
}

template <class M>
__global__ void __launch_bounds__(kScanBlock) scan_top_kernel(const Job *__restrict__ job) {
  pdl_enter();
  using T = typename M::T;
  const Job &J = *job;
  __shared__ T s_warp[32];
  __shared__ T s_incl[kScanBlock];
  __shared__ T s_carry;
  uint32_t lo, hi;
  M::range(J, lo, hi);
  const uint32_t nb = (hi - lo + kScanBlock - 1) / kScanBlock;
  // tiles before the range (earlier chunks of the document) are done: their
  // inclusive prefix is the carry into the range
  if (threadIdx.x == 0)
    s_carry = lo == 0 ? M::identity() : M::combine(M::stored(J, lo - 1), M::load(J, lo - 1));
  __syncthreads();
  for (uint32_t base = 0; base < nb; base += kScanBlock) {
    const uint32_t b = base + threadIdx.x;
    const T v = b < nb ? M::agg(J)[b] : M::identity();
    T total;
    const T incl = block_inclusive<M>(v, s_warp, total);
    s_incl[threadIdx.x] = incl;
    __syncthreads();
    // exclusive prefix of block b: carry . (inclusive of b-1 within this chunk)
    const T carry = s_carry;
    const T excl = threadIdx.x ? M::combine(carry, s_incl[threadIdx.x - 1]) : carry;
    if (b < nb) M::pre(J)[b] = excl;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = M::combine(carry, total);
    __syncthreads();
  }
}

template <class M>
__global__ void __launch_bounds__(kScanBlock) scan_down_kernel(const Job *__restrict__ job) {
  pdl_enter();
  using T = typename M::T;
  const Job &J = *job;
  __shared__ T s_warp[32];
  __shared__ T s_incl[kScanBlock];
  uint32_t lo, n;
  M::range(J, lo, n);
  for (uint32_t b = blockIdx.x; lo + b * kScanBlock < n; b += gridDim.x) {
    const uint32_t t = lo + b * kScanBlock + threadIdx.x;
    const T self = t < n ? M::load(J, t) : M::identity();
    T total;
    const T incl = block_inclusive<M>(self, s_warp, total);
    s_incl[threadIdx.x] = incl;
    __syncthreads();
    if (t < n) {
      T excl;
      if (self.head) {
        excl = M::identity();
      } else {
        const T pre = M::pre(J)[b];
        excl = threadIdx.x ? M::combine(pre, s_incl[threadIdx.x - 1]) : pre;
      }
      M::store(J, t, excl, self);
    }
    __syncthreads();  // s_incl is reused by the next scan block
  }
}

// The whole scan in one thread block, for parsers of at most kSmallTiles
// tiles (of the stage the scan serves): the block walks the range in steps of
// kScanBlock tiles and carries
// the inclusive prefix from one step to the next (the three launches above
// cost more than they save on a few thousand tiles).  With SPT (stage 2) the
// same block then builds the sparse table of tile minima in shared memory,
// one level from the one before (level k: minimum over the 2^k tiles ending
// at a tile), and the jump pointers from it (no jump_kernel launch).
template <class M, bool SPT>
__global__ void __launch_bounds__(kScanBlock) scan_single_kernel(const Job *__restrict__ job) {
  pdl_enter();
  using T = typename M::T;
  const Job &J = *job;
  __shared__ T s_warp[32];
  __shared__ T s_incl[kScanBlock];
  __shared__ T s_carry;
  uint32_t lo, n;
  M::range(J, lo, n);
  if (threadIdx.x == 0)
    s_carry = lo == 0 ? M::identity() : M::combine(M::stored(J, lo - 1), M::load(J, lo - 1));
  __syncthreads();
  for (uint32_t base = lo; base < n; base += kScanBlock) {
    const uint32_t t = base + threadIdx.x;
    const T self = t < n ? M::load(J, t) : M::identity();
    T total;
    const T incl = block_inclusive<M>(self, s_warp, total);
    s_incl[threadIdx.x] = incl;
    __syncthreads();
    const T carry = s_carry;
    if (t < n) {
      const T excl = self.head ? M::identity()
                               : (threadIdx.x ? M::combine(carry, s_incl[threadIdx.x - 1]) : carry);
      M::store(J, t, excl, self);
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry = M::combine(carry, total);
    __syncthreads();
  }
  if constexpr (SPT) {
    // Whole-document runs only (lo == 0, n <= kSmallTiles).  Every level of
    // the sparse table stays in shared memory (dynamic: spt_levels rows of
    // n), and each tile's jump pointer is found there by binary lifting, as
    // jump_kernel does from the table in global memory.
    extern __shared__ int32_t s_spt[];
    for (uint32_t t = threadIdx.x; t < n; t += kScanBlock) s_spt[t] = J.s2_pre[t].low;
    __syncthreads();
    for (uint32_t k = 1; k < J.spt_levels; k++) {
      const int32_t *in = s_spt + (k - 1) * n;
      int32_t *out = s_spt + k * n;
      const uint32_t step = 1u << (k - 1);
      for (uint32_t t = threadIdx.x; t < n; t += kScanBlock)
        out[t] = t >= step ? min(in[t], in[t - step]) : in[t];
      __syncthreads();
    }
    for (uint32_t t = threadIdx.x; t < n; t += kScanBlock) {
      const int64_t lo_d = s2_first(J, s2_doc(J, t));
      const int32_t x = s_spt[t];
      int64_t c = (int64_t)t - 1;
      for (int k = (int)J.spt_levels - 1; k >= 0 && c >= lo_d; k--) {
        const int64_t w = 1ll << k;
        if (c - w + 1 >= lo_d && s_spt[(uint32_t)k * n + (uint32_t)c] >= x) c -= w;
      }
      J.s2_pre[t].jump = c >= lo_d ? (uint32_t)c : kNoTile;
    }
  }
}

template __global__ void scan_single_kernel<M1, false>(const Job *);
template __global__ void scan_single_kernel<M2, true>(const Job *);

template __global__ void scan_up_kernel<M1>(const Job *);
template __global__ void scan_top_kernel<M1>(const Job *);
template __global__ void scan_down_kernel<M1>(const Job *);
template __global__ void scan_up_kernel<M2>(const Job *);
template __global__ void scan_top_kernel<M2>(const Job *);
template __global__ void scan_down_kernel<M2>(const Job *);

void launch_scan1(const Job *job, uint32_t blocks, cudaStream_t s, bool pdl) {
  launch_k(pdl, scan_up_kernel<M1>, blocks, kScanBlock, 0, s, job);
  launch_k(pdl, scan_top_kernel<M1>, 1, kScanBlock, 0, s, job);
  launch_k(pdl, scan_down_kernel<M1>, blocks, kScanBlock, 0, s, job);
}
void launch_scan2(const Job *job, uint32_t blocks, cudaStream_t s, bool pdl) {
  launch_k(pdl, scan_up_kernel<M2>, blocks, kScanBlock, 0, s, job);
  launch_k(pdl, scan_top_kernel<M2>, 1, kScanBlock, 0, s, job);
  launch_k(pdl, scan_down_kernel<M2>, blocks, kScanBlock, 0, s, job);
}
void launch_scan1_small(const Job *job, cudaStream_t s, bool pdl) {
  launch_k(pdl, scan_single_kernel<M1, false>, 1, kScanBlock, 0, s, job);
}
void launch_scan2_spt_small(const Job *job, size_t spt_smem, cudaStream_t s, bool pdl) {
  launch_k(pdl, scan_single_kernel<M2, true>, 1, kScanBlock, spt_smem, s, job);
}
// The sparse table in shared memory may exceed a launch's default limit.
cudaError_t prepare_scan2_spt_small(size_t spt_smem) {
  return cudaFuncSetAttribute(scan_single_kernel<M2, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spt_smem);
}

// ---- nearest earlier tile with a lower `low` -----------------------------------
// Sparse table of minima: level k holds min(low[t - 2^k + 1 .. t]).  Each
// launch derives four levels from level `src` (sixteen reads per tile).
__global__ void spt_build_kernel(const Job *__restrict__ job, uint32_t src) {
  pdl_enter();
  const Job &J = *job;
  uint32_t lo, n;
  s2_range(J, lo, n);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t t = lo + blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    if (src == 0) J.spt[t] = J.s2_pre[t].low;
    if (src + 1 >= J.spt_levels) continue;
    const int32_t *in = J.spt + (uint64_t)src * J.spt_stride;
    const uint32_t step = 1u << src;
    int32_t mn = src == 0 ? J.s2_pre[t].low : in[t];
#pragma unroll
    for (uint32_t i = 1; i < 16; i++) {
      const int64_t q = (int64_t)t - (int64_t)i * step;
      if (q >= 0) mn = min(mn, src == 0 ? J.s2_pre[q].low : in[q]);
      if ((i & (i + 1)) == 0) {  // i = 1, 3, 7, 15: window of 2, 4, 8, 16 entries
        const uint32_t lev = src + (31 - __clz(i + 1));
        if (lev < J.spt_levels) J.spt[(uint64_t)lev * J.spt_stride + t] = mn;
      }
    }
  }
}

// Largest c in [lo, from] with low(c) < x, or -1 (binary lifting).
__device__ __forceinline__ int64_t last_lower(const Job &J, int64_t from, int64_t lo, int32_t x) {
  int64_t c = from;
  for (int k = (int)J.spt_levels - 1; k >= 0 && c >= lo; k--) {
    const int64_t w = 1ll << k;
    if (c - w + 1 >= lo && J.spt[(uint64_t)k * J.spt_stride + c] >= x) c -= w;
  }
  return c >= lo ? c : -1;
}

__global__ void jump_kernel(const Job *__restrict__ job) {
  pdl_enter();
  const Job &J = *job;
  uint32_t lo, n;
  s2_range(J, lo, n);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t t = lo + blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    const uint32_t d = s2_doc(J, t);
    const int64_t c = last_lower(J, (int64_t)t - 1, s2_first(J, d), J.s2_pre[t].low);
    J.s2_pre[t].jump = c < 0 ? kNoTile : (uint32_t)c;
  }
}

// For every tile, the open container of each level [max(1, low), d_start]
// entering it: (kind << 63) | absolute tape index of its opener, or ~0 when
// there is none (an invalid document).  Level L of tile t is stored at
// front[idx_base + tile_off[t] + t + (d_start - L)]: a tile needs at most one
// more level than it has tokens, and the global tile index keeps documents
// apart.  One warp per tile: the nearest earlier tile whose lowest depth is
// below a level holds that level's container among its survivors, and one
// such tile serves the whole range of levels down to its own lowest depth,
// so the warp walks the chain of those tiles (jump pointers) once and copies
// each range with all lanes.
__global__ void frontier_kernel(const Job *__restrict__ job) {
  pdl_enter();
  const Job &J = *job;
  uint32_t t_lo, t_hi;
  s2_range(J, t_lo, t_hi);
  const int lane = threadIdx.x & 31;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t t = t_lo + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < t_hi; t += nw) {
    const uint32_t d = s2_doc(J, t);
    const uint32_t j_min = s2_first(J, d);
    if (J.doc_flags[d] & (kFlagUtf8 | kFlagUnclosed | kFlagCapacity)) continue;
    const S2Pre me = J.s2_pre[t];
    const int32_t lo = max(1, me.low), hi = me.d_start;
    if (hi < lo) continue;
    const uint64_t ib = idx_base(J, d);
    uint64_t *out = J.front + ib + J.tile_off[t] + t;
    int64_t c = (int64_t)t - 1;
    int32_t clow = c >= (int64_t)j_min ? J.s2_pre[c].low : 0;
    int32_t lev = hi;
    while (lev >= lo) {
      while (c >= (int64_t)j_min && clow >= lev) {
        const uint32_t jp = J.s2_pre[c].jump;
        c = jp == kNoTile ? -1 : (int64_t)jp;
        if (c >= (int64_t)j_min) clow = J.s2_pre[c].low;
      }
      if (c >= (int64_t)j_min) {  // levels (clow, lev] come from tile c's survivors
        const int32_t bottom = max(lo, clow + 1);
        const uint32_t *sv = J.surv + ib + J.tile_off[c];
        const uint64_t ts = J.s2_pre[c].tape_start;
        for (int32_t L = lev - lane; L >= bottom; L -= 32) {
          const uint32_t e = sv[L - clow - 1];
          out[hi - L] = ((uint64_t)(e >> 31) << 63) | (ts + (e & 0xFFFFu));
        }
        lev = bottom - 1;
      } else {  // no container: an invalid document
        for (int32_t L = lev - lane; L >= lo; L -= 32) out[hi - L] = ~0ull;
        lev = lo - 1;
      }
    }
  }
}

}  // namespace sj
