// setup.cu -- the first and last kernels of a run: tiles per document, and
// the per-document results with the error precedence.
#include "sj_internal.cuh"

namespace sj {

// Tiles per document (one block scan over the documents); resets the
// per-document state and the tile tickets.
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
    uint32_t incl = warp_incl_u32(nt, lane);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const uint32_t v = s_warp[lane];
      s_warp[lane] = warp_incl_u32(v, lane) - v;  // exclusive
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
    J.counters[kCtrTiles] = s_carry;
    J.counters[kCtrTicket1] = 0;
    J.counters[kCtrTicketBuild] = 0;
    J.counters[kCtrTicketNum] = 0;
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
