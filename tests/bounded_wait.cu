// Test harness (compiled by tests/test_zy_bounded_wait.py with a small
// SJ_SPIN_LIMIT, linked with the library's stage1.cu): runs the single-pass
// stage-1 kernel on a two-tile document whose first tile no warp ever takes
// (the ticket counter starts at 1), so the second tile's look-back waits on a
// status word that nothing publishes.  The wait must give up, mark the
// document INTERNAL and let the kernel finish.
#include <cuda_runtime.h>
#include <string.h>

#include "sj_internal.cuh"

namespace sj {
__global__ void stage1_kernel(const Job *job);
}

extern "C" int bw_run(uint32_t *flags_out) {
  const uint64_t len = 2 * sj::kTileBytes;
  uint8_t *doc = nullptr;
  uint64_t *doc_off = nullptr, *s1_count = nullptr;
  uint32_t *u32 = nullptr, *idx = nullptr;
  sj::Job *d_job = nullptr;
  if (cudaMalloc(&doc, len) || cudaMalloc(&doc_off, 2 * sizeof(uint64_t)) ||
      cudaMalloc(&s1_count, 2 * sizeof(uint64_t)) || cudaMalloc(&u32, 64 * sizeof(uint32_t)) ||
      cudaMalloc(&idx, len * sizeof(uint32_t)) || cudaMalloc(&d_job, sizeof(sj::Job)))
    return -1;
  cudaMemset(doc, ' ', len);
  const uint64_t off[2] = {0, len};
  cudaMemcpy(doc_off, off, sizeof(off), cudaMemcpyHostToDevice);
  cudaMemset(s1_count, 0, 2 * sizeof(uint64_t));
  cudaMemset(u32, 0, 64 * sizeof(uint32_t));
  // u32: [0..3] counters, [8..9] tile_first, [16..17] s1_state, [24..25] tile_cnt,
  // [32..33] tile_off, [40] doc_flags, [41] doc_nidx
  const uint32_t counters[4] = {1, 0, 2, 0};  // ticket from 1: tile 0 is never taken
  const uint32_t tile_first[2] = {0, 2};
  cudaMemcpy(u32, counters, sizeof(counters), cudaMemcpyHostToDevice);
  cudaMemcpy(u32 + 8, tile_first, sizeof(tile_first), cudaMemcpyHostToDevice);
  sj::Job J;
  memset(&J, 0, sizeof(J));
  J.base = doc;
  J.doc_off = doc_off;
  J.n_docs = 1;
  J.max_depth = sj::kMaxDepthLimit;
  J.max_doc_len = len;
  J.tile_first = u32 + 8;
  J.counters = u32;
  J.s1_state = u32 + 16;
  J.s1_count = s1_count;
  J.tile_cnt = u32 + 24;
  J.tile_off = u32 + 32;
  J.idx = idx;
  J.doc_flags = u32 + 40;
  J.doc_nidx = u32 + 41;
  cudaMemcpy(d_job, &J, sizeof(J), cudaMemcpyHostToDevice);
  sj::stage1_kernel<<<1, 32 * sj::kS1Warps>>>(d_job);
  cudaError_t e = cudaDeviceSynchronize();
  uint32_t flags = 0xFFFFFFFFu;
  if (e == cudaSuccess) e = cudaMemcpy(&flags, u32 + 40, sizeof(flags), cudaMemcpyDeviceToHost);
  cudaFree(doc); cudaFree(doc_off); cudaFree(s1_count); cudaFree(u32); cudaFree(idx); cudaFree(d_job);
  if (e != cudaSuccess) return (int)e;
  *flags_out = flags;
  return 0;
}
