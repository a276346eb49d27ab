// api.cu -- the C ABI of include/sj.h: parser objects, launches, results.
//
// A run is a fixed sequence of kernels on one stream (see enqueue_run):
// setup (tiles per document), stage 1 (blocks, tile scan, flatten), stage 2
// (reduce, tile scan, frontier, build) and finalize (per-document results),
// bracketed by a host-to-device copy of the run descriptor and the document
// offsets and a device-to-host copy of the results.  The sequence is captured
// once per (parser, bucket of document counts) as a CUDA graph and replayed.
//
// One large document in pinned host memory is parsed as it arrives
// (enqueue_chunked): a second stream copies it chunk by chunk while the
// kernels run stage 1 on each chunk that has landed and stage 2 on every tile
// whose tokens are known to end in landed bytes.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "sj_internal.cuh"

namespace sj {
__global__ void setup_kernel(Job *job, const Job *hjob, const uint64_t *hoff, uint32_t n_off);
__global__ void stage1_blocks_kernel(const Job *job);
__global__ void stage1_flatten_kernel(const Job *job);
__global__ void stage2_reduce_kernel(const Job *job);
__global__ void stage2_reduce_sub_kernel(const Job *job);
__global__ void stage2_build_kernel(const Job *job);
__global__ void stage2_build_sub_kernel(const Job *job);
__global__ void stage2_build_small_kernel(const Job *job);
__global__ void numbers_kernel(const Job *job);
__global__ void numbers_split_kernel(const Job *job);
__global__ void finalize_kernel(const Job *job);
__global__ void spt_build_kernel(const Job *job, uint32_t src);
__global__ void jump_kernel(const Job *job);
__global__ void frontier_kernel(const Job *job);
__global__ void chunk_range_kernel(const Job *job, uint32_t lo1, uint32_t hi1, int mode,
                                   uint32_t c, int last);
void launch_scan1(const Job *job, uint32_t blocks, cudaStream_t s, bool pdl);
void launch_scan2(const Job *job, uint32_t blocks, cudaStream_t s, bool pdl);
void launch_scan1_small(const Job *job, cudaStream_t s, bool pdl);
void launch_scan2_spt_small(const Job *job, size_t spt_smem, cudaStream_t s, bool pdl);
cudaError_t prepare_scan2_spt_small(size_t spt_smem);
}  // namespace sj

using sj::Job;

static thread_local int g_last_cuda_error = 0;

struct sj_parser {
  int device = 0;
  uint64_t max_bytes = 0;
  uint32_t max_docs = 0;
  uint32_t max_depth = 0;
  uint64_t max_tiles = 0;
  // device memory
  uint8_t *d_input = nullptr;
  uint64_t *d_doc_off = nullptr;
  uint32_t *d_tile_first = nullptr;
  uint32_t *d_counters = nullptr;
  uint32_t *d_tile_cnt = nullptr;
  uint32_t *d_tile_off = nullptr;
  sj::S1Agg *d_s1_rec = nullptr;
  sj::S1Pre *d_s1_pre = nullptr;
  uint64_t *d_s1_blk = nullptr;
  sj::S2Agg *d_s2_rec = nullptr;
  sj::S2Pre *d_s2_pre = nullptr;
  sj::S2Agg *d_scan_agg = nullptr;
  sj::S2Agg *d_scan_pre = nullptr;
  sj::S1Agg *d_scan_agg1 = nullptr;
  sj::S1Agg *d_scan_pre1 = nullptr;
  int32_t *d_spt = nullptr;
  uint32_t *d_slen = nullptr;
  ulonglong2 *d_s1_qx = nullptr;
  uint64_t *d_meta = nullptr;
  uint16_t *d_open_g = nullptr;
  uint8_t *d_unesc = nullptr;
  uint32_t *d_nlist = nullptr;
  uint64_t *d_numv = nullptr;  // small parsers only
  uint32_t *d_tile_nnum = nullptr;
  uint64_t *d_front = nullptr;
  uint32_t *d_surv = nullptr;
  uint32_t *d_idx = nullptr;
  uint64_t *d_tape = nullptr;
  uint8_t *d_strings = nullptr;
  uint32_t *d_doc_flags = nullptr;
  uint32_t *d_doc_nidx = nullptr;
  unsigned long long *d_doc_err = nullptr;
  uint64_t *d_doc_tape = nullptr;
  uint64_t *d_doc_str = nullptr;
  sj_doc_result *d_results = nullptr;
  Job *d_job = nullptr;
  // pinned host memory
  Job *h_job = nullptr;
  uint64_t *h_doc_off = nullptr;
  sj_doc_result *h_results = nullptr;
  // their addresses on the device (small runs read and write them in place)
  Job *h_job_dev = nullptr;
  uint64_t *h_doc_off_dev = nullptr;
  sj_doc_result *h_results_dev = nullptr;
  // at most kSmallTiles stage-2 tiles: one-block scans, sparse table built
  // with scan 2; with `sub`, stage-2 tiles of a quarter on whole runs
  bool small = false, sub = false;
  size_t spt_smem = 0;  // small: the one-block sparse table's shared memory
  // launch shapes
  int s1_grid = 0, fl_grid = 0, s2r_grid = 0, s2b_grid = 0, fin_grid = 0, aux_grid = 0;
  // The most blocks a launch can use: the kernels loop over tiles (4 per
  // block of the main kernels, 8 per block of the frontier) and documents, so
  // a parser for small inputs launches no blocks that would find no work.
  int tile_blocks = 1, aux_blocks = 1, doc_blocks = 1;
  int num_grid = 0;
  int sms = 0;
  int occ[4] = {1, 1, 1, 1};  // most resident blocks per SM: s1 blocks, flatten, reduce, build
  uint32_t scan_blocks = 0, scan_grid = 0, spt_levels = 0;
  uint64_t device_bytes = 0;  // cudaMalloc'ed by this parser
  // graph cache: one captured run per document-count bucket (powers of two)
  static constexpr int kBuckets = 33;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graphs[kBuckets] = {};
  cudaEvent_t done = nullptr;
  static constexpr int kStages = 9;
  cudaEvent_t prof[kStages + 1] = {};
  // chunked runs over a host document
  static constexpr uint32_t kMaxChunks = 64;
  static_assert(kMaxChunks <= (uint32_t)sj::kMaxChunkSlots, "a stage-2 bound slot per chunk");
  uint64_t host_chunk = 512ull << 20;  // largest chunk; 0 = never chunk
  cudaStream_t copy_stream = nullptr;
  cudaStream_t aux_stream = nullptr;  // the numbers kernel, beside the tile scan and frontier
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_start = nullptr;
  cudaEvent_t ev_chunk[kMaxChunks] = {};
  cudaStream_t s1_stream = nullptr;  // stage 1 of the chunks, ahead of stage 2
  cudaEvent_t ev_setup = nullptr;
  cudaEvent_t ev_s1[kMaxChunks] = {};
  bool chunked_run = false;
  bool profiling = false;
  bool profiled_run = false;
  bool pending = false;  // an async parse is in flight
  uint32_t last_docs = 0;
  uint64_t last_len = 0;
};

static int cuda_fail(cudaError_t e) {
  g_last_cuda_error = (int)e;
  return e == cudaErrorMemoryAllocation ? SJ_MEMALLOC : SJ_INTERNAL;
}
#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

template <class T>
static int dalloc(sj_parser *p, T **ptr, uint64_t n) {
  const size_t bytes = (size_t)(n ? n : 1) * sizeof(T);
  CK(cudaMalloc((void **)ptr, bytes));
  p->device_bytes += bytes;
  return SJ_SUCCESS;
}

extern "C" void sj_parser_destroy(sj_parser *p) {
  if (!p) return;
  if (p->pending) cudaEventSynchronize(p->done);
  for (cudaGraphExec_t g : p->graphs)
    if (g) cudaGraphExecDestroy(g);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  if (p->aux_stream) cudaStreamDestroy(p->aux_stream);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  if (p->s1_stream) cudaStreamDestroy(p->s1_stream);
  if (p->ev_setup) cudaEventDestroy(p->ev_setup);
  for (cudaEvent_t e : p->ev_s1)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_chunk)
    if (e) cudaEventDestroy(e);
  if (p->done) cudaEventDestroy(p->done);
  for (cudaEvent_t e : p->prof)
    if (e) cudaEventDestroy(e);
  void *dev[] = {p->d_input, p->d_doc_off, p->d_tile_first, p->d_counters, p->d_tile_cnt,
                 p->d_tile_off, p->d_s1_rec, p->d_s1_pre, p->d_s1_blk, p->d_s2_rec, p->d_s2_pre,
                 p->d_scan_agg, p->d_scan_pre, p->d_scan_agg1, p->d_scan_pre1, p->d_spt, p->d_slen, p->d_front, p->d_surv,
                 p->d_idx, p->d_tape, p->d_strings, p->d_doc_flags, p->d_doc_nidx, p->d_doc_err,
                 p->d_doc_tape, p->d_doc_str, p->d_results, p->d_job, p->d_s1_qx, p->d_meta,
                 p->d_open_g, p->d_unesc, p->d_nlist, p->d_numv, p->d_tile_nnum};
  for (void *q : dev)
    if (q) cudaFree(q);
  if (p->h_job) cudaFreeHost(p->h_job);
  if (p->h_doc_off) cudaFreeHost(p->h_doc_off);
  if (p->h_results) cudaFreeHost(p->h_results);
  delete p;
}

static int create_impl(sj_parser *p, uint64_t max_bytes, uint32_t max_docs, uint32_t max_depth) {
  CK(cudaGetDevice(&p->device));
  p->max_bytes = max_bytes;
  p->max_docs = max_docs;
  p->max_depth = max_depth;
  p->max_tiles = max_bytes / sj::kTileBytes + (uint64_t)max_docs + 1;
  const uint64_t tiles = p->max_tiles;
  // A parser of at most kSubTiles tiles splits each stage-1 tile in four for
  // stage 2 on whole-document runs (its stage-2 arrays hold four times the
  // tiles); a parser of at most kSmallTiles stage-2 tiles scans in one block.
  p->sub = tiles <= sj::kSubTiles;
  const uint64_t tiles2 = p->sub ? tiles << sj::kSmallShift : tiles;
  p->small = tiles2 <= sj::kSmallTiles;
  int r;
  if ((r = dalloc(p, &p->d_input, max_bytes + 64))) return r;
  if ((r = dalloc(p, &p->d_doc_off, (uint64_t)max_docs + 1))) return r;
  if ((r = dalloc(p, &p->d_tile_first, (uint64_t)max_docs + 1))) return r;
  if ((r = dalloc(p, &p->d_counters, sj::kCounters))) return r;
  p->scan_blocks = (uint32_t)((tiles + sj::kScanBlock - 1) / sj::kScanBlock);
  p->scan_grid = 0;  // set with the SM count below
  p->spt_levels = 2;
  while ((1ull << (p->spt_levels - 1)) <= tiles2) p->spt_levels++;
  if ((r = dalloc(p, &p->d_tile_cnt, tiles2))) return r;
  if ((r = dalloc(p, &p->d_tile_off, tiles2))) return r;
  if ((r = dalloc(p, &p->d_s1_rec, tiles))) return r;
  if ((r = dalloc(p, &p->d_s1_pre, tiles))) return r;
  if ((r = dalloc(p, &p->d_s1_blk, tiles * 64))) return r;
  if ((r = dalloc(p, &p->d_s2_rec, tiles2))) return r;
  if ((r = dalloc(p, &p->d_s2_pre, tiles2))) return r;
  if ((r = dalloc(p, &p->d_scan_agg, p->scan_blocks))) return r;
  if ((r = dalloc(p, &p->d_scan_pre, p->scan_blocks))) return r;
  if ((r = dalloc(p, &p->d_scan_agg1, p->scan_blocks))) return r;
  if ((r = dalloc(p, &p->d_scan_pre1, p->scan_blocks))) return r;
  if ((r = dalloc(p, &p->d_spt, (uint64_t)p->spt_levels * tiles2))) return r;
  if (p->small) {
    p->spt_smem = (size_t)p->spt_levels * tiles2 * sizeof(int32_t);
    // the limit of the function, for every parser alike: the largest table
    // (13 levels of kSmallTiles)
    CK(sj::prepare_scan2_spt_small((size_t)13 * sj::kSmallTiles * sizeof(int32_t)));
  }
  if ((r = dalloc(p, &p->d_slen, max_bytes + 16))) return r;
  if ((r = dalloc(p, &p->d_s1_qx, tiles * 32))) return r;
  if ((r = dalloc(p, &p->d_meta, max_bytes + 16))) return r;
  if ((r = dalloc(p, &p->d_unesc, max_bytes + 64 + 16))) return r;
  if ((r = dalloc(p, &p->d_nlist, max_bytes + 16))) return r;
  if (p->small && (r = dalloc(p, &p->d_numv, max_bytes + 16))) return r;  // per index slot
  if ((r = dalloc(p, &p->d_tile_nnum, tiles2))) return r;
  if ((r = dalloc(p, &p->d_front, max_bytes + tiles2 + 16))) return r;
  if ((r = dalloc(p, &p->d_surv, max_bytes + 16))) return r;
  if ((r = dalloc(p, &p->d_idx, max_bytes + 16))) return r;
  if ((r = dalloc(p, &p->d_tape, max_bytes + 3ull * max_docs + 8))) return r;
  if ((r = dalloc(p, &p->d_strings, (5 * max_bytes) / 2 + 8ull * max_docs + 64))) return r;
  if ((r = dalloc(p, &p->d_doc_flags, max_docs))) return r;
  if ((r = dalloc(p, &p->d_doc_nidx, max_docs))) return r;
  if ((r = dalloc(p, &p->d_doc_err, max_docs))) return r;
  if ((r = dalloc(p, &p->d_doc_tape, max_docs))) return r;
  if ((r = dalloc(p, &p->d_doc_str, max_docs))) return r;
  if ((r = dalloc(p, &p->d_results, max_docs))) return r;
  if ((r = dalloc(p, &p->d_job, 1))) return r;
  CK(cudaMemset(p->d_counters, 0, sj::kCounters * sizeof(uint32_t)));
  CK(cudaMallocHost((void **)&p->h_job, sizeof(Job)));
  CK(cudaMallocHost((void **)&p->h_doc_off, ((size_t)max_docs + 1) * sizeof(uint64_t)));
  CK(cudaMallocHost((void **)&p->h_results, (size_t)max_docs * sizeof(sj_doc_result)));
  CK(cudaHostGetDevicePointer((void **)&p->h_job_dev, p->h_job, 0));
  CK(cudaHostGetDevicePointer((void **)&p->h_doc_off_dev, p->h_doc_off, 0));
  CK(cudaHostGetDevicePointer((void **)&p->h_results_dev, p->h_results, 0));
  CK(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming));
  for (cudaEvent_t &e : p->prof) CK(cudaEventCreate(&e));
  CK(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&p->aux_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming));
  for (cudaEvent_t &e : p->ev_chunk) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  CK(cudaStreamCreateWithFlags(&p->s1_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&p->ev_setup, cudaEventDisableTiming));
  for (cudaEvent_t &e : p->ev_s1) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));

  int sms = 0, occ1 = 0, occf = 0, occ2r = 0, occ2b = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, sj::stage1_blocks_kernel,
                                                   32 * sj::kS1Warps, 0));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occf, sj::stage1_flatten_kernel,
                                                   32 * sj::kS1Warps, 0));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2r, sj::stage2_reduce_kernel,
                                                   sj::kS2Threads, 0));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2b, sj::stage2_build_kernel,
                                                   sj::kS2Threads, 0));
  p->sms = sms;
  p->scan_grid = p->scan_blocks < (uint32_t)(2 * sms) ? p->scan_blocks : (uint32_t)(2 * sms);
  p->occ[0] = occ1 > 0 ? occ1 : 1;
  p->occ[1] = occf > 0 ? occf : 1;
  p->occ[2] = occ2r > 0 ? occ2r : 1;
  p->occ[3] = occ2b > 0 ? occ2b : 1;
  // default launch: every SM full (the grids are grid-stride loops over tiles)
  p->s1_grid = sms * p->occ[0];
  p->fl_grid = sms * p->occ[1];
  p->s2r_grid = sms * p->occ[2];
  p->s2b_grid = sms * p->occ[3];
  // level tables of the reduce warps (zero between tiles)
  // (a reduce launch never has more blocks than its tiles can use: tables for
  // at most that many blocks)
  const uint64_t reduce_blocks = std::min<uint64_t>((uint64_t)p->s2r_grid, (tiles2 + 3) / 4);
  const uint64_t open_entries = reduce_blocks * (sj::kS2Threads / 32) * sj::kOpenGlobal;
  if ((r = dalloc(p, &p->d_open_g, open_entries))) return r;
  CK(cudaMemset(p->d_open_g, 0, open_entries * sizeof(uint16_t)));
  int occn = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occn, sj::numbers_kernel, 128, 0));
  // half its occupancy: the numbers kernel runs beside the build pass, and at
  // full occupancy its blocks, launched first, hold the build's off the SMs
  // (1 GiB document: 12 blocks per SM 8.56 ms, 6 blocks 8.50, 4 blocks 8.60,
  // 2 blocks 8.72)
  p->num_grid = sms * (occn > 1 ? occn / 2 : 1);
  p->fin_grid = sms * 4;
  p->aux_grid = sms * 8;
  p->tile_blocks = (int)((tiles2 + 3) / 4);
  p->aux_blocks = (int)((tiles2 + 7) / 8);
  p->doc_blocks = (int)((max_docs + 255) / 256);

  Job &J = *p->h_job;
  memset(&J, 0, sizeof(J));
  J.doc_off = p->d_doc_off;
  J.max_depth = max_depth;
  J.max_doc_len = sj::kMaxDocBytes;
  J.tile_first = p->d_tile_first;
  J.counters = p->d_counters;
  J.tile_cnt = p->d_tile_cnt;
  J.tile_off = p->d_tile_off;
  J.s1_rec = p->d_s1_rec;
  J.s1_pre = p->d_s1_pre;
  J.s1_blk = p->d_s1_blk;
  J.s2_rec = p->d_s2_rec;
  J.s2_pre = p->d_s2_pre;
  J.scan_agg = p->d_scan_agg;
  J.scan_pre = p->d_scan_pre;
  J.scan_agg1 = p->d_scan_agg1;
  J.scan_pre1 = p->d_scan_pre1;
  J.spt = p->d_spt;
  J.spt_stride = (uint32_t)tiles2;
  J.spt_levels = p->spt_levels;
  J.slen = p->d_slen;
  J.s1_qx = p->d_s1_qx;
  J.meta = p->d_meta;
  J.open_g = p->d_open_g;
  J.unesc = p->d_unesc;
  J.nlist = p->d_nlist;
  J.numv = p->d_numv;
  J.tile_nnum = p->d_tile_nnum;
  J.front = p->d_front;
  J.surv = p->d_surv;
  J.idx = p->d_idx;
  J.tape = p->d_tape;
  J.strings = p->d_strings;
  J.doc_flags = p->d_doc_flags;
  J.doc_nidx = p->d_doc_nidx;
  J.doc_err = p->d_doc_err;
  J.doc_tape = p->d_doc_tape;
  J.doc_str = p->d_doc_str;
  J.results = p->d_results;
  return SJ_SUCCESS;
}

extern "C" sj_status sj_parser_create(sj_parser **out, uint64_t max_bytes, uint32_t max_docs,
                                      uint32_t max_depth) {
  if (!out) return SJ_INVALID_ARG;
  *out = nullptr;
  if (max_docs == 0) max_docs = 1;
  if (max_depth == 0) max_depth = 4096;
  if (max_depth > sj::kMaxDepthLimit || max_bytes == 0) return SJ_INVALID_ARG;
  sj_parser *p = new (std::nothrow) sj_parser();
  if (!p) return SJ_MEMALLOC;
  int r = create_impl(p, max_bytes, max_docs, max_depth);
  if (r) {
    sj_parser_destroy(p);
    return r;
  }
  *out = p;
  return SJ_SUCCESS;
}

static inline int cap(int grid, int most) { return grid < most ? grid : most; }

// The kernels of one run, in order.  With `ev`, an event is recorded before
// the first kernel and after each of the stages named in STAGE_NAMES.  With
// `pdl` a kernel that follows another kernel on the same stream is launched
// with programmatic stream serialization (sj::launch_k), so that it is
// launched as soon as the blocks of the one before have exited; every run
// uses it but the profiled runs, whose events between kernels time each
// stage alone.
static void enqueue_stage1(sj_parser *p, cudaStream_t s, cudaEvent_t *ev, bool pdl) {
  sj::launch_k(pdl, sj::stage1_blocks_kernel, cap(p->s1_grid, p->tile_blocks), 32 * sj::kS1Warps, 0, s,
               (const Job *)p->d_job);
  if (ev) cudaEventRecord(ev[2], s);
  if (p->small) sj::launch_scan1_small(p->d_job, s, pdl);
  else sj::launch_scan1(p->d_job, p->scan_grid, s, pdl);
  if (ev) cudaEventRecord(ev[3], s);
  sj::launch_k(pdl, sj::stage1_flatten_kernel, cap(p->fl_grid, p->tile_blocks), 32 * sj::kS1Warps, 0, s,
               (const Job *)p->d_job);
  if (ev) cudaEventRecord(ev[4], s);
}

// Stage 2.  numbers_kernel needs the reduce pass's number lists and the tile
// scan's first tape slots, and writes only its tokens' tape words and
// errors, so (except in profiled runs, which time each stage alone) it runs
// on a second stream from the tile scan on, beside the sparse-table,
// frontier and build kernels, joined after the build pass.  Small whole runs
// use little of the GPU in their scan and frontier kernels, so there the
// numbers run beside those instead (numbers_split_kernel: four warps per
// tile, 32 numbers each, the last warp the rest), from the reduce pass on,
// leaving values and tags for the build pass, joined before it.
// `whole`: the run covers whole documents from tile 0 (not a round of a
// chunked run), so a small parser may build the sparse table with scan 2.
static void enqueue_stage2(sj_parser *p, cudaStream_t s, cudaEvent_t *ev, bool whole, bool pdl) {
  const bool small = p->small && whole;
  const bool sub = p->sub && whole;  // the run's s2_shift
  const Job *job = p->d_job;
  auto numbers = [&](cudaStream_t st) {
    if (small) sj::numbers_split_kernel<<<p->tile_blocks * 4, 128, 0, st>>>(p->d_job);
    else sj::numbers_kernel<<<cap(p->num_grid, p->tile_blocks), 128, 0, st>>>(p->d_job);
  };
  auto fork_numbers = [&]() {
    if (ev) return;
    cudaEventRecord(p->ev_fork, s);
    cudaStreamWaitEvent(p->aux_stream, p->ev_fork, 0);
    numbers(p->aux_stream);
    cudaEventRecord(p->ev_join, p->aux_stream);
  };
  sj::launch_k(pdl, sub ? sj::stage2_reduce_sub_kernel : sj::stage2_reduce_kernel,
               cap(p->s2r_grid, p->tile_blocks), sj::kS2Threads, 0, s, job);
  if (ev) cudaEventRecord(ev[5], s);
  if (small) {
    fork_numbers();
    sj::launch_scan2_spt_small(job, p->spt_smem, s, pdl);  // scan, sparse table, jump pointers
  } else {
    sj::launch_scan2(job, p->scan_grid, s, pdl);
    fork_numbers();
    for (uint32_t src = 0; src + 1 < p->spt_levels; src += 4)
      sj::launch_k(pdl, sj::spt_build_kernel, cap(p->aux_grid, p->aux_blocks), 256, 0, s, job, src);
    sj::launch_k(pdl, sj::jump_kernel, cap(p->aux_grid, p->aux_blocks), 256, 0, s, job);
  }
  sj::launch_k(pdl, sj::frontier_kernel, cap(p->aux_grid, p->aux_blocks), 256, 0, s, job);
  if (ev) cudaEventRecord(ev[6], s);
  if (ev) numbers(s);
  if (ev) cudaEventRecord(ev[7], s);
  if (small) {
    if (!ev) cudaStreamWaitEvent(s, p->ev_join, 0);
    if (sub) sj::stage2_build_sub_kernel<<<cap(p->s2b_grid, p->tile_blocks), sj::kS2Threads, 0, s>>>(p->d_job);
    else sj::stage2_build_small_kernel<<<cap(p->s2b_grid, p->tile_blocks), sj::kS2Threads, 0, s>>>(p->d_job);
    if (ev) cudaEventRecord(ev[8], s);
  } else {
    sj::launch_k(pdl, sj::stage2_build_kernel, cap(p->s2b_grid, p->tile_blocks), sj::kS2Threads, 0, s, job);
    if (ev) cudaEventRecord(ev[8], s);
    if (!ev) cudaStreamWaitEvent(s, p->ev_join, 0);
  }
}

// With `zc` the set-up kernel reads the run descriptor and the offsets of
// n_off documents from pinned host memory (no copy before the run).
static void enqueue_run(sj_parser *p, cudaStream_t s, cudaEvent_t *ev, bool zc, uint32_t n_off) {
  if (ev) cudaEventRecord(ev[0], s);
  sj::setup_kernel<<<1, 1024, 0, s>>>(p->d_job, zc ? p->h_job_dev : nullptr,
                                      zc ? p->h_doc_off_dev : nullptr, zc ? n_off : 0u);
  if (ev) cudaEventRecord(ev[1], s);
  const bool pdl = !ev;
  enqueue_stage1(p, s, ev, pdl);
  enqueue_stage2(p, s, ev, true, pdl);
  sj::finalize_kernel<<<cap(p->fin_grid, p->doc_blocks), 256, 0, s>>>(p->d_job);
  if (ev) cudaEventRecord(ev[9], s);
}

static uint32_t kernels_per_run(const sj_parser *p) {
  if (p->small)
    return 2 /* setup, blocks */ + 1 + 1 /* scan1, flatten */ + 1 + 1 /* reduce; scan2, sparse
         table and jump pointers */ + 1 /* frontier */ + 1 /* numbers */ + 1 + 1 /* build, finalize */;
  return 2 /* setup, blocks */ + 3 + 1 /* scan1, flatten */ + 1 + 3 /* reduce, scan2 */ +
         (p->spt_levels + 2) / 4 + 2 /* sparse table, jump, frontier */ + 1 /* numbers */ +
         1 + 1 /* build, finalize */;
}

// Whether a run of n_docs documents (its graph bucket) exchanges its
// descriptor, offsets and results through pinned host memory.
static bool zero_copy(const sj_parser *p, uint32_t n_docs);

// The launch sequence of one run, captured once per bucket of document
// counts: the kernels read the count from the run descriptor, and the copies
// of the offsets and results move a whole bucket (the smallest power of two
// not below the count, at most max_docs).
static uint32_t bucket_of(const sj_parser *p, uint32_t n_docs, int *b) {
  int k = 0;
  while ((1ull << k) < n_docs) k++;
  *b = k;
  return (uint32_t)((1ull << k) < p->max_docs ? (1ull << k) : p->max_docs);
}

static int ensure_graph(sj_parser *p, uint32_t n_docs, cudaGraphExec_t *out) {
  int b;
  const uint32_t nb = bucket_of(p, n_docs, &b);
  if (p->graphs[b]) {
    *out = p->graphs[b];
    return SJ_SUCCESS;
  }
  cudaStream_t s = p->cap_stream;
  cudaGraph_t g = nullptr;
  const bool zc = nb <= sj::kZeroCopyDocs;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  if (!zc) {
    cudaMemcpyAsync(p->d_job, p->h_job, sizeof(Job), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->d_doc_off, p->h_doc_off, ((size_t)nb + 1) * sizeof(uint64_t),
                    cudaMemcpyHostToDevice, s);
  }
  enqueue_run(p, s, nullptr, zc, nb + 1);
  if (!zc)
    cudaMemcpyAsync(p->h_results, p->d_results, (size_t)nb * sizeof(sj_doc_result),
                    cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaGraphInstantiate(&p->graphs[b], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    p->graphs[b] = nullptr;
    return cuda_fail(e);
  }
  *out = p->graphs[b];
  return SJ_SUCCESS;
}

static bool zero_copy(const sj_parser *p, uint32_t n_docs) {
  int b;
  return bucket_of(p, n_docs, &b) <= sj::kZeroCopyDocs;
}

static bool is_device_ptr(const void *ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device's address of pinned (page-locked) host memory, or null.
static const uint8_t *pinned_device_ptr(const void *ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? static_cast<const uint8_t *>(a.devicePointer) : nullptr;
}

static int wait_pending(sj_parser *p) {
  if (!p->pending) return SJ_SUCCESS;
  p->pending = false;
  CK(cudaEventSynchronize(p->done));
  return SJ_SUCCESS;
}

// One document of `len` bytes in pinned host memory, parsed while it is copied
// (Sec. 3: stage 1 and stage 2 may run over a stream of chunks).  The copy
// stream moves the chunks in order, each followed by an event; a stage-1
// stream waits for chunk c, runs stage 1 on its tiles (the tile scans carry
// the state of the tiles before) and notes the stage-2 bound the chunk
// allows; the run's stream waits for that, runs stage 2 on the tiles up to
// the bound (chunk_range_kernel), and after the last chunk on all that
// remain.
static int enqueue_chunked(sj_parser *p, const uint8_t *host, uint64_t len, cudaStream_t s) {
  // Chunk sizes: a small first chunk (nothing overlaps its copy), then
  // growing by 7/4 up to host_chunk: the copies run about 1.75 times as fast
  // as the parse (~211 against ~121 GB/s), so each chunk lands as the kernels
  // finish the one before (doubling made the copies the bottleneck: 2% slower
  // end to end).  The last of kMaxChunks chunks takes whatever remains.
  const uint64_t tile = sj::kTileBytes;
  const uint64_t cmax = p->host_chunk;
  uint64_t sz = (cmax / 16 + tile - 1) / tile * tile;
  uint64_t at[sj_parser::kMaxChunks + 1];
  uint32_t nc = 0;
  at[0] = 0;
  while (at[nc] < len) {
    const uint64_t o = at[nc];
    const uint64_t n = nc + 1 == sj_parser::kMaxChunks || len - o < sz ? len - o : sz;
    at[++nc] = o + n;
    const uint64_t grown = (sz * 7 / 4 + tile - 1) / tile * tile;
    sz = grown < cmax ? grown : cmax;
  }
  CK(cudaMemcpyAsync(p->d_job, p->h_job, sizeof(Job), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->d_doc_off, p->h_doc_off, 2 * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  // the input buffer is free once the work queued before this run is done
  CK(cudaEventRecord(p->ev_start, s));
  CK(cudaStreamWaitEvent(p->copy_stream, p->ev_start, 0));
  for (uint32_t c = 0; c < nc; c++) {
    CK(cudaMemcpyAsync(p->d_input + at[c], host + at[c], at[c + 1] - at[c], cudaMemcpyHostToDevice,
                       p->copy_stream));
    CK(cudaEventRecord(p->ev_chunk[c], p->copy_stream));
  }
  sj::setup_kernel<<<1, 1024, 0, s>>>(p->d_job, nullptr, nullptr, 0u);
  // stage 1 of every chunk on its own stream, as the chunks land: it reads
  // landed bytes and writes the arrays of its own tiles only (its tile scan
  // has its own scratch), so it runs beside stage 2 of the chunks before
  CK(cudaEventRecord(p->ev_setup, s));
  CK(cudaStreamWaitEvent(p->s1_stream, p->ev_setup, 0));
  for (uint32_t c = 0; c < nc; c++) {
    CK(cudaStreamWaitEvent(p->s1_stream, p->ev_chunk[c], 0));
    sj::chunk_range_kernel<<<1, 32, 0, p->s1_stream>>>(
        p->d_job, (uint32_t)(at[c] / tile), (uint32_t)((at[c + 1] + tile - 1) / tile), 0, c, 0);
    enqueue_stage1(p, p->s1_stream, nullptr, true);
    sj::launch_k(true, sj::chunk_range_kernel, 1, 32, 0, p->s1_stream, (const Job *)p->d_job, 0u, 0u, 1, c, 0);
    CK(cudaEventRecord(p->ev_s1[c], p->s1_stream));
  }
  for (uint32_t c = 0; c < nc; c++) {
    CK(cudaStreamWaitEvent(s, p->ev_s1[c], 0));
    sj::chunk_range_kernel<<<1, 32, 0, s>>>(p->d_job, 0, 0, 2, c, c + 1 == nc);
    enqueue_stage2(p, s, nullptr, false, true);
  }
  sj::finalize_kernel<<<cap(p->fin_grid, p->doc_blocks), 256, 0, s>>>(p->d_job);
  CK(cudaMemcpyAsync(p->h_results, p->d_results, sizeof(sj_doc_result), cudaMemcpyDeviceToHost, s));
  CK(cudaGetLastError());
  return SJ_SUCCESS;
}

// Queue one run over n_docs documents whose offsets are in h_doc_off.
static int launch(sj_parser *p, const uint8_t *bytes, uint64_t total, uint32_t n_docs,
                  cudaStream_t stream) {
  int r;
  if ((r = wait_pending(p))) return r;
  const uint8_t *base = bytes, *src = nullptr;
  bool chunked = false;
  if (!is_device_ptr(bytes)) {
    // one document in pinned host memory: parsed while it is copied when it
    // spans several chunks, else stage 1 reads it over the host link and
    // writes the device copy; any other host input is copied first
    src = n_docs == 1 && total ? pinned_device_ptr(bytes) : nullptr;
    chunked = src && p->host_chunk && total > p->host_chunk && !p->profiling;
    if (chunked) src = nullptr;
    else if (!src) CK(cudaMemcpyAsync(p->d_input, bytes, total, cudaMemcpyHostToDevice, stream));
    base = p->d_input;
  }
  p->h_job->base = base;
  p->h_job->src = src;
  // the scratch copy of escaped strings keeps the input's alignment modulo 16
  // (the build pass stages both windows alike)
  p->h_job->unesc = p->d_unesc + (((uintptr_t)base + p->h_doc_off[0]) & 15u);
  p->h_job->n_docs = n_docs;
  // stage-2 tiles of a quarter on a small parser's whole-document runs
  p->h_job->s2_shift = p->sub && !chunked ? sj::kSmallShift : 0u;
  // the graph of a small bucket writes the results straight to pinned host
  // memory; every other run writes them on the device and copies them back
  const bool zc = !chunked && !p->profiling && zero_copy(p, n_docs);
  p->h_job->results = zc ? p->h_results_dev : p->d_results;
  p->chunked_run = chunked;
  if (chunked) {
    if ((r = enqueue_chunked(p, bytes, total, stream))) return r;
    p->profiled_run = false;
  } else if (p->profiling) {
    // the same sequence as the graph, with events between the kernels
    CK(cudaMemcpyAsync(p->d_job, p->h_job, sizeof(Job), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(p->d_doc_off, p->h_doc_off, ((size_t)n_docs + 1) * sizeof(uint64_t),
                       cudaMemcpyHostToDevice, stream));
    enqueue_run(p, stream, p->prof, false, 0);
    CK(cudaMemcpyAsync(p->h_results, p->d_results, (size_t)n_docs * sizeof(sj_doc_result),
                       cudaMemcpyDeviceToHost, stream));
    CK(cudaGetLastError());
    p->profiled_run = true;
  } else {
    cudaGraphExec_t g;
    if ((r = ensure_graph(p, n_docs, &g))) return r;
    CK(cudaGraphLaunch(g, stream));
    p->profiled_run = false;
  }
  CK(cudaEventRecord(p->done, stream));
  p->pending = true;
  p->last_docs = n_docs;
  return SJ_SUCCESS;
}

static void fill_result(sj_parser *p, sj_result *out) {
  const sj_doc_result &r = p->h_results[0];
  out->error = r.error;
  out->reserved = 0;
  out->n_indices = r.n_indices;
  out->tape_words = r.tape_words;
  out->string_bytes = r.string_bytes;
  out->indices = p->d_idx;
  out->tape = p->d_tape;
  out->strings = p->d_strings;
}

extern "C" sj_status sj_parse_async(sj_parser *p, const uint8_t *bytes, uint64_t len, void *stream) {
  if (!p || (!bytes && len)) return SJ_INVALID_ARG;
  if (len > p->max_bytes) return SJ_CAPACITY;
  int r;
  if ((r = wait_pending(p))) return r;
  p->h_doc_off[0] = 0;
  p->h_doc_off[1] = len;
  p->last_len = len;
  static const uint8_t empty[16] = {0};
  return launch(p, len ? bytes : empty, len, 1, (cudaStream_t)stream);
}

extern "C" sj_status sj_parse_wait(sj_parser *p, sj_result *out) {
  if (!p || !out) return SJ_INVALID_ARG;
  if (!p->pending) return SJ_INVALID_ARG;
  int r;
  if ((r = wait_pending(p))) return r;
  CK(cudaGetLastError());
  fill_result(p, out);
  return SJ_SUCCESS;
}

extern "C" sj_status sj_parse(sj_parser *p, const uint8_t *bytes, uint64_t len, void *stream,
                              sj_result *out) {
  if (!out) return SJ_INVALID_ARG;
  int r = sj_parse_async(p, bytes, len, stream);
  if (r) return r;
  return sj_parse_wait(p, out);
}

extern "C" sj_status sj_parse_batch_async(sj_parser *p, const uint8_t *bytes,
                                          const uint64_t *doc_offsets, uint32_t n_docs,
                                          void *stream) {
  if (!p || !doc_offsets || n_docs == 0) return SJ_INVALID_ARG;
  if (n_docs > p->max_docs) return SJ_CAPACITY;
  for (uint32_t i = 0; i < n_docs; i++)
    if (doc_offsets[i + 1] < doc_offsets[i]) return SJ_INVALID_ARG;
  const uint64_t total = doc_offsets[n_docs] - doc_offsets[0];
  if (total > p->max_bytes) return SJ_CAPACITY;
  if (!bytes && total) return SJ_INVALID_ARG;
  int r;
  if ((r = wait_pending(p))) return r;
  const bool dev = total ? is_device_ptr(bytes) : false;
  // documents are addressed relative to the first one
  for (uint32_t i = 0; i <= n_docs; i++) p->h_doc_off[i] = doc_offsets[i] - doc_offsets[0];
  const uint8_t *first = bytes ? bytes + doc_offsets[0] : nullptr;
  static const uint8_t empty[16] = {0};
  if (!total) first = empty;
  (void)dev;
  return launch(p, first, total, n_docs, (cudaStream_t)stream);
}

extern "C" int sj_parse_query(sj_parser *p) {
  if (!p) return -SJ_INVALID_ARG;
  if (!p->pending) return 1;
  const cudaError_t e = cudaEventQuery(p->done);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  return -cuda_fail(e);
}

extern "C" sj_status sj_parse_batch_wait(sj_parser *p, sj_doc_result *out, const uint32_t **indices,
                                         const uint64_t **tape, const uint8_t **strings) {
  if (!p || !out || !p->pending) return SJ_INVALID_ARG;
  int r;
  if ((r = wait_pending(p))) return r;
  CK(cudaGetLastError());
  memcpy(out, p->h_results, (size_t)p->last_docs * sizeof(sj_doc_result));
  if (indices) *indices = p->d_idx;
  if (tape) *tape = p->d_tape;
  if (strings) *strings = p->d_strings;
  return SJ_SUCCESS;
}

extern "C" sj_status sj_parse_batch(sj_parser *p, const uint8_t *bytes, const uint64_t *doc_offsets,
                                    uint32_t n_docs, void *stream, sj_doc_result *out,
                                    const uint32_t **indices, const uint64_t **tape,
                                    const uint8_t **strings) {
  if (!out) return SJ_INVALID_ARG;
  int r = sj_parse_batch_async(p, bytes, doc_offsets, n_docs, stream);
  if (r) return r;
  return sj_parse_batch_wait(p, out, indices, tape, strings);
}

extern "C" uint64_t sj_parser_device_bytes(const sj_parser *p) { return p ? p->device_bytes : 0; }

extern "C" sj_status sj_parser_set_profiling(sj_parser *p, int enable) {
  if (!p) return SJ_INVALID_ARG;
  int r;
  if ((r = wait_pending(p))) return r;
  p->profiling = enable != 0;
  return SJ_SUCCESS;
}

extern "C" sj_status sj_parser_stage_times(sj_parser *p, float *ms, int n) {
  if (!p || !ms || n < sj_parser::kStages) return SJ_INVALID_ARG;
  if (!p->profiled_run) return SJ_INVALID_ARG;
  CK(cudaEventSynchronize(p->prof[sj_parser::kStages]));
  for (int i = 0; i < sj_parser::kStages; i++)
    CK(cudaEventElapsedTime(&ms[i], p->prof[i], p->prof[i + 1]));
  return SJ_SUCCESS;
}

extern "C" sj_status sj_parser_prepare(sj_parser *p, uint32_t max_docs) {
  if (!p) return SJ_INVALID_ARG;
  if (max_docs == 0 || max_docs > p->max_docs) max_docs = p->max_docs;
  for (uint64_t n = 1;; n <<= 1) {  // one graph per bucket (powers of two)
    cudaGraphExec_t g;
    const int r = ensure_graph(p, (uint32_t)(n < max_docs ? n : max_docs), &g);
    if (r) return r;
    if (n >= max_docs) break;
  }
  return SJ_SUCCESS;
}

extern "C" sj_status sj_parser_set_host_chunk(sj_parser *p, uint64_t chunk_bytes) {
  if (!p) return SJ_INVALID_ARG;
  int r;
  if ((r = wait_pending(p))) return r;
  p->host_chunk = (chunk_bytes + sj::kTileBytes - 1) / sj::kTileBytes * sj::kTileBytes;
  return SJ_SUCCESS;
}

extern "C" int sj_parser_kernels_per_run(const sj_parser *p) {
  return p ? (int)kernels_per_run(p) : 0;
}

// ---- launch shapes and their autotuner ----------------------------------
static void drop_graphs(sj_parser *p) {
  for (cudaGraphExec_t &g : p->graphs)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

extern "C" sj_status sj_parser_get_launch(const sj_parser *p, uint32_t *blocks_per_sm,
                                          uint32_t *max_blocks_per_sm) {
  if (!p || !blocks_per_sm) return SJ_INVALID_ARG;
  const int g[4] = {p->s1_grid, p->fl_grid, p->s2r_grid, p->s2b_grid};
  for (int k = 0; k < 4; k++) {
    blocks_per_sm[k] = (uint32_t)(g[k] / p->sms);
    if (max_blocks_per_sm) max_blocks_per_sm[k] = (uint32_t)p->occ[k];
  }
  return SJ_SUCCESS;
}

extern "C" sj_status sj_parser_set_launch(sj_parser *p, const uint32_t *blocks_per_sm) {
  if (!p || !blocks_per_sm) return SJ_INVALID_ARG;
  for (int k = 0; k < 4; k++)
    if (blocks_per_sm[k] < 1 || (int)blocks_per_sm[k] > p->occ[k]) return SJ_INVALID_ARG;
  int r;
  if ((r = wait_pending(p))) return r;
  p->s1_grid = p->sms * (int)blocks_per_sm[0];
  p->fl_grid = p->sms * (int)blocks_per_sm[1];
  p->s2r_grid = p->sms * (int)blocks_per_sm[2];  // the reduce level tables fit the largest grid
  p->s2b_grid = p->sms * (int)blocks_per_sm[3];
  drop_graphs(p);
  return SJ_SUCCESS;
}

// For each of the four main kernels in turn, try every resident-block count
// per SM its occupancy allows (the others fixed at their current choice),
// time the kernel with events over `reps` parses of the sample, and keep the
// fastest.  The stages of a run do not share launch shapes, so the kernels
// are tuned one at a time.
extern "C" sj_status sj_parser_autotune(sj_parser *p, const uint8_t *bytes, uint64_t len,
                                        void *stream, int reps, uint32_t *blocks_per_sm,
                                        float *best_ms) {
  if (!p || (!bytes && len) || reps < 1) return SJ_INVALID_ARG;
  if (len > p->max_bytes) return SJ_CAPACITY;
  int r;
  if ((r = wait_pending(p))) return r;
  const bool was_profiling = p->profiling;
  p->profiling = true;
  static const int stage_of[4] = {1, 3, 4, 7};  // index into the stage times
  uint32_t cur[4];
  sj_parser_get_launch(p, cur, nullptr);
  float best[4] = {0, 0, 0, 0};
  for (int k = 0; k < 4; k++) {
    uint32_t pick = cur[k];
    float pick_ms = 3.4e38f;
    for (int b = 1; b <= p->occ[k]; b++) {
      uint32_t trial[4] = {cur[0], cur[1], cur[2], cur[3]};
      trial[k] = (uint32_t)b;
      if ((r = sj_parser_set_launch(p, trial))) break;
      float sum = 0;
      for (int i = 0; i <= reps; i++) {  // the first run warms up
        if ((r = sj_parse_async(p, bytes, len, stream))) break;
        float ms[sj_parser::kStages];
        if ((r = sj_parser_stage_times(p, ms, sj_parser::kStages))) break;
        if (i) sum += ms[stage_of[k]];
      }
      if (r) break;
      const float avg = sum / (float)reps;
      if (avg < pick_ms) {
        pick_ms = avg;
        pick = (uint32_t)b;
      }
    }
    if (r) break;
    cur[k] = pick;
    best[k] = pick_ms;
  }
  wait_pending(p);
  p->profiling = was_profiling;
  const int r2 = sj_parser_set_launch(p, cur);
  if (r) return r;
  if (r2) return r2;
  if (blocks_per_sm)
    for (int k = 0; k < 4; k++) blocks_per_sm[k] = cur[k];
  if (best_ms)
    for (int k = 0; k < 4; k++) best_ms[k] = best[k];
  return SJ_SUCCESS;
}

extern "C" const char *sj_error_name(int code) {
  static const char *names[] = {"SUCCESS",        "CAPACITY",     "MEMALLOC",     "TAPE_ERROR",
                                "DEPTH_ERROR",    "STRING_ERROR", "T_ATOM_ERROR", "F_ATOM_ERROR",
                                "N_ATOM_ERROR",   "NUMBER_ERROR", "UTF8_ERROR",   "UNCLOSED_STRING",
                                "UNESCAPED_CHARS", "EMPTY",       "INVALID_ARG",  "INTERNAL"};
  if (code < 0 || code > 15) return "UNKNOWN";
  return names[code];
}

extern "C" int sj_last_cuda_error(void) { return g_last_cuda_error; }

extern "C" const char *sj_version(void) { return "sj-gb300 0.1 (sm_103a)"; }
