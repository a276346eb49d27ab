// noalloc.cu -- stage 1 (structural indices) of one document without any
// device allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: code that must not allocate device memory at the time it
// parses -- a process whose device memory is all handed to another
// framework's caching allocator, a latency-critical thread that cannot afford
// cudaMalloc's implicit device-wide synchronisation, or a library embedded in a
// host that owns every allocation.  Such a caller passes its own input and
// output buffers; the look-back scratch of the kernel lives in one file-scope
// device array that every GPU loading this library holds until the process
// exits.
//
// The scratch is sized for documents of at most kNoAllocMaxBytes (64 MiB).
// Every call shares it and leaves the last call's contents behind; the start
// of each call clears what must start at zero.  Two calls whose kernels
// overlap on the GPU (different streams, or different host threads on the same
// device) race on the scratch and give wrong results: serialise them.
#include <cuda_runtime.h>
#include <string.h>

#include <functional>
#include <mutex>

#include "sj_internal.cuh"

namespace sj {
__global__ void stage1_kernel(const Job *job);
}  // namespace sj

namespace {

constexpr uint64_t kNoAllocMaxBytes = 64ull << 20;
constexpr uint32_t kNoAllocTiles = (uint32_t)(kNoAllocMaxBytes / sj::kTileBytes) + 1;

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffJob = 0;
constexpr size_t kOffDocOff = align256(kOffJob + sizeof(sj::Job));
constexpr size_t kOffTileFirst = align256(kOffDocOff + 2 * sizeof(uint64_t));
constexpr size_t kOffCounters = align256(kOffTileFirst + 2 * sizeof(uint32_t));
constexpr size_t kOffDocFlags = align256(kOffCounters + 4 * sizeof(uint32_t));
constexpr size_t kOffDocNidx = align256(kOffDocFlags + sizeof(uint32_t));
constexpr size_t kOffS1State = align256(kOffDocNidx + sizeof(uint32_t));
constexpr size_t kOffS1Count = align256(kOffS1State + kNoAllocTiles * sizeof(uint32_t));
constexpr size_t kOffTileCnt = align256(kOffS1Count + kNoAllocTiles * sizeof(uint64_t));
constexpr size_t kOffTileOff = align256(kOffTileCnt + kNoAllocTiles * sizeof(uint32_t));
constexpr size_t kScratchBytes = align256(kOffTileOff + kNoAllocTiles * sizeof(uint32_t));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Fills the run descriptor and clears the look-back state of the scratch.
__global__ void noalloc_init_kernel(sj::Job job, uint64_t len, uint32_t n_tiles) {
  unsigned char *s = g_noalloc_scratch;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t stride = gridDim.x * blockDim.x;
  if (tid == 0) {
    *reinterpret_cast<sj::Job *>(s + kOffJob) = job;
    uint64_t *doc_off = reinterpret_cast<uint64_t *>(s + kOffDocOff);
    doc_off[0] = 0;
    doc_off[1] = len;
    uint32_t *tile_first = reinterpret_cast<uint32_t *>(s + kOffTileFirst);
    tile_first[0] = 0;
    tile_first[1] = n_tiles;
    uint32_t *counters = reinterpret_cast<uint32_t *>(s + kOffCounters);
    counters[0] = 0;
    counters[1] = 0;
    counters[2] = n_tiles;
    counters[3] = 0;
    *reinterpret_cast<uint32_t *>(s + kOffDocFlags) = 0;
    *reinterpret_cast<uint32_t *>(s + kOffDocNidx) = 0;
  }
  uint32_t *st = reinterpret_cast<uint32_t *>(s + kOffS1State);
  uint64_t *cnt = reinterpret_cast<uint64_t *>(s + kOffS1Count);
  for (uint32_t t = tid; t < n_tiles; t += stride) {
    st[t] = 0;
    cnt[t] = 0;
  }
}

// Copies the index count and the document flags to the caller's buffer.
__global__ void noalloc_finish_kernel(uint32_t *result) {
  const unsigned char *s = g_noalloc_scratch;
  result[0] = *reinterpret_cast<const uint32_t *>(s + kOffDocNidx);
  const uint32_t f = *reinterpret_cast<const uint32_t *>(s + kOffDocFlags);
  result[1] = (f & sj::kFlagUtf8 ? 1u : 0u) | (f & sj::kFlagUnclosed ? 2u : 0u) |
              (f & sj::kFlagInternal ? 4u : 0u);
}

// Per-device set-up: the device address of the scratch array and the launch
// shape of the stage-1 kernel.  The array's name is only a host-side stand-in
// in host code, so its device address is asked for once per device, with that
// device current.
constexpr int kMaxDevices = 64;
struct DeviceSetup {
  std::once_flag once;
  cudaError_t err = cudaSuccess;
  unsigned char *scratch = nullptr;
  int grid = 0;
};
DeviceSetup g_setup[kMaxDevices];

void setup_device(DeviceSetup &ds, int dev) {
  void *ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) { ds.err = e; return; }
  int sms = 0, occ = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sj::stage1_kernel, 32 * sj::kS1Warps, 0);
  if (e != cudaSuccess) { ds.err = e; return; }
  ds.scratch = static_cast<unsigned char *>(ptr);
  ds.grid = sms * (occ > 0 ? occ : 1);
}

}  // namespace

// Declared in include/sj.h.
extern "C" sj_status sj_stage1_indices_noalloc(const uint8_t *d_bytes, uint64_t len,
                                               uint32_t *d_indices, uint32_t *d_result,
                                               void *stream) {
  if ((!d_bytes && len) || !d_indices || !d_result) return SJ_INVALID_ARG;
  if (len > kNoAllocMaxBytes) return SJ_CAPACITY;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SJ_INTERNAL;
  DeviceSetup &ds = g_setup[dev];
  std::call_once(ds.once, setup_device, std::ref(ds), dev);
  if (ds.err != cudaSuccess || !ds.scratch) return SJ_INTERNAL;

  unsigned char *s = ds.scratch;
  sj::Job job;
  memset(&job, 0, sizeof(job));
  job.base = d_bytes;
  job.doc_off = reinterpret_cast<const uint64_t *>(s + kOffDocOff);
  job.n_docs = 1;
  job.max_depth = sj::kMaxDepthLimit;
  job.max_doc_len = kNoAllocMaxBytes;
  job.tile_first = reinterpret_cast<uint32_t *>(s + kOffTileFirst);
  job.counters = reinterpret_cast<uint32_t *>(s + kOffCounters);
  job.s1_state = reinterpret_cast<uint32_t *>(s + kOffS1State);
  job.s1_count = reinterpret_cast<uint64_t *>(s + kOffS1Count);
  job.tile_cnt = reinterpret_cast<uint32_t *>(s + kOffTileCnt);
  job.tile_off = reinterpret_cast<uint32_t *>(s + kOffTileOff);
  job.idx = d_indices;
  job.doc_flags = reinterpret_cast<uint32_t *>(s + kOffDocFlags);
  job.doc_nidx = reinterpret_cast<uint32_t *>(s + kOffDocNidx);

  uint32_t n_tiles = (uint32_t)((len + sj::kTileBytes - 1) / sj::kTileBytes);
  cudaStream_t st = (cudaStream_t)stream;
  // Each launch's own status: an error left by earlier, unrelated work is
  // neither blamed on this call nor cleared by it (no cudaGetLastError).
  {
    void *args[] = {&job, &len, &n_tiles};
    e = cudaLaunchKernel((const void *)noalloc_init_kernel, dim3(64), dim3(256), args, 0, st);
    if (e != cudaSuccess) return SJ_INTERNAL;
  }
  {
    const sj::Job *jp = reinterpret_cast<const sj::Job *>(s + kOffJob);
    void *args[] = {&jp};
    e = cudaLaunchKernel((const void *)sj::stage1_kernel, dim3(ds.grid), dim3(32 * sj::kS1Warps),
                         args, 0, st);
    if (e != cudaSuccess) return SJ_INTERNAL;
  }
  {
    void *args[] = {&d_result};
    e = cudaLaunchKernel((const void *)noalloc_finish_kernel, dim3(1), dim3(1), args, 0, st);
    if (e != cudaSuccess) return SJ_INTERNAL;
  }
  return SJ_SUCCESS;
}
