// query.cu -- distinct values at a key path over a device-resident tape: the
// paper's example query "select all distinct user.id" (Table "tab:userid").
//
// The tape makes the walk cheap (Sec. 3): an opener's payload is the index
// after its matching closer, so a container's children are visited by
// skipping whole sub-containers; a number takes two words, anything else one.
// One thread per tape word: the thread of every object opener scans that
// object's keys for the path's first key; when its value is an object it
// scans that object for the next key, and so on; an integer ('l') at the end
// of the path goes into a hash set (open addressing in device memory,
// atomicCAS on 64-bit keys), whose first insertion of a value also appends it
// to the output.  As in the paper's recursive search, the path may start at
// any object of the document.
#include <cuda_runtime.h>
#include <string.h>

#include <new>

#include "sj.h"

namespace sj {

constexpr uint32_t kMaxPath = 8;
constexpr uint32_t kMaxPathBytes = 256;
constexpr uint64_t kEmpty = ~0ull;  // free slot; the value -1 itself is kept in a flag

struct QueryDev {
  uint32_t path_len;
  uint32_t key_off[kMaxPath + 1];  // key k is key_bytes[key_off[k] .. key_off[k + 1])
  uint8_t key_bytes[kMaxPathBytes];
};

__device__ __forceinline__ uint8_t tag_of(uint64_t w) { return (uint8_t)(w >> 56); }
__device__ __forceinline__ uint64_t payload(uint64_t w) { return w & 0x00FFFFFFFFFFFFFFull; }

// Index of the tape word after the value starting at v (v + 1 at least, so
// that a walk always advances).
__device__ __forceinline__ uint64_t after_value(const uint64_t *tape, uint64_t v) {
  const uint64_t w = tape[v];
  const uint8_t t = tag_of(w);
  if (t == '{' || t == '[') return max(payload(w), v + 1);  // one past the matching closer
  if (t == 'l' || t == 'd') return v + 2;
  return v + 1;
}

// Does the string at buffer offset `off` equal key k of the path?
__device__ __forceinline__ bool key_is(const uint8_t *strings, uint64_t nstr, uint64_t off,
                                       const QueryDev &q, uint32_t k) {
  const uint32_t n = q.key_off[k + 1] - q.key_off[k];
  if (off + 4 + n > nstr) return false;
  const uint8_t *s = strings + off;
  const uint32_t len = (uint32_t)s[0] | ((uint32_t)s[1] << 8) | ((uint32_t)s[2] << 16) |
                       ((uint32_t)s[3] << 24);
  if (len != n) return false;
  for (uint32_t i = 0; i < n; i++)
    if (s[4 + i] != q.key_bytes[q.key_off[k] + i]) return false;
  return true;
}

// Value index of key k in the object opening at tape index o, or 0.  Every
// index stays below T (a tape of a failed parse is read without faults).
__device__ __forceinline__ uint64_t find_key(const uint64_t *tape, uint64_t T,
                                             const uint8_t *strings, uint64_t nstr, uint64_t o,
                                             const QueryDev &q, uint32_t k) {
  const uint64_t p = min(payload(tape[o]), T);
  if (p < o + 2) return 0;
  const uint64_t end = p - 1;  // the closer
  uint64_t j = o + 1;
  while (j + 1 < end) {
    const uint64_t kw = tape[j];
    if (tag_of(kw) != '"') return 0;  // not a tape of a valid object
    if (key_is(strings, nstr, payload(kw), q, k)) return j + 1;
    j = after_value(tape, j + 1);
  }
  return 0;
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {  // splitmix64 finaliser
  x ^= x >> 30;
  x *= 0xBF58476D1CE4E5B9ull;
  x ^= x >> 27;
  x *= 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void query_distinct_kernel(const uint64_t *__restrict__ tape, uint64_t T,
                                      const uint8_t *__restrict__ strings, uint64_t nstr,
                                      const QueryDev *__restrict__ qd,
                                      unsigned long long *__restrict__ table, uint64_t cap_mask,
                                      uint64_t *__restrict__ out, uint64_t max_out,
                                      unsigned long long *__restrict__ counters) {
  const QueryDev &q = *qd;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i + 1 < T; i += stride) {
    if (tag_of(tape[i]) != '{') continue;
    uint64_t o = i, v = 0;
    for (uint32_t k = 0; k < q.path_len; k++) {
      v = find_key(tape, T, strings, nstr, o, q, k);
      if (!v) break;
      if (k + 1 < q.path_len) {
        if (tag_of(tape[v]) != '{') { v = 0; break; }
        o = v;
      }
    }
    if (!v || tag_of(tape[v]) != 'l' || v + 1 >= T) continue;
    const uint64_t val = tape[v + 1];
    if (val == kEmpty) {  // the value -1
      if (atomicExch(&counters[2], 1ull) == 0) {
        const unsigned long long at = atomicAdd(&counters[0], 1ull);
        if (at < max_out) out[at] = val;
      }
      continue;
    }
    uint64_t h = mix64(val) & cap_mask;
    for (uint64_t probe = 0; probe <= cap_mask; probe++) {
      const unsigned long long prev = atomicCAS(&table[h], kEmpty, (unsigned long long)val);
      if (prev == kEmpty) {
        const unsigned long long at = atomicAdd(&counters[0], 1ull);
        if (at < max_out) out[at] = val;
        break;
      }
      if (prev == val) break;
      h = (h + 1) & cap_mask;
      if (probe == cap_mask) atomicExch(&counters[1], 1ull);  // table full
    }
  }
}

}  // namespace sj

struct sj_query {
  uint64_t max_values = 0, cap = 0;
  unsigned long long *d_table = nullptr;
  uint64_t *d_out = nullptr;
  unsigned long long *d_counters = nullptr;  // [0] distinct values, [1] table full, [2] saw -1
  sj::QueryDev *d_q = nullptr;
  sj::QueryDev *h_q = nullptr;
  unsigned long long *h_counters = nullptr;
  int grid = 0;
};

extern "C" void sj_query_destroy(sj_query *q) {
  if (!q) return;
  void *dev[] = {q->d_table, q->d_out, q->d_counters, q->d_q};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (q->h_q) cudaFreeHost(q->h_q);
  if (q->h_counters) cudaFreeHost(q->h_counters);
  delete q;
}

extern "C" sj_status sj_query_create(sj_query **out, uint64_t max_values) {
  if (!out || max_values == 0) return SJ_INVALID_ARG;
  *out = nullptr;
  sj_query *q = new (std::nothrow) sj_query();
  if (!q) return SJ_MEMALLOC;
  q->max_values = max_values;
  q->cap = 1024;
  while (q->cap < 2 * max_values) q->cap <<= 1;
  int sms = 0, dev = 0;
  bool ok = cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaMalloc((void **)&q->d_table, q->cap * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc((void **)&q->d_out, max_values * sizeof(uint64_t)) == cudaSuccess &&
            cudaMalloc((void **)&q->d_counters, 4 * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc((void **)&q->d_q, sizeof(sj::QueryDev)) == cudaSuccess &&
            cudaMallocHost((void **)&q->h_q, sizeof(sj::QueryDev)) == cudaSuccess &&
            cudaMallocHost((void **)&q->h_counters, 4 * sizeof(unsigned long long)) == cudaSuccess;
  if (!ok) {
    sj_query_destroy(q);
    return SJ_MEMALLOC;
  }
  q->grid = sms * 8;
  *out = q;
  return SJ_SUCCESS;
}

extern "C" sj_status sj_query_distinct(sj_query *q, const uint64_t *d_tape, uint64_t tape_words,
                                       const uint8_t *d_strings, uint64_t string_bytes,
                                       const char *const *path,
                                       uint32_t path_len, void *stream, uint64_t *n_values,
                                       const uint64_t **d_values) {
  if (!q || !d_tape || !d_strings || !path || path_len == 0 || path_len > sj::kMaxPath ||
      !n_values)
    return SJ_INVALID_ARG;
  sj::QueryDev &h = *q->h_q;
  h.path_len = path_len;
  uint32_t at = 0;
  for (uint32_t k = 0; k < path_len; k++) {
    if (!path[k]) return SJ_INVALID_ARG;
    const size_t n = strlen(path[k]);
    if (at + n > sj::kMaxPathBytes) return SJ_INVALID_ARG;
    h.key_off[k] = at;
    memcpy(h.key_bytes + at, path[k], n);
    at += (uint32_t)n;
  }
  h.key_off[path_len] = at;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(q->d_q, q->h_q, sizeof(sj::QueryDev), cudaMemcpyHostToDevice, s) ||
      cudaMemsetAsync(q->d_table, 0xFF, q->cap * sizeof(unsigned long long), s) ||
      cudaMemsetAsync(q->d_counters, 0, 4 * sizeof(unsigned long long), s))
    return SJ_INTERNAL;
  sj::query_distinct_kernel<<<q->grid, 256, 0, s>>>(d_tape, tape_words, d_strings, string_bytes,
                                                    q->d_q,
                                                    q->d_table, q->cap - 1, q->d_out,
                                                    q->max_values, q->d_counters);
  if (cudaMemcpyAsync(q->h_counters, q->d_counters, 4 * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost, s) ||
      cudaStreamSynchronize(s))
    return SJ_INTERNAL;
  if (q->h_counters[1] || q->h_counters[0] > q->max_values) return SJ_CAPACITY;
  *n_values = q->h_counters[0];
  if (d_values) *d_values = q->d_out;
  return SJ_SUCCESS;
}
