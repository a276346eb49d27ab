// server.cpp -- a continuous-batching parse server over the parser calls of
// sj.h (host code; every parse runs in the library's CUDA kernels).
//
// Requests are queued as they arrive.  Each slot owns a parser (its device
// buffers hold the results), a stream and a pinned staging buffer.  Whenever a
// slot is free and requests are waiting, the waiting requests (in arrival
// order, up to the slot's byte and document capacity) are packed into one
// batch and launched on that slot's stream, so batches of several slots run
// on the GPU at the same time.  A finished batch's results stay on the device
// until the caller releases every document of it; only then is the slot free
// again.  The number of slots is set by the device-memory budget: slots are
// created while the next one still fits.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <algorithm>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "sj.h"

namespace {

// Small batches (the common case at moderate load) run on a second, small
// parser of the slot: a parser of at most 512 tiles runs 10 launches per batch
// instead of 18 (one-block tile scans) and splits each tile in four for stage
// 2, so that a batch of a few small documents keeps more warps busy.
constexpr uint64_t kSmallBatchBytes = 768ull << 10;
constexpr uint32_t kSmallBatchDocs = 64;

struct Slot {
  sj_parser *p = nullptr;
  sj_parser *ps = nullptr;    // the small parser (none when p is no larger)
  sj_parser *used = nullptr;  // the parser of the batch in flight or held
  cudaStream_t stream = nullptr;
  uint8_t *h_stage = nullptr;  // pinned: the batch's bytes, copied to the device by the parser
  std::vector<uint64_t> offsets;
  std::vector<uint64_t> tickets;
  std::vector<sj_doc_result> results;
  const uint32_t *idx = nullptr;
  const uint64_t *tape = nullptr;
  const uint8_t *strs = nullptr;
  enum State { kFree, kRunning, kHeld } state = kFree;
  uint32_t unreleased = 0;
};

struct Pending {
  uint64_t ticket;
  const uint8_t *bytes;
  uint64_t len;
};

double now_s() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

}  // namespace

struct sj_server {
  sj_server_config cfg{};
  std::vector<Slot> slots;
  std::deque<Pending> queue;
  std::unordered_map<uint64_t, uint32_t> held;  // ticket -> slot of its result
  std::deque<sj_completion> ready;
  uint64_t next_ticket = 0;
  uint64_t device_bytes = 0;
  uint64_t batches = 0;
};

static void destroy_slot(Slot &s) {
  if (s.p) sj_parser_destroy(s.p);
  if (s.ps) sj_parser_destroy(s.ps);
  if (s.stream) cudaStreamDestroy(s.stream);
  if (s.h_stage) cudaFreeHost(s.h_stage);
  s = Slot{};
}

extern "C" void sj_server_destroy(sj_server *s) {
  if (!s) return;
  for (Slot &sl : s->slots) destroy_slot(sl);  // a parser waits for its queued run
  delete s;
}

extern "C" sj_status sj_server_create(sj_server **out, const sj_server_config *cfg) {
  if (!out || !cfg || cfg->max_batch_bytes == 0 || cfg->max_slots == 0) return SJ_INVALID_ARG;
  *out = nullptr;
  sj_server *s = new (std::nothrow) sj_server();
  if (!s) return SJ_MEMALLOC;
  s->cfg = *cfg;
  if (s->cfg.max_batch_docs == 0) s->cfg.max_batch_docs = 1;
  for (uint32_t i = 0; i < s->cfg.max_slots; i++) {
    Slot sl;
    int r = sj_parser_create(&sl.p, s->cfg.max_batch_bytes, s->cfg.max_batch_docs,
                             s->cfg.max_depth);
    if (r) {
      if (i == 0) {
        sj_server_destroy(s);
        return r;
      }
      break;
    }
    if (!r && (s->cfg.max_batch_bytes > kSmallBatchBytes || s->cfg.max_batch_docs > kSmallBatchDocs))
      r = sj_parser_create(&sl.ps, std::min(s->cfg.max_batch_bytes, kSmallBatchBytes),
                           std::min(s->cfg.max_batch_docs, kSmallBatchDocs), s->cfg.max_depth);
    if (r) {
      destroy_slot(sl);
      if (i == 0) {
        sj_server_destroy(s);
        return r;
      }
      break;
    }
    const uint64_t need = sj_parser_device_bytes(sl.p) + (sl.ps ? sj_parser_device_bytes(sl.ps) : 0);
    if (s->cfg.mem_budget && s->device_bytes + need > s->cfg.mem_budget) {
      destroy_slot(sl);
      if (i == 0) {
        sj_server_destroy(s);
        return SJ_CAPACITY;
      }
      break;
    }
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost((void **)&sl.h_stage, (size_t)s->cfg.max_batch_bytes) != cudaSuccess) {
      destroy_slot(sl);
      sj_server_destroy(s);
      return SJ_MEMALLOC;
    }
    // every batch size's run captured now, not on the first batch of that size
    // while requests wait
    if ((r = sj_parser_prepare(sl.p, s->cfg.max_batch_docs)) ||
        (sl.ps && (r = sj_parser_prepare(sl.ps, std::min(s->cfg.max_batch_docs, kSmallBatchDocs))))) {
      destroy_slot(sl);
      sj_server_destroy(s);
      return r;
    }
    sl.offsets.reserve((size_t)s->cfg.max_batch_docs + 1);
    sl.tickets.reserve(s->cfg.max_batch_docs);
    sl.results.resize(s->cfg.max_batch_docs);
    s->device_bytes += need;
    s->slots.push_back(std::move(sl));
  }
  *out = s;
  return SJ_SUCCESS;
}

extern "C" uint32_t sj_server_slots(const sj_server *s) { return s ? (uint32_t)s->slots.size() : 0; }
extern "C" uint64_t sj_server_device_bytes(const sj_server *s) { return s ? s->device_bytes : 0; }
extern "C" uint64_t sj_server_batches(const sj_server *s) { return s ? s->batches : 0; }

extern "C" sj_status sj_server_submit(sj_server *s, const uint8_t *bytes, uint64_t len,
                                      uint64_t *ticket) {
  if (!s || !ticket || (!bytes && len)) return SJ_INVALID_ARG;
  if (len > s->cfg.max_batch_bytes) return SJ_CAPACITY;
  *ticket = s->next_ticket++;
  s->queue.push_back(Pending{*ticket, bytes, len});
  return SJ_SUCCESS;
}

// Pack waiting requests into free slots and launch them.
static int launch_batches(sj_server *s) {
  for (uint32_t k = 0; k < s->slots.size() && !s->queue.empty(); k++) {
    Slot &sl = s->slots[k];
    if (sl.state != Slot::kFree) continue;
    sl.offsets.clear();
    sl.tickets.clear();
    sl.offsets.push_back(0);
    uint64_t total = 0;
    while (!s->queue.empty() && sl.tickets.size() < s->cfg.max_batch_docs &&
           total + s->queue.front().len <= s->cfg.max_batch_bytes) {
      const Pending &q = s->queue.front();
      if (q.len) memcpy(sl.h_stage + total, q.bytes, (size_t)q.len);
      total += q.len;
      sl.offsets.push_back(total);
      sl.tickets.push_back(q.ticket);
      s->queue.pop_front();
    }
    const bool small = sl.ps && total <= kSmallBatchBytes && sl.tickets.size() <= kSmallBatchDocs;
    sl.used = small ? sl.ps : sl.p;
    const int r = sj_parse_batch_async(sl.used, sl.h_stage, sl.offsets.data(),
                                       (uint32_t)sl.tickets.size(), sl.stream);
    if (r) return r;
    sl.state = Slot::kRunning;
    s->batches++;
  }
  return SJ_SUCCESS;
}

// Move finished batches' results to the ready list.
static int collect(sj_server *s) {
  for (uint32_t k = 0; k < s->slots.size(); k++) {
    Slot &sl = s->slots[k];
    if (sl.state != Slot::kRunning) continue;
    const int q = sj_parse_query(sl.used);
    if (q < 0) return -q;
    if (q == 0) continue;
    const int r = sj_parse_batch_wait(sl.used, sl.results.data(), &sl.idx, &sl.tape, &sl.strs);
    if (r) return r;
    const uint32_t n = (uint32_t)sl.tickets.size();
    for (uint32_t i = 0; i < n; i++) {
      const sj_doc_result &d = sl.results[i];
      sj_completion c;
      c.ticket = sl.tickets[i];
      c.error = d.error;
      c.slot = k;
      c.n_indices = d.n_indices;
      c.tape_words = d.tape_words;
      c.string_bytes = d.string_bytes;
      c.indices = sl.idx + d.indices_offset;
      c.tape = sl.tape + d.tape_offset;
      c.strings = sl.strs + d.strings_offset;
      s->ready.push_back(c);
      s->held[c.ticket] = k;
    }
    sl.unreleased = n;
    sl.state = n ? Slot::kHeld : Slot::kFree;
  }
  return SJ_SUCCESS;
}

extern "C" int sj_server_poll(sj_server *s, sj_completion *out, uint32_t max) {
  if (!s || (!out && max)) return -SJ_INVALID_ARG;
  int r;
  if ((r = collect(s))) return -r;
  if ((r = launch_batches(s))) return -r;
  uint32_t n = 0;
  while (n < max && !s->ready.empty()) {
    out[n++] = s->ready.front();
    s->ready.pop_front();
  }
  return (int)n;
}

extern "C" sj_status sj_server_release(sj_server *s, uint64_t ticket) {
  if (!s) return SJ_INVALID_ARG;
  auto it = s->held.find(ticket);
  if (it == s->held.end()) return SJ_INVALID_ARG;
  Slot &sl = s->slots[it->second];
  s->held.erase(it);
  if (sl.unreleased && --sl.unreleased == 0) sl.state = Slot::kFree;
  return SJ_SUCCESS;
}

extern "C" sj_status sj_server_replay(sj_server *s, const uint8_t *bytes, const uint64_t *offsets,
                                      const double *arrival_s, uint32_t n, double *latency_s,
                                      double *wall_s) {
  if (!s || !offsets || !arrival_s || !latency_s || (!bytes && n)) return SJ_INVALID_ARG;
  const uint64_t first = s->next_ticket;
  std::vector<sj_completion> comp(1024);
  const double t0 = now_s();
  uint32_t sent = 0, done = 0;
  while (done < n) {
    const double t = now_s() - t0;
    while (sent < n && arrival_s[sent] <= t) {
      uint64_t tk;
      const int r = sj_server_submit(s, bytes + offsets[sent], offsets[sent + 1] - offsets[sent], &tk);
      if (r) return r;
      sent++;
    }
    const int got = sj_server_poll(s, comp.data(), (uint32_t)comp.size());
    if (got < 0) return -got;
    if (got == 0) continue;
    const double tr = now_s() - t0;
    for (int i = 0; i < got; i++) {
      const uint64_t idx = comp[i].ticket - first;
      if (idx < n) latency_s[idx] = tr - arrival_s[idx];
      const int r = sj_server_release(s, comp[i].ticket);
      if (r) return r;
      done++;
    }
  }
  if (wall_s) *wall_s = now_s() - t0;
  return SJ_SUCCESS;
}
