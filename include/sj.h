/*
 * sj.h -- C ABI of a GB300 (sm_103a) implementation of the two-stage
 * validating JSON parser of "Parsing Gigabytes of JSON per Second"
 * (G. Langdale, D. Lemire).
 *
 * The problem statement (Sec. 3): bytes in; a tape of 64-bit words, a string
 * buffer and an error code out; the input is never modified.  Stage 1 (Sec.
 * 3.1) validates UTF-8 and flattens the structural and pseudo-structural
 * characters into a u32 index array; stage 2 (Sec. 3.2) builds the tape.
 *
 * Conventions shared by every call
 *  - All compute runs in CUDA kernels on the current device; there is no CPU
 *    fallback.  A call returns an sj_status (below).  A document's own parse
 *    result (valid or which error) is reported separately, in sj_result.error
 *    or sj_doc_result.error, as an sj_error code.
 *  - Input bytes may live in host or device memory (detected with
 *    cudaPointerGetAttributes).  They are read-only and need neither padding
 *    nor alignment.  Host input is first copied into a parser-owned device
 *    buffer; device input is read in place.
 *  - Outputs live in parser-owned device buffers and stay valid until the next
 *    call on the same parser.  The caller never frees them.
 *  - A parser is not thread-safe; use one parser per host thread.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).
 *  - No C++ exception, abort or exit crosses this boundary.
 *
 * Output layout (Sec. 3, Fig. "jsontape"; Sec. 3.2.2)
 *  - indices: u32 byte positions (relative to the document start) of the
 *    structural and pseudo-structural characters, ascending.
 *  - tape: u64 words, tag in bits 56..63 and a 56-bit payload.  Word 0 is
 *    'r' with payload T-1, word T-1 is 'r' with payload 0.  '{'/'[' carry one
 *    plus the index of the matching closer, '}'/']' the index of the opener.
 *    '"' carries the byte offset of the string in the string buffer.  'l' and
 *    'd' are followed by one word: a two's-complement int64, or the binary64
 *    bits of a correctly rounded double.  't', 'f', 'n' have payload 0.
 *  - strings: per string, in tape order, a u32 little-endian length, the
 *    UTF-8 bytes (escapes resolved, may contain NUL), and one NUL byte.
 */
#ifndef SJ_H
#define SJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Per-document parse result.  Names follow the paper's examples
 * (STRING_ERROR, NUMBER_ERROR, UTF8_ERROR, Sec. 3); the paper leaves the rest
 * of the set open ("etc."), this is the full set used here.  When several
 * problems exist the reported one is, in order: CAPACITY / EMPTY, UTF8_ERROR
 * (whole input, Sec. 3.1.5), UNCLOSED_STRING (end of stage 1), then the first
 * failing token in document order, with the grammar checked before the
 * token's content. */
typedef enum {
  SJ_SUCCESS = 0,
  SJ_CAPACITY = 1,         /* document too large (more than 2^32 - 256 bytes, or above max_bytes) */
  SJ_MEMALLOC = 2,
  SJ_TAPE_ERROR = 3,       /* grammar: misplaced token, unbalanced brackets, trailing content */
  SJ_DEPTH_ERROR = 4,      /* nesting deeper than max_depth */
  SJ_STRING_ERROR = 5,     /* bad escape or lone UTF-16 surrogate */
  SJ_T_ATOM_ERROR = 6,
  SJ_F_ATOM_ERROR = 7,
  SJ_N_ATOM_ERROR = 8,
  SJ_NUMBER_ERROR = 9,     /* grammar, int64 range, or a double that overflows */
  SJ_UTF8_ERROR = 10,
  SJ_UNCLOSED_STRING = 11,
  SJ_UNESCAPED_CHARS = 12, /* raw byte < 0x20 inside a string */
  SJ_EMPTY = 13,           /* no byte other than white space */
  SJ_INVALID_ARG = 14,
  SJ_INTERNAL = 15         /* a bounded wait gave up; should not happen */
} sj_error;

/* Status of a call (as opposed to the document result): SJ_SUCCESS,
 * SJ_INVALID_ARG, SJ_CAPACITY (input larger than the parser was created for),
 * SJ_MEMALLOC (a CUDA allocation failed) or SJ_INTERNAL (a CUDA runtime error;
 * sj_last_cuda_error() tells which). */
typedef int sj_status;

typedef struct sj_parser sj_parser;

/* Result of sj_parse.  Pointers are device pointers into parser-owned memory. */
typedef struct {
  int32_t error;            /* sj_error of the document */
  uint32_t reserved;
  uint64_t n_indices;       /* valid unless error is UTF8_ERROR, CAPACITY or EMPTY */
  uint64_t tape_words;      /* valid when error == SJ_SUCCESS */
  uint64_t string_bytes;    /* valid when error == SJ_SUCCESS */
  const uint32_t *indices;
  const uint64_t *tape;
  const uint8_t *strings;
} sj_result;

/* Per-document result of sj_parse_batch (host array, one per document).
 * Offsets are element offsets into the batch's indices / tape / strings
 * arrays; payloads inside a document's tape are relative to its own strings. */
typedef struct {
  int32_t error;
  uint32_t reserved;
  uint64_t n_indices;
  uint64_t tape_words;
  uint64_t string_bytes;
  uint64_t indices_offset;
  uint64_t tape_offset;
  uint64_t strings_offset;
} sj_doc_result;

/* Create a parser for inputs of at most max_bytes bytes in total (summed over
 * a batch) and at most max_docs documents per batch (0 = 1).  max_depth is
 * the nesting limit (0 = 4096; at most 4096); the root container has depth 1.
 * Allocates all device memory up front (about 45 bytes per input byte, 53
 * for a parser of at most 4 MiB, plus about 35 MB of per-warp tables;
 * sj_parser_device_bytes tells the total).
 * Returns SJ_SUCCESS and *out, or an error status and *out = NULL. */
sj_status sj_parser_create(sj_parser **out, uint64_t max_bytes, uint32_t max_docs,
                           uint32_t max_depth);

/* Free a parser and all its device memory.  NULL is ignored. */
void sj_parser_destroy(sj_parser *p);

/* Parse one document of len bytes and wait for it (stream-synchronous).
 * The paper's sj_parse(bytes, len): fills *out and returns SJ_SUCCESS, or an
 * error status (then *out is untouched). */
sj_status sj_parse(sj_parser *p, const uint8_t *bytes, uint64_t len, void *stream,
                   sj_result *out);

/* As sj_parse but does not wait: the kernels and a copy of the small result
 * header are queued on `stream`; call sj_parse_wait() before reading *out. */
sj_status sj_parse_async(sj_parser *p, const uint8_t *bytes, uint64_t len, void *stream);
sj_status sj_parse_wait(sj_parser *p, sj_result *out);

/* Parse n_docs independent documents in one graph-launched set of kernels.
 * Document i is bytes[doc_offsets[i] .. doc_offsets[i+1]); doc_offsets is a
 * host array of n_docs+1 non-decreasing values.  Carries reset at every
 * document start.  out is a host array of n_docs results.  The three device
 * pointers give the batch output arrays (may be NULL).  Synchronous. */
sj_status sj_parse_batch(sj_parser *p, const uint8_t *bytes, const uint64_t *doc_offsets,
                         uint32_t n_docs, void *stream, sj_doc_result *out,
                         const uint32_t **indices, const uint64_t **tape,
                         const uint8_t **strings);

/* sj_parse_batch in two halves.  sj_parse_batch_async queues the run on
 * `stream` and returns; host `bytes` should be pinned (cudaMallocHost) for the
 * copy to be asynchronous, and must stay unchanged until the run has finished.
 * sj_parse_query returns 1 when the queued run has finished (or none is
 * queued), 0 while it runs, and -status on a CUDA error.  sj_parse_batch_wait
 * waits for the run and fills the outputs as sj_parse_batch does. */
sj_status sj_parse_batch_async(sj_parser *p, const uint8_t *bytes, const uint64_t *doc_offsets,
                               uint32_t n_docs, void *stream);
int sj_parse_query(sj_parser *p);
sj_status sj_parse_batch_wait(sj_parser *p, sj_doc_result *out, const uint32_t **indices,
                              const uint64_t **tape, const uint8_t **strings);

/* Device memory held by a parser, in bytes. */
uint64_t sj_parser_device_bytes(const sj_parser *p);

/* ---- Serving: continuous batching ----------------------------------------
 * The paper parses one document per call; a server parses a stream of
 * requests.  Requests are queued in arrival order; whenever one of the
 * server's slots is free, the waiting requests (up to max_batch_bytes and
 * max_batch_docs) form one batch, launched on that slot's own stream, so
 * several batches are on the GPU at once.  Results stay in the slot's device
 * buffers until every document of the batch has been released.  Slots are
 * created, up to max_slots, while their device memory fits mem_budget
 * (0 = no budget).  Each slot also holds a small parser (768 KiB, 64
 * documents, counted in the budget) that runs the batches within those
 * limits with fewer launches.  Not thread-safe: one host thread drives a
 * server. */
typedef struct sj_server sj_server;
typedef struct {
  uint64_t mem_budget;       /* device bytes all slots may hold together (0 = unlimited) */
  uint64_t max_batch_bytes;  /* input bytes per batch; larger requests are refused */
  uint32_t max_batch_docs;   /* documents per batch */
  uint32_t max_slots;        /* batches in flight or held, at most */
  uint32_t max_depth;        /* as in sj_parser_create */
  uint32_t reserved;
} sj_server_config;

/* One finished request.  The pointers are device pointers to the document's
 * own indices, tape and strings (payloads relative to its strings), valid
 * until sj_server_release(ticket). */
typedef struct {
  uint64_t ticket;
  int32_t error;             /* sj_error of the document */
  uint32_t slot;
  uint64_t n_indices, tape_words, string_bytes;
  const uint32_t *indices;
  const uint64_t *tape;
  const uint8_t *strings;
} sj_completion;

sj_status sj_server_create(sj_server **out, const sj_server_config *cfg);
void sj_server_destroy(sj_server *s);
uint32_t sj_server_slots(const sj_server *s);
uint64_t sj_server_device_bytes(const sj_server *s);
uint64_t sj_server_batches(const sj_server *s);

/* Queue a request.  The bytes (host memory) are read when its batch is
 * formed, during a later sj_server_poll, and must stay valid until then.
 * Writes the request's ticket (consecutive from 0).  SJ_CAPACITY when len is
 * above max_batch_bytes. */
sj_status sj_server_submit(sj_server *s, const uint8_t *bytes, uint64_t len, uint64_t *ticket);

/* Collect finished batches, launch waiting requests on free slots, and write
 * up to max finished requests to out.  Returns their number, or -status. */
int sj_server_poll(sj_server *s, sj_completion *out, uint32_t max);

/* Give up a finished request's results. */
sj_status sj_server_release(sj_server *s, uint64_t ticket);

/* Replay an arrival trace: request i (bytes[offsets[i] .. offsets[i+1]),
 * host memory) is submitted once arrival_s[i] seconds have passed since the
 * call started (arrival_s non-decreasing); every result is released as soon
 * as it is seen.  latency_s[i] = the time its result was seen minus
 * arrival_s[i]; *wall_s = the time until the last result. */
sj_status sj_server_replay(sj_server *s, const uint8_t *bytes, const uint64_t *offsets,
                           const double *arrival_s, uint32_t n, double *latency_s,
                           double *wall_s);

/* Per-kernel timing.  With profiling on, runs launch their kernels directly
 * (not through the captured graph) with CUDA events recorded between them on
 * the caller's stream.  sj_parser_stage_times waits for the last run and
 * writes, in milliseconds, the durations of its 9 stages to ms[0..8]: setup,
 * stage-1 blocks, stage-1 tile scan, stage-1 flatten, stage-2 reduce, stage-2
 * tile scan and frontier, stage-2 numbers, stage-2 build, finalize.  n must be
 * at least 9. */
sj_status sj_parser_set_profiling(sj_parser *p, int enable);
sj_status sj_parser_stage_times(sj_parser *p, float *ms, int n);

/* Number of kernel launches in one run of this parser (over resident input,
 * or host input that is not chunked). */
int sj_parser_kernels_per_run(const sj_parser *p);

/* Capture now the runs (CUDA graphs) of every batch size up to max_docs
 * documents (0 = the parser's max_docs), which are otherwise captured on the
 * first run of each size (one graph per power-of-two bucket of document
 * counts).  A server calls it once per parser so that no capture happens
 * while requests wait. */
sj_status sj_parser_prepare(sj_parser *p, uint32_t max_docs);

/* Host documents that arrive in chunks.  A single document in pinned host
 * memory (cudaMallocHost / cudaHostRegister) longer than chunk_bytes is
 * parsed while it is copied: a second stream copies it chunk by chunk, and
 * the run's stream runs stage 1 on each chunk once it has landed and stage 2
 * on every tile whose tokens end in bytes that have landed (Sec. 3 notes that
 * the two stages can be interleaved over a stream of chunks).  Results are
 * identical to a parse of the same bytes in device memory.  chunk_bytes is
 * the largest chunk, rounded up to a multiple of 2048: the first chunk is
 * 1/16 of it and each next one 7/4 of the one before, up to it (the host link
 * copies about 1.75 times as fast as the kernels parse); at most 64 chunks, the last
 * taking what remains.  0 turns chunking off (stage 1 then reads the pinned
 * document over the host link itself); the default is 512 MiB.  Such runs
 * launch their kernels directly (no graph; about 20 launches per chunk) and
 * are not profiled: with profiling on, the document is not chunked. */
sj_status sj_parser_set_host_chunk(sj_parser *p, uint64_t chunk_bytes);

/* Launch shapes.  The four main kernels (stage-1 blocks, stage-1 flatten,
 * stage-2 reduce, stage-2 build) loop over tiles, so any grid covers any
 * input; the shape is the number of resident blocks per SM, from 1 to the
 * kernel's occupancy limit (max_blocks_per_sm, may be NULL).  A parser starts
 * with every kernel at its limit.  sj_parser_set_launch drops the captured
 * graphs (the next run captures again).  The paper has no counterpart: its
 * single-threaded parser has no launch shape. */
sj_status sj_parser_get_launch(const sj_parser *p, uint32_t *blocks_per_sm,
                               uint32_t *max_blocks_per_sm);
sj_status sj_parser_set_launch(sj_parser *p, const uint32_t *blocks_per_sm);

/* Autotuner: parses the sample (bytes, len; host or device) to time each of
 * the four main kernels at every allowed shape, one kernel at a time (reps
 * timed runs each, after one warm-up), keeps the fastest and writes the
 * choice and its kernel time (ms) to blocks_per_sm[4] / best_ms[4] (either may
 * be NULL).  Leaves profiling as it was.  Synchronous on `stream`. */
sj_status sj_parser_autotune(sj_parser *p, const uint8_t *bytes, uint64_t len, void *stream,
                             int reps, uint32_t *blocks_per_sm, float *best_ms);

/* Stage 1 only (structural indices) of one document, allocating nothing.
 * The paper has no counterpart: this entry exists for callers that cannot call
 * cudaMalloc when they parse (device memory owned by another allocator, or a
 * thread that must not trigger cudaMalloc's implicit synchronisation).  The
 * caller passes device buffers: d_bytes (len bytes, read-only), d_indices
 * (room for len u32 positions) and d_result (2 u32: the index count, then
 * flags 1 = invalid UTF-8, 2 = unclosed string, 4 = internal).  The kernel's
 * scratch is one static device array sized for len <= 64 MiB, held by every GPU
 * that loads the library until exit; larger inputs return SJ_CAPACITY.  The
 * first call on a device looks up that array's device address (set-up); make
 * it before any stream capture.  Calls share the array: calls that overlap on
 * the GPU race and must be serialised.  Queued on `stream`, not waited for. */
sj_status sj_stage1_indices_noalloc(const uint8_t *d_bytes, uint64_t len, uint32_t *d_indices,
                                    uint32_t *d_result, void *stream);

/* ---- Tape query ------------------------------------------------------------
 * Distinct integer values at a key path, e.g. {"user", "id"} -- the paper's
 * example query over a parsed document (Sec. 4.5, Table "tab:userid").  The
 * path may start at any object of the document; a value counts when every key
 * but the last names an object and the last names an int64 ('l').  The tape
 * and strings are a document's device outputs of a successful parse
 * (tape_words, string_bytes from its result); any other tape is read without
 * faults but gives no meaningful answer.  A query object owns a device hash
 * set for up to max_values distinct values (SJ_CAPACITY beyond).  The
 * values, in no particular order, stay in device memory owned by the query
 * until its next call.  Synchronous on `stream`. */
typedef struct sj_query sj_query;
sj_status sj_query_create(sj_query **out, uint64_t max_values);
void sj_query_destroy(sj_query *q);
sj_status sj_query_distinct(sj_query *q, const uint64_t *d_tape, uint64_t tape_words,
                            const uint8_t *d_strings, uint64_t string_bytes,
                            const char *const *path, uint32_t path_len, void *stream,
                            uint64_t *n_values, const uint64_t **d_values);

/* Name of an sj_error code ("SUCCESS", "TAPE_ERROR", ...). */
const char *sj_error_name(int code);

/* Last CUDA runtime error code seen by the library on this thread (0 = none). */
int sj_last_cuda_error(void);

/* Library version string. */
const char *sj_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SJ_H */
