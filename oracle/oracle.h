/*
 * oracle.h -- plain, slow, obviously-correct CPU reference for the two-stage
 * JSON parser of "Parsing Gigabytes of JSON per Second" (Langdale & Lemire).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this code.  It shares no
 * code, header, table or helper with the CUDA library; neither includes or
 * links the other.
 *
 * What it computes (each function cites the passage it follows):
 *   sjo_utf8_valid   -- UTF-8 well-formedness, Sec. 3.1.5, Table "tab:unicode".
 *   sjo_classify     -- byte classes of Sec. 3.1.2 (Table "tab:vectable",
 *                       right-hand side): the plain definition, no nibble tables.
 *   sjo_stage1       -- the structural + pseudo-structural index set of
 *                       Sec. 3.1.1-3.1.4 (Figs. "identifyescapedquotes",
 *                       "identifyquoteregion", "identifypseudo"), restated as a
 *                       byte-at-a-time scan, plus the unclosed-string flag.
 *   sjo_parse        -- the whole validating parse (Sec. 3 and 3.2): a plain
 *                       recursive descent over the bytes (RFC 8259 as the paper
 *                       restates it), building the tape of Sec. 3 / Fig.
 *                       "jsontape" and the string buffer of Sec. 3.2.2.
 *
 * Parity pins: see tests/test_oracle_*.py (paper worked examples, brute force
 * against Python's json and utf-8 codecs, invariants).  The error *category*
 * chosen among several wrong-document codes is pinned only by hand-written
 * cases ("parity unpinned" beyond them).
 */
#ifndef SJ_ORACLE_H
#define SJ_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes; the numbering is the public one of include/sj.h, restated
 * here so that the oracle does not include the library header. */
enum {
  SJO_SUCCESS = 0, SJO_CAPACITY = 1, SJO_MEMALLOC = 2, SJO_TAPE_ERROR = 3,
  SJO_DEPTH_ERROR = 4, SJO_STRING_ERROR = 5, SJO_T_ATOM_ERROR = 6,
  SJO_F_ATOM_ERROR = 7, SJO_N_ATOM_ERROR = 8, SJO_NUMBER_ERROR = 9,
  SJO_UTF8_ERROR = 10, SJO_UNCLOSED_STRING = 11, SJO_UNESCAPED_CHARS = 12,
  SJO_EMPTY = 13, SJO_INVALID_ARG = 14, SJO_INTERNAL = 15
};

typedef struct {
  int32_t  error;
  uint32_t pad_;
  uint64_t n_indices;     /* stage-1 index count (valid unless UTF8/CAPACITY/EMPTY) */
  uint64_t tape_words;    /* valid on SUCCESS */
  uint64_t string_bytes;  /* valid on SUCCESS */
  uint64_t n_tokens;      /* token starts seen by the descent (for the O2 cross-check) */
} sjo_result;

/* 1 if buf[0..len) is well-formed UTF-8 (Table "tab:unicode"), else 0. */
int sjo_utf8_valid(const uint8_t *buf, uint64_t len);

/* Validate n fixed-width records of width w packed in buf; ok[i] = validity
 * of record i.  A convenience loop over sjo_utf8_valid for exhaustive tests. */
void sjo_utf8_valid_many(const uint8_t *buf, uint64_t n, uint32_t w, uint8_t *ok);

/* Class bits of one byte: 1 ',' 2 ':' 4 '[]{}' 8 '\t\n\r' 16 ' ' (Sec. 3.1.2). */
int sjo_classify(uint8_t c);

/* Stage-1 index set of buf (Sec. 3.1).  Writes at most cap positions into idx,
 * sets *n to the full count and *unclosed to the final in-string state.
 * Returns 0, or 1 if cap was too small. */
int sjo_stage1(const uint8_t *buf, uint64_t len, uint32_t *idx, uint64_t cap,
               uint64_t *n, int *unclosed);

/* Run sjo_stage1 over n fixed-width records (width w) and write, per record,
 * a w-byte 0/1 mask of indexed positions and the unclosed flag. */
void sjo_stage1_many(const uint8_t *buf, uint64_t n, uint32_t w,
                     uint8_t *mask, uint8_t *unclosed);

/* Full validating parse.  Capacities: idx >= len, tape >= len + 3 words,
 * strings >= 3*len + 8 bytes, tokens >= len (or tokens == NULL).
 * max_depth == 0 means 4096.  Returns res->error. */
int sjo_parse(const uint8_t *buf, uint64_t len, uint32_t max_depth,
              uint32_t *idx, uint64_t idx_cap,
              uint64_t *tape, uint64_t tape_cap,
              uint8_t *strings, uint64_t strings_cap,
              uint32_t *tokens, uint64_t tokens_cap,
              sjo_result *res);

/* Parse n documents (concatenated, offsets[n+1]) one after the other, only
 * the error codes are kept.  Used for exhaustive accept/reject tests and for
 * the batched CPU baseline. */
void sjo_parse_many_errors(const uint8_t *buf, const uint64_t *offsets,
                           uint64_t n, uint32_t max_depth, int32_t *errors);

#ifdef __cplusplus
}
#endif
#endif
