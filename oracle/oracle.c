/*
 * oracle.c -- plain CPU reference of the validating two-stage JSON parse of
 * "Parsing Gigabytes of JSON per Second" (Langdale & Lemire).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Deliberately simple: byte at a
 * time, no SIMD, no tables beyond the plain definitions, no code shared with
 * the CUDA library.
 *
 * Readings of the paper where it is silent (the same list is kept in the
 * design notes of the repository):
 *  - byte -1 is a virtual white-space byte: a root atom at byte 0 is indexed;
 *  - the backslash-run parity is counted over all bytes, in or out of strings
 *    (Fig. "identifyescapedquotes" is applied to every byte);
 *  - opening quotes are indexed, closing quotes are not (Fig. "identifypseudo",
 *    last line);
 *  - an atom or number must be followed by white space, one of ",:[]{}" or the
 *    end of the input;
 *  - integers outside [-2^63, 2^63) are errors (Sec. 3, stage 2), there is no
 *    fallback to a double; "-0" is the integer 0;
 *  - doubles are correctly rounded (round to nearest, ties to even); an
 *    infinite result is an error, underflow to a subnormal or zero is not;
 *  - lone or reversed UTF-16 surrogates in \u escapes are string errors;
 *  - strings are packed in tape order: u32 little-endian length, the bytes,
 *    one NUL; the tape payload is the byte offset of the length field;
 *  - root word 0 points at the last word (T-1), the last word points at 0;
 *  - error precedence: CAPACITY/EMPTY, UTF8, UNCLOSED_STRING, then the first
 *    failing token in document order (grammar before content at a token).
 */
#define _GNU_SOURCE
#include "oracle.h"

#include <errno.h>
#include <locale.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Sec. 3.1.5, Table "tab:unicode": well-formed UTF-8 byte sequences.        */
/* ------------------------------------------------------------------------ */
int sjo_utf8_valid(const uint8_t *b, uint64_t len) {
  uint64_t i = 0;
  while (i < len) {
    uint8_t c = b[i];
    uint8_t lo2 = 0x80, hi2 = 0xBF; /* allowed range of the 2nd byte */
    int need;                        /* continuation bytes after the lead */
    if (c <= 0x7F) { i += 1; continue; }
    else if (c >= 0xC2 && c <= 0xDF) need = 1;
    else if (c == 0xE0) { need = 2; lo2 = 0xA0; }
    else if ((c >= 0xE1 && c <= 0xEC) || c == 0xEE || c == 0xEF) need = 2;
    else if (c == 0xED) { need = 2; hi2 = 0x9F; }
    else if (c == 0xF0) { need = 3; lo2 = 0x90; }
    else if (c >= 0xF1 && c <= 0xF3) need = 3;
    else if (c == 0xF4) { need = 3; hi2 = 0x8F; }
    else return 0; /* 80..C1 as a lead, F5..FF */
    if (i + (uint64_t)need >= len) return 0; /* truncated at the end */
    if (b[i + 1] < lo2 || b[i + 1] > hi2) return 0;
    for (int k = 2; k <= need; k++)
      if (b[i + k] < 0x80 || b[i + k] > 0xBF) return 0;
    i += (uint64_t)need + 1;
  }
  return 1;
}

void sjo_utf8_valid_many(const uint8_t *buf, uint64_t n, uint32_t w, uint8_t *ok) {
  for (uint64_t r = 0; r < n; r++) ok[r] = (uint8_t)sjo_utf8_valid(buf + r * w, w);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1.2: the desired classes (right-hand side of Table "tab:vectable"). */
/* ------------------------------------------------------------------------ */
int sjo_classify(uint8_t c) {
  if (c == ',') return 1;
  if (c == ':') return 2;
  if (c == '[' || c == ']' || c == '{' || c == '}') return 4;
  if (c == '\t' || c == '\n' || c == '\r') return 8;
  if (c == ' ') return 16;
  return 0;
}

static int is_ws(uint8_t c) { return (sjo_classify(c) & 0x18) != 0; }
static int is_op(uint8_t c) { return (sjo_classify(c) & 0x7) != 0; }

/* ------------------------------------------------------------------------ */
/* Sec. 3.1.1-3.1.4 restated one byte at a time.                             */
/*  - a quote is a real quote iff the run of backslashes right before it has  */
/*    even length (Fig. "identifyescapedquotes");                             */
/*  - the in-string state flips at every real quote (Fig.                     */
/*    "identifyquoteregion"); the opening quote is inside, the closing one is */
/*    not;                                                                    */
/*  - outside strings, structural characters and opening quotes are indexed, */
/*    and so is every other non-white-space byte whose predecessor is        */
/*    white space, structural or a real quote (Sec. 3.1.3, Fig.              */
/*    "identifypseudo"); the predecessor of byte 0 is white space.           */
/* ------------------------------------------------------------------------ */
int sjo_stage1(const uint8_t *b, uint64_t len, uint32_t *idx, uint64_t cap,
               uint64_t *n_out, int *unclosed) {
  uint64_t n = 0;
  uint64_t bs_run = 0;   /* consecutive backslashes right before byte i */
  int in_str = 0;        /* inside a string (after an opening quote)     */
  int prev_sep = 1;      /* predecessor is white space / structural / quote */
  int overflow = 0;
  for (uint64_t i = 0; i < len; i++) {
    uint8_t c = b[i];
    int real_quote = (c == '"') && (bs_run % 2 == 0);
    int indexed = 0;
    if (in_str) {
      if (real_quote) { in_str = 0; prev_sep = 1; }  /* closing quote, not indexed */
      /* other bytes inside a string: nothing; prev_sep is irrelevant inside */
    } else {
      if (real_quote) { indexed = 1; in_str = 1; prev_sep = 1; }
      else if (is_op(c)) { indexed = 1; prev_sep = 1; }
      else if (is_ws(c)) { prev_sep = 1; }
      else { indexed = prev_sep; prev_sep = 0; }
    }
    if (indexed) {
      if (n < cap) idx[n] = (uint32_t)i; else overflow = 1;
      n++;
    }
    bs_run = (c == '\\') ? bs_run + 1 : 0;
  }
  *n_out = n;
  *unclosed = in_str;
  return overflow;
}

void sjo_stage1_many(const uint8_t *buf, uint64_t n, uint32_t w,
                     uint8_t *mask, uint8_t *unclosed) {
  uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * (w ? w : 1));
  for (uint64_t r = 0; r < n; r++) {
    uint64_t cnt = 0; int uc = 0;
    sjo_stage1(buf + r * w, w, tmp, w, &cnt, &uc);
    memset(mask + r * w, 0, w);
    for (uint64_t k = 0; k < cnt; k++) mask[r * w + tmp[k]] = 1;
    unclosed[r] = (uint8_t)uc;
  }
  free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3 / 3.2: recursive descent over the bytes, building the tape.        */
/* ------------------------------------------------------------------------ */
typedef struct {
  const uint8_t *b;
  uint64_t len, pos;
  uint32_t max_depth;
  uint64_t *tape; uint64_t tape_cap, tn;
  uint8_t *sb; uint64_t sb_cap, sn;
  uint32_t *tok; uint64_t tok_cap, ntok;
  int err;
  locale_t cloc;
} P;

#define TAG(c) ((uint64_t)(uint8_t)(c) << 56)

static void skip_ws(P *p) {
  while (p->pos < p->len && is_ws(p->b[p->pos])) p->pos++;
}

static int put_word(P *p, uint64_t w) {
  if (p->tn >= p->tape_cap) { p->err = SJO_CAPACITY; return 0; }
  p->tape[p->tn++] = w;
  return 1;
}

static void note_token(P *p) {
  if (p->tok && p->ntok < p->tok_cap) p->tok[p->ntok] = (uint32_t)p->pos;
  p->ntok++;
}

/* Terminator rule for atoms and numbers: white space, ",:[]{}", or the end. */
static int at_terminator(P *p, uint64_t q) {
  return q >= p->len || is_ws(p->b[q]) || is_op(p->b[q]);
}

static int hexval(uint8_t c) {
  if (c >= '0' && c <= '9') return c - '0';
  if (c >= 'a' && c <= 'f') return c - 'a' + 10;
  if (c >= 'A' && c <= 'F') return c - 'A' + 10;
  return -1;
}

static int read_u4(P *p, uint64_t q, uint32_t *cu) {
  /* expects the 4 hex digits at q .. q+3 */
  if (q + 4 > p->len) return 0;
  uint32_t v = 0;
  for (int k = 0; k < 4; k++) {
    int h = hexval(p->b[q + k]);
    if (h < 0) return 0;
    v = v * 16 + (uint32_t)h;
  }
  *cu = v;
  return 1;
}

static int sb_put(P *p, uint8_t c) {
  if (p->sn >= p->sb_cap) { p->err = SJO_CAPACITY; return 0; }
  p->sb[p->sn++] = c;
  return 1;
}

/* Encode one Unicode scalar value as UTF-8 (RFC 3629). */
static int sb_put_cp(P *p, uint32_t cp) {
  if (cp < 0x80) return sb_put(p, (uint8_t)cp);
  if (cp < 0x800)
    return sb_put(p, (uint8_t)(0xC0 | (cp >> 6))) && sb_put(p, (uint8_t)(0x80 | (cp & 0x3F)));
  if (cp < 0x10000)
    return sb_put(p, (uint8_t)(0xE0 | (cp >> 12))) &&
           sb_put(p, (uint8_t)(0x80 | ((cp >> 6) & 0x3F))) &&
           sb_put(p, (uint8_t)(0x80 | (cp & 0x3F)));
  return sb_put(p, (uint8_t)(0xF0 | (cp >> 18))) &&
         sb_put(p, (uint8_t)(0x80 | ((cp >> 12) & 0x3F))) &&
         sb_put(p, (uint8_t)(0x80 | ((cp >> 6) & 0x3F))) &&
         sb_put(p, (uint8_t)(0x80 | (cp & 0x3F)));
}

/* Sec. 3.2.2: validate and normalise one string; p->pos is at the opening
 * quote.  Writes the '"' tape word and the (length, bytes, NUL) record. */
static int parse_string(P *p) {
  uint64_t off = p->sn;
  if (!put_word(p, TAG('"') | off)) return 0;
  for (int k = 0; k < 4; k++) if (!sb_put(p, 0)) return 0; /* length, patched below */
  uint64_t q = p->pos + 1;
  for (;;) {
    if (q >= p->len) { p->err = SJO_UNCLOSED_STRING; return 0; }
    uint8_t c = p->b[q];
    if (c == '"') { q++; break; }
    if (c < 0x20) { p->err = SJO_UNESCAPED_CHARS; return 0; }
    if (c != '\\') { if (!sb_put(p, c)) return 0; q++; continue; }
    if (q + 1 >= p->len) { p->err = SJO_STRING_ERROR; return 0; }
    uint8_t e = p->b[q + 1];
    uint8_t out = 0;
    switch (e) {
      case '"': out = '"'; break;
      case '\\': out = '\\'; break;
      case '/': out = '/'; break;
      case 'b': out = '\b'; break;
      case 'f': out = '\f'; break;
      case 'n': out = '\n'; break;
      case 'r': out = '\r'; break;
      case 't': out = '\t'; break;
      case 'u': {
        uint32_t cu;
        if (!read_u4(p, q + 2, &cu)) { p->err = SJO_STRING_ERROR; return 0; }
        q += 6;
        if (cu >= 0xDC00 && cu <= 0xDFFF) { p->err = SJO_STRING_ERROR; return 0; }
        if (cu >= 0xD800 && cu <= 0xDBFF) {
          uint32_t lo;
          if (q + 1 >= p->len || p->b[q] != '\\' || p->b[q + 1] != 'u' ||
              !read_u4(p, q + 2, &lo) || lo < 0xDC00 || lo > 0xDFFF) {
            p->err = SJO_STRING_ERROR; return 0;
          }
          q += 6;
          cu = 0x10000 + ((cu - 0xD800) << 10) + (lo - 0xDC00);
        }
        if (!sb_put_cp(p, cu)) return 0;
        continue;
      }
      default: p->err = SJO_STRING_ERROR; return 0;
    }
    if (!sb_put(p, out)) return 0;
    q += 2;
  }
  uint64_t slen = p->sn - off - 4;
  if (slen > 0xFFFFFFFFull) { p->err = SJO_CAPACITY; return 0; }
  p->sb[off + 0] = (uint8_t)(slen);
  p->sb[off + 1] = (uint8_t)(slen >> 8);
  p->sb[off + 2] = (uint8_t)(slen >> 16);
  p->sb[off + 3] = (uint8_t)(slen >> 24);
  if (!sb_put(p, 0)) return 0;
  p->pos = q;
  return 1;
}

static int is_digit(uint8_t c) { return c >= '0' && c <= '9'; }

/* Sec. 3.2.1: RFC 8259 number grammar, int64 range, correctly rounded double. */
static int parse_number(P *p) {
  uint64_t s = p->pos, q = s;
  int neg = 0, is_int = 1;
  if (q < p->len && p->b[q] == '-') { neg = 1; q++; }
  if (q >= p->len || !is_digit(p->b[q])) { p->err = SJO_NUMBER_ERROR; return 0; }
  if (p->b[q] == '0') q++;
  else while (q < p->len && is_digit(p->b[q])) q++;
  uint64_t int_end = q;
  if (q < p->len && p->b[q] == '.') {
    is_int = 0; q++;
    if (q >= p->len || !is_digit(p->b[q])) { p->err = SJO_NUMBER_ERROR; return 0; }
    while (q < p->len && is_digit(p->b[q])) q++;
  }
  if (q < p->len && (p->b[q] == 'e' || p->b[q] == 'E')) {
    is_int = 0; q++;
    if (q < p->len && (p->b[q] == '+' || p->b[q] == '-')) q++;
    if (q >= p->len || !is_digit(p->b[q])) { p->err = SJO_NUMBER_ERROR; return 0; }
    while (q < p->len && is_digit(p->b[q])) q++;
  }
  if (!at_terminator(p, q)) { p->err = SJO_NUMBER_ERROR; return 0; }
  if (is_int) {
    /* exact magnitude with overflow detection; limit 2^63 - 1 or 2^63 */
    uint64_t mag = 0, lim = neg ? 0x8000000000000000ull : 0x7FFFFFFFFFFFFFFFull;
    for (uint64_t k = s + (uint64_t)neg; k < int_end; k++) {
      uint64_t d = (uint64_t)(p->b[k] - '0');
      if (mag > (lim - d) / 10) { p->err = SJO_NUMBER_ERROR; return 0; }
      mag = mag * 10 + d;
    }
    uint64_t v = neg ? (uint64_t)0 - mag : mag;
    if (!put_word(p, TAG('l'))) return 0;
    if (!put_word(p, v)) return 0;
  } else {
    uint64_t n = q - s;
    char small[128];
    char *lex = n < sizeof(small) ? small : (char *)malloc(n + 1);
    if (!lex) { p->err = SJO_MEMALLOC; return 0; }
    memcpy(lex, p->b + s, n);
    lex[n] = 0;
    double d = strtod_l(lex, NULL, p->cloc);
    if (lex != small) free(lex);
    if (isinf(d)) { p->err = SJO_NUMBER_ERROR; return 0; }
    uint64_t bits;
    memcpy(&bits, &d, 8);
    if (!put_word(p, TAG('d'))) return 0;
    if (!put_word(p, bits)) return 0;
  }
  p->pos = q;
  return 1;
}

static int parse_atom(P *p, const char *word, int err, char tag) {
  uint64_t n = strlen(word);
  if (p->pos + n > p->len || memcmp(p->b + p->pos, word, n) != 0 ||
      !at_terminator(p, p->pos + n)) {
    p->err = err; return 0;
  }
  if (!put_word(p, TAG(tag))) return 0;
  p->pos += n;
  return 1;
}

static int parse_value(P *p, uint32_t depth);

/* Objects and arrays (Sec. 3, stage 2): the opener word is patched once the
 * matching closer is written, with one plus the closer's tape index; the
 * closer word holds the opener's tape index (Fig. "jsontape"). */
static int parse_container(P *p, uint32_t depth, int is_obj) {
  uint8_t open = is_obj ? '{' : '[', close = is_obj ? '}' : ']';
  if (depth + 1 > p->max_depth) { p->err = SJO_DEPTH_ERROR; return 0; }
  uint64_t at = p->tn;
  if (!put_word(p, TAG(open))) return 0;
  p->pos++;
  skip_ws(p);
  if (p->pos < p->len && p->b[p->pos] == close) {
    note_token(p);
  } else {
    for (;;) {
      if (p->pos >= p->len) { p->err = SJO_TAPE_ERROR; return 0; }
      if (is_obj) {
        if (p->b[p->pos] != '"') { p->err = SJO_TAPE_ERROR; return 0; }
        note_token(p);
        if (!parse_string(p)) return 0;
        skip_ws(p);
        if (p->pos >= p->len || p->b[p->pos] != ':') { p->err = SJO_TAPE_ERROR; return 0; }
        note_token(p);
        p->pos++;
        skip_ws(p);
      }
      if (!parse_value(p, depth + 1)) return 0;
      skip_ws(p);
      if (p->pos >= p->len) { p->err = SJO_TAPE_ERROR; return 0; }
      if (p->b[p->pos] == ',') { note_token(p); p->pos++; skip_ws(p); continue; }
      if (p->b[p->pos] == close) { note_token(p); break; }
      p->err = SJO_TAPE_ERROR;
      return 0;
    }
  }
  uint64_t end = p->tn;
  if (!put_word(p, TAG(close) | at)) return 0;
  p->tape[at] = TAG(open) | (end + 1);
  p->pos++;
  return 1;
}

/* Dispatch on the first byte of a value (Sec. 3, stage 2; Sec. 3.1.3). */
static int parse_value(P *p, uint32_t depth) {
  if (p->pos >= p->len) { p->err = SJO_TAPE_ERROR; return 0; }
  uint8_t c = p->b[p->pos];
  note_token(p);
  switch (c) {
    case '{': return parse_container(p, depth, 1);
    case '[': return parse_container(p, depth, 0);
    case '"': return parse_string(p);
    case 't': return parse_atom(p, "true", SJO_T_ATOM_ERROR, 't');
    case 'f': return parse_atom(p, "false", SJO_F_ATOM_ERROR, 'f');
    case 'n': return parse_atom(p, "null", SJO_N_ATOM_ERROR, 'n');
    default:
      if (c == '-' || is_digit(c)) return parse_number(p);
      p->err = SJO_TAPE_ERROR;
      return 0;
  }
}

int sjo_parse(const uint8_t *buf, uint64_t len, uint32_t max_depth,
              uint32_t *idx, uint64_t idx_cap,
              uint64_t *tape, uint64_t tape_cap,
              uint8_t *strings, uint64_t strings_cap,
              uint32_t *tokens, uint64_t tokens_cap,
              sjo_result *res) {
  memset(res, 0, sizeof(*res));
  if (max_depth == 0) max_depth = 4096;
  /* O0: sizes.  Documents must leave room for u32 positions and tape words. */
  if (len > 0xFFFFFF00ull) { res->error = SJO_CAPACITY; return res->error; }
  uint64_t k = 0;
  while (k < len && is_ws(buf[k])) k++;
  if (k == len) { res->error = SJO_EMPTY; return res->error; }
  /* O1: UTF-8 over the whole input (Sec. 3.1.5). */
  if (!sjo_utf8_valid(buf, len)) { res->error = SJO_UTF8_ERROR; return res->error; }
  /* O2: stage-1 index set; an unclosed string is reported before stage 2. */
  uint64_t nidx = 0; int unclosed = 0;
  if (sjo_stage1(buf, len, idx, idx_cap, &nidx, &unclosed)) {
    res->error = SJO_CAPACITY; return res->error;
  }
  res->n_indices = nidx;
  if (unclosed) { res->error = SJO_UNCLOSED_STRING; return res->error; }
  /* O3: descent. */
  P p;
  memset(&p, 0, sizeof(p));
  p.b = buf; p.len = len; p.max_depth = max_depth;
  p.tape = tape; p.tape_cap = tape_cap;
  p.sb = strings; p.sb_cap = strings_cap;
  p.tok = tokens; p.tok_cap = tokens ? tokens_cap : 0;
  p.cloc = newlocale(LC_NUMERIC_MASK, "C", (locale_t)0);
  if (!p.cloc) { res->error = SJO_MEMALLOC; return res->error; }
  if (put_word(&p, TAG('r'))) {
    skip_ws(&p);
    if (parse_value(&p, 0)) {
      skip_ws(&p);
      if (p.pos != p.len) p.err = SJO_TAPE_ERROR; /* trailing content */
    }
  }
  if (!p.err && put_word(&p, TAG('r'))) {
    tape[0] = TAG('r') | (p.tn - 1);
  }
  freelocale(p.cloc);
  res->error = p.err;
  res->tape_words = p.err ? 0 : p.tn;
  res->string_bytes = p.err ? 0 : p.sn;
  res->n_tokens = p.ntok;
  return res->error;
}

void sjo_parse_many_errors(const uint8_t *buf, const uint64_t *offsets,
                           uint64_t n, uint32_t max_depth, int32_t *errors) {
  uint64_t maxlen = 0;
  for (uint64_t d = 0; d < n; d++)
    if (offsets[d + 1] - offsets[d] > maxlen) maxlen = offsets[d + 1] - offsets[d];
  uint64_t cap = maxlen + 8;
  uint32_t *idx = (uint32_t *)malloc(sizeof(uint32_t) * cap);
  uint64_t *tape = (uint64_t *)malloc(sizeof(uint64_t) * (cap + 3));
  uint8_t *sb = (uint8_t *)malloc(3 * cap + 8);
  for (uint64_t d = 0; d < n; d++) {
    sjo_result r;
    if (!idx || !tape || !sb) { errors[d] = SJO_MEMALLOC; continue; }
    sjo_parse(buf + offsets[d], offsets[d + 1] - offsets[d], max_depth, idx, cap,
              tape, cap + 3, sb, 3 * cap + 8, NULL, 0, &r);
    errors[d] = r.error;
  }
  free(idx); free(tape); free(sb);
}
