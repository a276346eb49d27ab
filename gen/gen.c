/*
 * gen.c -- seeded synthetic JSON documents shaped like the paper's workloads
 * (Sec. 4.2, Tables "tab:test-datasets" / "tab:test-datasets-size").
 *
 * Input generation only: this file holds none of the parser's arithmetic.
 * Numbers are emitted as random digit strings, never by formatting a binary
 * value.  The same generator feeds the oracle and the CUDA library.
 *
 * Random numbers: splitmix64 (Steele, Lea, Flood 2014), one stream per seed.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t s; } rng_t;

static uint64_t rnext(rng_t *r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double runif(rng_t *r) { return (double)(rnext(r) >> 11) * (1.0 / 9007199254740992.0); }
static uint64_t rbelow(rng_t *r, uint64_t n) { return n ? rnext(r) % n : 0; }
static int64_t rrange(rng_t *r, int64_t lo, int64_t hi) { /* inclusive */
  return lo + (int64_t)rbelow(r, (uint64_t)(hi - lo + 1));
}

typedef struct {
  uint8_t *b;
  uint64_t n, cap;
  int overflow;
} wbuf;

static void put(wbuf *w, uint8_t c) {
  if (w->n < w->cap) w->b[w->n] = c; else w->overflow = 1;
  w->n++;
}
static void puts_(wbuf *w, const char *s) { while (*s) put(w, (uint8_t)*s++); }

typedef struct {
  int pretty;            /* 2-space pretty printing */
  double nonascii_p;     /* per string character: probability of a non-ASCII scalar */
  double escape_p;       /* per string character: probability of an escape */
  double long_string_p;  /* per string: probability of a 64..300 character string */
  double straddle_p;     /* per string: probability of an escape run placed on a block edge */
  int str_min, str_max;  /* string length range (characters) */
  int max_nest;          /* nesting levels below a record */
  double deep_p;         /* per record: probability of a deep chain */
  int deep_levels;       /* absolute depth reached by a deep chain */
} recopt;

static void newline(wbuf *w, const recopt *o, int level) {
  if (!o->pretty) return;
  put(w, '\n');
  for (int i = 0; i < level; i++) { put(w, ' '); put(w, ' '); }
}

static const char KEYCH[] = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789_";

static void emit_key(wbuf *w, rng_t *r) {
  int n = (int)rrange(r, 3, 12);
  put(w, '"');
  for (int i = 0; i < n; i++) put(w, (uint8_t)KEYCH[rbelow(r, sizeof(KEYCH) - 1)]);
  put(w, '"');
}

static void emit_hex4(wbuf *w, uint32_t v) {
  static const char H[] = "0123456789abcdefABCDEF";
  for (int s = 12; s >= 0; s -= 4) {
    uint32_t d = (v >> s) & 15;
    /* mix upper and lower case hex digits */
    put(w, (uint8_t)(d < 10 ? H[d] : ((v ^ (uint32_t)s) & 1 ? H[d] : H[d + 6])));
  }
}

/* One Unicode scalar value, raw UTF-8; 2/3/4-byte sequences in ratio 5:3:2. */
static void emit_nonascii(wbuf *w, rng_t *r) {
  double u = runif(r);
  uint32_t cp;
  if (u < 0.5) cp = (uint32_t)rrange(r, 0x80, 0x7FF);
  else if (u < 0.8) {
    do cp = (uint32_t)rrange(r, 0x800, 0xFFFF); while (cp >= 0xD800 && cp <= 0xDFFF);
  } else cp = (uint32_t)rrange(r, 0x10000, 0x10FFFF);
  if (cp < 0x800) { put(w, (uint8_t)(0xC0 | (cp >> 6))); put(w, (uint8_t)(0x80 | (cp & 63))); }
  else if (cp < 0x10000) {
    put(w, (uint8_t)(0xE0 | (cp >> 12))); put(w, (uint8_t)(0x80 | ((cp >> 6) & 63)));
    put(w, (uint8_t)(0x80 | (cp & 63)));
  } else {
    put(w, (uint8_t)(0xF0 | (cp >> 18))); put(w, (uint8_t)(0x80 | ((cp >> 12) & 63)));
    put(w, (uint8_t)(0x80 | ((cp >> 6) & 63))); put(w, (uint8_t)(0x80 | (cp & 63)));
  }
}

/* An escape; backslash runs of 1..5 are formed as legal escape sequences. */
static void emit_escape(wbuf *w, rng_t *r, double nonascii_p) {
  int k = (int)rbelow(r, 9);
  switch (k) {
    case 0: puts_(w, "\\n"); break;                 /* run of 1 */
    case 1: puts_(w, "\\\\"); break;                /* run of 2 */
    case 2: puts_(w, "\\\\\\\""); break;            /* run of 3 */
    case 3: puts_(w, "\\\\\\\\"); break;            /* run of 4 */
    case 4: puts_(w, "\\\\\\\\\\n"); break;         /* run of 5 */
    case 5: puts_(w, "\\\""); break;
    case 6: { /* \uXXXX, BMP, not a surrogate */
      uint32_t v;
      do v = (uint32_t)rrange(r, 1, 0xFFFF); while (v >= 0xD800 && v <= 0xDFFF);
      puts_(w, "\\u"); emit_hex4(w, v); break;
    }
    case 7: if (nonascii_p > 0) { /* surrogate pair */
        puts_(w, "\\u"); emit_hex4(w, (uint32_t)rrange(r, 0xD800, 0xDBFF));
        puts_(w, "\\u"); emit_hex4(w, (uint32_t)rrange(r, 0xDC00, 0xDFFF));
        break;
      }
      /* fall through */
    default: { static const char *E[] = {"\\t", "\\r", "\\/", "\\b", "\\f"};
      puts_(w, E[rbelow(r, 5)]); break; }
  }
}

static void emit_plain_char(wbuf *w, rng_t *r) {
  /* printable ASCII except '"' and '\\', with some spaces and punctuation that
   * would be structural outside a string */
  uint8_t c;
  do c = (uint8_t)rrange(r, 0x20, 0x7E); while (c == '"' || c == '\\');
  put(w, c);
}

static void emit_string(wbuf *w, rng_t *r, const recopt *o) {
  int n;
  if (runif(r) < o->long_string_p) n = (int)rrange(r, 64, 300);
  else n = (int)rrange(r, o->str_min, o->str_max);
  put(w, '"');
  if (runif(r) < o->straddle_p) {
    /* pad with plain characters so that an escape run lands on a 64-byte,
     * 2 KiB or 128 KiB edge (only when the edge is near) */
    static const uint64_t G[] = {64, 2048, 131072};
    uint64_t g = G[rbelow(r, 3)];
    uint64_t d = g - (w->n % g);
    uint64_t back = (uint64_t)rrange(r, 1, 4);
    if (d > back && d - back <= 96) {
      for (uint64_t i = 0; i < d - back; i++) put(w, 'x');
      puts_(w, runif(r) < 0.5 ? "\\\\\\\"" : "\\\\\\\\\\n");
    }
  }
  for (int i = 0; i < n; i++) {
    double u = runif(r);
    if (u < o->escape_p) emit_escape(w, r, o->nonascii_p);
    else if (u < o->escape_p + o->nonascii_p) emit_nonascii(w, r);
    else emit_plain_char(w, r);
  }
  put(w, '"');
}

static void emit_digits(wbuf *w, rng_t *r, int n, int first_nonzero) {
  for (int i = 0; i < n; i++)
    put(w, (uint8_t)('0' + ((i == 0 && first_nonzero) ? rrange(r, 1, 9) : rrange(r, 0, 9))));
}

static void emit_int(wbuf *w, rng_t *r) {
  int64_t v = rrange(r, -1000000000, 1000000000);
  char tmp[24]; int k = 0;
  uint64_t m = v < 0 ? (uint64_t)(-v) : (uint64_t)v;
  do { tmp[k++] = (char)('0' + m % 10); m /= 10; } while (m);
  if (v < 0) put(w, '-');
  while (k) put(w, (uint8_t)tmp[--k]);
}

/* A decimal with `sig` significant digits, `ip` of them before the point
 * (ip <= 0: leading "0." and -ip zeros), optional exponent. */
static void emit_decimal(wbuf *w, rng_t *r, int sig, int ip, int expo, int has_exp) {
  if (ip <= 0) {
    puts_(w, "0.");
    for (int i = 0; i < -ip; i++) put(w, '0');
    emit_digits(w, r, sig, 1);
  } else if (ip >= sig) {
    emit_digits(w, r, sig, 1);
    for (int i = sig; i < ip; i++) put(w, '0');
    puts_(w, ".0");
  } else {
    emit_digits(w, r, ip, 1);
    put(w, '.');
    emit_digits(w, r, sig - ip, 0);
  }
  if (has_exp) {
    put(w, runif(r) < 0.5 ? 'e' : 'E');
    if (expo < 0) { put(w, '-'); expo = -expo; }
    else if (runif(r) < 0.5) put(w, '+');
    char tmp[8]; int k = 0;
    do { tmp[k++] = (char)('0' + expo % 10); expo /= 10; } while (expo);
    while (k) put(w, (uint8_t)tmp[--k]);
  }
}

static void emit_double(wbuf *w, rng_t *r) {
  int sig = (int)rrange(r, 1, 17);
  if (runif(r) < 0.5) put(w, '-');
  if (runif(r) < 0.15) emit_decimal(w, r, sig, 1, (int)rrange(r, -300, 300), 1);
  else emit_decimal(w, r, sig, (int)rrange(r, -3, 9), 0, 0);
}

static void emit_value(wbuf *w, rng_t *r, const recopt *o, int level, int nest_left);

static void emit_object(wbuf *w, rng_t *r, const recopt *o, int level, int nest_left, int fields) {
  put(w, '{');
  for (int i = 0; i < fields; i++) {
    if (i) put(w, ',');
    newline(w, o, level + 1);
    emit_key(w, r);
    put(w, ':');
    if (o->pretty) put(w, ' ');
    emit_value(w, r, o, level + 1, nest_left);
  }
  if (fields) newline(w, o, level);
  put(w, '}');
}

static void emit_array(wbuf *w, rng_t *r, const recopt *o, int level, int nest_left, int items) {
  put(w, '[');
  for (int i = 0; i < items; i++) {
    if (i) put(w, ',');
    newline(w, o, level + 1);
    emit_value(w, r, o, level + 1, nest_left);
  }
  if (items) newline(w, o, level);
  put(w, ']');
}

static void emit_value(wbuf *w, rng_t *r, const recopt *o, int level, int nest_left) {
  double u = runif(r);
  if (u < 0.05) { puts_(w, "true"); return; }
  if (u < 0.10) { puts_(w, "false"); return; }
  if (u < 0.15) { puts_(w, "null"); return; }
  if (nest_left > 0 && u < 0.23) {
    emit_object(w, r, o, level, nest_left - 1, (int)rrange(r, 0, 6)); return;
  }
  if (nest_left > 0 && u < 0.30) {
    emit_array(w, r, o, level, nest_left - 1, (int)rrange(r, 0, 6)); return;
  }
  if (u < 0.62) { emit_string(w, r, o); return; }
  if (u < 0.82) { emit_int(w, r); return; }
  emit_double(w, r);
}

/* A chain of objects and arrays down to absolute depth `to`. */
static void emit_deep(wbuf *w, rng_t *r, const recopt *o, int level, int to) {
  int n = to - level;
  for (int i = 0; i < n; i++) {
    if (i & 1) { put(w, '['); }
    else { put(w, '{'); emit_key(w, r); put(w, ':'); }
  }
  emit_value(w, r, o, to, 0);
  for (int i = n - 1; i >= 0; i--) put(w, (i & 1) ? ']' : '}');
}

static void emit_record(wbuf *w, rng_t *r, const recopt *o, int level) {
  if (o->deep_p > 0 && runif(r) < o->deep_p) {
    put(w, '{');
    newline(w, o, level + 1);
    emit_key(w, r);
    put(w, ':');
    emit_deep(w, r, o, level + 1, o->deep_levels);
    newline(w, o, level);
    put(w, '}');
    return;
  }
  emit_object(w, r, o, level, o->max_nest, (int)rrange(r, 3, 9));
}

static void init_opts(recopt *o, int pretty, double nonascii_p) {
  memset(o, 0, sizeof(*o));
  o->pretty = pretty;
  o->nonascii_p = nonascii_p;
  o->escape_p = 0.05;
  o->long_string_p = nonascii_p > 0 ? 0.02 : 0.0;
  o->straddle_p = nonascii_p > 0 ? 0.02 : 0.0;
  o->str_min = 0;
  o->str_max = 40;
  o->max_nest = 4;   /* record at level 1 (or 2 in a root array) -> depth <= 6 */
}

/* Records.  root_array == 0: one root object whose fields are records (the
 * 64 KB configuration); root_array == 1: a root array of records (the 1 GB
 * configuration).  The document is the first one of at least `target` bytes. */
uint64_t sjg_records(uint64_t seed, uint64_t target, int root_array, int pretty,
                     double nonascii_p, double deep_p, int deep_levels,
                     uint8_t *out, uint64_t cap) {
  rng_t r = {seed * 0x2545F4914F6CDD1Dull + 0x1234567ull};
  recopt o;
  init_opts(&o, pretty, nonascii_p);
  o.deep_p = deep_p;
  o.deep_levels = deep_levels;
  wbuf w = {out, 0, cap, 0};
  put(&w, root_array ? '[' : '{');
  uint64_t i = 0;
  do {
    if (i) put(&w, ',');
    newline(&w, &o, 1);
    if (!root_array) {
      emit_key(&w, &r);
      put(&w, ':');
      if (pretty) put(&w, ' ');
    }
    emit_record(&w, &r, &o, 1);
    i++;
  } while (w.n + 2 < target && !w.overflow);
  newline(&w, &o, 0);
  put(&w, root_array ? ']' : '}');
  if (pretty) put(&w, '\n');
  return w.overflow ? 0 : w.n;
}

/* A coordinate: an integer part uniform in [-(lim - 1), lim - 1] and random
 * fraction digits up to 15..17 significant digits, so |value| < lim; 1% are
 * written in exponent form (the same digits with one before the point and
 * the exponent moving the point back; a value below 1 keeps the plain form). */
static void emit_coord(wbuf *w, rng_t *r, int lim) {
  int sig = (int)rrange(r, 15, 17);
  int64_t ipart = rrange(r, -(lim - 1), lim - 1);
  const int expo_form = runif(r) < 0.01;
  uint64_t m = ipart < 0 ? (uint64_t)(-ipart) : (uint64_t)ipart;
  if (ipart < 0 || (ipart == 0 && runif(r) < 0.5)) put(w, '-');
  char tmp[8]; int k = 0;
  do { tmp[k++] = (char)('0' + m % 10); m /= 10; } while (m);
  int ip_digits = (ipart == 0) ? 0 : k;
  if (expo_form && ip_digits > 0) {
    put(w, (uint8_t)tmp[--k]);
    put(w, '.');
    while (k) put(w, (uint8_t)tmp[--k]);
    emit_digits(w, r, sig - ip_digits, 0);
    put(w, runif(r) < 0.5 ? 'e' : 'E');
    if (runif(r) < 0.5) put(w, '+');
    put(w, (uint8_t)('0' + (ip_digits - 1)));
    return;
  }
  while (k) put(w, (uint8_t)tmp[--k]);
  put(w, '.');
  emit_digits(w, r, sig - ip_digits, 0);
}

/* Number-heavy GeoJSON-like document: an object wrapping an array of polygons,
 * each an array of U[50,300] [lon,lat] pairs, minimal white space; the first
 * document of at least `target` bytes (canada.json stand-in). */
uint64_t sjg_geo(uint64_t seed, uint64_t target, uint8_t *out, uint64_t cap) {
  rng_t r = {seed * 0x2545F4914F6CDD1Dull + 0x7777ull};
  wbuf w = {out, 0, cap, 0};
  puts_(&w, "{\"type\":\"MultiPolygon\",\"coordinates\":[");
  uint64_t p = 0;
  do {
    if (p) put(&w, ',');
    put(&w, '[');
    int pairs = (int)rrange(&r, 50, 300);
    for (int i = 0; i < pairs; i++) {
      if (i) put(&w, ',');
      put(&w, '[');
      emit_coord(&w, &r, 180);
      put(&w, ',');
      emit_coord(&w, &r, 90);
      put(&w, ']');
    }
    put(&w, ']');
    p++;
  } while (w.n + 2 < target && !w.overflow);
  puts_(&w, "]}");
  return w.overflow ? 0 : w.n;
}

/* String-heavy records: long strings with many escapes and non-ASCII text. */
uint64_t sjg_strings(uint64_t seed, uint64_t target, uint8_t *out, uint64_t cap) {
  rng_t r = {seed * 0x2545F4914F6CDD1Dull + 0x5151ull};
  recopt o;
  init_opts(&o, 0, 0.25);
  o.escape_p = 0.15;
  o.str_min = 20;
  o.str_max = 400;
  o.long_string_p = 0.1;
  o.straddle_p = 0.1;
  o.max_nest = 1;
  wbuf w = {out, 0, cap, 0};
  put(&w, '[');
  uint64_t i = 0;
  do {
    if (i) put(&w, ',');
    emit_string(&w, &r, &o);
    if ((i & 3) == 3) { put(&w, ','); emit_record(&w, &r, &o, 1); }
    i++;
  } while (w.n + 2 < target && !w.overflow);
  put(&w, ']');
  return w.overflow ? 0 : w.n;
}

/* ---- tweets: a stand-in for twitter.json (the paper's user.id query,
 * Table "tab:userid"): {"statuses": [tweet, ...], "search_metadata": {...}}.
 * Each tweet carries "id", "text", "user": {"id", "name", "screen_name",
 * "followers_count", ...}, counters, "entities" and, for 1 in 8, a
 * "retweeted_status" with its own "user".  User ids come from a pool of
 * n_users values, so the distinct count is below the number of users. */
static void emit_uint_digits(wbuf *w, uint64_t v) {
  char t[24];
  int n = 0;
  do { t[n++] = (char)('0' + v % 10); v /= 10; } while (v);
  while (n) put(w, (uint8_t)t[--n]);
}

static void emit_text(wbuf *w, rng_t *r, const recopt *o, int lo, int hi) {
  recopt t = *o;
  t.str_min = lo;
  t.str_max = hi;
  t.long_string_p = 0;
  t.straddle_p = 0;
  emit_string(w, r, &t);
}

static void emit_user(wbuf *w, rng_t *r, const recopt *o, const uint64_t *pool, uint64_t n_users) {
  const uint64_t id = pool[rbelow(r, n_users)];
  puts_(w, "{\"id\":"); emit_uint_digits(w, id);
  puts_(w, ",\"id_str\":\""); emit_uint_digits(w, id); put(w, '"');
  puts_(w, ",\"name\":"); emit_text(w, r, o, 3, 20);
  puts_(w, ",\"screen_name\":"); emit_key(w, r);
  puts_(w, ",\"location\":"); emit_text(w, r, o, 0, 24);
  puts_(w, ",\"description\":"); emit_text(w, r, o, 0, 120);
  puts_(w, ",\"followers_count\":"); emit_uint_digits(w, rbelow(r, 2000000));
  puts_(w, ",\"friends_count\":"); emit_uint_digits(w, rbelow(r, 5000));
  puts_(w, ",\"verified\":"); puts_(w, rbelow(r, 10) ? "false" : "true");
  puts_(w, ",\"profile_image_url\":null}");
}

static void emit_tweet(wbuf *w, rng_t *r, const recopt *o, const uint64_t *pool, uint64_t n_users,
                       int nested) {
  puts_(w, "{\"created_at\":"); emit_text(w, r, o, 30, 30);
  puts_(w, ",\"id\":"); emit_uint_digits(w, 500000000000000000ull + rbelow(r, 400000000000000000ull));
  puts_(w, ",\"text\":"); emit_text(w, r, o, 20, 140);
  puts_(w, ",\"user\":"); emit_user(w, r, o, pool, n_users);
  puts_(w, ",\"retweet_count\":"); emit_uint_digits(w, rbelow(r, 10000));
  puts_(w, ",\"favorite_count\":"); emit_uint_digits(w, rbelow(r, 10000));
  puts_(w, ",\"entities\":{\"hashtags\":[");
  const int nh = (int)rbelow(r, 3);
  for (int i = 0; i < nh; i++) {
    if (i) put(w, ',');
    puts_(w, "{\"text\":"); emit_key(w, r); puts_(w, ",\"indices\":[");
    emit_uint_digits(w, rbelow(r, 100)); put(w, ','); emit_uint_digits(w, rbelow(r, 140));
    puts_(w, "]}");
  }
  puts_(w, "],\"urls\":[]}");
  puts_(w, ",\"favorited\":false,\"lang\":\"en\"");
  if (!nested && rbelow(r, 8) == 0) {
    puts_(w, ",\"retweeted_status\":");
    emit_tweet(w, r, o, pool, n_users, 1);
  }
  put(w, '}');
}

uint64_t sjg_tweets(uint64_t seed, uint64_t target, uint64_t n_users, uint8_t *out, uint64_t cap) {
  rng_t r = {seed * 0x9E3779B97F4A7C15ull + 7};
  wbuf w = {out, 0, cap, 0};
  recopt o;
  init_opts(&o, 0, 0.03);
  if (n_users == 0) n_users = 1;
  if (n_users > 1000000) n_users = 1000000;
  static uint64_t pool[1000000];
  for (uint64_t i = 0; i < n_users; i++) pool[i] = 1000 + rbelow(&r, 4000000000ull);
  puts_(&w, "{\"statuses\":[");
  int first = 1;
  while (w.n + 8 < target) {
    if (!first) put(&w, ',');
    first = 0;
    emit_tweet(&w, &r, &o, pool, n_users, 0);
  }
  puts_(&w, "],\"search_metadata\":{\"count\":100,\"max_id\":null}}");
  return w.overflow ? 0 : w.n;
}
