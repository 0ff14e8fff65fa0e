/*
 * Oracle: raw Deflate (RFC 1951) decoder.  TEST INFRASTRUCTURE ONLY.
 *
 * CODAG Sec. II-A: Deflate is dictionary (LZ77) coding whose literals and
 * length/offset pairs are Huffman coded; Sec. IV-F gives the back-reference
 * copy (including the case where the length exceeds the offset and the
 * window repeats, which this decoder defines by copying one byte at a time).
 * The stream format is RFC 1951 Sec. 3.2, followed in its own order:
 *   3.2.3 block loop (BFINAL, BTYPE), 3.2.4 stored blocks, 3.2.2 canonical
 *   code construction, 3.2.6 fixed codes, 3.2.7 dynamic code lengths,
 *   3.2.5 length and distance bases/extra bits.
 * Bits are taken least significant first from each byte; Huffman codes are
 * matched one bit at a time, most significant code bit first.
 *
 * Readings where the RFC leaves acceptance open (chosen to agree with zlib,
 * so that zlib can serve as an independent check of this decoder):
 *   - HLIT + 257 > 286 or HDIST + 1 > 30 is BAD_HUFFMAN;
 *   - an over-subscribed code is BAD_HUFFMAN; an incomplete code is
 *     BAD_HUFFMAN unless it is a single code of length 1 (lit/len and
 *     distance codes) or, for distance codes only, has no codes at all;
 *     the code-length code must be complete;
 *   - reading a code whose prefix no code can extend is BAD_HUFFMAN, as is
 *     decoding lit/len symbol 286/287 or distance symbol 30/31;
 *   - a missing end-of-block code (length of symbol 256 is 0) is BAD_HUFFMAN;
 *   - a repeat code 16 with no previous length, or a repeat running past
 *     HLIT + HDIST lengths, is BAD_HUFFMAN;
 *   - a distance reaching before the chunk's first output byte is
 *     BAD_DISTANCE (chunks have no preset dictionary);
 *   - BTYPE 3 is BAD_HEADER; bytes after the final block are ignored.
 * Error order: the first problem met while decoding in stream order wins;
 * for a stored block: TRUNCATED header, BAD_STORED_LEN, OUTPUT_OVERFLOW,
 * then TRUNCATED data; for a match: BAD_DISTANCE before OUTPUT_OVERFLOW.
 */
#include <string.h>
#include "oracle.h"

#define INF_MAXBITS 15

typedef struct {
  const uint8_t *p;
  size_t n;
  size_t bitpos; /* absolute bit position in the stream */
} inf_in;

static int inf_bits(inf_in *s, int k, uint32_t *v) {
  uint32_t x = 0;
  for (int i = 0; i < k; i++) {
    if (s->bitpos >= s->n * 8) return ORC_TRUNCATED;
    uint32_t b = (s->p[s->bitpos / 8] >> (s->bitpos % 8)) & 1;
    x |= b << i;
    s->bitpos++;
  }
  *v = x;
  return ORC_OK;
}

/* A canonical Huffman code (RFC 1951 Sec. 3.2.2). */
typedef struct {
  int count[INF_MAXBITS + 1];   /* number of codes of each length */
  int first[INF_MAXBITS + 1];   /* first code of each length */
  int offset[INF_MAXBITS + 1];  /* index in `symbols` of that first code */
  int symbols[320];             /* symbols ordered by (length, symbol) */
  uint32_t kraft;               /* sum of 2^(15 - len) over all codes */
} inf_code;

/* Build a code from lengths[0..n).  kind: 0 = code-length code,
 * 1 = lit/len, 2 = distance.  Returns ORC_OK or ORC_BAD_HUFFMAN. */
static int inf_build(inf_code *c, const int *lengths, int n, int kind) {
  memset(c, 0, sizeof(*c));
  for (int i = 0; i < n; i++) c->count[lengths[i]]++;
  c->count[0] = 0;
  int maxlen = 0;
  uint32_t kraft = 0;
  for (int len = 1; len <= INF_MAXBITS; len++) {
    kraft += (uint32_t)c->count[len] << (INF_MAXBITS - len);
    if (c->count[len]) maxlen = len;
  }
  c->kraft = kraft;
  if (kraft > (1u << INF_MAXBITS)) return ORC_BAD_HUFFMAN; /* over-subscribed */
  if (kraft < (1u << INF_MAXBITS)) {                         /* incomplete */
    int ok = 0;
    if (kind != 0 && maxlen == 1) ok = 1;
    if (kind == 2 && maxlen == 0) ok = 1;
    if (!ok) return ORC_BAD_HUFFMAN;
  }
  int code = 0, idx = 0;
  for (int len = 1; len <= INF_MAXBITS; len++) {
    code = (code + c->count[len - 1]) << 1;
    c->first[len] = code;
    c->offset[len] = idx;
    idx += c->count[len];
  }
  int fill[INF_MAXBITS + 1];
  memcpy(fill, c->offset, sizeof(fill));
  for (int i = 0; i < n; i++)
    if (lengths[i]) c->symbols[fill[lengths[i]]++] = i;
  return ORC_OK;
}

/* Decode one symbol, one bit at a time. */
static int inf_decode(inf_in *s, const inf_code *c, int *sym) {
  int code = 0;
  if (c->kraft == 0) return ORC_BAD_HUFFMAN; /* no code can be read at all */
  for (int len = 1; len <= INF_MAXBITS; len++) {
    uint32_t b;
    int st = inf_bits(s, 1, &b);
    if (st != ORC_OK) return st;
    code = (code << 1) | (int)b;
    int k = code - c->first[len];
    if (k >= 0 && k < c->count[len]) {
      *sym = c->symbols[c->offset[len] + k];
      return ORC_OK;
    }
    /* prefixes at or above ceil(kraft * 2^len / 2^15) start no code */
    uint32_t valid = (c->kraft + (1u << (INF_MAXBITS - len)) - 1) >> (INF_MAXBITS - len);
    if ((uint32_t)code >= valid) return ORC_BAD_HUFFMAN;
  }
  return ORC_BAD_HUFFMAN;
}

/* RFC 1951 Sec. 3.2.5 */
static const int inf_len_base[29] = {3,  4,  5,  6,  7,  8,  9,  10, 11, 13,
                                     15, 17, 19, 23, 27, 31, 35, 43, 51, 59,
                                     67, 83, 99, 115, 131, 163, 195, 227, 258};
static const int inf_len_extra[29] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 1,
                                      1, 1, 2, 2, 2, 2, 3, 3, 3, 3,
                                      4, 4, 4, 4, 5, 5, 5, 5, 0};
static const int inf_dist_base[30] = {
    1,    2,    3,    4,    5,    7,     9,     13,    17,  25,
    33,   49,   65,   97,   129,  193,   257,   385,   513, 769,
    1025, 1537, 2049, 3073, 4097, 6145, 8193, 12289, 16385, 24577};
static const int inf_dist_extra[30] = {0, 0, 0, 0, 1, 1, 2,  2,  3,  3,
                                       4, 4, 5, 5, 6, 6, 7,  7,  8,  8,
                                       9, 9, 10, 10, 11, 11, 12, 12, 13, 13};

/* Code-length code order, RFC 1951 Sec. 3.2.7 */
static const int inf_clen_order[19] = {16, 17, 18, 0, 8,  7, 9,  6, 10, 5,
                                       11, 4,  12, 3, 13, 2, 14, 1, 15};

typedef struct {
  uint8_t *out;
  size_t cap, n;
  int store;
} inf_out;

static int inf_codes(inf_in *s, inf_out *o, const inf_code *lit, const inf_code *dist) {
  for (;;) {
    int sym, st;
    if ((st = inf_decode(s, lit, &sym)) != ORC_OK) return st;
    if (sym < 256) {
      if (o->n >= o->cap) return ORC_OUTPUT_OVERFLOW;
      if (o->store) o->out[o->n] = (uint8_t)sym;
      o->n++;
    } else if (sym == 256) {
      return ORC_OK;
    } else {
      sym -= 257;
      if (sym >= 29) return ORC_BAD_HUFFMAN;
      uint32_t e;
      if ((st = inf_bits(s, inf_len_extra[sym], &e)) != ORC_OK) return st;
      size_t len = (size_t)inf_len_base[sym] + e;
      int dsym;
      if ((st = inf_decode(s, dist, &dsym)) != ORC_OK) return st;
      if (dsym >= 30) return ORC_BAD_HUFFMAN;
      if ((st = inf_bits(s, inf_dist_extra[dsym], &e)) != ORC_OK) return st;
      size_t d = (size_t)inf_dist_base[dsym] + e;
      if (d > o->n) return ORC_BAD_DISTANCE;
      if (len > o->cap - o->n) return ORC_OUTPUT_OVERFLOW;
      for (size_t i = 0; i < len; i++) { /* byte at a time: defines overlap */
        if (o->store) o->out[o->n] = o->out[o->n - d];
        o->n++;
      }
    }
  }
}

static int inf_stored(inf_in *s, inf_out *o) {
  s->bitpos = (s->bitpos + 7) / 8 * 8; /* skip to a byte boundary */
  uint32_t len, nlen;
  int st;
  if ((st = inf_bits(s, 16, &len)) != ORC_OK) return st;
  if ((st = inf_bits(s, 16, &nlen)) != ORC_OK) return st;
  if (len != (~nlen & 0xffffu)) return ORC_BAD_STORED_LEN;
  if (len > o->cap - o->n) return ORC_OUTPUT_OVERFLOW;
  size_t at = s->bitpos / 8;
  if (len > s->n - at) return ORC_TRUNCATED;
  if (o->store) memcpy(o->out + o->n, s->p + at, len);
  o->n += len;
  s->bitpos += (size_t)len * 8;
  return ORC_OK;
}

static int inf_fixed(inf_in *s, inf_out *o) {
  int lengths[288];
  inf_code lit, dist;
  for (int i = 0; i < 144; i++) lengths[i] = 8;
  for (int i = 144; i < 256; i++) lengths[i] = 9;
  for (int i = 256; i < 280; i++) lengths[i] = 7;
  for (int i = 280; i < 288; i++) lengths[i] = 8;
  inf_build(&lit, lengths, 288, 1);
  for (int i = 0; i < 32; i++) lengths[i] = 5;
  inf_build(&dist, lengths, 32, 2);
  return inf_codes(s, o, &lit, &dist);
}

static int inf_dynamic(inf_in *s, inf_out *o) {
  uint32_t hlit, hdist, hclen;
  int st;
  if ((st = inf_bits(s, 5, &hlit)) != ORC_OK) return st;
  if ((st = inf_bits(s, 5, &hdist)) != ORC_OK) return st;
  if ((st = inf_bits(s, 4, &hclen)) != ORC_OK) return st;
  int nlen = (int)hlit + 257, ndist = (int)hdist + 1, ncode = (int)hclen + 4;
  if (nlen > 286 || ndist > 30) return ORC_BAD_HUFFMAN;
  int lengths[320];
  memset(lengths, 0, sizeof(lengths));
  for (int i = 0; i < ncode; i++) {
    uint32_t v;
    if ((st = inf_bits(s, 3, &v)) != ORC_OK) return st;
    lengths[inf_clen_order[i]] = (int)v;
  }
  inf_code clen;
  if ((st = inf_build(&clen, lengths, 19, 0)) != ORC_OK) return st;
  int have = 0;
  while (have < nlen + ndist) {
    int sym;
    if ((st = inf_decode(s, &clen, &sym)) != ORC_OK) return st;
    if (sym < 16) {
      lengths[have++] = sym;
      continue;
    }
    int rep, val = 0;
    uint32_t e;
    if (sym == 16) {
      if (have == 0) return ORC_BAD_HUFFMAN;
      val = lengths[have - 1];
      if ((st = inf_bits(s, 2, &e)) != ORC_OK) return st;
      rep = 3 + (int)e;
    } else if (sym == 17) {
      if ((st = inf_bits(s, 3, &e)) != ORC_OK) return st;
      rep = 3 + (int)e;
    } else {
      if ((st = inf_bits(s, 7, &e)) != ORC_OK) return st;
      rep = 11 + (int)e;
    }
    if (have + rep > nlen + ndist) return ORC_BAD_HUFFMAN;
    while (rep--) lengths[have++] = val;
  }
  if (lengths[256] == 0) return ORC_BAD_HUFFMAN;
  inf_code lit, dist;
  if ((st = inf_build(&lit, lengths, nlen, 1)) != ORC_OK) return st;
  if ((st = inf_build(&dist, lengths + nlen, ndist, 2)) != ORC_OK) return st;
  return inf_codes(s, o, &lit, &dist);
}

int oracle_inflate(const uint8_t *in, size_t n_in, uint8_t *out, size_t cap,
                   size_t *n_out) {
  inf_in s = {in, n_in, 0};
  inf_out o = {out, cap, 0, out != NULL};
  int st = ORC_OK;
  for (;;) {
    uint32_t bfinal, btype;
    if ((st = inf_bits(&s, 1, &bfinal)) != ORC_OK) break;
    if ((st = inf_bits(&s, 2, &btype)) != ORC_OK) break;
    if (btype == 0)
      st = inf_stored(&s, &o);
    else if (btype == 1)
      st = inf_fixed(&s, &o);
    else if (btype == 2)
      st = inf_dynamic(&s, &o);
    else
      st = ORC_BAD_HEADER;
    if (st != ORC_OK || bfinal) break;
  }
  *n_out = o.n;
  if (st == ORC_OK && cap != SIZE_MAX && o.n < cap) return ORC_OUTPUT_UNDERFLOW;
  return st;
}
