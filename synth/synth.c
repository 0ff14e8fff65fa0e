/*
 * Seeded synthetic inputs: column generators and ENCODERS for ORC integer
 * RLE v1 / v2, plus plaintext generators for the Deflate workloads.
 *
 * This module only produces inputs.  It holds no decoding arithmetic and is
 * shared by the tests, the benchmark and the oracle's round-trip pins; the
 * oracle and the GPU library never include or import it.
 *
 * Every random draw comes from splitmix64 keyed by (seed, stream, chunk), and
 * all distributions are built from integer arithmetic only, so a (seed,
 * chunk) pair gives the same bytes on any host.
 *
 * Column shapes (stand-ins for the paper's datasets, which are not public in
 * this form; CODAG Sec. V-B, Tables 4 and 5):
 *   RLE v1: groups chosen by count, 70% runs (length U[3,130], delta
 *           U[-128,127], base ~ N(0, 2^20)) and 30% literal groups (count
 *           U[1,128], values log-uniform in [1, 2^40] with a random sign);
 *           the last group is clipped to the chunk; a remainder under 3
 *           becomes literals.
 *   RLE v2: runs chosen by count, 25% SHORT_REPEAT (3-10 repeats of a 1-8 byte
 *           value), 35% DIRECT (length U[1,512], width ~ N(12,4) clamped to
 *           [1,64] with a 5% tail U[13,64], rounded up to an encodable
 *           width), 15% PATCHED_BASE (length U[16,512], 5% outliers up to
 *           2^48), 25% DELTA (length U[2,512], monotone timestamps near
 *           1.6e12, geometric steps of mean 30; 10% of them fixed-step).
 *   Deflate plaintext: 50% CSV-like rows (digits, commas, newlines, tokens
 *           from a 20-token vocabulary drawn Zipf s = 1.1), 30% little-endian
 *           int32 columns with deltas U[-16,16], 20% uniform random bytes.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

/* ---------------------------------------------------------------- RNG --- */
typedef struct { uint64_t s; } rng_t;

static uint64_t rng_next(rng_t *r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static rng_t rng_make(uint64_t seed, uint64_t stream, uint64_t chunk) {
  rng_t r = {seed * 0x9E3779B97F4A7C15ull ^ (stream << 48) ^ (chunk * 0xD1B54A32D192ED03ull)};
  rng_next(&r);
  rng_next(&r);
  return r;
}

/* uniform in [0, n) (n >= 1), Lemire multiply */
static uint64_t rng_below(rng_t *r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}

static int64_t rng_range(rng_t *r, int64_t lo, int64_t hi) {
  return lo + (int64_t)rng_below(r, (uint64_t)(hi - lo) + 1);
}

/* approximately N(0, 1) scaled by 2^16: Irwin-Hall sum of 12 uniforms */
static int64_t rng_normal16(rng_t *r) {
  int64_t s = 0;
  for (int i = 0; i < 12; i++) s += (int64_t)(rng_next(r) >> 48);
  return s - 6 * 65536;
}

/* log-uniform-ish in [1, 2^bits): uniform octave, uniform inside it */
static uint64_t rng_loguniform(rng_t *r, int bits) {
  int k = (int)rng_below(r, (uint64_t)bits);
  uint64_t lo = (uint64_t)1 << k;
  return lo + rng_below(r, lo);
}

/* geometric on {1, 2, ...} with p = 2185/65536 (mean ~30) */
static uint64_t rng_geometric30(rng_t *r) {
  uint64_t n = 1;
  for (;;) {
    uint64_t x = rng_next(r);
    for (int i = 0; i < 4; i++, x >>= 16, n++)
      if ((x & 0xffff) < 2185) return n;
  }
}

/* ------------------------------------------------------------ helpers --- */
static uint64_t zz(int64_t v) { return ((uint64_t)v << 1) ^ (uint64_t)(v >> 63); }

static int bits_needed(uint64_t v) {
  int b = 0;
  while (v) { b++; v >>= 1; }
  return b;
}

typedef struct {
  uint8_t *p;
  uint64_t n, cap;
  int overflow;
} wbuf;

static void put_byte(wbuf *w, uint8_t b) {
  if (w->n < w->cap) w->p[w->n] = b;
  else w->overflow = 1;
  w->n++;
}

static void put_varint(wbuf *w, uint64_t v) {
  while (v >= 0x80) {
    put_byte(w, (uint8_t)(v | 0x80));
    v >>= 7;
  }
  put_byte(w, (uint8_t)v);
}

/* MSB-first bit packer for one section, padded to a byte at the end */
typedef struct {
  wbuf *w;
  uint8_t cur;
  int nbits;
} bitpack;

static void bp_put(bitpack *b, uint64_t v, int width) {
  for (int k = width - 1; k >= 0; k--) {
    b->cur = (uint8_t)((b->cur << 1) | ((v >> k) & 1));
    if (++b->nbits == 8) {
      put_byte(b->w, b->cur);
      b->cur = 0;
      b->nbits = 0;
    }
  }
}

static void bp_flush(bitpack *b) {
  if (b->nbits) put_byte(b->w, (uint8_t)(b->cur << (8 - b->nbits)));
  b->cur = 0;
  b->nbits = 0;
}

/* RLE v2 5-bit width codes */
static const int W_TABLE[32] = {1,  2,  3,  4,  5,  6,  7,  8,  9,  10, 11,
                                12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22,
                                23, 24, 26, 28, 30, 32, 40, 48, 56, 64};

static int width_code(int w) { /* smallest code whose width >= w (w >= 1) */
  for (int k = 0; k < 32; k++)
    if (W_TABLE[k] >= w) return k;
  return 31;
}

/* ------------------------------------------------------------- RLE v1 --- */
/* Generate and encode one RLE v1 chunk of n values.  values (nullable)
 * receives the column; returns the encoded size (may exceed cap: then
 * nothing past cap was written and the caller must retry with more room). */
uint64_t synth_rle_v1_chunk(uint64_t seed, uint64_t chunk, int is_signed, uint64_t n,
                            int64_t *values, uint8_t *enc, uint64_t cap) {
  rng_t r = rng_make(seed, 1, chunk);
  wbuf w = {enc, 0, cap, 0};
  uint64_t pos = 0;
  while (pos < n) {
    uint64_t rem = n - pos;
    int run = rng_below(&r, 100) < 70;
    if (run && rem >= 3) {
      uint64_t len = (uint64_t)rng_range(&r, 3, 130);
      if (len > rem) len = rem;
      int64_t delta = rng_range(&r, -128, 127);
      int64_t base = rng_normal16(&r) * 16; /* N(0, 2^20) */
      if (!is_signed && base < 0) base = -base;
      put_byte(&w, (uint8_t)(len - 3));
      put_byte(&w, (uint8_t)(int8_t)delta);
      put_varint(&w, is_signed ? zz(base) : (uint64_t)base);
      for (uint64_t i = 0; i < len; i++)
        if (values) values[pos + i] = (int64_t)((uint64_t)base + i * (uint64_t)delta);
      pos += len;
    } else {
      uint64_t cnt = (uint64_t)rng_range(&r, 1, 128);
      if (cnt > rem) cnt = rem;
      put_byte(&w, (uint8_t)(256 - cnt));
      for (uint64_t i = 0; i < cnt; i++) {
        int64_t v = (int64_t)rng_loguniform(&r, 40);
        if (is_signed && (rng_next(&r) & 1)) v = -v;
        put_varint(&w, is_signed ? zz(v) : (uint64_t)v);
        if (values) values[pos + i] = v;
      }
      pos += cnt;
    }
  }
  return w.n;
}

/* ----------------------------------------------------------- byte RLE --- */
/* One ORC byte RLE chunk of n bytes, shaped like a low-cardinality byte or
 * packed-boolean column: 55% runs (length uniform 3..130, value from a
 * 16-symbol alphabet), 45% literal groups (1..128 bytes, 3/4 from the
 * alphabet, 1/4 uniform).  Same calling convention as synth_rle_v1_chunk,
 * with the decoded bytes in `values`. */
uint64_t synth_byte_rle_chunk(uint64_t seed, uint64_t chunk, uint64_t n, uint8_t *values,
                              uint8_t *enc, uint64_t cap) {
  rng_t r = rng_make(seed, 5, chunk);
  wbuf w = {enc, 0, cap, 0};
  uint8_t alpha[16];
  for (int i = 0; i < 16; i++) alpha[i] = (uint8_t)rng_next(&r);
  uint64_t pos = 0;
  while (pos < n) {
    uint64_t rem = n - pos;
    if (rem >= 3 && rng_below(&r, 100) < 55) {
      uint64_t len = (uint64_t)rng_range(&r, 3, 130);
      if (len > rem) len = rem;
      uint8_t v = alpha[rng_below(&r, 16)];
      put_byte(&w, (uint8_t)(len - 3));
      put_byte(&w, v);
      for (uint64_t i = 0; i < len; i++)
        if (values) values[pos + i] = v;
      pos += len;
    } else {
      uint64_t cnt = (uint64_t)rng_range(&r, 1, 128);
      if (cnt > rem) cnt = rem;
      put_byte(&w, (uint8_t)(256 - cnt));
      for (uint64_t i = 0; i < cnt; i++) {
        uint8_t v = rng_below(&r, 4) ? alpha[rng_below(&r, 16)] : (uint8_t)rng_next(&r);
        put_byte(&w, v);
        if (values) values[pos + i] = v;
      }
      pos += cnt;
    }
  }
  return w.n;
}

/* ------------------------------------------------------------- RLE v2 --- */
static void v2_header2(wbuf *w, int enc, int wcode, uint64_t len) {
  put_byte(w, (uint8_t)((enc << 6) | (wcode << 1) | (int)((len - 1) >> 8)));
  put_byte(w, (uint8_t)((len - 1) & 0xff));
}

static int direct_width(rng_t *r) {
  int wbits;
  if (rng_below(r, 100) < 5) {
    wbits = (int)rng_range(r, 13, 64);
  } else {
    int64_t x = 12 * 65536 + 4 * rng_normal16(r); /* N(12, 4) in 1/65536 */
    wbits = (int)((x + 32768) >> 16);
    if (wbits < 1) wbits = 1;
    if (wbits > 64) wbits = 64;
  }
  return W_TABLE[width_code(wbits)];
}

static uint64_t rand_bits(rng_t *r, int bits) {
  return bits >= 64 ? rng_next(r) : rng_next(r) & (((uint64_t)1 << bits) - 1);
}

uint64_t synth_rle_v2_chunk(uint64_t seed, uint64_t chunk, int is_signed, uint64_t n,
                            int64_t *values, uint8_t *enc, uint64_t cap) {
  rng_t r = rng_make(seed, 2, chunk);
  wbuf w = {enc, 0, cap, 0};
  uint64_t pos = 0;
  uint64_t tmp[512];
  while (pos < n) {
    uint64_t rem = n - pos;
    uint64_t pick = rng_below(&r, 100);
    if (pick < 25 && rem >= 3) { /* SHORT_REPEAT */
      uint64_t cnt = (uint64_t)rng_range(&r, 3, 10);
      if (cnt > rem) cnt = rem;
      int nb = (int)rng_range(&r, 1, 8);
      uint64_t u = rand_bits(&r, 8 * nb);
      int64_t v = is_signed ? (int64_t)((u >> 1) ^ (0 - (u & 1))) : (int64_t)u;
      uint64_t e = is_signed ? zz(v) : (uint64_t)v;
      int bytes = (bits_needed(e) + 7) / 8;
      if (bytes == 0) bytes = 1;
      put_byte(&w, (uint8_t)(((bytes - 1) << 3) | (int)(cnt - 3)));
      for (int k = bytes - 1; k >= 0; k--) put_byte(&w, (uint8_t)(e >> (8 * k)));
      for (uint64_t i = 0; i < cnt; i++)
        if (values) values[pos + i] = v;
      pos += cnt;
    } else if (pick < 60 || (pick < 25 && rem < 3)) { /* DIRECT */
      uint64_t len = (uint64_t)rng_range(&r, 1, 512);
      if (len > rem) len = rem;
      int wb = direct_width(&r);
      bitpack bp = {&w, 0, 0};
      v2_header2(&w, 1, width_code(wb), len);
      for (uint64_t i = 0; i < len; i++) {
        uint64_t u = rand_bits(&r, wb);
        bp_put(&bp, u, wb);
        if (values)
          values[pos + i] = is_signed ? (int64_t)((u >> 1) ^ (0 - (u & 1))) : (int64_t)u;
      }
      bp_flush(&bp);
      pos += len;
    } else if (pick < 75) { /* PATCHED_BASE */
      uint64_t len = (uint64_t)rng_range(&r, 16, 512);
      if (len > rem) len = rem;
      int64_t base = rng_range(&r, is_signed ? -(1 << 20) : 0, 1 << 20);
      int wcap = direct_width(&r);
      if (wcap > 24) wcap = 24;
      int wb = W_TABLE[width_code(wcap)];
      uint64_t patch[512];
      int npatch = 0, maxpatch_bits = 1;
      for (uint64_t i = 0; i < len; i++) {
        tmp[i] = rand_bits(&r, wb);
        patch[i] = 0;
        if (npatch < 29 && rng_below(&r, 100) < 5) {
          int pb = 48 - wb;
          uint64_t p = 1 + rng_below(&r, ((uint64_t)1 << pb) - 1);
          patch[i] = p;
          npatch++;
          if (bits_needed(p) > maxpatch_bits) maxpatch_bits = bits_needed(p);
        }
      }
      int pw = W_TABLE[width_code(maxpatch_bits)];
      /* patch entries: (gap, patch); gaps over 255 use (255, 0) fillers */
      uint64_t egap[32], epatch[32];
      int ne = 0, maxgap_bits = 1;
      uint64_t last = 0;
      for (uint64_t i = 0; i < len; i++) {
        if (!patch[i]) continue;
        uint64_t gap = i - last;
        while (gap > 255) {
          egap[ne] = 255;
          epatch[ne] = 0;
          ne++;
          gap -= 255;
        }
        egap[ne] = gap;
        epatch[ne] = patch[i];
        ne++;
        last = i;
      }
      for (int e = 0; e < ne; e++)
        if (bits_needed(egap[e]) > maxgap_bits) maxgap_bits = bits_needed(egap[e]);
      uint64_t mag = (uint64_t)(base < 0 ? -base : base);
      int bw = (bits_needed(mag) + 1 + 7) / 8;
      v2_header2(&w, 2, width_code(wb), len);
      put_byte(&w, (uint8_t)(((bw - 1) << 5) | width_code(pw)));
      put_byte(&w, (uint8_t)(((maxgap_bits - 1) << 5) | ne));
      uint64_t sm = mag | (base < 0 ? (uint64_t)1 << (8 * bw - 1) : 0);
      for (int k = bw - 1; k >= 0; k--) put_byte(&w, (uint8_t)(sm >> (8 * k)));
      bitpack bp = {&w, 0, 0};
      for (uint64_t i = 0; i < len; i++) bp_put(&bp, tmp[i], wb);
      bp_flush(&bp);
      int ew = W_TABLE[width_code(maxgap_bits + pw)];
      for (int e = 0; e < ne; e++) bp_put(&bp, (egap[e] << pw) | epatch[e], ew);
      bp_flush(&bp);
      for (uint64_t i = 0; i < len; i++)
        if (values)
          values[pos + i] = (int64_t)((uint64_t)base + (tmp[i] | (patch[i] << wb)));
      pos += len;
    } else { /* DELTA */
      uint64_t len = (uint64_t)rng_range(&r, 2, 512);
      if (len > rem) len = rem;
      int64_t base = 1600000000000ll + (int64_t)rng_below(&r, 1000000000ull);
      int down = rng_below(&r, 100) < 15;
      int fixed = rng_below(&r, 100) < 10;
      uint64_t fstep = 1 + rng_below(&r, 60);
      tmp[0] = (uint64_t)base;
      for (uint64_t i = 1; i < len; i++) {
        uint64_t s = fixed ? fstep : rng_geometric30(&r);
        tmp[i] = down ? tmp[i - 1] - s : tmp[i - 1] + s;
      }
      int64_t delta = len >= 2 ? (int64_t)(tmp[1] - tmp[0]) : 0;
      uint64_t maxd = 0;
      int all_same = 1;
      for (uint64_t i = 2; i < len; i++) {
        uint64_t d = down ? tmp[i - 1] - tmp[i] : tmp[i] - tmp[i - 1];
        if (d > maxd) maxd = d;
        if ((int64_t)(tmp[i] - tmp[i - 1]) != delta) all_same = 0;
      }
      if (all_same || len < 3) {
        v2_header2(&w, 3, 0, len);
        put_varint(&w, is_signed ? zz(base) : (uint64_t)base);
        put_varint(&w, zz(delta));
      } else {
        int wb = bits_needed(maxd);
        if (wb < 2) wb = 2; /* width 1 has no DELTA code */
        int code = width_code(wb);
        wb = W_TABLE[code];
        v2_header2(&w, 3, code, len);
        put_varint(&w, is_signed ? zz(base) : (uint64_t)base);
        put_varint(&w, zz(delta));
        bitpack bp = {&w, 0, 0};
        for (uint64_t i = 2; i < len; i++)
          bp_put(&bp, down ? tmp[i - 1] - tmp[i] : tmp[i] - tmp[i - 1], wb);
        bp_flush(&bp);
      }
      for (uint64_t i = 0; i < len; i++)
        if (values) values[pos + i] = (int64_t)tmp[i];
      pos += len;
    }
  }
  return w.n;
}

/* ------------------------------------------------ Deflate plaintexts --- */
static const uint32_t ZIPF20_CDF[20] = {
    1345767730u, 1973590576u, 2375507904u, 2668397618u, 2897538777u,
    3085039840u, 3243296599u, 3379934482u, 3499968225u, 3606866355u,
    3703124649u, 3790596988u, 3870696970u, 3944526359u, 4012960012u,
    4076703839u, 4136335416u, 4192333137u, 4245097555u, 4294967295u};

/* kind: 0 = CSV-like rows, 1 = int32 column with small deltas, 2 = random.
 * kind < 0 picks it from the (seed, chunk) draw (50/30/20). Returns kind. */
int synth_plaintext(uint64_t seed, uint64_t chunk, int kind, uint8_t *out, uint64_t n) {
  rng_t r = rng_make(seed, 3, chunk);
  if (kind < 0) {
    uint64_t k = rng_below(&r, 100);
    kind = k < 50 ? 0 : k < 80 ? 1 : 2;
  }
  if (kind == 0) {
    static const char alpha[] = "abcdefghijklmnopqrstuvwxyz0123456789-._/";
    char vocab[20][9];
    int vlen[20];
    rng_t vr = rng_make(seed, 4, 0); /* one vocabulary per seed */
    for (int t = 0; t < 20; t++) {
      vlen[t] = (int)rng_range(&vr, 2, 8);
      for (int i = 0; i < vlen[t]; i++) vocab[t][i] = alpha[rng_below(&vr, 40)];
    }
    uint64_t pos = 0;
    while (pos < n) {
      int fields = (int)rng_range(&r, 6, 10);
      for (int f = 0; f < fields && pos < n; f++) {
        char tok[32];
        int tl = 0;
        if (rng_below(&r, 100) < 60) {
          uint32_t u = (uint32_t)(rng_next(&r) >> 32);
          int t = 0;
          while (t < 19 && u > ZIPF20_CDF[t]) t++;
          memcpy(tok, vocab[t], (size_t)vlen[t]);
          tl = vlen[t];
        } else {
          int digits = (int)rng_range(&r, 1, 7);
          for (int d = 0; d < digits; d++) tok[tl++] = (char)('0' + rng_below(&r, 10));
          if (rng_below(&r, 100) < 30) {
            tok[tl++] = '.';
            tok[tl++] = (char)('0' + rng_below(&r, 10));
            tok[tl++] = (char)('0' + rng_below(&r, 10));
          }
        }
        tok[tl++] = f == fields - 1 ? '\n' : ',';
        for (int i = 0; i < tl && pos < n; i++) out[pos++] = (uint8_t)tok[i];
      }
    }
  } else if (kind == 1) {
    int64_t v = rng_range(&r, -(1ll << 30), 1ll << 30);
    for (uint64_t pos = 0; pos < n; pos += 4) {
      uint32_t u = (uint32_t)v;
      for (int k = 0; k < 4 && pos + k < n; k++) out[pos + k] = (uint8_t)(u >> (8 * k));
      v += rng_range(&r, -16, 16);
    }
  } else {
    for (uint64_t pos = 0; pos < n; pos += 8) {
      uint64_t x = rng_next(&r);
      for (int k = 0; k < 8 && pos + k < n; k++) out[pos + k] = (uint8_t)(x >> (8 * k));
    }
  }
  return kind;
}
