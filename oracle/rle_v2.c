/*
 * Oracle: ORC integer RLE version 2 decoder.  TEST INFRASTRUCTURE ONLY.
 *
 * CODAG Sec. II-A: RLE v2 combines run-length and delta encoding (plus bit
 * packing) over RLE v1; Sec. V-A evaluates the Apache ORC form.  The format
 * followed is ORC v1 integer RLE version 2.  The top two bits of a run's
 * first byte select the sub-encoding:
 *
 *   0 SHORT_REPEAT  1 byte header: bits 5-3 = value bytes - 1, bits 2-0 =
 *                   count - 3; then the value, big-endian; repeated count times
 *   1 DIRECT        2 byte header: bits 5-1 of byte 0 = encoded width W,
 *                   bit 0 + byte 1 = length - 1 (9 bits); then L values of W
 *                   bits, MSB first, padded to a byte
 *   2 PATCHED_BASE  4 byte header: W and L as DIRECT; byte 2 = (base bytes-1)
 *                   << 5 | encoded patch width PW; byte 3 = (patch gap width
 *                   - 1) << 5 | patch list length; then the base (big-endian
 *                   sign-magnitude), L data values of W bits (padded), the
 *                   patch list (padded); value = base + (data | patch << W)
 *   3 DELTA         2 byte header: encoded width (0 = fixed delta), length;
 *                   base varint, delta-base zigzag varint, then L-2 deltas of
 *                   W bits added (delta base >= 0) or subtracted (< 0)
 *
 * Encoded widths (5 bits) k = 0..23 mean k + 1 bits; 24..31 mean 26, 28, 30,
 * 32, 40, 48, 56, 64.  In DELTA only, code 0 means width 0 (fixed delta).
 *
 * Readings where the spec is silent (all arithmetic wraps modulo 2^64):
 *   - signed columns zigzag SHORT_REPEAT and DIRECT values and the DELTA base;
 *     PATCHED_BASE data are unsigned offsets from the sign-magnitude base;
 *   - a patch-list entry is PGW + PW bits rounded up to the next encodable
 *     width (the "closest fixed bits" rule of the ORC writers); PGW + PW > 64
 *     is BAD_HEADER; an entry with gap 255 and patch 0 only advances the
 *     position by 255; patch positions must stay below L and strictly
 *     increase (a gap of 0 after a patch would patch one value twice), else
 *     BAD_HEADER; a filler run that reaches the end of the list adds no patch;
 *   - a DELTA run with W != 0 and L = 1 yields only the base;
 *   - padding bits are ignored.
 * Error order within a run: header and field problems in stream order, then
 * OUTPUT_OVERFLOW for the whole run.
 */
#include <string.h>
#include "oracle.h"

static const int v2_width_table[32] = {
    1,  2,  3,  4,  5,  6,  7,  8,  9,  10, 11, 12, 13, 14, 15, 16,
    17, 18, 19, 20, 21, 22, 23, 24, 26, 28, 30, 32, 40, 48, 56, 64};

typedef struct {
  const uint8_t *p;
  size_t n, pos;
} v2_in;

static int v2_byte(v2_in *s, uint8_t *b) {
  if (s->pos >= s->n) return ORC_TRUNCATED;
  *b = s->p[s->pos++];
  return ORC_OK;
}

static int v2_varint(v2_in *s, uint64_t *v) {
  uint64_t x = 0;
  for (int k = 0; k < 10; k++) {
    uint8_t b;
    if (v2_byte(s, &b) != ORC_OK) return ORC_TRUNCATED;
    if (7 * k < 64) x |= (uint64_t)(b & 0x7f) << (7 * k);
    if ((b & 0x80) == 0) {
      *v = x;
      return ORC_OK;
    }
  }
  return ORC_BAD_HEADER;
}

static uint64_t v2_unzigzag(uint64_t u) { return (u >> 1) ^ (0 - (u & 1)); }

/* Read `count` values of `w` bits each, most significant bit first, from a
 * section starting at the current byte; the section is padded to a byte. */
static int v2_unpack(v2_in *s, size_t count, int w, uint64_t *vals) {
  size_t nbits = count * (size_t)w;
  size_t nbytes = (nbits + 7) / 8;
  if (nbytes > s->n - s->pos) return ORC_TRUNCATED;
  const uint8_t *sec = s->p + s->pos;
  size_t bit = 0;
  for (size_t i = 0; i < count; i++) {
    uint64_t v = 0;
    for (int k = 0; k < w; k++, bit++) {
      int b = (sec[bit / 8] >> (7 - bit % 8)) & 1;
      v = (v << 1) | (uint64_t)b;
    }
    vals[i] = v;
  }
  s->pos += nbytes;
  return ORC_OK;
}

static int v2_closest_fixed_bits(int n) {
  for (int k = 0; k < 32; k++)
    if (v2_width_table[k] >= n) return v2_width_table[k];
  return 64;
}

static void v2_put(uint8_t *out, size_t idx, uint64_t v) {
  for (int k = 0; k < 8; k++) out[idx * 8 + k] = (uint8_t)(v >> (8 * k));
}

int oracle_rle_v2(const uint8_t *in, size_t n_in, int is_signed,
                  uint8_t *out, size_t cap, size_t *n_out) {
  v2_in s = {in, n_in, 0};
  size_t count = 0;
  int store = out != NULL;
  uint64_t vals[512];
  if (cap != SIZE_MAX && cap % 8 != 0) return ORC_BAD_SPAN;
  size_t cap_values = cap == SIZE_MAX ? SIZE_MAX : cap / 8;
  *n_out = 0;
  while (s.pos < s.n) {
    uint8_t b0 = s.p[s.pos++];
    int enc = b0 >> 6;
    size_t len = 0;
    int st;
    if (enc == 0) { /* SHORT_REPEAT */
      int nbytes = ((b0 >> 3) & 7) + 1;
      len = (size_t)(b0 & 7) + 3;
      uint64_t v = 0;
      for (int k = 0; k < nbytes; k++) {
        uint8_t b;
        if ((st = v2_byte(&s, &b)) != ORC_OK) return st;
        v = (v << 8) | b;
      }
      if (is_signed) v = v2_unzigzag(v);
      for (size_t i = 0; i < len; i++) vals[i] = v;
    } else {
      uint8_t b1;
      if ((st = v2_byte(&s, &b1)) != ORC_OK) return st;
      int wcode = (b0 >> 1) & 31;
      len = ((size_t)(b0 & 1) << 8 | b1) + 1;
      if (enc == 1) { /* DIRECT */
        int w = v2_width_table[wcode];
        if ((st = v2_unpack(&s, len, w, vals)) != ORC_OK) return st;
        if (is_signed)
          for (size_t i = 0; i < len; i++) vals[i] = v2_unzigzag(vals[i]);
      } else if (enc == 2) { /* PATCHED_BASE */
        int w = v2_width_table[wcode];
        uint8_t b2, b3;
        if ((st = v2_byte(&s, &b2)) != ORC_OK) return st;
        if ((st = v2_byte(&s, &b3)) != ORC_OK) return st;
        int base_bytes = (b2 >> 5) + 1;
        int pw = v2_width_table[b2 & 31];
        int pgw = (b3 >> 5) + 1;
        int pll = b3 & 31;
        if (pgw + pw > 64) return ORC_BAD_HEADER;
        uint64_t mag = 0;
        for (int k = 0; k < base_bytes; k++) {
          uint8_t b;
          if ((st = v2_byte(&s, &b)) != ORC_OK) return st;
          mag = (mag << 8) | b;
        }
        uint64_t sign_bit = (uint64_t)1 << (8 * base_bytes - 1);
        uint64_t base = (mag & sign_bit) ? 0 - (mag & ~sign_bit) : mag;
        if ((st = v2_unpack(&s, len, w, vals)) != ORC_OK) return st;
        uint64_t entries[32];
        int ew = v2_closest_fixed_bits(pgw + pw);
        if ((st = v2_unpack(&s, (size_t)pll, ew, entries)) != ORC_OK) return st;
        /* walk the patch list: positions accumulate gaps from 0 */
        uint64_t pos = 0, prev = 0;
        int have_prev = 0;
        for (int e = 0; e < pll; e++) {
          uint64_t gap = entries[e] >> pw; /* pw <= 63: pgw >= 1 and pgw + pw <= 64 */
          uint64_t patch = entries[e] & (((uint64_t)1 << pw) - 1);
          pos += gap;
          if (gap == 255 && patch == 0) continue; /* filler entry */
          if (pos >= len || (have_prev && pos <= prev)) return ORC_BAD_HEADER;
          vals[pos] |= w == 64 ? 0 : patch << w;
          prev = pos;
          have_prev = 1;
        }
        for (size_t i = 0; i < len; i++) vals[i] = base + vals[i];
      } else { /* DELTA */
        int w = wcode == 0 ? 0 : v2_width_table[wcode];
        uint64_t base, dz;
        if ((st = v2_varint(&s, &base)) != ORC_OK) return st;
        if (is_signed) base = v2_unzigzag(base);
        if ((st = v2_varint(&s, &dz)) != ORC_OK) return st;
        uint64_t delta = v2_unzigzag(dz);
        vals[0] = base;
        if (w == 0) {
          for (size_t i = 1; i < len; i++) vals[i] = vals[i - 1] + delta;
        } else if (len >= 2) {
          uint64_t d[512];
          if ((st = v2_unpack(&s, len - 2, w, d)) != ORC_OK) return st;
          vals[1] = base + delta;
          int negative = (int64_t)delta < 0;
          for (size_t i = 2; i < len; i++)
            vals[i] = negative ? vals[i - 1] - d[i - 2] : vals[i - 1] + d[i - 2];
        }
      }
    }
    if (len > cap_values - count) return ORC_OUTPUT_OVERFLOW;
    for (size_t i = 0; i < len; i++) {
      if (store) v2_put(out, count, vals[i]);
      count++;
    }
    *n_out = count * 8;
  }
  *n_out = count * 8;
  if (cap != SIZE_MAX && count < cap_values) return ORC_OUTPUT_UNDERFLOW;
  return ORC_OK;
}
