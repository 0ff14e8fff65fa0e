/*
 * Oracle: ORC integer RLE version 1 decoder.  TEST INFRASTRUCTURE ONLY.
 *
 * CODAG Sec. II-A describes RLE v1 as encoding each run by a value and a run
 * length; Sec. V-A evaluates the Apache ORC form of it.  The byte format
 * followed here is the ORC v1 integer RLE (version 1):
 *
 *   control byte h, read as a signed 8-bit number
 *     h in [0, 127]   : a run of h + 3 values, then one signed delta byte d,
 *                       then a base varint b; value i of the run = b + i*d
 *     h in [-128, -1] : -h literal values follow, each one varint
 *   varint: base-128, least significant 7-bit group first, bit 7 set on every
 *           byte but the last; at most 10 bytes (bits past 64 are dropped)
 *   signed columns store base and literals zigzag-encoded, (u >> 1) ^ -(u & 1);
 *   the delta byte is a plain two's-complement int8 in both cases.
 *
 * Arithmetic wraps modulo 2^64 (readings of the spec: unsigned 64-bit math).
 * Error order within a group: header/varint problems in stream order first
 * (TRUNCATED, BAD_HEADER), then OUTPUT_OVERFLOW for the whole group.
 */
#include <string.h>
#include "oracle.h"

typedef struct {
  const uint8_t *p;
  size_t n, pos;
} v1_in;

/* One varint; returns ORC_OK, ORC_TRUNCATED or ORC_BAD_HEADER. */
static int v1_varint(v1_in *s, uint64_t *v) {
  uint64_t x = 0;
  for (int k = 0; k < 10; k++) {
    if (s->pos >= s->n) return ORC_TRUNCATED;
    uint8_t b = s->p[s->pos++];
    if (7 * k < 64) x |= (uint64_t)(b & 0x7f) << (7 * k);
    if ((b & 0x80) == 0) {
      *v = x;
      return ORC_OK;
    }
  }
  return ORC_BAD_HEADER; /* an 11th byte would be needed */
}

static uint64_t v1_unzigzag(uint64_t u) { return (u >> 1) ^ (0 - (u & 1)); }

static void v1_put(uint8_t *out, size_t idx, uint64_t v) {
  for (int k = 0; k < 8; k++) out[idx * 8 + k] = (uint8_t)(v >> (8 * k));
}

int oracle_rle_v1(const uint8_t *in, size_t n_in, int is_signed,
                  uint8_t *out, size_t cap, size_t *n_out) {
  v1_in s = {in, n_in, 0};
  size_t count = 0; /* values produced */
  int store = out != NULL;
  if (cap != SIZE_MAX && cap % 8 != 0) return ORC_BAD_SPAN;
  size_t cap_values = cap == SIZE_MAX ? SIZE_MAX : cap / 8;
  *n_out = 0;
  while (s.pos < s.n) {
    int8_t h = (int8_t)s.p[s.pos++];
    if (h >= 0) {
      size_t len = (size_t)h + 3;
      if (s.pos >= s.n) return ORC_TRUNCATED;
      int8_t d = (int8_t)s.p[s.pos++];
      uint64_t base;
      int st = v1_varint(&s, &base);
      if (st != ORC_OK) return st;
      if (is_signed) base = v1_unzigzag(base);
      if (len > cap_values - count) return ORC_OUTPUT_OVERFLOW;
      for (size_t i = 0; i < len; i++) {
        uint64_t v = base + (uint64_t)i * (uint64_t)(int64_t)d;
        if (store) v1_put(out, count, v);
        count++;
      }
    } else {
      size_t len = (size_t)(-(int)h);
      uint64_t vals[128];
      for (size_t i = 0; i < len; i++) {
        int st = v1_varint(&s, &vals[i]);
        if (st != ORC_OK) return st;
        if (is_signed) vals[i] = v1_unzigzag(vals[i]);
      }
      if (len > cap_values - count) return ORC_OUTPUT_OVERFLOW;
      for (size_t i = 0; i < len; i++) {
        if (store) v1_put(out, count, vals[i]);
        count++;
      }
    }
    *n_out = count * 8;
  }
  *n_out = count * 8;
  if (cap != SIZE_MAX && count < cap_values) return ORC_OUTPUT_UNDERFLOW;
  return ORC_OK;
}
