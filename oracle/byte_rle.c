/*
 * Oracle: ORC byte RLE and boolean RLE decoders.  TEST INFRASTRUCTURE ONLY.
 *
 * CODAG Sec. V-A notes that encodings beyond the evaluated three can be
 * enabled through the same decoding structure; ORC's byte run-length
 * encoding (used for byte columns and, over packed bits, for boolean columns
 * and present streams) is such an encoding.  The byte format followed here
 * is the ORC v1 byte RLE:
 *
 *   control byte h, read as a signed 8-bit number
 *     h in [0, 127]   : a run: the next byte, repeated h + 3 times
 *     h in [-128, -1] : -h literal bytes follow, copied as they are
 *
 * Boolean RLE is byte RLE over bytes that each hold eight booleans, most
 * significant bit first.  The boolean decoder writes one output byte (0 or
 * 1) per boolean; its output span is the number of booleans n, the stream
 * must decode to exactly ceil(n / 8) bytes, and the unused low bits of the
 * last byte are ignored (readings: ORC keeps the value count outside the
 * stream).
 *
 * Error order within a group: TRUNCATED (the run byte or the literals run
 * past the chunk) before OUTPUT_OVERFLOW for the whole group.  Every control
 * byte is valid, so there is no BAD_HEADER.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

int oracle_byte_rle(const uint8_t *in, size_t n_in, uint8_t *out, size_t cap, size_t *n_out) {
  size_t pos = 0, count = 0;
  int store = out != NULL;
  *n_out = 0;
  while (pos < n_in) {
    int8_t h = (int8_t)in[pos++];
    if (h >= 0) {
      size_t len = (size_t)h + 3;
      if (pos >= n_in) { *n_out = count; return ORC_TRUNCATED; }
      uint8_t v = in[pos++];
      if (len > cap - count) { *n_out = count; return ORC_OUTPUT_OVERFLOW; }
      if (store)
        for (size_t i = 0; i < len; i++) out[count + i] = v;
      count += len;
    } else {
      size_t len = (size_t)(-(int)h);
      if (n_in - pos < len) { *n_out = count; return ORC_TRUNCATED; }
      if (len > cap - count) { *n_out = count; return ORC_OUTPUT_OVERFLOW; }
      if (store)
        for (size_t i = 0; i < len; i++) out[count + i] = in[pos + i];
      pos += len;
      count += len;
    }
  }
  *n_out = count;
  if (cap != SIZE_MAX && count < cap) return ORC_OUTPUT_UNDERFLOW;
  return ORC_OK;
}

int oracle_bool_rle(const uint8_t *in, size_t n_in, uint8_t *out, size_t cap, size_t *n_out) {
  /* decode the packed bytes first, then expand bit by bit */
  size_t nbytes_cap = cap == SIZE_MAX ? SIZE_MAX : (cap + 7) / 8;
  size_t got = 0;
  *n_out = 0;
  if (out == NULL) { /* sizing: 8 booleans per decoded byte */
    int st = oracle_byte_rle(in, n_in, NULL, nbytes_cap, &got);
    *n_out = got * 8;
    return st;
  }
  uint8_t *packed = (uint8_t *)malloc(nbytes_cap ? nbytes_cap : 1);
  if (!packed) return ORC_BAD_HEADER;
  int st = oracle_byte_rle(in, n_in, packed, nbytes_cap, &got);
  size_t nb = got * 8 < cap ? got * 8 : cap;
  for (size_t j = 0; j < nb; j++) out[j] = (uint8_t)((packed[j / 8] >> (7 - j % 8)) & 1);
  free(packed);
  *n_out = nb;
  return st;
}
