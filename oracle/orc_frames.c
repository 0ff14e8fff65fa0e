/*
 * Oracle: ORC compressed streams with zlib (raw Deflate) compression chunks.
 * TEST INFRASTRUCTURE ONLY.
 *
 * CODAG decodes chunks of standard formats in place (Sec. I and II-B:
 * compressed data as stored by existing systems, no re-encoding); ORC stores
 * each compressed column stream as a sequence of compression chunks, each
 * with a 3-byte header.  The layout followed here is the ORC v1 one:
 *
 *   header: 3 bytes, little endian, value v; length = v >> 1 body bytes
 *           follow; bit 0 set: the body is stored as is ("original"),
 *           clear: the body is a raw Deflate stream (RFC 1951)
 *   output: the bodies' decoded bytes, one after another
 *
 * Readings: every compressed body is a complete Deflate stream of its own (no
 * window shared between bodies; bytes after its final block are ignored,
 * as for the plain Deflate format); a body may be empty only when stored (an
 * empty Deflate body has no block and is TRUNCATED); a header or body that
 * runs past the input is TRUNCATED; the status of a bad body is the Deflate
 * one; the whole stream must fill the output span (OVERFLOW as soon as a body
 * would pass it, UNDERFLOW at the end).
 */
#include <stdint.h>
#include "oracle.h"

int oracle_orc_zlib(const uint8_t *in, size_t n_in, uint8_t *out, size_t cap, size_t *n_out) {
  size_t pos = 0, count = 0;
  *n_out = 0;
  while (pos < n_in) {
    if (n_in - pos < 3) { *n_out = count; return ORC_TRUNCATED; }
    uint32_t v = (uint32_t)in[pos] | ((uint32_t)in[pos + 1] << 8) | ((uint32_t)in[pos + 2] << 16);
    pos += 3;
    size_t len = v >> 1;
    if (n_in - pos < len) { *n_out = count; return ORC_TRUNCATED; }
    if (v & 1) { /* original bytes */
      if (len > cap - count) { *n_out = count; return ORC_OUTPUT_OVERFLOW; }
      if (out)
        for (size_t i = 0; i < len; i++) out[count + i] = in[pos + i];
      count += len;
    } else { /* a raw Deflate body, decoded into what is left of the span */
      size_t got = 0;
      int st = oracle_inflate(in + pos, len, out ? out + count : NULL,
                              cap == SIZE_MAX ? SIZE_MAX : cap - count, &got);
      if (st == ORC_OUTPUT_UNDERFLOW) st = ORC_OK; /* the span continues with the next body */
      if (st != ORC_OK) { *n_out = count + got; return st; }
      count += got;
    }
    pos += len;
  }
  *n_out = count;
  if (cap != SIZE_MAX && count < cap) return ORC_OUTPUT_UNDERFLOW;
  return ORC_OK;
}
