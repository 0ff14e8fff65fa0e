/*
 * Oracle: per-chunk dispatch and plain loops over chunk ranges.
 * TEST INFRASTRUCTURE ONLY.
 *
 * CODAG Sec. II-B: chunks are compressed independently and the container's
 * offset metadata lets each decode on its own; this file is that loop, one
 * chunk after another.
 */
#include <stdint.h>
#include "oracle.h"

int oracle_decode_chunk(int format, const uint8_t *in, size_t n_in,
                        uint8_t *out, size_t cap, size_t *n_out) {
  switch (format) {
    case ORC_FMT_RLE_V1_I64: return oracle_rle_v1(in, n_in, 1, out, cap, n_out);
    case ORC_FMT_RLE_V1_U64: return oracle_rle_v1(in, n_in, 0, out, cap, n_out);
    case ORC_FMT_RLE_V2_I64: return oracle_rle_v2(in, n_in, 1, out, cap, n_out);
    case ORC_FMT_RLE_V2_U64: return oracle_rle_v2(in, n_in, 0, out, cap, n_out);
    case ORC_FMT_DEFLATE: return oracle_inflate(in, n_in, out, cap, n_out);
    case ORC_FMT_BYTE_RLE: return oracle_byte_rle(in, n_in, out, cap, n_out);
    case ORC_FMT_BOOL_RLE: return oracle_bool_rle(in, n_in, out, cap, n_out);
    case ORC_FMT_ORC_ZLIB: return oracle_orc_zlib(in, n_in, out, cap, n_out);
    default: *n_out = 0; return ORC_BAD_HEADER;
  }
}

void oracle_decode_range(int format, const uint8_t *formats,
                         const uint8_t *comp, const uint64_t *comp_off,
                         uint8_t *out, const uint64_t *out_off,
                         int32_t *status, uint64_t first, uint64_t last) {
  for (uint64_t c = first; c < last; c++) {
    int f = formats ? formats[c] : format;
    size_t n_out = 0;
    status[c] = oracle_decode_chunk(f, comp + comp_off[c], comp_off[c + 1] - comp_off[c],
                                    out + out_off[c], out_off[c + 1] - out_off[c], &n_out);
  }
}

void oracle_sizes_range(int format, const uint8_t *formats,
                        const uint8_t *comp, const uint64_t *comp_off,
                        uint64_t *sizes, int32_t *status,
                        uint64_t first, uint64_t last) {
  for (uint64_t c = first; c < last; c++) {
    int f = formats ? formats[c] : format;
    size_t n_out = 0;
    status[c] = oracle_decode_chunk(f, comp + comp_off[c], comp_off[c + 1] - comp_off[c],
                                    NULL, SIZE_MAX, &n_out);
    sizes[c] = n_out;
  }
}
