/*
 * Oracle decoders: plain, slow, single-threaded CPU reference implementations
 * of the three chunk formats the GPU library decodes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call
 * this code; only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * path: every constant below is written out here again on purpose.
 *
 * What is decoded (CODAG, Sec. II-A and Sec. V-A): each chunk is an
 * independently compressed byte stream that decodes on its own; a chunk's
 * output must fill its output span exactly.
 *
 *   - ORC integer RLE v1 (run / literal groups, Sec. II-A "RLE v1"),
 *   - ORC integer RLE v2 (SHORT_REPEAT / DIRECT / PATCHED_BASE / DELTA,
 *     Sec. II-A "RLE v2 ... leverages delta encoding"),
 *   - raw Deflate, RFC 1951 (Sec. II-A "Deflate ... Huffman tree").
 *
 * RLE outputs are little-endian 64-bit integers (8 bytes per value); Deflate
 * outputs bytes.  Every function returns one of the status codes below; the
 * numeric values are the same ones the GPU library reports per chunk.
 */
#ifndef CODAG_ORACLE_H
#define CODAG_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_OK = 0,
  ORC_TRUNCATED = 1,        /* the stream needs bytes past the chunk's end   */
  ORC_OUTPUT_OVERFLOW = 2,  /* decoding would write past the output span     */
  ORC_OUTPUT_UNDERFLOW = 3, /* the stream ended before the span was filled   */
  ORC_BAD_HEADER = 4,       /* malformed header, varint, block type or patch */
  ORC_BAD_HUFFMAN = 5,      /* bad code lengths, invalid code or symbol      */
  ORC_BAD_DISTANCE = 6,     /* back-reference before the start of the chunk  */
  ORC_BAD_STORED_LEN = 7,   /* stored block LEN != ~NLEN                     */
  ORC_BAD_SPAN = 8          /* RLE output span is not a multiple of 8 bytes  */
};

/* Format identifiers (same numbering as the library's). */
enum {
  ORC_FMT_RLE_V1_I64 = 1,
  ORC_FMT_RLE_V2_I64 = 2,
  ORC_FMT_DEFLATE = 3,
  ORC_FMT_RLE_V1_U64 = 4,
  ORC_FMT_RLE_V2_U64 = 5,
  ORC_FMT_BYTE_RLE = 6,  /* ORC byte RLE: bytes out                        */
  ORC_FMT_BOOL_RLE = 7,  /* ORC boolean RLE: one 0/1 byte per boolean out  */
  ORC_FMT_ORC_ZLIB = 8   /* ORC compressed stream: 3-byte framed Deflate   */
};

/*
 * Decode one chunk.  `in`/`n_in` is the compressed chunk.  `out` receives at
 * most `cap` bytes (RLE: cap must be a multiple of 8).  `*n_out` receives the
 * number of bytes the stream decodes to (when the status is OK, OVERFLOW is
 * reported as soon as the stream would pass `cap`).  `out` may be NULL when
 * cap is 0 and only the decoded size is wanted: pass cap = SIZE_MAX with
 * out = NULL to size a stream (no bytes are stored then).
 */
int oracle_rle_v1(const uint8_t *in, size_t n_in, int is_signed,
                  uint8_t *out, size_t cap, size_t *n_out);
int oracle_rle_v2(const uint8_t *in, size_t n_in, int is_signed,
                  uint8_t *out, size_t cap, size_t *n_out);
int oracle_inflate(const uint8_t *in, size_t n_in,
                   uint8_t *out, size_t cap, size_t *n_out);
int oracle_byte_rle(const uint8_t *in, size_t n_in, uint8_t *out, size_t cap, size_t *n_out);
/* cap = number of booleans; sizing (out = NULL) gives 8 per decoded byte */
int oracle_bool_rle(const uint8_t *in, size_t n_in, uint8_t *out, size_t cap, size_t *n_out);
int oracle_orc_zlib(const uint8_t *in, size_t n_in, uint8_t *out, size_t cap, size_t *n_out);

/* Dispatch on a format identifier (unknown format -> ORC_BAD_HEADER). */
int oracle_decode_chunk(int format, const uint8_t *in, size_t n_in,
                        uint8_t *out, size_t cap, size_t *n_out);

/*
 * Decode chunks [first, last) of a chunked buffer laid out like the library's
 * arguments: chunk c is comp[comp_off[c] .. comp_off[c+1]) and decodes into
 * out[out_off[c] .. out_off[c+1]).  `formats` is either NULL (every chunk has
 * `format`) or a per-chunk format array.  Writes status[c] for each chunk.
 * Plain loop; callers may run disjoint ranges on several threads.
 */
void oracle_decode_range(int format, const uint8_t *formats,
                         const uint8_t *comp, const uint64_t *comp_off,
                         uint8_t *out, const uint64_t *out_off,
                         int32_t *status, uint64_t first, uint64_t last);

/* Decoded size of chunks [first, last) in bytes (status per chunk). */
void oracle_sizes_range(int format, const uint8_t *formats,
                        const uint8_t *comp, const uint64_t *comp_off,
                        uint64_t *sizes, int32_t *status,
                        uint64_t first, uint64_t last);

#ifdef __cplusplus
}
#endif
#endif
