// ORC compressed streams with zlib compression: a sequence of compression
// chunks, each a 3-byte little-endian header v (v >> 1 body bytes follow;
// bit 0 set: stored as is, clear: a raw Deflate stream) and its body; the
// output is the bodies' decoded bytes one after another.  CODAG decodes data
// as existing systems store it (Sec. I, Sec. II-B); this is how ORC stores
// a compressed column stream.  One warp per stream: the bodies are decoded
// in order, each compressed one by the Deflate decoder through a view of
// the staging ring that starts at the body (the ring only moves forward).
// Readings: every compressed body is a complete Deflate stream of its own
// (no shared window; bytes after its final block are ignored); a header or
// body that runs past the stream is TRUNCATED; a bad body reports its
// Deflate status; the stream must fill its output span.
#pragma once

#include "kernels.cuh"

namespace codag {

template <bool STORE, class Ring>
__device__ PartResult orc_zlib_decode(Ring& ring, uint8_t* scratch, int64_t n_in,
                                      uint8_t* __restrict__ out, uint64_t cap) {
  const uint32_t lane = lane_id();
  const uint64_t limit = STORE ? cap : ~0ull;
  int64_t pos = 0;
  uint64_t count = 0;
  while (pos < n_in) {
    if (n_in - pos < 3) return part_error(ST_TRUNCATED, pos, count);
    if (!ring.ensure(pos, pos + 3)) return part_error(ST_TIMEOUT, 0, count);
    const uint32_t v = (uint32_t)ring.byte(pos) | ((uint32_t)ring.byte(pos + 1) << 8) |
                       ((uint32_t)ring.byte(pos + 2) << 16);
    const int64_t body = pos + 3;
    const int64_t len = (int64_t)(v >> 1);
    if (n_in - body < len) return part_error(ST_TRUNCATED, pos, count);
    if (v & 1u) {  // stored body
      if ((uint64_t)len > limit - count) return part_error(ST_OVERFLOW, pos, count);
      if (STORE) {
        constexpr int64_t PIECE = Ring::MAX_SPAN - 16 < 512 ? Ring::MAX_SPAN - 16 : 512;
        for (int64_t k0 = 0; k0 < len; k0 += PIECE) {
          const int64_t piece = len - k0 < PIECE ? len - k0 : PIECE;
          if (!ring.ensure(body + k0, body + k0 + piece)) return part_error(ST_TIMEOUT, 0, count);
          for (int64_t k = lane; k < piece; k += 32) out[count + k0 + k] = ring.byte(body + k0 + k);
        }
        __syncwarp();
      }
      count += (uint64_t)len;
    } else {  // raw Deflate body into what is left of the span
      OffsetRing<Ring> sub;
      sub.in = &ring;
      sub.base = body;
      uint64_t prod = 0;
      int32_t st = inflate_decode<STORE, kLitTB, kDistTB, kWin>(sub, scratch, len, out + count,
                                                               limit - count, &prod);
      if (st == ST_UNDERFLOW) st = ST_OK;  // the span continues with the next body
      if (st != ST_OK) return part_error(st, st == ST_TIMEOUT ? 0 : pos, count + prod);
      count += prod;
    }
    pos = body + len;
  }
  if (STORE && count < cap) return part_error(ST_UNDERFLOW, n_in, count);
  return PartResult{ST_OK, -1, count};
}

}  // namespace codag
