// ORC byte RLE and boolean RLE, one warp per chunk.  CODAG Sec. V-A: other
// encodings are enabled through the same structure (a chunk per decoding
// unit, the staged input stream, warp-wide writes); ORC's byte run-length
// encoding is one.  Stream format: control byte h (int8); h >= 0: the next
// byte repeated h + 3 times; h < 0: -h literal bytes.  Boolean RLE is byte
// RLE over bytes of eight booleans, most significant bit first; it is
// written out as one 0/1 byte per boolean, and its output span is the
// number of booleans (the stream must decode to exactly ceil(span / 8)
// bytes; the unused low bits of the last byte are dropped).
//
// Work split: as a plain call, a CTA takes a chunk (like the integer RLE
// kernels): one warp walks the control bytes and publishes segment starts,
// every warp decodes segments; in the batch kernel a warp takes a chunk.
// Inside a warp every lane reads the control byte (identical state); a run's
// bytes and a literal group's bytes are written by all lanes, lane i taking
// byte i (booleans: output byte i), as coalesced stores.
// Status order matches the oracle: TRUNCATED before OUTPUT_OVERFLOW of the
// same group; there is no BAD_HEADER (every control byte is valid).
#pragma once

#include "rle_v1.cuh"  // publish_split

namespace codag {

// Decode part of one chunk (n_in bytes through `in`, starting at a group
// boundary whose first decoded byte is count0) into out, through the groups
// that start before decoded byte hi_v (hi_v = ~0: to the end of the stream,
// and report OUTPUT_UNDERFLOW).  cap: the output span in bytes (booleans: in
// booleans); STORE = false sizes the stream.  count of the result: output
// bytes (or booleans).  Error positions are relative to the part's start.
template <bool STORE, class In>
__device__ PartResult byte_rle_part(In& in, int64_t n_in, bool bools, uint8_t* __restrict__ out,
                                    uint64_t cap, uint64_t count0, uint64_t hi_v) {
  const uint32_t lane = lane_id();
  const uint64_t cap_bytes = !STORE ? ~0ull : bools ? cap / 8 + ((cap & 7) ? 1 : 0) : cap;
  const bool last = hi_v == ~0ull;
  int64_t pos = 0;
  uint64_t count = count0;  // decoded bytes
  while (pos < n_in) {
    if (count >= hi_v) return PartResult{ST_OK, -1, bools ? 8 * count : count};
    const int64_t want = n_in - pos < 130 ? n_in - pos : 130;
    if (!in.ensure(pos, pos + want)) return part_error(ST_TIMEOUT, 0, count);
    const int h = (int8_t)in.byte(pos);
    const uint32_t len = h >= 0 ? (uint32_t)h + 3 : (uint32_t)(-h);
    const int64_t src = pos + 1;  // run: the value byte; literals: the first byte
    if (h >= 0 ? src >= n_in : n_in - src < (int64_t)len)
      return part_error(ST_TRUNCATED, pos, bools ? 8 * count : count);
    if (count > cap_bytes || len > cap_bytes - count)
      return part_error(ST_OVERFLOW, pos, bools ? 8 * count : count);
    if (STORE) {
      const uint32_t v = in.byte(src);
      if (!bools) {
        uint8_t* o = out + count;
        if (h >= 0) {
          for (uint32_t i = lane; i < len; i += 32) o[i] = (uint8_t)v;
        } else {  // every lane reads in every step (a register ring reads by shuffles)
          for (uint32_t ib = 0; ib < len; ib += 32) {
            const uint32_t i = ib + lane;
            const uint8_t b = in.byte(src + (i < len ? i : len - 1));
            if (i < len) o[i] = b;
          }
        }
      } else {
        const uint64_t lo = 8 * count;
        const uint64_t hi = 8 * (count + len) < cap ? 8 * (count + len) : cap;
        for (uint64_t jb = lo; jb < hi; jb += 32) {
          const uint64_t j = jb + lane;
          const uint64_t jj = j < hi ? j : hi - 1;
          const uint32_t b = h >= 0 ? v : in.byte(src + (int64_t)(jj / 8 - count));
          if (j < hi) out[j] = (uint8_t)((b >> (7 - (uint32_t)(j & 7))) & 1u);
        }
      }
    }
    pos = h >= 0 ? src + 1 : src + len;
    count += len;
  }
  if (last && STORE && count < cap_bytes)
    return part_error(ST_UNDERFLOW, n_in, bools ? 8 * count : count);
  return PartResult{ST_OK, -1, bools ? 8 * count : count};
}

// One whole chunk (one warp).
template <bool STORE, class In>
__device__ __forceinline__ PartResult byte_rle_decode(In& in, int64_t n_in, bool bools,
                                                      uint8_t* __restrict__ out, uint64_t cap) {
  return byte_rle_part<STORE>(in, n_in, bools, out, cap, 0, ~0ull);
}

// Walk a chunk's control bytes (one warp) and record where parts start, in
// decoded bytes; same contract as rle_v1_walk.  A group's extent follows from
// its control byte alone, so the walk reads one byte per group.  Lenient like
// rle_v1_walk_staged: it does not check that a group's bytes are present.
template <class In>
__device__ __forceinline__ bool byte_rle_walk(In& in, int64_t n_in, const uint64_t* target, int nsplit,
                                              int64_t* split_pos, uint64_t* split_cnt,
                                              volatile uint32_t* published = nullptr) {
  int64_t pos = 0;
  uint64_t count = 0;
  int k = 1;
  uint64_t tk = target[1];
  bool waited_out = false;  // a staging wait ran out: the splits are not usable
  while (pos < n_in) {
    if (count >= tk) {
      do {
        publish_split(k, pos, count, split_pos, split_cnt, published);
        if (++k > nsplit) return true;
        tk = target[k];
      } while (count >= tk);
    }
    if (!in.ensure(pos, pos + 1)) {
      waited_out = true;
      break;
    }
    const int h = (int8_t)in.byte(pos);
    count += h >= 0 ? (uint32_t)h + 3 : (uint32_t)(-h);
    pos += h >= 0 ? 2 : 1 - h;
  }
  for (; k <= nsplit; k++) publish_split(k, pos, count, split_pos, split_cnt, published);
  return !waited_out;
}

}  // namespace codag
