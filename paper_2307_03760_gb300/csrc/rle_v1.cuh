// ORC integer RLE v1 decoder, one warp per chunk (CODAG Sec. II-A, RLE v1;
// Sec. VI-A evaluates the ORC form).  Stream format: control byte h (int8);
// h >= 0: run of h+3 values = base + i*delta (int8 delta byte, base varint);
// h < 0: -h literal varints.  Signed columns zigzag base and literals.
//
// Work split inside the warp:
//   - group headers are read by every lane (identical state, Sec. V-D);
//   - a varint is decoded from one 8-byte window with shifts and masks
//     instead of a byte-at-a-time loop;
//   - a literal group's varint boundaries are found warp-parallel: each lane
//     tests 4 bytes of a 128-byte window for the stop bit, __ballot_sync
//     gives a 128-bit terminator map, __popc ranks every terminator, and the
//     ranked end offsets go to shared memory; lane j then decodes varint j;
//   - runs are written by all lanes, value i = base + i*delta (the paper's
//     write_run primitive, Table 2), as coalesced 8-byte stores.
// Status order matches the oracle: header/varint problems in stream order
// (TRUNCATED, BAD_HEADER) before OUTPUT_OVERFLOW of the same group.
#pragma once

#include "ring.cuh"

namespace codag {

// shared scratch beyond the ring: u16 end offsets of up to 128 varints
constexpr int kRleV1Scratch = 128 * 2;

// Decode the low 7-bit groups of an 8-byte window (byte k -> bits 7k..7k+6).
__device__ __forceinline__ uint64_t varint_compact8(uint64_t x) {
  return (x & 0x7full) | ((x >> 1) & (0x7full << 7)) | ((x >> 2) & (0x7full << 14)) |
         ((x >> 3) & (0x7full << 21)) | ((x >> 4) & (0x7full << 28)) |
         ((x >> 5) & (0x7full << 35)) | ((x >> 6) & (0x7full << 42)) |
         ((x >> 7) & (0x7full << 49));
}

// Varint at chunk position p (bytes resident through p+16).  Returns a status;
// on success *v and *len (1..10).  `avail` = chunk bytes from p to the end.
template <class Ring>
__device__ __forceinline__ int32_t varint_at(const Ring& ring, int64_t p, int64_t avail,
                                             uint64_t* v, int* len) {
  const uint64_t x = ring.u64(p);
  uint64_t term = ~x & 0x8080808080808080ull;
  if (avail < 8) term &= lowmask64(8 * (uint32_t)(avail < 0 ? 0 : avail));
  if (term) {
    const int k = (__ffsll((long long)term) - 1) >> 3;  // terminator byte index
    *len = k + 1;
    *v = varint_compact8(x & lowmask64(8 * (k + 1)));
    return ST_OK;
  }
  if (avail <= 8) return ST_TRUNCATED;
  const uint64_t y = ring.u64(p + 8);
  uint64_t t2 = ~y & 0x8080ull;
  if (avail < 10) t2 &= lowmask64(8 * (uint32_t)(avail - 8));
  if (!t2) return avail >= 10 ? ST_BAD_HEADER : ST_TRUNCATED;
  const int k = (__ffsll((long long)t2) - 1) >> 3;  // 0 or 1
  *len = 9 + k;
  uint64_t r = varint_compact8(x) | ((y & 0x7full) << 56);
  if (k == 1) r |= ((y >> 8) & 0x1ull) << 63;
  *v = r;
  return ST_OK;
}

// One group's header and extent.  For a literal group the varint ends are
// left in `ends` (offsets from the group's first varint byte).  Returns
// ST_OK, ST_TRUNCATED or ST_BAD_HEADER; the ring must be positioned so that
// `in.ensure` can bring in the group.
struct V1Group {
  int literal;      // 1: -h literals, 0: a run
  uint32_t len;     // values
  int64_t g;        // literal: first varint byte
  int64_t end;      // end of the group
  uint64_t base;    // run: base (not yet unzigzagged)
  int64_t delta;    // run: delta
};

template <class In>
__device__ __forceinline__ int32_t v1_parse_group(In& in, int64_t pos, int64_t n_in, uint16_t* ends,
                                                  V1Group& gr) {
  const uint32_t lane = lane_id();
  const uint64_t w = in.u64(pos);
  const int h = (int8_t)(w & 0xff);
  if (h >= 0) {
    gr.literal = 0;
    gr.len = (uint32_t)h + 3;
    if (pos + 1 >= n_in) return ST_TRUNCATED;
    gr.delta = (int8_t)((w >> 8) & 0xff);
    int vlen;
    const int32_t st = varint_at(in, pos + 2, n_in - (pos + 2), &gr.base, &vlen);
    gr.end = pos + 2 + vlen;
    return st;
  }
  gr.literal = 1;
  const int cnt = -h;
  gr.len = (uint32_t)cnt;
  const int64_t g = pos + 1;  // first varint byte
  gr.g = g;
  const int64_t avail = n_in - g;
  const int64_t span = avail < 1280 + 128 ? avail : 1280 + 128;
  if (span > 0 && !in.ensure(g, g + span)) return ST_TIMEOUT;
  // 1. find up to cnt varint terminators, 128 bytes per step
  int found = 0;
  int64_t p = g;
  bool no_stop = false;
  while (found < cnt && p < n_in && p - g <= 1280) {
    uint32_t T[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
      const int64_t q = p + lane + 32 * m;
      const uint8_t b = q < n_in ? in.byte(q) : 0x80;
      T[m] = __ballot_sync(FULL, b < 0x80);
    }
    const int c0 = __popc(T[0]), c1 = __popc(T[1]), c2 = __popc(T[2]), c3 = __popc(T[3]);
    const int total = c0 + c1 + c2 + c3;
    if (total == 0) {
      no_stop = true;
      break;
    }
#pragma unroll
    for (int m = 0; m < 4; m++) {
      if ((T[m] >> lane) & 1u) {
        const int before = m == 0 ? 0 : m == 1 ? c0 : m == 2 ? c0 + c1 : c0 + c1 + c2;
        const int idx = found + before + __popc(T[m] & lanemask_lt());
        if (idx < cnt) ends[idx] = (uint16_t)(p + lane + 32 * m - g);
      }
    }
    found += total < cnt - found ? total : cnt - found;
    __syncwarp();
    p = g + ends[found - 1] + 1;
  }
  __syncwarp();
  // 2. every varint is at most 10 bytes; the first bad one in stream order
  for (int j0 = 0; j0 < found; j0 += 32) {
    const int j = j0 + (int)lane;
    bool bad = false;
    if (j < found) {
      const int s = j == 0 ? 0 : ends[j - 1] + 1;
      bad = ends[j] - s + 1 > 10;
    }
    if (__ballot_sync(FULL, bad)) return ST_BAD_HEADER;
  }
  if (found < cnt) {
    const int64_t seen = no_stop ? ((n_in - p) < 128 ? (n_in - p) : 128) : (n_in - p);
    if (p - g > 1280) return ST_BAD_HEADER;
    return seen >= 10 ? ST_BAD_HEADER : ST_TRUNCATED;
  }
  gr.end = g + ends[cnt - 1] + 1;
  return ST_OK;
}

// When `published` is given, split k is made visible to the CTA's other
// warps as soon as it is known (*published = k + 1 after a block fence).
__device__ __forceinline__ void publish_split(int k, int64_t pos, uint64_t count, int64_t* split_pos,
                                              uint64_t* split_cnt, volatile uint32_t* published) {
  if (lane_id() == 0) {
    split_pos[k] = pos;
    split_cnt[k] = count;
    if (published) {
      __threadfence_block();
      *published = (uint32_t)k + 1;
    }
  }
}

// Walk an RLE v1 stream's groups (one warp) and record where parts start;
// same contract as rle_v2_walk.
template <class In>
__device__ __forceinline__ void rle_v1_walk(In& in, uint16_t* ends, int64_t n_in,
                                            const uint64_t* target, int nsplit, int64_t* split_pos,
                                            uint64_t* split_cnt,
                                            volatile uint32_t* published = nullptr) {
  int64_t pos = 0;
  uint64_t count = 0;
  int k = 1;
  while (pos < n_in && k <= nsplit) {
    while (k <= nsplit && count >= target[k]) {
      publish_split(k, pos, count, split_pos, split_cnt, published);
      k++;
    }
    if (k > nsplit) break;
    if (!in.ensure(pos, pos + 24)) break;
    V1Group gr;
    if (v1_parse_group(in, pos, n_in, ends, gr) != ST_OK) break;
    __syncwarp();
    count += gr.len;
    pos = gr.end;
  }
  for (; k <= nsplit; k++) publish_split(k, pos, count, split_pos, split_cnt, published);
}

// Decode part of one RLE v1 chunk; same contract as rle_v2_part.
template <bool STORE, class In>
__device__ PartResult rle_v1_part(In& in, uint16_t* ends, int64_t n_in, bool is_signed,
                                  uint64_t* __restrict__ out, uint64_t cap_values, uint64_t count0,
                                  uint64_t hi_v) {
  const uint32_t lane = lane_id();
  const bool last = hi_v == ~0ull;
  int64_t pos = 0;
  uint64_t count = count0;
  while (pos < n_in) {
    if (count >= hi_v) return PartResult{ST_OK, -1, count};
    if (!in.ensure(pos, pos + 24)) return part_error(ST_TIMEOUT, 0, count);
    V1Group gr;
    const int32_t st = v1_parse_group(in, pos, n_in, ends, gr);
    if (st != ST_OK) return part_error(st, st == ST_TIMEOUT ? 0 : pos, count);
    if (count > cap_values || gr.len > cap_values - count) return part_error(ST_OVERFLOW, pos, count);
    if (STORE) {
      uint64_t* o = out + count;
      if (!gr.literal) {
        const uint64_t base = is_signed ? unzigzag(gr.base) : gr.base;
        for (uint32_t i = lane; i < gr.len; i += 32) o[i] = base + (uint64_t)i * (uint64_t)gr.delta;
      } else {
        for (int j = (int)lane; j < (int)gr.len; j += 32) {  // lane j decodes varint j
          const int s = j == 0 ? 0 : ends[j - 1] + 1;
          uint64_t v;
          int vlen;
          varint_at(in, gr.g + s, n_in - (gr.g + s), &v, &vlen);
          o[j] = is_signed ? unzigzag(v) : v;
        }
      }
    }
    count += gr.len;
    pos = gr.end;
    __syncwarp();
  }
  if (last && STORE && count < cap_values) return part_error(ST_UNDERFLOW, n_in, count);
  return PartResult{ST_OK, -1, count};
}

}  // namespace codag
