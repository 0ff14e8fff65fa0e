// ORC integer RLE v1 decoder (CODAG Sec. II-A, RLE v1; Sec. V-A evaluates
// the ORC form).  Stream format: control byte h (int8); h >= 0: run of h+3
// values = base + i*delta (int8 delta byte, base varint); h < 0: -h literal
// varints.  Signed columns zigzag base and literals.
//
// As for RLE v2, the plain kernels give a chunk one CTA whose warps decode
// group-aligned segments; the functions here decode one part with one warp.
//
// Work split inside the warp:
//   - group headers are read by every lane (identical state, Sec. IV-D);
//   - a varint is decoded from one 8-byte window with shifts and masks
//     instead of a byte-at-a-time loop;
//   - a literal group's varint boundaries are found warp-parallel: each lane
//     tests 4 bytes of a 128-byte window for the stop bit, __ballot_sync
//     gives a 128-bit terminator map, __popc ranks every terminator, and the
//     ranked end offsets go to shared memory; lane j then decodes varint j;
//   - when the chunk is staged whole, the CTA first builds a terminator
//     bitmap of it, so that skipping or splitting a literal group is a
//     rank/select over 32 words (1 KiB of stream) per warp step;
//   - runs are written by all lanes, value i = base + i*delta (the paper's
//     write_run primitive, Table 2), as coalesced 8-byte stores.
// Status order matches the oracle: header/varint problems in stream order
// (TRUNCATED, BAD_HEADER) before OUTPUT_OVERFLOW of the same group.
#pragma once

#include "ring.cuh"

namespace codag {

// shared scratch beyond the ring: u16 end offsets of up to 128 varints
constexpr int kRleV1Scratch = 128 * 2;

// Terminator bitmap of a chunk staged whole in shared memory: bit i of word t
// is set when stage byte 32t + i is a chunk byte below 0x80 (the last byte of
// a varint, or a header or delta byte).  With it, the k-th varint end after a
// position is a rank/select query instead of a byte scan.  A rank directory
// beside it holds, for every word, the set bits in all earlier words.
struct V1Bitmap {
  const uint32_t* bm;  // shared; nullptr: no bitmap (ring input)
  uint32_t off;        // stage position of position 0 of the input view
  uint32_t last_word;  // words from last_word on are zero (32 more are readable)
};

// Bitmap words a CTA builds for a chunk ending at stage position `end`.
__host__ __device__ __forceinline__ uint32_t v1_bitmap_words(uint32_t end) { return (end + 31) / 32 + 32; }

// Built by every warp of the CTA: warp w takes a block of words, one ballot
// per word, then ranks them with a warp scan; the block offsets come from the
// other warps' totals (`tot`: one shared word per warp).  Contains a CTA
// barrier; the caller synchronises the CTA again before use.
__device__ __forceinline__ void v1_build_bitmap(const uint8_t* stage, uint32_t skew, uint32_t n_in,
                                                uint32_t* bm, uint32_t* rk, uint32_t* tot) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t end = skew + n_in;
  const uint32_t words = v1_bitmap_words(end);
  const uint32_t per = ((words + nw - 1) / nw + 31) & ~31u;
  const uint32_t t_lo = warp * per;
  const uint32_t t_hi = t_lo + per < words ? t_lo + per : words;
  uint32_t run = 0;
  for (uint32_t t0 = t_lo; t0 < t_hi; t0 += 32) {
    uint32_t mine = 0;
    for (uint32_t k = 0; k < 32; k++) {
      const uint32_t p = 32 * (t0 + k) + lane;
      const uint32_t b = __ballot_sync(FULL, p >= skew && p < end && stage[p] < 0x80);
      if (lane == k) mine = b;
    }
    const uint32_t c = __popc(mine);
    const uint32_t incl = warp_incl_scan32(c);
    if (t0 + lane < t_hi) {
      bm[t0 + lane] = mine;
      rk[t0 + lane] = run + incl - c;
    }
    run += __shfl_sync(FULL, incl, 31);
  }
  if (lane == 0) tot[warp] = run;
  __syncthreads();
  uint32_t off = 0;
  for (uint32_t v = 0; v < warp; v++) off += tot[v];
  for (uint32_t t = t_lo + lane; t < t_hi; t += 32) rk[t] += off;
}

// Position (0..31) of the r-th set bit (r >= 1) of w, which has >= r set bits.
__device__ __forceinline__ uint32_t select_bit(uint32_t w, uint32_t r) {
  uint32_t pos = 0, c;
  c = __popc(w & 0xffffu);
  if (r > c) { r -= c; w >>= 16; pos += 16; }
  c = __popc(w & 0xffu);
  if (r > c) { r -= c; w >>= 8; pos += 8; }
  c = __popc(w & 0xfu);
  if (r > c) { r -= c; w >>= 4; pos += 4; }
  c = __popc(w & 0x3u);
  if (r > c) { r -= c; w >>= 2; pos += 2; }
  return pos + ((r > (w & 1u)) ? 1u : 0u);
}

// Decode the low 7-bit groups of an 8-byte window (byte k -> bits 7k..7k+6):
// drop the stop bits, then close the gaps pairwise, 7-bit groups into
// 14-bit, 14 into 28, 28 into 56, in three shift-and-merge steps.
__device__ __forceinline__ uint64_t varint_compact8(uint64_t x) {
  x &= 0x7f7f7f7f7f7f7f7full;
  x = (x & 0x007f007f007f007full) | ((x & 0x7f007f007f007f00ull) >> 1);
  x = (x & 0x00003fff00003fffull) | ((x & 0x3fff00003fff0000ull) >> 2);
  return (x & 0x000000000fffffffull) | ((x & 0x0fffffff00000000ull) >> 4);
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
                                                  V1Group& gr, const V1Bitmap& vb = V1Bitmap{nullptr, 0, 0}) {
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
  if (vb.bm) {
    // Fast path: the cnt varint ends from one window of 32 bitmap words
    // (1 KiB).  Lane j finds the word holding rank j by a binary search over
    // the warp's prefix counts, then the bit within it.  Groups that do not
    // end inside the window, or hold a varint longer than 10 bytes, take the
    // exact byte scan below, which also decides their status.
    const uint32_t sp = vb.off + (uint32_t)g;
    const uint32_t w0 = sp >> 5;
    uint32_t word = vb.bm[w0 + lane];
    if (lane == 0) word &= ~0u << (sp & 31);
    const uint32_t c = __popc(word);
    const uint32_t S = warp_incl_scan32(c);
    if (__shfl_sync(FULL, S, 31) >= (uint32_t)cnt) {
      const uint32_t excl = S - c;
      bool bad = false;
      uint32_t prev_end = sp - 1;
      for (uint32_t j0 = 0; j0 < (uint32_t)cnt; j0 += 32) {
        const uint32_t j = j0 + lane;
        uint32_t k = 0;
#pragma unroll
        for (uint32_t step = 16; step; step >>= 1)
          if (__shfl_sync(FULL, S, k + step - 1) <= j) k += step;
        const uint32_t wk = __shfl_sync(FULL, word, k);
        const uint32_t ek = __shfl_sync(FULL, excl, k);
        const uint32_t e = (w0 + k) * 32 + select_bit(wk, j - ek + 1);
        uint32_t prv = __shfl_up_sync(FULL, e, 1);
        if (lane == 0) prv = prev_end;
        if (j < (uint32_t)cnt) {
          ends[j] = (uint16_t)(e - sp);
          bad |= e - prv > 10;
        }
        prev_end = __shfl_sync(FULL, e, 31);
      }
      if (!__any_sync(FULL, bad)) {
        __syncwarp();
        gr.end = g + ends[cnt - 1] + 1;
        return ST_OK;
      }
      __syncwarp();
    }
  }
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
__device__ __forceinline__ bool rle_v1_walk(In& in, uint16_t* ends, int64_t n_in,
                                            const uint64_t* target, int nsplit, int64_t* split_pos,
                                            uint64_t* split_cnt,
                                            volatile uint32_t* published = nullptr) {
  int64_t pos = 0;
  uint64_t count = 0;
  int k = 1;
  bool waited_out = false;  // a staging wait ran out: the splits are not usable
  while (pos < n_in && k <= nsplit) {
    while (k <= nsplit && count >= target[k]) {
      publish_split(k, pos, count, split_pos, split_cnt, published);
      k++;
    }
    if (k > nsplit) break;
    if (!in.ensure(pos, pos + 24)) {
      waited_out = true;
      break;
    }
    V1Group gr;
    const int32_t st = v1_parse_group(in, pos, n_in, ends, gr);
    if (st != ST_OK) {
      waited_out = st == ST_TIMEOUT;
      break;
    }
    __syncwarp();
    count += gr.len;
    pos = gr.end;
  }
  for (; k <= nsplit; k++) publish_split(k, pos, count, split_pos, split_cnt, published);
  return !waited_out;
}

// Walk of a staged chunk (one warp) with its terminator bitmap and rank
// directory: same contract as rle_v1_walk, but a literal group is skipped in
// one step: its end is the (rank + cnt)-th set bit, whose word is the first
// with a directory entry that reaches that rank (one ballot over 32 words).
// The walk is lenient: it does not check varint lengths, and it stops at a
// group it cannot skip (the remaining splits get that position).  This is
// safe because a malformed stream decodes exactly like a well-formed one up
// to its first error: every group before it is skipped exactly, so the part
// containing the first error starts at or before it and reports it, and
// every later part starts after it, so the first error in stream order still
// wins when the part statuses are combined.
__device__ __forceinline__ void rle_v1_walk_staged(const StagedInput& in, const uint32_t* bm,
                                                   const uint32_t* rk, uint32_t n_in,
                                                   const uint64_t* target, int nsplit,
                                                   int64_t* split_pos, uint64_t* split_cnt,
                                                   volatile uint32_t* published) {
  const uint32_t lane = lane_id();
  const uint32_t skew = (uint32_t)in.skew;
  const uint32_t last_word = (skew + n_in + 31) >> 5;
  uint32_t pos = 0;
  uint64_t count = 0;
  int k = 1;
  uint64_t tk = target[1];
  while (pos < n_in) {
    if (count >= tk) {
      do {
        publish_split(k, pos, count, split_pos, split_cnt, published);
        if (++k > nsplit) return;
        tk = target[k];
      } while (count >= tk);
    }
    const int h = (int8_t)in.byte(pos);
    if (h >= 0) {  // run: header, delta byte, base varint
      if (pos + 2 >= n_in) break;
      uint64_t v;
      int vlen;
      if (varint_at(in, pos + 2, (int64_t)n_in - (pos + 2), &v, &vlen) != ST_OK) break;
      pos += 2 + (uint32_t)vlen;
      count += (uint32_t)h + 3;
    } else {  // literal group: the end of its -h-th varint
      const uint32_t sp = pos + 1 + skew;
      const uint32_t w0 = sp >> 5;
      const uint32_t T = rk[w0] + __popc(bm[w0] & ((1u << (sp & 31)) - 1u)) + (uint32_t)(-h);
      bool found = false;
      for (uint32_t wb = w0; wb < last_word; wb += 32) {
        const uint32_t t = wb + lane;
        const uint32_t hit = __ballot_sync(FULL, rk[t + 1] >= T);
        if (hit) {
          const uint32_t bit = select_bit(bm[t], T - rk[t]);  // meaningful in lane L only
          const int L = __ffs(hit) - 1;
          pos = (wb + (uint32_t)L) * 32 + __shfl_sync(FULL, bit, L) - skew + 1;
          found = true;
          break;
        }
      }
      if (!found) break;
      count += (uint32_t)(-h);
    }
  }
  for (; k <= nsplit; k++) publish_split(k, pos, count, split_pos, split_cnt, published);
}

// Group table of a staged chunk, for a walk that follows one shared-memory
// load per group: nx[p] = byte length | value count << 16 of a group whose
// header is at position p, for every position p < n_in (a header or not;
// the walk only reads the chain from position 0), or 0 where the group
// cannot be skipped (it runs past the chunk or spans more than 41 bitmap
// words).  Run: the base varint ends at the first terminator within 10 bytes
// after the delta byte.  Literal group: its end is the (rank + cnt)-th set
// bit, found by binary search over the rank directory.  Lenient like
// rle_v1_walk_staged.  Built by every thread of the CTA; the caller
// synchronises the CTA before use.
__device__ __forceinline__ void v1_build_next(const uint8_t* stage, uint32_t skew, uint32_t n_in,
                                              const uint32_t* bm, const uint32_t* rk,
                                              uint32_t last_word, uint32_t* nx) {
  for (uint32_t p = threadIdx.x; p < n_in; p += blockDim.x) {
    const uint32_t sp = skew + p;
    const uint32_t h = stage[sp];
    uint32_t v = 0;
    if (h < 0x80) {  // run: header, delta byte, base varint
      const uint32_t q = sp + 2;
      const uint32_t w = q >> 5;
      const uint64_t win = ((((uint64_t)bm[w + 1]) << 32) | bm[w]) >> (q & 31);
      const uint32_t t10 = (uint32_t)win & 0x3ffu;
      if (t10) v = (2u + (uint32_t)__ffs(t10)) | ((h + 3u) << 16);
    } else {  // literal group of 256 - h varints
      const uint32_t cnt = 256u - h;
      const uint32_t gq = sp + 1;
      const uint32_t w0 = gq >> 5;
      const uint32_t T = rk[w0] + __popc(bm[w0] & ((1u << (gq & 31)) - 1u)) + cnt;
      const uint32_t t_max = w0 + 41 < last_word + 30 ? w0 + 41 : last_word + 30;
      if (rk[t_max + 1] >= T) {
        uint32_t lo = w0, hi = t_max;  // smallest t in [lo, hi] with rk[t + 1] >= T
        while (lo < hi) {
          const uint32_t mid = (lo + hi) >> 1;
          if (rk[mid + 1] >= T) hi = mid;
          else lo = mid + 1;
        }
        const uint32_t e = lo * 32 + select_bit(bm[lo], T - rk[lo]);
        v = (e - sp + 1) | (cnt << 16);
      }
    }
    nx[p] = v;
  }
}

// Walk (one warp) along the group table; same contract as rle_v1_walk.
__device__ __forceinline__ void rle_v1_walk_next(const uint32_t* nx, uint32_t n_in,
                                                 const uint64_t* target, int nsplit,
                                                 int64_t* split_pos, uint64_t* split_cnt,
                                                 volatile uint32_t* published) {
  uint32_t pos = 0;
  uint64_t count = 0;
  int k = 1;
  uint64_t tk = target[1];
  while (pos < n_in) {
    if (count >= tk) {
      do {
        publish_split(k, pos, count, split_pos, split_cnt, published);
        if (++k > nsplit) return;
        tk = target[k];
      } while (count >= tk);
    }
    const uint32_t v = nx[pos];
    if (!v) break;
    count += v >> 16;
    pos += v & 0xffffu;
  }
  for (; k <= nsplit; k++) publish_split(k, pos, count, split_pos, split_cnt, published);
}

// Decode a literal group of cnt varints whose first byte is at view position
// g straight from the terminator bitmap: lane j finds the end of varint j
// (binary search over the warp's prefix counts, then the bit in the word),
// the previous lane's end gives its start, and the value is decoded and
// stored in the same step.  Returns false, having stored at most part of the
// group, when the group does not end within one 32-word window or holds a
// varint longer than 10 bytes; the caller then takes the exact path, which
// decides the status.  On success *end is the view position after the group.
template <class In>
__device__ __forceinline__ bool v1_literal_direct(const In& in, const V1Bitmap& vb, uint32_t g,
                                                  uint32_t cnt, bool is_signed,
                                                  uint64_t* __restrict__ o, int64_t* end) {
  const uint32_t lane = lane_id();
  const uint32_t sp = vb.off + g;
  const uint32_t w0 = sp >> 5;
  uint32_t word = vb.bm[w0 + lane];
  if (lane == 0) word &= ~0u << (sp & 31);
  const uint32_t c = __popc(word);
  const uint32_t S = warp_incl_scan32(c);
  if (__shfl_sync(FULL, S, 31) < cnt) return false;
  const uint32_t excl = S - c;
  bool bad = false;
  uint32_t prev_end = sp - 1, e = 0;
  for (uint32_t j0 = 0; j0 < cnt; j0 += 32) {
    const uint32_t j = j0 + lane;
    uint32_t k = 0;
#pragma unroll
    for (uint32_t step = 16; step; step >>= 1)
      if (__shfl_sync(FULL, S, k + step - 1) <= j) k += step;
    const uint32_t wk = __shfl_sync(FULL, word, k);
    const uint32_t ek = __shfl_sync(FULL, excl, k);
    e = (w0 + k) * 32 + select_bit(wk, j - ek + 1);
    uint32_t prv = __shfl_up_sync(FULL, e, 1);
    if (lane == 0) prv = prev_end;
    const uint32_t len = e - prv;
    if (j < cnt) {
      bad |= len > 10;
      if (len <= 10) {
        const int64_t s0 = (int64_t)(prv + 1 - vb.off);
        const uint64_t x = in.u64(s0);
        uint64_t v;
        if (len <= 8) {
          v = varint_compact8(x & lowmask64(8 * len));
        } else {
          const uint64_t y = in.u64(s0 + 8);
          v = varint_compact8(x) | ((y & 0x7full) << 56);
          if (len == 10) v |= ((y >> 8) & 0x1ull) << 63;
        }
        o[j] = is_signed ? unzigzag(v) : v;
      }
    }
    prev_end = __shfl_sync(FULL, e, 31);
  }
  if (__any_sync(FULL, bad)) return false;
  *end = (int64_t)__shfl_sync(FULL, e, (int)((cnt - 1) & 31)) - (int64_t)vb.off + 1;
  return true;
}

// Decode part of one RLE v1 chunk; same contract as rle_v2_part.
template <bool STORE, class In>
__device__ PartResult rle_v1_part(In& in, uint16_t* ends, int64_t n_in, bool is_signed,
                                  uint64_t* __restrict__ out, uint64_t cap_values, uint64_t count0,
                                  uint64_t hi_v, const V1Bitmap& vb = V1Bitmap{nullptr, 0, 0}) {
  const uint32_t lane = lane_id();
  const bool last = hi_v == ~0ull;
  int64_t pos = 0;
  uint64_t count = count0;
  while (pos < n_in) {
    if (count >= hi_v) return PartResult{ST_OK, -1, count};
    if (!in.ensure(pos, pos + 24)) return part_error(ST_TIMEOUT, 0, count);
    if (STORE && vb.bm) {  // staged chunk: literal groups straight from the bitmap
      const int h = (int8_t)in.byte(pos);
      if (h < 0 && count <= cap_values && (uint64_t)(-h) <= cap_values - count) {
        int64_t end;
        if (v1_literal_direct(in, vb, (uint32_t)pos + 1, (uint32_t)(-h), is_signed, out + count,
                              &end)) {
          count += (uint32_t)(-h);
          pos = end;
          continue;
        }
      }
    }
    V1Group gr;
    const int32_t st = v1_parse_group(in, pos, n_in, ends, gr, vb);
    if (st != ST_OK) return part_error(st, st == ST_TIMEOUT ? 0 : pos, count);
    if (count > cap_values || gr.len > cap_values - count) return part_error(ST_OVERFLOW, pos, count);
    if (STORE) {
      uint64_t* o = out + count;
      if (!gr.literal) {
        const uint64_t base = is_signed ? unzigzag(gr.base) : gr.base;
        uint64_t v = base + (uint64_t)lane * (uint64_t)gr.delta;  // value i = base + i * delta
        const uint64_t step = 32ull * (uint64_t)gr.delta;
        for (uint32_t i = lane; i < gr.len; i += 32, v += step) o[i] = v;
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
