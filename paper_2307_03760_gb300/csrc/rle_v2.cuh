// ORC integer RLE v2 decoder (CODAG Sec. II-A, RLE v2; Sec. V-A evaluates
// the ORC form).  The top two bits of a run's first byte select
// SHORT_REPEAT / DIRECT / PATCHED_BASE / DELTA.
//
// A chunk is decoded by one CTA in the plain kernels (a walk over the run
// headers cuts it into segments at run boundaries, and each warp decodes the
// segments it claims) and by one or more warps in the batch kernel.  The
// functions here decode one part (a run-aligned sub-stream) with one warp.
//
// Work split inside the warp:
//   - run headers are parsed by every lane (identical state);
//   - bit-packed sections (MSB first, widths 1..64) are unpacked 32 values at
//     a time, lane i taking value i: one unaligned 8-byte read from the
//     staging ring, a byte swap and two shifts (any width <= 64 fits: widths
//     that are not multiples of 8 are <= 30 bits);
//   - PATCHED_BASE patch entries are decoded one per lane, their positions
//     are a warp prefix sum of the gaps; a run of values up to 25 bits is
//     unpacked like a DIRECT run and each patch-holding lane then rewrites
//     its value, wider runs mark patched values in a 512-bit shared bitmap
//     for the unpack loop;
//   - DELTA runs are a warp-wide inclusive prefix sum per 32 deltas
//     (__shfl_up_sync), carried across pieces;
//   - outputs are coalesced 8-byte stores.
// Status order matches the oracle: field problems in stream order, then
// OUTPUT_OVERFLOW of the same run.
#pragma once

#include "rle_v1.cuh"  // varint_at
#include "ring.cuh"

namespace codag {

// shared scratch beyond the ring: 16-word patch bitmap + 32 patch values
constexpr int kRleV2Scratch = 16 * 4 + 32 * 8;

// 5-bit encoded width -> bits
__device__ __forceinline__ int v2_width(int code) {
  return code < 24 ? code + 1 : (code < 27 ? 26 + 2 * (code - 24) : 32 + 8 * (code - 27));
}

// smallest encodable width >= n
__device__ __forceinline__ int v2_closest_fixed_bits(int n) {
  if (n <= 1) return 1;
  if (n <= 24) return n;
  if (n <= 32) return (n + 1) & ~1;
  return (n + 7) & ~7;
}

// value i (width w) of a packed section starting at chunk position sec
template <class Ring>
__device__ __forceinline__ uint64_t v2_unpack(const Ring& ring, int64_t sec, uint64_t i, int w) {
  const uint64_t bit = i * (uint64_t)w;
  const uint64_t x = load_be64(ring, sec + (int64_t)(bit >> 3));
  return (x << (bit & 7)) >> (64 - w);
}

// value at bit offset `bit` (width w <= 25) of a packed section at chunk
// position sec: one unaligned big-endian 4-byte read and two 32-bit shifts
template <class In>
__device__ __forceinline__ uint32_t v2_unpack32(const In& in, uint32_t sec, uint32_t bit, int w) {
  const uint32_t x = load_be32(in, sec + (bit >> 3));
  return (x << (bit & 7)) >> (32 - w);
}

// Four consecutive w-bit fields (w <= 14) starting at bit `bit` of a packed
// section at chunk position sec: one unaligned 8-byte read; after the
// sub-byte shift 57 bits remain, enough for 4 x 14.  The first two fields are
// the top 2w bits of the high word, the last two the top 2w bits of the word
// that starts 2w bits further on.
template <class In>
__device__ __forceinline__ void v2_unpack4(const In& in, uint32_t sec, uint32_t bit, int w, uint32_t& v0,
                                           uint32_t& v1, uint32_t& v2, uint32_t& v3) {
  const uint64_t x = load_be64(in, sec + (bit >> 3)) << (bit & 7);
  const uint32_t hi = (uint32_t)(x >> 32);
  const uint32_t mid = (uint32_t)(x >> (32 - 2 * w));
  v0 = hi >> (32 - w);
  v1 = (hi << w) >> (32 - w);
  v2 = mid >> (32 - w);
  v3 = (mid << w) >> (32 - w);
}

__device__ __forceinline__ uint64_t unzigzag32(uint32_t v) {
  return (uint64_t)(int64_t)(int32_t)((v >> 1) ^ (0u - (v & 1u)));
}

// One run's header fields and byte extent (everything that the header alone
// decides).  Returns ST_OK, ST_TRUNCATED or ST_BAD_HEADER.
struct V2Run {
  uint32_t enc, len;
  int w;
  int64_t sec, nbytes, end;    // data section, its size, end of the run
  int bw, pw, pll, ew;         // PATCHED_BASE
  int64_t psec, pbytes;
  uint64_t basev, dz;          // DELTA base and zigzagged delta base
  uint32_t b0;
};

template <class In>
__device__ __forceinline__ int32_t v2_parse_run(const In& in, int64_t pos, int64_t n_in, V2Run& r) {
  const uint64_t hdr = in.u64(pos);
  const uint32_t b0 = (uint32_t)(hdr & 0xff);
  r.b0 = b0;
  r.enc = b0 >> 6;
  if (r.enc == 0) {  // SHORT_REPEAT
    const int nb = ((b0 >> 3) & 7) + 1;
    r.len = (b0 & 7) + 3;
    r.w = nb;
    r.end = pos + 1 + nb;
    return r.end > n_in ? ST_TRUNCATED : ST_OK;
  }
  if (pos + 2 > n_in) return ST_TRUNCATED;
  const uint32_t b1 = (uint32_t)((hdr >> 8) & 0xff);
  const int wcode = (b0 >> 1) & 31;
  r.len = (((b0 & 1) << 8) | b1) + 1;
  if (r.enc == 1) {  // DIRECT
    r.w = v2_width(wcode);
    r.sec = pos + 2;
    r.nbytes = ((int64_t)r.len * r.w + 7) >> 3;
    r.end = r.sec + r.nbytes;
    return r.end > n_in ? ST_TRUNCATED : ST_OK;
  }
  if (r.enc == 2) {  // PATCHED_BASE
    r.w = v2_width(wcode);
    if (pos + 4 > n_in) return ST_TRUNCATED;
    const uint32_t b2 = (uint32_t)((hdr >> 16) & 0xff);
    const uint32_t b3 = (uint32_t)((hdr >> 24) & 0xff);
    r.bw = (b2 >> 5) + 1;
    r.pw = v2_width(b2 & 31);
    const int pgw = (b3 >> 5) + 1;
    r.pll = b3 & 31;
    if (pgw + r.pw > 64) return ST_BAD_HEADER;
    if (pos + 4 + r.bw > n_in) return ST_TRUNCATED;
    r.sec = pos + 4 + r.bw;
    r.nbytes = ((int64_t)r.len * r.w + 7) >> 3;
    if (r.sec + r.nbytes > n_in) return ST_TRUNCATED;
    r.ew = v2_closest_fixed_bits(pgw + r.pw);
    r.psec = r.sec + r.nbytes;
    r.pbytes = ((int64_t)r.pll * r.ew + 7) >> 3;
    r.end = r.psec + r.pbytes;
    return r.end > n_in ? ST_TRUNCATED : ST_OK;
  }
  // DELTA
  r.w = wcode == 0 ? 0 : v2_width(wcode);
  int l1, l2;
  int32_t st = varint_at(in, pos + 2, n_in - (pos + 2), &r.basev, &l1);
  if (st != ST_OK) return st;
  st = varint_at(in, pos + 2 + l1, n_in - (pos + 2 + l1), &r.dz, &l2);
  if (st != ST_OK) return st;
  r.sec = pos + 2 + l1 + l2;
  r.nbytes = (r.w != 0 && r.len >= 2) ? ((int64_t)(r.len - 2) * r.w + 7) >> 3 : 0;
  r.end = r.sec + r.nbytes;
  return r.end > n_in ? ST_TRUNCATED : ST_OK;
}

// Walk an RLE v2 stream's run headers (one warp, identical state in every
// lane) and record where parts start: for k = 1..nsplit, the first run whose
// first value index is >= target[k].  Where the walk stops early (a header
// error, or the end of the stream) the remaining splits get that position,
// so the last part finds the error again.  split_pos / split_cnt: shared.
// Returns false when a staging wait ran out (the splits are then unusable).
template <class In>
__device__ __forceinline__ bool rle_v2_walk(In& in, int64_t n_in, const uint64_t* target,
                                            int nsplit, int64_t* split_pos, uint64_t* split_cnt,
                                            volatile uint32_t* published = nullptr) {
  int64_t pos = 0;
  uint64_t count = 0;
  int k = 1;
  bool waited_out = false;
  while (pos < n_in && k <= nsplit) {
    while (k <= nsplit && count >= target[k]) {
      publish_split(k, pos, count, split_pos, split_cnt, published);
      k++;
    }
    if (k > nsplit) break;
    if (!in.ensure(pos, pos + 40)) {
      waited_out = true;
      break;
    }
    V2Run r;
    if (v2_parse_run(in, pos, n_in, r) != ST_OK) break;
    count += r.len;
    pos = r.end;
  }
  for (; k <= nsplit; k++) publish_split(k, pos, count, split_pos, split_cnt, published);
  return !waited_out;
}

// Extent of the run at pos for the staged walk: its value count and end,
// from the header bytes alone, without the field checks of v2_parse_run
// (lenient, like rle_v1_walk_staged: exact on well-formed runs, and the part
// decoders check every run).  Returns false where it cannot tell (a DELTA
// varint that is malformed or runs past the chunk); the caller stops there.
template <class In>
__device__ __forceinline__ bool v2_run_extent(const In& in, uint32_t pos, uint32_t n_in, uint32_t* len,
                                              uint32_t* end) {
  const uint64_t hdr = in.u64(pos);
  const uint32_t b0 = (uint32_t)hdr & 0xffu;
  const uint32_t enc = b0 >> 6;
  if (enc == 0) {
    *len = (b0 & 7) + 3;
    *end = pos + 2 + ((b0 >> 3) & 7);
    return true;
  }
  const uint32_t L = ((((b0 & 1) << 8) | ((uint32_t)(hdr >> 8) & 0xffu))) + 1;
  const uint32_t code = (b0 >> 1) & 31;
  const uint32_t w = (enc == 3 && code == 0) ? 0u : (uint32_t)v2_width((int)code);
  *len = L;
  if (enc == 1) {
    *end = pos + 2 + ((L * w + 7) >> 3);
    return true;
  }
  if (enc == 2) {
    const uint32_t b2 = (uint32_t)(hdr >> 16) & 0xffu, b3 = (uint32_t)(hdr >> 24) & 0xffu;
    const uint32_t ew = (uint32_t)v2_closest_fixed_bits((int)((b3 >> 5) + 1) + v2_width((int)(b2 & 31)));
    *end = pos + 4 + ((b2 >> 5) + 1) + ((L * w + 7) >> 3) + (((b3 & 31) * ew + 7) >> 3);
    return true;
  }
  // DELTA: header, base varint, delta-base varint, packed deltas
  const uint64_t x = in.u64(pos + 2);
  const uint64_t t1 = ~x & 0x8080808080808080ull;
  const uint64_t t2 = t1 & (t1 - 1);
  uint32_t vb;  // bytes of both varints
  if (t2) {
    vb = (uint32_t)(__ffsll((long long)t2) >> 3);
  } else {  // longer than the 8-byte window
    uint64_t v;
    int l1, l2;
    if (varint_at(in, pos + 2, (int64_t)n_in - (pos + 2), &v, &l1) != ST_OK) return false;
    if (varint_at(in, pos + 2 + l1, (int64_t)n_in - (pos + 2 + l1), &v, &l2) != ST_OK) return false;
    vb = (uint32_t)(l1 + l2);
  }
  *end = pos + 2 + vb + ((w != 0 && L >= 2) ? (((L - 2) * w + 7) >> 3) : 0u);
  return true;
}

// Staged walk (one warp) with v2_run_extent; same contract as rle_v2_walk.
// Safe for the reason given at rle_v1_walk_staged: runs before the first
// malformed one are skipped exactly.
template <class In>
__device__ __forceinline__ void rle_v2_walk_staged(const In& in, uint32_t n_in, const uint64_t* target,
                                                   int nsplit, int64_t* split_pos, uint64_t* split_cnt,
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
    uint32_t len, end;
    if (!v2_run_extent(in, pos, n_in, &len, &end)) break;
    count += len;
    pos = end;
  }
  for (; k <= nsplit; k++) publish_split(k, pos, count, split_pos, split_cnt, published);
}

// Width of a 5-bit width code, in four integer operations.
__device__ __forceinline__ uint32_t v2_width_u(uint32_t code) {
  const uint32_t wide = code < 27u ? 2u * code - 22u : 8u * code - 184u;
  return code < 24u ? code + 1u : wide;
}

// The staged walk of rle_v2_walk_staged with every step in 32-bit arithmetic
// straight from the stage words: the walk is one dependent chain per chunk
// (the critical path of its CTA), so each run costs as few dependent
// instructions as the header allows.  Same splits, same stop rule (a DELTA
// varint that v2_run_extent could not size ends the walk).  Needs value
// counts below 2^32 (targets in 32 bits).
__device__ __forceinline__ void rle_v2_walk_lean(const StagedInput& in, uint32_t n_in,
                                                 const uint64_t* target, uint32_t nseg,
                                                 int64_t* split_pos, uint64_t* split_cnt,
                                                 volatile uint32_t* published) {
  const uint8_t* buf = in.buf;
  const uint32_t skew = (uint32_t)in.skew;
  uint32_t pos = 0, count = 0, k = 1;
  uint32_t tk = (uint32_t)target[1];
  while (pos < n_in) {
    if (count >= tk) {
      do {
        publish_split((int)k, pos, count, split_pos, split_cnt, published);
        if (++k >= nseg) return;
        tk = (uint32_t)target[k];
      } while (count >= tk);
    }
    const uint32_t r = pos + skew;
    const uint32_t* wp = reinterpret_cast<const uint32_t*>(buf + (r & ~3u));
    const uint32_t h = __funnelshift_r(wp[0], wp[1], (r & 3u) << 3);  // bytes pos .. pos+3
    const uint32_t enc = (h >> 6) & 3u;
    uint32_t len, ext;
    if (enc == 0) {  // SHORT_REPEAT: header + value bytes
      len = (h & 7u) + 3u;
      ext = ((h >> 3) & 7u) + 2u;
    } else {
      len = (((h & 1u) << 8) | ((h >> 8) & 0xffu)) + 1u;
      const uint32_t code = (h >> 1) & 31u;
      if (enc == 1) {  // DIRECT
        ext = 2u + ((len * v2_width_u(code) + 7u) >> 3);
      } else if (enc == 2) {  // PATCHED_BASE
        const uint32_t b2 = (h >> 16) & 0xffu, b3 = h >> 24;
        const uint32_t ew = (uint32_t)v2_closest_fixed_bits((int)((b3 >> 5) + 1u + v2_width_u(b2 & 31u)));
        ext = 4u + (b2 >> 5) + 1u + ((len * v2_width_u(code) + 7u) >> 3) + (((b3 & 31u) * ew + 7u) >> 3);
      } else {  // DELTA: header, two varints, packed deltas
        const uint64_t x = in.u64(pos + 2);
        const uint64_t t1 = ~x & 0x8080808080808080ull;
        const uint64_t t2 = t1 & (t1 - 1);
        uint32_t vb;
        if (t2) {
          vb = (uint32_t)(__ffsll((long long)t2) >> 3);
        } else {  // longer than the 8-byte window
          uint64_t v;
          int l1, l2;
          if (varint_at(in, pos + 2, (int64_t)n_in - (pos + 2), &v, &l1) != ST_OK) break;
          if (varint_at(in, pos + 2 + l1, (int64_t)n_in - (pos + 2 + l1), &v, &l2) != ST_OK) break;
          vb = (uint32_t)(l1 + l2);
        }
        const uint32_t w = code == 0 ? 0u : v2_width_u(code);
        ext = 2u + vb + ((w != 0 && len >= 2) ? (((len - 2u) * w + 7u) >> 3) : 0u);
      }
    }
    count += len;
    pos += ext;
  }
  for (; k < nseg; k++) publish_split((int)k, pos, count, split_pos, split_cnt, published);
}

// Decode part of one RLE v2 chunk.  The part's stream starts at a run
// boundary (position 0 of `in`, n_in bytes to the chunk end) whose first
// value index is count0; it decodes every run that starts before value hi_v
// (hi_v = ~0: to the end of the stream, and report OUTPUT_UNDERFLOW).
// out: the chunk's output; cap_values: its span; STORE = false sizes only.
// Error positions are relative to the part's start.
template <bool STORE, class In>
__device__ PartResult rle_v2_part(In& in, uint8_t* scratch, int64_t n_in, bool is_signed,
                                  uint64_t* __restrict__ out, uint64_t cap_values, uint64_t count0,
                                  uint64_t hi_v) {
  const uint32_t lane = lane_id();
  uint32_t* bitmap = reinterpret_cast<uint32_t*>(scratch);
  uint64_t* pvals = reinterpret_cast<uint64_t*>(scratch + 64);
  const bool last = hi_v == ~0ull;
  int64_t pos = 0;
  uint64_t count = count0;
  while (pos < n_in) {
    if (count >= hi_v) return PartResult{ST_OK, -1, count};
    if (!in.ensure(pos, pos + 40)) return part_error(ST_TIMEOUT, 0, count);
    V2Run r;
    const int32_t st = v2_parse_run(in, pos, n_in, r);
    if (st != ST_OK) return part_error(st, pos, count);
    const uint32_t len = r.len;
    const int w = r.w;
    if (r.enc == 2) {  // patch list validity belongs to the run's own checks
      const uint64_t mag = load_be64(in, pos + 4) >> (64 - 8 * r.bw);
      const uint64_t sign = 1ull << (8 * r.bw - 1);
      const uint64_t base = (mag & sign) ? 0ull - (mag & ~sign) : mag;
      // one entry per lane, read straight from global memory (at most 31
      // entries) so the staging ring only ever moves forward; positions are
      // the prefix sum of the gaps
      uint64_t gap = 0, patch = 0;
      if ((int)lane < r.pll) {
        const uint64_t bit = (uint64_t)lane * (uint64_t)r.ew;
        const int64_t at = r.psec + (int64_t)(bit >> 3);
        uint64_t x = 0;
        if (resident_input<In>::value) {  // a chunk staged whole: one 8-byte read in shared memory
          x = load_be64(in, at);
          if (n_in - at < 8) x &= ~0ull << (8 * (uint32_t)(8 - (n_in - at)));  // bytes past the chunk: 0
        } else {  // a ring only moves forward: the entries come from global memory
          const uint8_t* src = in.chunk_ptr();
#pragma unroll
          for (int k = 0; k < 8; k++) x = (x << 8) | (at + k < n_in ? (uint64_t)__ldg(src + at + k) : 0ull);
        }
        const uint64_t e = (x << (bit & 7)) >> (64 - r.ew);
        gap = e >> r.pw;  // pw <= 63 here
        patch = e & lowmask64(r.pw);
      }
      const bool real = (int)lane < r.pll && !(gap == 255 && patch == 0);
      // positions as a 32-bit scan: a gap above 0xffff (only in a malformed
      // entry) is clamped, which keeps its position and every later one at or
      // past the run length, so the stream is rejected as with exact sums
      const uint32_t ppos = warp_incl_scan32(gap > 0xffffull ? 0xffffu : (uint32_t)gap);
      const uint32_t before = __ballot_sync(FULL, real) & lanemask_lt();
      const int prev = before ? 31 - __clz(before) : 0;
      const uint32_t prev_pos = __shfl_sync(FULL, ppos, prev);
      const bool bad = real && (ppos >= len || (before != 0 && ppos <= prev_pos));
      if (__ballot_sync(FULL, bad)) return part_error(ST_BAD_HEADER, pos, count);
      if (count > cap_values || len > cap_values - count) return part_error(ST_OVERFLOW, pos, count);
      if (STORE && w <= 25) {
        // the whole run is resident: unpack it like a DIRECT run (two values
        // per lane and step, 32-bit arithmetic), then each lane that holds a
        // patch rewrites its one patched value (after the warp's stores)
        if (!in.ensure(r.sec, r.sec + r.nbytes + 8)) return part_error(ST_TIMEOUT, 0, count);
        uint64_t* o = out + count;
        const uint32_t sec32 = (uint32_t)r.sec;
        const uint32_t step = 32u * (uint32_t)w;
        uint32_t bit = lane * (uint32_t)w;
        uint32_t i = lane;
        for (; i + 32 < len; i += 64, bit += 2 * step) {
          const uint32_t va = v2_unpack32(in, sec32, bit, w);
          const uint32_t vb = v2_unpack32(in, sec32, bit + step, w);
          o[i] = base + va;
          o[i + 32] = base + vb;
        }
        if (i < len) o[i] = base + v2_unpack32(in, sec32, bit, w);
        __syncwarp();
        if (real) o[ppos] = base + ((uint64_t)v2_unpack32(in, sec32, ppos * (uint32_t)w, w) | (patch << w));
        __syncwarp();
      } else if (STORE) {
        // wide values stream through the ring 32 at a time: patches are
        // merged in the unpack loop through a 512-bit bitmap of positions
        if (lane < 16) bitmap[lane] = 0;
        __syncwarp();
        if (real) {
          atomicOr(&bitmap[ppos >> 5], 1u << (ppos & 31));
          pvals[__popc(before)] = patch;
        }
        __syncwarp();
        uint32_t carry = 0;
        uint64_t* o = out + count;
        for (uint32_t i0 = 0; i0 < len; i0 += 32) {
          const int64_t lo = r.sec + (((int64_t)i0 * w) >> 3);
          if (!in.ensure(lo, lo + 4 * w + 16)) return part_error(ST_TIMEOUT, 0, count);
          const uint32_t word = bitmap[i0 >> 5];
          const uint32_t i = i0 + lane;
          if (i < len) {
            uint64_t v = v2_unpack(in, r.sec, i, w);
            if ((word >> lane) & 1u) {
              const uint64_t pv = pvals[carry + __popc(word & lanemask_lt())];
              if (w < 64) v |= pv << w;
            }
            o[i] = base + v;
          }
          carry += __popc(word);
        }
        __syncwarp();
      }
    } else {
      if (count > cap_values || len > cap_values - count) return part_error(ST_OVERFLOW, pos, count);
      if (STORE) {
        uint64_t* o = out + count;
        if (r.enc == 0) {  // SHORT_REPEAT
          uint64_t v = load_be64(in, pos + 1) >> (64 - 8 * w);
          if (is_signed) v = unzigzag(v);
          if (lane < len) o[lane] = v;
        } else if (r.enc == 1) {  // DIRECT
          if (w <= 14) {  // whole run resident; four values per lane from one 8-byte read
            if (!in.ensure(r.sec, r.sec + r.nbytes + 8)) return part_error(ST_TIMEOUT, 0, count);
            const uint32_t sec32 = (uint32_t)r.sec;
            uint32_t i0 = 0;
            // lane l takes values i0 + 4l .. i0 + 4l + 3 and stores them with two
            // 16-byte stores; the first value goes alone when that aligns them
            if (reinterpret_cast<uintptr_t>(o) & 8) {
              const uint32_t v = v2_unpack32(in, sec32, 0, w);
              if (lane == 0) o[0] = is_signed ? unzigzag32(v) : (uint64_t)v;
              i0 = 1;
            }
            for (; i0 < len; i0 += 128) {
              const uint32_t i = i0 + 4 * lane;
              if (i < len) {
                uint32_t a0, a1, a2, a3;
                v2_unpack4(in, sec32, i * (uint32_t)w, w, a0, a1, a2, a3);
                const uint64_t x0 = is_signed ? unzigzag32(a0) : (uint64_t)a0;
                const uint64_t x1 = is_signed ? unzigzag32(a1) : (uint64_t)a1;
                const uint64_t x2 = is_signed ? unzigzag32(a2) : (uint64_t)a2;
                const uint64_t x3 = is_signed ? unzigzag32(a3) : (uint64_t)a3;
                if (i + 3 < len) {
                  *reinterpret_cast<ulonglong2*>(o + i) = make_ulonglong2(x0, x1);
                  *reinterpret_cast<ulonglong2*>(o + i + 2) = make_ulonglong2(x2, x3);
                } else {
                  o[i] = x0;
                  if (i + 1 < len) o[i + 1] = x1;
                  if (i + 2 < len) o[i + 2] = x2;
                }
              }
            }
          } else if (w <= 25) {  // whole run resident at once (<= 1600 bytes), 32-bit unpack
            if (!in.ensure(r.sec, r.sec + r.nbytes + 8)) return part_error(ST_TIMEOUT, 0, count);
            const uint32_t sec32 = (uint32_t)r.sec;
            const uint32_t step = 32u * (uint32_t)w;
            uint32_t bit = lane * (uint32_t)w;
            uint32_t i = lane;
            for (; i + 32 < len; i += 64, bit += 2 * step) {  // two values per lane and step
              const uint32_t va = v2_unpack32(in, sec32, bit, w);
              const uint32_t vb = v2_unpack32(in, sec32, bit + step, w);
              o[i] = is_signed ? unzigzag32(va) : (uint64_t)va;
              o[i + 32] = is_signed ? unzigzag32(vb) : (uint64_t)vb;
            }
            if (i < len) {
              const uint32_t v = v2_unpack32(in, sec32, bit, w);
              o[i] = is_signed ? unzigzag32(v) : (uint64_t)v;
            }
          } else {
            for (uint32_t i0 = 0; i0 < len; i0 += 32) {
              const int64_t lo = r.sec + (((int64_t)i0 * w) >> 3);
              if (!in.ensure(lo, lo + 4 * w + 16)) return part_error(ST_TIMEOUT, 0, count);
              const uint32_t i = i0 + lane;
              if (i < len) {
                uint64_t v = v2_unpack(in, r.sec, i, w);
                if (is_signed) v = unzigzag(v);
                o[i] = v;
              }
            }
          }
        } else {  // DELTA
          uint64_t basev = r.basev;
          if (is_signed) basev = unzigzag(basev);
          const uint64_t delta = unzigzag(r.dz);
          if (w == 0 || len < 3) {  // value i = base + i * delta, as a running sum
            uint64_t v = basev + (uint64_t)lane * delta;
            const uint64_t step = 32ull * delta;
            for (uint32_t i = lane; i < len; i += 32, v += step) o[i] = v;
          } else {
            const bool negative = (int64_t)delta < 0;
            if (lane == 0) o[0] = basev;
            if (lane == 1) o[1] = basev + delta;
            uint64_t carry = basev + delta;
            const uint32_t nd = len - 2;
            if (w <= 26) {  // deltas of <= 26 bits: 64 of them sum below 2^32
              if (!in.ensure(r.sec, r.sec + r.nbytes + 8)) return part_error(ST_TIMEOUT, 0, count);
              const uint32_t sec32 = (uint32_t)r.sec;
              uint64_t* od = o + 2;  // value j of the prefix-summed part
              uint32_t j0 = 0;
              // Lane i takes deltas j0 + 2i and j0 + 2i + 1 (one 8-byte read), so
              // one 32-value scan covers 64 deltas and each lane stores both
              // values with one 16-byte store; the first delta goes alone when
              // that keeps the pairs 16-byte aligned.
              if (reinterpret_cast<uintptr_t>(od) & 8) {
                const uint32_t d = v2_unpack32(in, sec32, 0, w);
                carry = negative ? carry - (uint64_t)d : carry + (uint64_t)d;
                if (lane == 0) od[0] = carry;
                j0 = 1;
              }
              // deltas of <= 14 bits: four per lane from one 8-byte read, one
              // scan per 128 deltas (their sum stays below 2^21), two 16-byte
              // stores per lane
              if (w <= 14)
                for (; j0 < nd; j0 += 128) {
                  const uint32_t j = j0 + 4 * lane;
                  uint32_t d0 = 0, d1 = 0, d2 = 0, d3 = 0;
                  if (j < nd) {
                    v2_unpack4(in, sec32, j * (uint32_t)w, w, d0, d1, d2, d3);
                    const uint32_t left = nd - j;
                    if (left < 4) {
                      d3 = 0;
                      if (left < 3) d2 = 0;
                      if (left < 2) d1 = 0;
                    }
                  }
                  const uint32_t sum = d0 + d1 + d2 + d3;
                  const uint32_t incl = warp_incl_scan32(sum);
                  const uint32_t p0 = incl - sum + d0, p1 = p0 + d1, p2 = p1 + d2;
                  const uint64_t s0 = negative ? carry - (uint64_t)p0 : carry + (uint64_t)p0;
                  const uint64_t s1 = negative ? carry - (uint64_t)p1 : carry + (uint64_t)p1;
                  const uint64_t s2 = negative ? carry - (uint64_t)p2 : carry + (uint64_t)p2;
                  const uint64_t s3 = negative ? carry - (uint64_t)incl : carry + (uint64_t)incl;
                  if (j + 3 < nd) {
                    *reinterpret_cast<ulonglong2*>(od + j) = make_ulonglong2(s0, s1);
                    *reinterpret_cast<ulonglong2*>(od + j + 2) = make_ulonglong2(s2, s3);
                  } else if (j < nd) {
                    od[j] = s0;
                    if (j + 1 < nd) od[j + 1] = s1;
                    if (j + 2 < nd) od[j + 2] = s2;
                  }
                  const uint64_t tot = __shfl_sync(FULL, incl, 31);
                  carry = negative ? carry - tot : carry + tot;
                }
              for (; j0 < nd; j0 += 64) {
                const uint32_t j = j0 + 2 * lane;
                uint32_t da = 0, db = 0;
                if (j < nd) {
                  const uint32_t b = j * (uint32_t)w;
                  const uint64_t x = load_be64(in, sec32 + (b >> 3)) << (b & 7);
                  da = (uint32_t)(x >> (64 - w));
                  if (j + 1 < nd) db = (uint32_t)((x << w) >> (64 - w));
                }
                const uint32_t incl = warp_incl_scan32(da + db);
                const uint64_t s1 = negative ? carry - (uint64_t)(incl - db) : carry + (uint64_t)(incl - db);
                const uint64_t s2 = negative ? carry - (uint64_t)incl : carry + (uint64_t)incl;
                if (j + 1 < nd) *reinterpret_cast<ulonglong2*>(od + j) = make_ulonglong2(s1, s2);
                else if (j < nd) od[j] = s1;
                const uint64_t tot = __shfl_sync(FULL, incl, 31);
                carry = negative ? carry - tot : carry + tot;
              }
            } else {
              for (uint32_t j0 = 0; j0 < nd; j0 += 32) {
                const int64_t lo = r.sec + (((int64_t)j0 * w) >> 3);
                if (!in.ensure(lo, lo + 4 * w + 16)) return part_error(ST_TIMEOUT, 0, count);
                const uint32_t j = j0 + lane;
                uint64_t d = j < nd ? v2_unpack(in, r.sec, j, w) : 0;
                if (negative) d = 0ull - d;
                const uint64_t s = warp_incl_scan64(d) + carry;
                if (j < nd) o[2 + j] = s;
                carry = shfl64(s, 31);
              }
            }
          }
        }
      }
    }
    count += len;
    pos = r.end;
  }
  if (last && STORE && count < cap_values) return part_error(ST_UNDERFLOW, n_in, count);
  return PartResult{ST_OK, -1, count};
}

}  // namespace codag
