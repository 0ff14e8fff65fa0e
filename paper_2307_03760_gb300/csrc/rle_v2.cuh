// ORC integer RLE v2 decoder, one warp per chunk (CODAG Sec. II-A, RLE v2;
// Sec. VI-A evaluates the ORC form).  The top two bits of a run's first byte
// select SHORT_REPEAT / DIRECT / PATCHED_BASE / DELTA.
//
// Work split inside the warp:
//   - run headers are parsed by every lane (identical state);
//   - bit-packed sections (MSB first, widths 1..64) are unpacked 32 values at
//     a time, lane i taking value i: one unaligned 8-byte read from the
//     staging ring, a byte swap and two shifts (any width <= 64 fits: widths
//     that are not multiples of 8 are <= 30 bits);
//   - PATCHED_BASE patch entries are decoded one per lane, their positions
//     are a warp prefix sum of the gaps, and a 512-bit shared bitmap marks
//     the patched values for the unpack loop;
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
  const uint64_t x = bswap64(ring.u64(sec + (int64_t)(bit >> 3)));
  return (x << (bit & 7)) >> (64 - w);
}

template <bool STORE, class Ring>
__device__ int32_t rle_v2_decode(Ring& ring, uint8_t* scratch, int64_t n_in, bool is_signed,
                                 uint64_t* __restrict__ out, uint64_t cap_values,
                                 uint64_t* produced) {
  const uint32_t lane = lane_id();
  uint32_t* bitmap = reinterpret_cast<uint32_t*>(scratch);
  uint64_t* pvals = reinterpret_cast<uint64_t*>(scratch + 64);
  int64_t pos = 0;
  uint64_t count = 0;
  *produced = 0;
  while (pos < n_in) {
    if (!ring.ensure(pos, pos + 40)) return ST_TIMEOUT;
    const uint64_t hdr = ring.u64(pos);
    const uint32_t b0 = (uint32_t)(hdr & 0xff);
    const uint32_t enc = b0 >> 6;
    if (enc == 0) {  // SHORT_REPEAT
      const int nb = ((b0 >> 3) & 7) + 1;
      const uint32_t len = (b0 & 7) + 3;
      if (pos + 1 + nb > n_in) return ST_TRUNCATED;
      uint64_t v = bswap64(ring.u64(pos + 1)) >> (64 - 8 * nb);
      if (is_signed) v = unzigzag(v);
      if (len > cap_values - count) return ST_OVERFLOW;
      if (STORE && lane < len) out[count + lane] = v;
      count += len;
      pos += 1 + nb;
    } else {
      if (pos + 2 > n_in) return ST_TRUNCATED;
      const uint32_t b1 = (uint32_t)((hdr >> 8) & 0xff);
      const int wcode = (b0 >> 1) & 31;
      const uint32_t len = (((b0 & 1) << 8) | b1) + 1;
      if (enc == 1) {  // DIRECT
        const int w = v2_width(wcode);
        const int64_t sec = pos + 2;
        const int64_t nbytes = ((int64_t)len * w + 7) >> 3;
        if (sec + nbytes > n_in) return ST_TRUNCATED;
        if (len > cap_values - count) return ST_OVERFLOW;
        if (STORE) {
          for (uint32_t i0 = 0; i0 < len; i0 += 32) {
            const int64_t lo = sec + (((int64_t)i0 * w) >> 3);
            if (!ring.ensure(lo, lo + 4 * w + 16)) return ST_TIMEOUT;
            const uint32_t i = i0 + lane;
            if (i < len) {
              uint64_t v = v2_unpack(ring, sec, i, w);
              if (is_signed) v = unzigzag(v);
              out[count + i] = v;
            }
          }
        }
        count += len;
        pos = sec + nbytes;
      } else if (enc == 2) {  // PATCHED_BASE
        const int w = v2_width(wcode);
        if (pos + 4 > n_in) return ST_TRUNCATED;
        const uint32_t b2 = (uint32_t)((hdr >> 16) & 0xff);
        const uint32_t b3 = (uint32_t)((hdr >> 24) & 0xff);
        const int bw = (b2 >> 5) + 1;
        const int pw = v2_width(b2 & 31);
        const int pgw = (b3 >> 5) + 1;
        const int pll = b3 & 31;
        if (pgw + pw > 64) return ST_BAD_HEADER;
        if (pos + 4 + bw > n_in) return ST_TRUNCATED;
        const uint64_t mag = bswap64(ring.u64(pos + 4)) >> (64 - 8 * bw);
        const uint64_t sign = 1ull << (8 * bw - 1);
        const uint64_t base = (mag & sign) ? 0ull - (mag & ~sign) : mag;
        const int64_t sec = pos + 4 + bw;
        const int64_t nbytes = ((int64_t)len * w + 7) >> 3;
        if (sec + nbytes > n_in) return ST_TRUNCATED;
        const int ew = v2_closest_fixed_bits(pgw + pw);
        const int64_t psec = sec + nbytes;
        const int64_t pbytes = ((int64_t)pll * ew + 7) >> 3;
        if (psec + pbytes > n_in) return ST_TRUNCATED;
        // patch list: one entry per lane, read straight from global memory
        // (at most 31 entries) so the staging ring only ever moves forward;
        // positions = prefix sum of the gaps
        uint64_t gap = 0, patch = 0;
        if ((int)lane < pll) {
          const uint64_t bit = (uint64_t)lane * (uint64_t)ew;
          const int64_t at = psec + (int64_t)(bit >> 3);
          const uint8_t* src = ring.chunk_ptr();
          uint64_t x = 0;
#pragma unroll
          for (int k = 0; k < 8; k++) {
            const uint64_t b = at + k < n_in ? (uint64_t)__ldg(src + at + k) : 0ull;
            x = (x << 8) | b;
          }
          const uint64_t e = (x << (bit & 7)) >> (64 - ew);
          gap = e >> pw;  // pw <= 63 here
          patch = e & lowmask64(pw);
        }
        const bool real = (int)lane < pll && !(gap == 255 && patch == 0);
        const uint64_t ppos = warp_incl_scan64(gap);
        const uint32_t real_mask = __ballot_sync(FULL, real);
        const uint32_t before = real_mask & lanemask_lt();
        const int prev = before ? 31 - __clz(before) : 0;
        const uint64_t prev_pos = shfl64(ppos, prev);
        const bool bad = real && (ppos >= len || (before != 0 && ppos <= prev_pos));
        if (__ballot_sync(FULL, bad)) return ST_BAD_HEADER;
        if (len > cap_values - count) return ST_OVERFLOW;
        if (STORE) {
          if (lane < 16) bitmap[lane] = 0;
          __syncwarp();
          if (real) {
            atomicOr(&bitmap[ppos >> 5], 1u << (ppos & 31));
            pvals[__popc(before)] = patch;
          }
          __syncwarp();
          uint32_t carry = 0;
          for (uint32_t i0 = 0; i0 < len; i0 += 32) {
            const int64_t lo = sec + (((int64_t)i0 * w) >> 3);
            if (!ring.ensure(lo, lo + 4 * w + 16)) return ST_TIMEOUT;
            const uint32_t word = bitmap[i0 >> 5];
            const uint32_t i = i0 + lane;
            if (i < len) {
              uint64_t v = v2_unpack(ring, sec, i, w);
              if ((word >> lane) & 1u) {
                const uint64_t pv = pvals[carry + __popc(word & lanemask_lt())];
                if (w < 64) v |= pv << w;
              }
              out[count + i] = base + v;
            }
            carry += __popc(word);
          }
        }
        count += len;
        pos = psec + pbytes;
      } else {  // DELTA
        const int w = wcode == 0 ? 0 : v2_width(wcode);
        uint64_t basev, dz;
        int l1, l2;
        int32_t st = varint_at(ring, pos + 2, n_in - (pos + 2), &basev, &l1);
        if (st != ST_OK) return st;
        if (is_signed) basev = unzigzag(basev);
        st = varint_at(ring, pos + 2 + l1, n_in - (pos + 2 + l1), &dz, &l2);
        if (st != ST_OK) return st;
        const uint64_t delta = unzigzag(dz);
        const int64_t sec = pos + 2 + l1 + l2;
        int64_t nbytes = 0;
        if (w != 0 && len >= 2) {
          nbytes = ((int64_t)(len - 2) * w + 7) >> 3;
          if (sec + nbytes > n_in) return ST_TRUNCATED;
        }
        if (len > cap_values - count) return ST_OVERFLOW;
        if (STORE) {
          uint64_t* o = out + count;
          if (w == 0 || len < 3) {
            for (uint32_t i = lane; i < len; i += 32) o[i] = basev + (uint64_t)i * delta;
          } else {
            const bool negative = (int64_t)delta < 0;
            if (lane == 0) o[0] = basev;
            if (lane == 1) o[1] = basev + delta;
            uint64_t carry = basev + delta;
            const uint32_t nd = len - 2;
            for (uint32_t j0 = 0; j0 < nd; j0 += 32) {
              const int64_t lo = sec + (((int64_t)j0 * w) >> 3);
              if (!ring.ensure(lo, lo + 4 * w + 16)) return ST_TIMEOUT;
              const uint32_t j = j0 + lane;
              uint64_t d = j < nd ? v2_unpack(ring, sec, j, w) : 0;
              if (negative) d = 0ull - d;
              const uint64_t s = warp_incl_scan64(d) + carry;
              if (j < nd) o[2 + j] = s;
              carry = shfl64(s, 31);
            }
          }
        }
        count += len;
        pos = sec + nbytes;
      }
    }
    *produced = count;
  }
  *produced = count;
  if (STORE && count < cap_values) return ST_UNDERFLOW;
  return ST_OK;
}

}  // namespace codag
