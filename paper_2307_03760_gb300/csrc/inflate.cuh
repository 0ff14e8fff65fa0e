// Raw Deflate (RFC 1951) decoder, one warp per chunk (CODAG Sec. II-A,
// Deflate; Sec. V-F for the dictionary copy primitive).
//
// Work split inside the warp:
//   - the bit stream is consumed by every lane from a 64-bit register buffer
//     refilled from the shared staging ring (identical state in all lanes);
//   - Huffman codes are decoded by one lookup in a shared-memory table
//     indexed by the next TB stream bits (codes longer than TB bits, which
//     are rare by construction of Huffman codes, fall back to a canonical
//     search over lengths TB+1..15);
//   - tables are built warp-parallel for every block: __match_any_sync ranks
//     symbols of equal length (canonical order), and each lane fills table
//     entries by locating the code that prefixes the entry's bits;
//   - output goes into a shared-memory window that mirrors the last WIN
//     bytes of the chunk's output; literals are stored by one lane, matches
//     (the paper's memcpy(off, len), Table 2) are copied by all lanes, lane i
//     taking byte i, with overlapping matches (len > dist) handled by reading
//     position (i mod dist) of the source window (Sec. V-F); sources farther
//     back than the window are read back from global memory;
//   - the window is flushed to global memory with coalesced 16-byte stores.
//
// Status order matches the oracle: the first problem met in stream order;
// code-length problems before symbol validity (a code whose bits run past the
// chunk end is TRUNCATED even where the padded bits would be invalid).
#pragma once

#include "ring.cuh"

namespace codag {

// table entry: bits 0-3 code length, 4-6 kind, 8-11 extra bits, 16-31 value
enum : uint32_t {
  K_LIT = 0,      // literal byte / code-length symbol
  K_BASE = 1,     // length or distance base with extra bits
  K_EOB = 2,      // end of block
  K_BADSYM = 3,   // valid code, invalid symbol (286, 287, distance 30, 31)
  K_BADCODE = 4,  // bits that no code can start with
  K_LONG = 5,     // code longer than the table's index width
};

__device__ __forceinline__ uint32_t ent_len(uint32_t e) { return e & 15u; }
__device__ __forceinline__ uint32_t ent_kind(uint32_t e) { return (e >> 4) & 7u; }
__device__ __forceinline__ uint32_t ent_extra(uint32_t e) { return (e >> 8) & 15u; }
__device__ __forceinline__ uint32_t ent_val(uint32_t e) { return e >> 16; }
__device__ __forceinline__ uint32_t make_ent(uint32_t len, uint32_t kind, uint32_t extra,
                                             uint32_t val) {
  return len | (kind << 4) | (extra << 8) | (val << 16);
}

// RFC 1951 Sec. 3.2.5 in closed form: length symbol 257+i, distance code d.
__device__ __forceinline__ uint32_t len_sym_entry(uint32_t len, uint32_t i) {
  if (i < 8) return make_ent(len, K_BASE, 0, 3 + i);
  if (i == 28) return make_ent(len, K_BASE, 0, 258);
  const uint32_t e = (i >> 2) - 1;
  return make_ent(len, K_BASE, e, ((4u + (i & 3u)) << e) + 3u);
}
__device__ __forceinline__ uint32_t dist_sym_entry(uint32_t len, uint32_t d) {
  if (d < 4) return make_ent(len, K_BASE, 0, 1 + d);
  const uint32_t e = (d >> 1) - 1;
  return make_ent(len, K_BASE, e, ((2u + (d & 1u)) << e) + 1u);
}

// Code-length code order, RFC 1951 Sec. 3.2.7.
static __constant__ uint8_t kClenOrder[19] = {16, 17, 18, 0, 8,  7, 9,  6, 10, 5,
                                       11, 4,  12, 3, 13, 2, 14, 1, 15};

// A canonical code in shared memory.
struct HCode {
  uint32_t* table;   // 1 << tb entries
  uint16_t* sorted;  // symbols by (length, symbol)
  uint16_t* first;   // [16] first code of each length
  uint16_t* count;   // [16] codes of each length
  uint16_t* offset;  // [16] index in sorted of each length's first code
  uint32_t kraft;    // sum of 2^(15 - len)
  int tb;            // table index bits
  int kind;          // 0 code-length code, 1 lit/len, 2 distance
};

// Entry for symbol `sym` with code length `len`.
__device__ __forceinline__ uint32_t sym_entry(int kind, uint32_t len, uint32_t sym) {
  if (kind == 0) return make_ent(len, K_LIT, 0, sym);
  if (kind == 1) {
    if (sym < 256) return make_ent(len, K_LIT, 0, sym);
    if (sym == 256) return make_ent(len, K_EOB, 0, 0);
    if (sym <= 285) return len_sym_entry(len, sym - 257);
    return make_ent(len, K_BADSYM, 0, 0);
  }
  if (sym < 30) return dist_sym_entry(len, sym);
  return make_ent(len, K_BADSYM, 0, 0);
}

// Build the canonical code for lens[0..n) (RFC 1951 Sec. 3.2.2).  Returns
// ST_OK or ST_BAD_HUFFMAN (over-subscribed, or incomplete except a single
// length-1 code for lit/len and distance codes, or no codes for distance).
static __device__ __noinline__ int32_t build_code(HCode& c, const uint8_t* lens, int n, uint16_t* scratch16) {
  const uint32_t lane = lane_id();
  uint16_t* run = scratch16;  // [16] running counters
  if (lane < 16) {
    c.count[lane] = 0;
    run[lane] = 0;
  }
  __syncwarp();
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int j = j0 + (int)lane;
    const uint32_t L = j < n ? lens[j] : 0u;
    const uint32_t mask = __match_any_sync(FULL, L);
    if (L != 0 && (int)lane == __ffs(mask) - 1) c.count[L] += (uint16_t)__popc(mask);
    __syncwarp();
  }
  __syncwarp();
  // Kraft sum, first code and offset of each length (every lane, same values)
  uint32_t kraft = 0;
  int maxlen = 0;
  uint32_t code = 0, idx = 0, prev = 0;
  for (int L = 1; L <= 15; L++) {
    const uint32_t cnt = c.count[L];
    kraft += cnt << (15 - L);
    if (cnt) maxlen = L;
    code = (code + prev) << 1;
    if (lane == 0) {
      c.first[L] = (uint16_t)code;
      c.offset[L] = (uint16_t)idx;
    }
    idx += cnt;
    prev = cnt;
  }
  c.kraft = kraft;
  if (kraft > (1u << 15)) return ST_BAD_HUFFMAN;
  if (kraft < (1u << 15)) {
    const bool ok = (c.kind != 0 && maxlen == 1) || (c.kind == 2 && maxlen == 0);
    if (!ok) return ST_BAD_HUFFMAN;
  }
  __syncwarp();
  // place symbols in canonical order
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int j = j0 + (int)lane;
    const uint32_t L = j < n ? lens[j] : 0u;
    const uint32_t mask = __match_any_sync(FULL, L);
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if ((int)lane == leader && L != 0) base = run[L];
    base = __shfl_sync(FULL, base, leader);
    if (L != 0) c.sorted[c.offset[L] + base + __popc(mask & lanemask_lt())] = (uint16_t)j;
    __syncwarp();
    if ((int)lane == leader && L != 0) run[L] = (uint16_t)(base + __popc(mask));
    __syncwarp();
  }
  __syncwarp();
  // fill the table: entry e holds the code whose bits prefix e (stream order)
  const int tb = c.tb;
  for (int e = (int)lane; e < (1 << tb); e += 32) {
    const uint32_t rev = __brev((uint32_t)e) >> (32 - tb);  // code bits MSB first
    uint32_t ent;
    if (kraft == 0) {
      ent = make_ent(0, K_BADCODE, 0, 0);
    } else {
      ent = make_ent(0, K_LONG, 0, 0);
      for (int L = 1; L <= tb; L++) {
        const uint32_t cc = rev >> (tb - L);
        const uint32_t k = cc - c.first[L];
        if (k < c.count[L]) {
          ent = sym_entry(c.kind, (uint32_t)L, c.sorted[c.offset[L] + k]);
          break;
        }
        const uint32_t valid = (kraft + (1u << (15 - L)) - 1) >> (15 - L);
        if (cc >= valid) {
          ent = make_ent((uint32_t)L, K_BADCODE, 0, 0);
          break;
        }
      }
    }
    c.table[e] = ent;
  }
  __syncwarp();
  return ST_OK;
}

// Decode a code longer than the table width from the next 15 stream bits.
static __device__ __noinline__ uint32_t decode_long(const HCode& c, uint64_t bits) {
  const uint32_t rev = __brev((uint32_t)bits) >> 17;  // 15 bits, MSB first
  for (int L = c.tb + 1; L <= 15; L++) {
    const uint32_t cc = rev >> (15 - L);
    const uint32_t k = cc - c.first[L];
    if (k < c.count[L]) return sym_entry(c.kind, (uint32_t)L, c.sorted[c.offset[L] + k]);
    const uint32_t valid = (c.kraft + (1u << (15 - L)) - 1) >> (15 - L);
    if (cc >= valid) return make_ent((uint32_t)L, K_BADCODE, 0, 0);
  }
  return make_ent(15, K_BADCODE, 0, 0);
}

template <int LIT_TB, int DIST_TB, int WIN>
struct InflateSmem {
  static constexpr int LIT_ENTRIES = 1 << LIT_TB;
  static constexpr int DIST_ENTRIES = 1 << DIST_TB;
  static_assert(DIST_ENTRIES >= 128, "distance table also holds the 7-bit code-length table");
  // byte offsets within the decoder's scratch area
  static constexpr int OFF_LIT = 0;
  static constexpr int OFF_DIST = OFF_LIT + 4 * LIT_ENTRIES;
  static constexpr int OFF_WIN = OFF_DIST + 4 * DIST_ENTRIES;
  static constexpr int OFF_LSORT = OFF_WIN + WIN;
  static constexpr int OFF_DSORT = OFF_LSORT + 2 * 288;
  static constexpr int OFF_META = OFF_DSORT + 2 * 32;  // 7 x u16[16]
  static constexpr int OFF_LENS = OFF_META + 7 * 32;
  static constexpr int BYTES = (OFF_LENS + 320 + 15) & ~15;
};

// Bit reader over the staging ring; all lanes hold the same state.
template <class Ring>
struct BitIn {
  Ring* ring;
  uint64_t bb;     // next bits, LSB first; zero past the chunk end
  int nb;          // valid bits in bb
  int64_t pos;     // absolute bit position of bb's bit 0
  int64_t endbits; // chunk length in bits

  __device__ __forceinline__ bool refill() {
    const int64_t byte = pos >> 3;
    if (!ring->ensure(byte, byte + 8)) return false;
    const uint32_t sh = (uint32_t)(pos & 7);
    uint64_t x = ring->u64(byte) >> sh;
    const int64_t avail = endbits - pos;
    if (avail < 64) x &= lowmask64(avail < 0 ? 0u : (uint32_t)avail);
    bb = x;
    nb = 64 - (int)sh;
    return true;
  }
  __device__ __forceinline__ void consume(uint32_t k) {
    bb >>= k;
    nb -= (int)k;
    pos += k;
  }
  __device__ __forceinline__ int64_t avail() const { return endbits - pos; }
};

// Decode one raw Deflate chunk.  out: the chunk's output; cap: its span in
// bytes (STORE = false sizes the stream and ignores out/cap).
template <bool STORE, int LIT_TB, int DIST_TB, int WIN, class Ring>
__device__ int32_t inflate_decode(Ring& ring, uint8_t* scratch, int64_t n_in,
                                  uint8_t* __restrict__ out, uint64_t cap, uint64_t* produced) {
  using SM = InflateSmem<LIT_TB, DIST_TB, WIN>;
  constexpr uint32_t WMASK = WIN - 1;
  constexpr int64_t FLUSH_T = WIN / 4;
  constexpr int64_t NEAR_MAX = WIN - 512;
  static_assert(WIN >= 2048 && (WIN & (WIN - 1)) == 0, "window: power of two >= 2048");
  const uint32_t lane = lane_id();
  uint32_t* lit_tab = reinterpret_cast<uint32_t*>(scratch + SM::OFF_LIT);
  uint32_t* dist_tab = reinterpret_cast<uint32_t*>(scratch + SM::OFF_DIST);
  uint8_t* win = scratch + SM::OFF_WIN;
  uint16_t* meta = reinterpret_cast<uint16_t*>(scratch + SM::OFF_META);
  uint8_t* lens = scratch + SM::OFF_LENS;
  HCode lit{lit_tab, reinterpret_cast<uint16_t*>(scratch + SM::OFF_LSORT), meta, meta + 16,
            meta + 32, 0, LIT_TB, 1};
  HCode dist{dist_tab, reinterpret_cast<uint16_t*>(scratch + SM::OFF_DSORT), meta + 48, meta + 64,
             meta + 80, 0, DIST_TB, 2};
  uint16_t* run16 = meta + 96;

  BitIn<Ring> in{&ring, 0, 0, 0, n_in * 8};
  const uint32_t oaddr = (uint32_t)reinterpret_cast<uintptr_t>(out);
  const uint64_t limit = STORE ? cap : ~0ull;
  uint64_t wpos = 0;     // bytes produced
  uint64_t flushed = 0;  // bytes already in global memory
  int fixed_ready = 0;   // the fixed tables are built in lit/dist
  int32_t st = ST_OK;
  *produced = 0;

  // write window bytes of output [flushed, to) to global memory; `to` is either
  // a 16-byte boundary of the global address or the end of the output
  auto flush = [&](uint64_t to) {
    uint64_t f = flushed;
    const uint64_t head_end = (((uint64_t)oaddr + f + 15) & ~15ull) - oaddr;
    if (f < head_end) {  // unaligned head (first flush only)
      const uint64_t h = (head_end < to ? head_end : to) - f;
      if (lane < h) out[f + lane] = win[(oaddr + (uint32_t)(f + lane)) & WMASK];
      f += h;
    }
    const uint64_t body_end = f + ((to - f) & ~15ull);
    for (uint64_t b = f + 16 * lane; b < body_end; b += 512) {
      const uint4 v = *reinterpret_cast<const uint4*>(win + ((oaddr + (uint32_t)b) & WMASK));
      *reinterpret_cast<uint4*>(out + b) = v;
    }
    f = body_end;
    if (f < to && lane < to - f) out[f + lane] = win[(oaddr + (uint32_t)(f + lane)) & WMASK];
    flushed = to;
  };

  if (!in.refill()) return ST_TIMEOUT;
  for (;;) {
    // block header
    if (in.avail() < 3) { st = ST_TRUNCATED; break; }
    if (in.nb < 48 && !in.refill()) return ST_TIMEOUT;
    const uint32_t bfinal = (uint32_t)(in.bb & 1);
    const uint32_t btype = (uint32_t)((in.bb >> 1) & 3);
    in.consume(3);
    if (btype == 3) { st = ST_BAD_HEADER; break; }
    if (btype == 0) {  // stored block
      const uint32_t skip = (uint32_t)((8 - (in.pos & 7)) & 7);
      if (in.avail() < (int64_t)skip + 32) { st = ST_TRUNCATED; break; }
      in.consume(skip);
      if (!in.refill()) return ST_TIMEOUT;
      const uint32_t len = (uint32_t)(in.bb & 0xffff);
      const uint32_t nlen = (uint32_t)((in.bb >> 16) & 0xffff);
      if (len != (~nlen & 0xffffu)) { st = ST_BAD_STORED_LEN; break; }
      if (len > limit - wpos) { st = ST_OVERFLOW; break; }
      const int64_t src = (in.pos >> 3) + 4;
      if (src + (int64_t)len > n_in) { st = ST_TRUNCATED; break; }
      if (STORE) {
        constexpr uint32_t PIECE = WIN / 4 < 1024 ? WIN / 4 : 1024;
        for (uint32_t k0 = 0; k0 < len; k0 += PIECE) {
          const uint32_t piece = len - k0 < PIECE ? len - k0 : PIECE;
          if (!ring.ensure(src + k0, src + k0 + piece)) return ST_TIMEOUT;
          for (uint32_t k = lane; k < piece; k += 32)
            win[(oaddr + (uint32_t)(wpos + k0 + k)) & WMASK] = ring.byte(src + k0 + k);
          __syncwarp();
          const uint64_t w2 = wpos + k0 + piece;
          if (w2 - flushed >= (uint64_t)FLUSH_T) flush((((uint64_t)oaddr + w2) & ~15ull) - oaddr);
          __syncwarp();
        }
      }
      wpos += len;
      in.pos += 32 + 8 * (int64_t)len;
      in.nb = 0;
      if (!in.refill()) return ST_TIMEOUT;
    } else {
      if (btype == 1) {  // fixed codes, RFC 1951 Sec. 3.2.6
        if (!fixed_ready) {
          for (int j = (int)lane; j < 320; j += 32) {
            uint8_t L;
            if (j < 288) L = j < 144 ? 8 : j < 256 ? 9 : j < 280 ? 7 : 8;
            else L = 5;
            lens[j] = L;
          }
          __syncwarp();
          build_code(lit, lens, 288, run16);
          build_code(dist, lens + 288, 32, run16);
          fixed_ready = 1;
        }
      } else {  // dynamic codes, RFC 1951 Sec. 3.2.7
        fixed_ready = 0;
        if (in.avail() < 14) { st = ST_TRUNCATED; break; }
        if (in.nb < 48 && !in.refill()) return ST_TIMEOUT;
        const int nlen = (int)(in.bb & 31) + 257;
        const int ndist = (int)((in.bb >> 5) & 31) + 1;
        const int ncode = (int)((in.bb >> 10) & 15) + 4;
        in.consume(14);
        if (nlen > 286 || ndist > 30) { st = ST_BAD_HUFFMAN; break; }
        if (in.avail() < 3 * ncode) { st = ST_TRUNCATED; break; }
        if (!in.refill()) return ST_TIMEOUT;
        // code-length code lengths; 19 x 3 = 57 bits fit one refill
        if (lane < 19) lens[kClenOrder[lane]] = (int)lane < ncode ? (uint8_t)((in.bb >> (3 * lane)) & 7) : 0;
        __syncwarp();
        in.consume(3 * ncode);
        HCode cl{dist_tab, dist.sorted, dist.first, dist.count, dist.offset, 0, 7, 0};
        if (build_code(cl, lens, 19, run16) != ST_OK) { st = ST_BAD_HUFFMAN; break; }
        const int total = nlen + ndist;
        int have = 0;
        bool bad = false;
        while (have < total) {
          if (in.nb < 16 && !in.refill()) return ST_TIMEOUT;
          const uint32_t e = dist_tab[in.bb & 127];
          const uint32_t L = ent_len(e);
          if ((int64_t)L > in.avail()) { st = ST_TRUNCATED; bad = true; break; }
          if (ent_kind(e) != K_LIT) { st = ST_BAD_HUFFMAN; bad = true; break; }
          in.consume(L);
          const uint32_t sym = ent_val(e);
          if (sym < 16) {
            if (lane == 0) lens[have] = (uint8_t)sym;
            have++;
            continue;
          }
          uint32_t rep, val = 0;
          if (sym == 16) {
            if (have == 0) { st = ST_BAD_HUFFMAN; bad = true; break; }
            __syncwarp();
            val = lens[have - 1];
            if (in.avail() < 2) { st = ST_TRUNCATED; bad = true; break; }
            rep = 3 + (uint32_t)(in.bb & 3);
            in.consume(2);
          } else if (sym == 17) {
            if (in.avail() < 3) { st = ST_TRUNCATED; bad = true; break; }
            rep = 3 + (uint32_t)(in.bb & 7);
            in.consume(3);
          } else {
            if (in.avail() < 7) { st = ST_TRUNCATED; bad = true; break; }
            rep = 11 + (uint32_t)(in.bb & 127);
            in.consume(7);
          }
          if (have + (int)rep > total) { st = ST_BAD_HUFFMAN; bad = true; break; }
          for (uint32_t k = lane; k < rep; k += 32) lens[have + k] = (uint8_t)val;
          have += (int)rep;
        }
        if (bad) break;
        __syncwarp();
        if (lens[256] == 0) { st = ST_BAD_HUFFMAN; break; }
        if (build_code(lit, lens, nlen, run16) != ST_OK) { st = ST_BAD_HUFFMAN; break; }
        if (build_code(dist, lens + nlen, ndist, run16) != ST_OK) { st = ST_BAD_HUFFMAN; break; }
      }
      // symbol loop
      bool done = false;
      for (;;) {
        if (in.nb < 48 && !in.refill()) return ST_TIMEOUT;
        uint32_t e = lit_tab[in.bb & ((1u << LIT_TB) - 1)];
        if (ent_kind(e) == K_LONG) e = decode_long(lit, in.bb);
        uint32_t L = ent_len(e);
        uint32_t kind = ent_kind(e);
        if ((int64_t)L > in.avail()) { st = ST_TRUNCATED; break; }
        if (kind == K_BADCODE || kind == K_BADSYM) { st = ST_BAD_HUFFMAN; break; }
        in.consume(L);
        if (kind == K_LIT) {
          if (wpos >= limit) { st = ST_OVERFLOW; break; }
          if (STORE && lane == 0) win[(oaddr + (uint32_t)wpos) & WMASK] = (uint8_t)ent_val(e);
          wpos++;
          if (STORE && wpos - flushed >= (uint64_t)FLUSH_T) {
            __syncwarp();
            flush((((uint64_t)oaddr + wpos) & ~15ull) - oaddr);
            __syncwarp();
          }
          continue;
        }
        if (kind == K_EOB) { done = true; break; }
        // length
        uint32_t x = ent_extra(e);
        if ((int64_t)x > in.avail()) { st = ST_TRUNCATED; break; }
        const uint32_t mlen = ent_val(e) + (uint32_t)(in.bb & ((1u << x) - 1));
        in.consume(x);
        // distance
        e = dist_tab[in.bb & ((1u << DIST_TB) - 1)];
        if (ent_kind(e) == K_LONG) e = decode_long(dist, in.bb);
        L = ent_len(e);
        kind = ent_kind(e);
        if ((int64_t)L > in.avail()) { st = ST_TRUNCATED; break; }
        if (kind == K_BADCODE || kind == K_BADSYM) { st = ST_BAD_HUFFMAN; break; }
        in.consume(L);
        x = ent_extra(e);
        if ((int64_t)x > in.avail()) { st = ST_TRUNCATED; break; }
        const uint32_t d = ent_val(e) + (uint32_t)(in.bb & ((1u << x) - 1));
        in.consume(x);
        if ((uint64_t)d > wpos) { st = ST_BAD_DISTANCE; break; }
        if ((uint64_t)mlen > limit - wpos) { st = ST_OVERFLOW; break; }
        if (STORE) {
          __syncwarp();
          const uint64_t s0 = wpos - d;
          if ((int64_t)d <= NEAR_MAX) {
            for (uint32_t i = lane; i < mlen; i += 32) {
              const uint32_t k = d >= mlen ? i : i % d;
              win[(oaddr + (uint32_t)(wpos + i)) & WMASK] = win[(oaddr + (uint32_t)(s0 + k)) & WMASK];
            }
          } else {  // far source: already flushed to global memory
            for (uint32_t i = lane; i < mlen; i += 32)
              win[(oaddr + (uint32_t)(wpos + i)) & WMASK] = __ldcg(out + s0 + i);
          }
          __syncwarp();
        }
        wpos += mlen;
        if (STORE && wpos - flushed >= (uint64_t)FLUSH_T) {
          __syncwarp();
          flush((((uint64_t)oaddr + wpos) & ~15ull) - oaddr);
          __syncwarp();
        }
      }
      if (!done) break;
    }
    if (STORE && wpos - flushed >= (uint64_t)FLUSH_T) {
      __syncwarp();
      flush((((uint64_t)oaddr + wpos) & ~15ull) - oaddr);
      __syncwarp();
    }
    if (bfinal) break;
  }
  if (STORE) {
    __syncwarp();
    if (wpos > flushed) flush(wpos);
    __syncwarp();
  }
  *produced = wpos;
  if (st != ST_OK) return st;
  if (STORE && wpos < cap) return ST_UNDERFLOW;
  return ST_OK;
}

}  // namespace codag
