// Raw Deflate (RFC 1951) decoder, one warp per chunk (CODAG Sec. II-A,
// Deflate; Sec. IV-F for the dictionary copy primitive).
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
//   - output and match sources live in global memory (the chunk's own output
//     span, served by L1/L2): literals are stored by one lane; a match (the
//     paper's memcpy(off, len), Table 2) is copied by all lanes, lane i
//     taking byte i, with overlapping matches (len > dist) handled by reading
//     position (i mod dist) of the source (Sec. IV-F); in the lean loop a
//     short match's source bytes are loaded when it is decoded and stored
//     when the next match is decoded, so the load overlaps decoding;
//   - a shared-memory window of the last WIN output bytes is a template
//     option (WIN > 0: flushed with 16-byte stores); every kernel compiles it
//     with WIN = 0, since the window cost more occupancy than it saved.
//
// Status order matches the oracle: the first problem met in stream order;
// code-length problems before symbol validity (a code whose bits run past the
// chunk end is TRUNCATED even where the padded bits would be invalid).
#pragma once

#include "ring.cuh"

namespace codag {

// table entry: bits 0-3 code length, 4-6 kind, 8-11 extra bits, 16-30 value,
// bit 31 set for literals (so a literal is recognised by the sign alone)
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
__device__ __forceinline__ uint32_t ent_val(uint32_t e) { return (e >> 16) & 0x7fffu; }
__device__ __forceinline__ uint32_t make_ent(uint32_t len, uint32_t kind, uint32_t extra,
                                             uint32_t val) {
  return len | (kind << 4) | (extra << 8) | (val << 16) | (kind == 0 ? 0x80000000u : 0u);
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

// Shared-memory tables hold 16-bit entries: bits 0-3 code length, 4-11 value
// (literal byte, length-symbol index 0-28, distance code 0-29, or
// code-length symbol), 12-14 kind, bit 15 set for literals.  Base and extra
// bits of lengths and distances come from the two small constant tables
// below (all lanes read the same entry, a broadcast).
constexpr uint32_t len_info(uint32_t i) {  // base | extra << 16, RFC 1951 Sec. 3.2.5
  return i < 8 ? 3 + i : i == 28 ? 258u
                       : ((((4u + (i & 3u)) << ((i >> 2) - 1)) + 3u) | (((i >> 2) - 1) << 16));
}
constexpr uint32_t dist_info(uint32_t d) {
  return d < 4 ? 1 + d : ((((2u + (d & 1u)) << ((d >> 1) - 1)) + 1u) | (((d >> 1) - 1) << 16));
}
static __constant__ uint32_t kLenInfo[29] = {
    len_info(0),  len_info(1),  len_info(2),  len_info(3),  len_info(4),  len_info(5),
    len_info(6),  len_info(7),  len_info(8),  len_info(9),  len_info(10), len_info(11),
    len_info(12), len_info(13), len_info(14), len_info(15), len_info(16), len_info(17),
    len_info(18), len_info(19), len_info(20), len_info(21), len_info(22), len_info(23),
    len_info(24), len_info(25), len_info(26), len_info(27), len_info(28)};
static __constant__ uint32_t kDistInfo[30] = {
    dist_info(0),  dist_info(1),  dist_info(2),  dist_info(3),  dist_info(4),  dist_info(5),
    dist_info(6),  dist_info(7),  dist_info(8),  dist_info(9),  dist_info(10), dist_info(11),
    dist_info(12), dist_info(13), dist_info(14), dist_info(15), dist_info(16), dist_info(17),
    dist_info(18), dist_info(19), dist_info(20), dist_info(21), dist_info(22), dist_info(23),
    dist_info(24), dist_info(25), dist_info(26), dist_info(27), dist_info(28), dist_info(29)};

__device__ __forceinline__ uint16_t e16(uint32_t len, uint32_t kind, uint32_t val) {
  return (uint16_t)(len | (val << 4) | (kind << 12) | (kind == K_LIT ? 0x8000u : 0u));
}

// 16-bit entry for symbol `sym` with code length `len`.
__device__ __forceinline__ uint16_t sym_entry16(int kind, uint32_t len, uint32_t sym) {
  if (kind == 0) return e16(len, K_LIT, sym);
  if (kind == 1) {
    if (sym < 256) return e16(len, K_LIT, sym);
    if (sym == 256) return e16(len, K_EOB, 0);
    if (sym <= 285) return e16(len, K_BASE, sym - 257);
    return e16(len, K_BADSYM, 0);
  }
  if (sym < 30) return e16(len, K_BASE, sym);
  return e16(len, K_BADSYM, 0);
}

// Full entry (the 32-bit form the exact decoding path works with).
__device__ __forceinline__ uint32_t expand16(int kind, uint32_t e) {
  const uint32_t len = e & 15u, val = (e >> 4) & 0xffu;
  if (e & 0x8000u) return make_ent(len, K_LIT, 0, val);
  const uint32_t k = (e >> 12) & 7u;
  if (k == K_BASE) {
    const uint32_t info = kind == 1 ? kLenInfo[val] : kDistInfo[val];
    return make_ent(len, K_BASE, info >> 16, info & 0xffffu);
  }
  return make_ent(len, k, 0, val);
}

// Code-length code order, RFC 1951 Sec. 3.2.7.
static __constant__ uint8_t kClenOrder[19] = {16, 17, 18, 0, 8,  7, 9,  6, 10, 5,
                                       11, 4,  12, 3, 13, 2, 14, 1, 15};

// A canonical code in shared memory.
struct HCode {
  uint16_t* table;   // 1 << tb entries (16-bit form)
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
    uint16_t ent;
    if (kraft == 0) {
      ent = e16(0, K_BADCODE, 0);
    } else {
      ent = e16(0, K_LONG, 0);
      for (int L = 1; L <= tb; L++) {
        const uint32_t cc = rev >> (tb - L);
        const uint32_t k = cc - c.first[L];
        if (k < c.count[L]) {
          ent = sym_entry16(c.kind, (uint32_t)L, c.sorted[c.offset[L] + k]);
          break;
        }
        const uint32_t valid = (kraft + (1u << (15 - L)) - 1) >> (15 - L);
        if (cc >= valid) {
          ent = e16((uint32_t)L, K_BADCODE, 0);
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
  static constexpr int OFF_DIST = OFF_LIT + 2 * LIT_ENTRIES;
  static constexpr int OFF_WIN = OFF_DIST + 2 * DIST_ENTRIES;
  static constexpr int OFF_LSORT = OFF_WIN + WIN;  // WIN = 0: no shared window
  static constexpr int OFF_DSORT = OFF_LSORT + 2 * 288;
  static constexpr int OFF_META = OFF_DSORT + 2 * 32;  // 7 x u16[16]
  static constexpr int OFF_LENS = OFF_META + 7 * 32;
  static constexpr int BYTES = (OFF_LENS + 320 + 15) & ~15;
};

// Bit reader over the staging ring; all lanes hold the same state.
// bb holds nb valid stream bits (least significant = next); inpos is the
// next byte not yet loaded.  Bits past the chunk end read as zero.
template <class In>
struct BitIn {
  In* in;
  uint64_t bb;
  uint32_t nb;
  uint32_t inpos;
  uint32_t n_in;

  // Top up to >= 56 bits (or every remaining byte near the end).
  __device__ __forceinline__ bool refill() {
    // keep 8 bytes behind inpos resident: a stored block starts up to 8
    // bytes before the next unloaded byte
    const uint32_t keep = inpos >= 8 ? inpos - 8 : 0;
    if (inpos + 8 <= n_in) {  // branchless refill: 8 real bytes are there
      if (!in->ensure(keep, inpos + 8)) return false;
      bb |= in->u64(inpos) << nb;
      inpos += (63 - nb) >> 3;
      nb |= 56;
      return true;
    }
    if (inpos < n_in && !in->ensure(keep, n_in)) return false;
    while (nb <= 56 && inpos < n_in) {
      bb |= (uint64_t)in->byte(inpos) << nb;
      nb += 8;
      inpos++;
    }
    return true;
  }
  __device__ __forceinline__ uint32_t avail() const { return nb + 8u * (n_in - inpos); }
  __device__ __forceinline__ void consume(uint32_t k) {
    bb >>= k;
    nb -= k;
  }
  // byte position of the next unconsumed bit (which must be byte aligned)
  __device__ __forceinline__ uint32_t byte_pos() const { return inpos - (nb >> 3); }
  __device__ __forceinline__ void seek_byte(uint32_t p) {
    inpos = p;
    bb = 0;
    nb = 0;
  }
};

// Decode one raw Deflate chunk.  out: the chunk's output; cap: its span in
// bytes (STORE = false sizes the stream and ignores out/cap).  Chunks must be
// below 512 MiB compressed and 4 GiB decoded (32-bit positions).
template <bool STORE, int LIT_TB, int DIST_TB, int WIN, class Ring>
__device__ int32_t inflate_decode(Ring& ring, uint8_t* scratch, int64_t n_in64,
                                  uint8_t* __restrict__ out, uint64_t cap64, uint64_t* produced) {
  using SM = InflateSmem<LIT_TB, DIST_TB, WIN>;
  constexpr uint32_t WMASK = WIN == 0 ? 0 : WIN - 1;
  constexpr uint32_t FLUSH_T = WIN == 0 ? 0xffffffffu : WIN / 4;
  constexpr uint32_t NEAR_MAX = WIN == 0 ? 0xffffffffu : WIN - 512;
  constexpr uint32_t LITMASK = (1u << LIT_TB) - 1;
  constexpr uint32_t DISTMASK = (1u << DIST_TB) - 1;
  static_assert(WIN == 0 || (WIN >= 2048 && (WIN & (WIN - 1)) == 0), "window: 0 or a power of two >= 2048");
  constexpr bool GWIN = WIN == 0;  // output and match sources in global memory
  *produced = 0;
  if (n_in64 >= (int64_t)1 << 29 || (STORE && cap64 > 0xffffffffull)) return ST_BAD_SPAN;
  const uint32_t lane = lane_id();
  uint16_t* lit_tab = reinterpret_cast<uint16_t*>(scratch + SM::OFF_LIT);
  uint16_t* dist_tab = reinterpret_cast<uint16_t*>(scratch + SM::OFF_DIST);
  uint8_t* win = scratch + SM::OFF_WIN;
  uint16_t* meta = reinterpret_cast<uint16_t*>(scratch + SM::OFF_META);
  uint8_t* lens = scratch + SM::OFF_LENS;
  HCode lit{lit_tab, reinterpret_cast<uint16_t*>(scratch + SM::OFF_LSORT), meta, meta + 16,
            meta + 32, 0, LIT_TB, 1};
  HCode dist{dist_tab, reinterpret_cast<uint16_t*>(scratch + SM::OFF_DSORT), meta + 48, meta + 64,
             meta + 80, 0, DIST_TB, 2};
  uint16_t* run16 = meta + 96;

  const uint32_t n_in = (uint32_t)n_in64;
  BitIn<Ring> in{&ring, 0, 0, 0, n_in};
  const uint32_t oaddr = (uint32_t)reinterpret_cast<uintptr_t>(out);
  const uint32_t limit = STORE ? (uint32_t)cap64 : 0xffffffffu;
  uint32_t wpos = 0;     // bytes produced
  uint32_t flushed = 0;  // bytes already in global memory
  int fixed_ready = 0;   // the fixed tables are built in lit/dist
  int32_t st = ST_OK;

  // write window bytes of output [flushed, to) to global memory; `to` is either
  // a 16-byte boundary of the global address or the end of the output
  auto flush = [&](uint32_t to) {
    uint32_t f = flushed;
    const uint32_t head_end = ((oaddr + f + 15u) & ~15u) - oaddr;
    if (f < head_end) {  // unaligned head (first flush only)
      const uint32_t h = (head_end < to ? head_end : to) - f;
      if (lane < h) out[f + lane] = win[(oaddr + f + lane) & WMASK];
      f += h;
    }
    const uint32_t body_end = f + ((to - f) & ~15u);
    for (uint32_t b = f + 16 * lane; b < body_end; b += 512)
      *reinterpret_cast<uint4*>(out + b) = *reinterpret_cast<const uint4*>(win + ((oaddr + b) & WMASK));
    f = body_end;
    if (f < to && lane < to - f) out[f + lane] = win[(oaddr + f + lane) & WMASK];
    flushed = to;
  };
  // Far-match copies in flight: the source bytes (one per lane) are loaded
  // from global memory when the match is decoded and written to the window
  // later, so the load latency overlaps the decoding of later symbols.  A
  // copy is committed before anything could read or flush its bytes.
  struct PendingCopy {
    uint32_t dst, len, v;
  };
  PendingCopy pend_a{0, 0, 0}, pend_b{0, 0, 0};  // a is the older
  auto commit = [&](PendingCopy& p) {
    if (p.len) {
      if (lane < p.len) win[(oaddr + p.dst + lane) & WMASK] = (uint8_t)p.v;
      p.len = 0;
    }
  };
  auto commit_all = [&]() {
    commit(pend_a);
    commit(pend_b);
  };
  auto maybe_flush = [&]() {
    if (STORE && !GWIN && wpos - flushed >= FLUSH_T) {
      commit_all();
      __syncwarp();
      flush(((oaddr + wpos) & ~15u) - oaddr);
      __syncwarp();
    }
  };

  if (!in.refill()) return ST_TIMEOUT;
  for (;;) {
    // block header
    if (in.nb < 32 && !in.refill()) return ST_TIMEOUT;
    if (in.avail() < 3) { st = ST_TRUNCATED; break; }
    const uint32_t bfinal = (uint32_t)(in.bb & 1);
    const uint32_t btype = (uint32_t)((in.bb >> 1) & 3);
    in.consume(3);
    if (btype == 3) { st = ST_BAD_HEADER; break; }
    if (btype == 0) {  // stored block, RFC 1951 Sec. 3.2.4
      in.consume(in.nb & 7);  // to a byte boundary
      if (in.nb < 32 && !in.refill()) return ST_TIMEOUT;
      if (in.avail() < 32) { st = ST_TRUNCATED; break; }
      const uint32_t len = (uint32_t)(in.bb & 0xffff);
      const uint32_t nlen = (uint32_t)((in.bb >> 16) & 0xffff);
      if (len != (~nlen & 0xffffu)) { st = ST_BAD_STORED_LEN; break; }
      if (len > limit - wpos) { st = ST_OVERFLOW; break; }
      in.consume(32);
      const uint32_t src = in.byte_pos();
      if (len > n_in - src) { st = ST_TRUNCATED; break; }
      if (STORE && GWIN) {
        constexpr uint32_t GPIECE = Ring::MAX_SPAN - 16 < 512 ? Ring::MAX_SPAN - 16 : 512;
        for (uint32_t k0 = 0; k0 < len; k0 += GPIECE) {
          const uint32_t piece = len - k0 < GPIECE ? len - k0 : GPIECE;
          if (!ring.ensure(src + k0, src + k0 + piece + 8)) return ST_TIMEOUT;
          // every lane reads in every step (a register ring reads by shuffles)
          for (uint32_t kb = 0; kb < piece; kb += 32) {
            const uint32_t k = kb + lane;
            const uint8_t v = ring.byte(src + k0 + (k < piece ? k : piece - 1));
            if (k < piece) out[wpos + k0 + k] = v;
          }
        }
        __syncwarp();
      } else if (STORE) {
        commit_all();
        constexpr uint32_t PIECE0 = WIN / 4 < 1024 ? WIN / 4 : 1024;
        constexpr uint32_t PIECE = PIECE0 < Ring::MAX_SPAN - 16 ? PIECE0 : Ring::MAX_SPAN - 16;
        for (uint32_t k0 = 0; k0 < len; k0 += PIECE) {
          const uint32_t piece = len - k0 < PIECE ? len - k0 : PIECE;
          if (!ring.ensure(src + k0, src + k0 + piece + 8)) return ST_TIMEOUT;
          for (uint32_t k = 4 * lane; k < piece; k += 128) {
            const uint32_t v = ring.u32(src + k0 + k);
            const uint32_t at = oaddr + wpos + k0 + k;
            const uint32_t n4 = piece - k < 4 ? piece - k : 4;
            for (uint32_t t = 0; t < n4; t++) win[(at + t) & WMASK] = (uint8_t)(v >> (8 * t));
          }
          __syncwarp();
          const uint32_t w2 = wpos + k0 + piece;
          if (w2 - flushed >= FLUSH_T) flush(((oaddr + w2) & ~15u) - oaddr);
          __syncwarp();
        }
      }
      wpos += len;
      in.seek_byte(src + len);
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
        if (in.nb < 32 && !in.refill()) return ST_TIMEOUT;
        if (in.avail() < 14) { st = ST_TRUNCATED; break; }
        const int nlen = (int)(in.bb & 31) + 257;
        const int ndist = (int)((in.bb >> 5) & 31) + 1;
        const int ncode = (int)((in.bb >> 10) & 15) + 4;
        in.consume(14);
        if (nlen > 286 || ndist > 30) { st = ST_BAD_HUFFMAN; break; }
        if (!in.refill()) return ST_TIMEOUT;
        if (in.avail() < (uint32_t)(3 * ncode)) { st = ST_TRUNCATED; break; }
        // code-length code lengths; 19 x 3 = 57 bits: two reads
        uint64_t cl = in.bb;
        const uint32_t first_n = ncode < 18 ? ncode : 18;
        in.consume(3 * first_n);
        if (ncode > 18) {
          if (!in.refill()) return ST_TIMEOUT;
          cl = (cl & lowmask64(54)) | ((in.bb & 7) << 54);
          in.consume(3);
        }
        if (lane < 19) lens[kClenOrder[lane]] = (int)lane < ncode ? (uint8_t)((cl >> (3 * lane)) & 7) : 0;
        __syncwarp();
        HCode cl_code{dist_tab, dist.sorted, dist.first, dist.count, dist.offset, 0, 7, 0};
        if (build_code(cl_code, lens, 19, run16) != ST_OK) { st = ST_BAD_HUFFMAN; break; }
        const int total = nlen + ndist;
        int have = 0;
        bool bad = false;
        while (have < total) {
          if (in.nb < 16 && !in.refill()) return ST_TIMEOUT;
          const uint32_t e = expand16(0, dist_tab[in.bb & 127]);
          const uint32_t L = ent_len(e);
          if (L > in.avail()) { st = ST_TRUNCATED; bad = true; break; }
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
      // symbol loop.  Fast path while 8 input bytes and 258 output bytes
      // remain: no code can then run past the input or the output, so only
      // code validity and distances are checked.
      bool done = false;
      for (;;) {
        // Lean loop for the common symbols (literals; lengths and distances
        // whose codes fit the tables) far from both ends.  Nothing is
        // consumed for a symbol it does not finish; the exact path below
        // takes every other case.
        if (GWIN && STORE) {
          // A short non-overlapping match is loaded (lane i: byte i) when it is
          // decoded but stored only when the next match is decoded (before
          // that one reads its source) or the loop ends, so the load latency
          // of the source (earlier output, in L1/L2) overlaps the decoding in
          // between.  Literals land after the pending bytes, so order holds.
          uint32_t pdst = 0, plen = 0, pval = 0;
          while (in.inpos + 8 <= n_in && wpos + 258 <= limit) {
            if (in.nb < 48) {
              if (!ring.ensure(in.inpos >= 8 ? in.inpos - 8 : 0, in.inpos + 8)) return ST_TIMEOUT;
              in.bb |= ring.u64(in.inpos) << in.nb;
              in.inpos += (63 - in.nb) >> 3;
              in.nb |= 56;
            }
            uint32_t e = lit_tab[in.bb & LITMASK];
            if (e & 0x8000u) {  // up to 4 table literals (<= 10 bits each; >= 48 bits here)
              uint8_t* o = out + wpos;
              int k = 0;
              do {
                in.consume(e & 15u);
                if (lane == 0) o[k] = (uint8_t)(e >> 4);
                e = lit_tab[in.bb & LITMASK];
              } while ((e & 0x8000u) && ++k < 4);
              wpos += (uint32_t)k + ((e & 0x8000u) ? 0u : 1u);
              continue;
            }
            if ((e >> 12) != K_BASE) break;  // EOB, long or bad code
            const uint32_t li = kLenInfo[(e >> 4) & 0xffu];
            const uint32_t L = e & 15u, x = li >> 16;
            const uint32_t ed = dist_tab[(in.bb >> (L + x)) & DISTMASK];
            if ((ed >> 12) != K_BASE) break;
            const uint32_t di = kDistInfo[(ed >> 4) & 0xffu];
            const uint32_t Ld = ed & 15u, xd = di >> 16;
            const uint32_t mlen = (li & 0xffffu) + ((uint32_t)(in.bb >> L) & ((1u << x) - 1));
            const uint32_t d = (di & 0xffffu) + ((uint32_t)(in.bb >> (L + x + Ld)) & ((1u << xd) - 1));
            if (d > wpos) break;  // the exact path reports BAD_DISTANCE
            in.consume(L + x + Ld + xd);
            uint8_t* o = out + wpos;
            const uint8_t* src = o - d;
            if (plen) {  // store the pending match
              if (lane < plen) out[pdst + lane] = (uint8_t)pval;
              plen = 0;
            }
            __syncwarp();
            if (d >= mlen && mlen <= 32) {
              pval = lane < mlen ? src[lane] : 0u;
              pdst = wpos;
              plen = mlen;
            } else if (d >= mlen) {
              for (uint32_t i = lane; i < mlen; i += 32) o[i] = src[i];
            } else {  // overlap: byte i repeats source byte i mod d (exact float division here)
              const float r = __frcp_ru((float)d);
              uint32_t kk = lane - d * (uint32_t)__float2uint_rz((float)lane * r);
              const uint32_t step = 32u - d * (uint32_t)__float2uint_rz(32.0f * r);
              for (uint32_t i = lane; i < mlen; i += 32) {
                o[i] = src[kk];
                kk += step;
                if (kk >= d) kk -= d;
              }
            }
            wpos += mlen;
          }
          if (plen && lane < plen) out[pdst + lane] = (uint8_t)pval;
          __syncwarp();
        }
        const bool fast = in.inpos + 8 <= n_in && wpos + 258 <= limit;
        if (in.nb < 48 && !in.refill()) return ST_TIMEOUT;
        uint32_t e = expand16(1, lit_tab[in.bb & LITMASK]);
        if (fast && ent_kind(e) == K_LIT) {  // up to 3 literals per refill (<= 45 bits)
          int k = 0;
          do {
            in.consume(ent_len(e));
            if (STORE && lane == 0) {
              if (GWIN) out[wpos] = (uint8_t)ent_val(e);
              else win[(oaddr + wpos) & WMASK] = (uint8_t)ent_val(e);
            }
            wpos++;
            e = expand16(1, lit_tab[in.bb & LITMASK]);
          } while (ent_kind(e) == K_LIT && ++k < 3);
          maybe_flush();
          continue;
        }
        if (ent_kind(e) == K_LONG) e = decode_long(lit, in.bb);
        uint32_t L = ent_len(e);
        uint32_t kind = ent_kind(e);
        if (!fast && L > in.avail()) { st = ST_TRUNCATED; break; }
        if (kind >= K_BADSYM) { st = ST_BAD_HUFFMAN; break; }
        in.consume(L);
        if (kind == K_LIT) {
          if (!fast && wpos >= limit) { st = ST_OVERFLOW; break; }
          if (STORE && lane == 0) {
            if (GWIN) out[wpos] = (uint8_t)ent_val(e);
            else win[(oaddr + wpos) & WMASK] = (uint8_t)ent_val(e);
          }
          wpos++;
          maybe_flush();
          continue;
        }
        if (kind == K_EOB) { done = true; break; }
        // length
        uint32_t x = ent_extra(e);
        if (!fast && x > in.avail()) { st = ST_TRUNCATED; break; }
        const uint32_t mlen = ent_val(e) + (uint32_t)(in.bb & ((1u << x) - 1));
        in.consume(x);
        // distance
        e = expand16(2, dist_tab[in.bb & DISTMASK]);
        if (ent_kind(e) == K_LONG) e = decode_long(dist, in.bb);
        L = ent_len(e);
        kind = ent_kind(e);
        if (!fast && L > in.avail()) { st = ST_TRUNCATED; break; }
        if (kind >= K_BADSYM) { st = ST_BAD_HUFFMAN; break; }
        in.consume(L);
        x = ent_extra(e);
        if (!fast && x > in.avail()) { st = ST_TRUNCATED; break; }
        const uint32_t d = ent_val(e) + (uint32_t)(in.bb & ((1u << x) - 1));
        in.consume(x);
        if (d > wpos) { st = ST_BAD_DISTANCE; break; }
        if (!fast && mlen > limit - wpos) { st = ST_OVERFLOW; break; }
        if (STORE && GWIN) {
          // source bytes are earlier output of this warp, in global memory
          const uint32_t s0 = wpos - d;
          __syncwarp();
          if (d >= mlen) {
            for (uint32_t i = lane; i < mlen; i += 32) out[wpos + i] = out[s0 + i];
          } else {  // overlap: byte i repeats source byte i mod d
            uint32_t k = lane % d;
            const uint32_t step = 32 % d;
            for (uint32_t i = lane; i < mlen; i += 32) {
              out[wpos + i] = out[s0 + k];
              k += step;
              if (k >= d) k -= d;
            }
          }
        } else if (STORE) {
          const uint32_t s0 = wpos - d;
          if (d > NEAR_MAX && mlen <= 32) {
            // far source, already in global memory: load now, write later
            if (pend_a.len && pend_b.len) {  // both slots busy: retire the older
              commit(pend_a);
              pend_a = pend_b;
              pend_b.len = 0;
            }
            const PendingCopy nw{wpos, mlen, lane < mlen ? (uint32_t)__ldcg(out + s0 + lane) : 0u};
            if (!pend_a.len) pend_a = nw;
            else pend_b = nw;
          } else if (d > NEAR_MAX) {  // long far copy: synchronous
            commit_all();
            for (uint32_t i = lane; i < mlen; i += 32)
              win[(oaddr + wpos + i) & WMASK] = __ldcg(out + s0 + i);
            __syncwarp();
          } else {
            // near source in the window; it may overlap a pending far copy
            const uint32_t rd_end = s0 + (d < mlen ? d : mlen);
            if ((pend_a.len && s0 < pend_a.dst + pend_a.len && pend_a.dst < rd_end) ||
                (pend_b.len && s0 < pend_b.dst + pend_b.len && pend_b.dst < rd_end))
              commit_all();
            __syncwarp();
            if (d >= mlen) {
              for (uint32_t i = lane; i < mlen; i += 32)
                win[(oaddr + wpos + i) & WMASK] = win[(oaddr + s0 + i) & WMASK];
            } else {  // overlap: byte i repeats source byte i mod d
              uint32_t k = lane % d;
              const uint32_t step = 32 % d;
              for (uint32_t i = lane; i < mlen; i += 32) {
                win[(oaddr + wpos + i) & WMASK] = win[(oaddr + s0 + k) & WMASK];
                k += step;
                if (k >= d) k -= d;
              }
            }
          }
        }
        wpos += mlen;
        maybe_flush();
      }
      if (!done) break;
    }
    maybe_flush();
    if (bfinal) break;
  }
  if (STORE && !GWIN) {
    commit_all();
    __syncwarp();
    if (wpos > flushed) flush(wpos);
    __syncwarp();
  }
  if (STORE && GWIN) __syncwarp();
  *produced = wpos;
  if (st != ST_OK) return st;
  if (STORE && wpos < limit) return ST_UNDERFLOW;
  return ST_OK;
}

}  // namespace codag
