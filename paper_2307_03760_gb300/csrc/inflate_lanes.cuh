// Raw Deflate (RFC 1951) in two passes: Huffman decoding with one LANE per
// chunk, then the LZ77 copies with one WARP per chunk (CODAG Sec. II-A,
// Deflate; Sec. IV-F, the dictionary copy of Alg. 2).
//
// Why two passes.  Decoding one chunk is one serial chain of table lookups.
// A warp that walks that chain with all 32 lanes issues every instruction 32
// times for one symbol; here a warp walks 32 chains at once, one per lane.
// What a lane cannot do well alone is the copy of a match (up to 258 bytes,
// sources in global memory): those are left to a second kernel in which a
// warp writes 32 consecutive output bytes per step.
//
// Pass 1, inflate_huffman_kernel (one CTA of kHufWarps warps per SM, lanes
// claim chunks from a global counter until none is left):
//   - every lane owns interleaved shared-memory tables (element k of lane l
//     at [k * 32 + l], so lanes that touch the same element index hit
//     different banks): an 8-bit lit/len table and a 7-bit distance table,
//     built by the lane itself per dynamic block (RFC 1951 Sec. 3.2.2); codes
//     longer than the table index resolve through per-length limits; fixed
//     blocks (Sec. 3.2.6) use one table pair per CTA (9-bit lit/len index,
//     so every fixed code is in the table).  The tables take 47 KB a warp,
//     so 4 warps (128 chunks) fit per SM;
//   - the lane reads its chunk from global memory through a four-word
//     register queue (the next words are in flight while the current ones are
//     decoded) into a 64-bit bit buffer;
//   - literals are stored straight to their output byte; everything else is
//     a 32-bit copy command appended to the chunk's command list:
//       match      (bit 31 = 0): R literals precede it (bits 0-7), length - 3
//                  (bits 8-15), distance - 1 (bits 16-30);
//       literals   (bits 31,30 = 1,0): R literals (bits 0-15), no match;
//       stored     (bits 31,30 = 1,1): LEN bytes (bits 0-15) of a stored
//                  block, copied by pass 2 from the compressed input; the
//                  block's input offset is parked in its first four output
//                  bytes (stored blocks of fewer than 4 bytes are literals);
//   - every check of the serial decoder is made here, in stream order, so a
//     chunk's status is final after this pass;
//   - chunk c's commands go to its region of the command pool, a quarter of
//     a word per byte of its output span plus two (words
//     [U_c / 4 + 2 c, U_{c+1} / 4 + 2 c + 2) with U_c the output offset from
//     the launch's first chunk), so chunks with disjoint output spans never
//     share pool words; a chunk whose commands do not fit its region, or
//     whose region is past the pool, is marked kDeferred and decoded later
//     by the one-warp decoder (inflate.cuh).
//
// Pass 2, inflate_lz77_kernel (one warp per chunk, many warps per SM): the
// commands are read 32 at a time, a warp prefix sum gives each one's output
// position, and the chunk's output is then written 32 bytes per step, lane i
// taking byte b + i: a literal byte is already in place, a stored byte comes
// from the input, a match byte from output position p - distance.  A source
// inside the current 32 bytes comes from the lane that holds it; chains of
// such sources (overlapping matches, Sec. IV-F) resolve by pointer jumping
// over shuffles, at most five rounds.
#pragma once

#include <cstddef>

#include "kernels.cuh"

namespace codag {

constexpr int kLaneLTB = 8;   // lit/len table index bits of a lane's (dynamic) code
constexpr int kFixLTB = 9;    // lit/len table index bits of the fixed code (every code fits)
constexpr int kLaneDTB = 7;   // distance (and code-length) table index bits
constexpr int kHufWarps = 4;  // warps per CTA of the Huffman kernel (one CTA per SM)
constexpr int kLz77Warps = 8;  // warps per CTA of the copy kernel
// Chunks that decode to more than this are left to the one-warp decoder
// (kDeferred): one lane decodes a chunk at about the speed of one warp, so a
// few long chunks would hold the whole Huffman pass (a 1 MiB chunk on one
// lane takes some 150 ms), while the one-warp pass runs them with the SM to
// fewer decoders.
constexpr uint32_t kHufMaxOut = 128u * 1024u;
// The sizes pass knows no output span: it leaves chunks of more compressed
// bytes than this to the one-warp decoder instead.
constexpr uint64_t kHufMaxInSizes = 64u * 1024u;

// Table entry (16 bits): bits 0-3 code length, 4-12 value, 13-15 kind.
// Values: a literal byte; a code-length symbol; a length symbol as index
// (0-28) | extra bits << 5; a distance code (0-29) | extra bits << 5.
__device__ __forceinline__ uint32_t lent(uint32_t len, uint32_t kind, uint32_t val) {
  return len | (val << 4) | (kind << 13);
}
__device__ __forceinline__ uint32_t lane_len_extra(uint32_t i) { return (i < 8 || i == 28) ? 0u : (i >> 2) - 1; }
__device__ __forceinline__ uint32_t lane_dist_extra(uint32_t d) { return d < 4 ? 0u : (d >> 1) - 1; }

// kind: 0 code-length code, 1 lit/len, 2 distance
__device__ __forceinline__ uint32_t lane_sym_entry(int kind, uint32_t len, uint32_t sym) {
  if (kind == 0) return lent(len, K_LIT, sym);
  if (kind == 1) {
    if (sym < 256) return lent(len, K_LIT, sym);
    if (sym == 256) return lent(len, K_EOB, 0);
    if (sym <= 285) return lent(len, K_BASE, (sym - 257) | (lane_len_extra(sym - 257) << 5));
    return lent(len, K_BADSYM, 0);
  }
  if (sym < 30) return lent(len, K_BASE, sym | (lane_dist_extra(sym) << 5));
  return lent(len, K_BADSYM, 0);
}

// Per-warp shared memory: interleaved per-lane arrays.
struct LaneTables {
  // lit and dist, one after the other, also hold the lane's code lengths
  // (up to 316) while a header is read; lsort then holds the code-length
  // code's table
  uint16_t lit[(1 << kLaneLTB) * 32];
  uint16_t dist[(1 << kLaneDTB) * 32];
  uint16_t lsort[288 * 32];  // table entries of the symbols, in canonical order
  uint16_t dsort[32 * 32];
  uint16_t lmeta[2 * (15 - kLaneLTB) * 32];  // limits, then bases, of lengths LTB+1..15
  uint16_t dmeta[2 * (15 - kLaneDTB) * 32];
};
// Per-CTA shared memory: the fixed codes' tables and the base values of
// lengths and distances (RFC 1951 Sec. 3.2.5, 3.2.6).
struct HufCta {
  uint16_t flit[1 << kFixLTB];
  uint16_t fdist[1 << kLaneDTB];
  uint32_t len_base[32];
  uint32_t dist_base[32];
};
constexpr int kHufSmem = kHufWarps * (int)sizeof(LaneTables) + (int)sizeof(HufCta);

// Counts, or running positions, of code lengths 0..15 in four registers of
// four 16-bit fields (no local memory for a per-lane array).
struct Len16 {
  uint64_t r0 = 0, r1 = 0, r2 = 0, r3 = 0;
  __device__ __forceinline__ uint32_t get(uint32_t L) const {
    const uint32_t g = L >> 2;
    const uint64_t r = g == 0 ? r0 : g == 1 ? r1 : g == 2 ? r2 : r3;
    return (uint32_t)(r >> (16 * (L & 3))) & 0xffffu;
  }
  __device__ __forceinline__ void add(uint32_t L, uint32_t v) {
    const uint64_t inc = (uint64_t)v << (16 * (L & 3));
    const uint32_t g = L >> 2;
    r0 += g == 0 ? inc : 0;
    r1 += g == 1 ? inc : 0;
    r2 += g == 2 ? inc : 0;
    r3 += g == 3 ? inc : 0;
  }
};

// Build a lane's canonical code (RFC 1951 Sec. 3.2.2) from lens[k * 32],
// k < n.  tab / sorted / meta are the lane's interleaved arrays (already
// offset by the lane).  Every per-lane array, the code lengths included, is
// a column of the same interleaved grid of 16-bit elements, so a lane never
// writes another lane's data, whatever point of its build each lane has
// reached.  Returns ST_OK or ST_BAD_HUFFMAN with the serial decoder's
// acceptance rules: over-subscribed codes are rejected, and incomplete ones
// too except a single length-1 code (lit/len, distance) or no code at all
// (distance).
template <int TB>
__device__ int32_t lane_build(const uint16_t* lens, int n, int kind, uint16_t* tab, uint16_t* sorted,
                              uint16_t* meta) {
  Len16 cnt;
  for (int k = 0; k < n; k++) cnt.add(lens[k * 32], 1);
  uint32_t kraft = 0, maxlen = 0, nshort = 0;
  uint32_t first[16], offset[16];
  {
    uint32_t code = 0, idx = 0, prev = 0;
#pragma unroll
    for (int L = 1; L <= 15; L++) {
      const uint32_t c = cnt.get(L);
      kraft += c << (15 - L);
      maxlen = c ? (uint32_t)L : maxlen;
      code = (code + prev) << 1;
      first[L] = code;
      offset[L] = idx;
      idx += c;
      prev = c;
      if (L == TB) nshort = idx;
    }
  }
  if (kraft > (1u << 15)) return ST_BAD_HUFFMAN;
  if (kraft < (1u << 15) && !((kind != 0 && maxlen == 1) || (kind == 2 && maxlen == 0)))
    return ST_BAD_HUFFMAN;
  // symbols in canonical order (by length, then symbol)
  Len16 pos;
#pragma unroll
  for (int L = 1; L <= 15; L++) pos.add(L, offset[L]);
  for (int k = 0; k < n; k++) {
    const uint32_t L = lens[k * 32];
    if (L) {
      const uint32_t p = pos.get(L);
      pos.add(L, 1);
      sorted[p * 32] = (uint16_t)lane_sym_entry(kind, L, (uint32_t)k);
    }
  }
  // table: entry t in code order (prefix t, most significant code bit
  // first) lives at the bit-reversed index, since the stream gives the code's
  // first bit first; canonical codes of length <= TB tile the prefixes in
  // order, so one sweep with a cursor fills the table
  const uint32_t dflt = kraft == 0 ? lent(0, K_BADCODE, 0)
                        : kraft < (1u << 15) ? lent(1, K_BADCODE, 0)
                                             : lent(0, K_LONG, 0);
  uint32_t idx = 0, end = 0, ent = dflt;
  for (uint32_t t = 0; t < (1u << TB); t++) {
    if (t == end && idx < nshort) {
      ent = sorted[idx * 32];
      end += 1u << (TB - (ent & 15));
      idx++;
    }
    tab[(__brev(t) >> (32 - TB)) * 32] = (uint16_t)(t < end ? ent : dflt);
  }
  // longer codes: per length, the end of its codes left-justified to 15 bits
  // (limits increase with the length) and the index offset into sorted
#pragma unroll
  for (int L = TB + 1; L <= 15; L++) {
    meta[(L - TB - 1) * 32] = (uint16_t)((first[L] + cnt.get(L)) << (15 - L));
    meta[(15 - TB + L - TB - 1) * 32] = (uint16_t)(offset[L] - first[L]);
  }
  return ST_OK;
}

// A code longer than TB bits, from the next 15 stream bits: its table entry
// (sorted holds the entries of all symbols in canonical order).  Only
// complete codes have such entries, so the search always ends at a code; NS
// bounds the index into sorted all the same.
template <int TB, uint32_t NS>
__device__ __forceinline__ uint32_t lane_long(uint64_t bb, const uint16_t* meta, const uint16_t* sorted) {
  const uint32_t rev = __brev((uint32_t)bb) >> 17;
  uint32_t L = 15;
#pragma unroll
  for (int i = 15 - TB - 1; i >= 0; i--)
    if (rev < meta[i * 32]) L = TB + 1 + i;
  const uint32_t base = meta[(15 - TB + L - TB - 1) * 32];
  const uint32_t k = (base + (rev >> (15 - L))) & 0xffffu;
  return sorted[(k < NS ? k : NS - 1) * 32];
}

// Per-lane bit reader over global memory.  Reader position r = chunk
// position + skew, where g8 (the chunk start rounded down to 8) is reader
// position 0; q0..q3 are the words at reader positions 8 qk .. 8 qk + 31.
struct LaneIn {
  const uint8_t* g8;
  const uint8_t* end;  // end of the readable buffer
  uint32_t skew;
  uint32_t nbits;  // 8 x chunk bytes
  uint32_t qk;
  uint32_t ipos;   // next reader position to load into bb
  uint32_t nb;     // valid bits in bb
  uint64_t bb;
  uint64_t q0, q1, q2, q3;

  // the word at reader position 8 k; bytes past the buffer read as zero
  __device__ static __noinline__ uint64_t word_tail(const uint8_t* p, const uint8_t* end) {
    uint64_t v = 0;
    for (int b = 0; b < 8; b++)
      if (p + b < end) v |= (uint64_t)__ldg(p + b) << (8 * b);
    return v;
  }
  __device__ __forceinline__ uint64_t word(uint32_t k) const {
    const uint8_t* p = g8 + 8ull * k;
    if (p + 8 <= end) return __ldg(reinterpret_cast<const unsigned long long*>(p));
    return word_tail(p, end);
  }
  __device__ __forceinline__ void seek(uint32_t chunk_pos) {
    ipos = chunk_pos + skew;
    qk = ipos >> 3;
    q0 = word(qk);
    q1 = word(qk + 1);
    q2 = word(qk + 2);
    q3 = word(qk + 3);
    bb = 0;
    nb = 0;
  }
  // Top up to >= 56 valid bits.  Safe to repeat: bits past nb are rewritten
  // with the same stream bits.
  __device__ __forceinline__ void refill() {
    const uint32_t sh = (ipos & 7) * 8;
    const bool lo = sh < 32;
    const uint32_t a = lo ? (uint32_t)q0 : (uint32_t)(q0 >> 32);
    const uint32_t b = lo ? (uint32_t)(q0 >> 32) : (uint32_t)q1;
    const uint32_t c = lo ? (uint32_t)q1 : (uint32_t)(q1 >> 32);
    const uint64_t v = ((uint64_t)__funnelshift_r(b, c, sh) << 32) | __funnelshift_r(a, b, sh);
    bb |= v << nb;
    ipos += (63 - nb) >> 3;
    nb |= 56;
    if ((ipos >> 3) != qk) {
      q0 = q1;
      q1 = q2;
      q2 = q3;
      qk++;
      q3 = word(qk + 3);
    }
  }
  __device__ __forceinline__ uint32_t used() const { return 8 * (ipos - skew) - nb; }
  __device__ __forceinline__ uint32_t avail() const { return nbits - used(); }
  __device__ __forceinline__ void consume(uint32_t k) {
    bb >>= k;
    nb -= k;
  }
};

// The command pool of a launch and its bookkeeping.
struct HufArgs {
  uint32_t* cmd;        // command pool (this launch's part)
  uint64_t pool_words;  // its size in words
  uint32_t* ncmd;       // per chunk: commands written
  uint32_t* counter;    // chunk claims, zeroed before the launch
  unsigned long long* need;  // pool words the launch needs (atomic max; a hint for the host)
};

// Start of chunk c's command region (see the file header).
__device__ __forceinline__ uint64_t cmd_region(const Args& a, uint64_t c) {
  return (a.out_off[c] - a.out_off[0]) / 4 + 2 * c;
}

enum : uint32_t { LS_NEED_CHUNK = 0, LS_NEED_HEADER = 1, LS_IN_BLOCK = 2, LS_GONE = 3 };

template <bool STORE>
struct LaneDec {
  const Args* a;
  const HufArgs* h;
  LaneTables* T;
  const HufCta* F;
  uint32_t lane;
  uint32_t state;
  uint64_t c;
  uint32_t bfinal;
  uint32_t wpos, cap;
  uint32_t run;   // literals since the last command
  uint32_t ncmd;
  uint32_t ccap;  // command words of the chunk's slot
  bool stuck;     // the fast step met a symbol it leaves to step()
  bool first;     // the lane has not claimed a chunk yet
  uint8_t* out;
  uint32_t* cmd;
  const uint16_t* lt;  // lit/len table, element stride ls, index mask lm
  uint32_t lm;
  const uint16_t* dt;  // distance table, element stride ds
  uint32_t ls, ds;
  LaneIn in;

  __device__ __forceinline__ void emit_cmd(uint32_t v) {
    if (ncmd < ccap) cmd[ncmd] = v;
    ncmd++;
  }
  __device__ __forceinline__ void emit_literal(uint32_t byte) {
    if (STORE) {
      out[wpos] = (uint8_t)byte;
      if (++run == 255) {
        emit_cmd(0x80000000u | 255u);
        run = 0;
      }
    }
    wpos++;
  }
  __device__ void finish(int32_t st) {
    if (STORE && st == ST_OK && wpos < cap) st = ST_UNDERFLOW;
    if (STORE && st == ST_OK) {
      if (run) emit_cmd(0x80000000u | run);
      run = 0;
      if (ncmd > ccap) st = kDeferred;
      h->ncmd[c] = ncmd;
    }
    a->status[c] = st;
    if (!STORE) a->sizes[c] = wpos;
    state = LS_NEED_CHUNK;
  }

  // Take the next chunk (state LS_NEED_CHUNK).  A lane's first chunk is
  // fixed: lane l of warp w (of W in the grid) takes chunk l * W + w, so a
  // call with fewer chunks than lanes spreads them over every warp (fewer
  // lanes per warp diverge less and each chunk's chain advances faster);
  // later chunks come from the counter, past the first 32 W.
  __device__ void claim() {
    const uint32_t W = gridDim.x * (blockDim.x >> 5);
    if (first) {
      first = false;
      c = (uint64_t)lane * W + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    } else {
      c = 32ull * W + atomicAdd(h->counter, 1u);
    }
    if (c >= a->n) {
      state = LS_GONE;
      return;
    }
    const uint64_t total = a->comp_off[a->n];
    const uint64_t cs = a->comp_off[c], ce = a->comp_off[c + 1];
    wpos = 0;
    run = 0;
    ncmd = 0;
    stuck = false;
    ccap = 0;
    cap = 0xffffffffu;
    if (ce < cs || ce > total) {
      finish(ST_BAD_SPAN);
      return;
    }
    const uint64_t n_in = ce - cs;
    if (STORE) {
      const uint64_t os = a->out_off[c], oe = a->out_off[c + 1];
      if (oe < os) {
        finish(ST_BAD_SPAN);
        return;
      }
      if (oe - os > 0xffffffffull) {
        finish(ST_BAD_SPAN);
        return;
      }
      cap = (uint32_t)(oe - os);
      if (cap > kHufMaxOut) {
        finish(kDeferred);
        return;
      }
      out = a->out + os;
      // the region of a chunk with a valid span; one past the pool (or an
      // output start before the launch's first) leaves the chunk to the
      // one-warp decoder
      const uint64_t o0 = a->out_off[0];
      if (os < o0) {
        finish(kDeferred);
        return;
      }
      const uint64_t r0 = cmd_region(*a, c), r1 = (oe - o0) / 4 + 2 * c + 2;
      if (r1 > h->pool_words) {
        finish(kDeferred);
        return;
      }
      cmd = h->cmd + r0;
      ccap = (uint32_t)((r1 - r0) < 0xffffffffull ? r1 - r0 : 0xffffffffull);
    }
    if (n_in >= (1ull << 29)) {
      finish(ST_BAD_SPAN);
      return;
    }
    if (!STORE && n_in > kHufMaxInSizes) {
      finish(kDeferred);
      return;
    }
    const uint8_t* chunk = a->comp + cs;
    in.g8 = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(chunk) & ~uintptr_t(7));
    in.skew = (uint32_t)(chunk - in.g8);
    in.end = a->comp + total;
    in.nbits = (uint32_t)(8 * n_in);
    in.seek(0);
    state = LS_NEED_HEADER;
  }

  // One block header (state LS_NEED_HEADER); a stored block is handled whole.
  __device__ void header() {
    in.refill();
    uint32_t avail = in.avail();
    if (avail < 3) return finish(ST_TRUNCATED);
    bfinal = (uint32_t)(in.bb & 1);
    const uint32_t btype = (uint32_t)((in.bb >> 1) & 3);
    in.consume(3);
    if (btype == 3) return finish(ST_BAD_HEADER);
    if (btype == 0) return stored();
    if (btype == 1) {
      lt = F->flit;
      lm = (1u << kFixLTB) - 1;
      dt = F->fdist;
      ls = ds = 1;
      state = LS_IN_BLOCK;
      return;
    }
    dynamic();
  }

  // RFC 1951 Sec. 3.2.4
  __device__ void stored() {
    in.consume(in.nb & 7);
    in.refill();
    if (in.avail() < 32) return finish(ST_TRUNCATED);
    const uint32_t len = (uint32_t)(in.bb & 0xffff);
    const uint32_t nlen = (uint32_t)((in.bb >> 16) & 0xffff);
    if (len != (~nlen & 0xffffu)) return finish(ST_BAD_STORED_LEN);
    if (STORE && len > cap - wpos) return finish(ST_OVERFLOW);
    in.consume(32);
    const uint32_t src = in.used() >> 3;
    const uint32_t n_in = in.nbits >> 3;
    if (len > n_in - src) return finish(ST_TRUNCATED);
    if (STORE && len >= 4) {
      if (run) emit_cmd(0x80000000u | run);
      run = 0;
      emit_cmd(0xC0000000u | len);
      // the block's input offset, parked in its first four output bytes
      out[wpos] = (uint8_t)src;
      out[wpos + 1] = (uint8_t)(src >> 8);
      out[wpos + 2] = (uint8_t)(src >> 16);
      out[wpos + 3] = (uint8_t)(src >> 24);
      wpos += len;
    } else if (STORE) {
      const uint8_t* p = in.g8 + in.skew + src;
      for (uint32_t i = 0; i < len; i++) emit_literal(__ldg(p + i));
    } else {
      wpos += len;
    }
    in.seek(src + len);
    if (bfinal) finish(ST_OK);
  }

  // RFC 1951 Sec. 3.2.7: code lengths, then the lane's own tables.  The
  // code lengths run through lit into dist (lit is the struct's first
  // array), the code-length code's table lives in lsort meanwhile, and the
  // lit/len code is built first: its sweep overwrites only lengths already
  // read, and the distance lengths (index >= 257) lie in dist.
  __device__ void dynamic() {
    static_assert((1 << kLaneLTB) + (1 << kLaneDTB) >= 286 + 30, "code lengths fit lit + dist");
    static_assert(offsetof(LaneTables, dist) == sizeof(uint16_t) * (1 << kLaneLTB) * 32, "dist follows lit");
    uint16_t* lens = T->lit + lane;
    uint16_t* dtab = T->dist + lane;
    uint16_t* ctab = T->lsort + lane;
    in.refill();
    if (in.avail() < 14) return finish(ST_TRUNCATED);
    const int nlen = (int)(in.bb & 31) + 257;
    const int ndist = (int)((in.bb >> 5) & 31) + 1;
    const int ncode = (int)((in.bb >> 10) & 15) + 4;
    in.consume(14);
    if (nlen > 286 || ndist > 30) return finish(ST_BAD_HUFFMAN);
    in.refill();
    if (in.avail() < (uint32_t)(3 * ncode)) return finish(ST_TRUNCATED);
    uint64_t cl = in.bb;
    const int first_n = ncode < 18 ? ncode : 18;
    in.consume(3 * first_n);
    if (ncode > 18) {
      in.refill();
      cl = (cl & lowmask64(54)) | ((in.bb & 7) << 54);
      in.consume(3);
    }
    for (int i = 0; i < 19; i++)
      lens[kClenOrder[i] * 32] = i < ncode ? (uint16_t)((cl >> (3 * i)) & 7) : 0;
    if (lane_build<kLaneDTB>(lens, 19, 0, ctab, T->dsort + lane, T->dmeta + lane) != ST_OK)
      return finish(ST_BAD_HUFFMAN);
    const int total = nlen + ndist;
    int have = 0;
    while (have < total) {
      in.refill();
      const uint32_t avail = in.avail();
      const uint32_t e = ctab[(uint32_t)(in.bb & 127) * 32];
      const uint32_t L = e & 15;
      if (L > avail) return finish(ST_TRUNCATED);
      if ((e >> 13) != K_LIT) return finish(ST_BAD_HUFFMAN);
      in.consume(L);
      const uint32_t sym = (e >> 4) & 0x1ff;
      if (sym < 16) {
        lens[have * 32] = (uint16_t)sym;
        have++;
        continue;
      }
      uint32_t rep, val = 0;
      if (sym == 16) {
        if (have == 0) return finish(ST_BAD_HUFFMAN);
        val = lens[(have - 1) * 32];
        if (avail - L < 2) return finish(ST_TRUNCATED);
        rep = 3 + (uint32_t)(in.bb & 3);
        in.consume(2);
      } else if (sym == 17) {
        if (avail - L < 3) return finish(ST_TRUNCATED);
        rep = 3 + (uint32_t)(in.bb & 7);
        in.consume(3);
      } else {
        if (avail - L < 7) return finish(ST_TRUNCATED);
        rep = 11 + (uint32_t)(in.bb & 127);
        in.consume(7);
      }
      if (have + (int)rep > total) return finish(ST_BAD_HUFFMAN);
      for (uint32_t j = 0; j < rep; j++) lens[(have + (int)j) * 32] = (uint16_t)val;
      have += (int)rep;
    }
    if (lens[256 * 32] == 0) return finish(ST_BAD_HUFFMAN);
    if (lane_build<kLaneLTB>(lens, nlen, 1, T->lit + lane, T->lsort + lane, T->lmeta + lane) != ST_OK)
      return finish(ST_BAD_HUFFMAN);
    if (lane_build<kLaneDTB>(lens + nlen * 32, ndist, 2, dtab, T->dsort + lane, T->dmeta + lane) != ST_OK)
      return finish(ST_BAD_HUFFMAN);
    lt = T->lit + lane;
    lm = (1u << kLaneLTB) - 1;
    dt = dtab;
    ls = ds = 32;
    state = LS_IN_BLOCK;
  }

  // The common step, far from both ends of the chunk: a literal (two when
  // the next code is a table literal too) or a length/distance pair.  Both
  // outcomes are computed and the stores predicated, so the lanes of a warp
  // (each on its own chunk) follow one instruction stream whatever symbol
  // each meets; only codes longer than the tables and the rare cases branch.
  // End of block, invalid codes and distances park the lane (stuck): the
  // next service phase decodes the same symbol again with step(), which makes
  // every check; nothing is consumed before that.
  __device__ __forceinline__ void fast_step() {
    constexpr uint32_t DM = (1u << kLaneDTB) - 1;
    in.refill();
    const uint64_t bb = in.bb;
    uint32_t e = lt[((uint32_t)bb & lm) * ls];
    if ((e >> 13) == K_LONG) e = lane_long<kLaneLTB, 288>(bb, T->lmeta + lane, T->lsort + lane);
    const uint32_t k = e >> 13;
    const bool islit = k == K_LIT;
    const uint32_t L = e & 15;
    const uint32_t x = islit ? 0u : (e >> 9) & 7;
    const uint32_t s1 = L + x;
    const uint64_t b1 = bb >> s1;
    const uint16_t* t2 = islit ? lt : dt;
    uint32_t e2 = t2[((uint32_t)b1 & (islit ? lm : DM)) * (islit ? ls : ds)];
    if (!islit && (e2 >> 13) == K_LONG) e2 = lane_long<kLaneDTB, 32>(b1, T->dmeta + lane, T->dsort + lane);
    const uint32_t k2 = e2 >> 13;
    const uint32_t L2 = e2 & 15;
    const uint32_t x2 = (e2 >> 9) & 15;
    const uint32_t mlen = F->len_base[(e >> 4) & 31] + ((uint32_t)(bb >> L) & ((1u << x) - 1));
    const uint32_t d = F->dist_base[(e2 >> 4) & 31] + ((uint32_t)(b1 >> L2) & ((1u << x2) - 1));
    if (k > K_BASE || (!islit && (k2 != K_BASE || d > wpos))) {
      stuck = true;
      return;
    }
    const bool two = islit && k2 == K_LIT && (!STORE || wpos + 1 < cap);
    in.consume(islit ? (two ? L + L2 : L) : s1 + L2 + x2);
    const uint32_t n = two ? 2u : 1u;
    if (STORE) {
      const bool flush = islit && run + n > 255;
      if (islit) out[wpos] = (uint8_t)(e >> 4);
      if (two) out[wpos + 1] = (uint8_t)(e2 >> 4);
      const bool put = flush || !islit;
      const uint32_t cv = islit ? (0x80000000u | run) : (run | ((mlen - 3) << 8) | ((d - 1) << 16));
      if (put && ncmd < ccap) cmd[ncmd] = cv;
      ncmd += put ? 1u : 0u;
      run = islit ? (flush ? n : run + n) : 0u;
    }
    wpos += islit ? n : mlen;
  }
  // whether fast_step() may run: 48 bits (the longest step) are left in the
  // chunk and 258 + 2 bytes in the output span
  __device__ __forceinline__ bool fast_ok() const {
    return in.avail() >= 64 && (!STORE || cap - wpos >= 260);
  }

  // One symbol (state LS_IN_BLOCK), and a second one when both are table
  // literals.  The checks and their order are the serial decoder's.
  __device__ void step() {
    constexpr uint32_t DM = (1u << kLaneDTB) - 1;
    in.refill();
    uint32_t avail = in.avail();
    uint32_t e = lt[((uint32_t)in.bb & lm) * ls];
    if ((e >> 13) == K_LONG) e = lane_long<kLaneLTB, 288>(in.bb, T->lmeta + lane, T->lsort + lane);
    const uint32_t L = e & 15;
    const uint32_t k = e >> 13;
    if (L > avail) return finish(ST_TRUNCATED);
    if (k >= K_BADSYM) return finish(ST_BAD_HUFFMAN);
    if (k == K_EOB) {
      in.consume(L);
      if (bfinal) return finish(ST_OK);
      state = LS_NEED_HEADER;
      return;
    }
    if (k == K_LIT) {
      if (STORE && wpos >= cap) return finish(ST_OVERFLOW);
      in.consume(L);
      avail -= L;
      emit_literal((e >> 4) & 0xffu);
      const uint32_t e2 = lt[((uint32_t)in.bb & lm) * ls];
      if ((e2 >> 13) == K_LIT && (e2 & 15) <= avail && (!STORE || wpos < cap)) {
        in.consume(e2 & 15);
        emit_literal((e2 >> 4) & 0xffu);
      }
      return;
    }
    // length, then distance
    const uint32_t v = (e >> 4) & 0x1ff;
    const uint32_t x = v >> 5;
    if (L + x > avail) return finish(ST_TRUNCATED);
    const uint32_t mlen = F->len_base[v & 31] + ((uint32_t)(in.bb >> L) & ((1u << x) - 1));
    in.consume(L + x);
    avail -= L + x;
    uint32_t ed = dt[(uint32_t)(in.bb & DM) * ds];
    if ((ed >> 13) == K_LONG) ed = lane_long<kLaneDTB, 32>(in.bb, T->dmeta + lane, T->dsort + lane);
    const uint32_t Ld = ed & 15;
    if (Ld > avail) return finish(ST_TRUNCATED);
    if ((ed >> 13) != K_BASE) return finish(ST_BAD_HUFFMAN);
    const uint32_t vd = (ed >> 4) & 0x1ff;
    const uint32_t xd = vd >> 5;
    if (Ld + xd > avail) return finish(ST_TRUNCATED);
    const uint32_t d = F->dist_base[vd & 31] + ((uint32_t)(in.bb >> Ld) & ((1u << xd) - 1));
    in.consume(Ld + xd);
    if (d > wpos) return finish(ST_BAD_DISTANCE);
    if (STORE && mlen > cap - wpos) return finish(ST_OVERFLOW);
    if (STORE) {
      emit_cmd(run | ((mlen - 3) << 8) | ((d - 1) << 16));
      run = 0;
    }
    wpos += mlen;
  }
};

// Fixed codes (RFC 1951 Sec. 3.2.6) and the length / distance bases, for
// the CTA.  Lit/len prefixes in code order: 7-bit codes 0-23 are symbols
// 256-279, 8-bit codes 48-191 are 0-143, 8-bit codes 192-199 are 280-287,
// 9-bit codes 400-511 are 144-255; distance codes are 5 bits.
__device__ __forceinline__ void huf_cta_init(HufCta* F) {
  for (uint32_t t = threadIdx.x; t < (1u << kFixLTB); t += blockDim.x) {
    uint32_t sym, L;
    if ((t >> 2) < 24) { sym = 256 + (t >> 2); L = 7; }
    else if ((t >> 1) < 192) { sym = (t >> 1) - 48; L = 8; }
    else if ((t >> 1) < 200) { sym = 280 + (t >> 1) - 192; L = 8; }
    else { sym = 144 + t - 400; L = 9; }
    F->flit[__brev(t) >> (32 - kFixLTB)] = (uint16_t)lane_sym_entry(1, L, sym);
  }
  for (uint32_t t = threadIdx.x; t < (1u << kLaneDTB); t += blockDim.x)
    F->fdist[__brev(t) >> (32 - kLaneDTB)] = (uint16_t)lane_sym_entry(2, 5, t >> 2);
  for (uint32_t i = threadIdx.x; i < 32; i += blockDim.x) {
    F->len_base[i] = i < 29 ? (kLenInfo[i] & 0xffffu) : 0u;
    F->dist_base[i] = i < 30 ? (kDistInfo[i] & 0xffffu) : 0u;
  }
}

// Pass 1 body: every lane decodes chunks it claims until none is left.
// Lanes waiting for a block header (or a new chunk) are served together once
// a quarter of the live lanes wait, so that header work (serial per lane)
// overlaps across lanes.
template <bool STORE>
__device__ void huffman_body(const Args& a, const HufArgs& h) {
  extern __shared__ __align__(128) uint8_t smem[];
  HufCta* F = reinterpret_cast<HufCta*>(smem + kHufWarps * sizeof(LaneTables));
  huf_cta_init(F);
  if (STORE && blockIdx.x == 0 && threadIdx.x == 0)  // the pool this launch needs, for the next call
    atomicMax(h.need, (unsigned long long)((a.out_off[a.n] - a.out_off[0]) / 4 + 2 * a.n + 2));
  __syncthreads();
  LaneDec<STORE> s;
  s.a = &a;
  s.h = &h;
  s.T = reinterpret_cast<LaneTables*>(smem) + (threadIdx.x >> 5);
  s.F = F;
  s.lane = lane_id();
  s.state = LS_NEED_CHUNK;
  s.first = true;
  for (;;) {
    while (s.state == LS_NEED_CHUNK) s.claim();
    if (__all_sync(FULL, s.state == LS_GONE)) break;
    while (__any_sync(FULL, s.state == LS_NEED_HEADER)) {
      if (s.state == LS_NEED_HEADER) s.header();
      while (s.state == LS_NEED_CHUNK) s.claim();
    }
    // hot loop: only the fast step; it ends when no lane can take one, or
    // every 8 steps when a quarter of the live lanes wait (header, new
    // chunk, or a symbol the fast step leaves to the exact one)
    for (uint32_t it = 0;; it++) {
      const bool act = s.state == LS_IN_BLOCK && !s.stuck && s.fast_ok();
      const uint32_t am = __ballot_sync(FULL, act);
      if (!am) break;
      if ((it & 7) == 7) {
        const uint32_t live = __ballot_sync(FULL, s.state != LS_GONE);
        if (4 * __popc(am) <= 3 * __popc(live)) break;
      }
      if (act) s.fast_step();
    }
    // service: lanes in a block that cannot take a fast step take exact
    // steps until they can again (or leave the block), a bounded number
    for (int j = 0; j < 64; j++) {
      const bool need = s.state == LS_IN_BLOCK && (s.stuck || !s.fast_ok());
      if (!__any_sync(FULL, need)) break;
      if (need) {
        s.stuck = false;
        s.step();
      }
    }
  }
}

// Pass 2 body: the copies of chunk c (one warp).
__device__ __forceinline__ void lz77_chunk(const Args& a, const HufArgs& h, uint64_t c) {
  if (a.status[c] != ST_OK) return;  // errors keep an unspecified output; deferred chunks come later
  const uint32_t lane = lane_id();
  const uint64_t os = a.out_off[c];
  const uint32_t cap = (uint32_t)(a.out_off[c + 1] - os);
  const uint64_t cs = a.comp_off[c];
  const uint32_t n_in = (uint32_t)(a.comp_off[c + 1] - cs);
  uint8_t* out = a.out + os;
  const uint8_t* in = a.comp + cs;
  const uint32_t* cmd = h.cmd + cmd_region(a, c);
  const uint32_t ncmd = h.ncmd[c];
  uint32_t opos = 0;
  for (uint32_t g = 0; g < ncmd; g += 32) {
    const uint32_t j = g + lane;
    const uint32_t v = j < ncmd ? cmd[j] : 0x80000000u;  // past the end: 0 literals
    // rm = R | M << 8 (M: match or stored length), bit 31 stored; aux =
    // distance (match) or input offset (stored)
    uint32_t len, rm, aux;
    if (!(v >> 31)) {
      const uint32_t m = ((v >> 8) & 255u) + 3;
      len = (v & 255u) + m;
      rm = (v & 255u) | (m << 8);
      aux = (v >> 16) + 1;
    } else if (!((v >> 30) & 1)) {
      len = v & 0xffffu;
      rm = len;
      aux = 0;
    } else {
      len = v & 0xffffu;
      rm = 0x80000000u | (len << 8);
      aux = 0;
    }
    const uint32_t incl = warp_incl_scan32(len);
    const uint32_t start = opos + incl - len;
    const uint32_t gend0 = opos + __shfl_sync(FULL, incl, 31);
    const uint32_t gend = gend0 < cap ? gend0 : cap;  // defensive: never past the span
    if ((rm >> 31) && start + 4 <= cap)  // stored: the parked input offset
      aux = (uint32_t)out[start] | ((uint32_t)out[start + 1] << 8) | ((uint32_t)out[start + 2] << 16) |
            ((uint32_t)out[start + 3] << 24);
    __syncwarp();
    for (uint32_t b = opos; b < gend; b += 32) {
      const uint32_t p = b + lane;
      const uint32_t starts = __reduce_or_sync(FULL, (len && start >= b && start < b + 32) ? 1u << (start - b) : 0u);
      const uint32_t before = __popc(__ballot_sync(FULL, len && start < b));
      const uint32_t jl = before + __popc(starts & (0xffffffffu >> (31 - lane))) - 1;
      const uint32_t cstart = __shfl_sync(FULL, start, jl);
      const uint32_t crm = __shfl_sync(FULL, rm, jl);
      const uint32_t caux = __shfl_sync(FULL, aux, jl);
      const uint32_t o = p - cstart;
      const bool live = p < gend;
      const bool stored = crm >> 31;
      const bool lit = !stored && o < (crm & 255u);
      const uint32_t src = p - caux;  // match source (wraps when invalid)
      const bool inwin = live && !stored && !lit && caux <= p && src >= b;
      // every lane loads its value: a literal lane its own (already written)
      // byte, which a later lane of this window may copy.  (Gating that load
      // on a warp vote whose result only this branch used hung the warp on
      // GB300; an unconditional coalesced load costs little.)
      uint32_t val = 0;
      if (live) {
        if (stored) {
          const uint32_t q = caux + o;
          if (q < n_in) val = __ldg(in + q);
        } else if (lit) {
          val = out[p];
        } else if (!inwin && caux <= p) {
          val = out[src];
        }
      }
      bool ready = !inwin;
      uint32_t sl = inwin ? src - b : lane;
      // every source lane is below its reader, so five rounds resolve any chain
      for (int r = 0; r < 5 && !__all_sync(FULL, ready); r++) {
        const uint32_t v2 = __shfl_sync(FULL, val, sl);
        const bool r2 = __shfl_sync(FULL, ready, sl);
        const uint32_t s2 = __shfl_sync(FULL, sl, sl);
        if (!ready) {
          if (r2) {
            val = v2;
            ready = true;
          } else {
            sl = s2;
          }
        }
      }
      if (live && !lit) out[p] = (uint8_t)val;
      __syncwarp();
    }
    opos = gend;
  }
}

}  // namespace codag
