// Per-decoder input staging ring (CODAG Sec. IV-E, "coalesced on-demand
// reading": a warp refills an input buffer with whole cache lines when it has
// room, and decoding then reads from the buffer).
//
// GB300 form: the ring is NSLOT slots of SLOT bytes in shared memory.  Each
// slot is filled by one 1-D TMA bulk copy (cp.async.bulk, 16-byte aligned
// source and size) issued by lane 0 and completed on the slot's mbarrier; the
// ragged tail (< 16 bytes at the end of the readable range) is fetched with
// plain byte loads.  Refills are issued up to NSLOT slots ahead of the lowest
// position the decoder still needs, so the next slots are in flight while the
// current one is decoded.  Every lane keeps an identical copy of the ring
// state, like every other piece of decoder state.
//
// Positions are chunk-relative byte offsets.  Ring position r = chunk
// position + skew, where skew (0..15) aligns ring position 0 to 16 bytes.
// ensure(lo, hi) makes chunk bytes [lo, hi) resident and releases every slot
// below lo; hi - lo must not exceed (NSLOT - 1) * SLOT.  Bytes past the end
// of the readable range are never fetched: reads there return stale data and
// the decoders bound every read by the chunk length themselves.
#pragma once

#include "common.cuh"

namespace codag {

template <int SLOT_, int NSLOT_>
struct InRing {
  static constexpr int SLOT = SLOT_;
  static constexpr int NSLOT = NSLOT_;
  static constexpr int BYTES = SLOT * NSLOT;
  static constexpr int MAX_SPAN = (NSLOT - 1) * SLOT;
  static_assert((SLOT & (SLOT - 1)) == 0 && SLOT >= 64, "slot: power of two >= 64");
  static_assert((NSLOT & (NSLOT - 1)) == 0 && NSLOT >= 2, "nslot: power of two >= 2");
  // shared memory this ring needs: data + one mbarrier per slot
  static constexpr int SMEM = BYTES + 8 * NSLOT;

  uint8_t* buf;        // shared, BYTES, 128-byte aligned
  uint64_t* bar;       // shared, NSLOT mbarriers
  const uint8_t* gsrc; // 16-byte aligned global address of ring position 0
  int64_t skew;        // chunk start - gsrc
  int64_t limit;       // readable ring positions: [0, limit)
  uint32_t issued;     // slots issued for this chunk
  uint32_t ready;      // slots waited for (in order)
  uint32_t parity;     // per-slot mbarrier phase parity (persists across chunks)

  // Once per warp: carve the ring out of `smem` and initialise barriers.
  __device__ __forceinline__ void init(uint8_t* smem) {
    buf = smem;
    bar = reinterpret_cast<uint64_t*>(smem + BYTES);
    parity = 0;
    if (lane_id() == 0) {
      for (int s = 0; s < NSLOT; s++) mbar_init(&bar[s], 1);
      fence_mbar_init();
      fence_proxy_async_smem();
    }
    __syncwarp();
  }

  // Start a chunk of `len` bytes at `chunk`; `buf_end` bounds every read.
  __device__ __forceinline__ void start(const uint8_t* chunk, int64_t len, const uint8_t* buf_end) {
    gsrc = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(chunk) & ~uintptr_t(15));
    skew = chunk - gsrc;
    int64_t lim = (skew + len + 15) & ~int64_t(15);
    int64_t hard = buf_end - gsrc;
    limit = lim < hard ? lim : hard;
    issued = 0;
    ready = 0;
  }

  __device__ __forceinline__ void issue_next() {
    const uint32_t k = issued;
    const int s = k & (NSLOT - 1);
    const int64_t off = (int64_t)k * SLOT;
    int64_t bytes = limit - off;
    if (bytes > SLOT) bytes = SLOT;
    if (bytes > 0) {
      const uint32_t bulk = (uint32_t)bytes & ~15u;
      const uint32_t tail = (uint32_t)bytes - bulk;
      if (lane_id() == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[s], bulk);
        if (bulk) tma_load_1d(buf + s * SLOT, gsrc + off, bulk, &bar[s]);
      }
      if (lane_id() < tail) buf[s * SLOT + bulk + lane_id()] = __ldg(gsrc + off + bulk + lane_id());
    }
    issued = k + 1;
  }

  // Wait for slot `ready`; false if the bounded wait ran out.  A wait for
  // bytes the decoder needs is bounded by work_wait_ns(); the drain at the
  // end of a chunk (own copies in flight) by kMaxWaitNs.
  __device__ __forceinline__ bool wait_next(bool draining = false) {
    const uint32_t k = ready;
    const int s = k & (NSLOT - 1);
    if ((int64_t)k * SLOT < limit) {
      if (!mbar_wait_bounded(&bar[s], (parity >> s) & 1u, draining ? kMaxWaitNs : work_wait_ns()))
        return false;
      parity ^= 1u << s;
    }
    ready = k + 1;
    return true;
  }

  // Make chunk bytes [lo, hi) resident, release slots below lo and keep up to
  // NSLOT slots in flight.  False on a wait timeout.
  __device__ __forceinline__ bool ensure(int64_t lo, int64_t hi) {
    const int64_t rhi = hi + skew;
    if (rhi <= (int64_t)ready * SLOT) return true;
    __syncwarp();  // every lane's reads of released slots precede their refill
    const uint32_t k_lo = (uint32_t)((lo + skew) / SLOT);
    const uint32_t k_hi = (uint32_t)((rhi + SLOT - 1) / SLOT);
    while (issued < k_lo + NSLOT && (int64_t)issued * SLOT < limit) {
      // the buffer slot being refilled must have been waited for first
      while (ready + NSLOT <= issued)
        if (!wait_next()) return false;
      issue_next();
    }
    while (ready < k_hi) {
      if (ready >= issued) {  // past the readable range: nothing to wait for
        ready = k_hi;
        break;
      }
      if (!wait_next()) return false;
    }
    __syncwarp();
    return true;
  }

  // Wait for every copy still in flight (end of a chunk).
  __device__ __forceinline__ bool drain() {
    while (ready < issued)
      if (!wait_next(true)) return false;
    __syncwarp();
    return true;
  }

  __device__ __forceinline__ const uint8_t* chunk_ptr() const { return gsrc + skew; }

  // --- reads (chunk positions; the bytes must be resident) ---------------
  __device__ __forceinline__ uint8_t byte(int64_t p) const {
    return buf[(uint32_t)(p + skew) & (BYTES - 1)];
  }
  // 4 bytes starting at p, little-endian (byte p in bits 0..7).  Only the low
  // bits of p matter for the ring index, so 32-bit positions are enough.
  __device__ __forceinline__ uint32_t u32(uint32_t p) const {
    const uint32_t r = p + (uint32_t)skew;
    const uint32_t a = r & ~3u;
    const uint32_t lo = *reinterpret_cast<const uint32_t*>(buf + (a & (BYTES - 1)));
    const uint32_t hi = *reinterpret_cast<const uint32_t*>(buf + ((a + 4) & (BYTES - 1)));
    return __funnelshift_r(lo, hi, (r & 3u) * 8);
  }
  // 8 bytes starting at p, little-endian (byte p in bits 0..7)
  __device__ __forceinline__ uint64_t u64(int64_t p) const {
    const uint32_t r = (uint32_t)p + (uint32_t)skew;
    const uint32_t a = r & ~3u;
    const uint32_t sh = (r & 3u) * 8;
    const uint32_t w0 = *reinterpret_cast<const uint32_t*>(buf + (a & (BYTES - 1)));
    const uint32_t w1 = *reinterpret_cast<const uint32_t*>(buf + ((a + 4) & (BYTES - 1)));
    const uint32_t w2 = *reinterpret_cast<const uint32_t*>(buf + ((a + 8) & (BYTES - 1)));
    return ((uint64_t)__funnelshift_r(w1, w2, sh) << 32) | __funnelshift_r(w0, w1, sh);
  }
  // The same reads in big-endian byte order (byte p most significant): the
  // unaligned shift and the byte swap are one byte permute per result word.
  __device__ __forceinline__ uint32_t u32be(uint32_t p) const {
    const uint32_t r = p + (uint32_t)skew;
    const uint32_t a = r & ~3u;
    const uint32_t sel = 0x0123u + (r & 3u) * 0x1111u;
    const uint32_t w0 = *reinterpret_cast<const uint32_t*>(buf + (a & (BYTES - 1)));
    const uint32_t w1 = *reinterpret_cast<const uint32_t*>(buf + ((a + 4) & (BYTES - 1)));
    return __byte_perm(w0, w1, sel);
  }
  __device__ __forceinline__ uint64_t u64be(int64_t p) const {
    const uint32_t r = (uint32_t)p + (uint32_t)skew;
    const uint32_t a = r & ~3u;
    const uint32_t sel = 0x0123u + (r & 3u) * 0x1111u;
    const uint32_t w0 = *reinterpret_cast<const uint32_t*>(buf + (a & (BYTES - 1)));
    const uint32_t w1 = *reinterpret_cast<const uint32_t*>(buf + ((a + 4) & (BYTES - 1)));
    const uint32_t w2 = *reinterpret_cast<const uint32_t*>(buf + ((a + 8) & (BYTES - 1)));
    return ((uint64_t)__byte_perm(w0, w1, sel) << 32) | __byte_perm(w1, w2, sel);
  }
};

// Register staging ring (CODAG Sec. IV-E, the register input buffer): the
// warp keeps a 512-byte window of the chunk in registers, 8 bytes per lane in
// each of two 256-byte halves, plus the next 256 bytes already requested;
// ensure() slides the window forward by halves.  A read takes its bytes from
// the lane that holds them (__shfl_sync), so it needs no shared memory; every
// lane keeps the same window state.  Positions and the readable range are
// those of InRing; an ensure() span must not exceed MAX_SPAN.  Every read is
// a warp-wide shuffle, so all 32 lanes must make each read together (a lane
// may ask for a different position than the others); decoders that use it
// keep their per-lane loops at a warp-uniform trip count.
struct RegRing {
  static constexpr int HALF = 256;
  static constexpr int MAX_SPAN = HALF;
  static constexpr int SMEM = 0;
  const uint8_t* gsrc;  // 16-byte aligned global address of ring position 0
  int64_t skew;         // chunk start - gsrc
  int64_t limit;        // readable ring positions: [0, limit)
  int64_t base;         // ring position of the window start (a multiple of HALF)
  uint64_t h0, h1, nx;  // this lane's 8 bytes of the two halves and the next one

  __device__ __forceinline__ void init(uint8_t*) {}
  // 8 bytes at ring position r (a multiple of 8); bytes past the readable
  // range read as zero
  __device__ __forceinline__ uint64_t fetch(int64_t r) const {
    if (r + 8 <= limit) return __ldg(reinterpret_cast<const unsigned long long*>(gsrc + r));
    uint64_t v = 0;
    for (int k = 0; k < 8; k++)
      if (r + k < limit) v |= (uint64_t)__ldg(gsrc + r + k) << (8 * k);
    return v;
  }
  __device__ __forceinline__ void start(const uint8_t* chunk, int64_t, const uint8_t* buf_end) {
    gsrc = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(chunk) & ~uintptr_t(15));
    skew = chunk - gsrc;
    limit = buf_end - gsrc;
    base = 0;
    const int64_t l8 = 8 * (int64_t)lane_id();
    h0 = fetch(l8);
    h1 = fetch(HALF + l8);
    nx = fetch(2 * HALF + l8);
  }
  __device__ __forceinline__ bool ensure(int64_t lo, int64_t hi) {
    hi += skew;
    while (hi > base + 2 * HALF) {
      h0 = h1;
      h1 = nx;
      base += HALF;
      nx = fetch(base + 2 * HALF + 8 * (int64_t)lane_id());
    }
    return lo + skew >= base;
  }
  __device__ __forceinline__ bool drain() { return true; }
  __device__ __forceinline__ const uint8_t* chunk_ptr() const { return gsrc + skew; }
  // the 8 bytes at ring position r (a multiple of 8 inside the window)
  __device__ __forceinline__ uint64_t word(int64_t r) const {
    const uint32_t o = (uint32_t)(r - base);
    const int src = (int)((o >> 3) & 31);
    const uint64_t a = shfl64(h0, src), b = shfl64(h1, src);
    return o >= (uint32_t)HALF ? b : a;
  }
  __device__ __forceinline__ uint8_t byte(int64_t p) const {
    const int64_t r = p + skew;
    return (uint8_t)(word(r & ~int64_t(7)) >> (8 * (uint32_t)(r & 7)));
  }
  __device__ __forceinline__ uint64_t u64(int64_t p) const {
    const int64_t r = p + skew;
    const int64_t a = r & ~int64_t(7);
    const uint32_t sh = 8 * (uint32_t)(r & 7);
    const uint64_t w0 = word(a), w1 = word(a + 8);
    return sh ? (w0 >> sh) | (w1 << (64 - sh)) : w0;
  }
  __device__ __forceinline__ uint32_t u32(uint32_t p) const { return (uint32_t)u64(p); }
  __device__ __forceinline__ uint32_t u32be(uint32_t p) const { return bswap32(u32(p)); }
  __device__ __forceinline__ uint64_t u64be(int64_t p) const { return bswap64(u64(p)); }
};

// Input that is wholly resident in shared memory: a CTA stages a whole
// compressed chunk at once (TMA bulk copies on one mbarrier) and its warps
// read it with the same interface as the ring, without further waits.
struct StagedInput {
  const uint8_t* buf;   // shared; position 0 = gsrc
  const uint8_t* gsrc;  // 16-byte aligned global address of position 0
  int64_t skew;         // chunk start - gsrc

  __device__ __forceinline__ bool ensure(int64_t, int64_t) { return true; }
  __device__ __forceinline__ bool drain() { return true; }
  __device__ __forceinline__ const uint8_t* chunk_ptr() const { return gsrc + skew; }
  __device__ __forceinline__ uint8_t byte(int64_t p) const { return buf[(uint32_t)(p + skew)]; }
  __device__ __forceinline__ uint32_t u32(uint32_t p) const {
    const uint32_t r = p + (uint32_t)skew;
    const uint32_t a = r & ~3u;
    const uint32_t lo = *reinterpret_cast<const uint32_t*>(buf + a);
    const uint32_t hi = *reinterpret_cast<const uint32_t*>(buf + a + 4);
    return __funnelshift_r(lo, hi, (r & 3u) * 8);
  }
  __device__ __forceinline__ uint64_t u64(int64_t p) const {
    const uint32_t r = (uint32_t)p + (uint32_t)skew;
    const uint32_t a = r & ~3u;
    const uint32_t sh = (r & 3u) * 8;
    const uint32_t w0 = *reinterpret_cast<const uint32_t*>(buf + a);
    const uint32_t w1 = *reinterpret_cast<const uint32_t*>(buf + a + 4);
    const uint32_t w2 = *reinterpret_cast<const uint32_t*>(buf + a + 8);
    return ((uint64_t)__funnelshift_r(w1, w2, sh) << 32) | __funnelshift_r(w0, w1, sh);
  }
  // big-endian, as for InRing
  __device__ __forceinline__ uint32_t u32be(uint32_t p) const {
    const uint32_t r = p + (uint32_t)skew;
    const uint32_t a = r & ~3u;
    const uint32_t sel = 0x0123u + (r & 3u) * 0x1111u;
    const uint32_t w0 = *reinterpret_cast<const uint32_t*>(buf + a);
    const uint32_t w1 = *reinterpret_cast<const uint32_t*>(buf + a + 4);
    return __byte_perm(w0, w1, sel);
  }
  __device__ __forceinline__ uint64_t u64be(int64_t p) const {
    const uint32_t r = (uint32_t)p + (uint32_t)skew;
    const uint32_t a = r & ~3u;
    const uint32_t sel = 0x0123u + (r & 3u) * 0x1111u;
    const uint32_t w0 = *reinterpret_cast<const uint32_t*>(buf + a);
    const uint32_t w1 = *reinterpret_cast<const uint32_t*>(buf + a + 4);
    const uint32_t w2 = *reinterpret_cast<const uint32_t*>(buf + a + 8);
    return ((uint64_t)__byte_perm(w0, w1, sel) << 32) | __byte_perm(w1, w2, sel);
  }
};

// View of an input shifted by `base` bytes: a part decoder reads its own
// sub-stream (starting at a run boundary) with positions from 0.
template <class In>
struct OffsetIn {
  In* in;
  int64_t base;
  __device__ __forceinline__ bool ensure(int64_t lo, int64_t hi) { return in->ensure(lo + base, hi + base); }
  __device__ __forceinline__ const uint8_t* chunk_ptr() const { return in->chunk_ptr() + base; }
  __device__ __forceinline__ uint8_t byte(int64_t p) const { return in->byte(p + base); }
  __device__ __forceinline__ uint32_t u32(uint32_t p) const { return in->u32(p + (uint32_t)base); }
  __device__ __forceinline__ uint64_t u64(int64_t p) const { return in->u64(p + base); }
  __device__ __forceinline__ uint32_t u32be(uint32_t p) const { return in->u32be(p + (uint32_t)base); }
  __device__ __forceinline__ uint64_t u64be(int64_t p) const { return in->u64be(p + base); }
};

// The same view over a staging ring, for decoders that need the ring's span.
template <class Ring>
struct OffsetRing : OffsetIn<Ring> {
  static constexpr int MAX_SPAN = Ring::MAX_SPAN;
};

// Inputs whose every chunk byte is resident in shared memory (any position
// can be read at any time, without ensure()).
template <class In>
struct resident_input {
  static constexpr bool value = false;
};
template <>
struct resident_input<StagedInput> {
  static constexpr bool value = true;
};
template <class In>
struct resident_input<OffsetIn<In>> : resident_input<In> {};

// Big-endian 4- and 8-byte reads at chunk position p (MSB-first bit fields).
template <class In>
__device__ __forceinline__ uint32_t load_be32(const In& in, uint32_t p) { return in.u32be(p); }
template <class In>
__device__ __forceinline__ uint64_t load_be64(const In& in, int64_t p) { return in.u64be(p); }

// Bytes a staged chunk of n_in bytes needs: 16-byte alignment skew in front,
// and reads of up to 16 bytes past the last position (stale but in bounds).
__host__ __device__ __forceinline__ int64_t staged_bytes(int64_t n_in) { return n_in + 15 + 32; }

}  // namespace codag
