// One chunk (or one part of an RLE chunk), end to end, for any format:
// bounds checks on the offsets metadata (CODAG Sec. II-B: each chunk is
// located by its compressed and uncompressed offsets), staging-ring start,
// the format decoder, and the drain of in-flight staging copies.
#pragma once

#include "kernels.cuh"
#include "orc_frames.cuh"  // after kernels.cuh: uses the Deflate table sizes

namespace codag {

// Combinable status: the earliest error in stream order wins; a timeout wins
// over everything; ~0 means OK.
__device__ __forceinline__ unsigned long long status_key(const PartResult& r) {
  if (r.status == ST_OK) return ~0ull;
  if (r.status == ST_TIMEOUT) return (unsigned long long)ST_TIMEOUT;
  return ((unsigned long long)(r.err_pos + 1) << 4) | (unsigned long long)r.status;
}
__device__ __forceinline__ int32_t key_status(unsigned long long k) {
  return k == ~0ull ? ST_OK : (int32_t)(k & 15);
}

// Offsets checks for chunk c: its compressed range and (STORE) output span.
struct ChunkGeom {
  int32_t bad;  // ST_OK or ST_BAD_SPAN
  uint64_t cs;  // compressed start
  int64_t n_in; // compressed bytes
  uint64_t os;  // output start (STORE)
  uint64_t cap; // output span (STORE; ~0 when sizing)
};

template <int FAMILY, bool STORE>
__device__ __forceinline__ ChunkGeom chunk_geom(const Args& a, uint64_t c) {
  ChunkGeom g{ST_OK, 0, 0, 0, ~0ull};
  const uint64_t total = a.comp_off[a.n];
  const uint64_t cs = a.comp_off[c], ce = a.comp_off[c + 1];
  if (ce < cs || ce > total) { g.bad = ST_BAD_SPAN; return g; }
  g.cs = cs;
  g.n_in = (int64_t)(ce - cs);
  if (STORE) {
    g.os = a.out_off[c];
    const uint64_t oe = a.out_off[c + 1];
    if (oe < g.os) { g.bad = ST_BAD_SPAN; return g; }
    g.cap = oe - g.os;
    if (FAMILY <= 2 && ((g.cap & 7) || (g.os & 7))) g.bad = ST_BAD_SPAN;
  }
  return g;
}

// Value index where part k of K starts (parts split the output evenly).
__device__ __forceinline__ uint64_t part_target(uint64_t cap_v, uint32_t k, uint32_t K) {
  if (k >= K) return ~0ull;
  const uint64_t q = cap_v / K, rem = cap_v % K;
  return q * k + (k < rem ? k : rem);
}

// Segments of a chunk staged whole by the plain RLE kernels (K warps): about
// kSegValues values each (kSegValuesV1 for RLE v1, kSegBytesByteRle decoded
// bytes for byte RLE), at least K, at most kMaxSeg.
template <int FAMILY>
__host__ __device__ __forceinline__ uint32_t rle_seg_count(uint64_t cap_v, uint32_t K) {
  const uint64_t want = cap_v / (FAMILY == 1 ? kSegValuesV1 : FAMILY == 4 ? kSegBytesByteRle : kSegValues);
  return want < K ? K : want > (uint64_t)kMaxSeg ? (uint32_t)kMaxSeg : (uint32_t)want;
}

// Decode one part: the sub-stream of `in` starting at byte `base` (a run or
// group boundary whose first value index is count0), through the runs that
// start before value hi.  Error positions come back chunk-relative.
template <int FAMILY, bool STORE, class In>
__device__ __forceinline__ PartResult decode_rle_part(In& in, uint8_t* scratch, const Args& a,
                                                      const ChunkGeom& g, int format, int64_t base,
                                                      uint64_t count0, uint64_t hi,
                                                      V1Bitmap vb = V1Bitmap{nullptr, 0, 0}) {
  OffsetIn<In> sub{&in, base};
  uint64_t* out = reinterpret_cast<uint64_t*>(a.out + g.os);
  const uint64_t cap_v = g.cap / 8;
  PartResult r;
  vb.off += (uint32_t)base;
  if (FAMILY == 4) {  // byte / boolean RLE: counts are decoded bytes (booleans)
    r = byte_rle_part<STORE>(sub, g.n_in - base, format == FMT_BOOL_RLE, a.out + g.os, g.cap, count0, hi);
    if (r.status != ST_OK && r.status != ST_TIMEOUT) r.err_pos += base;
    return r;
  }
  if (FAMILY == 1)
    r = rle_v1_part<STORE>(sub, reinterpret_cast<uint16_t*>(scratch), g.n_in - base,
                           format == FMT_RLE_V1_I64, out, cap_v, count0, hi, vb);
  else
    r = rle_v2_part<STORE>(sub, scratch, g.n_in - base, format == FMT_RLE_V2_I64, out, cap_v,
                           count0, hi);
  if (r.status != ST_OK && r.status != ST_TIMEOUT) r.err_pos += base;
  r.count *= 8;
  return r;
}

// Walk a chunk (one warp) to the start of part k: returns (position, count),
// and false when a staging wait ran out on the way.
template <int FAMILY, class In>
__device__ __forceinline__ bool walk_to(In& in, uint8_t* scratch, int64_t n_in, uint64_t target,
                                        int64_t* pos, uint64_t* count) {
  uint64_t t[2] = {0, target};
  int64_t sp[2];
  uint64_t sc[2];
  bool ok;
  if (FAMILY == 1)
    ok = rle_v1_walk(in, reinterpret_cast<uint16_t*>(scratch), n_in, t, 1, sp, sc);
  else
    ok = rle_v2_walk(in, n_in, t, 1, sp, sc);
  // every lane computed the same values; lane 0 stored them
  *pos = (int64_t)shfl64((uint64_t)sp[1], 0);
  *count = shfl64(sc[1], 0);
  return ok;
}

// Part k of K of chunk c through a per-warp staging ring (batch kernel): the
// warp walks to its start, then decodes its runs from there.
template <int FAMILY, bool STORE, class Ring, int WIN = kWin>
__device__ __forceinline__ PartResult decode_part(Ring& ring, uint8_t* scratch, const Args& a,
                                                  uint64_t c, int format, uint32_t k, uint32_t K) {
  const ChunkGeom g = chunk_geom<FAMILY, STORE>(a, c);
  if (g.bad != ST_OK) return PartResult{g.bad, 0, 0};
  ring.start(a.comp + g.cs, g.n_in, a.comp + a.comp_off[a.n]);
  PartResult r;
  if (FAMILY == 3) {
    uint64_t prod = 0;
    const int32_t st =
        inflate_decode<STORE, kLitTB, kDistTB, WIN>(ring, scratch, g.n_in, a.out + g.os, g.cap, &prod);
    r = PartResult{st, 0, prod};
  } else if (FAMILY == 4) {
    r = byte_rle_decode<STORE>(ring, g.n_in, format == FMT_BOOL_RLE, a.out + g.os, g.cap);
  } else if (FAMILY == 5) {
    r = orc_zlib_decode<STORE>(ring, scratch, g.n_in, a.out + g.os, g.cap);
  } else {
    const uint64_t cap_v = g.cap / 8;
    int64_t base = 0;
    uint64_t count0 = 0;
    bool walked = true;
    if (k > 0) walked = walk_to<FAMILY>(ring, scratch, g.n_in, part_target(cap_v, k, K), &base, &count0);
    const uint64_t hi = (k + 1 < K) ? part_target(cap_v, k + 1, K) : ~0ull;
    if (walked) r = decode_rle_part<FAMILY, STORE>(ring, scratch, a, g, format, base, count0, hi);
    else r = PartResult{ST_TIMEOUT, 0, 0};
  }
  // bounded wait for this warp's own copies still in flight, also after a timeout
  if (!ring.drain()) r.status = ST_TIMEOUT;
  return r;
}

// Wait (bounded by work_wait_ns()) until at least k + 1 segment starts are
// published, napping nap_ns between looks.
__device__ __forceinline__ bool wait_published(volatile uint32_t* published, uint32_t k,
                                               uint32_t nap_ns = 128) {
  if (*published > k) return true;
  const uint64_t limit = work_wait_ns();
  if (limit == 0) return false;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t polls = 0; polls < kMaxWaitPolls; polls++) {
    __nanosleep(nap_ns);
    if (*published > k) return true;
    if (globaltimer_ns() - t0 > limit) return false;
  }
  return false;
}

// Plain RLE kernels: one CTA per chunk, K warps.  Shared memory:
// [stage][K scratch][mbarrier][key][published][claimed][segment tables]
// [RLE v1: terminator bitmap of the stage].
//
// A chunk that fits the stage is copied in whole by TMA (warp 0, one
// mbarrier).  Its output is cut into nseg segments of about equal numbers of
// values.  Warp 0 walks the run headers once and publishes where each
// segment starts (a run boundary) as soon as its walk reaches it; every warp,
// warp 0 included once its walk is done, claims segments with an atomic
// counter and decodes each one in place as soon as its start is known.
// Statuses combine by an atomic minimum over (stream position, code).
//
// A larger chunk is streamed: warp 0 walks it through a ring to the K part
// starts, then each warp streams its own part through a ring of its own.
template <int FAMILY, bool STORE>
__device__ __forceinline__ void rle_cta_body(const Args& a, int stage_bytes) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t K = blockDim.x >> 5;
  const uint32_t warp = threadIdx.x >> 5;
  const uint64_t c = blockIdx.x;
  uint8_t* stage = smem;
  uint8_t* scratch = smem + stage_bytes + warp * kRleScratch;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + stage_bytes + K * kRleScratch);
  unsigned long long* key = reinterpret_cast<unsigned long long*>(bar + 1);
  uint32_t* published = reinterpret_cast<uint32_t*>(bar + 2);
  uint32_t* claimed = published + 1;
  int64_t* split_pos = reinterpret_cast<int64_t*>(bar + 3);      // [kMaxSeg + 1]
  uint64_t* split_cnt = reinterpret_cast<uint64_t*>(split_pos + kMaxSeg + 1);
  uint64_t* target = split_cnt + kMaxSeg + 1;
  uint32_t* bitmap = reinterpret_cast<uint32_t*>(smem + stage_bytes + K * kRleScratch + kRleCtaExtra);
  const ChunkGeom g = chunk_geom<FAMILY, STORE>(a, c);
  if (g.bad != ST_OK) {
    if (threadIdx.x == 0) {
      a.status[c] = g.bad;
      if (!STORE) a.sizes[c] = 0;
    }
    return;
  }
  const uint8_t* chunk = a.comp + g.cs;
  const uint8_t* buf_end = a.comp + a.comp_off[a.n];
  const uint8_t* gsrc = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(chunk) & ~uintptr_t(15));
  const int64_t skew = chunk - gsrc;
  const bool staged = staged_bytes(g.n_in) <= stage_bytes;
  // output units the segments split: values (RLE), decoded bytes (byte /
  // boolean RLE)
  const uint64_t cap_v = FAMILY != 4 ? g.cap / 8 : a.format == FMT_BOOL_RLE ? (g.cap + 7) / 8 : g.cap;
  // segments: about kSegValues values each, at least K, at most kMaxSeg
  const uint32_t nseg = (staged && STORE) ? rle_seg_count<FAMILY>(cap_v, K) : K;
  // RLE v2 segment starts written by the walk pass (rle_v2_walk_kernel)
  const uint2* segt = (FAMILY == 2 && STORE && staged && nseg > 1 && a.seg) ? a.seg + c * kMaxSeg : nullptr;
  const bool prewalked = segt && segt[0].x == 1u;
  if (prewalked)
    for (uint32_t t = 1 + threadIdx.x; t < nseg; t += blockDim.x) {
      const uint2 e = segt[t];
      split_pos[t] = e.x;
      split_cnt[t] = e.y;
    }
  if (threadIdx.x == 0) {
    *key = ~0ull;
    *published = prewalked ? nseg : 1;
    *claimed = 0;
    split_pos[0] = 0;
    split_cnt[0] = 0;
    if (staged) {
      mbar_init(bar, 1);
      fence_mbar_init();
      fence_proxy_async_smem();
    }
  }
  for (uint32_t t = threadIdx.x; t <= nseg; t += blockDim.x) target[t] = part_target(cap_v, t, nseg);
  __syncthreads();
  if (staged) {
    // readable: [gsrc, buf_end); copy up to the chunk end rounded to 16
    int64_t bytes = (skew + g.n_in + 15) & ~int64_t(15);
    if (bytes > buf_end - gsrc) bytes = buf_end - gsrc;
    const uint32_t bulk = (uint32_t)bytes & ~15u;
    const uint32_t tail = (uint32_t)bytes - bulk;
    if (warp == 0) {
      if (lane_id() == 0) {
        mbar_arrive_expect_tx(bar, bulk);
        for (uint32_t off = 0; off < bulk; off += 16384) {
          const uint32_t piece = bulk - off < 16384 ? bulk - off : 16384;
          tma_load_1d(stage + off, gsrc + off, piece, bar);
        }
      }
      if (lane_id() < tail) stage[bulk + lane_id()] = __ldg(gsrc + bulk + lane_id());
    }
    bool ok = mbar_wait_bounded(bar, 0, work_wait_ns());
    // a wait that ran out still waits (kMaxWaitNs) for the copies in flight
    // before the CTA stops; the chunk reports TIMEOUT either way
    if (!ok) mbar_wait_bounded(bar, 0);
    ok = __syncthreads_and(ok);  // CTA-uniform; also publishes warp 0's tail bytes
    StagedInput in{stage, gsrc, skew};
    V1Bitmap vb{nullptr, (uint32_t)skew, 0};
    uint32_t nx_off = 0;  // RLE v1: stage offset of the group table (0: none)
    if (FAMILY == 1 && ok) {
      uint32_t* rank = bitmap + rle_v1_bitmap_words(stage_bytes);
      v1_build_bitmap(stage, (uint32_t)skew, (uint32_t)g.n_in, bitmap, rank,
                      rank + rle_v1_bitmap_words(stage_bytes));
      vb.bm = bitmap;
      vb.last_word = ((uint32_t)skew + (uint32_t)g.n_in + 31) >> 5;
      __syncthreads();
      // the group table goes to the unused tail of the stage when it fits
      nx_off = ((uint32_t)skew + (uint32_t)g.n_in + 48 + 15) & ~15u;
      if (nseg > 1 && nx_off + 4 * (uint32_t)g.n_in <= (uint32_t)stage_bytes) {
        v1_build_next(stage, (uint32_t)skew, (uint32_t)g.n_in, bitmap, rank, vb.last_word,
                      reinterpret_cast<uint32_t*>(stage + nx_off));
        __syncthreads();
      } else {
        nx_off = 0;
      }
    }
    if (!ok) {
      if (threadIdx.x == 0) *key = status_key(PartResult{ST_TIMEOUT, 0, 0});
    } else {
      if (warp == 0 && nseg > 1 && !prewalked) {
        if (FAMILY == 1 && nx_off)
          rle_v1_walk_next(reinterpret_cast<const uint32_t*>(stage + nx_off), (uint32_t)g.n_in,
                           target, (int)nseg - 1, split_pos, split_cnt, published);
        else if (FAMILY == 1)
          rle_v1_walk_staged(in, bitmap, bitmap + rle_v1_bitmap_words(stage_bytes),
                             (uint32_t)g.n_in, target, (int)nseg - 1, split_pos, split_cnt,
                             published);
        else if (FAMILY == 4)
          byte_rle_walk(in, g.n_in, target, (int)nseg - 1, split_pos, split_cnt, published);
        else if (cap_v < (1ull << 32))
          rle_v2_walk_lean(in, (uint32_t)g.n_in, target, nseg, split_pos, split_cnt, published);
        else
          rle_v2_walk_staged(in, (uint32_t)g.n_in, target, (int)nseg - 1, split_pos, split_cnt,
                             published);
      }
      for (;;) {
        uint32_t k = 0;
        if (lane_id() == 0) k = atomicAdd(claimed, 1u);
        k = __shfl_sync(FULL, k, 0);
        if (k >= nseg) break;
        PartResult r;
        // byte RLE: a segment start comes about every 130 control bytes of
        // a serial walk, so a longer nap costs no latency and spares the
        // walker's issue slots
        if (!wait_published(published, k, FAMILY == 4 ? 1024u : 128u)) {
          r = PartResult{ST_TIMEOUT, 0, 0};
        } else {
          __threadfence_block();
          const uint64_t hi = k + 1 < nseg ? target[k + 1] : ~0ull;
          r = decode_rle_part<FAMILY, STORE>(in, scratch, a, g, a.format, split_pos[k],
                                             split_cnt[k], hi, vb);
        }
        if (lane_id() == 0 && r.status != ST_OK) atomicMin(key, status_key(r));
        if (!STORE && k + 1 == nseg && lane_id() == 0) a.sizes[c] = r.count;
        if (r.status == ST_TIMEOUT) break;
      }
    }
  } else {
    RleRing ring;
    ring.init(stage + warp * RleRing::SMEM);
    bool ok = true;
    if (warp == 0 && K > 1) {
      ring.start(chunk, g.n_in, buf_end);
      if (FAMILY == 1)
        ok = rle_v1_walk(ring, reinterpret_cast<uint16_t*>(scratch), g.n_in, target, (int)K - 1,
                         split_pos, split_cnt);
      else if (FAMILY == 4)
        ok = byte_rle_walk(ring, g.n_in, target, (int)K - 1, split_pos, split_cnt);
      else
        ok = rle_v2_walk(ring, g.n_in, target, (int)K - 1, split_pos, split_cnt);
      ok = ring.drain() && ok;
    }
    // a walk whose wait ran out leaves unusable splits: the chunk times out
    ok = __syncthreads_and(ok);
    // this part's sub-stream, through a ring started at its first byte
    PartResult r{ST_TIMEOUT, 0, 0};
    if (ok) {
      const int64_t base = split_pos[warp];
      ChunkGeom sub = g;
      sub.n_in = g.n_in - base;
      ring.start(chunk + base, sub.n_in, buf_end);
      const uint64_t hi = warp + 1 < K ? target[warp + 1] : ~0ull;
      r = decode_rle_part<FAMILY, STORE>(ring, scratch, a, sub, a.format, 0, split_cnt[warp], hi);
      if (r.status != ST_OK && r.status != ST_TIMEOUT) r.err_pos += base;
      if (!ring.drain()) r.status = ST_TIMEOUT;
    }
    if (lane_id() == 0 && r.status != ST_OK) atomicMin(key, status_key(r));
    if (!STORE && warp == K - 1 && lane_id() == 0) a.sizes[c] = r.count;
  }
  __syncthreads();
  if (threadIdx.x == 0) a.status[c] = key_status(*key);
}

// Walk pass of the plain RLE v2 call (one warp per chunk): for every chunk
// that the decode pass (a.parts warps per CTA, a.stage_bytes of stage) stages
// whole and cuts into nseg > 1 segments, walk its run headers through a TMA
// ring and write where each segment starts, as rle_v2_walk_staged would
// publish it.  Every chunk's walk runs at once here, instead of one walk at a
// time on the critical path of each decode CTA.  A chunk that the walk pass
// leaves (other geometry, a value count past 32 bits, a wait that ran out)
// gets flag 0, and its decode CTA walks it itself.
__device__ __forceinline__ void rle_v2_walk_body(const Args& a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t warp = threadIdx.x >> 5;
  const uint64_t c = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= a.n) return;
  RleRing ring;
  ring.init(smem + warp * RleRing::SMEM);
  uint2* segt = a.seg + c * kMaxSeg;
  const ChunkGeom g = chunk_geom<2, true>(a, c);
  const uint64_t cap_v = g.cap / 8;
  const uint32_t nseg = rle_seg_count<2>(cap_v, (uint32_t)a.parts);
  if (g.bad != ST_OK || staged_bytes(g.n_in) > a.stage_bytes || nseg <= 1 || cap_v >= (1ull << 32)) {
    if (lane_id() == 0) segt[0] = make_uint2(0u, 0u);
    return;
  }
  const uint32_t n_in = (uint32_t)g.n_in;
  const uint32_t q = (uint32_t)(cap_v / nseg), rem = (uint32_t)(cap_v % nseg);
  ring.start(a.comp + g.cs, g.n_in, a.comp + a.comp_off[a.n]);
  uint32_t pos = 0, count = 0, k = 1;
  uint32_t tk = q + (1 < rem ? 1 : rem);  // part_target(cap_v, 1, nseg)
  bool ok = true;
  while (pos < n_in) {
    if (count >= tk) {
      do {
        if (lane_id() == 0) segt[k] = make_uint2(pos, count);
        if (++k >= nseg) break;
        tk = q * k + (k < rem ? k : rem);
      } while (count >= tk);
      if (k >= nseg) break;
    }
    if (!ring.ensure(pos, pos + 40)) {
      ok = false;
      break;
    }
    uint32_t len, end;
    if (!v2_run_extent(ring, pos, n_in, &len, &end)) break;
    count += len;
    pos = end;
  }
  if (ok)
    for (; k < nseg; k++)
      if (lane_id() == 0) segt[k] = make_uint2(pos, count);
  if (!ring.drain()) ok = false;
  if (lane_id() == 0) segt[0] = make_uint2(ok ? 1u : 0u, 0u);
}

// Plain kernels with one warp per chunk: Deflate (FAMILY 3), byte /
// boolean RLE (FAMILY 4) and ORC zlib streams (FAMILY 5).
// Ring: the shared-memory TMA ring (DeflateRing) or the register ring
// (RegRing, no shared memory for the input); per-warp shared memory holds
// the ring and the decoder scratch (Deflate tables; none for byte RLE).
template <int FAMILY, bool STORE, class Ring = DeflateRing>
__device__ __forceinline__ void warp_chunk_body(const Args& a) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr int kWarpSmem = warp_chunk_smem(FAMILY, Ring::SMEM);
  const uint32_t warp = threadIdx.x >> 5;
  const uint64_t c = (uint64_t)blockIdx.x * kWarpsPerBlock + warp;
  if (c >= a.n) return;
  if (a.deferred_only && a.status[c] != kDeferred) return;
  uint8_t* region = smem + warp * kWarpSmem;
  Ring ring;
  ring.init(region);
  const PartResult r = decode_part<FAMILY, STORE>(ring, region + Ring::SMEM, a, c, a.format, 0, 1);
  if (lane_id() == 0) {
    a.status[c] = r.status;
    if (!STORE) a.sizes[c] = r.count;
  }
}

}  // namespace codag
