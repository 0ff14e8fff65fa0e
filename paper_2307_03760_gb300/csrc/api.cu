// Host side of the C ABI (include/codag.h): argument checks, the per-device
// workspace, kernel launches and the batch graph.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/codag.h"
#include "kernels.cuh"
#include "inflate_lanes.cuh"  // after kernels.cuh: uses Args

using namespace codag;

namespace {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_batch_ctas_per_sm{0};
// plain RLE v2: walk pass before the decode pass (1) or the walk inside each
// decode CTA (0, the default: faster on GB300 for the 128 KiB-chunk column,
// 104 against 127 us); codag_set_walk_pass
std::atomic<int> g_walk_pass{0};
// the walk pass's table is kMaxSeg * 8 bytes per chunk: calls with more
// chunks than this walk inside the decode CTAs
constexpr uint64_t kMaxWalkChunks = 1ull << 18;
std::atomic<int> g_batch_shape{kBatchShapeDefault};  // index into batch_shape()
std::atomic<uint32_t> g_split_lg{kSplitLgDefault}, g_split_max{kSplitMaxDefault};
std::atomic<int> g_parts_per_chunk{0};
std::atomic<int> g_reg_ring[8];  // per decoder family: 1 = register staging ring
std::atomic<uint64_t> g_pool_limit{0};  // Deflate command pool bound in bytes (0: none)
std::atomic<uint64_t> g_wait_limit{100ull * 1000 * 1000};  // work-wait bound of the kernels, ns

codag_status fail(codag_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

codag_status cuda_fail(cudaError_t e, const char* what) {
  return fail(CODAG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr int kMaxDevices = 64;

// Host-to-host decode (codag_decompress_host): two copy streams, kPipeDecode
// decode streams (slices decode concurrently, so that small slices still fill
// the GPU), events per slice, and device copies of the two offsets arrays.
constexpr uint64_t kSliceBytes = 16ull << 20;
constexpr int kMaxSlices = 64;
constexpr int kPipeDecode = 4;

// Two-pass Deflate command pool: its first size in words (enough for about
// 64 MiB of output), grown to what an earlier call needed.
constexpr uint64_t kHufPoolInitWords = 1ull << 24;
struct HostPipe {
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaStream_t dec[kPipeDecode] = {};
  cudaEvent_t start = nullptr, done = nullptr;
  cudaEvent_t copied[kMaxSlices] = {}, decoded[kMaxSlices] = {};
  bool used = false;         // `done` marks the end of an earlier call
  uint64_t* offs = nullptr;  // comp offsets, then out offsets
  uint64_t offs_cap = 0;     // words
};

struct Workspace {
  HostPipe pipe;
  int32_t* status = nullptr;     // per-chunk status of the last plain call
  uint64_t status_cap = 0;
  uint64_t last_n = 0;
  uint32_t* order = nullptr;     // batch claim order
  unsigned long long* keys = nullptr;  // batch combined status of multi-part chunks
  uint64_t order_cap = 0;
  uint32_t* counters = nullptr;  // kBatchCounterWords words
  bool attrs_set = false;
  int sm_count = 0;
  int smem_per_sm = 0;     // shared memory per SM, bytes
  int smem_reserved = 0;   // shared memory the system keeps per CTA
  int smem_optin = 0;      // largest dynamic shared memory per CTA
  // dynamic shared memory per CTA of the CTA-per-chunk RLE kernels at the
  // CTAs per SM that threads and registers allow, by kernel (decode or
  // sizes: their register counts differ), family (1, 2, 4) and warps per CTA
  // (1..16); 0 = not known yet, -1 = unknown
  mutable int rle_avail[2][5][17] = {};
  // two-pass Deflate: the copy-command pool, the per-chunk command counts,
  // chunk-claim counters (one per concurrent slice of codag_decompress_host,
  // one for plain calls), and the pool size the last call needed (a device
  // word, copied to pinned host memory after each call; the next call sizes
  // its pool from it)
  uint32_t* hcmd = nullptr;
  uint64_t hcmd_words = 0;
  uint32_t* hncmd = nullptr;
  uint64_t hncmd_cap = 0;
  uint32_t* hctr = nullptr;
  unsigned long long* hneed = nullptr;
  unsigned long long* hneed_host = nullptr;
  // RLE v2 walk pass: kMaxSeg segment-start entries per chunk
  uint2* seg = nullptr;
  uint64_t seg_cap = 0;  // chunks
};

std::mutex g_mu;
Workspace g_ws[kMaxDevices];

codag_status current_ws(Workspace** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(CODAG_EINVAL, "device index out of range");
  Workspace& w = g_ws[dev];
  if (!w.attrs_set) {
    struct {
      const void* fn;
      int bytes;
    } attrs[] = {{(const void*)rle_v1_kernel, -1},
                 {(const void*)rle_v1_sizes_kernel, -1},
                 {(const void*)rle_v2_kernel, -1},
                 {(const void*)rle_v2_sizes_kernel, -1},
                 {(const void*)byte_rle_cta_kernel, -1},
                 {(const void*)inflate_kernel, kWarpsPerBlock * kDeflateWarp},
                 {(const void*)inflate_sizes_kernel, kWarpsPerBlock * kDeflateWarp},
                 {(const void*)orc_zlib_kernel, kWarpsPerBlock * kDeflateWarp},
                 {(const void*)orc_zlib_sizes_kernel, kWarpsPerBlock * kDeflateWarp},
                 {(const void*)byte_rle_kernel, kWarpsPerBlock * warp_chunk_smem(4, RleRing::SMEM)},
                 {(const void*)byte_rle_sizes_kernel, kWarpsPerBlock * warp_chunk_smem(4, RleRing::SMEM)},
                 {(const void*)inflate_reg_kernel, kWarpsPerBlock * warp_chunk_smem(3, 0)},
                 {(const void*)inflate_huffman_kernel, kHufSmem},
                 {(const void*)inflate_huffman_sizes_kernel, kHufSmem}};
    e = cudaDeviceGetAttribute(&w.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&w.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&w.smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&w.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    for (auto& at : attrs) {
      // -1: a CTA-per-chunk RLE kernel, whose stage is sized at launch
      // (rle_stage_bytes), up to the largest dynamic shared memory of a CTA
      const int bytes = at.bytes >= 0 ? at.bytes : w.smem_optin > kRleMaxSmem ? w.smem_optin : kRleMaxSmem;
      e = cudaFuncSetAttribute(at.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    }
    for (int i = 0; i < kBatchShapes; i++) {
      const BatchShape b = batch_shape(i);
      e = cudaFuncSetAttribute(b.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, b.smem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    }
    e = cudaMalloc(&w.counters, kBatchCounterWords * sizeof(uint32_t));
    if (e != cudaSuccess) return fail(CODAG_ENOMEM, "workspace allocation failed");
    w.attrs_set = true;
  }
  *out = &w;
  return CODAG_OK;
}

codag_status grow_status(Workspace& w, uint64_t n) {
  if (n <= w.status_cap) return CODAG_OK;
  if (w.status) cudaFree(w.status);
  w.status = nullptr;
  w.status_cap = 0;
  uint64_t cap = n < 1024 ? 1024 : n + n / 4;
  if (cudaMalloc(&w.status, cap * sizeof(int32_t)) != cudaSuccess)
    return fail(CODAG_ENOMEM, "status workspace allocation failed");
  w.status_cap = cap;
  return CODAG_OK;
}

codag_status grow_order(Workspace& w, uint64_t n) {
  if (n <= w.order_cap) return CODAG_OK;
  if (w.order) cudaFree(w.order);
  if (w.keys) cudaFree(w.keys);
  w.order = nullptr;
  w.keys = nullptr;
  w.order_cap = 0;
  uint64_t cap = n < 1024 ? 1024 : n + n / 4;
  if (cudaMalloc(&w.order, cap * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&w.keys, cap * sizeof(unsigned long long)) != cudaSuccess)
    return fail(CODAG_ENOMEM, "order workspace allocation failed");
  w.order_cap = cap;
  return CODAG_OK;
}

// The walk pass's segment table for n chunks, or nullptr when the call walks
// inside its decode CTAs (not RLE v2, the walk pass switched off, too many
// chunks, or no memory for the table).
uint2* walk_table(Workspace& w, int fam, uint64_t n, bool store) {
  if (fam != 2 || !store || g_walk_pass.load() != 1 || n > kMaxWalkChunks) return nullptr;
  if (n > w.seg_cap) {
    if (w.seg) cudaFree(w.seg);
    w.seg = nullptr;
    w.seg_cap = 0;
    const uint64_t cap = n < 1024 ? 1024 : (n + n / 4 < kMaxWalkChunks ? n + n / 4 : kMaxWalkChunks);
    if (cudaMalloc(&w.seg, cap * kMaxSeg * sizeof(uint2)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    w.seg_cap = cap;
  }
  return w.seg;
}

bool is_rle(int f) {
  return f == CODAG_ORC_RLE_V1_I64 || f == CODAG_ORC_RLE_V1_U64 || f == CODAG_ORC_RLE_V2_I64 ||
         f == CODAG_ORC_RLE_V2_U64;
}
int family_of(int f) {
  if (f == CODAG_ORC_RLE_V1_I64 || f == CODAG_ORC_RLE_V1_U64) return 1;
  if (f == CODAG_ORC_RLE_V2_I64 || f == CODAG_ORC_RLE_V2_U64) return 2;
  if (f == CODAG_DEFLATE_RAW) return 3;
  if (f == CODAG_ORC_BYTE_RLE || f == CODAG_ORC_BOOL_RLE) return 4;
  if (f == CODAG_ORC_ZLIB) return 5;
  return 0;
}

codag_status check_common(const void* comp, const uint64_t* comp_offsets, uint64_t n) {
  if (!comp || !comp_offsets) return fail(CODAG_EINVAL, "NULL comp or comp_offsets");
  if (reinterpret_cast<uintptr_t>(comp) & 15) return fail(CODAG_EINVAL, "comp must be 16-byte aligned");
  if (n > (1ull << 32) - 1) return fail(CODAG_EINVAL, "too many chunks (max 2^32 - 1)");
  return CODAG_OK;
}

// One launch's share of the two-pass Deflate scratch.
struct DeflateRun {
  uint32_t* cmd = nullptr;  // the launch's part of the command pool
  uint64_t pool_words = 0;  // its size
  uint32_t* ncmd = nullptr; // the launch's first chunk's count
  uint32_t* counter = nullptr;
  unsigned long long* need = nullptr;
};

// Size the two-pass Deflate scratch for a call of n chunks (store: with the
// command pool).  The pool grows to what an earlier call needed (plus a
// quarter); a chunk whose region lies past it is decoded by the one-warp
// decoder instead, so the pool size is a speed setting only.
codag_status deflate_prepare(Workspace& w, uint64_t n, bool store, uint64_t known_words = 0) {
  if (!w.hctr) {
    if (cudaMalloc(&w.hctr, (kMaxSlices + 1) * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&w.hneed, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(w.hneed, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaHostAlloc(&w.hneed_host, sizeof(unsigned long long), cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return fail(CODAG_ENOMEM, "Deflate workspace allocation failed");
    }
    *w.hneed_host = 0;
  }
  if (!store) return CODAG_OK;
  const unsigned long long need =
      known_words ? known_words : *reinterpret_cast<volatile unsigned long long*>(w.hneed_host);
  uint64_t words = need > kHufPoolInitWords ? need : kHufPoolInitWords;
  const uint64_t limit = g_pool_limit.load() / sizeof(uint32_t);
  if (limit && words > limit) words = limit;
  if (words > w.hcmd_words) {
    if (w.hcmd) cudaFree(w.hcmd);
    w.hcmd = nullptr;
    w.hcmd_words = 0;
    const uint64_t alloc = words + words / 4;
    if (cudaMalloc(&w.hcmd, alloc * sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      return fail(CODAG_ENOMEM, "Deflate command pool allocation failed");
    }
    w.hcmd_words = alloc;
  }
  if (n > w.hncmd_cap) {
    if (w.hncmd) cudaFree(w.hncmd);
    w.hncmd = nullptr;
    w.hncmd_cap = 0;
    const uint64_t alloc = n < 1024 ? 1024 : n + n / 4;
    if (cudaMalloc(&w.hncmd, alloc * sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      return fail(CODAG_ENOMEM, "Deflate count allocation failed");
    }
    w.hncmd_cap = alloc;
  }
  return CODAG_OK;
}

// The scratch of chunks [first, first + n) of a prepared call, claimed
// through counter `slot` (0 .. kMaxSlices); region: the pool word where
// chunk `first`'s region starts (its output offset from the call's first
// chunk / 4 + 2 first), so that slices decoded at the same time never share
// pool words.
DeflateRun deflate_run(const Workspace& w, uint64_t region, uint64_t first, int slot) {
  DeflateRun r;
  uint64_t words = w.hcmd_words;
  const uint64_t limit = g_pool_limit.load() / sizeof(uint32_t);
  if (limit && words > limit) words = limit;
  r.cmd = w.hcmd ? w.hcmd + (region < words ? region : words) : nullptr;
  r.pool_words = w.hcmd && region < words ? words - region : 0;
  r.ncmd = w.hncmd ? w.hncmd + first : nullptr;
  r.counter = w.hctr + slot;
  r.need = w.hneed;
  return r;
}

codag_status launch_kernel(const Workspace& ws, int format, const void* comp,
                           const uint64_t* comp_offsets, uint64_t n, void* out,
                           const uint64_t* out_offsets, uint64_t* sizes, bool store,
                           int32_t* status, cudaStream_t stream, const DeflateRun* dr = nullptr,
                           uint2* seg = nullptr);

codag_status launch_plain(int format, const void* comp, const uint64_t* comp_offsets, uint64_t n,
                          void* out, const uint64_t* out_offsets, uint64_t* sizes, bool store,
                          cudaStream_t stream) {
  const int fam = family_of(format);
  if (!fam) return fail(CODAG_EINVAL, "unknown format");
  if (n == 0) return CODAG_OK;
  codag_status s = check_common(comp, comp_offsets, n);
  if (s != CODAG_OK) return s;
  if (store) {
    if (!out || !out_offsets) return fail(CODAG_EINVAL, "NULL out or out_offsets");
    if (is_rle(format) && (reinterpret_cast<uintptr_t>(out) & 7))
      return fail(CODAG_EINVAL, "RLE out must be 8-byte aligned");
  } else if (!sizes) {
    return fail(CODAG_EINVAL, "NULL sizes_out");
  }
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace* w;
  if ((s = current_ws(&w)) != CODAG_OK) return s;
  if ((s = grow_status(*w, n)) != CODAG_OK) return s;
  w->last_n = n;
  if (fam == 3) {
    if ((s = deflate_prepare(*w, n, store)) != CODAG_OK) return s;
    const DeflateRun dr = deflate_run(*w, 0, 0, kMaxSlices);
    s = launch_kernel(*w, format, comp, comp_offsets, n, out, out_offsets, sizes, store, w->status,
                      stream, &dr);
    if (s == CODAG_OK && store) {
      const cudaError_t e = cudaMemcpyAsync(w->hneed_host, w->hneed, sizeof(unsigned long long),
                                            cudaMemcpyDeviceToHost, stream);
      if (e != cudaSuccess) return cuda_fail(e, "Deflate need copy");
    }
    return s;
  }
  return launch_kernel(*w, format, comp, comp_offsets, n, out, out_offsets, sizes, store, w->status,
                       stream, nullptr, walk_table(*w, fam, n, store));
}

// Whole-chunk stage of a CTA-per-chunk RLE launch (family fam, `parts`
// warps): at least kRleStageBytes (and room for the per-warp rings of the
// fallback path), widened to all the shared memory that the CTAs per SM
// allowed by threads and registers leave free, so that more chunks are
// staged whole without costing occupancy.
int rle_stage_bytes(const Workspace& w, const void* fn, int fam, int parts, bool store) {
  int stage = kRleStageBytes;
  if (stage < parts * RleRing::SMEM) stage = parts * RleRing::SMEM;
  // cached per kernel, family and warps: the dynamic shared memory a CTA may have
  // while as many CTAs fit per SM as threads and registers allow.  A CTA's
  // share is its dynamic shared memory plus the memory the system reserves
  // for it, allocated in 128-byte units (measured on GB300 with ncu: one
  // byte over takes a CTA per SM away).
  int& avail = w.rle_avail[store ? 1 : 0][fam][parts];
  if (avail == 0) {
    int ctas = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, fn, 32 * parts, 0) != cudaSuccess || ctas <= 0 ||
        w.smem_per_sm <= 0) {
      cudaGetLastError();
      avail = -1;
    } else {
      const int share = (w.smem_per_sm / ctas) & ~127;
      avail = share - w.smem_reserved;
      if (avail > w.smem_optin) avail = w.smem_optin;
    }
  }
  if (avail <= 0) return stage;
  const int other = parts * kRleScratch + kRleCtaExtra;
  const int budget = avail - other;
  // RLE v1 adds a terminator bitmap of about a quarter of the stage (+384 B)
  int wide = fam == 1 ? (budget - 384) / 5 * 4 : budget;
  wide &= ~255;
  while (fam == 1 && wide > 0 && wide + rle_v1_bitmap_bytes(wide) > budget) wide -= 256;
  return wide > stage ? wide : stage;
}

// One plain decode (or sizes) launch over chunks [0, n) of the given arrays,
// statuses to `status`.  Arguments are checked and g_mu is held by the caller.
codag_status launch_kernel(const Workspace& ws, int format, const void* comp,
                           const uint64_t* comp_offsets, uint64_t n, void* out,
                           const uint64_t* out_offsets, uint64_t* sizes, bool store,
                           int32_t* status, cudaStream_t stream, const DeflateRun* dr,
                           uint2* seg) {
  const Workspace* w = &ws;
  const int fam = family_of(format);
  Args a{};
  a.comp = static_cast<const uint8_t*>(comp);
  a.comp_off = comp_offsets;
  a.n = n;
  a.out = static_cast<uint8_t*>(out);
  a.out_off = out_offsets;
  a.sizes = sizes;
  a.status = status;
  a.format = format;
  const void* fn;
  unsigned grid, block;
  size_t smem;
  // decode kernels of Deflate and byte / boolean RLE may stage their input
  // in registers instead of a shared-memory ring (codag_set_input_staging);
  // byte / boolean RLE then runs a warp per chunk, else a CTA per chunk
  const bool reg = store && (fam == 3 || fam == 4) && g_reg_ring[fam].load() == 1;
  if (fam == 3 && !reg && dr) {
    // two passes: Huffman decoding a lane per chunk, then the copies a warp
    // per chunk, then the one-warp decoder for chunks left to it
    HufArgs h{dr->cmd, dr->pool_words, dr->ncmd, dr->counter, dr->need};
    cudaError_t e = cudaMemsetAsync(dr->counter, 0, sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    // one CTA per SM (fewer for fewer chunks than SMs): the lanes' first
    // chunks are spread over every warp
    const unsigned g1 = (unsigned)(n < (uint64_t)w->sm_count ? n : (uint64_t)w->sm_count);
    if (!store) {
      // then the one-warp sizes kernel for the chunks the lanes left to it
      inflate_huffman_sizes_kernel<<<g1, 32 * kHufWarps, kHufSmem, stream>>>(a, h);
      Args b = a;
      b.deferred_only = 1;
      inflate_sizes_kernel<<<(unsigned)((n + kWarpsPerBlock - 1) / kWarpsPerBlock), kThreads,
                             kWarpsPerBlock * kDeflateWarp, stream>>>(b);
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "decode launch");
      g_launches.fetch_add(2);
      return CODAG_OK;
    }
    inflate_huffman_kernel<<<g1, 32 * kHufWarps, kHufSmem, stream>>>(a, h);
    inflate_lz77_kernel<<<(unsigned)((n + kLz77Warps - 1) / kLz77Warps), 32 * kLz77Warps, 0, stream>>>(a, h);
    Args b = a;
    b.deferred_only = 1;
    inflate_kernel<<<(unsigned)((n + kWarpsPerBlock - 1) / kWarpsPerBlock), kThreads,
                     kWarpsPerBlock * kDeflateWarp, stream>>>(b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    g_launches.fetch_add(3);
    return CODAG_OK;
  }
  if (fam == 3 || fam == 5 || (fam == 4 && (!store || reg))) {
    grid = (unsigned)((n + kWarpsPerBlock - 1) / kWarpsPerBlock);
    block = kThreads;
    const int ring_smem = reg ? 0 : fam == 4 ? RleRing::SMEM : DeflateRing::SMEM;
    smem = (size_t)kWarpsPerBlock * warp_chunk_smem(fam == 5 ? 3 : fam, ring_smem);
    if (fam == 3)
      fn = !store ? (const void*)inflate_sizes_kernel : reg ? (const void*)inflate_reg_kernel : (const void*)inflate_kernel;
    else if (fam == 4)
      fn = !store ? (const void*)byte_rle_sizes_kernel : reg ? (const void*)byte_rle_reg_kernel : (const void*)byte_rle_kernel;
    else
      fn = store ? (const void*)orc_zlib_kernel : (const void*)orc_zlib_sizes_kernel;
  } else {
    // parts per chunk: enough warps to fill the GPU, at most 16 per chunk
    int parts = g_parts_per_chunk.load();
    if (!store) parts = 1;
    if (parts <= 0) {
      parts = 1;
      while (parts < 16 && (uint64_t)parts * n < (uint64_t)w->sm_count * 32) parts *= 2;
    }
    grid = (unsigned)n;
    block = 32u * (unsigned)parts;
    if (fam == 1) fn = store ? (const void*)rle_v1_kernel : (const void*)rle_v1_sizes_kernel;
    else if (fam == 4) fn = (const void*)byte_rle_cta_kernel;
    else fn = store ? (const void*)rle_v2_kernel : (const void*)rle_v2_sizes_kernel;
    const int stage = rle_stage_bytes(*w, fn, fam, parts, store);
    a.stage_bytes = stage;
    smem = (size_t)stage + (size_t)parts * kRleScratch + kRleCtaExtra;
    if (fam == 1) smem += (size_t)rle_v1_bitmap_bytes(stage);
    if (fam == 2 && store && seg && parts > 1) {
      // walk pass: every chunk's segment starts, before the decode pass
      a.seg = seg;
      a.parts = parts;
      rle_v2_walk_kernel<<<(unsigned)((n + kWarpsPerBlock - 1) / kWarpsPerBlock), kThreads,
                           kWarpsPerBlock * RleRing::SMEM, stream>>>(a);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "walk launch");
      g_launches.fetch_add(1);
    }
  }
  void* params[] = {&a};
  cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(block), params, smem, stream);
  if (e != cudaSuccess) return cuda_fail(e, "decode launch");
  g_launches.fetch_add(1);
  return CODAG_OK;
}

codag_status init_pipe(HostPipe& p) {
  if (p.h2d) return CODAG_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&p.h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p.d2h, cudaStreamNonBlocking);
  for (int i = 0; i < kPipeDecode && e == cudaSuccess; i++)
    e = cudaStreamCreateWithFlags(&p.dec[i], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming);
  for (int i = 0; i < kMaxSlices && e == cudaSuccess; i++) {
    e = cudaEventCreateWithFlags(&p.copied[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.decoded[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    p.h2d = nullptr;  // retried on the next call; the objects made so far are kept alive
    return cuda_fail(e, "copy stream / event creation");
  }
  return CODAG_OK;
}

codag_status grow_offs(HostPipe& p, uint64_t words) {
  if (words <= p.offs_cap) return CODAG_OK;
  if (p.offs) cudaFree(p.offs);
  p.offs = nullptr;
  p.offs_cap = 0;
  const uint64_t cap = words < 2048 ? 2048 : words + words / 4;
  if (cudaMalloc(&p.offs, cap * sizeof(uint64_t)) != cudaSuccess)
    return fail(CODAG_ENOMEM, "offsets workspace allocation failed");
  p.offs_cap = cap;
  return CODAG_OK;
}

// Slice boundaries (chunk indices, first 0, last n): about kSliceBytes of
// output each, but at least min_chunks chunks (enough decoders for
// kPipeDecode concurrent slices to fill the GPU), at most kMaxSlices, no
// empty slice.
std::vector<uint64_t> plan_slices(const uint64_t* out_offsets, uint64_t n, uint64_t min_chunks) {
  const uint64_t o0 = out_offsets[0], total = out_offsets[n] - o0;
  uint64_t S = (total + kSliceBytes - 1) / kSliceBytes;
  if (min_chunks && S > n / min_chunks) S = n / min_chunks;
  if (S > (uint64_t)kMaxSlices) S = kMaxSlices;
  if (S > n) S = n;
  if (S < 1) S = 1;
  std::vector<uint64_t> b{0};
  for (uint64_t s = 1; s < S; s++) {
    const uint64_t target = o0 + (total / S) * s;
    uint64_t lo = b.back() + 1, hi = n;  // first c in [lo, n) with out_offsets[c] >= target
    while (lo < hi) {
      const uint64_t mid = lo + (hi - lo) / 2;
      if (out_offsets[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    if (lo < n) b.push_back(lo);
  }
  b.push_back(n);
  return b;
}

// Enqueue the batch path with the given scratch (status, order, keys, counters).
codag_status enqueue_batch(const Workspace& w, const uint8_t* formats, const void* comp,
                           const uint64_t* comp_offsets, uint64_t n, void* out,
                           const uint64_t* out_offsets, int32_t* status, uint32_t* order,
                           unsigned long long* keys, uint32_t* counters, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(counters, 0, kBatchCounterWords * sizeof(uint32_t), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0xff, n * sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  const unsigned og = (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  order_hist_kernel<<<og, 256, 0, stream>>>(formats, comp_offsets, out_offsets, n, counters + 1);
  order_scatter_kernel<<<og, 256, 0, stream>>>(formats, comp_offsets, out_offsets, n,
                                               counters + 1, counters + 1 + kBuckets, order);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "order launch");
  Args a{};
  a.comp = static_cast<const uint8_t*>(comp);
  a.comp_off = comp_offsets;
  a.n = n;
  a.out = static_cast<uint8_t*>(out);
  a.out_off = out_offsets;
  a.status = status;
  a.formats = formats;
  a.order = order;
  a.counter = counters;
  a.keys = keys;
  a.split_lg = g_split_lg.load();
  a.split_max = g_split_max.load();
  const BatchShape b = batch_shape(g_batch_shape.load());
  int fit = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, b.fn, kThreads, b.smem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  int per_sm = g_batch_ctas_per_sm.load();
  if (per_sm <= 0 || per_sm > fit) per_sm = fit;
  if (per_sm < 1) per_sm = 1;
  const uint64_t grid = (uint64_t)per_sm * (uint64_t)w.sm_count;
  void* params[] = {&a};
  e = cudaLaunchKernel(b.fn, dim3((unsigned)grid), dim3(kThreads), params, (size_t)b.smem, stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  batch_finalize_kernel<<<og, 256, 0, stream>>>(formats, comp_offsets, out_offsets, n, keys, status,
                                                a.split_lg, a.split_max);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  g_launches.fetch_add(4);
  return CODAG_OK;
}

codag_status check_batch(const uint8_t* formats, const void* comp, const uint64_t* comp_offsets,
                         uint64_t n, void* out, const uint64_t* out_offsets) {
  codag_status s = check_common(comp, comp_offsets, n);
  if (s != CODAG_OK) return s;
  if (!formats || !out || !out_offsets) return fail(CODAG_EINVAL, "NULL formats, out or out_offsets");
  if (reinterpret_cast<uintptr_t>(out) & 7) return fail(CODAG_EINVAL, "out must be 8-byte aligned");
  return CODAG_OK;
}

}  // namespace

namespace codag {
// For entry points defined in other translation units.
void note_launches(uint64_t n) { g_launches.fetch_add(n); }
void note_error(const std::string& msg) { g_last_error = msg; }
int batch_shape_selected() { return g_batch_shape.load(); }
}  // namespace codag

struct codag_graph_s {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  uint32_t* order = nullptr;
  unsigned long long* keys = nullptr;
  uint32_t* counters = nullptr;
};

extern "C" {

codag_status codag_decompress(int format, const void* comp, const uint64_t* comp_offsets,
                              uint64_t n_chunks, void* out, const uint64_t* out_offsets,
                              cudaStream_t stream) {
  return launch_plain(format, comp, comp_offsets, n_chunks, out, out_offsets, nullptr, true, stream);
}

codag_status codag_decompressed_sizes(int format, const void* comp, const uint64_t* comp_offsets,
                                      uint64_t n_chunks, uint64_t* sizes_out, cudaStream_t stream) {
  return launch_plain(format, comp, comp_offsets, n_chunks, nullptr, nullptr, sizes_out, false,
                      stream);
}

codag_status codag_decompress_host(int format, const void* h_comp, const uint64_t* h_comp_offsets,
                                   uint64_t n, void* h_out, const uint64_t* h_out_offsets,
                                   void* d_comp, void* d_out, int32_t* h_status,
                                   cudaStream_t stream) {
  if (!family_of(format)) return fail(CODAG_EINVAL, "unknown format");
  if (n == 0) return CODAG_OK;
  if (!h_comp || !h_comp_offsets || !h_out || !h_out_offsets || !d_comp || !d_out)
    return fail(CODAG_EINVAL, "codag_decompress_host: NULL pointer");
  codag_status s = check_common(d_comp, h_comp_offsets, n);
  if (s != CODAG_OK) return s;
  if (is_rle(format) && (reinterpret_cast<uintptr_t>(d_out) & 7))
    return fail(CODAG_EINVAL, "RLE out must be 8-byte aligned");
  for (uint64_t c = 0; c < n; c++)
    if (h_comp_offsets[c + 1] < h_comp_offsets[c] || h_out_offsets[c + 1] < h_out_offsets[c])
      return fail(CODAG_EINVAL, "codag_decompress_host: offsets must be non-decreasing");
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace* w;
  if ((s = current_ws(&w)) != CODAG_OK) return s;
  if ((s = grow_status(*w, n)) != CODAG_OK) return s;
  HostPipe& p = w->pipe;
  if ((s = init_pipe(p)) != CODAG_OK) return s;
  if ((s = grow_offs(p, 2 * (n + 1))) != CODAG_OK) return s;
  // the pool this call needs is known here from the host offsets
  if (family_of(format) == 3 &&
      (s = deflate_prepare(*w, n, true, (h_out_offsets[n] - h_out_offsets[0]) / 4 + 2 * n + 2)) != CODAG_OK)
    return s;
  w->last_n = n;
  // decoders resident per SM: a Deflate chunk is one lane of the Huffman
  // pass (32 * kHufWarps per SM), a byte RLE or ORC zlib chunk one warp
  // (about 40), an RLE chunk a CTA (a few); kPipeDecode slices in flight
  // should fill them
  const int fam = family_of(format);
  const uint64_t per_sm = fam == 3 ? 32 * kHufWarps : fam >= 4 ? 40 : 8;
  const uint64_t min_chunks = (uint64_t)w->sm_count * per_sm / kPipeDecode;
  const std::vector<uint64_t> bounds = plan_slices(h_out_offsets, n, min_chunks);
  uint2* seg = walk_table(*w, fam, n, true);
  uint64_t* d_coff = p.offs;
  uint64_t* d_ooff = p.offs + (n + 1);
  const uint8_t* hc = static_cast<const uint8_t*>(h_comp);
  uint8_t* dc = static_cast<uint8_t*>(d_comp);
  uint8_t* ho = static_cast<uint8_t*>(h_out);
  uint8_t* dd = static_cast<uint8_t*>(d_out);

  // order: earlier work on `stream` and an earlier host call (which shares
  // the offsets copy and the statuses) before the first copy
  cudaError_t e = cudaEventRecord(p.start, stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p.h2d, p.start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p.d2h, p.start, 0);
  if (e == cudaSuccess && p.used) e = cudaStreamWaitEvent(p.h2d, p.done, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_coff, h_comp_offsets, (n + 1) * 8, cudaMemcpyHostToDevice, p.h2d);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_ooff, h_out_offsets, (n + 1) * 8, cudaMemcpyHostToDevice, p.h2d);
  if (e != cudaSuccess) return cuda_fail(e, "codag_decompress_host setup");
  // A slice's kernels read its chunks' bytes and, for the 16-byte alignment
  // of a staged copy, up to 15 bytes before the first chunk: those belong to
  // the previous slice, whose copy is earlier on the same stream.
  uint64_t copied_to = h_comp_offsets[0];
  for (size_t k = 0; k + 1 < bounds.size(); k++) {
    const uint64_t a = bounds[k], b = bounds[k + 1];
    const uint64_t hi = h_comp_offsets[b];
    if (hi > copied_to)
      e = cudaMemcpyAsync(dc + copied_to, hc + copied_to, hi - copied_to, cudaMemcpyHostToDevice, p.h2d);
    copied_to = hi > copied_to ? hi : copied_to;
    cudaStream_t ds = p.dec[k % kPipeDecode];
    if (e == cudaSuccess) e = cudaEventRecord(p.copied[k], p.h2d);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ds, p.copied[k], 0);
    if (e != cudaSuccess) return cuda_fail(e, "codag_decompress_host copy in");
    const DeflateRun dr = deflate_run(*w, (h_out_offsets[a] - h_out_offsets[0]) / 4 + 2 * a, a, (int)k);
    s = launch_kernel(*w, format, d_comp, d_coff + a, b - a, d_out, d_ooff + a, nullptr, true,
                      w->status + a, ds, family_of(format) == 3 ? &dr : nullptr,
                      seg ? seg + a * kMaxSeg : nullptr);
    if (s != CODAG_OK) return s;
    e = cudaEventRecord(p.decoded[k], ds);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p.d2h, p.decoded[k], 0);
    const uint64_t ob = h_out_offsets[a], oe = h_out_offsets[b];
    if (e == cudaSuccess && oe > ob)
      e = cudaMemcpyAsync(ho + ob, dd + ob, oe - ob, cudaMemcpyDeviceToHost, p.d2h);
    if (e != cudaSuccess) return cuda_fail(e, "codag_decompress_host copy out");
  }
  if (h_status) e = cudaMemcpyAsync(h_status, w->status, n * 4, cudaMemcpyDeviceToHost, p.d2h);
  if (e == cudaSuccess && family_of(format) == 3)
    e = cudaMemcpyAsync(w->hneed_host, w->hneed, sizeof(unsigned long long), cudaMemcpyDeviceToHost, p.d2h);
  if (e == cudaSuccess) e = cudaEventRecord(p.done, p.d2h);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, p.done, 0);
  if (e != cudaSuccess) return cuda_fail(e, "codag_decompress_host finish");
  p.used = true;
  return CODAG_OK;
}

codag_status codag_decompress_batch(const uint8_t* formats, const void* comp,
                                    const uint64_t* comp_offsets, uint64_t n_chunks, void* out,
                                    const uint64_t* out_offsets, int32_t* chunk_status,
                                    cudaStream_t stream) {
  if (n_chunks == 0) return CODAG_OK;
  codag_status s = check_batch(formats, comp, comp_offsets, n_chunks, out, out_offsets);
  if (s != CODAG_OK) return s;
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace* w;
  if ((s = current_ws(&w)) != CODAG_OK) return s;
  if ((s = grow_order(*w, n_chunks)) != CODAG_OK) return s;
  if (!chunk_status) {
    if ((s = grow_status(*w, n_chunks)) != CODAG_OK) return s;
    w->last_n = n_chunks;
    chunk_status = w->status;
  }
  return enqueue_batch(*w, formats, comp, comp_offsets, n_chunks, out, out_offsets, chunk_status,
                       w->order, w->keys, w->counters, stream);
}

uint64_t codag_batch_scratch_bytes(uint64_t n_chunks) {
  // keys (8 per chunk), counters (256-byte block), order (4 per chunk)
  return n_chunks * 8 + 256 * ((kBatchCounterWords * 4 + 255) / 256) + n_chunks * 4 + 256;
}

codag_status codag_decompress_batch_ws(const uint8_t* formats, const void* comp,
                                       const uint64_t* comp_offsets, uint64_t n_chunks, void* out,
                                       const uint64_t* out_offsets, int32_t* chunk_status,
                                       void* scratch, uint64_t scratch_bytes, cudaStream_t stream) {
  if (n_chunks == 0) return CODAG_OK;
  codag_status s = check_batch(formats, comp, comp_offsets, n_chunks, out, out_offsets);
  if (s != CODAG_OK) return s;
  if (!chunk_status || !scratch) return fail(CODAG_EINVAL, "NULL chunk_status or scratch");
  if (reinterpret_cast<uintptr_t>(scratch) & 255) return fail(CODAG_EINVAL, "scratch must be 256-byte aligned");
  if (scratch_bytes < codag_batch_scratch_bytes(n_chunks))
    return fail(CODAG_EINVAL, "scratch smaller than codag_batch_scratch_bytes(n_chunks)");
  uint8_t* base = static_cast<uint8_t*>(scratch);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(base);
  uint32_t* counters = reinterpret_cast<uint32_t*>(base + ((n_chunks * 8 + 255) & ~255ull));
  uint32_t* order = counters + 64 * ((kBatchCounterWords + 63) / 64);
  Workspace* w;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if ((s = current_ws(&w)) != CODAG_OK) return s;
  }
  return enqueue_batch(*w, formats, comp, comp_offsets, n_chunks, out, out_offsets, chunk_status,
                       order, keys, counters, stream);
}

codag_status codag_last_chunk_status(int32_t* host_status, uint64_t n, cudaStream_t stream) {
  if (n == 0) return CODAG_OK;
  if (!host_status) return fail(CODAG_EINVAL, "NULL host_status");
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace* w;
  codag_status s;
  if ((s = current_ws(&w)) != CODAG_OK) return s;
  if (n > w->last_n || !w->status) return fail(CODAG_EINVAL, "n exceeds the last call's chunk count");
  cudaError_t e = cudaMemcpyAsync(host_status, w->status, n * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, stream);
  if (e != cudaSuccess) return cuda_fail(e, "status copy");
  e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  for (uint64_t i = 0; i < n; i++)
    if (host_status[i] != CODAG_CHUNK_OK) return CODAG_ECORRUPT;
  return CODAG_OK;
}

codag_status codag_batch_graph_create(const uint8_t* formats, const void* comp,
                                      const uint64_t* comp_offsets, uint64_t n_chunks, void* out,
                                      const uint64_t* out_offsets, int32_t* chunk_status,
                                      cudaStream_t stream, codag_graph* graph_out) {
  if (!graph_out) return fail(CODAG_EINVAL, "NULL graph_out");
  *graph_out = nullptr;
  if (n_chunks == 0 || !chunk_status) return fail(CODAG_EINVAL, "n_chunks == 0 or NULL chunk_status");
  codag_status s = check_batch(formats, comp, comp_offsets, n_chunks, out, out_offsets);
  if (s != CODAG_OK) return s;
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace* w;
  if ((s = current_ws(&w)) != CODAG_OK) return s;
  codag_graph g = new codag_graph_s();
  if (cudaMalloc(&g->order, n_chunks * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&g->keys, n_chunks * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&g->counters, kBatchCounterWords * sizeof(uint32_t)) != cudaSuccess) {
    if (g->order) cudaFree(g->order);
    if (g->keys) cudaFree(g->keys);
    delete g;
    return fail(CODAG_ENOMEM, "graph scratch allocation failed");
  }
  cudaStream_t cap;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(g->order);
    cudaFree(g->keys);
    cudaFree(g->counters);
    delete g;
    return cuda_fail(e, "capture stream");
  }
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const uint64_t before = g_launches.load();
    s = enqueue_batch(*w, formats, comp, comp_offsets, n_chunks, out, out_offsets, chunk_status,
                      g->order, g->keys, g->counters, cap);
    g_launches.store(before);  // captured, not launched
    cudaError_t e2 = cudaStreamEndCapture(cap, &g->graph);
    if (s == CODAG_OK && e2 != cudaSuccess) s = cuda_fail(e2, "end capture");
    if (s == CODAG_OK) {
      e2 = cudaGraphInstantiate(&g->exec, g->graph, 0);
      if (e2 != cudaSuccess) s = cuda_fail(e2, "graph instantiate");
    }
  } else {
    s = cuda_fail(e, "begin capture");
  }
  cudaStreamDestroy(cap);
  (void)stream;
  if (s != CODAG_OK) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    cudaFree(g->order);
    cudaFree(g->keys);
    cudaFree(g->counters);
    delete g;
    return s;
  }
  *graph_out = g;
  return CODAG_OK;
}

codag_status codag_batch_graph_launch(codag_graph graph, cudaStream_t stream) {
  if (!graph || !graph->exec) return fail(CODAG_EINVAL, "NULL graph");
  cudaError_t e = cudaGraphLaunch(graph->exec, stream);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  g_launches.fetch_add(4);
  return CODAG_OK;
}

codag_status codag_batch_graph_destroy(codag_graph graph) {
  if (!graph) return CODAG_OK;
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  if (graph->graph) cudaGraphDestroy(graph->graph);
  if (graph->order) cudaFree(graph->order);
  if (graph->keys) cudaFree(graph->keys);
  if (graph->counters) cudaFree(graph->counters);
  delete graph;
  return CODAG_OK;
}

codag_status codag_set_batch_ctas_per_sm(int ctas_per_sm) {
  if (ctas_per_sm < 0 || ctas_per_sm > 64) return fail(CODAG_EINVAL, "ctas_per_sm out of range");
  g_batch_ctas_per_sm.store(ctas_per_sm);
  return CODAG_OK;
}

int codag_get_batch_ctas_per_sm(void) { return g_batch_ctas_per_sm.load(); }

int codag_batch_staging_shapes(int* slot_bytes, int* slots, int cap) {
  for (int i = 0; i < kBatchShapes && i < cap; i++) {
    const BatchShape b = batch_shape(i);
    if (slot_bytes) slot_bytes[i] = b.slot;
    if (slots) slots[i] = b.slots;
  }
  return kBatchShapes;
}

codag_status codag_set_batch_staging(int slot_bytes, int slots) {
  if (slot_bytes == 0 && slots == 0) {
    g_batch_shape.store(kBatchShapeDefault);
    return CODAG_OK;
  }
  for (int i = 0; i < kBatchShapes; i++) {
    const BatchShape b = batch_shape(i);
    if (b.slot == slot_bytes && b.slots == slots) {
      g_batch_shape.store(i);
      return CODAG_OK;
    }
  }
  return fail(CODAG_EINVAL, "codag_set_batch_staging: no batch kernel is compiled for a ring of " +
                                std::to_string(slot_bytes) + " x " + std::to_string(slots) + " bytes");
}

codag_status codag_get_batch_staging(int* slot_bytes, int* slots) {
  if (!slot_bytes || !slots) return fail(CODAG_EINVAL, "codag_get_batch_staging: NULL argument");
  const BatchShape b = batch_shape(g_batch_shape.load());
  *slot_bytes = b.slot;
  *slots = b.slots;
  return CODAG_OK;
}

codag_status codag_set_walk_pass(int format, int mode) {
  if (family_of(format) != 2) return fail(CODAG_EINVAL, "codag_set_walk_pass: RLE v2 formats only");
  if (mode != 0 && mode != 1) return fail(CODAG_EINVAL, "codag_set_walk_pass: mode must be 0 or 1");
  g_walk_pass.store(mode);
  return CODAG_OK;
}

int codag_get_walk_pass(int format) { return family_of(format) == 2 ? g_walk_pass.load() : -1; }

codag_status codag_set_batch_split(int split_log2, int max_parts) {
  if (split_log2 == 0 && max_parts == 0) {
    g_split_lg.store(kSplitLgDefault);
    g_split_max.store(kSplitMaxDefault);
    return CODAG_OK;
  }
  if (split_log2 < 8 || split_log2 > 40)
    return fail(CODAG_EINVAL, "codag_set_batch_split: split_log2 must be in [8, 40]");
  if (max_parts < 1 || max_parts > (int)kSplitMaxLimit)
    return fail(CODAG_EINVAL, "codag_set_batch_split: max_parts must be in [1, 32]");
  g_split_lg.store((uint32_t)split_log2);
  g_split_max.store((uint32_t)max_parts);
  return CODAG_OK;
}

codag_status codag_get_batch_split(int* split_log2, int* max_parts) {
  if (!split_log2 || !max_parts) return fail(CODAG_EINVAL, "codag_get_batch_split: NULL argument");
  *split_log2 = (int)g_split_lg.load();
  *max_parts = (int)g_split_max.load();
  return CODAG_OK;
}

codag_status codag_set_parts_per_chunk(int parts) {
  if (parts < 0 || parts > 16) return fail(CODAG_EINVAL, "parts per chunk must be 0..16");
  g_parts_per_chunk.store(parts);
  return CODAG_OK;
}

int codag_get_parts_per_chunk(void) { return g_parts_per_chunk.load(); }

codag_status codag_set_input_staging(int format, int mode) {
  const int fam = family_of(format);
  if (fam != 3 && fam != 4) return fail(CODAG_EINVAL, "input staging applies to Deflate and byte / boolean RLE");
  if (mode != 0 && mode != 1) return fail(CODAG_EINVAL, "input staging mode: 0 (shared ring) or 1 (registers)");
  g_reg_ring[fam].store(mode);
  return CODAG_OK;
}

int codag_get_input_staging(int format) {
  const int fam = family_of(format);
  return (fam == 3 || fam == 4) ? g_reg_ring[fam].load() : -1;
}

codag_status codag_set_wait_limit_ns(uint64_t ns) {
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace* w;
  codag_status s = current_ws(&w);  // the kernels' modules are loaded
  if (s != CODAG_OK) return s;
  cudaError_t e = set_wait_limit_rle(ns);
  if (e == cudaSuccess) e = set_wait_limit_inflate(ns);
  if (e == cudaSuccess) e = set_wait_limit_batch(ns);
  if (e == cudaSuccess) e = set_wait_limit_batch_small(ns);
  if (e == cudaSuccess) e = set_wait_limit_batch_large(ns);
  if (e != cudaSuccess) return cuda_fail(e, "wait limit");
  g_wait_limit.store(ns);
  return CODAG_OK;
}

uint64_t codag_get_wait_limit_ns(void) { return g_wait_limit.load(); }

codag_status codag_set_deflate_pool_limit(uint64_t bytes) {
  g_pool_limit.store(bytes);
  return CODAG_OK;
}

uint64_t codag_get_deflate_pool_limit(void) { return g_pool_limit.load(); }

uint64_t codag_kernel_launches(void) { return g_launches.load(); }

const char* codag_last_error(void) { return g_last_error.c_str(); }

const char* codag_version(void) { return "codag-gb300 0.1"; }

}  // extern "C"
