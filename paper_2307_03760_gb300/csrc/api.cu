// Host side of the C ABI (include/codag.h): argument checks, the per-device
// workspace, kernel launches and the batch graph.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/codag.h"
#include "kernels.cuh"

using namespace codag;

namespace {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_batch_ctas_per_sm{0};
std::atomic<int> g_parts_per_chunk{0};

codag_status fail(codag_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

codag_status cuda_fail(cudaError_t e, const char* what) {
  return fail(CODAG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr int kMaxDevices = 64;

struct Workspace {
  int32_t* status = nullptr;     // per-chunk status of the last plain call
  uint64_t status_cap = 0;
  uint64_t last_n = 0;
  uint32_t* order = nullptr;     // batch claim order
  unsigned long long* keys = nullptr;  // batch combined status of multi-part chunks
  uint64_t order_cap = 0;
  uint32_t* counters = nullptr;  // kBatchCounterWords words
  bool attrs_set = false;
  int sm_count = 0;
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
    } attrs[] = {{(const void*)rle_v1_kernel, kRleMaxSmem},
                 {(const void*)rle_v1_sizes_kernel, kRleMaxSmem},
                 {(const void*)rle_v2_kernel, kRleMaxSmem},
                 {(const void*)rle_v2_sizes_kernel, kRleMaxSmem},
                 {(const void*)inflate_kernel, kWarpsPerBlock * kDeflateWarp},
                 {(const void*)inflate_sizes_kernel, kWarpsPerBlock * kDeflateWarp},
                 {(const void*)batch_kernel, kBatchSmem}};
    for (auto& at : attrs) {
      e = cudaFuncSetAttribute(at.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, at.bytes);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    }
    e = cudaDeviceGetAttribute(&w.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
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

bool is_rle(int f) {
  return f == CODAG_ORC_RLE_V1_I64 || f == CODAG_ORC_RLE_V1_U64 || f == CODAG_ORC_RLE_V2_I64 ||
         f == CODAG_ORC_RLE_V2_U64;
}
int family_of(int f) {
  if (f == CODAG_ORC_RLE_V1_I64 || f == CODAG_ORC_RLE_V1_U64) return 1;
  if (f == CODAG_ORC_RLE_V2_I64 || f == CODAG_ORC_RLE_V2_U64) return 2;
  if (f == CODAG_DEFLATE_RAW) return 3;
  return 0;
}

codag_status check_common(const void* comp, const uint64_t* comp_offsets, uint64_t n) {
  if (!comp || !comp_offsets) return fail(CODAG_EINVAL, "NULL comp or comp_offsets");
  if (reinterpret_cast<uintptr_t>(comp) & 15) return fail(CODAG_EINVAL, "comp must be 16-byte aligned");
  if (n > (1ull << 32) - 1) return fail(CODAG_EINVAL, "too many chunks (max 2^32 - 1)");
  return CODAG_OK;
}

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
  Args a{};
  a.comp = static_cast<const uint8_t*>(comp);
  a.comp_off = comp_offsets;
  a.n = n;
  a.out = static_cast<uint8_t*>(out);
  a.out_off = out_offsets;
  a.sizes = sizes;
  a.status = w->status;
  a.format = format;
  const void* fn;
  unsigned grid, block;
  size_t smem;
  if (fam == 3) {
    grid = (unsigned)((n + kWarpsPerBlock - 1) / kWarpsPerBlock);
    block = kThreads;
    smem = (size_t)kWarpsPerBlock * kDeflateWarp;
    fn = store ? (const void*)inflate_kernel : (const void*)inflate_sizes_kernel;
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
    int stage = kRleStageBytes;
    if (stage < parts * RleRing::SMEM) stage = parts * RleRing::SMEM;  // ring fallback fits
    a.stage_bytes = stage;
    smem = (size_t)stage + (size_t)parts * kRleScratch + kRleCtaExtra;
    if (fam == 1) fn = store ? (const void*)rle_v1_kernel : (const void*)rle_v1_sizes_kernel;
    else fn = store ? (const void*)rle_v2_kernel : (const void*)rle_v2_sizes_kernel;
  }
  void* params[] = {&a};
  cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(block), params, smem, stream);
  if (e != cudaSuccess) return cuda_fail(e, "decode launch");
  g_launches.fetch_add(1);
  return CODAG_OK;
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
  int fit = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, batch_kernel, kThreads, kBatchSmem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  int per_sm = g_batch_ctas_per_sm.load();
  if (per_sm <= 0 || per_sm > fit) per_sm = fit;
  if (per_sm < 1) per_sm = 1;
  const uint64_t grid = (uint64_t)per_sm * (uint64_t)w.sm_count;
  batch_kernel<<<(unsigned)grid, kThreads, kBatchSmem, stream>>>(a);
  batch_finalize_kernel<<<og, 256, 0, stream>>>(formats, comp_offsets, out_offsets, n, keys, status);
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

codag_status codag_set_parts_per_chunk(int parts) {
  if (parts < 0 || parts > 16 || (parts & (parts - 1)))
    return fail(CODAG_EINVAL, "parts per chunk must be 0 or a power of two <= 16");
  g_parts_per_chunk.store(parts);
  return CODAG_OK;
}

int codag_get_parts_per_chunk(void) { return g_parts_per_chunk.load(); }

uint64_t codag_kernel_launches(void) { return g_launches.load(); }

const char* codag_last_error(void) { return g_last_error.c_str(); }

const char* codag_version(void) { return "codag-gb300 0.1"; }

}  // extern "C"
