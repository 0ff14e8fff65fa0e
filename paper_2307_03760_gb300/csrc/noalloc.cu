// codag_decompress_batch_noalloc: the mixed-format batch decode for callers
// that cannot let a library allocate device memory.
//
// Who needs it: programs that account for every byte of device memory
// themselves (a fixed budget or their own pool, where an allocation behind
// their back breaks the accounting), and latency-critical loops where the
// first-call cudaMalloc of the ordinary entry point, which can synchronise the
// whole device, is not acceptable.
//
// How: the batch kernel's scratch (claim counter, size histogram, claim
// order, combined status of split chunks) lives in the file-scope array
// below instead of the library workspace.  The array is part of the library
// image, so every GPU that loads the library holds it (about 385 KiB) until
// the process exits.  Host code may not use the array's name as a device
// address; the first call on each device, with that device current, asks the
// runtime for the array's address with cudaGetSymbolAddress and keeps it.
// That first call also sets the shared-memory attribute of every compiled
// shape of the batch kernel, so make it before any stream capture.
//
// All calls on a device share the one array and it keeps the last call's
// contents: each call clears the parts that must start at zero (or all ones)
// before its kernels run.  Calls whose work overlaps on the GPU (for example
// on two streams) race on the array and must not be issued.
#include <mutex>
#include <string>

#include "../../include/codag.h"
#include "kernels.cuh"

namespace codag {
void note_launches(uint64_t n);
void note_error(const std::string& msg);
int batch_shape_selected();
}  // namespace codag

using namespace codag;

namespace {

constexpr uint64_t kMaxChunks = CODAG_NOALLOC_MAX_CHUNKS;
// byte layout: combined status keys (u64 per chunk), counters, claim order
constexpr size_t kKeysOff = 0;
constexpr size_t kCountersOff = kKeysOff + kMaxChunks * 8;
constexpr size_t kOrderOff = kCountersOff + ((kBatchCounterWords * 4 + 255) & ~size_t(255));
constexpr size_t kScratchBytes = kOrderOff + kMaxChunks * 4;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

struct DeviceSetup {
  bool ready = false;
  uint8_t* scratch = nullptr;  // device address of g_noalloc_scratch
  int sm_count = 0;
  int fit[kBatchShapes] = {};  // resident batch CTAs per SM, per ring shape
};

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

codag_status fail(codag_status s, const std::string& msg) {
  note_error(msg);
  return s;
}

// Once per device, with the device current: find the array and size the grid.
codag_status setup_current_device(DeviceSetup** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CODAG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(CODAG_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(CODAG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    e = cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
      return fail(CODAG_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
    for (int i = 0; i < kBatchShapes; i++) {
      const BatchShape b = batch_shape(i);
      e = cudaFuncSetAttribute(b.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, b.smem);
      if (e != cudaSuccess)
        return fail(CODAG_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s.fit[i], b.fn, kThreads, b.smem);
      if (e != cudaSuccess)
        return fail(CODAG_ECUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
    }
    s.scratch = static_cast<uint8_t*>(p);
    s.ready = true;
  }
  *out = &s;
  return CODAG_OK;
}

}  // namespace

extern "C" codag_status codag_decompress_batch_noalloc(const uint8_t* formats, const void* comp,
                                                       const uint64_t* comp_offsets,
                                                       uint64_t n_chunks, void* out,
                                                       const uint64_t* out_offsets,
                                                       int32_t* chunk_status,
                                                       cudaStream_t stream) {
  if (n_chunks == 0) return CODAG_OK;
  if (n_chunks > kMaxChunks)
    return fail(CODAG_EINVAL, "codag_decompress_batch_noalloc: n_chunks " + std::to_string(n_chunks) +
                                  " exceeds the maximum of " + std::to_string(kMaxChunks));
  if (!formats || !comp || !comp_offsets || !out || !out_offsets || !chunk_status)
    return fail(CODAG_EINVAL, "codag_decompress_batch_noalloc: NULL argument");
  if (reinterpret_cast<uintptr_t>(comp) & 15) return fail(CODAG_EINVAL, "comp must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(out) & 7) return fail(CODAG_EINVAL, "out must be 8-byte aligned");
  DeviceSetup* s;
  codag_status st = setup_current_device(&s);
  if (st != CODAG_OK) return st;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(s->scratch + kKeysOff);
  uint32_t* counters = reinterpret_cast<uint32_t*>(s->scratch + kCountersOff);
  uint32_t* order = reinterpret_cast<uint32_t*>(s->scratch + kOrderOff);

  // the counter, histogram and cursors start at zero, the keys at all ones
  cudaError_t e = cudaMemsetAsync(counters, 0, kBatchCounterWords * sizeof(uint32_t), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0xff, n_chunks * 8, stream);
  if (e != cudaSuccess) return fail(CODAG_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  const unsigned og = (unsigned)((n_chunks + 255) / 256 < 1024 ? (n_chunks + 255) / 256 : 1024);
  order_hist_kernel<<<og, 256, 0, stream>>>(formats, comp_offsets, out_offsets, n_chunks, counters + 1);
  order_scatter_kernel<<<og, 256, 0, stream>>>(formats, comp_offsets, out_offsets, n_chunks,
                                               counters + 1, counters + 1 + kBuckets, order);
  Args a{};
  a.comp = static_cast<const uint8_t*>(comp);
  a.comp_off = comp_offsets;
  a.n = n_chunks;
  a.out = static_cast<uint8_t*>(out);
  a.out_off = out_offsets;
  a.status = chunk_status;
  a.formats = formats;
  a.order = order;
  a.counter = counters;
  a.keys = keys;
  int split_lg = 0, split_max = 0;
  codag_get_batch_split(&split_lg, &split_max);
  a.split_lg = (uint32_t)split_lg;
  a.split_max = (uint32_t)split_max;
  const int shape = batch_shape_selected();
  const BatchShape b = batch_shape(shape);
  int per_sm = codag_get_batch_ctas_per_sm();
  if (per_sm <= 0 || per_sm > s->fit[shape]) per_sm = s->fit[shape];
  if (per_sm < 1) per_sm = 1;
  const uint64_t grid = (uint64_t)per_sm * (uint64_t)s->sm_count;
  void* params[] = {&a};
  e = cudaLaunchKernel(b.fn, dim3((unsigned)grid), dim3(kThreads), params, (size_t)b.smem, stream);
  if (e != cudaSuccess) return fail(CODAG_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  batch_finalize_kernel<<<og, 256, 0, stream>>>(formats, comp_offsets, out_offsets, n_chunks, keys,
                                                chunk_status, a.split_lg, a.split_max);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CODAG_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  note_launches(4);
  return CODAG_OK;
}
