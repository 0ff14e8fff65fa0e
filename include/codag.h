/*
 * codag.h - chunk-parallel GPU decompression for ORC integer RLE v1/v2 and
 * raw Deflate (C ABI of libcodag.so, built for sm_103a).
 *
 * The operation (CODAG, Sec. II-B "Parallelizing Decompression"): a column
 * is split into chunks that were compressed independently; metadata gives
 * each chunk's compressed and uncompressed offsets, so every chunk decodes on
 * its own.  One call decodes many chunks of one format (or, in the batch
 * call, of mixed formats) on one GPU.  The formats are the three the paper
 * evaluates (Sec. V-A): ORC integer RLE version 1 and version 2 and Deflate
 * (RFC 1951, raw: no zlib or gzip wrapper, no preset dictionary).
 *
 * Memory layout shared by every call (all pointers are DEVICE pointers
 * unless noted; the caller owns every buffer):
 *   comp          concatenated compressed chunks; must be 16-byte aligned
 *                 (any cudaMalloc pointer is) and readable over
 *                 [comp, comp + comp_offsets[n_chunks]).
 *   comp_offsets  uint64[n_chunks + 1], byte offsets into comp; chunk c is
 *                 comp[comp_offsets[c] .. comp_offsets[c+1]).  Non-decreasing.
 *   out           output buffer; chunk c decodes into
 *                 out[out_offsets[c] .. out_offsets[c+1]), and must fill that
 *                 span exactly.  For the RLE formats the output is
 *                 little-endian 64-bit integers: out must be 8-byte aligned
 *                 and every RLE offset a multiple of 8.
 *   out_offsets   uint64[n_chunks + 1], byte offsets into out.
 *
 * Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 * default stream).  Argument problems are reported synchronously by the
 * return value and nothing is launched.  Problems with the DATA are reported
 * per chunk on the device (CODAG_CHUNK_* codes below): the call still returns
 * CODAG_OK, the bad chunk's output span is left unspecified, and the other
 * chunks decode normally.  Per-chunk status is read with
 * codag_last_chunk_status() (plain calls) or from the caller's chunk_status
 * array (batch calls).  No call ever traps or faults the GPU on bad data, and
 * every device-side wait is bounded (CODAG_CHUNK_TIMEOUT).
 *
 * Library-owned memory: a per-device workspace (per-chunk status of the last
 * plain call, batch claim counter and order) allocated with cudaMalloc on
 * first use and grown on demand; it lives until process exit.  Calls on the
 * same device share it, so plain calls that overlap on different streams
 * must not rely on codag_last_chunk_status().
 */
#ifndef CODAG_H
#define CODAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cudaStream_t;

/* Chunk formats (CODAG Sec. V-A).  _I64 columns are signed (ORC zigzag
 * encoding of bases, literals and deltas as the ORC format defines), _U64
 * unsigned. */
typedef enum {
  CODAG_ORC_RLE_V1_I64 = 1,
  CODAG_ORC_RLE_V2_I64 = 2,
  CODAG_DEFLATE_RAW = 3,
  CODAG_ORC_RLE_V1_U64 = 4,
  CODAG_ORC_RLE_V2_U64 = 5,
  /* ORC byte RLE (byte columns; output bytes) and boolean RLE (byte RLE over
   * bytes of eight booleans, most significant bit first; output one 0/1 byte
   * per boolean, output span = number of booleans, the stream must decode to
   * exactly ceil(span / 8) bytes).  Not evaluated in the paper; Sec. V-A
   * notes that other encodings can be enabled the same way. */
  CODAG_ORC_BYTE_RLE = 6,
  CODAG_ORC_BOOL_RLE = 7,
  /* An ORC compressed stream with zlib compression: compression chunks of a
   * 3-byte little-endian header v (v >> 1 body bytes follow; bit 0 set: the
   * body is stored as is, clear: it is a raw Deflate stream of its own) and
   * the body; the output is the bodies' decoded bytes in order (Sec. I and
   * II-B: data decoded as existing systems store it). */
  CODAG_ORC_ZLIB = 8
} codag_format;

/* Call status (host side). */
typedef enum {
  CODAG_OK = 0,
  CODAG_EINVAL = 1,   /* bad argument: pointer, alignment, format, size */
  CODAG_ECUDA = 2,    /* a CUDA runtime call failed (see codag_last_error) */
  CODAG_ENOMEM = 3,   /* workspace allocation failed */
  CODAG_ECORRUPT = 4, /* reserved: returned by helpers that read statuses */
  CODAG_ETIMEOUT = 5  /* a bounded host wait ran out */
} codag_status;

/* Per-chunk status (device side), one int32 per chunk. */
enum {
  CODAG_CHUNK_OK = 0,
  CODAG_CHUNK_TRUNCATED = 1,        /* stream needs bytes past the chunk end   */
  CODAG_CHUNK_OUTPUT_OVERFLOW = 2,  /* decodes to more than the output span   */
  CODAG_CHUNK_OUTPUT_UNDERFLOW = 3, /* decodes to less than the output span   */
  CODAG_CHUNK_BAD_HEADER = 4,       /* bad header, varint, block type, patch  */
  CODAG_CHUNK_BAD_HUFFMAN = 5,      /* bad code lengths, code or symbol       */
  CODAG_CHUNK_BAD_DISTANCE = 6,     /* back-reference before the chunk start  */
  CODAG_CHUNK_BAD_STORED_LEN = 7,   /* Deflate stored block LEN != ~NLEN      */
  CODAG_CHUNK_BAD_SPAN = 8,         /* offsets decrease, pass the buffer end, or
                                       an RLE span is not a multiple of 8     */
  CODAG_CHUNK_TIMEOUT = 9           /* a bounded device wait ran out          */
};

/*
 * codag_decompress - decode n_chunks chunks of one format.
 *
 * CODAG Sec. IV-C/IV-D (warp-level decompression) and Sec. IV-E/IV-F
 * (coalesced on-demand reading and writing): an RLE chunk is decoded by one
 * CTA whose warps decode segments of it after one warp has walked the run
 * headers, its compressed bytes staged in shared memory with 1-D TMA bulk
 * copies.  Raw Deflate runs in two passes: Huffman decoding with one lane
 * per chunk, which stores literals in place and writes 32-bit copy commands
 * to a library pool (about a quarter of the decoded size; see
 * codag_set_deflate_pool_limit), then the LZ77 copies with one warp per
 * chunk writing 32 consecutive output bytes per step; a chunk whose
 * commands do not fit its part of the pool, or whose output span is over
 * 128 KiB (one lane would hold the pass back), is decoded by one warp
 * instead (the same result).  Output is written with coalesced stores.
 *
 * format        one of codag_format.
 * comp, comp_offsets, out, out_offsets: see the layout above (device).
 * n_chunks      number of chunks; 0 is a no-op returning CODAG_OK.
 * stream        CUDA stream the work is enqueued on.
 * Returns CODAG_OK once enqueued; CODAG_EINVAL for a NULL pointer (with
 * n_chunks > 0), an unknown format, comp not 16-byte aligned or an RLE out
 * not 8-byte aligned; CODAG_ENOMEM / CODAG_ECUDA on runtime failure.  The
 * per-chunk status goes to the library workspace (codag_last_chunk_status).
 */
codag_status codag_decompress(int format, const void *comp, const uint64_t *comp_offsets,
                              uint64_t n_chunks, void *out, const uint64_t *out_offsets,
                              cudaStream_t stream);

/*
 * codag_decompress_host - codag_decompress from HOST memory to HOST memory,
 * with the copies overlapped with decoding.
 *
 * The paper's pipeline (Sec. II-B) reads compressed chunks from storage into
 * GPU memory, decodes them and hands the output on; this call is that end to
 * end step for data that starts and ends in host memory.  The chunks are cut
 * into slices of about 16 MiB of output (fewer, larger slices when the
 * chunks are too few to keep the GPU busy); slice i's host-to-device copy,
 * its decode and its device-to-host copy are ordered by events across
 * internal streams (one for each copy direction and four for decoding), so
 * copies in both directions overlap the decoding of other slices, and up to
 * four slices decode at once.
 *
 * h_comp        HOST, concatenated compressed chunks (layout of comp above).
 * h_comp_offsets, h_out_offsets: HOST uint64[n_chunks + 1], read during the
 *               call; both must be non-decreasing.
 * h_out         HOST output buffer, written at h_out[h_out_offsets[c] ..].
 * d_comp        DEVICE buffer of at least h_comp_offsets[n_chunks] bytes,
 *               16-byte aligned: the compressed bytes are copied to the same
 *               offsets in it.
 * d_out         DEVICE buffer of at least h_out_offsets[n_chunks] bytes
 *               (8-byte aligned for the RLE formats).
 * h_status      HOST int32[n_chunks] for the per-chunk status, or NULL; the
 *               status also stays in the workspace (codag_last_chunk_status).
 * stream        the call is asynchronous with respect to `stream` like
 *               codag_decompress: work enqueued on it before the call is
 *               ordered before the copies, and work enqueued after it waits
 *               for the last read-back.  h_comp, h_out and h_status must stay valid until
 *               then; they should be page-locked (cudaHostAlloc or
 *               cudaHostRegister), or the copies do not overlap.
 * Calls on one device run one after another on the device (they share the
 * workspace and the copy streams).  Returns as codag_decompress, plus
 * CODAG_EINVAL when an offsets array decreases or d_comp / d_out is NULL.
 * The library has no counterpart in the paper for the slicing itself.
 */
codag_status codag_decompress_host(int format, const void *h_comp, const uint64_t *h_comp_offsets,
                                   uint64_t n_chunks, void *h_out, const uint64_t *h_out_offsets,
                                   void *d_comp, void *d_out, int32_t *h_status,
                                   cudaStream_t stream);

/*
 * codag_decompressed_sizes - decoded size in bytes of each chunk.
 *
 * Chunked formats normally carry uncompressed offsets (CODAG Sec. II-B); this
 * query recovers them when they are missing.  RLE v1/v2 walk the stream
 * without storing values (cheap); raw Deflate stores no size, so the Deflate
 * query decodes every symbol without writing output (about the cost of a
 * decode).  sizes_out: device uint64[n_chunks], written asynchronously.  A
 * chunk that fails to decode gets its size up to the error and a non-zero
 * status in the workspace (codag_last_chunk_status).  Returns as
 * codag_decompress (sizes_out must be non-NULL).
 */
codag_status codag_decompressed_sizes(int format, const void *comp, const uint64_t *comp_offsets,
                                      uint64_t n_chunks, uint64_t *sizes_out,
                                      cudaStream_t stream);

/*
 * codag_decompress_batch - decode a batch of chunks of mixed formats in one
 * persistent, work-stealing launch (CODAG Sec. II-B chunk parallelism; the
 * batching itself is this library's, not the paper's).
 *
 * formats       device uint8[n_chunks], a codag_format per chunk (an unknown
 *               value marks that chunk CODAG_CHUNK_BAD_HEADER).
 * chunk_status  device int32[n_chunks] for per-chunk status, or NULL to use
 *               the library workspace (codag_last_chunk_status).
 * Other arguments as codag_decompress.  Chunks are claimed largest first
 * (by log2 of compressed + uncompressed bytes); an RLE chunk of 2^b bytes
 * (compressed + decoded) is split into clamp(2^(b-16), 1, 16) parts decoded
 * by different warps.  The enqueued work is two memsets, two small ordering
 * kernels, the persistent decode kernel and a status-combining kernel; it
 * allocates nothing once the workspace is large enough, so it may be
 * captured into a CUDA graph after one warm-up call of at least this size.
 */
codag_status codag_decompress_batch(const uint8_t *formats, const void *comp,
                                    const uint64_t *comp_offsets, uint64_t n_chunks, void *out,
                                    const uint64_t *out_offsets, int32_t *chunk_status,
                                    cudaStream_t stream);

/*
 * codag_last_chunk_status - copy the per-chunk status of the last plain call
 * (codag_decompress, codag_decompressed_sizes, or a batch call without
 * chunk_status) on the current device into host_status[0..n).  Synchronises
 * `stream`.  host_status is HOST memory.  Returns CODAG_EINVAL if n exceeds
 * the last call's chunk count, CODAG_ECORRUPT (after copying) if any chunk is
 * not CODAG_CHUNK_OK.
 */
codag_status codag_last_chunk_status(int32_t *host_status, uint64_t n, cudaStream_t stream);

/*
 * codag_decompress_batch_ws - codag_decompress_batch with caller-provided
 * scratch (device memory, 256-byte aligned, at least
 * codag_batch_scratch_bytes(n_chunks) bytes) instead of the shared library
 * workspace, so that batches on several streams may run at the same time
 * (each with its own scratch).  chunk_status is required.  Nothing is
 * allocated; the scratch is only used by the work this call enqueues.
 */
uint64_t codag_batch_scratch_bytes(uint64_t n_chunks);
codag_status codag_decompress_batch_ws(const uint8_t *formats, const void *comp,
                                       const uint64_t *comp_offsets, uint64_t n_chunks, void *out,
                                       const uint64_t *out_offsets, int32_t *chunk_status,
                                       void *scratch, uint64_t scratch_bytes, cudaStream_t stream);

/*
 * codag_decompress_batch_noalloc - the batch decode above, for callers that
 * cannot let a library allocate device memory: programs that budget or pool
 * every byte of device memory themselves, and latency-critical loops that
 * cannot afford the device-wide synchronisation a first-call cudaMalloc may
 * cause.  The paper has no counterpart; this is an interface choice of this
 * library.
 *
 * It allocates nothing.  Its scratch (claim counter, size histogram, claim
 * order, combined status of split chunks) is a fixed array compiled into the
 * library, so every GPU that loads the library holds it (about 385 KiB)
 * until the process exits.  At most
 * CODAG_NOALLOC_MAX_CHUNKS chunks per call: a larger n_chunks returns
 * CODAG_EINVAL and enqueues nothing.  chunk_status (device int32[n_chunks])
 * is required; the other arguments are those of codag_decompress_batch.
 * The first call on each device does a one-time set-up (it looks up the
 * array's device address and sets the kernel's shared-memory limit) with
 * that device current; make that first call before any stream capture.
 * Every call on a device shares the one array: each call clears what must
 * start at zero, but calls whose work overlaps on the GPU (for example on
 * two streams) race on it, so issue them one after another.
 */
#define CODAG_NOALLOC_MAX_CHUNKS 32768
codag_status codag_decompress_batch_noalloc(const uint8_t *formats, const void *comp,
                                            const uint64_t *comp_offsets, uint64_t n_chunks,
                                            void *out, const uint64_t *out_offsets,
                                            int32_t *chunk_status, cudaStream_t stream);

/*
 * A batch decode captured once into a CUDA graph and replayed.  create
 * captures codag_decompress_batch for fixed arguments (all pointers stay
 * owned by the caller and must outlive the graph) with a private claim
 * counter and order buffer, so several graphs may run concurrently.
 * chunk_status must be non-NULL.  launch enqueues one replay on `stream`.
 */
typedef struct codag_graph_s *codag_graph;
codag_status codag_batch_graph_create(const uint8_t *formats, const void *comp,
                                      const uint64_t *comp_offsets, uint64_t n_chunks, void *out,
                                      const uint64_t *out_offsets, int32_t *chunk_status,
                                      cudaStream_t stream, codag_graph *graph_out);
codag_status codag_batch_graph_launch(codag_graph graph, cudaStream_t stream);
codag_status codag_batch_graph_destroy(codag_graph graph);

/*
 * Launch shape of the persistent batch kernel: resident CTAs (4 decoder
 * warps each) per SM.  0 = as many as fit (the default).  Used by the
 * autotuner; takes effect for later calls and graph captures.
 */
codag_status codag_set_batch_ctas_per_sm(int ctas_per_sm);
int codag_get_batch_ctas_per_sm(void);

/*
 * Header walk of the plain RLE v2 calls (codag_decompress and
 * codag_decompress_host with an RLE v2 format; CODAG Sec. II-B: decoders
 * start independently where the stream's boundaries are known).  A chunk staged whole is cut into segments of
 * about 1024 values that start at run boundaries, found by walking its run
 * headers.  mode 0 (the default): each chunk's CTA walks its own chunk while
 * its other warps decode the segments already found.  mode 1: a walk pass,
 * one warp per chunk, walks every chunk at once and writes the segment
 * starts (512 bytes of library workspace per chunk, calls of up to 2^18
 * chunks); the decode pass then decodes segments with no wait.  Other
 * formats: CODAG_EINVAL (get: -1).  Takes effect for later calls; both modes
 * decode the same bytes.  Used by the autotuner.
 */
codag_status codag_set_walk_pass(int format, int mode);
int codag_get_walk_pass(int format);

/*
 * Input staging of the batch kernel (CODAG Sec. IV-E: each decoder warp
 * reads its chunk through a ring of input slots that the copy engine fills
 * ahead of the decoder).  The batch kernel is compiled for a fixed set of
 * ring shapes, SLOT bytes per slot x SLOTS slots per warp:
 * 256 x 8, 512 x 8, 1024 x 4 (the default) and 2048 x 4.  A deeper ring keeps
 * more input in flight per warp; a smaller one leaves room for more CTAs per
 * SM.  codag_batch_staging_shapes writes up to `cap` shapes into the two
 * arrays (either may be NULL) and returns how many are compiled.
 * codag_set_batch_staging selects one (0, 0 = the default; any shape not
 * compiled: CODAG_EINVAL, selection unchanged).  Takes effect for later calls
 * and graph captures of the batch entry points, the no-alloc one included.
 * Used by the autotuner; every shape decodes the same bytes.
 */
int codag_batch_staging_shapes(int *slot_bytes, int *slots, int cap);
codag_status codag_set_batch_staging(int slot_bytes, int slots);
codag_status codag_get_batch_staging(int *slot_bytes, int *slots);

/*
 * Chunk-to-warp mapping of the batch kernel for RLE chunks (CODAG Sec. IV-C:
 * one warp per chunk, generalised to parts of one chunk).  A chunk whose
 * compressed plus decoded size is 2^b to 2^(b+1) - 1 bytes is decoded by
 * min(2^(b - split_log2), max_parts) warps when b > split_log2, else by one;
 * each warp walks the run headers to its part's first value and decodes its
 * part.  Deflate, byte RLE and ORC zlib chunks are always decoded whole.
 * split_log2 in [8, 40], max_parts in [1, 32] (1: never split); (0, 0) = the
 * default (16, 16); otherwise CODAG_EINVAL.  Takes effect for later calls and
 * graph captures, the no-alloc entry point included.  Used by the autotuner;
 * every mapping decodes the same bytes.
 */
codag_status codag_set_batch_split(int split_log2, int max_parts);
codag_status codag_get_batch_split(int *split_log2, int *max_parts);

/*
 * Warps per chunk for the plain RLE calls (codag_decompress with an RLE
 * format): one CTA per chunk runs this many warps.  A chunk staged whole in
 * shared memory is cut into segments of about 1024 values (256 for RLE v1):
 * one warp walks the run headers and publishes where each segment starts,
 * and every warp claims segments and decodes them; a larger chunk is cut
 * into one part per warp.  0 = automatic (the default: the smallest power of
 * two that gives at least 32 warps per SM, at most 16); otherwise 1..16.
 * Used by the autotuner.
 */
codag_status codag_set_parts_per_chunk(int parts);
int codag_get_parts_per_chunk(void);

/*
 * Input staging of the one-warp-per-chunk decode kernels (CODAG Sec. IV-E and
 * its register input buffer): mode 0 stages compressed bytes in a per-warp
 * shared-memory ring filled by TMA bulk copies (default); mode 1 keeps a
 * 512-byte window in the warp's registers, refilled by coalesced loads, and
 * reads it with __shfl_sync (no shared memory for the input).  format: a
 * Deflate or byte / boolean RLE format (the setting is per decoder family;
 * RLE v1/v2 always stage in shared memory).  For Deflate, mode 0 selects the
 * two-pass decoder (see codag_decompress) and mode 1 the one-warp decoder
 * with the register ring.  Process-wide; an autotuner choice.  Returns
 * CODAG_EINVAL for another format or mode; the getter returns -1 for another
 * format.
 */
codag_status codag_set_input_staging(int format, int mode);
int codag_get_input_staging(int format);

/*
 * codag_set_deflate_pool_limit - upper bound, in bytes, on the command pool
 * of the two-pass Deflate decoder (0, the default: no bound).  Chunk c owns
 * the pool words from (out_offsets[c] - out_offsets[0]) / 4 + 2c on (a
 * quarter of the decoded size of the call, plus two words a chunk); the
 * pool starts at 64 MiB and grows to what the previous call needed, and a
 * chunk whose part lies past it or past this bound is decoded by the
 * one-warp decoder instead, with the same result.  For callers that
 * bound the library's device memory, and for tests of that fallback.  The
 * library's addition; the paper has no counterpart.  Process-wide.
 */
codag_status codag_set_deflate_pool_limit(uint64_t bytes);
uint64_t codag_get_deflate_pool_limit(void);

/*
 * codag_set_wait_limit_ns - bound, in nanoseconds, of every device wait on
 * work in progress: a staging copy a decoder needs next, or a segment start
 * another warp of the chunk publishes.  Default 100 ms (100000000); 0 makes
 * such a wait give up unless it is already complete.  A wait that runs out
 * ends the chunk with CODAG_CHUNK_TIMEOUT (no other status), after the
 * decoder has waited, bounded by the default, for its own copies in flight.
 * For tests of that path and for callers that prefer a bounded stall; the
 * library's addition, the paper has none.  Process-wide; applies to calls
 * enqueued after it returns (do not call it while decodes are in flight).
 * Returns CODAG_ECUDA if the value cannot be set on the current device.
 */
codag_status codag_set_wait_limit_ns(uint64_t ns);
uint64_t codag_get_wait_limit_ns(void);

/* Number of kernel launches the library enqueued since load (all calls). */
uint64_t codag_kernel_launches(void);

/* Human-readable text of the last error on this thread ("" if none). */
const char *codag_last_error(void);

/* Library version, e.g. "codag-gb300 0.1". */
const char *codag_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CODAG_H */
