/*
 * sprintz_gb300.h — C ABI of the GB300 (sm_103a) Sprintz codec.
 *
 * Sprintz (Blalock, Madden, Guttag, "Sprintz: Time Series Compression for the
 * Internet of Things", IMWUT 2018) compresses a multivariate integer time
 * series — T samples of D columns, every element a w-bit integer, stored
 * row-major (Sec. 2.1, Definitions 2.1-2.3) — in blocks of B = 8 rows:
 * forecast each sample (delta coding, Sec. 4.2.1, or the FIRE online
 * forecaster, Sec. 4.2.2 / Algorithm 3), zigzag the errors, store each
 * column's bit width in a header and bit-pack the errors (Sec. 4.3), replace
 * runs of all-zero blocks by their count (Sec. 4.1, Algorithm 1), and
 * optionally Huffman-code the packed bytes (Sec. 4.4).  Decoding inverts each
 * step (Algorithm 2).
 *
 * Conventions for every entry point:
 *   - Data pointers (src, dst, workspace, out_size) are DEVICE pointers
 *     owned by the caller; the library never allocates on these calls and
 *     never frees caller memory.
 *   - Samples are little-endian, row-major, w in {8, 16} bits, 1 <= D <= 1024.
 *     Their signedness does not matter: all arithmetic is modulo 2^w.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream).  Argument checks are synchronous and return a
 *     negative SPRINTZ_ERR_* code before anything is enqueued.  Errors that
 *     depend on the data (a corrupt stream, a wait that timed out) are
 *     recorded in the context's device status word, read by
 *     sprintz_get_status().
 *   - The stream format is fixed: a 64-byte header, a 16-byte entry per chunk
 *     of `chunk_rows` rows (the forecaster restarts at each chunk), the chunk
 *     bodies (groups of `group_blocks` record headers, then their payloads),
 *     then the rows % 8 trailing rows stored raw.  The same input and options
 *     always give the same bytes.
 */
#ifndef SPRINTZ_GB300_H
#define SPRINTZ_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPRINTZ_OK 0
#define SPRINTZ_ERR_INVALID_ARG (-1)   /* a null pointer, bad D, bad option */
#define SPRINTZ_ERR_UNSUPPORTED_W (-2) /* w is not 8 or 16 */
#define SPRINTZ_ERR_DST_TOO_SMALL (-3) /* dst_cap below what the call may write */
#define SPRINTZ_ERR_WS_TOO_SMALL (-4)  /* workspace below the *_workspace_size() */
#define SPRINTZ_ERR_CORRUPT (-5)       /* a stream that is not a valid Sprintz stream */
#define SPRINTZ_ERR_TIMEOUT (-6)       /* a bounded device wait gave up */
#define SPRINTZ_ERR_CUDA (-7)          /* a CUDA runtime call failed */
#define SPRINTZ_ERR_UNSUPPORTED (-8)   /* a valid option this build does not run */

/* Codec options (the paper's knobs, Sec. 4.1 and 5.2: SprintzDelta,
 * SprintzFIRE, SprintzFIRE+Huf). */
typedef struct {
  uint8_t forecaster;   /* 0 = delta coding (Sec. 4.2.1); 1 = FIRE as used in practice, alpha
                           per block and one averaged update (Sec. 4.2.2); 2 = double delta,
                           the a = 2, b = -1 model of Sec. 4.2.2; 3 = FIRE in its
                           per-sample form (Algorithm 3), alpha and a step at every sample */
  uint8_t huffman;      /* 1 = Huffman-code the bit-packed bytes (Sec. 4.4) */
  uint8_t group_blocks; /* G, 1..8: record headers stored together (Sec. 4.3); the paper uses 2 */
  uint8_t learn_shift;  /* FIRE: alpha = accumulator >> learn_shift; 1 gives eta = 1/2 (Sec. 4.2.2) */
  uint32_t chunk_rows;  /* rows per chunk, multiple of 8; the forecaster restarts at each chunk;
                           0 = one chunk for the whole series (the paper's single stream) */
  uint32_t huff_chunks; /* consecutive chunks sharing one Huffman table (huffman = 1), >= 1.
                           A coded chunk is a jump table of u32 offsets followed by
                           independently decodable sub-blocks of 2048 packed bytes; with
                           huffman = 1 a chunk body may not exceed 2^31 bytes
                           (SPRINTZ_ERR_INVALID_ARG) */
} sprintz_opts;

/* Shape and options of a stream, as recorded in its 64-byte header. */
typedef struct {
  uint64_t rows;
  uint32_t D;
  uint32_t w;
  sprintz_opts opts;
  uint32_t n_chunks;
  uint32_t tail_rows;
  uint64_t data_off;    /* first chunk body */
  uint64_t tail_off;    /* the raw trailing rows */
  uint64_t total_bytes; /* stream size */
} sprintz_info;

typedef struct sprintz_ctx sprintz_ctx;

/* Create a context on `device` (allocates its 4-byte device status word and
 * queries the device).  Returns SPRINTZ_OK and sets *out, or an error. */
int sprintz_ctx_create(sprintz_ctx **out, int device);
void sprintz_ctx_destroy(sprintz_ctx *ctx);

/* Largest stream sprintz_compress() can write for this shape and options:
 * header + chunk table (+ Huffman tables) + for each chunk, one header group
 * per G records and D*w bytes per block + the raw tail.  0 if the arguments
 * are invalid. */
uint64_t sprintz_max_compressed_size(uint64_t rows, uint32_t D, uint32_t w,
                                     const sprintz_opts *opts);

/* Device workspace bytes sprintz_compress() / sprintz_decompress() need for
 * this shape and options (may be 0).  Workspace contents need not be
 * initialised and are not preserved. */
uint64_t sprintz_compress_workspace_size(uint64_t rows, uint32_t D, uint32_t w,
                                         const sprintz_opts *opts);
uint64_t sprintz_decompress_workspace_size(const sprintz_info *info);

/* Compress `rows` x `D` samples at `src` (Algorithm 1 over every chunk).
 * Writes the stream to dst (capacity dst_cap >= sprintz_max_compressed_size)
 * and its size in bytes to the device uint64 *d_out_size.  The workspace must
 * hold sprintz_compress_workspace_size() bytes.  src and dst must not
 * overlap. */
int sprintz_compress(sprintz_ctx *ctx, const void *src, uint64_t rows, uint32_t D, uint32_t w,
                     const sprintz_opts *opts, void *dst, uint64_t dst_cap,
                     uint64_t *d_out_size, void *workspace, uint64_t ws_bytes, void *stream);

/* Decompress a stream of src_size bytes at src (Algorithm 2 over every
 * chunk) into dst (rows x D samples, capacity dst_cap bytes).  `info` is the
 * stream's header as parsed on the host by sprintz_query() (the caller keeps
 * a host copy of the first 64 bytes; the host reads no device data here); the
 * device checks it against the stream and flags SPRINTZ_ERR_CORRUPT on a
 * mismatch. */
int sprintz_decompress(sprintz_ctx *ctx, const void *src, uint64_t src_size,
                       const sprintz_info *info, void *dst, uint64_t dst_cap, void *workspace,
                       uint64_t ws_bytes, void *stream);

/* Decompress rows [row_begin, row_end) of a stream into dst
 * ((row_end - row_begin) x D samples, capacity dst_cap bytes, any alignment):
 * Algorithm 2 over only the chunks that cover those rows -- every chunk
 * decodes on its own, since the forecaster restarts at each one -- and the
 * raw tail rows when the range reaches them.  The covering chunks are decoded
 * into the workspace (sprintz_decompress_rows_workspace_size() bytes) and
 * the rows copied out.  Streams with Huffman coding, or whose chunks no range
 * decoder takes, are decoded whole into the workspace first (a larger
 * workspace, same result).  row_end <= row_begin does nothing;
 * row_end > rows is SPRINTZ_ERR_INVALID_ARG.  `info` as for
 * sprintz_decompress(); the device checks the header and flags
 * SPRINTZ_ERR_CORRUPT. */
uint64_t sprintz_decompress_rows_workspace_size(const sprintz_info *info, uint64_t row_begin, uint64_t row_end);
int sprintz_decompress_rows(sprintz_ctx *ctx, const void *src, uint64_t src_size, const sprintz_info *info,
                            uint64_t row_begin, uint64_t row_end, void *dst, uint64_t dst_cap, void *workspace,
                            uint64_t ws_bytes, void *stream);

/* Append n_rows rows (rows x D samples at `rows`, the stream's w and D) to a
 * compressed stream: dst receives the stream of the old series followed by
 * the new rows, byte for byte what sprintz_compress() of the whole series
 * writes, and *d_out_size its size.  Chunks restart the forecaster, so the
 * old stream's complete chunks are copied as they are; its last chunk if it
 * is partial and its raw tail rows are decoded (Algorithm 2) and encoded
 * again with the new rows (Algorithm 1) in the workspace
 * (sprintz_append_workspace_size() bytes), and one kernel joins the two.
 *   - `info` is the old stream's header as parsed by sprintz_query() (a host
 *     copy); the device checks it against the stream (SPRINTZ_ERR_CORRUPT).
 *   - dst_cap >= sprintz_max_compressed_size(info->rows + n_rows, ...);
 *     dst must not overlap src or rows (the old stream is not grown in
 *     place: its chunk table precedes its bodies).
 *   - Huffman-coded streams, and streams with chunk_rows = 0 whose one chunk
 *     no range decoder takes, are SPRINTZ_ERR_UNSUPPORTED. */
uint64_t sprintz_append_workspace_size(const sprintz_info *info, uint64_t n_rows);
int sprintz_append(sprintz_ctx *ctx, const void *src, uint64_t src_size, const sprintz_info *info,
                   const void *rows, uint64_t n_rows, void *dst, uint64_t dst_cap, uint64_t *d_out_size,
                   void *workspace, uint64_t ws_bytes, void *stream);

/* Pack n device buffers back to back (for storing or moving many compressed
 * streams with one copy; the paper has no counterpart).  Buffer k is
 * d_src_ptrs[k] (a device array of n device addresses) and holds d_sizes[k]
 * bytes (device array, e.g. the out_size words of a batched compress); dst
 * receives them in order with no gaps, d_offsets[k] (device array of n + 1
 * words) where each starts and d_offsets[n] the total -- an exclusive scan
 * taken on the device, so the host reads nothing.  A total above dst_cap
 * copies nothing and records SPRINTZ_ERR_DST_TOO_SMALL in the status word.
 * The sources must not overlap dst. */
int sprintz_pack(sprintz_ctx *ctx, const uint64_t *d_src_ptrs, const uint64_t *d_sizes, uint32_t n, void *dst,
                 uint64_t dst_cap, uint64_t *d_offsets, void *stream);

/* ---- Batches of independent streams --------------------------------------
 * Many streams of uneven length, width and D encoded or decoded by one
 * persistent kernel launch over the chunk groups of all of them.  The paper
 * compresses one stream at a time; a batch is a set of independent streams,
 * and every stream's bytes are exactly those sprintz_compress() would write.
 *
 * sprintz_batch_plan() checks the items, uploads their descriptors into the
 * workspace (one host-to-device copy, stream-ordered) and records the launch
 * shape in the context; sprintz_batch_run() then only enqueues memsets and
 * kernels, so it may be repeated (or captured in a CUDA graph) for the same
 * buffers.  A context holds one plan at a time.  Batches need D <= 32 for
 * every stream, 8-byte-aligned sample buffers (except range outputs), and no
 * Huffman coding (SPRINTZ_ERR_UNSUPPORTED otherwise).  A decompress item with
 * row_end > row_begin is a range request: only the chunks covering those rows
 * are decoded (chunks restart the forecaster, so any chunk decodes alone). */
typedef struct {
  const void *src;     /* compress: rows x D samples; decompress: the stream */
  uint64_t src_bytes;  /* decompress: stream size in bytes; compress: unused */
  void *dst;           /* compress: stream buffer; decompress: rows x D samples */
  uint64_t dst_cap;    /* bytes available at dst */
  uint64_t *out_size;  /* compress: device uint64 receiving the stream size */
  uint64_t rows;       /* shape and options (decompress: from sprintz_query) */
  uint32_t D;
  uint32_t w;
  sprintz_opts opts;
  uint64_t row_begin;  /* decompress: rows [row_begin, row_end) only, when row_end > row_begin; */
  uint64_t row_end;    /*   dst then receives exactly those rows; 0, 0 = the whole stream */
} sprintz_batch_item;

/* Launch schedule of a batched launch: the knobs that change its speed but
 * never its bytes.  0 in a field means the library's default.
 *   ctas_per_sm     persistent CTAs of 4 warps per SM (clamped to what fits).
 *   ring_segments   decompress: TMA ring segments per chunk, 2 or 4.
 *   prefetch_bytes  L2 bulk prefetch this many bytes ahead of each chunk's
 *                   reads (rounded down to 16); 1 = no prefetch.
 *   order           work order inside each (w, D) class of streams (the
 *                   classes come one after another, heaviest chunk groups
 *                   first): 1 = stream order, 2 = longest stream first,
 *                   3 = round robin over the class's streams.
 * Defaults: as many CTAs per SM as fit (7 compress, 6 decompress); compress
 * round robin without prefetch; decompress 2 ring segments, 8 KB prefetch,
 * longest stream first. */
typedef struct {
  uint32_t ctas_per_sm;
  uint32_t ring_segments;
  uint32_t prefetch_bytes;
  uint32_t order;
} sprintz_schedule;

/* Workspace bytes for a batch (compress = 1 or 0) under any schedule; 0 if
 * an item is invalid. */
uint64_t sprintz_batch_workspace_size(sprintz_ctx *ctx, const sprintz_batch_item *items, uint32_t n,
                                      int compress);
/* Plan with the schedule the context's autotuner chose for a batch of this
 * kind (device, direction, forecasters, mix of widths and column counts,
 * size), else the defaults. */
int sprintz_batch_plan(sprintz_ctx *ctx, const sprintz_batch_item *items, uint32_t n, int compress,
                       void *workspace, uint64_t ws_bytes, void *stream);
/* Plan with an explicit schedule (NULL = the defaults). */
int sprintz_batch_plan_schedule(sprintz_ctx *ctx, const sprintz_batch_item *items, uint32_t n, int compress,
                                const sprintz_schedule *schedule, void *workspace, uint64_t ws_bytes,
                                void *stream);
int sprintz_batch_run(sprintz_ctx *ctx, void *workspace, uint64_t ws_bytes, void *stream);
/* The resolved schedule of the context's current plan. */
int sprintz_batch_schedule(sprintz_ctx *ctx, sprintz_schedule *out);

/* Autotuner: plan the batch under a set of candidate schedules, run each
 * (the outputs are written, identically, every time) and time it with CUDA
 * events on `stream` (synchronous), searching one knob at a time from the
 * defaults.  The fastest schedule is remembered in the context for batches
 * of the same kind (and in the text file named by SPRINTZ_SCHEDULE_CACHE, if
 * set, which later contexts read), and the batch is left planned with it.
 * *chosen and *ms (either may be NULL) receive it and its time. */
int sprintz_batch_autotune(sprintz_ctx *ctx, const sprintz_batch_item *items, uint32_t n, int compress,
                           void *workspace, uint64_t ws_bytes, void *stream, sprintz_schedule *chosen,
                           float *ms);

/* Compression for callers that cannot allocate device memory.  (The paper has
 * no counterpart: this is a deployment variant of sprintz_compress.)
 *
 * Some callers cannot call cudaMalloc: a process whose own pool allocator has
 * taken all free device memory, or a serving request path that must not let
 * cudaMalloc/cudaFree implicitly synchronize the device.  This entry point
 * needs no context and no workspace: the encoder's scratch (chunk ticket,
 * look-back words, status word) lives in a fixed 512 KiB array in device
 * memory that the library defines; every GPU that loads the library holds it
 * until the process exits.  It allocates nothing and frees nothing.
 *   - Same arguments, stream bytes and *d_out_size as sprintz_compress() on
 *     the same input; the current device is used.
 *   - Limit: at most 65,536 chunks per call (2^26 rows at chunk_rows = 1024),
 *     and chunks that fit the encoder's shared-memory paths; larger calls
 *     return SPRINTZ_ERR_WS_TOO_SMALL before anything is enqueued.  Huffman
 *     returns SPRINTZ_ERR_UNSUPPORTED.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process: after cudaDeviceReset() on that device it is stale, so this
 *     entry point must not be used on a device once it has been reset.
 *   - Every call shares the one array and each call clears what must start at
 *     zero; two calls whose work overlaps on the GPU (different streams, or
 *     different host threads) race and corrupt each other's output.
 *   - A device-side failure (a bounded wait that gave up) sets *d_out_size to
 *     0. */
int sprintz_compress_noalloc(const void *src, uint64_t rows, uint32_t D, uint32_t w,
                             const sprintz_opts *opts, void *dst, uint64_t dst_cap,
                             uint64_t *d_out_size, void *stream);

/* The forecasting step alone, the subroutine that the FIRE Speed experiment
 * of Sec. 5.6 times: inverse = 0 turns samples into their forecast errors,
 * inverse = 1 rebuilds the samples from such errors.  Neither changes the
 * size: errors are signed w-bit values stored as w-bit two's complement in
 * the samples' row-major layout.
 *   - forecaster 0..3 as in sprintz_opts, learn_shift as there.
 *   - The forecaster restarts every chunk_rows rows (a multiple of 8; 0 =
 *     one chunk, a single sequential pass per column), as in the codec.
 *   - Whole 8-row blocks are transformed; the rows % 8 trailing rows are
 *     copied unchanged.
 *   - src and dst: rows x D samples, 8-byte aligned (else
 *     SPRINTZ_ERR_UNSUPPORTED); dst may equal src.  No workspace.
 *   - 2^32 rows or more with chunk_rows = 0 is SPRINTZ_ERR_UNSUPPORTED. */
int sprintz_forecast(sprintz_ctx *ctx, const void *src, uint64_t rows, uint32_t D, uint32_t w,
                     uint32_t forecaster, uint32_t learn_shift, uint32_t chunk_rows, int inverse, void *dst,
                     void *stream);

/* Float data (Sec. 5.8: quantize, then compress the integers).  Each column
 * of a row-major rows x D float32 series (1 <= D <= 1024) is offset and
 * rescaled linearly so that its minimum and maximum map to 0 and 2^w - 1,
 * then floored: in double precision, every operation rounded on its own,
 *   s = (2^w - 1) / (max - min)  (0 for a constant column),
 *   code = min(floor((x - min) * s), 2^w - 1).
 * The codes are rows x D little-endian w-bit samples, ready for
 * sprintz_compress.  lo_hi (device, 2 D doubles) receives min and max of each
 * column; the inverse needs it.  NaN inputs are not supported.  The
 * workspace holds sprintz_quant_workspace_size(D) bytes (0 for a bad D). */
uint64_t sprintz_quant_workspace_size(uint32_t D);
int sprintz_quantize(sprintz_ctx *ctx, const float *src, uint64_t rows, uint32_t D, uint32_t w, void *codes,
                     double *lo_hi, void *workspace, uint64_t ws_bytes, void *stream);

/* The inverse map: x = (float)(code * h + min), h = (max - min) / (2^w - 1),
 * each operation rounded on its own.  No workspace. */
int sprintz_dequantize(sprintz_ctx *ctx, const void *codes, uint64_t rows, uint32_t D, uint32_t w,
                       const double *lo_hi, float *dst, void *stream);

/* The quantization error of Sec. 5.8, per column: the mean squared error of
 * the reconstruction over the column's (population) variance, in double; 0
 * for a constant column.  nmse: device, D doubles.  The sums are double
 * atomics, so their rounding depends on the order of the additions. */
int sprintz_quant_nmse(sprintz_ctx *ctx, const float *src, const void *codes, uint64_t rows, uint32_t D,
                       uint32_t w, const double *lo_hi, double *nmse, void *workspace, uint64_t ws_bytes,
                       void *stream);

/* Parse a HOST copy of a stream's first n >= 64 bytes. */
int sprintz_query(const void *host_header, uint64_t n, sprintz_info *out);

/* Failure detection, for tests of the error path (both 0 = normal use):
 *   wait_limit        polls the single-stream encoder's look-back (the wait
 *                     for an earlier chunk group's offset) makes before it
 *                     gives up with SPRINTZ_ERR_TIMEOUT (0 = about 4 million,
 *                     a few seconds at most);
 *   skip_first_group  1 = the next single-stream compressions on this
 *                     context never take their first chunk group, so the
 *                     later groups wait for a predecessor that never
 *                     publishes its offset: every such wait runs out, the
 *                     kernel still returns, and sprintz_get_status() reports
 *                     SPRINTZ_ERR_TIMEOUT (the bytes written are not a valid
 *                     stream).
 * Nothing faults or hangs: the waits are bounded and the kernels exit. */
int sprintz_ctx_set_failure_test(sprintz_ctx *ctx, uint32_t wait_limit, uint32_t skip_first_group);

/* Wait for `stream`, return the first data-dependent error recorded since
 * the last call (SPRINTZ_OK if none) and clear it. */
int sprintz_get_status(sprintz_ctx *ctx, void *stream);

/* Static description of an error code. */
const char *sprintz_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
