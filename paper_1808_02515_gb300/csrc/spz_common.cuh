// Shared definitions of the CUDA Sprintz codec (sm_103a).
//
// Stream format (identical bytes for every implementation of it):
//   [0, 64)         header: "SPZ1", version 1, w, forecaster, flags (bit 0 =
//                   Huffman), D (u16), G, learn_shift, chunk_rows (u32),
//                   huff_chunks (u32), n_chunks (u32), rows (u64), tail_rows
//                   (u32), reserved (u32), data_off, tail_off, total (u64)
//   [64, +16/chunk) chunk table: u64 body offset from data_off, u32 record
//                   count, u32 packed bytes
//   Huffman tables  128 bytes per segment of huff_chunks chunks (flag set)
//   data_off        chunk bodies; each body is groups of G records: the G
//                   records' width codes (log2(w) bits each, record s column j
//                   at bit (s*D + j)*log2(w), LSB first, zero padded to a byte),
//                   then the records' payloads
//   tail_off        rows % 8 trailing rows, raw
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <vector>

#include "../../include/sprintz_gb300.h"

namespace spz {

constexpr int kBlockRows = 8;          // B (Sec. 4.1)
constexpr uint32_t kHdrBytes = 64;
constexpr uint32_t kEntryBytes = 16;
constexpr uint32_t kHuffTableBytes = 128;
constexpr uint32_t kMaxRun = 65535;    // run counts are 16-bit
constexpr uint32_t kMaxD = 1024;
constexpr int kFcDelta = 0;       // x_{i-1} (Sec. 4.2.1)
constexpr int kFcFire = 1;        // FIRE, block form: alpha per block, one averaged update (Sec. 4.2.2)
constexpr int kFcDDelta = 2;      // double delta x_{i-1} + delta_{i-1} (Sec. 4.2.2, a = 2, b = -1)
constexpr int kFcFireSample = 3;  // FIRE per sample (Algorithm 3 without Sec. 4.2.2's changes): alpha and a step every sample

// Everything about a stream's layout that the host knows before launch.
struct Geom {
  uint64_t rows;
  uint64_t full_rows;      // rows - rows % 8
  uint64_t chunk_rows;     // rows per chunk (the last may be shorter)
  uint32_t chunk_rows_opt; // the option as given (0 = one chunk)
  uint64_t data_off;
  uint64_t tail_rows;
  uint32_t n_chunks;
  uint32_t D;
  uint32_t w;
  uint32_t wb;             // bytes per element
  uint32_t G;
  uint32_t hb;             // header bits per code: log2(w)
  uint32_t hdr_bytes;      // ceil(G*D*hb/8)
  uint32_t col_major;      // D*w <= 32
  uint32_t forecaster;
  uint32_t learn_shift;
  uint32_t huffman;
  uint32_t huff_chunks;
  uint32_t n_segments;
  uint32_t max_blocks;     // blocks in the largest chunk
  uint64_t max_body;       // largest possible body of one chunk
};

__host__ __device__ inline uint64_t max_body_bytes(uint64_t n_blocks, uint32_t D, uint32_t w,
                                                   uint32_t G) {
  uint64_t hdr = ((uint64_t)G * D * (w == 8 ? 3u : 4u) + 7) / 8;
  return (n_blocks + G - 1) / G * hdr + n_blocks * (uint64_t)D * w;
}

// Bytes of a chunk's rows as stored in the uncompressed series.
__host__ __device__ inline uint64_t chunk_raw_bytes(const Geom &g, uint64_t rows) {
  return rows * g.D * g.wb;
}

// Bytes between the staged 8-row blocks of consecutive chunks of a warp
// (lane-per-column kernels).  When a row is a whole number of 8-byte words,
// the stride is padded so that chunk k's block starts k * D * wb bytes (mod
// 128) into the shared-memory banks: one row of all the warp's chunks then
// falls into disjoint banks.
__host__ __device__ inline uint32_t blk_stage_stride(uint32_t D, uint32_t wb) {
  const uint32_t row = D * wb, blk = kBlockRows * row;
  if (row % 8) return blk;
  return blk + ((row - blk) & 127u);
}

__device__ __forceinline__ void set_status(int *status, int code) {
  atomicCAS(status, 0, code);
}

// Width code <-> stored width (a width of w-1 is promoted to w; code w-1
// means w).
__device__ __forceinline__ uint32_t code_to_width(uint32_t c, uint32_t w) {
  return c == w - 1 ? w : c;
}
__device__ __forceinline__ uint32_t width_to_code(uint32_t n, uint32_t w) {
  return n == w ? w - 1 : n;
}

// Sign-extend the low W bits.
template <int W>
__device__ __forceinline__ int32_t sext(uint32_t v) {
  return (int32_t)(v << (32 - W)) >> (32 - W);
}

__device__ __forceinline__ int32_t sign_of(int32_t v) { return (v > 0) - (v < 0); }

// Zigzag of a signed W-bit value (Sec. 4.3) as an unsigned W-bit value.
template <int W>
__device__ __forceinline__ uint32_t zigzag(int32_t e) {
  return ((uint32_t)e << 1 ^ (uint32_t)(e >> 31)) & ((1u << W) - 1u);
}
template <int W>
__device__ __forceinline__ int32_t unzigzag(uint32_t z) {
  return (int32_t)(z >> 1) ^ -(int32_t)(z & 1u);
}

// Bits needed for v (0 for 0).
__device__ __forceinline__ uint32_t bit_len(uint32_t v) { return 32u - __clz(v); }

// Little-endian loads/stores of one w-bit sample from byte memory.
template <int W>
__device__ __forceinline__ uint32_t load_sample(const uint8_t *p) {
  if (W == 8) return p[0];
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8);
}
template <int W>
__device__ __forceinline__ void store_sample(uint8_t *p, uint32_t v) {
  p[0] = (uint8_t)v;
  if (W == 16) p[1] = (uint8_t)(v >> 8);
}

// Read `n` (<= 25) bits starting at bit position `bit` of a byte array.
__device__ __forceinline__ uint32_t read_bits(const uint8_t *base, uint64_t bit, uint32_t n) {
  const uint8_t *p = base + (bit >> 3);
  uint32_t s = (uint32_t)(bit & 7);
  uint32_t need = (s + n + 7) >> 3;  // 0..4 bytes
  uint32_t v = 0;
  for (uint32_t k = 0; k < need; ++k) v |= (uint32_t)p[k] << (8 * k);
  return n ? (v >> s) & (0xFFFFFFFFu >> (32 - n)) : 0u;
}

// FIRE fixed-point step shared by encoder and decoder: floor(wrap_2w(alpha *
// delta) / 2^w) modulo 2^w, returned unreduced in its low w bits.
template <int W>
__device__ __forceinline__ uint32_t fire_pred_delta(int32_t alpha, int32_t delta) {
  return (uint32_t)((uint32_t)alpha * (uint32_t)delta) >> W;
}

// The accumulator is a signed 2w-bit integer (wraps at 2w bits).
template <int W>
__device__ __forceinline__ int32_t wrap_acc(int32_t v) {
  if (W == 16) return v;
  return (int32_t)(int16_t)v;
}

// Relaxed/acquire 64-bit global accesses for the encoder's offset scan.
__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
// Relaxed gpu-scope accesses: for flags whose own word is the only data
// exchanged (no L1 invalidation, no fence).
__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// L2 eviction policies (createpolicy) and global accesses that carry one:
// data read once and streamed through is marked evict_first, data written
// now and read back soon (the encoder's body slots) evict_last.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// Read-only (non-coherent) 8-byte load with an L2 policy.
__device__ __forceinline__ unsigned long long ldg_u64_hint(const unsigned long long *p, uint64_t pol) {
  unsigned long long v;
  asm("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}
// 16-byte load / store with an L2 policy (data this kernel writes).
__device__ __forceinline__ uint4 ld_v4_hint(const void *p, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_v4_hint(void *p, uint4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w), "l"(pol)
               : "memory");
}

// Bulk prefetch of [p, p + bytes) into L2 (TMA unit; p and bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Prefetch the 16-byte-aligned part of [lo, hi) that lies inside [buf_lo, buf_hi).
__device__ __forceinline__ void prefetch_l2_range(uintptr_t lo, uintptr_t hi, uintptr_t buf_lo,
                                                  uintptr_t buf_hi) {
  uintptr_t a = (lo > buf_lo ? lo : buf_lo);
  a = (a + 15) & ~(uintptr_t)15;
  uintptr_t b = hi < buf_hi ? hi : buf_hi;
  b &= ~(uintptr_t)15;
  if (b > a) prefetch_l2_bulk((const void *)a, (uint32_t)(b - a));
}

// mbarrier and TMA bulk-copy helpers (shared-memory addresses are 32-bit).
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// Global -> shared bulk copy completing on `bar` (16-byte aligned, multiple of 16).
__device__ __forceinline__ void tma_load_1d(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Wait for the phase of `bar` with the given parity; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
  const uint32_t a = smem_addr(bar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Copy n bytes with every thread of the grid: 16-byte vectors when source
// and destination share their alignment modulo 16, else 4-byte words when
// they share it modulo 4, else bytes.
__device__ __forceinline__ void grid_copy(uint8_t *dst, const uint8_t *src, uint64_t n) {
  const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  const uintptr_t mis = ((uintptr_t)dst ^ (uintptr_t)src);
  const uint32_t vec = (mis & 15) == 0 ? 16u : ((mis & 3) == 0 ? 4u : 1u);
  uint64_t head = vec == 1 ? 0 : ((vec - ((uintptr_t)dst & (vec - 1))) & (vec - 1));
  if (head > n) head = n;
  for (uint64_t k = t0; k < head; k += nt) dst[k] = src[k];
  const uint64_t nv = vec == 1 ? 0 : (n - head) / vec;
  if (vec == 16) {
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src + head);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst + head);
    for (uint64_t k = t0; k < nv; k += nt) d4[k] = s4[k];
  } else if (vec == 4) {
    const uint32_t *s4 = reinterpret_cast<const uint32_t *>(src + head);
    uint32_t *d4 = reinterpret_cast<uint32_t *>(dst + head);
    for (uint64_t k = t0; k < nv; k += nt) d4[k] = s4[k];
  }
  for (uint64_t k = head + nv * vec + t0; k < n; k += nt) dst[k] = src[k];
}

// Host helpers --------------------------------------------------------------

struct LaunchCfg {
  int sm_count;
  int max_smem_optin;
  uint32_t wait_limit;        // look-back polls before SPRINTZ_ERR_TIMEOUT (0: the default)
  uint32_t skip_first_group;  // failure test: single-stream encoders start their ticket at 1
};

int make_geom(uint64_t rows, uint32_t D, uint32_t w, const sprintz_opts *o, Geom *g);

// Float quantization (spz_quant.cu).
int launch_quantize(const LaunchCfg &cfg, const float *x, uint64_t rows, uint32_t D, uint32_t w, uint8_t *codes,
                    double *lo_hi, uint8_t *ws, cudaStream_t stream);
int launch_dequantize(const LaunchCfg &cfg, const uint8_t *codes, uint64_t rows, uint32_t D, uint32_t w,
                      const double *lo_hi, float *y, cudaStream_t stream);
int launch_quant_nmse(const LaunchCfg &cfg, const float *x, const uint8_t *codes, uint64_t rows, uint32_t D,
                      uint32_t w, const double *lo_hi, double *nmse, uint8_t *ws, cudaStream_t stream);

// Forecast transform alone (spz_forecast.cu).
int launch_forecast(const LaunchCfg &cfg, const uint8_t *src, uint64_t rows, uint32_t D, uint32_t w,
                    uint32_t forecaster, uint32_t learn_shift, uint32_t chunk_rows, bool inverse, uint8_t *dst,
                    cudaStream_t stream);

// Encoder / decoder launchers (spz_encode.cu, spz_decode.cu).
uint64_t encode_workspace_bytes(const Geom &g, const LaunchCfg &cfg);
int launch_encode(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint8_t *dst,
                  uint64_t dst_cap, uint64_t *d_out_size, uint8_t *ws, uint64_t ws_bytes,
                  int *d_status, cudaStream_t stream);
int launch_encode_fast(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint8_t *dst,
                       uint64_t dst_cap, uint64_t *d_out_size, uint8_t *ws, uint64_t ws_bytes,
                       int *d_status, cudaStream_t stream);
uint64_t decode_workspace_bytes(const Geom &g, const LaunchCfg &cfg);
// Huffman stage (spz_huff.cu)
uint64_t huff_encode_workspace_bytes(const Geom &g, const LaunchCfg &cfg);
int launch_encode_huffman(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint8_t *dst,
                          uint64_t dst_cap, uint64_t *d_out_size, uint8_t *ws, uint64_t ws_bytes,
                          int *d_status, cudaStream_t stream);
uint64_t huff_decode_workspace_bytes(const Geom &g, const LaunchCfg &cfg);
int launch_decode_huffman(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint64_t src_size,
                          uint8_t *dst, uint64_t dst_cap, uint8_t *ws, uint64_t ws_bytes, int *d_status,
                          cudaStream_t stream);

// Batched launches: the host part of a plan (device descriptors live in the
// workspace at the recorded offsets).
struct BatchPlan {
  int compress;
  uint32_t n;
  uint32_t grid;
  uint32_t region;        // shared bytes per warp
  uint64_t slot_region;   // encode: slot bytes per warp; decode: nonzero if any range request
  uint64_t items_off;     // descriptor table
  uint64_t work_off;      // work list: one u64 (stream << 40 | chunk group) per work item
  uint64_t n_work;
  uint64_t slots_off;     // encode: slots; decode: range temporaries
  uint64_t zero_bytes;    // ticket (+ encode: look-back words) to clear at [0, zero_bytes)
  uint64_t ws_total;
  sprintz_schedule sched; // the schedule the plan was built with (defaults filled in)
  void *ws;
};
// A work entry: stream index (< 2^24) and chunk group of that stream.
constexpr uint32_t kWorkGroupBits = 40;
constexpr uint32_t kMaxBatchStreams = 1u << 24;
// The work list's classes (one per (w, D) pair) and each SM's home class:
// warps take work from their SM's home class first, so that the warps of an
// SM run one specialisation at a time (the instruction cache holds one), and
// move on to the other classes once it is exhausted.  The table precedes
// the work entries in the workspace; the class tickets are the first
// kClassTicketBytes of the workspace.
constexpr uint32_t kMaxBatchClasses = 64;
constexpr uint32_t kMaxHomeSm = 512;
constexpr uint64_t kClassTicketBytes = 4 * kMaxBatchClasses;
struct BatchClasses {
  uint32_t n_classes;
  uint32_t n_sm;                          // SM ids are taken modulo n_sm
  uint64_t start[kMaxBatchClasses + 1];   // work entries [start[c], start[c + 1]) are class c's
  uint8_t home[kMaxHomeSm];
};
constexpr uint64_t kClassTableBytes = (sizeof(BatchClasses) + 255) & ~255ull;
// Resolve the 0 (= default) fields of a schedule for one direction.
sprintz_schedule batch_default_schedule(int compress);
// Build the plan and the descriptor image (host bytes to copy to ws +
// items_off and ws + work_off).  Returns SPRINTZ_OK or an error.
int plan_batch_encode(const sprintz_batch_item *items, uint32_t n, const LaunchCfg &cfg,
                      const sprintz_schedule &sched, int *d_status, uint8_t *ws, BatchPlan *plan,
                      std::vector<uint8_t> *items_img, std::vector<uint64_t> *work_img);
int run_batch_encode(const BatchPlan &plan, cudaStream_t stream);
int plan_batch_decode(const sprintz_batch_item *items, uint32_t n, const LaunchCfg &cfg,
                      const sprintz_schedule &sched, int *d_status, uint8_t *ws, BatchPlan *plan,
                      std::vector<uint8_t> *items_img, std::vector<uint64_t> *work_img);
int run_batch_decode(const BatchPlan &plan, cudaStream_t stream);
// The work image of a batch: the class table (kClassTableBytes), then per
// (w, D) class (classes in a fixed order, the heaviest groups first) the
// chunk groups of the class's streams in the schedule's order; every
// stream's groups stay in increasing order.  SMs get home classes in
// proportion to the classes' chunk groups.
void batch_work_list(const std::vector<uint32_t> &w, const std::vector<uint32_t> &D,
                     const std::vector<uint64_t> &groups, uint32_t order, uint32_t sm_count,
                     std::vector<uint64_t> *image, uint64_t *n_work);
// The next work entry of a warp of a batched kernel (the same value in every
// lane): from the SM's home class while it lasts, then from the others in
// turn.  False when every class is exhausted.
__device__ __forceinline__ bool batch_next(const BatchClasses *cls, const uint64_t *work, uint32_t *tickets,
                                           uint32_t &c, uint64_t *entry) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nc = cls->n_classes;
  for (uint32_t tried = 0; tried < nc; ++tried) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&tickets[c], 1u);
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    const uint64_t s0 = cls->start[c], n = cls->start[c + 1] - s0;
    if (t < n) {
      *entry = __ldg(work + s0 + t);
      return true;
    }
    c = c + 1 == nc ? 0 : c + 1;
  }
  return false;
}
__device__ __forceinline__ uint32_t batch_home(const BatchClasses *cls) {
  uint32_t smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  return cls->n_classes ? cls->home[smid % cls->n_sm] : 0u;
}
int launch_decode(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint64_t src_size,
                  uint8_t *dst, uint64_t dst_cap, uint8_t *ws, uint64_t ws_bytes, int *d_status,
                  cudaStream_t stream);
// Decode chunks [c_begin, c_end) of a stream without Huffman coding into dst
// (8-byte aligned; it receives rows from c_begin * chunk_rows on) with the
// lane or the wide decoder; no header check and no tail.  Returns
// SPRINTZ_ERR_UNSUPPORTED when neither decoder takes this stream.
bool decode_chunks_supported(const Geom &g, const LaunchCfg &cfg);
int launch_decode_chunks(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint64_t src_size,
                         uint32_t c_begin, uint32_t c_end, uint8_t *dst, uint64_t dst_cap, int *d_status,
                         cudaStream_t stream);
// Rows [row_begin, row_end) of a stream into out (any alignment).
uint64_t decode_rows_workspace_bytes(const Geom &g, const LaunchCfg &cfg, uint64_t row_begin, uint64_t row_end);
int launch_decode_rows(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint64_t src_size,
                       uint64_t row_begin, uint64_t row_end, uint8_t *out, uint8_t *ws, uint64_t ws_bytes,
                       int *d_status, cudaStream_t stream);
// Buffers back to back, offsets by a device-side exclusive scan (spz_append.cu).
int launch_pack(const LaunchCfg &cfg, const uint64_t *srcs, const uint64_t *sizes, uint32_t n, uint8_t *dst,
                uint64_t dst_cap, uint64_t *offsets, int *d_status, uint32_t *d_ok, cudaStream_t stream);
// A stream followed by n_new more rows (spz_append.cu).
uint64_t append_workspace_bytes(const Geom &g_old, const LaunchCfg &cfg, uint64_t n_new);
int launch_append(const Geom &g_old, const LaunchCfg &cfg, const uint8_t *src, uint64_t src_size,
                  uint64_t old_tail_off, const uint8_t *rows, uint64_t n_new, uint8_t *dst, uint64_t dst_cap,
                  uint64_t *d_out_size, uint8_t *ws, uint64_t ws_bytes, int *d_status, cudaStream_t stream);

}  // namespace spz
