// Sprintz encoder on sm_103a.
//
// One CTA encodes one chunk at a time (a chunk is an independent Sprintz
// stream of chunk_rows rows: the forecaster restarts at zero).  Chunks are
// taken in order from an atomic ticket, so every chunk a CTA waits on is
// already running.  Per chunk:
//   1. the chunk's rows are staged in shared memory (128-bit loads);
//   2. FIRE only: one thread per column runs the block-level recurrence of
//      alpha (Algorithm 3 with alpha fixed per block, one averaged update per
//      block from the gradients of rows 0, 2, 4, 6 — Sec. 4.2.2);
//   3. every (block, column) recomputes its 8 errors, zigzags them and takes
//      the width from the OR of the column (Sec. 4.3), promoting w-1 to w;
//   4. blocks whose widths are all zero merge into runs; records, groups of G
//      record headers and payload offsets are laid out (Algorithm 1);
//   5. headers and payloads are packed into a shared-memory copy of the body
//      (column-major if D*w <= 32, else row-major — Sec. 4.3);
//   6. a decoupled look-back over the chunks' body sizes (single pass,
//      bounded waits) gives the body's offset in the stream;
//   7. the body and its chunk-table entry are written; the last chunk writes
//      the raw tail, the stream header and the stream size.
// Chunks too large for shared memory use a per-CTA global scratch slot and
// read their rows straight from the source.
#include <stdlib.h>

#include <algorithm>
#include <mutex>

#include "spz_common.cuh"

namespace spz {

constexpr int kEncThreads = 256;
constexpr uint64_t kFlagAggregate = 1ull << 62;
constexpr uint64_t kFlagPrefix = 2ull << 62;
constexpr uint64_t kValueMask = (1ull << 62) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;  // a few seconds at most, then SPRINTZ_ERR_TIMEOUT

struct EncLayout {
  uint64_t x, width, alpha, bsum, rec_first, rec_run, rec_off, body, total;
};

__host__ __device__ inline EncLayout enc_layout(const Geom &g, bool stage_rows) {
  EncLayout L;
  uint64_t o = 0;
  uint64_t nb = g.max_blocks;
  auto take = [&](uint64_t bytes) {
    uint64_t r = o;
    o += (bytes + 15) & ~15ull;
    return r;
  };
  L.x = stage_rows ? take(nb * kBlockRows * g.D * g.wb) : 0;
  L.width = take(nb * g.D);
  L.alpha = take(g.forecaster == kFcFire ? nb * g.D * 4
                 : g.forecaster == kFcFireSample ? nb * kBlockRows * g.D * 4 : 0);
  L.bsum = take(nb * 4);
  L.rec_first = take(nb * 4);
  L.rec_run = take(nb * 4);
  L.rec_off = take(nb * 4);
  L.body = take(g.max_body + 16);  // +16: the unaligned copy reads one word past the end
  L.total = o;
  return L;
}

struct EncParams {
  const uint8_t *src;
  uint8_t *dst;
  uint64_t dst_cap;
  uint64_t *out_size;
  uint32_t *ticket;
  uint64_t *lookback;
  int *status;
  uint8_t *scratch;
  uint64_t scratch_per_cta;
  uint32_t stage_rows;  // 1: rows and working arrays in shared memory
  uint32_t spin_limit;  // look-back polls before SPRINTZ_ERR_TIMEOUT (0: kSpinLimit)
  Geom g;
};

// Clear the ticket and look-back words of a single-stream launch; the
// failure test starts the ticket at 1, so that chunk group 0 is never taken
// and its successors' look-backs run out.
static int init_ticket(uint8_t *ws, uint64_t zero_bytes, const LaunchCfg &cfg, cudaStream_t stream) {
  if (cudaMemsetAsync(ws, 0, zero_bytes, stream) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  if (cfg.skip_first_group && cudaMemsetAsync(ws, 1, 1, stream) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  return SPRINTZ_OK;
}

// ---------------------------------------------------------------------------
// Small device helpers
// ---------------------------------------------------------------------------

// Copy n bytes between arbitrary addresses with the whole CTA; 16-byte
// vector accesses when both ends share the alignment.
__device__ void cta_copy(uint8_t *dst, const uint8_t *src, uint64_t n) {
  uint64_t head = (16 - ((uintptr_t)dst & 15)) & 15;
  if (head > n) head = n;
  bool vec = (((uintptr_t)dst + head) & 15) == 0 && (((uintptr_t)src + head) & 15) == 0;
  if (!vec) {
    for (uint64_t k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
    return;
  }
  for (uint64_t k = threadIdx.x; k < head; k += blockDim.x) dst[k] = src[k];
  uint64_t n16 = (n - head) / 16;
  const uint4 *s4 = reinterpret_cast<const uint4 *>(src + head);
  uint4 *d4 = reinterpret_cast<uint4 *>(dst + head);
  for (uint64_t k = threadIdx.x; k < n16; k += blockDim.x) d4[k] = s4[k];
  for (uint64_t k = head + n16 * 16 + threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

// Copy a 16-byte-aligned source buffer (shared or global, padded by 16
// readable bytes) to a destination of any alignment, 16-byte stores in the
// middle built from funnel-shifted source words.
__device__ void cta_copy_to_unaligned(uint8_t *dst, const uint8_t *src, uint64_t n) {
  uint64_t head = (16 - ((uintptr_t)dst & 15)) & 15;
  if (head > n) head = n;
  for (uint64_t k = threadIdx.x; k < head; k += blockDim.x) dst[k] = src[k];
  uint64_t n16 = (n - head) / 16;
  uint32_t sh = (uint32_t)(head & 3) * 8;
  const uint32_t *sw = reinterpret_cast<const uint32_t *>(src + (head & ~3ull));
  uint4 *d4 = reinterpret_cast<uint4 *>(dst + head);
  for (uint64_t k = threadIdx.x; k < n16; k += blockDim.x) {
    const uint32_t *p = sw + 4 * k;
    uint32_t a = p[0], b = p[1], c = p[2], d = p[3], e = p[4];
    uint4 v;
    v.x = __funnelshift_r(a, b, sh);
    v.y = __funnelshift_r(b, c, sh);
    v.z = __funnelshift_r(c, d, sh);
    v.w = __funnelshift_r(d, e, sh);
    d4[k] = v;
  }
  for (uint64_t k = head + n16 * 16 + threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

// OR `n` (<= 25) bits of v into a zero-initialised byte array at bit `bit`.
__device__ __forceinline__ void or_bits(uint8_t *base, uint64_t bit, uint32_t v, uint32_t n) {
  if (!n) return;
  uint8_t *p = base + (bit >> 3);
  uint32_t s = (uint32_t)(bit & 7);
  uint64_t x = (uint64_t)v << s;
  uint32_t nbytes = (s + n + 7) >> 3;
  for (uint32_t k = 0; k < nbytes; ++k) p[k] |= (uint8_t)(x >> (8 * k));
}

template <int W>
__device__ __forceinline__ uint32_t sample(const uint8_t *X, uint32_t D, uint64_t r, uint32_t j) {
  return load_sample<W>(X + ((uint64_t)r * D + j) * (W / 8));
}

// Forecast error of row r (chunk-relative), column j: delta predicts the
// previous sample (x_{-1} = 0); FIRE adds floor(alpha * delta_{r-1} / 2^w)
// (delta_{-1} = 0, delta_0 = x_0 - 0).
template <int W>
__device__ __forceinline__ int32_t error_at(const uint8_t *X, uint32_t D, uint64_t r, uint32_t j,
                                            uint32_t forecaster, int32_t alpha) {
  uint32_t x = sample<W>(X, D, r, j);
  uint32_t xp = r >= 1 ? sample<W>(X, D, r - 1, j) : 0u;
  if (forecaster == kFcDelta) return sext<W>(x - xp);
  uint32_t xpp = r >= 2 ? sample<W>(X, D, r - 2, j) : 0u;
  int32_t dp = r >= 1 ? sext<W>(xp - xpp) : 0;
  if (forecaster == kFcDDelta) return sext<W>(x - xp - (uint32_t)dp);
  return sext<W>(x - xp - fire_pred_delta<W>(alpha, dp));
}

// The alpha that error_at needs for row i of block b, column j.
__device__ __forceinline__ int32_t alpha_at(const Geom &g, const int32_t *alpha, uint32_t D, uint32_t b,
                                            uint32_t i, uint32_t j) {
  if (g.forecaster == kFcFire) return alpha[(uint64_t)b * D + j];
  if (g.forecaster == kFcFireSample) return alpha[((uint64_t)b * kBlockRows + i) * D + j];
  return 0;
}

__device__ void write_stream_header(uint8_t *h, const Geom &g, uint64_t tail_off, uint64_t total) {
  uint8_t b[64];
  for (int k = 0; k < 64; ++k) b[k] = 0;
  b[0] = 'S';
  b[1] = 'P';
  b[2] = 'Z';
  b[3] = '1';
  b[4] = 1;
  b[5] = (uint8_t)g.w;
  b[6] = (uint8_t)g.forecaster;
  b[7] = (uint8_t)(g.huffman ? 1 : 0);
  auto put = [&](int off, uint64_t v, int n) {
    for (int k = 0; k < n; ++k) b[off + k] = (uint8_t)(v >> (8 * k));
  };
  put(8, g.D, 2);
  b[10] = (uint8_t)g.G;
  b[11] = (uint8_t)g.learn_shift;
  put(12, g.chunk_rows_opt, 4);
  put(16, g.huffman ? g.huff_chunks : 0, 4);
  put(20, g.n_chunks, 4);
  put(24, g.rows, 8);
  put(32, g.tail_rows, 4);
  put(40, g.data_off, 8);
  put(48, tail_off, 8);
  put(56, total, 8);
  for (int k = 0; k < 64; ++k) h[k] = b[k];
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

template <int W>
__device__ void encode_chunk(const EncParams &p, uint8_t *mem, uint32_t c) {
  const Geom &g = p.g;
  const uint32_t D = g.D;
  const uint32_t wb = W / 8;
  const EncLayout L = enc_layout(g, p.stage_rows != 0);
  __shared__ uint32_t s_nrec;
  __shared__ uint32_t s_body;
  __shared__ uint64_t s_off;

  const uint64_t row0 = (uint64_t)c * g.chunk_rows;
  const uint64_t rows_c = min(g.chunk_rows, g.full_rows - row0);
  const uint32_t nb = (uint32_t)(rows_c / kBlockRows);
  const uint8_t *src_c = p.src + row0 * D * wb;

  uint8_t *width = mem + L.width;
  int32_t *alpha = reinterpret_cast<int32_t *>(mem + L.alpha);
  uint32_t *bsum = reinterpret_cast<uint32_t *>(mem + L.bsum);
  uint32_t *rec_first = reinterpret_cast<uint32_t *>(mem + L.rec_first);
  uint32_t *rec_run = reinterpret_cast<uint32_t *>(mem + L.rec_run);
  uint32_t *rec_off = reinterpret_cast<uint32_t *>(mem + L.rec_off);
  uint8_t *body = mem + L.body;

  // 1. rows
  const uint8_t *X = src_c;
  if (p.stage_rows) {
    cta_copy(mem + L.x, src_c, rows_c * D * wb);
    X = mem + L.x;
  }
  __syncthreads();

  // 2. FIRE per sample: alpha of every row, one thread per column
  // (Algorithm 3: alpha from the accumulator, then one gradient step).
  if (g.forecaster == kFcFireSample) {
    for (uint32_t j = threadIdx.x; j < D; j += blockDim.x) {
      int32_t acc = 0, dp = 0;
      uint32_t xp = 0;
      for (uint64_t r = 0; r < (uint64_t)nb * kBlockRows; ++r) {
        const int32_t a = acc >> g.learn_shift;
        alpha[r * D + j] = a;
        const uint32_t x = sample<W>(X, D, r, j);
        const int32_t e = sext<W>(x - xp - fire_pred_delta<W>(a, dp));
        acc = wrap_acc<W>((int32_t)((uint32_t)acc + (uint32_t)(sign_of(e) * dp)));
        dp = sext<W>(x - xp);
        xp = x;
      }
    }
    __syncthreads();
  }
  // 2. FIRE: alpha of every block, one thread per column.
  if (g.forecaster == kFcFire) {
    for (uint32_t j = threadIdx.x; j < D; j += blockDim.x) {
      int32_t acc = 0, dp = 0;
      uint32_t xp = 0;
      for (uint32_t b = 0; b < nb; ++b) {
        int32_t a = acc >> g.learn_shift;
        alpha[(uint64_t)b * D + j] = a;
        int32_t gsum = 0;
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          uint32_t x = sample<W>(X, D, (uint64_t)b * kBlockRows + i, j);
          if ((i & 1) == 0) {
            int32_t e = sext<W>(x - xp - fire_pred_delta<W>(a, dp));
            gsum += sign_of(e) * dp;
          }
          dp = sext<W>(x - xp);
          xp = x;
        }
        acc = wrap_acc<W>((int32_t)((uint32_t)acc + (uint32_t)(gsum >> 2)));
      }
    }
    __syncthreads();
  }

  // 3. widths of every (block, column)
  for (uint64_t q = threadIdx.x; q < (uint64_t)nb * D; q += blockDim.x) {
    uint32_t b = (uint32_t)(q / D), j = (uint32_t)(q % D);
    uint32_t o = 0;
#pragma unroll
    for (int i = 0; i < kBlockRows; ++i)
      o |= zigzag<W>(error_at<W>(X, D, (uint64_t)b * kBlockRows + i, j, g.forecaster,
                                 alpha_at(g, alpha, D, b, i, j)));
    uint32_t n = bit_len(o);
    width[q] = (uint8_t)(n == W - 1 ? W : n);
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
    uint32_t s = 0;
    for (uint32_t j = 0; j < D; ++j) s += width[(uint64_t)b * D + j];
    bsum[b] = s;
  }
  __syncthreads();

  // 4. records (runs of all-zero blocks and packed blocks) and their offsets
  if (threadIdx.x == 0) {
    uint32_t nrec = 0, run = 0, run_start = 0, pos = 0;
    auto emit = [&](uint32_t first, uint32_t runlen, uint32_t size) {
      if (nrec % g.G == 0) pos += g.hdr_bytes;
      rec_first[nrec] = first;
      rec_run[nrec] = runlen;
      rec_off[nrec] = pos;
      pos += size;
      nrec++;
    };
    for (uint32_t b = 0; b < nb; ++b) {
      uint32_t s = bsum[b];
      if (s == 0) {
        if (run == 0) run_start = b;
        if (++run == kMaxRun) {
          emit(run_start, run, 2);
          run = 0;
        }
        continue;
      }
      if (run) {
        emit(run_start, run, 2);
        run = 0;
      }
      emit(b, 0, g.col_major ? s : 8 * ((s + 7) / 8));
    }
    if (run) emit(run_start, run, 2);
    s_nrec = nrec;
    s_body = pos;
  }
  __syncthreads();
  const uint32_t nrec = s_nrec;
  const uint32_t body_bytes = s_body;

  // 5. pack: zero the body, then group headers and payloads (each work item
  //    owns whole bytes)
  for (uint32_t k = threadIdx.x; k < body_bytes; k += blockDim.x) body[k] = 0;
  __syncthreads();
  const uint32_t ngroups = (nrec + g.G - 1) / g.G;
  for (uint32_t q = threadIdx.x; q < ngroups; q += blockDim.x) {
    uint8_t *h = body + rec_off[q * g.G] - g.hdr_bytes;
    for (uint32_t s = 0; s < g.G; ++s) {
      uint32_t r = q * g.G + s;
      if (r >= nrec) break;
      if (rec_run[r]) continue;
      const uint8_t *wr = width + (uint64_t)rec_first[r] * D;
      for (uint32_t j = 0; j < D; ++j)
        or_bits(h, (uint64_t)(s * D + j) * g.hb, width_to_code(wr[j], W), g.hb);
    }
  }
  const uint32_t per = g.col_major ? D : kBlockRows;
  for (uint64_t q = threadIdx.x; q < (uint64_t)nrec * per; q += blockDim.x) {
    uint32_t r = (uint32_t)(q / per), k = (uint32_t)(q % per);
    uint8_t *out = body + rec_off[r];
    if (rec_run[r]) {
      if (k == 0) {
        out[0] = (uint8_t)rec_run[r];
        out[1] = (uint8_t)(rec_run[r] >> 8);
      }
      continue;
    }
    const uint32_t b = rec_first[r];
    const uint8_t *wr = width + (uint64_t)b * D;
    if (g.col_major) {
      // column k: its 8 values at bits i*n, exactly n bytes
      uint32_t off = 0;
      for (uint32_t j = 0; j < k; ++j) off += wr[j];
      uint32_t n = wr[k];
      if (!n) continue;
      uint64_t lo = 0, hi = 0;  // 128-bit little-endian bit buffer
      for (int i = 0; i < kBlockRows; ++i) {
        uint64_t z = zigzag<W>(error_at<W>(X, D, (uint64_t)b * kBlockRows + i, k, g.forecaster,
                                           alpha_at(g, alpha, D, b, i, k)));
        uint32_t bit = i * n;
        if (bit < 64) {
          lo |= z << bit;
          if (bit + n > 64) hi |= z >> (64 - bit);
        } else {
          hi |= z << (bit - 64);
        }
      }
      uint8_t *o = out + off;
      for (uint32_t t = 0; t < n; ++t) o[t] = (uint8_t)(t < 8 ? lo >> (8 * t) : hi >> (8 * (t - 8)));
    } else {
      // row k: columns at consecutive bit offsets, padded to R bytes
      uint32_t R = (bsum[b] + 7) / 8;
      uint8_t *o = out + (uint64_t)k * R;
      uint64_t acc = 0;
      uint32_t nacc = 0;
      const uint64_t row = (uint64_t)b * kBlockRows + k;
      for (uint32_t j = 0; j < D; ++j) {
        uint32_t n = wr[j];
        if (!n) continue;
        uint64_t z = zigzag<W>(error_at<W>(X, D, row, j, g.forecaster, alpha_at(g, alpha, D, b, k, j)));
        acc |= z << nacc;
        nacc += n;
        while (nacc >= 8) {
          *o++ = (uint8_t)acc;
          acc >>= 8;
          nacc -= 8;
        }
      }
      if (nacc) *o = (uint8_t)acc;
    }
  }
  __syncthreads();

  // 6. offset of this body: decoupled look-back over the preceding chunks
  if (threadIdx.x == 0) {
    uint64_t *lb = p.lookback;
    uint64_t prefix = 0;
    if (c == 0) {
      st_release_u64(&lb[0], kFlagPrefix | body_bytes);
    } else {
      st_release_u64(&lb[c], kFlagAggregate | body_bytes);
      int64_t k = (int64_t)c - 1;
      uint32_t spins = 0;
      while (k >= 0) {
        uint64_t v = ld_acquire_u64(&lb[k]);
        uint64_t flag = v & ~kValueMask;
        if (flag == 0) {
          if (++spins > (p.spin_limit ? p.spin_limit : kSpinLimit)) {
            set_status(p.status, SPRINTZ_ERR_TIMEOUT);
            break;
          }
          __nanosleep(64);
          continue;
        }
        prefix += v & kValueMask;
        if (flag == kFlagPrefix) break;
        --k;
      }
      st_release_u64(&lb[c], kFlagPrefix | (prefix + body_bytes));
    }
    s_off = prefix;
  }
  __syncthreads();
  const uint64_t off = s_off;

  // 7. body, chunk entry; the last chunk also writes tail, header and size
  uint64_t pos = g.data_off + off;
  if (pos + body_bytes <= p.dst_cap) {
    cta_copy_to_unaligned(p.dst + pos, body, body_bytes);
  } else if (threadIdx.x == 0) {
    set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
  }
  if (threadIdx.x < 16) {
    uint8_t *e = p.dst + kHdrBytes + (uint64_t)c * kEntryBytes;
    uint32_t t = threadIdx.x;
    uint64_t v = t < 8 ? off >> (8 * t) : (t < 12 ? (uint64_t)nrec >> (8 * (t - 8))
                                                  : (uint64_t)body_bytes >> (8 * (t - 12)));
    e[t] = (uint8_t)v;
  }
  if (c == g.n_chunks - 1) {
    const uint64_t tail_off = g.data_off + off + body_bytes;
    const uint64_t tail_bytes = g.tail_rows * D * wb;
    const uint64_t total = tail_off + tail_bytes;
    if (total <= p.dst_cap) {
      cta_copy(p.dst + tail_off, p.src + g.full_rows * D * wb, tail_bytes);
      if (threadIdx.x == 0) {
        write_stream_header(p.dst, g, tail_off, total);
        *p.out_size = total;
      }
    } else if (threadIdx.x == 0) {
      set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
    }
  }
  __syncthreads();
}

template <int W>
__global__ void __launch_bounds__(kEncThreads) k_encode(EncParams p) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_ticket;
  uint8_t *mem = p.stage_rows ? smem : p.scratch + (uint64_t)blockIdx.x * p.scratch_per_cta;
  for (;;) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(p.ticket, 1u);
    __syncthreads();
    const uint32_t c = s_ticket;
    __syncthreads();
    if (c >= p.g.n_chunks) break;
    encode_chunk<W>(p, mem, c);
  }
}

// Streams with no full block: header and raw tail only.
__global__ void k_encode_tail_only(EncParams p) {
  const Geom &g = p.g;
  const uint64_t tail_bytes = g.tail_rows * g.D * g.wb;
  const uint64_t total = g.data_off + tail_bytes;
  if (total > p.dst_cap) {
    if (threadIdx.x == 0) set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
    return;
  }
  cta_copy(p.dst + g.data_off, p.src, tail_bytes);
  if (threadIdx.x == 0) {
    write_stream_header(p.dst, g, g.data_off, total);
    *p.out_size = total;
  }
}

// ---------------------------------------------------------------------------
// Lane-per-column encoder (D <= 32)
//
// Persistent warps take groups of K = floor(32 / D) consecutive chunks from a
// ticket; lane k*D + j owns column j of chunk k.  Per group:
//   pass A  streams the rows block by block (a per-warp shared stage filled by
//           8-byte loads, one block of lookahead), runs the forecaster in
//           registers, takes every column's width and, with a segmented warp
//           scan, each block's size; the record logic of Algorithm 1 (runs of
//           all-zero blocks, groups of G headers) gives the body size;
//   look-back over chunk groups (bounded waits) gives the group's offset;
//   pass B  repeats the computation (its rows are still in L2: the grid is
//           sized so the groups in flight fit) and ORs header codes and
//           payload bits into a per-chunk shared ring addressed by absolute
//           output byte; completed 16-byte units are stored with one vector
//           store, only the bytes at the chunk's two ends with byte stores.
// ---------------------------------------------------------------------------

constexpr int kEncLaneThreads = 128;
constexpr int kEncLaneWarps = kEncLaneThreads / 32;
constexpr uint32_t kEncStage = 512;  // K * 8 rows * D * 2 bytes <= 512

struct EncLaneCfg {
  uint32_t window;  // ring bytes per chunk (power of two >= 64)
  uint32_t n_groups;
};

__host__ __device__ inline uint32_t enc_window_bytes(const Geom &g) {
  uint64_t maxpay = (uint64_t)g.D * g.w;  // bytes of a block at full width
  uint64_t need = 2ull * g.hdr_bytes + (uint64_t)(g.G + 1) * maxpay + 48;
  uint32_t wsz = 64;
  while (wsz < need) wsz <<= 1;
  return wsz;
}

// OR the low n (<= 16) bits of v into the ring at absolute bit position `abit`.
__device__ __forceinline__ void ring_or(uint32_t *ring, uint32_t ring_words, uint64_t abit,
                                        uint32_t v, uint32_t n) {
  if (!n || !v) return;
  const uint32_t wi = (uint32_t)(abit >> 5) & (ring_words - 1);
  const uint32_t sh = (uint32_t)abit & 31;
  atomicOr(&ring[wi], v << sh);
  if (sh + n > 32) atomicOr(&ring[(wi + 1) & (ring_words - 1)], v >> (32 - sh));
}

// Decoupled look-back over chunk groups with the whole warp: each lane reads
// one of the 32 nearest unread predecessors' words; the run of published
// aggregates up to the nearest inclusive prefix is summed at once.  The group
// publishes its aggregate first and its inclusive prefix last.  A published
// word carries its own value, so relaxed accesses suffice (acquire loads
// would invalidate the SM's L1 on every poll).  Polls back off exponentially
// and are bounded (SPRINTZ_ERR_TIMEOUT).  Returns the exclusive prefix in
// every lane.
__device__ uint64_t lookback_warp(uint64_t *lb, uint32_t grp, uint64_t total, int *status,
                                  uint32_t spin_limit) {
  const uint32_t limit = spin_limit ? spin_limit : kSpinLimit;
  const uint32_t lane = threadIdx.x & 31;
  if (grp == 0) {
    if (lane == 0) st_relaxed_u64(&lb[0], kFlagPrefix | total);
    return 0;
  }
  if (lane == 0) st_relaxed_u64(&lb[grp], kFlagAggregate | total);
  uint64_t prefix = 0;
  int64_t k = (int64_t)grp - 1;  // nearest predecessor not yet summed
  uint32_t spins = 0, ns = 64;
  while (true) {
    const int64_t idx = k - (int64_t)lane;
    const uint64_t w = idx >= 0 ? ld_relaxed_u64(&lb[idx]) : kFlagPrefix;  // before group 0: prefix 0
    const uint64_t flag = w & ~kValueMask;
    const uint32_t pend = __ballot_sync(0xFFFFFFFFu, flag == 0);
    const uint32_t pref = __ballot_sync(0xFFFFFFFFu, flag == kFlagPrefix);
    const uint32_t np = pref ? __ffs(pref) - 1 : 32u;  // lane of the nearest prefix
    const uint32_t nq = pend ? __ffs(pend) - 1 : 32u;  // lane of the nearest unpublished group
    const bool done = np < nq;
    const uint32_t take = done ? np + 1 : nq;
    uint64_t v = lane < take ? (w & kValueMask) : 0;
#pragma unroll
    for (uint32_t o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    prefix += v;
    if (done) break;
    k -= take;
    if (take == 0) {
      if (++spins > limit) {
        if (lane == 0) set_status(status, SPRINTZ_ERR_TIMEOUT);
        break;
      }
      __nanosleep(ns);
      ns = ns < 1024 ? ns * 2 : 1024;
    } else {
      ns = 64;
    }
  }
  if (lane == 0) st_relaxed_u64(&lb[grp], kFlagPrefix | (prefix + total));
  return prefix;
}

// Per-chunk state of one pass.
struct EncRun {
  uint32_t xp;   // x_{i-1}
  int32_t dp;    // delta_{i-1}
  int32_t acc;   // FIRE accumulator
  uint32_t run;  // blocks in the current zero run
  uint32_t nrec;
  uint64_t pos;  // body bytes laid out so far
  uint64_t hpos; // header of the open group
  bool open;     // a group is open (its header is incomplete)
  uint64_t flushed;  // body bytes already stored
};

template <int W, bool EMIT>
__device__ uint64_t encode_pass(const EncParams &p, const Geom &g, uint8_t *stage, uint32_t *ring,
                                uint32_t ring_words, bool live, uint32_t grp, uint32_t K,
                                uint32_t kk, uint32_t j, uint32_t lane, uint64_t row0, uint32_t nb,
                                uint64_t base /* absolute address of the body (EMIT) */,
                                uint32_t *nrec_out) {
  const uint32_t D = g.D;
  const uint32_t wb = W / 8;
  const uint32_t seg0 = lane - j;
  const uint32_t words_per = D * wb;  // 8-byte words of one chunk's block
  const uint32_t total_words = K * words_per;
  const uint32_t nb_max = (uint32_t)(min(g.chunk_rows, g.full_rows) / kBlockRows);
  EncRun st{};

  // which chunk, block word does each of this lane's (up to 2) stage words hold
  auto load_words = [&](uint32_t b, uint64_t *w) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const uint32_t q = lane + 32 * t;
      w[t] = 0;
      const uint32_t k2 = min(q / words_per, K - 1);
      const uint32_t lv = __shfl_sync(0xFFFFFFFFu, live ? nb : 0u, k2 * D);
      if (q < total_words && b < lv) {
        const uint64_t c2 = (uint64_t)grp * K + k2;
        const uint64_t r = c2 * g.chunk_rows + (uint64_t)b * kBlockRows;
        w[t] = __ldg(reinterpret_cast<const unsigned long long *>(p.src + r * D * wb) + (q % words_per));
      }
    }
  };

  uint64_t wcur[2], wnext[2];
  load_words(0, wcur);
  // L2 prefetch of the chunk's rows ahead (segment leader, pass A)
  const uintptr_t rows_lo = (uintptr_t)(p.src + row0 * D * wb);
  const uintptr_t rows_hi = rows_lo + (uint64_t)nb * kBlockRows * D * wb;
  uintptr_t pf = rows_lo;
  if (!EMIT && live && j == 0) {
    uintptr_t e2 = min(rows_hi, pf + 8192);
    prefetch_l2_range(pf, e2, rows_lo, rows_hi);
    pf = e2;
  }

  auto record = [&](bool is_run, uint32_t run_len, uint32_t total, uint32_t prefix, uint32_t n,
                    const uint32_t *z) {
    if (st.nrec % g.G == 0) {
      st.hpos = st.pos;
      st.pos += g.hdr_bytes;
      st.open = true;
    }
    const uint32_t s = st.nrec % g.G;
    uint32_t size;
    if (is_run) {
      size = 2;
      if (EMIT && j == 0) ring_or(ring, ring_words, ((uint64_t)base + st.pos) * 8, run_len, 16);
    } else {
      size = g.col_major ? total : 8 * ((total + 7) / 8);
      if (EMIT) {
        ring_or(ring, ring_words, ((uint64_t)base + st.hpos) * 8 + (uint64_t)(s * D + j) * g.hb,
                width_to_code(n, W), g.hb);
        if (n) {
          const uint64_t b0 = ((uint64_t)base + st.pos) * 8;
#pragma unroll
          for (int i = 0; i < kBlockRows; ++i) {
            const uint64_t bit = g.col_major ? b0 + (uint64_t)prefix * 8 + (uint64_t)i * n
                                             : b0 + (uint64_t)i * size + prefix;
            ring_or(ring, ring_words, bit, z[i], n);
          }
        }
      }
    }
    st.pos += size;
    st.nrec++;
    if (st.nrec % g.G == 0) st.open = false;
  };

  // store the completed 16-byte units of [flushed, limit) (absolute alignment);
  // units holding bytes outside [base, base + body) get byte stores
  auto flush = [&](uint64_t limit, bool final_) {
    const uint64_t a0 = base + st.flushed;
    const uint64_t a1 = final_ ? base + limit : ((base + limit) & ~15ull);
    if (a1 <= a0) return;
    const uint64_t u0 = a0 & ~15ull;
    const uint64_t nu = (a1 - u0 + 15) / 16;
    for (uint64_t u = j; u < nu; u += D) {
      const uint64_t ua = u0 + 16 * u;
      const uint32_t ri = (uint32_t)(ua >> 2) & (ring_words - 1);
      const uint4 v = *reinterpret_cast<const uint4 *>(&ring[ri]);
      if (ua >= base && ua + 16 <= a1) {
        *reinterpret_cast<uint4 *>(ua) = v;
      } else {
        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
        for (uint32_t k = 0; k < 16; ++k) {
          const uint64_t ab = ua + k;
          if (ab >= a0 && ab < a1) *reinterpret_cast<uint8_t *>(ab) = (uint8_t)(wv[k >> 2] >> (8 * (k & 3)));
        }
      }
      // a fully written unit is cleared for reuse; the last partial one keeps its bytes
      if (ua + 16 <= a1) *reinterpret_cast<uint4 *>(&ring[ri]) = make_uint4(0, 0, 0, 0);
    }
    st.flushed = (a1 & ~15ull) > base ? (a1 & ~15ull) - base : st.flushed;
    if (final_) st.flushed = limit;
  };

  for (uint32_t b = 0; b < nb_max; ++b) {
    // stage this block, start loading the next one
#pragma unroll
    for (int t = 0; t < 2; ++t)
      if (lane + 32 * t < total_words) reinterpret_cast<uint64_t *>(stage)[lane + 32 * t] = wcur[t];
    if (b + 1 < nb_max) load_words(b + 1, wnext);
    __syncwarp();
    const bool here = live && b < nb;
    uint32_t z[kBlockRows];
    uint32_t n = 0;
    if (here) {
      uint32_t x[kBlockRows];
#pragma unroll
      for (int i = 0; i < kBlockRows; ++i)
        x[i] = load_sample<W>(stage + kk * (kBlockRows * D * wb) + (i * D + j) * wb);
      uint32_t orz = 0;
      if (g.forecaster == kFcDelta) {
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          z[i] = zigzag<W>(sext<W>(x[i] - st.xp));
          st.xp = x[i];
          orz |= z[i];
        }
      } else if (g.forecaster == kFcDDelta) {
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          z[i] = zigzag<W>(sext<W>(x[i] - st.xp - (uint32_t)st.dp));
          orz |= z[i];
          st.dp = sext<W>(x[i] - st.xp);
          st.xp = x[i];
        }
      } else if (g.forecaster == kFcFireSample) {
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          const int32_t e = sext<W>(x[i] - st.xp - fire_pred_delta<W>(st.acc >> g.learn_shift, st.dp));
          st.acc = wrap_acc<W>((int32_t)((uint32_t)st.acc + (uint32_t)(sign_of(e) * st.dp)));
          z[i] = zigzag<W>(e);
          orz |= z[i];
          st.dp = sext<W>(x[i] - st.xp);
          st.xp = x[i];
        }
      } else {
        const int32_t a = st.acc >> g.learn_shift;
        int32_t gsum = 0;
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          const int32_t e = sext<W>(x[i] - st.xp - fire_pred_delta<W>(a, st.dp));
          if ((i & 1) == 0) gsum += sign_of(e) * st.dp;
          z[i] = zigzag<W>(e);
          orz |= z[i];
          st.dp = sext<W>(x[i] - st.xp);
          st.xp = x[i];
        }
        st.acc = wrap_acc<W>((int32_t)((uint32_t)st.acc + (uint32_t)(gsum >> 2)));
      }
      n = bit_len(orz);
      if (n == W - 1) n = W;
    }
    // segmented scan of the widths: this lane's offset and the block's total
    uint32_t v = n;
    for (uint32_t o = 1; o < D; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (j >= o) v += t;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, v, seg0 + D - 1);
    const uint32_t prefix = v - n;
    if (here) {
      if (total == 0) {
        if (++st.run == kMaxRun) {
          record(true, st.run, 0, 0, 0, z);
          st.run = 0;
        }
      } else {
        if (st.run) {
          record(true, st.run, 0, 0, 0, z);
          st.run = 0;
        }
        record(false, 0, total, prefix, n, z);
      }
      if (!EMIT && j == 0 && pf < rows_hi && rows_lo + (uint64_t)(b + 1) * kBlockRows * D * wb + 4096 > pf) {
        uintptr_t e2 = min(rows_hi, pf + 4096);
        prefetch_l2_range(pf, e2, rows_lo, rows_hi);
        pf = e2;
      }
    }
    if (EMIT) {
      __syncwarp();
      if (here) flush(st.open ? st.hpos : st.pos, false);
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 2; ++t) wcur[t] = wnext[t];
  }
  if (live) {
    if (st.run) record(true, st.run, 0, 0, 0, nullptr);
    st.open = false;
  }
  if (EMIT) {
    __syncwarp();
    if (live) flush(st.pos, true);
    __syncwarp();
  }
  *nrec_out = st.nrec;
  return st.pos;
}

template <int W>
__global__ void __launch_bounds__(kEncLaneThreads) k_encode_lanes(EncParams p, EncLaneCfg cfg) {
  extern __shared__ __align__(16) uint8_t smem[];
  const Geom &g = p.g;
  const uint32_t D = g.D;
  const uint32_t K = 32 / D;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t kk = lane / D, j = lane % D;
  const uint32_t seg0 = lane - j;
  uint8_t *stage = smem + warp * kEncStage;
  const uint32_t ring_words = cfg.window / 4;
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem + kEncLaneWarps * kEncStage +
                                                ((uint64_t)warp * K + min(kk, K - 1)) * cfg.window);
  const uint32_t wb = W / 8;

  for (;;) {
    uint32_t grp = 0;
    if (lane == 0) grp = atomicAdd(p.ticket, 1u);
    grp = __shfl_sync(0xFFFFFFFFu, grp, 0);
    if (grp >= cfg.n_groups) break;
    const uint64_t c64 = (uint64_t)grp * K + kk;
    const bool live = kk < K && c64 < g.n_chunks;
    const uint32_t c = (uint32_t)c64;
    const uint64_t row0 = c64 * g.chunk_rows;
    const uint32_t nb = live ? (uint32_t)(min(g.chunk_rows, g.full_rows - row0) / kBlockRows) : 0u;

    // pass A: body sizes
    uint32_t nrec = 0;
    const uint64_t S = encode_pass<W, false>(p, g, stage, ring, ring_words, live, grp, K, kk, j,
                                             lane, row0, nb, 0, &nrec);
    // this group's total and each chunk's offset inside it
    uint64_t v = (live && j == 0) ? S : 0;
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane >= o) v += t;
    }
    const uint64_t group_total = __shfl_sync(0xFFFFFFFFu, v, 31);
    const uint64_t excl = __shfl_sync(0xFFFFFFFFu, v, seg0) - __shfl_sync(0xFFFFFFFFu, (live && j == 0) ? S : 0ull, seg0);
    // look-back over groups
    const uint64_t prefix = lookback_warp(p.lookback, grp, group_total, p.status, p.spin_limit);
    const uint64_t off = prefix + excl;

    // pass B: the body at its place
    const uint64_t base = (uint64_t)(uintptr_t)(p.dst + g.data_off + off);
    if (live) {
      // clear this chunk's ring
      for (uint32_t t = j; t < ring_words / 4; t += D)
        reinterpret_cast<uint4 *>(ring)[t] = make_uint4(0, 0, 0, 0);
    }
    __syncwarp();
    const bool fits = g.data_off + prefix + group_total <= p.dst_cap;
    if (!fits && lane == 0) set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
    uint32_t nrec_b = 0;
    encode_pass<W, true>(p, g, stage, ring, ring_words, live && fits, grp, K, kk, j, lane, row0, nb,
                         base, &nrec_b);
    if (live && j == 0 && fits) {
      // chunk entry: body offset, record count, packed bytes (little-endian)
      uint8_t *e = p.dst + kHdrBytes + (uint64_t)c * kEntryBytes;
      const uint64_t w1 = (uint64_t)nrec | ((uint64_t)S << 32);
      for (int k = 0; k < 8; ++k) {
        e[k] = (uint8_t)(off >> (8 * k));
        e[8 + k] = (uint8_t)(w1 >> (8 * k));
      }
    }
    __syncwarp();
    if (c == g.n_chunks - 1 && live) {
      const uint64_t tail_off = g.data_off + off + S;
      const uint64_t tail_bytes = g.tail_rows * D * wb;
      const uint64_t total = tail_off + tail_bytes;
      if (total <= p.dst_cap) {
        for (uint64_t k = j; k < tail_bytes; k += D) p.dst[tail_off + k] = p.src[g.full_rows * D * wb + k];
        if (j == 0) {
          write_stream_header(p.dst, g, tail_off, total);
          *p.out_size = total;
        }
      } else if (j == 0) {
        set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Single-pass lane encoder (D <= 32): bodies assembled in private slots
//
// As the two-pass encoder, but each warp owns K body slots in the workspace
// (one per chunk it encodes).  One pass over the rows lays out the records
// and ORs header codes and payload bits into a per-chunk shared ring, whose
// completed 16-byte units go to the slot with one vector store each.  When
// the chunk ends its size is known: the look-back over chunk groups gives its
// offset and the chunk's lanes copy the slot to its place in the stream
// (16-byte stores, bytes only at the two unaligned ends).  Slots are reused
// by the same warp, so they stay in L2.
// ---------------------------------------------------------------------------

// Appends bit fields to the chunk's shared ring from bit position `bit` on:
// whole 32-bit words are OR-ed in as they fill, so one lane touches each
// word once (the first and last words may be shared with other writers).
struct BitSink {
  uint32_t *ring;
  uint32_t wmask, w, lo, fill;
  __device__ __forceinline__ BitSink(uint32_t *r, uint32_t wm, uint32_t bit)
      : ring(r), wmask(wm), w((bit >> 5) & wm), lo(0), fill(bit & 31) {}
  // v < 2^n, n <= 32
  __device__ __forceinline__ void put(uint32_t v, uint32_t n) {
    const uint32_t f = fill;
    lo |= v << f;
    fill = f + n;
    if (fill >= 32) {
      if (lo) atomicOr(&ring[w], lo);
      w = (w + 1) & wmask;
      lo = __funnelshift_l(v, 0u, f);  // the bits of v past the word
      fill -= 32;
    }
  }
  __device__ __forceinline__ void finish() {
    if (lo) atomicOr(&ring[w], lo);
  }
};

// Transposition tile of the row-major packer: per chunk, 8 rows of D entries
// (zigzagged error | width << 16).  A row takes an odd number of 16-byte
// units, so that the row owners' 16-byte loads of a quarter warp fall into
// distinct banks; chunks start D * 4 bytes apart modulo 128, so that the
// column owners' stores of one row do too.
__host__ __device__ inline uint32_t enc_tile_row(uint32_t D) { return (((D * 4 + 15) / 16) | 1u) * 16; }
__host__ __device__ inline uint32_t enc_tile_stride(uint32_t D) {
  const uint32_t t = kBlockRows * enc_tile_row(D);
  return t + ((((D * 4) - t) & 127u) + 15u & ~15u);
}
__host__ __device__ inline uint32_t enc_stage_bytes(uint32_t D, uint32_t wb) {
  return ((32 / D) * blk_stage_stride(D, wb) + 15) & ~15u;
}
// The tile exists only for row-major packing.
__host__ __device__ inline uint32_t enc_tile_bytes(const Geom &g) {
  return g.col_major ? 0u : enc_tile_stride(g.D);
}
__host__ __device__ inline uint32_t enc_slot_region(const Geom &g, uint32_t window) {
  const uint32_t K = 32 / g.D;
  return enc_stage_bytes(g.D, g.wb) + K * enc_tile_bytes(g) + K * window;
}

struct EncSlotCfg {
  uint32_t window;       // ring bytes per chunk (power of two)
  uint32_t n_groups;
  uint32_t slot_stride;  // bytes per chunk slot (multiple of 32, >= the largest body + 32)
  uint32_t pf_bytes;     // L2 bulk prefetch of the chunk's rows, this far ahead (0: none)
  uint8_t *slots;        // [warp][K] slots
};

// Encode chunk group `grp` of one stream with one warp: wsm is the warp's
// shared region (stage, then K rings), wslots its K body slots.
// cfg.pf_bytes > 0 prefetches the chunks' rows into L2 ahead of the reads
// (the batched kernel, whose streams are short, can gain; the single-stream
// kernel, whose one wave of warps covers the whole input, loses: its windows
// evict each other).
template <int W, int DT>
__device__ __forceinline__ void encode_group_slots(const EncParams &p, const EncSlotCfg &cfg, uint32_t grp,
                                                   uint8_t *wsm, uint8_t *wslots) {
  const Geom &g = p.g;
  const uint32_t D = DT ? (uint32_t)DT : g.D;  // a compile-time constant for common D
  const uint32_t K = 32 / D;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t kk = lane / D, j = lane % D;
  const uint32_t kc = kk < K ? kk : K - 1;
  const uint32_t seg0 = lane - j, last = seg0 + D - 1;
  const uint32_t wb = W / 8;
  const uint32_t G = g.G, hb = g.hb, H = g.hdr_bytes;
  (void)warp;
  uint8_t *stage = wsm;
  const uint32_t tile_stride = enc_tile_bytes(g), tile_rw = enc_tile_row(D) / 4;
  const uint32_t st_stride = blk_stage_stride(D, wb), st_bytes = enc_stage_bytes(D, wb);
  uint32_t *tile = reinterpret_cast<uint32_t *>(wsm + st_bytes + kc * tile_stride);
  uint32_t *ring = reinterpret_cast<uint32_t *>(wsm + st_bytes + K * tile_stride + (uint64_t)kc * cfg.window);
  const uint32_t ring_wmask = cfg.window / 4 - 1, ring_bitmask = cfg.window * 8 - 1;
  const uint32_t seg_mask = D == 32 ? 0xFFFFFFFFu : ((1u << D) - 1u) << seg0;
  // the chunk's header codes fit one word and combine by butterfly shuffles
  constexpr uint32_t HB = W == 8 ? 3u : 4u;
  constexpr bool kHdrShfl = DT >= 2 && (DT & (DT - 1)) == 0 && DT * HB <= 32;
  const bool colmaj = DT ? (DT * W <= 32) : (g.col_major != 0);
  uint8_t *slot = wslots + (uint64_t)kc * cfg.slot_stride;
  // L2 policies: the rows stream through (evict first); the body slot is
  // written now and read back at the chunk's end (evict last); the stream
  // itself is written once (evict first)
  const uint64_t pol_stream = l2_policy_evict_first(), pol_slot = l2_policy_evict_last();

  // cooperative stage loads: this lane's (up to two) 8-byte words of a block step
  const uint32_t words_per = D * wb, total_words = K * words_per;
  bool has[2];
  uint32_t k2[2], wq[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const uint32_t q = lane + 32 * t;
    has[t] = q < total_words;
    k2[t] = has[t] ? q / words_per : 0;
    wq[t] = has[t] ? q % words_per : 0;
  }
  const uint32_t row_stride = D * wb;
  const uint8_t *my_x = stage + kc * st_stride + j * wb;
  uint32_t st_word[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) st_word[t] = k2[t] * (st_stride / 8) + wq[t];
  const uint32_t nb_max = (uint32_t)(min(g.chunk_rows, g.full_rows) / kBlockRows);

  {
    const uint64_t c64 = (uint64_t)grp * K + kk;
    const bool live = kk < K && c64 < g.n_chunks;
    const uint64_t row0 = c64 * g.chunk_rows;
    const uint32_t nb = live ? (uint32_t)(min(g.chunk_rows, g.full_rows - row0) / kBlockRows) : 0u;
    const unsigned long long *srcw[2];
    uint32_t nbw[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      nbw[t] = __shfl_sync(0xFFFFFFFFu, nb, k2[t] * D);
      const uint64_t c2 = (uint64_t)grp * K + k2[t];
      srcw[t] = reinterpret_cast<const unsigned long long *>(p.src + c2 * g.chunk_rows * D * wb) + wq[t];
    }
    const uintptr_t rows_lo = (uintptr_t)(p.src + row0 * D * wb);
    const uintptr_t rows_hi = rows_lo + (uint64_t)nb * kBlockRows * D * wb;
    uintptr_t pf = rows_lo;
    const uint32_t pfb = cfg.pf_bytes;
    if (pfb && live && j == 0) {
      const uintptr_t e2 = min(rows_hi, pf + 2 * pfb);
      prefetch_l2_range(pf, e2, rows_lo, rows_hi);
      pf = e2;
    }
    if (live)
      for (uint32_t t = j; t < cfg.window / 16; t += D)
        reinterpret_cast<uint4 *>(ring)[t] = make_uint4(0, 0, 0, 0);

    uint32_t xp = 0, run = 0, nrec = 0, gs = 0, pos = 0, hpos = 0, flushed = 0;
    int32_t dp = 0, acc = 0;
    bool open = false;

    auto ror = [&](uint32_t bit, uint32_t v, uint32_t n) {
      if (!v) return;
      const uint32_t q = bit & ring_bitmask;
      const uint32_t wi = q >> 5, sh = q & 31;
      atomicOr(&ring[wi], v << sh);
      if (sh + n > 32) atomicOr(&ring[(wi + 1) & ring_wmask], v >> (32 - sh));
    };
    auto start_record = [&]() {
      if (gs == 0) {
        hpos = pos;
        pos += H;
        open = true;
      }
    };
    auto end_record = [&](uint32_t size) {
      pos += size;
      nrec++;
      if (++gs == G) {
        gs = 0;
        open = false;
      }
    };
    auto emit_run = [&](uint32_t len) {
      start_record();
      if (j == 0) ror(pos * 8, len, 16);
      end_record(2);
    };
    // completed bytes to the slot in whole 32-byte sectors (the last partial
    // 16-byte unit at the end of the chunk)
    auto flush = [&](uint32_t limit, bool fin) {
      const uint32_t u1 = fin ? (limit + 15) >> 4 : (limit >> 5) << 1;
      for (uint32_t u = (flushed >> 4) + j; u < u1; u += D) {
        uint4 *r4 = reinterpret_cast<uint4 *>(&ring[(u * 4) & ring_wmask]);
        st_v4_hint(slot + 16ull * u, *r4, pol_slot);
        *r4 = make_uint4(0, 0, 0, 0);
      }
      if (u1 * 16 > flushed) flushed = u1 * 16;
    };

    unsigned long long wcur[2], wnext[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) wcur[t] = (has[t] && nbw[t] > 0) ? ldg_u64_hint(srcw[t], pol_stream) : 0ull;
    __syncwarp();
    for (uint32_t b = 0; b < nb_max; ++b) {
#pragma unroll
      for (int t = 0; t < 2; ++t)
        if (has[t]) reinterpret_cast<unsigned long long *>(stage)[st_word[t]] = wcur[t];
#pragma unroll
      for (int t = 0; t < 2; ++t)
        wnext[t] = (has[t] && b + 1 < nbw[t]) ? ldg_u64_hint(srcw[t] + (uint64_t)(b + 1) * words_per, pol_stream)
                                              : 0ull;
      __syncwarp();
      const bool here = live && b < nb;
      uint32_t z[kBlockRows];
      uint32_t n = 0;
      if (here) {
        uint32_t x[kBlockRows];
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i)
          x[i] = W == 8 ? (uint32_t)my_x[i * row_stride]
                        : (uint32_t) * reinterpret_cast<const uint16_t *>(my_x + i * row_stride);
        uint32_t orz = 0;
        if (g.forecaster == kFcDelta) {
#pragma unroll
          for (int i = 0; i < kBlockRows; ++i) {
            z[i] = zigzag<W>(sext<W>(x[i] - xp));
            xp = x[i];
            orz |= z[i];
          }
        } else if (g.forecaster == kFcDDelta) {
          // double delta: predict x_{i-1} + delta_{i-1}
#pragma unroll
          for (int i = 0; i < kBlockRows; ++i) {
            z[i] = zigzag<W>(sext<W>(x[i] - xp - (uint32_t)dp));
            orz |= z[i];
            dp = sext<W>(x[i] - xp);
            xp = x[i];
          }
        } else if (g.forecaster == kFcFireSample) {
          // Algorithm 3 at every sample: alpha = acc >> shift, then
          // acc += sign(e) * delta_{i-1}
#pragma unroll
          for (int i = 0; i < kBlockRows; ++i) {
            const int32_t e = sext<W>(x[i] - xp - fire_pred_delta<W>(acc >> g.learn_shift, dp));
            acc = wrap_acc<W>((int32_t)((uint32_t)acc + (uint32_t)(sign_of(e) * dp)));
            z[i] = zigzag<W>(e);
            orz |= z[i];
            dp = sext<W>(x[i] - xp);
            xp = x[i];
          }
        } else {
          const int32_t a = acc >> g.learn_shift;
          int32_t gsum = 0;
#pragma unroll
          for (int i = 0; i < kBlockRows; ++i) {
            const int32_t e = sext<W>(x[i] - xp - fire_pred_delta<W>(a, dp));
            if ((i & 1) == 0) gsum += e == 0 ? 0 : (e > 0 ? dp : -dp);
            z[i] = zigzag<W>(e);
            orz |= z[i];
            dp = sext<W>(x[i] - xp);
            xp = x[i];
          }
          acc = wrap_acc<W>((int32_t)((uint32_t)acc + (uint32_t)(gsum >> 2)));
        }
        n = 32u - __clz(orz);
        if (n == W - 1) n = W;
      }
      // segmented scan of the widths: this lane's offset and the block's total
      uint32_t v = n;
#pragma unroll
      for (uint32_t o = 1; o < 32; o <<= 1) {
        if (o < D) {
          const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
          if (j >= o) v += t;
        }
      }
      const uint32_t total = __shfl_sync(0xFFFFFFFFu, v, last);
      if (DT != 0 && here && !colmaj) {
        const uint32_t nh = n << 16;
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) tile[i * tile_rw + j] = z[i] | nh;
      }
      __syncwarp();
      if (here) {
        if (total == 0) {
          if (++run == kMaxRun) {
            emit_run(run);
            run = 0;
          }
        } else {
          if (run) {
            emit_run(run);
            run = 0;
          }
          start_record();
          const uint32_t prefix = v - n;
          const uint32_t size = colmaj ? total : (total + 7) & ~7u;
          const uint32_t code = n == W ? W - 1 : n;
          if (kHdrShfl) {
            uint32_t hv = code << (j * HB);
#pragma unroll
            for (uint32_t o = 1; o < (DT ? (uint32_t)DT : 1u); o <<= 1) hv |= __shfl_xor_sync(seg_mask, hv, o);
            // lane 0 ORs the low part into the first word, lane 1 the rest into the next
            if (j < 2) {
              const uint32_t hbit = hpos * 8 + gs * D * HB, sh = hbit & 31;
              const uint32_t hw = j == 0 ? hv << sh : __funnelshift_l(hv, 0u, sh);
              if (hw) atomicOr(&ring[((hbit >> 5) + j) & ring_wmask], hw);
            }
          } else {
            ror(hpos * 8 + (gs * D + j) * hb, code, hb);
          }
          if (colmaj) {
            // column j: its 8 values of n bits, contiguous from byte pos + prefix
            if (n) {
              BitSink bs(ring, ring_wmask, (pos + prefix) * 8);
#pragma unroll
              for (int i = 0; i < kBlockRows; ++i) bs.put(z[i], n);
              bs.finish();
            }
          } else if (DT == 0) {
            // any column count (the batched kernel): each lane ORs its 8
            // fields into the ring, rows size bits apart
            if (n) {
              const uint32_t b0 = pos * 8 + prefix;
#pragma unroll
              for (int i = 0; i < kBlockRows; ++i) ror(b0 + i * size, z[i], n);
            }
          } else {
            // rows j, j + D, ...: each the concatenation of its D fields
            // (size bits per row), read from the tile 4 entries at a time and
            // appended two columns at a time
            for (uint32_t i = j; i < kBlockRows; i += D) {
              const uint4 *row = reinterpret_cast<const uint4 *>(tile + i * tile_rw);
              BitSink bs(ring, ring_wmask, pos * 8 + i * size);
#pragma unroll
              for (uint32_t c4 = 0; c4 < (D + 3) / 4; ++c4) {
                const uint4 q = row[c4];
                const uint32_t e[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (uint32_t h = 0; h < 4; h += 2) {
                  const uint32_t c = c4 * 4 + h;
                  if (c < D) {
                    const uint32_t n0 = e[h] >> 16, v0 = e[h] & 0xFFFFu;
                    if (c + 1 < D) {
                      const uint32_t n1 = e[h + 1] >> 16, v1 = e[h + 1] & 0xFFFFu;
                      bs.put(v0 | (v1 << n0), n0 + n1);
                    } else {
                      bs.put(v0, n0);
                    }
                  }
                }
              }
              bs.finish();
            }
          }
          end_record(size);
        }
        if (pfb && j == 0 && pf < rows_hi && rows_lo + (uint64_t)(b + 1) * kBlockRows * D * wb + pfb > pf) {
          const uintptr_t e2 = min(rows_hi, pf + pfb);
          prefetch_l2_range(pf, e2, rows_lo, rows_hi);
          pf = e2;
        }
      }
      __syncwarp();
      if (here) flush(open ? hpos : pos, false);
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 2; ++t) wcur[t] = wnext[t];
    }
    if (live) {
      if (run) emit_run(run);
      open = false;
    }
    __syncwarp();
    if (live) flush(pos, true);
    __syncwarp();
    const uint32_t S = pos;

    // offsets: this group's total, each chunk's place inside it, look-back
    uint64_t v = (live && j == 0) ? S : 0;
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane >= o) v += t;
    }
    const uint64_t group_total = __shfl_sync(0xFFFFFFFFu, v, 31);
    const uint64_t excl = __shfl_sync(0xFFFFFFFFu, v, seg0) - __shfl_sync(0xFFFFFFFFu, (uint64_t)S, seg0);
    const uint64_t prefix = lookback_warp(p.lookback, grp, group_total, p.status, p.spin_limit);
    const uint64_t off = prefix + excl;

    // the body to its place: bytes up to a 16-byte boundary, 16-byte units
    // assembled from the slot's words, bytes after the last unit
    if (live && g.data_off + off + S <= p.dst_cap) {
      uint8_t *d = p.dst + g.data_off + off;
      const uint32_t head = min((uint32_t)((16 - ((uintptr_t)d & 15)) & 15), S);
      for (uint32_t k = j; k < head; k += D) d[k] = slot[k];
      const uint32_t n16 = (S - head) / 16;
      // output unit u is slot bytes [head + 16u, +16): the tail of slot unit u
      // and the head of unit u + 1 (both inside the slot's 16 spare bytes)
      const uint32_t sh = (head & 3) * 8;
      const bool w1 = head & 4, w2 = head & 8;
      const uint4 *s4 = reinterpret_cast<const uint4 *>(slot);
      for (uint32_t u0 = j; u0 < n16; u0 += 2 * D) {
        uint4 A[2], B[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const uint32_t u = u0 + t * D;
          if (u < n16) {
            A[t] = ld_v4_hint(s4 + u, pol_stream);
            B[t] = ld_v4_hint(s4 + u + 1, pol_stream);
          }
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const uint32_t u = u0 + t * D;
          if (u < n16) {
            // words head/4 .. head/4 + 4 of the pair
            const uint32_t p0 = w2 ? A[t].z : A[t].x, p1 = w2 ? A[t].w : A[t].y;
            const uint32_t p2 = w2 ? B[t].x : A[t].z, p3 = w2 ? B[t].y : A[t].w;
            const uint32_t p4 = w2 ? B[t].z : B[t].x, p5 = w2 ? B[t].w : B[t].y;
            const uint32_t a0 = w1 ? p1 : p0, a1 = w1 ? p2 : p1, a2 = w1 ? p3 : p2;
            const uint32_t a3 = w1 ? p4 : p3, a4 = w1 ? p5 : p4;
            uint4 o;
            o.x = __funnelshift_r(a0, a1, sh);
            o.y = __funnelshift_r(a1, a2, sh);
            o.z = __funnelshift_r(a2, a3, sh);
            o.w = __funnelshift_r(a3, a4, sh);
            st_v4_hint(d + head + 16 * u, o, pol_stream);
          }
        }
      }
      for (uint32_t k = head + 16 * n16 + j; k < S; k += D) d[k] = slot[k];
      if (j == 0) {
        uint8_t *e = p.dst + kHdrBytes + c64 * kEntryBytes;
        const uint64_t w1 = (uint64_t)nrec | ((uint64_t)S << 32);
        for (int k = 0; k < 8; ++k) {
          e[k] = (uint8_t)(off >> (8 * k));
          e[8 + k] = (uint8_t)(w1 >> (8 * k));
        }
      }
      if (c64 == g.n_chunks - 1) {
        const uint64_t tail_off = g.data_off + off + S;
        const uint64_t tail_bytes = g.tail_rows * D * wb;
        const uint64_t tot = tail_off + tail_bytes;
        if (tot <= p.dst_cap) {
          for (uint64_t k = j; k < tail_bytes; k += D) p.dst[tail_off + k] = p.src[g.full_rows * D * wb + k];
          if (j == 0) {
            write_stream_header(p.dst, g, tail_off, tot);
            *p.out_size = tot;
          }
        } else if (j == 0) {
          set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
        }
      }
    } else if (live && j == 0) {
      set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
    }
    __syncwarp();
  }
}

template <int W, int DT>
__global__ void __launch_bounds__(kEncLaneThreads, 7) k_encode_slots(EncParams p, EncSlotCfg cfg) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t K = 32 / p.g.D;
  const uint32_t region = enc_slot_region(p.g, cfg.window);
  uint8_t *wsm = smem + (uint64_t)warp * region;
  const uint64_t gwarp = (uint64_t)blockIdx.x * kEncLaneWarps + warp;
  uint8_t *wslots = cfg.slots + gwarp * K * (uint64_t)cfg.slot_stride;
  for (;;) {
    uint32_t grp = 0;
    if (lane == 0) grp = atomicAdd(p.ticket, 1u);
    grp = __shfl_sync(0xFFFFFFFFu, grp, 0);
    if (grp >= cfg.n_groups) break;
    encode_group_slots<W, DT>(p, cfg, grp, wsm, wslots);
  }
}

// The slot encoder specialised for the column count (0: any D <= 32).
template <int W>
static const void *slot_encoder(uint32_t D) {
  switch (D) {
    case 1: return (const void *)k_encode_slots<W, 1>;
    case 2: return (const void *)k_encode_slots<W, 2>;
    case 3: return (const void *)k_encode_slots<W, 3>;
    case 4: return (const void *)k_encode_slots<W, 4>;
    case 8: return (const void *)k_encode_slots<W, 8>;
    case 16: return (const void *)k_encode_slots<W, 16>;
    default: return (const void *)k_encode_slots<W, 0>;
  }
}

// One stream of a batched encode.
struct EncBatchItem {
  EncParams p;    // its own look-back words, destination and size word
  EncSlotCfg cfg;
};
static_assert(sizeof(EncBatchItem) % 8 == 0, "descriptors are copied in 8-byte words");

// One chunk group of a batch item, through the slot encoder specialised for
// the item's column count (a call per group keeps each variant's code apart).
// The warp's region arrives as an offset into the dynamic shared memory, so
// that the callee addresses it as shared memory (32-bit addresses, shared
// atomics) rather than through generic pointers.
template <int W, int DT>
__device__ __noinline__ void encode_batch_group(const EncBatchItem &it, uint32_t grp, uint32_t wsm_off,
                                                uint8_t *wslots) {
  extern __shared__ __align__(16) uint8_t smem[];
  encode_group_slots<W, DT>(it.p, it.cfg, grp, smem + wsm_off, wslots);
}

// Variant table: [w == 16][D] (D = 0: any column count up to 32).  One
// indirect call site for every variant keeps the kernel's frame small.
typedef void (*EncBatchGroupFn)(const EncBatchItem &, uint32_t, uint32_t, uint8_t *);
#define SPZ_ENC_ROW(W)                                                                                  \
  {encode_batch_group<W, 0>,  encode_batch_group<W, 1>,  encode_batch_group<W, 2>,                      \
   encode_batch_group<W, 3>,  encode_batch_group<W, 4>,  encode_batch_group<W, 5>,                      \
   encode_batch_group<W, 6>,  encode_batch_group<W, 7>,  encode_batch_group<W, 8>,                      \
   encode_batch_group<W, 9>,  encode_batch_group<W, 10>, encode_batch_group<W, 11>,                     \
   encode_batch_group<W, 12>, encode_batch_group<W, 13>, encode_batch_group<W, 14>,                     \
   encode_batch_group<W, 15>, encode_batch_group<W, 16>}
__device__ EncBatchGroupFn g_enc_batch_fns[2][17] = {SPZ_ENC_ROW(8), SPZ_ENC_ROW(16)};
#undef SPZ_ENC_ROW

// Batched encode: persistent warps take work entries (stream, chunk group),
// one ticket per (w, D) class, from their SM's home class first.  Every
// stream's groups are in increasing order inside their class's list, so a
// group's look-back only waits on earlier groups of its own stream, all of
// which were taken earlier and are running or done.  Each warp copies its
// item's descriptor into shared memory once per group.
__global__ void __launch_bounds__(kEncLaneThreads, 7) k_encode_batch(const EncBatchItem *items,
                                                                    const BatchClasses *classes,
                                                                    const uint64_t *work, uint32_t *tickets,
                                                                    uint32_t region, uint8_t *slots,
                                                                    uint64_t slot_region) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ __align__(16) EncBatchItem s_it[kEncLaneWarps];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wsm_off = warp * region;
  const uint64_t gwarp = (uint64_t)blockIdx.x * kEncLaneWarps + warp;
  uint8_t *wslots = slots + gwarp * slot_region;
  constexpr uint32_t kWords = sizeof(EncBatchItem) / 8;
  uint32_t c = batch_home(classes);
  uint64_t e = 0;
  while (batch_next(classes, work, tickets, c, &e)) {
    const uint32_t s = (uint32_t)(e >> kWorkGroupBits);
    const uint32_t grp = (uint32_t)(e & ((1ull << kWorkGroupBits) - 1));
    const uint64_t *from = reinterpret_cast<const uint64_t *>(items + s);
    uint64_t *to = reinterpret_cast<uint64_t *>(&s_it[warp]);
    for (uint32_t k = lane; k < kWords; k += 32) to[k] = __ldg(from + k);
    __syncwarp();
    const EncBatchItem &it = s_it[warp];
    const uint32_t D = it.p.g.D;
    g_enc_batch_fns[it.p.g.w == 16][D <= 16 ? D : 0](it, grp, wsm_off, wslots);
    __syncwarp();
  }
}

// Streams of a batch without a full block: header and raw tail only.
__global__ void k_encode_batch_tails(const EncBatchItem *items) {
  const EncParams &p = items[blockIdx.x].p;
  const Geom &g = p.g;
  if (g.n_chunks != 0) return;
  const uint64_t tail_bytes = g.tail_rows * g.D * g.wb;
  const uint64_t total = g.data_off + tail_bytes;
  if (total > p.dst_cap) {
    if (threadIdx.x == 0) set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
    return;
  }
  for (uint64_t k = threadIdx.x; k < tail_bytes; k += blockDim.x) p.dst[g.data_off + k] = p.src[k];
  if (threadIdx.x == 0) {
    write_stream_header(p.dst, g, g.data_off, total);
    *p.out_size = total;
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

static uint64_t align256(uint64_t v) { return (v + 255) & ~255ull; }

// CTAs (of 4 warps) per SM for the lane encoder; SPRINTZ_ENC_CTAS_PER_SM
// overrides it for tuning.
static uint32_t enc_lane_ctas_per_sm() {
  static uint32_t v = [] {
    const char *e = getenv("SPRINTZ_ENC_CTAS_PER_SM");
    int x = e ? atoi(e) : 0;
    return (uint32_t)(x > 0 && x <= 32 ? x : 3);
  }();
  return v;
}

struct EncPlan {
  bool stage_rows;
  uint64_t smem;
  uint32_t grid;
  uint64_t scratch_per_cta;
};

static EncPlan enc_plan(const Geom &g, const LaunchCfg &cfg) {
  EncPlan pl{};
  EncLayout Ls = enc_layout(g, true);
  const uint64_t smem_limit = std::min<uint64_t>((uint64_t)cfg.max_smem_optin, 200u * 1024);
  pl.stage_rows = Ls.total <= smem_limit;
  if (pl.stage_rows) {
    pl.smem = Ls.total;
    int per_sm = 0;
    const void *fn = g.w == 8 ? (const void *)k_encode<8> : (const void *)k_encode<16>;
    if (pl.smem > 48 * 1024)
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kEncThreads, pl.smem) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    pl.grid = (uint32_t)std::min<uint64_t>(g.n_chunks, (uint64_t)cfg.sm_count * per_sm);
    pl.scratch_per_cta = 0;
  } else {
    pl.smem = 0;
    pl.grid = (uint32_t)std::min<uint64_t>(g.n_chunks, (uint64_t)cfg.sm_count * 2);
    pl.scratch_per_cta = align256(enc_layout(g, false).total);
  }
  if (pl.grid == 0) pl.grid = 1;
  return pl;
}

// Workspace of the encoders that need only the ticket, the look-back words and
// (for chunks too large for shared memory) per-CTA scratch.
static uint64_t encode_workspace_basic(const Geom &g, const LaunchCfg &cfg) {
  uint64_t base = align256(16 + 8ull * g.n_chunks);
  if (g.n_chunks == 0) return base;
  EncPlan pl = enc_plan(g, cfg);
  return base + (uint64_t)pl.grid * pl.scratch_per_cta;
}

// Plan of the single-pass slot encoder (grid 0: not applicable).
struct SlotPlan {
  EncSlotCfg sc;
  uint32_t grid;
  uint64_t smem;
  uint64_t ws_base;   // ticket + look-back words (aligned)
  uint64_t ws_total;
};

static uint32_t enc_slot_ctas_per_sm() {
  static uint32_t v = [] {
    const char *e = getenv("SPRINTZ_ENC_SLOT_CTAS_PER_SM");
    int x = e ? atoi(e) : 0;
    return (uint32_t)(x > 0 && x <= 32 ? x : 8);
  }();
  return v;
}

static SlotPlan slot_plan(const Geom &g, const LaunchCfg &cfg) {
  SlotPlan pl{};
  if (g.n_chunks == 0 || g.D > 32 || g.max_body >= (1ull << 28)) return pl;
  const uint32_t K = 32 / g.D;
  pl.sc.window = enc_window_bytes(g);
  pl.sc.n_groups = (uint32_t)((g.n_chunks + K - 1) / K);
  pl.sc.slot_stride = (uint32_t)(((g.max_body + 31) & ~31ull) + 32);
  pl.smem = (uint64_t)kEncLaneWarps * enc_slot_region(g, pl.sc.window);
  if (pl.smem > (uint64_t)cfg.max_smem_optin) return pl;
  const uint64_t want = (pl.sc.n_groups + kEncLaneWarps - 1) / kEncLaneWarps;
  pl.grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)cfg.sm_count *
                                                                          enc_slot_ctas_per_sm()));
  pl.ws_base = align256(16 + 8ull * pl.sc.n_groups);
  pl.ws_total = pl.ws_base + (uint64_t)pl.grid * kEncLaneWarps * K * pl.sc.slot_stride;
  return pl;
}



int launch_encode(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint8_t *dst,
                  uint64_t dst_cap, uint64_t *d_out_size, uint8_t *ws, uint64_t ws_bytes,
                  int *d_status, cudaStream_t stream) {
  EncParams p{};
  p.src = src;
  p.dst = dst;
  p.dst_cap = dst_cap;
  p.out_size = d_out_size;
  p.status = d_status;
  p.g = g;
  p.spin_limit = cfg.wait_limit;
  int rc = SPRINTZ_OK;
  if (g.n_chunks == 0) {
    k_encode_tail_only<<<1, 128, 0, stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
  }
  if (g.D <= 32 && ((uintptr_t)src & 7) == 0) {
    // lane-per-column encoder: persistent warps, a few per SM so that the
    // groups between their two passes stay in L2
    const uint32_t K = 32 / g.D;
    EncLaneCfg lc;
    lc.window = enc_window_bytes(g);
    lc.n_groups = (uint32_t)((g.n_chunks + K - 1) / K);
    const uint64_t smem = (uint64_t)kEncLaneWarps * kEncStage + (uint64_t)kEncLaneWarps * K * lc.window;
    if (smem > (uint64_t)cfg.max_smem_optin) return SPRINTZ_ERR_UNSUPPORTED;
    if (ws_bytes < 16 + 8ull * g.n_chunks) return SPRINTZ_ERR_WS_TOO_SMALL;
    p.ticket = reinterpret_cast<uint32_t *>(ws);
    p.lookback = reinterpret_cast<uint64_t *>(ws + 16);
    const void *fn = g.w == 8 ? (const void *)k_encode_lanes<8> : (const void *)k_encode_lanes<16>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return SPRINTZ_ERR_CUDA;
    const uint64_t want_ctas = (lc.n_groups + kEncLaneWarps - 1) / kEncLaneWarps;
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(want_ctas, (uint64_t)cfg.sm_count *
                                                                                   enc_lane_ctas_per_sm()));
    if ((rc = init_ticket(ws, 16 + 8ull * lc.n_groups, cfg, stream)) != SPRINTZ_OK) return rc;
    if (g.w == 8)
      k_encode_lanes<8><<<(uint32_t)grid, kEncLaneThreads, smem, stream>>>(p, lc);
    else
      k_encode_lanes<16><<<(uint32_t)grid, kEncLaneThreads, smem, stream>>>(p, lc);
    return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
  }
  EncPlan pl = enc_plan(g, cfg);
  uint64_t base = align256(16 + 8ull * g.n_chunks);
  if (ws_bytes < base + (uint64_t)pl.grid * pl.scratch_per_cta) return SPRINTZ_ERR_WS_TOO_SMALL;
  p.ticket = reinterpret_cast<uint32_t *>(ws);
  p.lookback = reinterpret_cast<uint64_t *>(ws + 16);
  p.scratch = ws + base;
  p.scratch_per_cta = pl.scratch_per_cta;
  p.stage_rows = pl.stage_rows ? 1 : 0;
  if ((rc = init_ticket(ws, 16 + 8ull * g.n_chunks, cfg, stream)) != SPRINTZ_OK) return rc;
  if (g.w == 8)
    k_encode<8><<<pl.grid, kEncThreads, pl.smem, stream>>>(p);
  else
    k_encode<16><<<pl.grid, kEncThreads, pl.smem, stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

}  // namespace spz

namespace spz {

// Compression through the fastest applicable encoder: the single-pass slot
// encoder when the workspace holds its slots, else launch_encode's choice.
// ---------------------------------------------------------------------------
// Column-per-thread encoder for wide rows (32 < D <= 1024)
//
// Persistent CTAs take chunks in order from a ticket; thread j owns column j.
// Per block: the column's 8 samples (the threads of a row read consecutive
// samples), its forecast errors, zigzag and width; a block-wide scan of the
// widths gives each thread its bit offset in a row and the record's size.
// Header codes and row fields are OR-ed into a shared ring (rows are
// row-major: D * w > 32); completed 32-byte sectors go to the CTA's slot in
// the workspace.  At the chunk's end the look-back over chunks gives its
// offset and the CTA copies the slot to its place in the stream.
// ---------------------------------------------------------------------------

struct EncWideCfg {
  uint32_t window;       // ring bytes (power of two)
  uint32_t slot_stride;  // bytes per CTA slot (multiple of 32)
  uint8_t *slots;
};

template <int W>
__global__ void __launch_bounds__(1024) k_encode_wide(EncParams p, EncWideCfg cfg) {
  extern __shared__ __align__(16) uint8_t wsm_[];
  __shared__ uint32_t s_wsum[2][32];
  __shared__ uint32_t s_grp;
  __shared__ uint64_t s_prefix;
  const Geom &g = p.g;
  const uint32_t D = g.D, j = threadIdx.x, lane = j & 31, warp = j >> 5, nwarps = blockDim.x >> 5;
  const bool col = j < D;
  constexpr uint32_t wb = W / 8;
  constexpr uint32_t HB = W == 8 ? 3u : 4u;
  const uint32_t G = g.G, H = g.hdr_bytes;
  uint32_t *ring = reinterpret_cast<uint32_t *>(wsm_);
  const uint32_t ring_wmask = cfg.window / 4 - 1;
  uint8_t *slot = cfg.slots + (uint64_t)blockIdx.x * cfg.slot_stride;
  auto ror = [&](uint32_t bit, uint32_t v, uint32_t n) {
    if (!v) return;
    const uint32_t wi = (bit >> 5) & ring_wmask, sh = bit & 31;
    atomicOr(&ring[wi], v << sh);
    if (sh + n > 32) atomicOr(&ring[(wi + 1) & ring_wmask], v >> (32 - sh));
  };
  uint32_t par = 0;
  for (;;) {
    __syncthreads();
    if (j == 0) s_grp = atomicAdd(p.ticket, 1u);
    for (uint32_t t = j; t < cfg.window / 16; t += blockDim.x) reinterpret_cast<uint4 *>(ring)[t] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const uint32_t c = s_grp;
    if (c >= g.n_chunks) break;
    const uint64_t row0 = (uint64_t)c * g.chunk_rows;
    const uint32_t nb = (uint32_t)(min((uint64_t)g.chunk_rows, g.full_rows - row0) / kBlockRows);
    const uint8_t *xs = p.src + row0 * D * wb + j * wb;
    const uint32_t row_stride = D * wb;
    uint32_t xp = 0, run = 0, nrec = 0, gs = 0, pos = 0, hpos = 0, flushed = 0;
    int32_t dp = 0, acc = 0;
    bool open = false;
    auto start_record = [&]() {
      if (gs == 0) {
        hpos = pos;
        pos += H;
        open = true;
      }
    };
    auto end_record = [&](uint32_t size) {
      pos += size;
      nrec++;
      if (++gs == G) {
        gs = 0;
        open = false;
      }
    };
    auto emit_run = [&](uint32_t len) {
      start_record();
      if (j == 0) ror(pos * 8, len, 16);
      end_record(2);
    };
    // completed bytes to the slot in whole 32-byte sectors (a final partial
    // 16-byte unit at the chunk's end)
    auto flush = [&](uint32_t limit, bool fin) {
      __syncthreads();
      const uint32_t u1 = fin ? (limit + 15) >> 4 : (limit >> 5) << 1;
      for (uint32_t u = (flushed >> 4) + j; u < u1; u += blockDim.x) {
        uint4 *r4 = reinterpret_cast<uint4 *>(&ring[(u * 4) & ring_wmask]);
        *reinterpret_cast<uint4 *>(slot + 16ull * u) = *r4;
        *r4 = make_uint4(0, 0, 0, 0);
      }
      if (u1 * 16 > flushed) flushed = u1 * 16;
      __syncthreads();
    };
    uint32_t xn[kBlockRows];
#pragma unroll
    for (int i = 0; i < kBlockRows; ++i)
      xn[i] = col && nb ? (W == 8 ? (uint32_t)xs[i * row_stride]
                                  : (uint32_t)*reinterpret_cast<const uint16_t *>(xs + i * row_stride))
                        : 0u;
    for (uint32_t b = 0; b < nb; ++b) {
      uint32_t x[kBlockRows];
#pragma unroll
      for (int i = 0; i < kBlockRows; ++i) x[i] = xn[i];
      if (b + 1 < nb && col) {
        const uint8_t *q = xs + (uint64_t)(b + 1) * kBlockRows * row_stride;
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i)
          xn[i] = W == 8 ? (uint32_t)q[i * row_stride] : (uint32_t)*reinterpret_cast<const uint16_t *>(q + i * row_stride);
      }
      uint32_t z[kBlockRows];
      uint32_t orz = 0;
      if (g.forecaster == kFcDelta) {
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          z[i] = zigzag<W>(sext<W>(x[i] - xp));
          xp = x[i];
          orz |= z[i];
        }
      } else if (g.forecaster == kFcDDelta) {
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          z[i] = zigzag<W>(sext<W>(x[i] - xp - (uint32_t)dp));
          orz |= z[i];
          dp = sext<W>(x[i] - xp);
          xp = x[i];
        }
      } else if (g.forecaster == kFcFireSample) {
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          const int32_t e = sext<W>(x[i] - xp - fire_pred_delta<W>(acc >> g.learn_shift, dp));
          acc = wrap_acc<W>((int32_t)((uint32_t)acc + (uint32_t)(sign_of(e) * dp)));
          z[i] = zigzag<W>(e);
          orz |= z[i];
          dp = sext<W>(x[i] - xp);
          xp = x[i];
        }
      } else {
        const int32_t a = acc >> g.learn_shift;
        int32_t gsum = 0;
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          const int32_t e = sext<W>(x[i] - xp - fire_pred_delta<W>(a, dp));
          if ((i & 1) == 0) gsum += sign_of(e) * dp;
          z[i] = zigzag<W>(e);
          orz |= z[i];
          dp = sext<W>(x[i] - xp);
          xp = x[i];
        }
        acc = wrap_acc<W>((int32_t)((uint32_t)acc + (uint32_t)(gsum >> 2)));
      }
      uint32_t n = 32u - __clz(orz);
      if (n == W - 1) n = W;
      if (!col) n = 0;
      // block-wide exclusive scan of the widths
      uint32_t v = n;
#pragma unroll
      for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += t;
      }
      if (lane == 31) s_wsum[par][warp] = v;
      __syncthreads();
      if (warp == 0) {
        uint32_t t = lane < nwarps ? s_wsum[par][lane] : 0u;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
          const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, t, o);
          if (lane >= o) t += u;
        }
        if (lane < nwarps) s_wsum[par][lane] = t;
      }
      __syncthreads();
      const uint32_t prefix = v - n + (warp ? s_wsum[par][warp - 1] : 0u);
      const uint32_t total = s_wsum[par][nwarps - 1];
      par ^= 1;
      if (total == 0) {
        if (++run == kMaxRun) {
          emit_run(run);
          run = 0;
        }
      } else {
        if (run) {
          emit_run(run);
          run = 0;
        }
        start_record();
        const uint32_t size = (total + 7) & ~7u;  // bits per row (row-major)
        if (col) {
          ror(hpos * 8 + (gs * D + j) * HB, n == W ? W - 1 : n, HB);
          if (n) {
            const uint32_t b0 = pos * 8 + prefix;
#pragma unroll
            for (int i = 0; i < kBlockRows; ++i) ror(b0 + i * size, z[i], n);
          }
        }
        end_record(size);
      }
      flush(open ? hpos : pos, false);
    }
    if (run) emit_run(run);
    open = false;
    flush(pos, true);
    const uint32_t S = pos;

    // offset of the body: look-back over chunks (warp 0), then the copy
    if (warp == 0) {
      const uint64_t pre = lookback_warp(p.lookback, c, S, p.status, p.spin_limit);
      if (lane == 0) s_prefix = pre;
    }
    __syncthreads();
    const uint64_t off = s_prefix;
    if (g.data_off + off + S <= p.dst_cap) {
      uint8_t *d = p.dst + g.data_off + off;
      const uint32_t head = min((uint32_t)((16 - ((uintptr_t)d & 15)) & 15), S);
      for (uint32_t k = j; k < head; k += blockDim.x) d[k] = slot[k];
      const uint32_t n16 = (S - head) / 16;
      const uint32_t sh = (head & 3) * 8;
      const bool w1 = head & 4, w2 = head & 8;
      const uint4 *s4 = reinterpret_cast<const uint4 *>(slot);
      for (uint32_t u = j; u < n16; u += blockDim.x) {
        const uint4 A = s4[u], B = s4[u + 1];
        const uint32_t p0 = w2 ? A.z : A.x, p1 = w2 ? A.w : A.y, p2 = w2 ? B.x : A.z, p3 = w2 ? B.y : A.w;
        const uint32_t p4 = w2 ? B.z : B.x, p5 = w2 ? B.w : B.y;
        const uint32_t a0 = w1 ? p1 : p0, a1 = w1 ? p2 : p1, a2 = w1 ? p3 : p2, a3 = w1 ? p4 : p3,
                       a4 = w1 ? p5 : p4;
        uint4 o;
        o.x = __funnelshift_r(a0, a1, sh);
        o.y = __funnelshift_r(a1, a2, sh);
        o.z = __funnelshift_r(a2, a3, sh);
        o.w = __funnelshift_r(a3, a4, sh);
        *reinterpret_cast<uint4 *>(d + head + 16 * u) = o;
      }
      for (uint32_t k = head + 16 * n16 + j; k < S; k += blockDim.x) d[k] = slot[k];
      if (j == 0) {
        uint8_t *e = p.dst + kHdrBytes + (uint64_t)c * kEntryBytes;
        const uint64_t w1v = (uint64_t)nrec | ((uint64_t)S << 32);
        for (int k = 0; k < 8; ++k) {
          e[k] = (uint8_t)(off >> (8 * k));
          e[8 + k] = (uint8_t)(w1v >> (8 * k));
        }
      }
      if (c == g.n_chunks - 1) {
        const uint64_t tail_off = g.data_off + off + S;
        const uint64_t tail_bytes = g.tail_rows * D * wb;
        const uint64_t tot = tail_off + tail_bytes;
        if (tot <= p.dst_cap) {
          for (uint64_t k = j; k < tail_bytes; k += blockDim.x) p.dst[tail_off + k] = p.src[g.full_rows * D * wb + k];
          if (j == 0) {
            write_stream_header(p.dst, g, tail_off, tot);
            *p.out_size = tot;
          }
        } else if (j == 0) {
          set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
        }
      }
    } else if (j == 0) {
      set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
    }
  }
}

struct WidePlan {
  EncWideCfg wc;
  uint32_t grid, threads;
  uint64_t smem, ws_base, ws_total;
};

static WidePlan wide_plan(const Geom &g, const LaunchCfg &cfg) {
  WidePlan pl{};
  if (g.n_chunks == 0 || g.D <= 32 || g.D > 1024 || g.max_body >= (1ull << 31)) return pl;
  pl.wc.window = enc_window_bytes(g);
  pl.smem = pl.wc.window;
  if (pl.smem > (uint64_t)cfg.max_smem_optin - 1024) return pl;
  pl.threads = (g.D + 31) & ~31u;
  pl.wc.slot_stride = (uint32_t)(((g.max_body + 31) & ~31ull) + 32);
  // persistent CTAs: up to 2048 / threads per SM, with the slots' total kept
  // below 1 GiB
  const uint64_t per_sm = std::max<uint64_t>(1, 2048 / pl.threads);
  uint64_t grid = std::min<uint64_t>(g.n_chunks, (uint64_t)cfg.sm_count * per_sm);
  while (grid > (uint64_t)cfg.sm_count && grid * pl.wc.slot_stride > (1ull << 30)) grid /= 2;
  pl.grid = (uint32_t)std::max<uint64_t>(1, grid);
  pl.ws_base = align256(16 + 8ull * g.n_chunks);
  pl.ws_total = pl.ws_base + (uint64_t)pl.grid * pl.wc.slot_stride;
  return pl;
}

static int launch_encode_wide(const Geom &g, const LaunchCfg &cfg, const WidePlan &pl, const uint8_t *src,
                              uint8_t *dst, uint64_t dst_cap, uint64_t *d_out_size, uint8_t *ws, int *d_status,
                              cudaStream_t stream) {
  EncParams p{};
  p.src = src;
  p.dst = dst;
  p.dst_cap = dst_cap;
  p.out_size = d_out_size;
  p.status = d_status;
  p.g = g;
  p.spin_limit = cfg.wait_limit;
  int rc = SPRINTZ_OK;
  p.ticket = reinterpret_cast<uint32_t *>(ws);
  p.lookback = reinterpret_cast<uint64_t *>(ws + 16);
  EncWideCfg wc = pl.wc;
  wc.slots = ws + pl.ws_base;
  const void *fn = g.w == 8 ? (const void *)k_encode_wide<8> : (const void *)k_encode_wide<16>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) != cudaSuccess)
    return SPRINTZ_ERR_CUDA;
  if ((rc = init_ticket(ws, 16 + 8ull * g.n_chunks, cfg, stream)) != SPRINTZ_OK) return rc;
  void *args[] = {&p, &wc};
  if (cudaLaunchKernel(fn, dim3(pl.grid), dim3(pl.threads), args, pl.smem, stream) != cudaSuccess)
    return SPRINTZ_ERR_CUDA;
  return SPRINTZ_OK;
}

uint64_t encode_workspace_bytes(const Geom &g, const LaunchCfg &cfg) {
  const SlotPlan sp = slot_plan(g, cfg);
  const WidePlan wp = wide_plan(g, cfg);
  return std::max<uint64_t>(std::max<uint64_t>(encode_workspace_basic(g, cfg), sp.grid ? sp.ws_total : 0ull),
                            wp.grid ? wp.ws_total : 0ull);
}

int launch_encode_fast(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint8_t *dst,
                       uint64_t dst_cap, uint64_t *d_out_size, uint8_t *ws, uint64_t ws_bytes,
                       int *d_status, cudaStream_t stream) {
  if (g.D > 32) {
    const WidePlan wp = wide_plan(g, cfg);
    if (wp.grid && ws_bytes >= wp.ws_total)
      return launch_encode_wide(g, cfg, wp, src, dst, dst_cap, d_out_size, ws, d_status, stream);
    return launch_encode(g, cfg, src, dst, dst_cap, d_out_size, ws, ws_bytes, d_status, stream);
  }
  const SlotPlan sp = slot_plan(g, cfg);
  if (!sp.grid || ((uintptr_t)src & 7) != 0 || ws_bytes < sp.ws_total)
    return launch_encode(g, cfg, src, dst, dst_cap, d_out_size, ws, ws_bytes, d_status, stream);
  EncParams p{};
  p.src = src;
  p.dst = dst;
  p.dst_cap = dst_cap;
  p.out_size = d_out_size;
  p.status = d_status;
  p.g = g;
  p.spin_limit = cfg.wait_limit;
  int rc = SPRINTZ_OK;
  p.ticket = reinterpret_cast<uint32_t *>(ws);
  p.lookback = reinterpret_cast<uint64_t *>(ws + 16);
  EncSlotCfg sc = sp.sc;
  sc.slots = ws + sp.ws_base;
  const void *fn = g.w == 8 ? slot_encoder<8>(g.D) : slot_encoder<16>(g.D);
  if (sp.smem > 48 * 1024 &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp.smem) != cudaSuccess)
    return SPRINTZ_ERR_CUDA;
  if ((rc = init_ticket(ws, 16 + 8ull * sc.n_groups, cfg, stream)) != SPRINTZ_OK) return rc;
  void *args[] = {&p, &sc};
  if (cudaLaunchKernel(fn, dim3(sp.grid), dim3(kEncLaneThreads), args, sp.smem, stream) != cudaSuccess)
    return SPRINTZ_ERR_CUDA;
  return SPRINTZ_OK;
}

// ---- batches ----------------------------------------------------------------

// The schedules the autotuner picks on a batch of 10,000 streams (rows
// log-uniform in 1e3..1e6, D = 1..16, u8 and u16): compress round robin
// inside each class (a group's predecessor in its stream is long done when
// it looks back) without prefetch; decompress longest stream first with an
// 8 KB L2 prefetch window.
sprintz_schedule batch_default_schedule(int compress) {
  sprintz_schedule s;
  s.ctas_per_sm = compress ? 7 : 6;  // as many as the kernels' register bounds allow
  s.ring_segments = 2;
  s.prefetch_bytes = compress ? 1 : 8192;
  s.order = compress ? 3 : 2;
  return s;
}

static sprintz_schedule resolve_schedule(const sprintz_schedule &in, int compress) {
  const sprintz_schedule d = batch_default_schedule(compress);
  sprintz_schedule s = in;
  if (!s.ctas_per_sm) s.ctas_per_sm = d.ctas_per_sm;
  if (s.ring_segments != 2 && s.ring_segments != 4) s.ring_segments = d.ring_segments;
  if (!s.prefetch_bytes) s.prefetch_bytes = d.prefetch_bytes;
  if (s.prefetch_bytes != 1) s.prefetch_bytes &= ~15u;
  if (s.order < 1 || s.order > 3) s.order = d.order;
  return s;
}

void batch_work_list(const std::vector<uint32_t> &w, const std::vector<uint32_t> &D,
                     const std::vector<uint64_t> &groups, uint32_t order, uint32_t sm_count,
                     std::vector<uint64_t> *image, uint64_t *n_work) {
  const uint32_t n = (uint32_t)w.size();
  // classes (w, D), heaviest groups first, then by w and D
  std::vector<uint32_t> idx(n);
  for (uint32_t i = 0; i < n; ++i) idx[i] = i;
  auto cls = [&](uint32_t i) { return (uint64_t)w[i] << 32 | D[i]; };
  std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) {
    if (cls(a) != cls(b)) {
      const uint64_t ga = (uint64_t)(32 / D[a]) * D[a] * w[a], gb = (uint64_t)(32 / D[b]) * D[b] * w[b];
      if (ga != gb) return ga > gb;
      return cls(a) < cls(b);
    }
    if (order == 2 && groups[a] != groups[b]) return groups[a] > groups[b];
    return a < b;
  });
  const uint64_t hdr_words = kClassTableBytes / 8;
  image->assign(hdr_words, 0);
  uint64_t total = 0;
  for (uint32_t i = 0; i < n; ++i) total += groups[i];
  image->reserve(hdr_words + total);
  BatchClasses tab;
  memset(&tab, 0, sizeof(tab));
  for (uint32_t a = 0; a < n;) {
    uint32_t b = a;
    while (b < n && cls(idx[b]) == cls(idx[a])) ++b;
    uint64_t cg = 0;
    for (uint32_t k = a; k < b; ++k) cg += groups[idx[k]];
    if (cg) {
      const uint32_t c = tab.n_classes < kMaxBatchClasses ? tab.n_classes++ : kMaxBatchClasses - 1;
      tab.start[c] = image->size() - hdr_words;
      if (order == 3) {
        // round robin: group r of every stream of the class that has one
        uint64_t rmax = 0;
        for (uint32_t k = a; k < b; ++k) rmax = std::max<uint64_t>(rmax, groups[idx[k]]);
        for (uint64_t r = 0; r < rmax; ++r)
          for (uint32_t k = a; k < b; ++k)
            if (r < groups[idx[k]]) image->push_back((uint64_t)idx[k] << kWorkGroupBits | r);
      } else {
        for (uint32_t k = a; k < b; ++k)
          for (uint64_t r = 0; r < groups[idx[k]]; ++r) image->push_back((uint64_t)idx[k] << kWorkGroupBits | r);
      }
      tab.start[c + 1] = image->size() - hdr_words;
    }
    a = b;
  }
  *n_work = image->size() - hdr_words;
  // home classes: SM s takes the class that holds the point (s + 1/2) / n_sm
  // of the work
  tab.n_sm = std::max<uint32_t>(1, std::min<uint32_t>(sm_count, kMaxHomeSm));
  for (uint32_t sm = 0; sm < tab.n_sm && tab.n_classes; ++sm) {
    const double p = (sm + 0.5) * (double)*n_work / tab.n_sm;
    uint32_t c = 0;
    while (c + 1 < tab.n_classes && (double)tab.start[c + 1] <= p) ++c;
    tab.home[sm] = (uint8_t)c;
  }
  memcpy(image->data(), &tab, sizeof(tab));
}

// CTAs of the batched encoder that fit one SM with `region` shared bytes per warp.
static uint32_t enc_batch_occupancy(uint32_t region, const LaunchCfg &cfg) {
  const uint64_t smem = (uint64_t)kEncLaneWarps * region;
  if (smem > (uint64_t)cfg.max_smem_optin) return 0;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_encode_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_encode_batch, kEncLaneThreads, smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  return (uint32_t)occ;
}

int plan_batch_encode(const sprintz_batch_item *items, uint32_t n, const LaunchCfg &cfg,
                      const sprintz_schedule &sched_in, int *d_status, uint8_t *ws, BatchPlan *pl,
                      std::vector<uint8_t> *img, std::vector<uint64_t> *work) {
  if (n > kMaxBatchStreams) return SPRINTZ_ERR_INVALID_ARG;
  const sprintz_schedule sched = resolve_schedule(sched_in, 1);
  std::vector<EncBatchItem> v(n);
  std::vector<uint32_t> vw(n), vD(n);
  std::vector<uint64_t> vgroups(n);
  uint64_t lb_words = 0;
  uint32_t region = kEncStage;
  uint64_t slot_region = 16;
  for (uint32_t i = 0; i < n; ++i) {
    const sprintz_batch_item &it = items[i];
    Geom g;
    int rc = make_geom(it.rows, it.D, it.w, &it.opts, &g);
    if (rc != SPRINTZ_OK) return rc;
    if (it.opts.huffman || g.D > 32 || g.max_body >= (1ull << 28)) return SPRINTZ_ERR_UNSUPPORTED;
    if (!it.dst || !it.out_size || (it.rows && !it.src)) return SPRINTZ_ERR_INVALID_ARG;
    if (((uintptr_t)it.src & 7) != 0) return SPRINTZ_ERR_UNSUPPORTED;
    if (it.dst_cap < sprintz_max_compressed_size(it.rows, it.D, it.w, &it.opts)) return SPRINTZ_ERR_DST_TOO_SMALL;
    const uint32_t K = 32 / g.D;
    EncBatchItem &e = v[i];
    memset(&e, 0, sizeof(e));
    e.p.src = (const uint8_t *)it.src;
    e.p.dst = (uint8_t *)it.dst;
    e.p.dst_cap = it.dst_cap;
    e.p.out_size = it.out_size;
    e.p.status = d_status;
    e.p.g = g;
    e.p.lookback = reinterpret_cast<uint64_t *>(ws + kClassTicketBytes + 8 * lb_words);
    e.cfg.window = enc_window_bytes(g);
    e.cfg.n_groups = (uint32_t)((g.n_chunks + K - 1) / K);
    e.cfg.slot_stride = (uint32_t)(((g.max_body + 31) & ~31ull) + 32);
    e.cfg.pf_bytes = sched.prefetch_bytes == 1 ? 0u : sched.prefetch_bytes;
    lb_words += e.cfg.n_groups;
    vw[i] = g.w;
    vD[i] = g.D;
    vgroups[i] = e.cfg.n_groups;
    if (g.n_chunks) {
      region = std::max<uint32_t>(region, enc_slot_region(g, e.cfg.window));
      slot_region = std::max<uint64_t>(slot_region, (uint64_t)K * e.cfg.slot_stride);
    }
  }
  uint64_t n_work = 0;
  batch_work_list(vw, vD, vgroups, sched.order, (uint32_t)cfg.sm_count, work, &n_work);
  memset(pl, 0, sizeof(*pl));
  pl->compress = 1;
  pl->n = n;
  pl->region = region;
  pl->slot_region = slot_region;
  pl->n_work = n_work;
  pl->zero_bytes = kClassTicketBytes + 8 * lb_words;
  pl->items_off = align256(pl->zero_bytes);
  pl->work_off = align256(pl->items_off + (uint64_t)n * sizeof(EncBatchItem));
  pl->slots_off = align256(pl->work_off + 8ull * work->size());
  const uint32_t occ = enc_batch_occupancy(region, cfg);
  if (!occ) return SPRINTZ_ERR_UNSUPPORTED;
  const uint64_t want = (pl->n_work + kEncLaneWarps - 1) / kEncLaneWarps;
  const uint64_t max_grid = std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)cfg.sm_count * occ));
  pl->grid = (uint32_t)std::max<uint64_t>(
      1, std::min<uint64_t>(want, (uint64_t)cfg.sm_count * std::min<uint32_t>(occ, sched.ctas_per_sm)));
  // the workspace holds the slots of the largest grid any schedule may take
  pl->ws_total = pl->slots_off + max_grid * kEncLaneWarps * slot_region;
  pl->sched = sched;
  pl->sched.ctas_per_sm = std::min<uint32_t>(occ, sched.ctas_per_sm);
  if (ws)
    for (auto &e : v) e.p.ticket = reinterpret_cast<uint32_t *>(ws);
  img->assign(reinterpret_cast<const uint8_t *>(v.data()),
              reinterpret_cast<const uint8_t *>(v.data()) + (size_t)n * sizeof(EncBatchItem));
  return SPRINTZ_OK;
}

int run_batch_encode(const BatchPlan &pl, cudaStream_t stream) {
  uint8_t *ws = (uint8_t *)pl.ws;
  const EncBatchItem *items = reinterpret_cast<const EncBatchItem *>(ws + pl.items_off);
  const BatchClasses *classes = reinterpret_cast<const BatchClasses *>(ws + pl.work_off);
  const uint64_t *work = reinterpret_cast<const uint64_t *>(ws + pl.work_off + kClassTableBytes);
  if (cudaMemsetAsync(ws, 0, pl.zero_bytes, stream) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  k_encode_batch_tails<<<pl.n, 128, 0, stream>>>(items);
  if (pl.n_work)
    k_encode_batch<<<pl.grid, kEncLaneThreads, (uint64_t)kEncLaneWarps * pl.region, stream>>>(
        items, classes, work, reinterpret_cast<uint32_t *>(ws), pl.region, ws + pl.slots_off, pl.slot_region);
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

}  // namespace spz

// ---------------------------------------------------------------------------
// Compression for callers that cannot allocate device memory
//
// Some callers cannot call cudaMalloc at all: a process whose own pool
// allocator has taken all free device memory and must see every allocation,
// or a request path in a serving system that may not let cudaMalloc/cudaFree
// implicitly synchronize the device while other streams are running.  For
// them sprintz_compress_noalloc() runs the same encoder with its scratch (the
// chunk ticket, the look-back words and a status word) in a fixed array that
// this library defines in device memory.  Every GPU that loads the library
// holds the array until the process exits.
// ---------------------------------------------------------------------------

namespace spz {

constexpr uint64_t kNoAllocMaxChunks = 65536;  // chunks per call
// ticket + one look-back word per chunk, rounded up as the encoders' own
// workspace layout rounds it, then the status word
constexpr uint64_t kNoAllocStatusOff = (16 + 8 * kNoAllocMaxChunks + 255) & ~255ull;
constexpr uint64_t kNoAllocBytes = kNoAllocStatusOff + 256;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

struct NoAllocDevice {
  std::once_flag once;
  int rc = SPRINTZ_OK;
  uint8_t *ptr = nullptr;  // device address of g_noalloc_scratch on this device
  LaunchCfg cfg{};
};
constexpr int kNoAllocMaxDevices = 64;
static NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];

// A device-side failure (a bounded wait that gave up) is reported as size 0.
__global__ void k_noalloc_finish(const int *status, uint64_t *out_size) {
  if (*status != 0) *out_size = 0;
}

}  // namespace spz

extern "C" int sprintz_compress_noalloc(const void *src, uint64_t rows, uint32_t D, uint32_t w,
                                        const sprintz_opts *opts, void *dst, uint64_t dst_cap,
                                        uint64_t *d_out_size, void *stream) {
  using namespace spz;
  if (!dst || !d_out_size || (rows && !src)) return SPRINTZ_ERR_INVALID_ARG;
  Geom g;
  int rc = make_geom(rows, D, w, opts, &g);
  if (rc != SPRINTZ_OK) return rc;
  if (opts->huffman) return SPRINTZ_ERR_UNSUPPORTED;
  if (dst_cap < sprintz_max_compressed_size(rows, D, w, opts)) return SPRINTZ_ERR_DST_TOO_SMALL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return SPRINTZ_ERR_UNSUPPORTED;
  NoAllocDevice &nd = g_noalloc_dev[dev];
  // first call on this device (device current): find the array's address.
  // It is kept for the process's life; a cudaDeviceReset() makes it stale.
  std::call_once(nd.once, [&nd, dev] {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess ||
        cudaDeviceGetAttribute(&nd.cfg.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nd.cfg.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess) {
      nd.rc = SPRINTZ_ERR_CUDA;
      return;
    }
    nd.ptr = static_cast<uint8_t *>(ptr);
  });
  if (nd.rc != SPRINTZ_OK) return nd.rc;
  // the fixed array bounds the call: at most kNoAllocMaxChunks chunks, and no
  // chunk so large that the encoder would need per-block global scratch.
  // The scratch needed is that of the path launch_encode() takes: the lane
  // encoder (D <= 32, 8-byte-aligned samples) needs the ticket and one word
  // per chunk; the CTA-per-chunk encoder also its per-CTA arrays when a chunk
  // does not fit shared memory.
  const bool lane_path = g.D <= 32 && ((uintptr_t)src & 7) == 0;
  const uint64_t need = g.n_chunks == 0 ? 0
                        : lane_path     ? 16 + 8ull * g.n_chunks
                                        : encode_workspace_basic(g, nd.cfg);
  if (g.n_chunks > kNoAllocMaxChunks || need > kNoAllocStatusOff) return SPRINTZ_ERR_WS_TOO_SMALL;
  int *status = reinterpret_cast<int *>(nd.ptr + kNoAllocStatusOff);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  rc = launch_encode(g, nd.cfg, (const uint8_t *)src, (uint8_t *)dst, dst_cap, d_out_size, nd.ptr,
                     kNoAllocStatusOff, status, s);
  if (rc != SPRINTZ_OK) return rc;
  k_noalloc_finish<<<1, 1, 0, s>>>(status, d_out_size);
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

