// Sprintz encoder on sm_103a.
//
// One CTA encodes one chunk at a time (a chunk is an independent Sprintz
// stream of chunk_rows rows: the forecaster restarts at zero).  Chunks are
// taken in order from an atomic ticket, so every chunk a CTA waits on is
// already running.  Per chunk:
//   1. the chunk's rows are staged in shared memory (128-bit loads);
//   2. FIRE only: one thread per column runs the block-level recurrence of
//      alpha (Algorithm 3 with alpha fixed per block, one averaged update per
//      block from the gradients of rows 0, 2, 4, 6 — Sec. 3.2.2);
//   3. every (block, column) recomputes its 8 errors, zigzags them and takes
//      the width from the OR of the column (Sec. 3.3), promoting w-1 to w;
//   4. blocks whose widths are all zero merge into runs; records, groups of G
//      record headers and payload offsets are laid out (Algorithm 1);
//   5. headers and payloads are packed into a shared-memory copy of the body
//      (column-major if D*w <= 32, else row-major — Sec. 3.3);
//   6. a decoupled look-back over the chunks' body sizes (single pass,
//      bounded waits) gives the body's offset in the stream;
//   7. the body and its chunk-table entry are written; the last chunk writes
//      the raw tail, the stream header and the stream size.
// Chunks too large for shared memory use a per-CTA global scratch slot and
// read their rows straight from the source.
#include <algorithm>

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
  L.alpha = take(g.forecaster == kFcFire ? nb * g.D * 4 : 0);
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
  Geom g;
};

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
  return sext<W>(x - xp - fire_pred_delta<W>(alpha, dp));
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
    int32_t a = g.forecaster == kFcFire ? alpha[q] : 0;
    uint32_t o = 0;
#pragma unroll
    for (int i = 0; i < kBlockRows; ++i)
      o |= zigzag<W>(error_at<W>(X, D, (uint64_t)b * kBlockRows + i, j, g.forecaster, a));
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
      int32_t a = g.forecaster == kFcFire ? alpha[(uint64_t)b * D + k] : 0;
      uint64_t lo = 0, hi = 0;  // 128-bit little-endian bit buffer
      for (int i = 0; i < kBlockRows; ++i) {
        uint64_t z = zigzag<W>(error_at<W>(X, D, (uint64_t)b * kBlockRows + i, k, g.forecaster, a));
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
        int32_t a = g.forecaster == kFcFire ? alpha[(uint64_t)b * D + j] : 0;
        uint64_t z = zigzag<W>(error_at<W>(X, D, row, j, g.forecaster, a));
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
          if (++spins > kSpinLimit) {
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
// Host side
// ---------------------------------------------------------------------------

static uint64_t align256(uint64_t v) { return (v + 255) & ~255ull; }

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

uint64_t encode_workspace_bytes(const Geom &g, const LaunchCfg &cfg) {
  uint64_t base = align256(16 + 8ull * g.n_chunks);
  if (g.n_chunks == 0) return base;
  EncPlan pl = enc_plan(g, cfg);
  return base + (uint64_t)pl.grid * pl.scratch_per_cta;
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
  if (g.n_chunks == 0) {
    k_encode_tail_only<<<1, 128, 0, stream>>>(p);
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
  if (cudaMemsetAsync(ws, 0, 16 + 8ull * g.n_chunks, stream) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  if (g.w == 8)
    k_encode<8><<<pl.grid, kEncThreads, pl.smem, stream>>>(p);
  else
    k_encode<16><<<pl.grid, kEncThreads, pl.smem, stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

}  // namespace spz
