// Sprintz decoder on sm_103a.
//
// Chunks are independent (the forecaster restarts at each one), and the
// chunk table gives every body's offset, so one CTA decodes one chunk with no
// inter-CTA communication.  Per chunk:
//   1. the chunk's body is staged in shared memory;
//   2. one thread walks the groups of record headers (the only serial part:
//      each group's position depends on the sizes of the records before it)
//      and lays out every record's first block, run length and payload
//      offset, validating every count and offset against the body;
//   3. all threads unpack the payloads in parallel — column-major items are
//      (record, column), row-major items are (record, row) — and un-zigzag
//      them into a shared tile of errors (runs leave zeros);
//   4. the forecast is inverted in place: delta as a per-column wrap-around
//      prefix sum split across threads; FIRE as one serial recurrence per
//      column (Algorithm 2 with Algorithm 3's predict/train, alpha fixed per
//      block, one averaged update per block — Sec. 4.2.2);
//   5. the tile is stored with 128-bit stores.
// CTA 0 also checks the stream header against the host's view of it and
// copies the raw trailing rows.  Chunks too large for shared memory use a
// per-CTA global scratch slot for the record arrays and work directly in the
// source and destination.
#include <stdlib.h>

#include <algorithm>

#include "spz_common.cuh"

namespace spz {

constexpr int kDecThreads = 256;

struct DecLayout {
  uint64_t body, x, rec_first, rec_run, rec_off, grp_off, part, total;
};

__host__ __device__ inline DecLayout dec_layout(const Geom &g, bool staged) {
  DecLayout L;
  uint64_t o = 0;
  uint64_t nb = g.max_blocks;
  auto take = [&](uint64_t bytes) {
    uint64_t r = o;
    o += (bytes + 15) & ~15ull;
    return r;
  };
  L.body = staged ? take(g.max_body + 32) : 0;
  L.x = staged ? take(nb * kBlockRows * g.D * g.wb) : 0;
  L.rec_first = take(nb * 4);
  L.rec_run = take(nb * 4);
  L.rec_off = take(nb * 4);
  L.grp_off = take(nb * 4);
  L.part = take((uint64_t)kDecThreads * 4);
  L.total = o;
  return L;
}

struct DecParams {
  uint32_t pf_win;   // L2 bulk-prefetch window of the lane decoder (bytes, multiple of 16)
  uint32_t pf_mode;  // unused (0)
  // lane decoder: decode chunks [c_begin, c_end); dst holds row c_begin * chunk_rows
  uint32_t c_begin;
  uint32_t c_end;
  const uint8_t *src;
  uint64_t src_size;
  uint8_t *dst;
  uint64_t dst_cap;
  int *status;
  uint8_t *scratch;
  uint64_t scratch_per_cta;
  uint32_t staged;
  Geom g;
};

__device__ __forceinline__ uint64_t le_u64(const uint8_t *p) {
  uint64_t v = 0;
  for (int k = 0; k < 8; ++k) v |= (uint64_t)p[k] << (8 * k);
  return v;
}
__device__ __forceinline__ uint32_t le_u32(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

// Copy n bytes with the whole CTA (16-byte vectors when both ends allow).
__device__ void cta_copy_dec(uint8_t *dst, const uint8_t *src, uint64_t n) {
  uint64_t head = (16 - ((uintptr_t)dst & 15)) & 15;
  if (head > n) head = n;
  bool vec = (((uintptr_t)src + head) & 15) == 0;
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

// Copy n bytes from a source of any alignment into a 16-byte-aligned
// destination, 16-byte loads of the aligned source span.
__device__ void cta_copy_from_unaligned(uint8_t *dst, const uint8_t *src, uint64_t n) {
  const uint32_t mis = (uint32_t)((uintptr_t)src & 15);
  if (mis == 0) {
    cta_copy_dec(dst, src, n);
    return;
  }
  // dst[k] = src[k] for k < n, via aligned 16-byte source words: source word
  // t covers src[16t - mis, 16t - mis + 16).
  const uint8_t *a = src - mis;
  uint64_t nw = (n + mis + 15) / 16;
  for (uint64_t t = threadIdx.x; t < nw; t += blockDim.x) {
    uint64_t lo = t * 16;  // offset from a
    if (t == 0 || t == nw - 1) {
      for (uint32_t k = 0; k < 16; ++k) {
        uint64_t o = lo + k;
        if (o >= mis && o - mis < n) dst[o - mis] = a[o];
      }
      continue;
    }
    uint4 v = *reinterpret_cast<const uint4 *>(a + lo);
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 16; ++k) dst[lo + k - mis] = (uint8_t)(w[k >> 2] >> (8 * (k & 3)));
  }
}

template <int W>
__device__ __forceinline__ uint32_t tile_get(const uint8_t *X, uint32_t D, uint64_t r, uint32_t j) {
  return load_sample<W>(X + ((uint64_t)r * D + j) * (W / 8));
}
template <int W>
__device__ __forceinline__ void tile_put(uint8_t *X, uint32_t D, uint64_t r, uint32_t j, uint32_t v) {
  store_sample<W>(X + ((uint64_t)r * D + j) * (W / 8), v);
}

__device__ __forceinline__ uint32_t header_code(const uint8_t *hdr, uint32_t idx, uint32_t hb) {
  return read_bits(hdr, (uint64_t)idx * hb, hb);
}

template <int W>
__device__ void decode_chunk(const DecParams &p, uint8_t *mem, uint32_t c, uint64_t data_bytes) {
  const Geom &g = p.g;
  const uint32_t D = g.D;
  const uint32_t wb = W / 8;
  const DecLayout L = dec_layout(g, p.staged != 0);
  __shared__ uint32_t s_bad;
  __shared__ uint32_t s_nrec;

  const uint64_t row0 = (uint64_t)c * g.chunk_rows;
  const uint64_t rows_c = min(g.chunk_rows, g.full_rows - row0);
  const uint32_t nb = (uint32_t)(rows_c / kBlockRows);
  uint8_t *dst_c = p.dst + row0 * D * wb;
  const uint64_t bytes_c = rows_c * D * wb;

  uint32_t *rec_first = reinterpret_cast<uint32_t *>(mem + L.rec_first);
  uint32_t *rec_run = reinterpret_cast<uint32_t *>(mem + L.rec_run);
  uint32_t *rec_off = reinterpret_cast<uint32_t *>(mem + L.rec_off);
  uint32_t *grp_off = reinterpret_cast<uint32_t *>(mem + L.grp_off);
  uint32_t *part = reinterpret_cast<uint32_t *>(mem + L.part);
  __syncthreads();  // the previous chunk's readers of s_bad / s_nrec are done

  // Chunk entry: body offset, record count, packed bytes; the body ends where
  // the next one starts (or at the tail).
  const uint8_t *e = p.src + kHdrBytes + (uint64_t)c * kEntryBytes;
  const uint64_t off = le_u64(e);
  const uint32_t nrec = le_u32(e + 8);
  const uint32_t packed = le_u32(e + 12);
  const uint64_t end = c + 1 < g.n_chunks ? le_u64(e + kEntryBytes) : data_bytes;
  if (threadIdx.x == 0) {
    bool bad = off > end || end > data_bytes || end - off != packed || nrec < 1 || nrec > nb ||
               packed > g.max_body;
    s_bad = bad;
    if (bad) set_status(p.status, SPRINTZ_ERR_CORRUPT);
  }
  __syncthreads();
  if (s_bad) return;

  // 1. body
  const uint8_t *src_body = p.src + g.data_off + off;
  const uint8_t *body = src_body;
  if (p.staged) {
    cta_copy_from_unaligned(mem + L.body, src_body, packed);
    body = mem + L.body;
  }
  uint8_t *X = p.staged ? mem + L.x : dst_c;
  // errors start at zero (run blocks keep them)
  if (p.staged) {
    uint4 z = make_uint4(0, 0, 0, 0);
    for (uint64_t k = threadIdx.x; k < (bytes_c + 15) / 16; k += blockDim.x)
      reinterpret_cast<uint4 *>(X)[k] = z;
  } else {
    for (uint64_t k = threadIdx.x; k < bytes_c; k += blockDim.x) X[k] = 0;
  }
  __syncthreads();

  // 2. walk the header groups
  if (threadIdx.x == 0) {
    uint64_t pos = 0;
    uint32_t blk = 0;
    bool bad = false;
    const uint32_t ngroups = (nrec + g.G - 1) / g.G;
    for (uint32_t q = 0; q < ngroups && !bad; ++q) {
      const uint64_t h = pos;
      grp_off[q] = (uint32_t)h;
      pos += g.hdr_bytes;
      if (pos > packed) {
        bad = true;
        break;
      }
      const uint8_t *hdr = body + h;
      for (uint32_t s = 0; s < g.G; ++s) {
        const uint32_t r = q * g.G + s;
        uint32_t sum = 0, any = 0;
        for (uint32_t j = 0; j < D; ++j) {
          uint32_t code = header_code(hdr, s * D + j, g.hb);
          any |= code;
          sum += code_to_width(code, W);
        }
        if (r >= nrec) {
          if (any) bad = true;  // unused slots hold zero codes
          continue;
        }
        rec_first[r] = blk;
        rec_off[r] = (uint32_t)pos;
        if (!any) {
          if (pos + 2 > packed) {
            bad = true;
            break;
          }
          uint32_t cnt = (uint32_t)body[pos] | ((uint32_t)body[pos + 1] << 8);
          pos += 2;
          if (cnt == 0 || blk + cnt > nb) {
            bad = true;
            break;
          }
          rec_run[r] = cnt;
          blk += cnt;
        } else {
          pos += g.col_major ? sum : 8 * ((sum + 7) / 8);
          if (pos > packed || blk + 1 > nb) {
            bad = true;
            break;
          }
          rec_run[r] = 0;
          blk += 1;
        }
      }
    }
    if (blk != nb || pos != packed) bad = true;
    s_bad = bad;
    s_nrec = nrec;
    if (bad) set_status(p.status, SPRINTZ_ERR_CORRUPT);
  }
  __syncthreads();
  if (s_bad) return;

  // 3. unpack + un-zigzag into the tile
  const uint32_t per = g.col_major ? D : kBlockRows;
  for (uint64_t q = threadIdx.x; q < (uint64_t)nrec * per; q += blockDim.x) {
    const uint32_t r = (uint32_t)(q / per), k = (uint32_t)(q % per);
    if (rec_run[r]) continue;
    const uint32_t b = rec_first[r];
    const uint8_t *hdr = body + grp_off[r / g.G];
    const uint32_t s = r % g.G;
    if (g.col_major) {
      uint32_t offb = 0;
      for (uint32_t j = 0; j < k; ++j) offb += code_to_width(header_code(hdr, s * D + j, g.hb), W);
      const uint32_t n = code_to_width(header_code(hdr, s * D + k, g.hb), W);
      if (!n) continue;
      const uint64_t bit0 = ((uint64_t)rec_off[r] + offb) * 8;
#pragma unroll
      for (int i = 0; i < kBlockRows; ++i) {
        uint32_t z = read_bits(body, bit0 + (uint64_t)i * n, n);
        tile_put<W>(X, D, (uint64_t)b * kBlockRows + i, k, (uint32_t)unzigzag<W>(z));
      }
    } else {
      uint32_t sum = 0;
      for (uint32_t j = 0; j < D; ++j) sum += code_to_width(header_code(hdr, s * D + j, g.hb), W);
      const uint32_t R = (sum + 7) / 8;
      uint64_t bit = ((uint64_t)rec_off[r] + (uint64_t)k * R) * 8;
      const uint64_t row = (uint64_t)b * kBlockRows + k;
      for (uint32_t j = 0; j < D; ++j) {
        const uint32_t n = code_to_width(header_code(hdr, s * D + j, g.hb), W);
        if (!n) continue;
        uint32_t z = read_bits(body, bit, n);
        bit += n;
        tile_put<W>(X, D, row, j, (uint32_t)unzigzag<W>(z));
      }
    }
  }
  __syncthreads();

  // 4. invert the forecast
  if (g.forecaster == kFcDelta) {
    // x_r = sum_{k <= r} e_k mod 2^w per column: segment sums, a scan of the
    // segment sums, then each segment re-summed from its offset.
    const uint32_t S = D >= blockDim.x ? 1u : blockDim.x / D;
    const uint64_t seg = (rows_c + S - 1) / S;
    const uint64_t items = (uint64_t)D * S;
    for (uint64_t t = threadIdx.x; t < items; t += blockDim.x) {
      const uint32_t j = (uint32_t)(t % D), sg = (uint32_t)(t / D);
      const uint64_t r0 = (uint64_t)sg * seg, r1 = min(rows_c, r0 + seg);
      uint32_t acc = 0;
      for (uint64_t r = r0; r < r1; ++r) acc += tile_get<W>(X, D, r, j);
      if (S > 1) part[t] = acc;
    }
    __syncthreads();
    if (S > 1) {
      for (uint32_t j = threadIdx.x; j < D; j += blockDim.x) {
        uint32_t run = 0;
        for (uint32_t sg = 0; sg < S; ++sg) {
          uint32_t v = part[sg * D + j];
          part[sg * D + j] = run;
          run += v;
        }
      }
    }
    __syncthreads();
    for (uint64_t t = threadIdx.x; t < items; t += blockDim.x) {
      const uint32_t j = (uint32_t)(t % D), sg = (uint32_t)(t / D);
      const uint64_t r0 = (uint64_t)sg * seg, r1 = min(rows_c, r0 + seg);
      uint32_t acc = S > 1 ? part[t] : 0u;
      for (uint64_t r = r0; r < r1; ++r) {
        acc += tile_get<W>(X, D, r, j);
        tile_put<W>(X, D, r, j, acc);
      }
    }
  } else {
    // FIRE: per column, delta_i = wrap_w(floor(alpha * delta_{i-1} / 2^w) + e_i)
    // computed as one multiply-add and shift in 32 bits, x_i = x_{i-1} + delta_i.
    // Double delta: delta_i = wrap_w(delta_{i-1} + e_i).  FIRE per sample:
    // alpha from the accumulator and acc += sign(e_i) * delta_{i-1} at every
    // row (Algorithm 3's per-sample form).
    for (uint32_t j = threadIdx.x; j < D; j += blockDim.x) {
      int32_t acc = 0, dp = 0;
      uint32_t xp = 0;
      for (uint32_t b = 0; b < nb; ++b) {
        const int32_t a = acc >> g.learn_shift;
        const uint32_t A = (uint32_t)a << (32 - 2 * W);
        int32_t gsum = 0;
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          const uint64_t r = (uint64_t)b * kBlockRows + i;
          const int32_t ev = sext<W>(tile_get<W>(X, D, r, j));
          int32_t d;
          if (g.forecaster == kFcDDelta) {
            d = sext<W>((uint32_t)dp + (uint32_t)ev);
          } else if (g.forecaster == kFcFireSample) {
            const uint32_t As = (uint32_t)(acc >> g.learn_shift) << (32 - 2 * W);
            d = (int32_t)(As * (uint32_t)dp + ((uint32_t)ev << (32 - W))) >> (32 - W);
            acc = wrap_acc<W>((int32_t)((uint32_t)acc + (uint32_t)(sign_of(ev) * dp)));
          } else {
            d = (int32_t)(A * (uint32_t)dp + ((uint32_t)ev << (32 - W))) >> (32 - W);
            if ((i & 1) == 0) gsum += sign_of(ev) * dp;
          }
          xp += (uint32_t)d;
          tile_put<W>(X, D, r, j, xp);
          dp = d;
        }
        if (g.forecaster == kFcFire) acc = wrap_acc<W>((int32_t)((uint32_t)acc + (uint32_t)(gsum >> 2)));
      }
    }
  }
  __syncthreads();

  // 5. store
  if (p.staged) {
    if (row0 * D * wb + bytes_c <= p.dst_cap) cta_copy_dec(dst_c, X, bytes_c);
  }
  __syncthreads();
}

template <int W>
__global__ void __launch_bounds__(kDecThreads) k_decode(DecParams p) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint64_t s_data_bytes;
  uint8_t *mem = p.staged ? smem : p.scratch + (uint64_t)blockIdx.x * p.scratch_per_cta;
  const Geom &g = p.g;
  if (threadIdx.x == 0) {
    // the chunk bodies end at tail_off; check it before trusting it
    uint64_t tail_off = le_u64(p.src + 48);
    uint64_t db = tail_off >= g.data_off && tail_off <= p.src_size ? tail_off - g.data_off : 0;
    if (!(tail_off >= g.data_off && tail_off <= p.src_size))
      set_status(p.status, SPRINTZ_ERR_CORRUPT);
    s_data_bytes = db;
  }
  __syncthreads();
  const uint64_t data_bytes = s_data_bytes;
  for (uint32_t c = blockIdx.x; c < g.n_chunks; c += gridDim.x) decode_chunk<W>(p, mem, c, data_bytes);
}

// The stream's 64-byte header agrees with the host's geometry and its sizes
// with the buffer; *tail_off receives the raw tail's offset.
__device__ bool header_matches(const Geom &g, const uint8_t *h, uint64_t src_size, uint64_t *tail_off_out) {
  bool ok = h[0] == 'S' && h[1] == 'P' && h[2] == 'Z' && h[3] == '1' && h[4] == 1 &&
            h[5] == g.w && h[6] == g.forecaster && h[7] == (g.huffman ? 1 : 0) &&
            (h[8] | (h[9] << 8)) == g.D && h[10] == g.G && h[11] == g.learn_shift &&
            le_u32(h + 12) == g.chunk_rows_opt && le_u32(h + 16) == (g.huffman ? g.huff_chunks : 0) &&
            le_u32(h + 20) == g.n_chunks && le_u64(h + 24) == g.rows &&
            le_u32(h + 32) == g.tail_rows && le_u32(h + 36) == 0 && le_u64(h + 40) == g.data_off;
  const uint64_t tail_off = le_u64(h + 48), total = le_u64(h + 56);
  ok = ok && tail_off >= g.data_off && total <= src_size && total == tail_off + g.tail_rows * g.D * g.wb;
  *tail_off_out = tail_off;
  return ok;
}

// Check the device header against the host's geometry and copy the tail.
__global__ void k_decode_header_tail(DecParams p) {
  const Geom &g = p.g;
  __shared__ uint32_t s_ok;
  __shared__ uint64_t s_tail_off;
  if (threadIdx.x == 0) {
    uint64_t tail_off = 0;
    const bool ok = header_matches(g, p.src, p.src_size, &tail_off);
    s_ok = ok;
    s_tail_off = tail_off;
    if (!ok) set_status(p.status, SPRINTZ_ERR_CORRUPT);
  }
  __syncthreads();
  if (!s_ok) return;
  const uint64_t tail_bytes = g.tail_rows * g.D * g.wb;
  uint8_t *d = p.dst + g.full_rows * g.D * g.wb;
  const uint8_t *s = p.src + s_tail_off;
  for (uint64_t k = threadIdx.x; k < tail_bytes; k += blockDim.x) d[k] = s[k];
}

// ---------------------------------------------------------------------------
// Lane-per-column decoder (D <= 32)
//
// A warp decodes K = floor(32 / D) consecutive chunks; lane k*D + j owns
// column j of chunk k for the whole chunk.  The D lanes of a chunk walk its
// header groups together (each reads its own width code; a segmented warp
// scan gives every lane its bit offset and the record's size), read their
// column's bits straight from the stream through L1, and run the inverse
// forecast in registers: FIRE's step delta_i = wrap_w(floor(alpha *
// delta_{i-1} / 2^w) + e_i) is one 32-bit multiply-add and one arithmetic
// shift (alpha pre-shifted by 32 - 2w, e_i by 32 - w).  Each block's rows are
// staged per warp in shared memory and written with 8-byte stores.
// ---------------------------------------------------------------------------


constexpr int kLaneThreads = 128;
constexpr int kLaneWarps = kLaneThreads / 32;


// n (<= 16) bits at bit position `bit` of 4-byte-aligned memory `w`.
__device__ __forceinline__ uint32_t bits_at(const uint32_t *w, uint64_t bit, uint32_t n) {
  const uint32_t *p = w + (bit >> 5);
  uint32_t lo = __ldg(p), hi = __ldg(p + 1);
  return __funnelshift_r(lo, hi, (uint32_t)bit & 31u) & ((1u << n) - 1u);
}

// Bits [bit, bit + n) (n <= 16) of a word array (two aligned 32-bit loads).
__device__ __forceinline__ uint32_t wbits(const uint32_t *w, uint32_t bit, uint32_t mask) {
  const uint32_t *q = w + (bit >> 5);
  return __funnelshift_r(__ldg(q), __ldg(q + 1), bit) & mask;
}

// Bits [bit, bit + n) read bytewise (no byte outside [0, (bit + n + 7) / 8) touched).
__device__ __forceinline__ uint32_t bbits(const uint8_t *b, uint32_t bit, uint32_t mask) {
  const uint8_t *q = b + (bit >> 3);
  const uint32_t n = 32 - __clz(mask);
  const uint32_t s = bit & 7;
  uint32_t v = q[0];
  if (s + n > 8) v |= (uint32_t)q[1] << 8;
  if (s + n > 16) v |= (uint32_t)q[2] << 16;
  return (v >> s) & mask;
}

// Shared-memory ring of the lane decoder: per chunk NSEG segments of SEG
// bytes (powers of two) hold the body bytes at ring offset (address mod
// NSEG*SEG); the segment leader keeps NSEG - 1 segments loading ahead with TMA
// bulk copies, each completing on its slot's mbarrier.
struct LaneRing {
  uint32_t seg;            // segment bytes, >= the largest header group
  uint32_t seg_shift;      // log2(seg)
  uint32_t nseg;           // segments per chunk ring
  uint32_t bars_off;       // per-warp offsets inside the warp's shared region
  uint32_t rings_off;
  uint32_t per_warp;       // bytes of shared memory per warp
  uint32_t mirror;         // bytes after each ring repeating its first bytes
};

constexpr uint32_t kRingWaitLimit = 1u << 22;
// Where a lane's samples go.  With at most 3 columns a row is 1-6 bytes, so
// a lane's per-row stores would each touch a sliver of a sector: those
// specialisations stage a block's rows per warp in shared memory and write
// them as 8-byte words.  Wider rows are stored straight from the lanes.
__host__ __device__ constexpr bool dec_staged(int DT) { return DT >= 1 && DT <= 3; }

// Decode chunk group `warp_id` (K consecutive chunks) of one stream with one
// warp whose shared region (stage, barriers, rings) starts at wsm.
template <int W, int DT>
__device__ __forceinline__ void decode_group(const DecParams &p, const LaneRing &rg, uint64_t warp_id,
                                             uint8_t *wsm) {
  const Geom &g = p.g;
  const uint32_t D = DT ? (uint32_t)DT : g.D;  // columns: a compile-time constant for common D
  const uint32_t K = 32 / D;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t kk = lane / D, j = lane % D;
  const uint32_t kc = kk < K ? kk : K - 1;  // idle lanes alias the last slot, never touch it
  const uint32_t seg0 = lane - j;            // first lane of this chunk's segment
  const uint32_t last = seg0 + D - 1;
  // this chunk's lanes (they take the same branches: their data is shared)
  const uint32_t seg_mask = D == 32 ? 0xFFFFFFFFu : ((1u << D) - 1u) << seg0;
  const uint64_t c64 = p.c_begin + warp_id * K + kk;
  uint8_t *stage = wsm;
  uint64_t *bars = reinterpret_cast<uint64_t *>(wsm + rg.bars_off) + kc * rg.nseg;
  const uint32_t ring_bytes = rg.seg * rg.nseg;
  uint8_t *ring = wsm + rg.rings_off + kc * (ring_bytes + rg.mirror);
  const uint32_t *ring32 = reinterpret_cast<const uint32_t *>(ring);
  const uint32_t wb = W / 8;
  // header bits and layout: compile-time for a specialised column count
  constexpr uint32_t hb = W == 8 ? 3u : 4u;
  const uint32_t G = g.G;
  const bool colmaj = DT ? (DT * W <= 32) : (g.col_major != 0);
  const uint32_t blk_bytes = kBlockRows * D * wb;  // one chunk's block of output
  const uint32_t stage_stride = blk_stage_stride(D, wb);
  const uint32_t gmax = g.hdr_bytes + G * D * W;   // largest header group (bytes)
  constexpr bool kDecDirect = !dec_staged(DT);

  // the chunk bodies end at tail_off
  const uint64_t tail_off = le_u64(p.src + 48);
  const bool hdr_ok = tail_off >= g.data_off && tail_off <= p.src_size;
  const uint64_t data_bytes = hdr_ok ? tail_off - g.data_off : 0;

  bool live = kk < K && c64 < p.c_end && hdr_ok;
  const uint32_t c = (uint32_t)c64;
  uint64_t off = 0, end = 0;
  uint32_t nrec = 0, packed = 0, nb = 0;
  if (live) {
    const uint8_t *e = p.src + kHdrBytes + (uint64_t)c * kEntryBytes;
    off = le_u64(e);
    nrec = le_u32(e + 8);
    packed = le_u32(e + 12);
    end = c + 1 < g.n_chunks ? le_u64(e + kEntryBytes) : data_bytes;
    const uint64_t row0 = (uint64_t)c * g.chunk_rows;
    nb = (uint32_t)(min(g.chunk_rows, g.full_rows - row0) / kBlockRows);
    if (off > end || end > data_bytes || end - off != packed || nrec < 1 || nrec > nb) {
      live = false;
      if (j == 0) set_status(p.status, SPRINTZ_ERR_CORRUPT);
    }
  }
  const uint8_t *body = p.src + g.data_off + off;

  // ---- ring set-up: the leader initialises the barriers and starts loading
  const uintptr_t B0 = (uintptr_t)body, B1 = B0 + packed;
  const uintptr_t buf_lo = ((uintptr_t)p.src + 15) & ~(uintptr_t)15;
  const uintptr_t buf_hi = ((uintptr_t)p.src + p.src_size) & ~(uintptr_t)15;
  const uint32_t ssh = rg.seg_shift;
  const uint64_t s_lo = live ? B0 >> ssh : 0, s_hi = live ? (B1 - 1) >> ssh : 0;
  // segment counters relative to the body's first segment s_lo
  const uint32_t n_segs = live ? (uint32_t)(s_hi - s_lo) + 1 : 0u;
  const uint32_t b0r = (uint32_t)(B0 & (rg.seg - 1));  // body start inside its first segment
  const uint32_t slot0 = (uint32_t)s_lo;
  uint32_t seg_base = 0, seg_issued = 0, seg_waited = 0;
  uint32_t parity = 0;  // bit h: parity of the next completion of slot h
  bool ring_ok = true;
  if (live && j == 0) {
    for (uint32_t h = 0; h < rg.nseg; ++h) mbar_init(&bars[h], 1);
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  __syncwarp();
  // issue the load of segment s into its slot (leader lane)
  auto issue = [&](uint64_t s) {
    const uint32_t h = (uint32_t)(s & (rg.nseg - 1));
    uintptr_t a = max((uintptr_t)(s << ssh), max(B0 & ~(uintptr_t)15, buf_lo));
    uintptr_t b = min((uintptr_t)((s + 1) << ssh), min((B1 + 15) & ~(uintptr_t)15, buf_hi));
    const uint32_t bytes = b > a ? (uint32_t)(b - a) : 0u;
    // slot 0's first bytes also go to the mirror after the ring, so that a
    // header group that wraps around reads on linearly
    const uintptr_t s0 = (uintptr_t)(s << ssh);
    const uintptr_t mb = h == 0 ? min(b, s0 + rg.mirror) : a;
    const uint32_t mbytes = mb > a ? (uint32_t)(mb - a) : 0u;
    mbar_arrive_expect_tx(&bars[h], bytes + mbytes);
    if (bytes) tma_load_1d(ring + (a & (ring_bytes - 1)), reinterpret_cast<const void *>(a), bytes, &bars[h]);
    if (mbytes) tma_load_1d(ring + ring_bytes + (a - s0), reinterpret_cast<const void *>(a), mbytes, &bars[h]);
    // body bytes in the buffer's last partial 16-byte unit: plain loads
    const uintptr_t t0 = max(buf_hi, max((uintptr_t)(s << ssh), B0));
    const uintptr_t t1 = min(B1, (uintptr_t)((s + 1) << ssh));
    for (uintptr_t q = t0; q < t1; ++q) {
      const uint8_t v = *reinterpret_cast<const uint8_t *>(q);
      ring[q & (ring_bytes - 1)] = v;
      if (h == 0 && q - s0 < rg.mirror) ring[ring_bytes + (q - s0)] = v;
    }
  };
  auto wait_upto = [&](uint32_t s) {
    while (seg_waited <= s && seg_waited < seg_issued) {
      const uint32_t h = (slot0 + seg_waited) & (rg.nseg - 1);
      if (!mbar_wait(&bars[h], (parity >> h) & 1u, kRingWaitLimit)) {
        ring_ok = false;
        return;
      }
      parity ^= 1u << h;
      seg_waited++;
    }
  };
  if (live) {
    const uint32_t first_end = min(n_segs, rg.nseg);
    if (j == 0)
      for (uint32_t r = 0; r < first_end; ++r) issue(s_lo + r);
    seg_issued = first_end;
  }
  // L2 prefetch ahead of the ring (segment leader)
  const uint32_t kPrefetchWin = p.pf_win;
  uintptr_t pf_end = B0 + (uintptr_t)rg.seg * rg.nseg;
  if (live && j == 0 && pf_end < B1) {
    const uintptr_t e2 = min(B1, pf_end + kPrefetchWin);
    prefetch_l2_range(pf_end & ~(uintptr_t)15, e2, buf_lo, buf_hi);
    pf_end = e2;
  }
  // ring bit of body bit `bit` inside the current header group: the group's
  // ring position plus the offset into it (mod 2^32), never past the mirror
  const uint32_t b0ring = (uint32_t)(B0 & (ring_bytes - 1));
  uint32_t gq = b0ring * 8;
  auto rbits = [&](uint32_t bit, uint32_t mask) {
    const uint32_t q = gq + bit;
    const uint32_t i0 = q >> 5;
    return __funnelshift_r(ring32[i0], ring32[i0 + 1], q) & mask;
  };

  // output mapping of this lane's (up to two) 8-byte words of each block step
  uint64_t *dptr[2];
  uint32_t src_word[2], from_lane[2];
  bool has[2];
  const uint32_t words_per = blk_bytes / 8, total_words = K * words_per;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const uint32_t q = lane + 32 * t;
    has[t] = q < total_words;
    const uint32_t k2 = has[t] ? q / words_per : 0;
    const uint32_t wq = has[t] ? q % words_per : 0;
    from_lane[t] = k2 * D;
    src_word[t] = k2 * (stage_stride / 8) + wq;
    const uint64_t r2 = (warp_id * K + k2) * g.chunk_rows;  // rows from chunk c_begin
    dptr[t] = reinterpret_cast<uint64_t *>(p.dst + r2 * D * wb) + wq;
  }
  const uint32_t row_stride = D * wb;
  // kDecDirect: each lane stores its samples straight to global memory;
  // otherwise a block's rows are staged and written as 8-byte words
  uint8_t *my_stage = kDecDirect ? p.dst + (warp_id * K + kc) * (uint64_t)g.chunk_rows * row_stride + j * wb
                                 : stage + kc * stage_stride + j * wb;
  auto put = [&](int i, uint32_t v) {
    if (W == 8)
      my_stage[i * row_stride] = (uint8_t)v;
    else
      *reinterpret_cast<uint16_t *>(my_stage + i * row_stride) = (uint16_t)v;
  };

  // walk state (body-relative bytes / bits)
  uint32_t gpos = 0, hdr = 0;
  uint32_t gslot = G, rec = 0, rem = 0;
  uint32_t pbit = 0, stride = 0, mask = 0;
  bool bad_any = false;
  // forecaster state
  uint32_t xp = 0;
  int32_t dp = 0, acc = 0;

  const uint32_t nb_max = (uint32_t)(min(g.chunk_rows, g.full_rows) / kBlockRows);
  for (uint32_t b = 0; b < nb_max; ++b) {
    const bool here = live && b < nb;
    const bool need = here && rem == 0;
    // a new record: its header group first (ring upkeep), then every lane
    // reads its width code and the full warp scans them (lanes without a
    // new record contribute nothing that is used)
    if (need && gslot == G) {
      {
        hdr = gpos;
        gpos += g.hdr_bytes;
        gslot = 0;
        gq = ((b0ring + hdr) & (ring_bytes - 1)) * 8 - hdr * 8;
        // ring: release segments before the group, load ahead, wait for the group
        const uint32_t r_cur = (b0r + hdr) >> ssh;
        if (seg_base < r_cur) {
          wait_upto(r_cur - 1);
          ring_ok = __all_sync(seg_mask, ring_ok);
          if (j == 0) fence_proxy_async_smem();
          while (seg_base < r_cur) {
            const uint32_t r_new = seg_base + rg.nseg;
            if (r_new < n_segs) {
              if (j == 0) issue(s_lo + r_new);
              seg_issued = r_new + 1;
            }
            seg_base++;
          }
          if (j == 0 && pf_end < B1 && hdr + rg.seg * rg.nseg + kPrefetchWin / 2 > (uint32_t)(pf_end - B0)) {
            const uintptr_t e2 = min(B1, pf_end + kPrefetchWin);
            prefetch_l2_range(pf_end & ~(uintptr_t)15, e2, buf_lo, buf_hi);
            pf_end = e2;
          }
        }
        // wait for the group's last segment unless it already arrived (the
        // condition is the same in every lane of the chunk)
        const uint32_t r_need = min(n_segs - 1, (b0r + hdr + gmax - 1) >> ssh);
        if (r_need >= seg_waited && seg_waited < seg_issued) {
          wait_upto(r_need);
          ring_ok = __all_sync(seg_mask, ring_ok);
        }
      }
    }
    // every lane reads its width code (reads stay inside the current group:
    // a group spans at most gmax bytes whatever the data) and the full warp
    // scans them; lanes without a new record contribute nothing that is used
    const uint32_t raw = rbits(hdr * 8 + (gslot * D + j) * hb, (1u << hb) - 1u);
    const uint32_t code = need ? raw : 0u;
    const uint32_t nw = code == (uint32_t)W - 1 ? (uint32_t)W : code;
    uint32_t v = nw;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      if (o < D) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (j >= o) v += t;
      }
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, v, last);
    // the new record, in select form: a zero-block run (all widths zero, a
    // u16 count) or a block whose column starts at bit pbit with rows stride
    // bits apart.  The walk stays in bounds whatever the data; a record or
    // byte count that overruns shows in the totals checked at the chunk's
    // end, a zero run count here.
    {
      const bool isrun = total == 0;
      const uint32_t cnt = rbits(gpos * 8, 0xFFFFu);
      const uint32_t prefix = v - nw;
      const uint32_t size = colmaj ? total : 8 * ((total + 7) / 8);
      const uint32_t rsize = isrun ? 2u : size;
      const uint32_t pb = colmaj ? (gpos + prefix) * 8 : gpos * 8 + prefix;
      bad_any |= need && isrun && cnt == 0;
      rem = need ? (isrun ? cnt : 1u) : rem;
      mask = need ? (isrun ? 0u : (1u << nw) - 1u) : mask;
      pbit = need ? (isrun ? gpos * 8 : pb) : pbit;
      stride = need ? (isrun ? 0u : (colmaj ? nw : size)) : stride;
      gpos += need ? rsize : 0u;
      gslot += need ? 1u : 0u;
      rec += need ? 1u : 0u;
    }
    const bool emit = here;
    if (emit) {
      // zigzagged errors of this lane's column, 8 rows (all zero in a run:
      // mask 0)
      uint32_t z[kBlockRows];
      if (W == 8 && DT != 0 && DT * W <= 32) {
        // column-major u8: the 8 values (stride = n <= 8 bits each) are
        // contiguous, 64 bits at most: three words, two funnel shifts, and
        // values 4..7 from the window 4n bits on
        const uint32_t q = gq + pbit;
        const uint32_t i0 = q >> 5;
        const uint32_t a0 = ring32[i0], a1 = ring32[i0 + 1], a2 = ring32[i0 + 2];
        const uint32_t lo = __funnelshift_r(a0, a1, q), hi = __funnelshift_r(a1, a2, q);
        const uint32_t mid = __funnelshift_rc(lo, hi, 4 * stride);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          z[i] = (lo >> (i * stride)) & mask;
          z[i + 4] = (mid >> (i * stride)) & mask;
        }
      } else {
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) z[i] = rbits(pbit + i * stride, mask);
      }
      if (g.forecaster == kFcDelta) {
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          xp += (z[i] >> 1) ^ (0u - (z[i] & 1u));
          put(i, xp);
        }
      } else if (g.forecaster == kFcDDelta) {
        // double delta: delta_i = wrap_w(delta_{i-1} + e_i)
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          const uint32_t ev = (z[i] >> 1) ^ (0u - (z[i] & 1u));
          const int32_t d = sext<W>((uint32_t)dp + ev);
          xp += (uint32_t)d;
          put(i, xp);
          dp = d;
        }
      } else if (g.forecaster == kFcFireSample) {
        // Algorithm 3 at every sample: alpha from the accumulator, the
        // delta as in the block form, then acc += sign(e_i) * delta_{i-1}
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          const uint32_t A = (uint32_t)(acc >> g.learn_shift) << (32 - 2 * W);
          const uint32_t ev = (z[i] >> 1) ^ (0u - (z[i] & 1u));
          const int32_t d = (int32_t)(A * (uint32_t)dp + (ev << (32 - W))) >> (32 - W);
          const int32_t sg = z[i] == 0 ? 0 : ((z[i] & 1u) ? -dp : dp);
          acc = wrap_acc<W>((int32_t)((uint32_t)acc + (uint32_t)sg));
          xp += (uint32_t)d;
          put(i, xp);
          dp = d;
        }
      } else {
        // delta_i = wrap_w(floor(alpha * delta_{i-1} / 2^w) + e_i): one
        // multiply-add and one shift on 32-bit values pre-shifted by 32 - w
        const uint32_t A = (uint32_t)(acc >> g.learn_shift) << (32 - 2 * W);
        int32_t gsum = 0;
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          const uint32_t ev = (z[i] >> 1) ^ (0u - (z[i] & 1u));  // e_i, two's complement
          const int32_t d = (int32_t)(A * (uint32_t)dp + (ev << (32 - W))) >> (32 - W);
          if ((i & 1) == 0) gsum += z[i] == 0 ? 0 : ((z[i] & 1u) ? -dp : dp);
          xp += (uint32_t)d;
          put(i, xp);
          dp = d;
        }
        acc = wrap_acc<W>((int32_t)((uint32_t)acc + (uint32_t)(gsum >> 2)));
      }
      rem--;
    }
    if (kDecDirect) {
      my_stage += kBlockRows * row_stride;
    } else {
      __syncwarp();
      // block rows of every chunk of the warp: 8-byte words
      const uint32_t boff = b * (blk_bytes / 8);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const bool e2 = __shfl_sync(0xFFFFFFFFu, emit, from_lane[t]);
        if (has[t] && e2) dptr[t][boff] = reinterpret_cast<const uint64_t *>(stage)[src_word[t]];
      }
      __syncwarp();
    }
  }
  // every record consumed, the body used up, no run past the chunk's end,
  // unused slots of the last group zero
  if (live) {
    bool bad = bad_any || rec != nrec || gpos != packed || rem != 0;
    for (uint32_t s = gslot; s < G && !bad; ++s)
      bad |= rbits(hdr * 8 + (s * D + j) * hb, (1u << hb) - 1u) != 0;
    if (bad || !ring_ok) set_status(p.status, ring_ok ? SPRINTZ_ERR_CORRUPT : SPRINTZ_ERR_TIMEOUT);
  }
  // no bulk copy may still be writing this warp's shared memory when it is
  // reused or the CTA exits; then the barriers are retired
  if (kk < K && c64 < p.c_end && hdr_ok) {
    ring_ok = true;
    wait_upto(0xFFFFFFFFu);
    if (!ring_ok && j == 0) set_status(p.status, SPRINTZ_ERR_TIMEOUT);
    if (j == 0 && seg_issued > 0)
      for (uint32_t h = 0; h < rg.nseg; ++h) mbar_inval(&bars[h]);
  }
  __syncwarp();
}

template <int W, int DT>
__global__ void __launch_bounds__(kLaneThreads, 7) k_decode_lanes(DecParams p, LaneRing rg) {
  extern __shared__ __align__(16) uint8_t dsm[];
  const uint32_t warp = threadIdx.x >> 5;
  const DecParams pp = p;
  const LaneRing rr = rg;
  decode_group<W, DT>(pp, rr, (uint64_t)blockIdx.x * kLaneWarps + warp, dsm + (uint64_t)warp * rr.per_warp);
}

// The lane decoder specialised for the column count (0: any D <= 32).
template <int W>
static const void *lane_decoder(uint32_t D) {
  switch (D) {
    case 1: return (const void *)k_decode_lanes<W, 1>;
    case 2: return (const void *)k_decode_lanes<W, 2>;
    case 3: return (const void *)k_decode_lanes<W, 3>;
    case 4: return (const void *)k_decode_lanes<W, 4>;
    case 8: return (const void *)k_decode_lanes<W, 8>;
    case 16: return (const void *)k_decode_lanes<W, 16>;
    default: return (const void *)k_decode_lanes<W, 0>;
  }
}

// ---------------------------------------------------------------------------
// Column-per-thread decoder for wide rows (32 < D <= 1024)
//
// One CTA decodes one chunk; thread j owns column j.  The chunk's record
// state is the same in every thread.  At each header group the CTA copies
// the group's bytes (at most gmax) into shared memory; every thread reads its
// width code there, a block-wide scan of the widths gives its bit offset and
// the record's size, and each thread unpacks, un-zigzags and inverts its
// column's forecast in registers, writing its samples of each row (the
// threads of a row write consecutive samples).
// ---------------------------------------------------------------------------

template <int W>
__global__ void __launch_bounds__(1024) k_decode_wide(DecParams p) {
  extern __shared__ __align__(16) uint8_t gsm[];  // the current header group (+ 8 spare bytes)
  __shared__ uint32_t s_wsum[2][32];              // per-warp width sums, two records in turn
  const Geom &g = p.g;
  const uint32_t D = g.D, j = threadIdx.x, lane = j & 31, warp = j >> 5;
  const uint32_t nwarps = blockDim.x >> 5;
  const bool col = j < D;
  constexpr uint32_t wb = W / 8;
  const uint32_t hb = g.hb, G = g.G, H = g.hdr_bytes;
  const uint32_t gmax = H + G * D * W;
  const uint64_t c = (uint64_t)p.c_begin + blockIdx.x;
  if (c >= p.c_end) return;

  const uint64_t tail_off = le_u64(p.src + 48);
  const bool hdr_ok = tail_off >= g.data_off && tail_off <= p.src_size;
  const uint64_t data_bytes = hdr_ok ? tail_off - g.data_off : 0;
  const uint8_t *e = p.src + kHdrBytes + c * kEntryBytes;
  const uint64_t off = le_u64(e);
  const uint32_t nrec = le_u32(e + 8);
  const uint32_t packed = le_u32(e + 12);
  const uint64_t end = c + 1 < g.n_chunks ? le_u64(e + kEntryBytes) : data_bytes;
  const uint64_t row0 = c * g.chunk_rows;
  const uint32_t nb = (uint32_t)(min((uint64_t)g.chunk_rows, g.full_rows - row0) / kBlockRows);
  if (!hdr_ok || off > end || end > data_bytes || end - off != packed || nrec < 1 || nrec > nb) {
    if (j == 0) set_status(p.status, SPRINTZ_ERR_CORRUPT);
    return;
  }
  const uint8_t *body = p.src + g.data_off + off;
  const uint32_t *g32 = reinterpret_cast<const uint32_t *>(gsm);
  uint32_t hdr = 0;  // body offset of the staged group
  // bits [bit, bit + n) of the body, bit inside the staged group
  auto rbits = [&](uint32_t bit, uint32_t mask) {
    const uint32_t q = bit - hdr * 8;
    const uint32_t i0 = q >> 5;
    return __funnelshift_r(g32[i0], g32[i0 + 1], q) & mask;
  };
  uint8_t *out = p.dst + (row0 - (uint64_t)p.c_begin * g.chunk_rows) * D * wb + j * wb;
  const uint32_t row_stride = D * wb;

  uint32_t gpos = 0, gslot = G, rec = 0, rem = 0, pbit = 0, stride = 0, mask = 0, par = 0;
  bool bad_any = false;
  uint32_t xp = 0;
  int32_t dp = 0, acc = 0;
  for (uint32_t b = 0; b < nb; ++b) {
    if (rem == 0) {
      if (gslot == G) {
        // stage the next group: [gpos, gpos + gmax) clipped to the body
        hdr = gpos;
        gpos += H;
        gslot = 0;
        __syncthreads();  // every thread is done with the previous group
        const uint32_t n = hdr < packed ? min(gmax, packed - hdr) : 0u;
        for (uint32_t k = j; k < (gmax + 8 + 3) / 4; k += blockDim.x) {
          uint32_t v = 0;
          for (uint32_t t = 0; t < 4; ++t) {
            const uint32_t q = 4 * k + t;
            if (q < n) v |= (uint32_t)body[hdr + q] << (8 * t);
          }
          reinterpret_cast<uint32_t *>(gsm)[k] = v;
        }
        __syncthreads();
      }
      const bool hdr_in = gpos <= packed;
      const uint32_t code = col && hdr_in ? rbits(hdr * 8 + (gslot * D + j) * hb, (1u << hb) - 1u) : 0u;
      const uint32_t nw = code == (uint32_t)W - 1 ? (uint32_t)W : code;
      // block-wide exclusive scan of the widths
      uint32_t v = nw;
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
      const uint32_t prefix = v - nw + (warp ? s_wsum[par][warp - 1] : 0u);
      const uint32_t total = s_wsum[par][nwarps - 1];
      par ^= 1;
      // the record: a zero-block run (u16 count) or a block
      const bool isrun = total == 0;
      const uint32_t cnt = rbits(gpos * 8, 0xFFFFu);
      const uint32_t size = g.col_major ? total : 8 * ((total + 7) / 8);
      const uint32_t rsize = isrun ? 2u : size;
      bad_any |= rec >= nrec || !hdr_in || gpos + rsize > packed || (isrun && (cnt == 0 || b + cnt > nb));
      rem = isrun ? cnt : 1u;
      mask = isrun ? 0u : (1u << nw) - 1u;
      pbit = isrun ? gpos * 8 : (g.col_major ? (gpos + prefix) * 8 : gpos * 8 + prefix);
      stride = isrun ? 0u : (g.col_major ? nw : size);
      gpos += rsize;
      gslot++;
      rec++;
    }
    if (col) {
      uint32_t z[kBlockRows];
#pragma unroll
      for (int i = 0; i < kBlockRows; ++i) z[i] = rbits(pbit + i * stride, mask);
      uint8_t *ob = out + (uint64_t)b * kBlockRows * row_stride;
      auto put = [&](int i, uint32_t x) {
        if (W == 8)
          ob[i * row_stride] = (uint8_t)x;
        else
          *reinterpret_cast<uint16_t *>(ob + i * row_stride) = (uint16_t)x;
      };
      if (g.forecaster == kFcDelta) {
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          xp += (z[i] >> 1) ^ (0u - (z[i] & 1u));
          put(i, xp);
        }
      } else if (g.forecaster == kFcDDelta) {
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          const int32_t d = sext<W>((uint32_t)dp + ((z[i] >> 1) ^ (0u - (z[i] & 1u))));
          xp += (uint32_t)d;
          put(i, xp);
          dp = d;
        }
      } else if (g.forecaster == kFcFireSample) {
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          const uint32_t A = (uint32_t)(acc >> g.learn_shift) << (32 - 2 * W);
          const uint32_t ev = (z[i] >> 1) ^ (0u - (z[i] & 1u));
          const int32_t d = (int32_t)(A * (uint32_t)dp + (ev << (32 - W))) >> (32 - W);
          acc = wrap_acc<W>((int32_t)((uint32_t)acc + (uint32_t)(z[i] == 0 ? 0 : ((z[i] & 1u) ? -dp : dp))));
          xp += (uint32_t)d;
          put(i, xp);
          dp = d;
        }
      } else {
        const uint32_t A = (uint32_t)(acc >> g.learn_shift) << (32 - 2 * W);
        int32_t gsum = 0;
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          const uint32_t ev = (z[i] >> 1) ^ (0u - (z[i] & 1u));
          const int32_t d = (int32_t)(A * (uint32_t)dp + (ev << (32 - W))) >> (32 - W);
          if ((i & 1) == 0) gsum += z[i] == 0 ? 0 : ((z[i] & 1u) ? -dp : dp);
          xp += (uint32_t)d;
          put(i, xp);
          dp = d;
        }
        acc = wrap_acc<W>((int32_t)((uint32_t)acc + (uint32_t)(gsum >> 2)));
      }
    }
    rem--;
  }
  // every record consumed, the body used up, unused slots of the last group zero
  bool bad = bad_any || rec != nrec || gpos != packed;
  if (!bad && col)
    for (uint32_t s = gslot; s < G && !bad; ++s) bad |= rbits(hdr * 8 + (s * D + j) * hb, (1u << hb) - 1u) != 0;
  if (bad) set_status(p.status, SPRINTZ_ERR_CORRUPT);
}

// One stream of a batched decode.
struct DecBatchItem {
  DecParams p;
  LaneRing rg;
  // range request (row_end > row_begin): p.dst is a temporary holding the
  // covering chunks; rows [row_begin, row_end) then go to out
  uint64_t row_begin, row_end;
  uint8_t *out;
};

static_assert(sizeof(DecBatchItem) % 8 == 0, "descriptors are copied in 8-byte words");

// One chunk group of a batch item through the lane decoder specialised for
// its column count (a call per group keeps each variant's code apart).  The
// warp's region arrives as an offset into the dynamic shared memory, so that
// the callee addresses it as shared memory rather than through generic
// pointers.
template <int W, int DT>
__device__ __noinline__ void decode_batch_group(const DecBatchItem &it, uint64_t grp, uint32_t wsm_off) {
  extern __shared__ __align__(16) uint8_t dsm[];
  decode_group<W, DT>(it.p, it.rg, grp, dsm + wsm_off);
}

// Variant table: [w == 16][D] (D = 0: any column count up to 32).  One
// indirect call site for every variant keeps the kernel's frame small.
typedef void (*DecBatchGroupFn)(const DecBatchItem &, uint64_t, uint32_t);
#define SPZ_DEC_ROW(W)                                                                                  \
  {decode_batch_group<W, 0>,  decode_batch_group<W, 1>,  decode_batch_group<W, 2>,                      \
   decode_batch_group<W, 3>,  decode_batch_group<W, 4>,  decode_batch_group<W, 5>,                      \
   decode_batch_group<W, 6>,  decode_batch_group<W, 7>,  decode_batch_group<W, 8>,                      \
   decode_batch_group<W, 9>,  decode_batch_group<W, 10>, decode_batch_group<W, 11>,                     \
   decode_batch_group<W, 12>, decode_batch_group<W, 13>, decode_batch_group<W, 14>,                     \
   decode_batch_group<W, 15>, decode_batch_group<W, 16>}
__device__ DecBatchGroupFn g_dec_batch_fns[2][17] = {SPZ_DEC_ROW(8), SPZ_DEC_ROW(16)};
#undef SPZ_DEC_ROW

// Batched decode: persistent warps take work entries (stream, chunk group),
// one ticket per (w, D) class, from their SM's home class first; each warp
// copies its item's descriptor into shared memory once per group.  Bounded at
// 6 CTAs per SM (80 registers): the per-D callees hold the stream's
// descriptor fields in registers, which the single-stream kernels read from
// the constant bank, and at 72 registers they reload some of them from local
// memory inside the block loop (measured 2-3 % slower; 64 registers spill far
// more and are 15 % slower).
__global__ void __launch_bounds__(kLaneThreads, 6) k_decode_batch(const DecBatchItem *items,
                                                                 const BatchClasses *classes,
                                                                 const uint64_t *work, uint32_t *tickets,
                                                                 uint32_t per_warp) {
  extern __shared__ __align__(16) uint8_t dsm[];
  __shared__ __align__(16) DecBatchItem s_it[kLaneWarps];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wsm_off = warp * per_warp;
  constexpr uint32_t kWords = sizeof(DecBatchItem) / 8;
  uint32_t c = batch_home(classes);
  uint64_t e = 0;
  while (batch_next(classes, work, tickets, c, &e)) {
    const uint32_t s = (uint32_t)(e >> kWorkGroupBits);
    const uint64_t grp = e & ((1ull << kWorkGroupBits) - 1);
    const uint64_t *from = reinterpret_cast<const uint64_t *>(items + s);
    uint64_t *to = reinterpret_cast<uint64_t *>(&s_it[warp]);
    for (uint32_t k = lane; k < kWords; k += 32) to[k] = __ldg(from + k);
    __syncwarp();
    const DecBatchItem &it = s_it[warp];
    const uint32_t D = it.p.g.D;
    g_dec_batch_fns[it.p.g.w == 16][D <= 16 ? D : 0](it, grp, wsm_off);
    __syncwarp();
  }
}

// Range requests: copy rows [row_begin, row_end) from the decoded covering
// chunks (and the raw trailing rows) to the request's output.
__global__ void k_decode_batch_rows(const DecBatchItem *items) {
  const DecBatchItem &it = items[blockIdx.y];
  if (it.row_end <= it.row_begin) return;
  const Geom &g = it.p.g;
  const uint64_t rb = (uint64_t)g.D * g.wb;
  const uint64_t r_full = min(it.row_end, g.full_rows);
  const uint64_t base_row = (uint64_t)it.p.c_begin * g.chunk_rows;
  const uint64_t n_mid = r_full > it.row_begin ? (r_full - it.row_begin) * rb : 0;
  const uint8_t *from = it.p.dst + (it.row_begin - base_row) * rb;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_mid;
       k += (uint64_t)gridDim.x * blockDim.x)
    it.out[k] = from[k];
  if (it.row_end > g.full_rows && blockIdx.x == 0) {
    const uint64_t t0 = max(it.row_begin, g.full_rows);
    const uint64_t tail_off = le_u64(it.p.src + 48);
    const uint64_t nb = (it.row_end - t0) * rb;
    const uint8_t *tail = it.p.src + tail_off + (t0 - g.full_rows) * rb;
    if (tail_off + (g.tail_rows * rb) <= it.p.src_size)
      for (uint64_t k = threadIdx.x; k < nb; k += blockDim.x) it.out[n_mid + k] = tail[k];
  }
}

// Header check and raw tail of every stream of a batch (one CTA per stream).
__global__ void k_decode_batch_tails(const DecBatchItem *items) {
  const bool ranged = items[blockIdx.x].row_end > items[blockIdx.x].row_begin;
  const DecParams &p = items[blockIdx.x].p;
  const Geom &g = p.g;
  __shared__ uint32_t s_ok;
  __shared__ uint64_t s_tail_off;
  if (threadIdx.x == 0) {
    const uint8_t *h = p.src;
    bool ok = h[0] == 'S' && h[1] == 'P' && h[2] == 'Z' && h[3] == '1' && h[4] == 1 &&
              h[5] == g.w && h[6] == g.forecaster && h[7] == (g.huffman ? 1 : 0) &&
              (h[8] | (h[9] << 8)) == g.D && h[10] == g.G && h[11] == g.learn_shift &&
              le_u32(h + 12) == g.chunk_rows_opt && le_u32(h + 16) == (g.huffman ? g.huff_chunks : 0) &&
              le_u32(h + 20) == g.n_chunks && le_u64(h + 24) == g.rows &&
              le_u32(h + 32) == g.tail_rows && le_u32(h + 36) == 0 && le_u64(h + 40) == g.data_off;
    const uint64_t tail_off = le_u64(h + 48), total = le_u64(h + 56);
    ok = ok && tail_off >= g.data_off && total <= p.src_size && total == tail_off + g.tail_rows * g.D * g.wb;
    s_ok = ok;
    s_tail_off = tail_off;
    if (!ok) set_status(p.status, SPRINTZ_ERR_CORRUPT);
  }
  __syncthreads();
  if (!s_ok || ranged) return;
  const uint64_t tail_bytes = g.tail_rows * g.D * g.wb;
  uint8_t *d = p.dst + g.full_rows * g.D * g.wb;
  const uint8_t *src = p.src + s_tail_off;
  for (uint64_t k = threadIdx.x; k < tail_bytes; k += blockDim.x) d[k] = src[k];
}

// min_seg: smallest ring segment (a power of two >= 64); the batched decoder
// takes 64 so that the rings of its narrowest streams (D = 1: 32 chunks per
// warp) do not set the shared memory of every warp.
static LaneRing lane_ring_plan(const Geom &g, const LaunchCfg &cfg, uint32_t nseg_want, bool staged,
                               uint32_t min_seg = 128) {
  LaneRing r{};
  const uint32_t K = 32 / g.D;
  const uint32_t gmax = g.hdr_bytes + g.G * g.D * g.w;
  r.seg = 64;
  r.seg_shift = 6;
  while (r.seg < min_seg) {
    r.seg <<= 1;
    r.seg_shift++;
  }
  // a group plus the words read past its end: 4 bytes, or 12 for the u8
  // column-major records read as three words
  const uint32_t slack = (g.w == 8 && g.col_major) ? 16u : 8u;
  r.mirror = (gmax + slack + 15) & ~15u;
  while (r.seg < r.mirror) {
    r.seg <<= 1;
    r.seg_shift++;
  }
  r.nseg = nseg_want;
  auto layout = [&](LaneRing &x) {
    x.bars_off = staged ? (K * blk_stage_stride(g.D, g.wb) + 15) & ~15u : 0u;
    x.rings_off = x.bars_off + ((K * x.nseg * 8 + 15) & ~15u);
    x.per_warp = x.rings_off + K * (x.nseg * x.seg + x.mirror);
  };
  layout(r);
  while (r.nseg > 2 && (uint64_t)r.per_warp * kLaneWarps > 64 * 1024) {
    r.nseg >>= 1;
    layout(r);
  }
  if ((uint64_t)r.per_warp * kLaneWarps > (uint64_t)cfg.max_smem_optin) r.per_warp = 0;  // does not fit
  return r;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

static uint64_t align256d(uint64_t v) { return (v + 255) & ~255ull; }

// Segments per chunk ring of the lane decoder (SPRINTZ_DEC_RING_SEGS: 2 or 4).
static uint32_t dec_ring_segments() {
  static const uint32_t v = [] {
    const char *e = getenv("SPRINTZ_DEC_RING_SEGS");
    int x = e ? atoi(e) : 0;
    return (uint32_t)(x == 2 || x == 4 || x == 8 ? x : 2);
  }();
  return v;
}

struct DecPlan {
  bool staged;
  uint64_t smem;
  uint32_t grid;
  uint64_t scratch_per_cta;
};

static DecPlan dec_plan(const Geom &g, const LaunchCfg &cfg) {
  DecPlan pl{};
  DecLayout Ls = dec_layout(g, true);
  const uint64_t smem_limit = std::min<uint64_t>((uint64_t)cfg.max_smem_optin, 200u * 1024);
  pl.staged = Ls.total <= smem_limit;
  if (pl.staged) {
    pl.smem = Ls.total;
    const void *fn = g.w == 8 ? (const void *)k_decode<8> : (const void *)k_decode<16>;
    if (pl.smem > 48 * 1024)
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    pl.grid = (uint32_t)std::min<uint64_t>(g.n_chunks, 1u << 30);
    pl.scratch_per_cta = 0;
  } else {
    pl.smem = 0;
    pl.grid = (uint32_t)std::min<uint64_t>(g.n_chunks, (uint64_t)cfg.sm_count * 2);
    pl.scratch_per_cta = align256d(dec_layout(g, false).total);
  }
  if (pl.grid == 0) pl.grid = 1;
  return pl;
}

// ---- batches ----------------------------------------------------------------

int plan_batch_decode(const sprintz_batch_item *items, uint32_t n, const LaunchCfg &cfg,
                      const sprintz_schedule &sched_in, int *d_status, uint8_t *ws, BatchPlan *pl,
                      std::vector<uint8_t> *img, std::vector<uint64_t> *work) {
  if (n > kMaxBatchStreams) return SPRINTZ_ERR_INVALID_ARG;
  sprintz_schedule sched = batch_default_schedule(0);
  if (sched_in.ctas_per_sm) sched.ctas_per_sm = sched_in.ctas_per_sm;
  if (sched_in.ring_segments == 2 || sched_in.ring_segments == 4) sched.ring_segments = sched_in.ring_segments;
  if (sched_in.prefetch_bytes) sched.prefetch_bytes = sched_in.prefetch_bytes == 1 ? 1u : sched_in.prefetch_bytes & ~15u;
  if (sched_in.order >= 1 && sched_in.order <= 3) sched.order = sched_in.order;
  std::vector<DecBatchItem> v(n);
  std::vector<uint64_t> temp_off(n, 0);
  std::vector<uint32_t> vw(n), vD(n);
  std::vector<uint64_t> vgroups(n);
  uint64_t temp_total = 0;
  bool any_ranged = false;
  uint32_t region = 0;
  const uint32_t win = sched.prefetch_bytes == 1 ? 0u : sched.prefetch_bytes;
  for (uint32_t i = 0; i < n; ++i) {
    const sprintz_batch_item &it = items[i];
    Geom g;
    int rc = make_geom(it.rows, it.D, it.w, &it.opts, &g);
    if (rc != SPRINTZ_OK) return rc;
    if (it.opts.huffman || g.D > 32 || g.max_body >= (1ull << 28)) return SPRINTZ_ERR_UNSUPPORTED;
    const bool ranged = it.row_end > it.row_begin;
    if (ranged && it.row_end > it.rows) return SPRINTZ_ERR_INVALID_ARG;
    const uint64_t want_rows = ranged ? it.row_end - it.row_begin : it.rows;
    if (!it.src || (want_rows && !it.dst)) return SPRINTZ_ERR_INVALID_ARG;
    if (!ranged && ((uintptr_t)it.dst & 7) != 0) return SPRINTZ_ERR_UNSUPPORTED;
    if (it.dst_cap < want_rows * it.D * g.wb) return SPRINTZ_ERR_DST_TOO_SMALL;
    if (it.src_bytes < g.data_off) return SPRINTZ_ERR_CORRUPT;
    DecBatchItem &d = v[i];
    memset(&d, 0, sizeof(d));
    d.p.src = (const uint8_t *)it.src;
    d.p.src_size = it.src_bytes;
    d.p.dst = (uint8_t *)it.dst;
    d.p.dst_cap = it.dst_cap;
    d.p.status = d_status;
    d.p.g = g;
    d.p.pf_win = win;
    d.p.c_begin = 0;
    d.p.c_end = g.n_chunks;
    if (ranged) {
      // decode the chunks covering the rows into a temporary of the workspace
      const uint64_t r_full = std::min<uint64_t>(it.row_end, g.full_rows);
      d.row_begin = it.row_begin;
      d.row_end = it.row_end;
      d.out = (uint8_t *)it.dst;
      if (r_full > it.row_begin) {
        d.p.c_begin = (uint32_t)(it.row_begin / g.chunk_rows);
        d.p.c_end = (uint32_t)((r_full + g.chunk_rows - 1) / g.chunk_rows);
      } else {
        d.p.c_begin = d.p.c_end = 0;
      }
      const uint64_t tmp_rows =
          std::min<uint64_t>((uint64_t)d.p.c_end * g.chunk_rows, g.full_rows) - (uint64_t)d.p.c_begin * g.chunk_rows;
      d.p.dst = nullptr;  // set below, once the temporaries' offset is known
      d.p.dst_cap = tmp_rows * g.D * g.wb;
      temp_off[i] = temp_total;
      temp_total = (temp_total + d.p.dst_cap + 255) & ~255ull;
      any_ranged = true;
    }
    if (g.n_chunks) {
      // the batch kernel stages the rows of D <= 3 in shared memory, as the
      // single-stream lane decoder does
      d.rg = lane_ring_plan(g, cfg, sched.ring_segments, dec_staged((int)g.D), 64);
      if (!d.rg.per_warp) d.rg = lane_ring_plan(g, cfg, 2, dec_staged((int)g.D), 64);
      if (!d.rg.per_warp) return SPRINTZ_ERR_UNSUPPORTED;
      region = std::max(region, d.rg.per_warp);
    }
    const uint64_t K = 32 / g.D;
    vw[i] = g.w;
    vD[i] = g.D;
    vgroups[i] = (d.p.c_end - d.p.c_begin + K - 1) / K;
  }
  // streams whose rings leave room in the widest warp region (set by the
  // narrowest streams) take larger segments: fewer segment changes per chunk
  for (uint32_t i = 0; i < n; ++i) {
    DecBatchItem &d = v[i];
    if (!d.p.g.n_chunks) continue;
    for (uint32_t ms = d.rg.seg * 2; ms <= 4096; ms *= 2) {
      const LaneRing r = lane_ring_plan(d.p.g, cfg, d.rg.nseg, dec_staged((int)d.p.g.D), ms);
      if (!r.per_warp || r.per_warp > region || r.nseg != d.rg.nseg) break;
      d.rg = r;
    }
  }
  uint64_t n_work = 0;
  batch_work_list(vw, vD, vgroups, sched.order, (uint32_t)cfg.sm_count, work, &n_work);
  memset(pl, 0, sizeof(*pl));
  pl->compress = 0;
  pl->n = n;
  pl->region = std::max<uint32_t>(region, 16);
  pl->n_work = n_work;
  pl->zero_bytes = kClassTicketBytes;  // the class tickets
  pl->items_off = align256d(kClassTicketBytes);
  pl->work_off = align256d(pl->items_off + (uint64_t)n * sizeof(DecBatchItem));
  pl->slots_off = align256d(pl->work_off + 8ull * work->size());  // range temporaries
  pl->ws_total = pl->slots_off + temp_total;
  pl->slot_region = any_ranged ? 1 : 0;
  for (uint32_t i = 0; i < n; ++i)
    if (v[i].row_end > v[i].row_begin) v[i].p.dst = ws ? ws + pl->slots_off + temp_off[i] : nullptr;
  const uint64_t smem = (uint64_t)kLaneWarps * pl->region;
  if (smem > (uint64_t)cfg.max_smem_optin) return SPRINTZ_ERR_UNSUPPORTED;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_decode_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_decode_batch, kLaneThreads, smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  const uint32_t per_sm = std::min<uint32_t>((uint32_t)occ, sched.ctas_per_sm);
  pl->grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((pl->n_work + kLaneWarps - 1) / kLaneWarps,
                                                                (uint64_t)cfg.sm_count * per_sm));
  pl->sched = sched;
  pl->sched.ctas_per_sm = per_sm;
  img->assign(reinterpret_cast<const uint8_t *>(v.data()),
              reinterpret_cast<const uint8_t *>(v.data()) + (size_t)n * sizeof(DecBatchItem));
  return SPRINTZ_OK;
}

int run_batch_decode(const BatchPlan &pl, cudaStream_t stream) {
  uint8_t *ws = (uint8_t *)pl.ws;
  const DecBatchItem *items = reinterpret_cast<const DecBatchItem *>(ws + pl.items_off);
  const BatchClasses *classes = reinterpret_cast<const BatchClasses *>(ws + pl.work_off);
  const uint64_t *work = reinterpret_cast<const uint64_t *>(ws + pl.work_off + kClassTableBytes);
  if (cudaMemsetAsync(ws, 0, pl.zero_bytes, stream) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  k_decode_batch_tails<<<pl.n, 128, 0, stream>>>(items);
  if (pl.n_work)
    k_decode_batch<<<pl.grid, kLaneThreads, (uint64_t)kLaneWarps * pl.region, stream>>>(
        items, classes, work, reinterpret_cast<uint32_t *>(ws), pl.region);
  if (pl.slot_region) k_decode_batch_rows<<<dim3(8, pl.n), 256, 0, stream>>>(items);
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

uint64_t decode_workspace_bytes(const Geom &g, const LaunchCfg &cfg) {
  if (g.n_chunks == 0) return 0;
  DecPlan pl = dec_plan(g, cfg);
  return (uint64_t)pl.grid * pl.scratch_per_cta;
}

int launch_decode(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint64_t src_size,
                  uint8_t *dst, uint64_t dst_cap, uint8_t *ws, uint64_t ws_bytes, int *d_status,
                  cudaStream_t stream) {
  DecParams p{};
  p.src = src;
  p.src_size = src_size;
  p.dst = dst;
  p.dst_cap = dst_cap;
  p.status = d_status;
  p.g = g;
  p.c_begin = 0;
  p.c_end = g.n_chunks;
  {
    static const uint32_t win = [] {
      const char *e = getenv("SPRINTZ_DEC_PF_WIN");
      int x = e ? atoi(e) : 0;
      return (uint32_t)(x >= 16 ? (x & ~15) : 2048);
    }();
    p.pf_win = win;
    p.pf_mode = 0;
  }
  k_decode_header_tail<<<1, 128, 0, stream>>>(p);
  LaneRing rg{};
  if (g.n_chunks > 0 && g.D <= 32 && ((uintptr_t)dst & 7) == 0 && g.max_body < (1ull << 28))
    rg = lane_ring_plan(g, cfg, dec_ring_segments(), dec_staged((int)g.D));
  if (rg.per_warp) {
    const uint64_t K = 32 / g.D;
    const uint64_t warps = (g.n_chunks + K - 1) / K;
    const uint64_t grid = (warps + kLaneWarps - 1) / kLaneWarps;
    if (grid > 0x7FFFFFFFull) return SPRINTZ_ERR_INVALID_ARG;
    const uint64_t smem = (uint64_t)rg.per_warp * kLaneWarps;
    const void *fn = g.w == 8 ? lane_decoder<8>(g.D) : lane_decoder<16>(g.D);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return SPRINTZ_ERR_CUDA;
    void *args[] = {&p, &rg};
    if (cudaLaunchKernel(fn, dim3((uint32_t)grid), dim3(kLaneThreads), args, smem, stream) != cudaSuccess)
      return SPRINTZ_ERR_CUDA;
  } else if (g.n_chunks > 0 && g.D > 32 && g.n_chunks <= 0x7FFFFFFFull) {
    const uint32_t threads = (g.D + 31) & ~31u;
    const uint64_t smem = (((uint64_t)g.hdr_bytes + (uint64_t)g.G * g.D * g.w + 8 + 15) & ~15ull);
    if (smem > (uint64_t)cfg.max_smem_optin) return SPRINTZ_ERR_UNSUPPORTED;
    const void *fn = g.w == 8 ? (const void *)k_decode_wide<8> : (const void *)k_decode_wide<16>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return SPRINTZ_ERR_CUDA;
    void *args[] = {&p};
    if (cudaLaunchKernel(fn, dim3((uint32_t)g.n_chunks), dim3(threads), args, smem, stream) != cudaSuccess)
      return SPRINTZ_ERR_CUDA;
  } else if (g.n_chunks > 0) {
    DecPlan pl = dec_plan(g, cfg);
    if (ws_bytes < (uint64_t)pl.grid * pl.scratch_per_cta) return SPRINTZ_ERR_WS_TOO_SMALL;
    p.scratch = ws;
    p.scratch_per_cta = pl.scratch_per_cta;
    p.staged = pl.staged ? 1 : 0;
    if (g.w == 8)
      k_decode<8><<<pl.grid, kDecThreads, pl.smem, stream>>>(p);
    else
      k_decode<16><<<pl.grid, kDecThreads, pl.smem, stream>>>(p);
  }
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}


// ---- ranges of rows ----------------------------------------------------------

bool decode_chunks_supported(const Geom &g, const LaunchCfg &cfg) {
  if (g.huffman || g.n_chunks == 0) return false;
  if (g.D <= 32) return g.max_body < (1ull << 28) && lane_ring_plan(g, cfg, dec_ring_segments(), dec_staged((int)g.D)).per_warp;
  const uint64_t smem = (((uint64_t)g.hdr_bytes + (uint64_t)g.G * g.D * g.w + 8 + 15) & ~15ull);
  return g.n_chunks <= 0x7FFFFFFFull && smem <= (uint64_t)cfg.max_smem_optin;
}

int launch_decode_chunks(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint64_t src_size,
                         uint32_t c_begin, uint32_t c_end, uint8_t *dst, uint64_t dst_cap, int *d_status,
                         cudaStream_t stream) {
  if (!decode_chunks_supported(g, cfg) || ((uintptr_t)dst & 7) != 0) return SPRINTZ_ERR_UNSUPPORTED;
  if (c_end <= c_begin) return SPRINTZ_OK;
  DecParams p{};
  p.src = src;
  p.src_size = src_size;
  p.dst = dst;
  p.dst_cap = dst_cap;
  p.status = d_status;
  p.g = g;
  p.c_begin = c_begin;
  p.c_end = c_end;
  p.pf_win = 2048;
  const uint64_t n = c_end - c_begin;
  if (g.D <= 32) {
    LaneRing rg = lane_ring_plan(g, cfg, dec_ring_segments(), dec_staged((int)g.D));
    const uint64_t K = 32 / g.D;
    const uint64_t grid = ((n + K - 1) / K + kLaneWarps - 1) / kLaneWarps;
    if (grid > 0x7FFFFFFFull) return SPRINTZ_ERR_INVALID_ARG;
    const uint64_t smem = (uint64_t)rg.per_warp * kLaneWarps;
    const void *fn = g.w == 8 ? lane_decoder<8>(g.D) : lane_decoder<16>(g.D);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return SPRINTZ_ERR_CUDA;
    void *args[] = {&p, &rg};
    if (cudaLaunchKernel(fn, dim3((uint32_t)grid), dim3(kLaneThreads), args, smem, stream) != cudaSuccess)
      return SPRINTZ_ERR_CUDA;
    return SPRINTZ_OK;
  }
  const uint32_t threads = (g.D + 31) & ~31u;
  const uint64_t smem = (((uint64_t)g.hdr_bytes + (uint64_t)g.G * g.D * g.w + 8 + 15) & ~15ull);
  const void *fn = g.w == 8 ? (const void *)k_decode_wide<8> : (const void *)k_decode_wide<16>;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return SPRINTZ_ERR_CUDA;
  void *args[] = {&p};
  if (cudaLaunchKernel(fn, dim3((uint32_t)n), dim3(threads), args, smem, stream) != cudaSuccess)
    return SPRINTZ_ERR_CUDA;
  return SPRINTZ_OK;
}

// Rows [row_begin, row_end) to out: the rows of the decoded chunks held at
// tmp (from row tmp_row0 on), then the raw tail rows from the stream; the
// header is checked first (every CTA checks it, one reports it).
__global__ void k_decode_rows_finish(DecParams p, uint64_t row_begin, uint64_t row_end, uint64_t tmp_row0,
                                     const uint8_t *tmp, uint8_t *out) {
  const Geom &g = p.g;
  __shared__ uint32_t s_ok;
  __shared__ uint64_t s_tail_off;
  if (threadIdx.x == 0) {
    uint64_t tail_off = 0;
    const bool ok = header_matches(g, p.src, p.src_size, &tail_off);
    s_ok = ok;
    s_tail_off = tail_off;
    if (!ok && blockIdx.x == 0) set_status(p.status, SPRINTZ_ERR_CORRUPT);
  }
  __syncthreads();
  if (!s_ok) return;
  const uint64_t rb = (uint64_t)g.D * g.wb;
  const uint64_t r_full = min(row_end, g.full_rows);
  const uint64_t n_mid = r_full > row_begin ? (r_full - row_begin) * rb : 0;
  if (n_mid) grid_copy(out, tmp + (row_begin - tmp_row0) * rb, n_mid);
  if (row_end > g.full_rows) {
    const uint64_t t0 = max(row_begin, g.full_rows);
    grid_copy(out + n_mid, p.src + s_tail_off + (t0 - g.full_rows) * rb, (row_end - t0) * rb);
  }
}

// Chunks that cover rows [row_begin, row_end) (none when the rows all lie
// in the raw tail).
static void covering_chunks(const Geom &g, uint64_t row_begin, uint64_t row_end, uint32_t *c0, uint32_t *c1) {
  const uint64_t r_full = std::min<uint64_t>(row_end, g.full_rows);
  if (r_full > row_begin) {
    *c0 = (uint32_t)(row_begin / g.chunk_rows);
    *c1 = (uint32_t)((r_full + g.chunk_rows - 1) / g.chunk_rows);
  } else {
    *c0 = *c1 = 0;
  }
}

uint64_t decode_rows_workspace_bytes(const Geom &g, const LaunchCfg &cfg, uint64_t row_begin, uint64_t row_end) {
  const uint64_t rb = (uint64_t)g.D * g.wb;
  if (decode_chunks_supported(g, cfg)) {
    uint32_t c0, c1;
    covering_chunks(g, row_begin, row_end, &c0, &c1);
    const uint64_t r1 = std::min<uint64_t>((uint64_t)c1 * g.chunk_rows, g.full_rows);
    return c1 > c0 ? align256d((r1 - (uint64_t)c0 * g.chunk_rows) * rb) : 0;
  }
  // every chunk decoded by the whole-stream decoder, then the rows copied
  const uint64_t inner = g.huffman ? huff_decode_workspace_bytes(g, cfg) : decode_workspace_bytes(g, cfg);
  return align256d(g.rows * rb) + inner;
}

int launch_decode_rows(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint64_t src_size,
                       uint64_t row_begin, uint64_t row_end, uint8_t *out, uint8_t *ws, uint64_t ws_bytes,
                       int *d_status, cudaStream_t stream) {
  if (row_end <= row_begin) return SPRINTZ_OK;
  if (ws_bytes < decode_rows_workspace_bytes(g, cfg, row_begin, row_end)) return SPRINTZ_ERR_WS_TOO_SMALL;
  DecParams p{};
  p.src = src;
  p.src_size = src_size;
  p.status = d_status;
  p.g = g;
  const uint64_t rb = (uint64_t)g.D * g.wb;
  uint64_t tmp_row0 = 0;
  int rc = SPRINTZ_OK;
  if (decode_chunks_supported(g, cfg)) {
    uint32_t c0, c1;
    covering_chunks(g, row_begin, row_end, &c0, &c1);
    tmp_row0 = (uint64_t)c0 * g.chunk_rows;
    const uint64_t r1 = std::min<uint64_t>((uint64_t)c1 * g.chunk_rows, g.full_rows);
    if (c1 > c0) rc = launch_decode_chunks(g, cfg, src, src_size, c0, c1, ws, (r1 - tmp_row0) * rb, d_status, stream);
  } else {
    const uint64_t tb = align256d(g.rows * rb);
    rc = g.huffman ? launch_decode_huffman(g, cfg, src, src_size, ws, g.rows * rb, ws + tb, ws_bytes - tb, d_status,
                                           stream)
                   : launch_decode(g, cfg, src, src_size, ws, g.rows * rb, ws + tb, ws_bytes - tb, d_status, stream);
  }
  if (rc != SPRINTZ_OK) return rc;
  const uint64_t bytes = (row_end - row_begin) * rb;
  const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((bytes + 4095) / 4096,
                                                                          (uint64_t)cfg.sm_count * 8));
  k_decode_rows_finish<<<grid, 256, 0, stream>>>(p, row_begin, row_end, tmp_row0, ws, out);
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

}  // namespace spz
