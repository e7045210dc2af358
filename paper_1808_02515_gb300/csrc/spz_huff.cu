// Huffman stage of the CUDA Sprintz codec (Sec. 4.4: byte symbols, applied to
// the bit-packed bytes).  The paper uses Huff0; this is our own canonical,
// length-limited code shared by a segment of `huff_chunks` consecutive chunks:
//   lengths   package-merge (Larmore & Hirschberg 1990) with maximum length 11,
//             leaves ordered by (frequency, symbol), a leaf before a package of
//             equal weight, one used symbol -> length 1;
//   codes     canonical (RFC 1951 Sec. 3.2.2: by length, then symbol), each
//             code's most significant bit first in the least-significant-bit-
//             first stream;
//   raw       a segment whose coded bytes (each chunk padded to a byte) are not
//             fewer than its packed bytes keeps an all-zero table and raw bodies.
//
//   sub-blocks each chunk's code is cut into n = ceil(packed / 2048) sub-blocks
//             of about equal packed size, each padded to a byte and preceded
//             (after the first) by a u32 jump-table offset, so that every
//             sub-block decodes on its own.
//
// Encode: the regular encoder writes the Huffman-free stream P into the
// workspace; k_huff_hist (CTAs over 64 KB slices of a segment) counts the
// segment's packed bytes; k_huff_lengths (a CTA per segment) runs
// package-merge and builds the canonical code table; k_huff_sizes (a warp per
// chunk) sums the coded bits of every sub-block; k_huff_decide (a CTA per
// segment) chooses raw or coded and places the chunks inside the segment;
// k_huff_scan places the segments; k_huff_encode (persistent warps, each
// over a contiguous range of sub-blocks, a sub-block at a time) writes the
// coded bytes, the jump tables and the chunk table, and
// k_huff_enc_finish the header and the raw tail.
// Decode: k_huff_dec_prep (a CTA per segment) checks the table (lengths <= 11,
// Kraft), builds its 11-bit lookup table and maps the segment's sub-blocks to
// their chunks; k_huff_decode (a thread per sub-block) decodes each sub-block
// into a Huffman-free stream in the workspace, and k_huff_dec_finish writes
// its header and tail; the regular decoder then decodes that stream.
#include <algorithm>

#include "spz_common.cuh"

namespace spz {

constexpr uint32_t kHuffMaxLen = 11;
constexpr int kHuffThreads = 256;
constexpr uint32_t kHuffLists = kHuffMaxLen;  // list 0 (leaves) .. list L-1
constexpr uint32_t kMaxItems = 511;           // 2 * 256 - 1

__device__ __forceinline__ uint64_t le64(const uint8_t *p) {
  uint64_t v = 0;
  for (int k = 0; k < 8; ++k) v |= (uint64_t)p[k] << (8 * k);
  return v;
}
__device__ __forceinline__ uint32_t le32(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
__device__ __forceinline__ void put_le(uint8_t *p, uint64_t v, int n) {
  for (int k = 0; k < n; ++k) p[k] = (uint8_t)(v >> (8 * k));
}

// Shared state of the length computation of one segment.
struct HuffSmem {
  uint64_t hist[256];
  uint32_t sorted_sym[256];  // used symbols by (frequency, symbol)
  uint64_t w[2][kMaxItems + 1];
  uint64_t wl[256];  // leaf weights in (frequency, symbol) order
  uint8_t leaf[kHuffLists][kMaxItems + 1];  // list k: item is a leaf (1) or a package (0)
  uint32_t list_len[kHuffLists];
  uint32_t take[kHuffLists];  // leaves of list k inside the selection
  uint8_t len[256];
  uint32_t code[256];
  uint32_t n_used;
  uint32_t bl_count[kHuffMaxLen + 1];
  uint32_t next_code[kHuffMaxLen + 2];
};

// Code lengths of the 256 byte symbols from sm.hist (whole CTA).
__device__ void huff_lengths(HuffSmem &sm) {
  const uint32_t t = threadIdx.x;
  if (t == 0) sm.n_used = 0;
  __syncthreads();
  const uint64_t f = sm.hist[t];
  if (f) atomicAdd(&sm.n_used, 1u);
  sm.len[t] = 0;
  __syncthreads();
  const uint32_t n = sm.n_used;
  // rank among used symbols by (frequency, symbol)
  if (f) {
    uint32_t r = 0;
    for (uint32_t u = 0; u < 256; ++u) {
      const uint64_t fu = sm.hist[u];
      r += fu && (fu < f || (fu == f && u < t));
    }
    sm.sorted_sym[r] = t;
  }
  __syncthreads();
  if (n == 0) return;
  if (n == 1) {
    if (t == 0) sm.len[sm.sorted_sym[0]] = 1;
    __syncthreads();
    return;
  }
  // list 0: the leaves; list k: merge(leaves, packages of list k-1).  The
  // merge is done in parallel: each leaf and each package finds its place by
  // a binary search in the other sorted sequence (a leaf goes before a
  // package of equal weight).
  if (t < n) {
    const uint64_t w0 = sm.hist[sm.sorted_sym[t]];
    sm.wl[t] = w0;
    sm.w[0][t] = w0;
    sm.leaf[0][t] = 1;
  }
  if (t == 0) sm.list_len[0] = n;
  __syncthreads();
  for (uint32_t k = 1; k < kHuffLists; ++k) {
    const uint64_t *A = sm.w[(k - 1) & 1];
    uint64_t *B = sm.w[k & 1];
    const uint32_t np = sm.list_len[k - 1] / 2;
    for (uint32_t i = t; i < n; i += blockDim.x) {
      // packages lighter than this leaf
      const uint64_t wv = sm.wl[i];
      uint32_t lo = 0, hi = np;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (A[2 * mid] + A[2 * mid + 1] < wv) lo = mid + 1;
        else hi = mid;
      }
      B[i + lo] = wv;
      sm.leaf[k][i + lo] = 1;
    }
    for (uint32_t q = t; q < np; q += blockDim.x) {
      // leaves no heavier than this package
      const uint64_t wv = A[2 * q] + A[2 * q + 1];
      uint32_t lo = 0, hi = n;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (sm.wl[mid] <= wv) lo = mid + 1;
        else hi = mid;
      }
      B[q + lo] = wv;
      sm.leaf[k][q + lo] = 0;
    }
    if (t == 0) sm.list_len[k] = n + np;
    __syncthreads();
  }
  // selection: the first 2n - 2 items of the last list; the packages among
  // them select the first 2p items of the list before, and so on
  {
    uint32_t m = 2 * n - 2;
    for (int k = (int)kHuffLists - 1; k >= 0; --k) {
      uint32_t leaves = 0;
      for (uint32_t base = 0; base < m; base += blockDim.x) {
        const uint32_t i = base + t;
        leaves += __syncthreads_count(i < m && sm.leaf[k][i]);
      }
      if (t == 0) sm.take[k] = leaves;
      m = 2 * (m - leaves);
    }
  }
  __syncthreads();
  // a leaf's length is the number of lists whose selection holds it
  if (t < n) {
    uint32_t l = 0;
    for (uint32_t k = 0; k < kHuffLists; ++k) l += t < sm.take[k];
    sm.len[sm.sorted_sym[t]] = (uint8_t)l;
  }
  __syncthreads();
}

// Canonical codes from sm.len (whole CTA).
__device__ void huff_codes(HuffSmem &sm) {
  const uint32_t t = threadIdx.x;
  if (t <= kHuffMaxLen) sm.bl_count[t] = 0;
  __syncthreads();
  if (sm.len[t]) atomicAdd(&sm.bl_count[sm.len[t]], 1u);
  __syncthreads();
  if (t == 0) {
    uint32_t code = 0;
    sm.bl_count[0] = 0;
    for (uint32_t bits = 1; bits <= kHuffMaxLen; ++bits) {
      code = (code + sm.bl_count[bits - 1]) << 1;
      sm.next_code[bits] = code;
    }
  }
  __syncthreads();
  const uint32_t l = sm.len[t];
  uint32_t c = 0;
  if (l) {
    uint32_t r = 0;
    for (uint32_t u = 0; u < t; ++u) r += sm.len[u] == l;
    c = sm.next_code[l] + r;
  }
  sm.code[t] = c;
  __syncthreads();
}

__device__ __forceinline__ uint32_t bitrev(uint32_t c, uint32_t l) { return l ? __brev(c) >> (32 - l) : 0u; }


// ---------------------------------------------------------------------------
// Sub-blocks
//
// A chunk body of `packed` bytes is coded as n = ceil(packed / kHuffSub)
// sub-blocks of q = ceil(packed / n) packed bytes (the last one may be
// shorter; an empty body has one empty sub-block).  Each is padded to a
// byte and decodes on its own; n - 1 u32 offsets in front of them say where
// sub-blocks 1..n-1 start, counted from the end of that jump table.  Huff0,
// the coder the paper uses, splits its blocks into separately decodable
// streams behind a table of their sizes in the same way (RFC 8878 Sec.
// 4.2.2).  One warp encodes, and one thread decodes, one sub-block, so the
// parallelism no longer depends on how wide a chunk's rows are.
// ---------------------------------------------------------------------------

constexpr uint32_t kHuffSub = 2048;
__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
constexpr uint32_t kHuffSubWords = (kHuffSub * kHuffMaxLen / 8 + 4) / 4 + 2;  // one sub-block's code
constexpr uint32_t kHuffBufWords = kHuffSubWords + kHuffSubWords / 16 + 2;      // the same, skewed
constexpr uint32_t kHuffInWords = (kHuffSub + 6) / 4 + (kHuffSub + 6) / 64 + 4;   // one sub-block, skewed
constexpr int kHuffWarps = 8;                                                 // warps per CTA
constexpr int kHuffEncWarps = 4;  // k_huff_encode: 5.7 KB of shared memory per warp
constexpr uint32_t kLutSize = 1u << kHuffMaxLen;
constexpr uint32_t kHuffDecThreads = 128;

__host__ __device__ __forceinline__ uint32_t huff_n_sub(uint32_t packed) {
  return packed == 0 ? 1u : (uint32_t)(((uint64_t)packed + kHuffSub - 1) / kHuffSub);
}

// Packed bytes [i0, i0 + n) of sub-block k of a body of `packed` bytes.
__device__ __forceinline__ void huff_sub_range(uint32_t packed, uint32_t k, uint64_t *i0, uint32_t *n) {
  const uint64_t ns = huff_n_sub(packed);
  const uint64_t q = (packed + ns - 1) / ns;
  const uint64_t a = umin64(packed, k * q), b = umin64(packed, (k + 1) * q);
  *i0 = a;
  *n = (uint32_t)(b - a);
}

// Chunks [c0, c1) of segment s.
__device__ __forceinline__ void seg_chunks(const Geom &g, uint32_t s, uint32_t *c0, uint32_t *c1) {
  const uint64_t a = (uint64_t)s * g.huff_chunks;
  *c0 = (uint32_t)a;
  *c1 = (uint32_t)umin64(g.n_chunks, a + g.huff_chunks);
}

__device__ __forceinline__ uint8_t *huff_table(uint8_t *base, const Geom &g, uint32_t s) {
  return base + kHdrBytes + (uint64_t)kEntryBytes * g.n_chunks + (uint64_t)kHuffTableBytes * s;
}

// Exclusive prefix of the segment totals (one CTA).
__global__ void __launch_bounds__(1024) k_huff_scan(const uint64_t *in, uint64_t *out, uint32_t n) {
  __shared__ uint64_t s_w[32];
  __shared__ uint64_t s_carry;
  const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    const uint64_t v = base + t < n ? in[base + t] : 0;
    uint64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint64_t z = lane < blockDim.x / 32 ? s_w[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
        if (lane >= o) z += y;
      }
      s_w[lane] = z;
    }
    __syncthreads();
    const uint64_t incl = x + (warp ? s_w[warp - 1] : 0) + s_carry;
    if (base + t < n) out[base + t] = incl - v;
    __syncthreads();
    if (t == blockDim.x - 1) s_carry = incl;
    __syncthreads();
  }
  if (t == 0) out[n] = s_carry;
}

// Block-wide exclusive scan of one value per thread (256 threads); returns
// the thread's exclusive prefix plus *carry, and advances *carry by the sum.
__device__ __forceinline__ uint64_t block_scan256(uint64_t v, uint64_t *s_w, uint64_t *carry) {
  const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t z = lane < 8 ? s_w[lane] : 0;
    for (int o = 1; o < 8; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
      if (lane >= o) z += y;
    }
    if (lane < 8) s_w[lane] = z;
  }
  __syncthreads();
  const uint64_t excl = x - v + (warp ? s_w[warp - 1] : 0) + *carry;
  __syncthreads();
  if (t == 255) *carry = excl + v;
  __syncthreads();
  return excl;
}

// ---------------------------------------------------------------------------
// Encode
// ---------------------------------------------------------------------------

struct HuffEncParams {
  const uint8_t *P;               // Huffman-free stream (regular encoder output)
  uint8_t *dst;
  uint64_t dst_cap;
  uint64_t *out_size;
  const uint8_t *src;             // raw samples (for the tail)
  int *status;
  Geom g;                         // the Huffman stream's geometry
  uint64_t p_data_off;            // data offset of P
  uint64_t p_body_cap;            // bytes of P after p_data_off
  uint32_t slots;                 // sub-block slots per chunk (sub-blocks of the largest body)
  uint32_t slices;                // histogram CTAs per segment
  uint64_t slice_bytes;           // packed bytes per histogram CTA
  unsigned long long *hist;       // [n_segments][256] byte counts
  uint32_t *codes;                // [n_segments][256] bit-reversed code | length << 16
  unsigned long long *seg_coded;  // [n_segments] coded bytes of the segment's chunks
  uint32_t *seg_raw;              // [n_segments] 1 = stored raw
  uint64_t *seg_total;            // [n_segments] bytes the segment takes in the stream
  uint64_t *seg_prefix;           // [n_segments + 1]
  uint64_t *chunk_coded;          // [n_chunks] coded bytes of each chunk
  uint64_t *chunk_pos;            // [n_chunks] offset of each chunk inside its segment
  uint32_t *sub_off;              // [n_chunks][slots] start of each sub-block inside its chunk
};

// Chunk c of P: body offset (from P's data), records, packed bytes.  The
// regular encoder wrote these; they are clamped to P and to the largest
// body all the same, so that a failed encode cannot send a read astray.
__device__ __forceinline__ void p_entry(const HuffEncParams &p, uint32_t c, uint64_t *off, uint32_t *nrec,
                                        uint32_t *packed) {
  const uint8_t *e = p.P + kHdrBytes + (uint64_t)c * kEntryBytes;
  const uint64_t o = min(le64(e), p.p_body_cap);
  *off = o;
  *nrec = le32(e + 8);
  *packed = (uint32_t)min(min((uint64_t)le32(e + 12), p.p_body_cap - o), p.g.max_body);
}

// Byte histogram of one slice of a segment's packed bytes (the segment's
// bodies are contiguous in P): per-warp counters, then global atomics.
__global__ void __launch_bounds__(kHuffWarps * 32) k_huff_hist(HuffEncParams p) {
  __shared__ uint32_t h[kHuffWarps][256];
  const Geom &g = p.g;
  const uint32_t s = blockIdx.x / p.slices, part = blockIdx.x % p.slices;
  uint32_t c0, c1;
  seg_chunks(g, s, &c0, &c1);
  uint64_t o0, o1;
  uint32_t nr, pk;
  p_entry(p, c0, &o0, &nr, &pk);
  p_entry(p, c1 - 1, &o1, &nr, &pk);
  o1 += pk;
  const uint64_t a = o0 + (uint64_t)part * p.slice_bytes;
  if (a >= o1) return;
  const uint64_t b = min(o1, a + p.slice_bytes);
  const uint32_t t = threadIdx.x, warp = t >> 5;
  for (uint32_t k = t; k < kHuffWarps * 256; k += blockDim.x) (&h[0][0])[k] = 0;
  __syncthreads();
  // aligned 32-bit words covering [a, b); P has slack after its last byte
  const uintptr_t base = (uintptr_t)(p.P + p.p_data_off);
  const uintptr_t A = base + a, B = base + b;
  for (uintptr_t q = (A & ~(uintptr_t)3) + 4 * (uintptr_t)t; q < B; q += 4 * (uintptr_t)blockDim.x) {
    const uint32_t v = *reinterpret_cast<const uint32_t *>(q);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (q + i >= A && q + i < B) atomicAdd(&h[warp][(v >> (8 * i)) & 255u], 1u);
  }
  __syncthreads();
  uint32_t sum = 0;
  for (int w = 0; w < kHuffWarps; ++w) sum += h[w][t];
  if (sum) atomicAdd(&p.hist[(uint64_t)s * 256 + t], (unsigned long long)sum);
}

// Code lengths, the table and the codes of one segment (one CTA).
__global__ void __launch_bounds__(kHuffThreads) k_huff_lengths(HuffEncParams p) {
  __shared__ HuffSmem sm;
  const uint32_t s = blockIdx.x, t = threadIdx.x;
  sm.hist[t] = p.hist[(uint64_t)s * 256 + t];
  __syncthreads();
  huff_lengths(sm);
  huff_codes(sm);
  const uint32_t l = sm.len[t];
  p.codes[(uint64_t)s * 256 + t] = bitrev(sm.code[t], l) | (l << 16);
  uint8_t *tab = huff_table(p.dst, p.g, s);
  if (t < 128) tab[t] = (uint8_t)(sm.len[2 * t] | (sm.len[2 * t + 1] << 4));
  if (t == 0) p.seg_coded[s] = 0;
}

// Coded size of every sub-block of a chunk (one warp per chunk).
__global__ void __launch_bounds__(kHuffWarps * 32) k_huff_sizes(HuffEncParams p) {
  __shared__ uint8_t s_len[kHuffWarps][256];
  const Geom &g = p.g;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t c64 = (uint64_t)blockIdx.x * kHuffWarps + warp;
  if (c64 >= g.n_chunks) return;
  const uint32_t c = (uint32_t)c64;
  const uint32_t s = c / g.huff_chunks;
  const uint32_t *cs = p.codes + (uint64_t)s * 256;
#pragma unroll
  for (int i = 0; i < 8; ++i) s_len[warp][lane + 32 * i] = (uint8_t)(cs[lane + 32 * i] >> 16);
  __syncwarp();
  uint64_t off;
  uint32_t nrec, packed;
  p_entry(p, c, &off, &nrec, &packed);
  const uint8_t *body = p.P + p.p_data_off + off;
  const uint32_t n_sub = huff_n_sub(packed);
  uint64_t run = 4ull * (n_sub - 1);
  for (uint32_t k = 0; k < n_sub; ++k) {
    uint64_t i0;
    uint32_t len;
    huff_sub_range(packed, k, &i0, &len);
    uint32_t bits = 0;
    for (uint64_t i = i0 + lane; i < i0 + len; i += 32) bits += s_len[warp][body[i]];
    for (int o = 16; o > 0; o >>= 1) bits += __shfl_xor_sync(0xFFFFFFFFu, bits, o);
    if (lane == 0) p.sub_off[(uint64_t)c * p.slots + k] = (uint32_t)run;
    run += (bits + 7) / 8;
  }
  if (lane == 0) {
    p.chunk_coded[c] = run;
    atomicAdd(&p.seg_coded[s], (unsigned long long)run);
  }
}

// Raw or coded, and every chunk's place inside its segment (one CTA per
// segment): a segment whose coded bytes are not fewer than its packed bytes
// keeps an all-zero table and raw bodies.
__global__ void __launch_bounds__(256) k_huff_decide(HuffEncParams p) {
  __shared__ uint64_t s_w[8];
  __shared__ uint64_t s_carry;
  __shared__ uint32_t s_raw;
  const Geom &g = p.g;
  const uint32_t s = blockIdx.x, t = threadIdx.x;
  uint32_t c0, c1;
  seg_chunks(g, s, &c0, &c1);
  if (t == 0) {
    uint64_t o0, o1;
    uint32_t nr, pk;
    p_entry(p, c0, &o0, &nr, &pk);
    p_entry(p, c1 - 1, &o1, &nr, &pk);
    const uint64_t packed_total = o1 + pk - o0;
    const uint32_t raw = packed_total == 0 || p.seg_coded[s] >= packed_total;
    s_raw = raw;
    p.seg_raw[s] = raw;
    s_carry = 0;
  }
  __syncthreads();
  const bool raw = s_raw != 0;
  if (raw && t < 128) huff_table(p.dst, g, s)[t] = 0;
  for (uint64_t base = c0; base < c1; base += 256) {
    const uint64_t c = base + t;
    uint64_t v = 0;
    if (c < c1) {
      uint64_t off;
      uint32_t nrec, packed;
      p_entry(p, (uint32_t)c, &off, &nrec, &packed);
      v = raw ? packed : p.chunk_coded[c];
    }
    const uint64_t excl = block_scan256(v, s_w, &s_carry);
    if (c < c1) p.chunk_pos[c] = excl;
  }
  if (t == 0) p.seg_total[s] = s_carry;
}

// One sub-block slot (chunk c, sub-block k) for k_huff_encode: its packed
// bytes are copied to shared memory with coalesced word loads; lanes code
// contiguous runs of them, a warp scan of their bit counts places them in a
// shared buffer (whole words stored, the words two lanes share OR-ed), and
// the coded bytes go to the stream in 4-byte stores.  Both shared buffers
// have a pad word after every 16, so that lanes working about 16 words apart
// hit different banks.  Sub-block 0 writes the chunk's table entry, the
// others their jump-table offsets.  s_code holds the code table of segment
// *cur_s; it is loaded again only when the slot's segment differs.
__device__ __forceinline__ void huff_encode_slot(const HuffEncParams &p, uint64_t slot, uint32_t lane,
                                                 uint16_t *s_code, uint32_t *sin, uint32_t *buf,
                                                 uint32_t *cur_s) {
  const Geom &g = p.g;
  const uint32_t c = (uint32_t)(slot / p.slots), k = (uint32_t)(slot % p.slots);
  const uint32_t s = c / g.huff_chunks;
  // every per-slot load issued at once (all in bounds for any slot), with
  // the segment's code table when it is a new one
  uint64_t off;
  uint32_t nrec, packed;
  p_entry(p, c, &off, &nrec, &packed);
  const bool raw = p.seg_raw[s] != 0;
  const uint64_t seg_base = p.seg_prefix[s], chunk_base = p.chunk_pos[c], coded = p.chunk_coded[c];
  const uint32_t start = p.sub_off[(uint64_t)c * p.slots + k];
  const bool new_table = s != *cur_s;
  uint32_t ce[8];
  if (new_table) {
    const uint32_t *cs = p.codes + (uint64_t)s * 256;
#pragma unroll
    for (int i = 0; i < 8; ++i) ce[i] = cs[lane + 32 * i];
  }
  const uint32_t n_sub = huff_n_sub(packed);
  if (k >= n_sub) return;
  const uint64_t cpos = seg_base + chunk_base;  // from data_off
  const uint64_t ctotal = raw ? packed : coded;
  if (g.data_off + cpos + ctotal > p.dst_cap) {
    if (lane == 0) set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
    return;
  }
  uint8_t *d = p.dst + g.data_off + cpos;
  if (k == 0 && lane == 0) {
    uint8_t *e = p.dst + kHdrBytes + (uint64_t)c * kEntryBytes;
    put_le(e, cpos, 8);
    put_le(e + 8, nrec, 4);
    put_le(e + 12, packed, 4);
  }
  uint64_t i0;
  uint32_t n;
  huff_sub_range(packed, k, &i0, &n);
  const uint8_t *in = p.P + p.p_data_off + off + i0;
  if (raw) {
    for (uint32_t i = lane; i < n; i += 32) d[i0 + i] = in[i];
    return;
  }
  const uint32_t jump = 4 * (n_sub - 1);
  if (k > 0 && lane < 4) d[4 * (k - 1) + lane] = (uint8_t)((start - jump) >> (8 * lane));
  if (new_table) {
#pragma unroll
    for (int i = 0; i < 8; ++i) s_code[lane + 32 * i] = (uint16_t)((ce[i] & 0x7FFu) | ((ce[i] >> 16) << 11));
    *cur_s = s;
  }
  // the sub-block's bytes: aligned words from up to 3 bytes before it to up
  // to 3 bytes after it (P has slack after its last byte)
  const uint32_t lead = (uint32_t)((uintptr_t)in & 3);
  const uint32_t *w32 = reinterpret_cast<const uint32_t *>((uintptr_t)in - lead);
  const uint32_t nw = (n + lead + 3) / 4;
  for (uint32_t q = lane; q < nw; q += 32) sin[q + (q >> 4)] = w32[q];
  __syncwarp();
  // each lane codes a run of `per` bytes, a multiple of 4, so that its bytes
  // come four at a time from one funnel-shifted pair of words
  const uint32_t per = ((n + 31) / 32 + 3) & ~3u;
  const uint32_t a = min(n, lane * per), b = min(n, a + per);
  const uint32_t sh_lead = 8 * lead;
  auto word4 = [&](uint32_t i) {  // bytes i .. i + 3 (i a multiple of 4)
    const uint32_t q = i >> 2;
    return __funnelshift_r(sin[q + (q >> 4)], sin[(q + 1) + ((q + 1) >> 4)], sh_lead);
  };
  uint32_t nb = 0;
  for (uint32_t i = a; i < b; i += 4) {
    const uint32_t w = word4(i), m = b - i;
#pragma unroll
    for (uint32_t t = 0; t < 4; ++t)
      if (t < m) nb += s_code[(w >> (8 * t)) & 255u] >> 11;
  }
  uint32_t incl = nb;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  auto pad = [](uint32_t w) { return w + (w >> 4); };
  for (uint32_t i = lane; i <= pad(total / 32 + 1); i += 32) buf[i] = 0;
  __syncwarp();
  // the lane's bits [bit0, bit0 + nb): whole words stored, its first word
  // (shared with the lane before) and last word (with the lane after) OR-ed
  const uint32_t bit0 = incl - nb;
  uint32_t wi = bit0 >> 5, nacc = bit0 & 31;
  bool first_shared = nacc != 0;
  uint64_t acc = 0;
  // two codes (at most 22 bits) join the accumulator (under 32 bits) before
  // a full word can leave it
  auto emit = [&]() {
    if (nacc >= 32) {
      if (first_shared) atomicOr(&buf[pad(wi)], (uint32_t)acc);
      else buf[pad(wi)] = (uint32_t)acc;
      first_shared = false;
      acc >>= 32;
      nacc -= 32;
      ++wi;
    }
  };
  for (uint32_t i = a; i < b; i += 4) {
    const uint32_t w = word4(i), m = b - i;
#pragma unroll
    for (uint32_t t = 0; t < 4; ++t) {
      if (t < m) {
        const uint32_t e = s_code[(w >> (8 * t)) & 255u];
        acc |= (uint64_t)(e & 0x7FFu) << nacc;
        nacc += e >> 11;
      }
      if (t & 1) emit();
    }
  }
  if (b > a && nacc > 0) atomicOr(&buf[pad(wi)], (uint32_t)acc);
  __syncwarp();
  // the coded bytes: a few head bytes until the destination is 4-byte
  // aligned, whole words (two buffer words funnel-shifted), tail bytes
  const uint32_t nbytes = (total + 7) / 8;
  uint8_t *dd = d + start;
  auto byte_of = [&](uint32_t i) { return (uint8_t)(buf[pad(i >> 2)] >> (8 * (i & 3))); };
  const uint32_t hb = min(nbytes, (uint32_t)((4 - ((uintptr_t)dd & 3)) & 3));
  if (lane < hb) dd[lane] = byte_of(lane);
  const uint32_t nout = (nbytes - hb) / 4, sh = 8 * (hb & 3);
  uint32_t *dw = reinterpret_cast<uint32_t *>(dd + hb);
  for (uint32_t m = lane; m < nout; m += 32) {
    const uint32_t w = (hb + 4 * m) >> 2;
    dw[m] = __funnelshift_r(buf[pad(w)], buf[pad(w + 1)], sh);
  }
  for (uint32_t i = hb + 4 * nout + lane; i < nbytes; i += 32) dd[i] = byte_of(i);
}

// Persistent warps, each over a contiguous range of sub-block slots (those of
// one or two segments, so that the code table is mostly loaded once).
__global__ void __launch_bounds__(kHuffEncWarps * 32) k_huff_encode(HuffEncParams p, uint64_t per_warp) {
  __shared__ uint16_t s_code[kHuffEncWarps][256];  // reversed code | length << 11
  __shared__ uint32_t s_in[kHuffEncWarps][kHuffInWords];
  __shared__ uint32_t s_buf[kHuffEncWarps][kHuffBufWords];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t total = (uint64_t)p.g.n_chunks * p.slots;
  const uint64_t first = ((uint64_t)blockIdx.x * kHuffEncWarps + warp) * per_warp;
  const uint64_t last = umin64(total, first + per_warp);
  uint32_t cur_s = 0xFFFFFFFFu;
  for (uint64_t slot = first; slot < last; ++slot) {
    huff_encode_slot(p, slot, lane, s_code[warp], s_in[warp], s_buf[warp], &cur_s);
    __syncwarp();  // the warp's shared buffers are reused by the next slot
  }
}

// Header and raw tail of the Huffman stream.
__global__ void k_huff_enc_finish(HuffEncParams p) {
  const Geom &g = p.g;
  const uint64_t tail_off = g.data_off + p.seg_prefix[g.n_segments];
  const uint64_t tail_bytes = g.tail_rows * g.D * g.wb;
  const uint64_t total = tail_off + tail_bytes;
  if (total > p.dst_cap) {
    if (threadIdx.x == 0) set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
    return;
  }
  for (uint64_t k = threadIdx.x; k < tail_bytes; k += blockDim.x)
    p.dst[tail_off + k] = p.src[g.full_rows * g.D * g.wb + k];
  if (threadIdx.x == 0) {
    uint8_t *h = p.dst;
    for (int k = 0; k < 64; ++k) h[k] = 0;
    h[0] = 'S';
    h[1] = 'P';
    h[2] = 'Z';
    h[3] = '1';
    h[4] = 1;
    h[5] = (uint8_t)g.w;
    h[6] = (uint8_t)g.forecaster;
    h[7] = 1;
    put_le(h + 8, g.D, 2);
    h[10] = (uint8_t)g.G;
    h[11] = (uint8_t)g.learn_shift;
    put_le(h + 12, g.chunk_rows_opt, 4);
    put_le(h + 16, g.huff_chunks, 4);
    put_le(h + 20, g.n_chunks, 4);
    put_le(h + 24, g.rows, 8);
    put_le(h + 32, g.tail_rows, 4);
    put_le(h + 40, g.data_off, 8);
    put_le(h + 48, tail_off, 8);
    put_le(h + 56, total, 8);
    *p.out_size = total;
  }
}

// ---------------------------------------------------------------------------
// Decode
// ---------------------------------------------------------------------------

struct HuffDecParams {
  const uint8_t *src;
  uint64_t src_size;
  uint8_t *P;            // Huffman-free stream to build
  uint64_t p_cap;
  int *status;
  Geom g;                // the Huffman stream's geometry
  uint64_t p_data_off;
  uint32_t slots;        // sub-block slots per chunk
  uint32_t parts;        // k_huff_decode CTAs per segment
  uint16_t *lut;         // [n_segments][2^11] symbol | length << 8 (0: no code)
  uint32_t *seg_flags;   // [n_segments] bit 0 raw, bit 1 invalid table
  uint64_t *seg_packed;  // [n_segments] packed bytes per segment, then its prefix
  uint64_t *seg_prefix;  // [n_segments + 1]
  uint64_t *chunk_poff;  // [n_chunks] packed offset of each chunk inside its segment
  uint64_t *chunk_sub0;  // [n_chunks] index of each chunk's first sub-block inside its segment
  uint64_t *seg_nsub;    // [n_segments] sub-blocks of each segment
  uint64_t seg_slots;    // sub-block entries per segment in sub_map: huff_chunks * slots
  uint64_t *sub_map;     // [n_segments][seg_slots] chunk << 32 | k of each sub-block
};

// Per segment: check its table (lengths <= 11, Kraft), build its 11-bit
// lookup table, and place its chunks' packed bodies.
__global__ void __launch_bounds__(256) k_huff_dec_prep(HuffDecParams p) {
  __shared__ uint8_t s_len[256];
  __shared__ uint32_t s_cnt[16];
  __shared__ uint16_t s_lut[kLutSize];
  __shared__ uint64_t s_w[8];
  __shared__ uint64_t s_carry, s_carry2;
  __shared__ uint32_t s_ok;
  const Geom &g = p.g;
  const uint32_t s = blockIdx.x, t = threadIdx.x;
  const uint8_t *tab = huff_table(const_cast<uint8_t *>(p.src), g, s);
  s_len[t] = (tab[t >> 1] >> ((t & 1) * 4)) & 15u;
  if (t < 16) s_cnt[t] = 0;
  if (t == 0) {
    s_ok = 1;
    s_carry = 0;
    s_carry2 = 0;
  }
  for (uint32_t k = t; k < kLutSize; k += blockDim.x) s_lut[k] = 0;
  __syncthreads();
  if (s_len[t]) atomicAdd(&s_cnt[s_len[t]], 1u);
  __syncthreads();
  if (t == 0) {
    for (uint32_t l = kHuffMaxLen + 1; l < 16; ++l)
      if (s_cnt[l]) s_ok = 0;
    uint64_t kraft = 0;
    for (uint32_t l = 1; l <= kHuffMaxLen; ++l) kraft += (uint64_t)s_cnt[l] << (kHuffMaxLen - l);
    if (kraft > (1ull << kHuffMaxLen)) s_ok = 0;
    uint32_t code = 0, prev = 0;
    for (uint32_t bits = 1; bits <= kHuffMaxLen; ++bits) {
      code = (code + prev) << 1;
      prev = s_cnt[bits];
      s_cnt[bits] = code;  // first code of this length
    }
  }
  const bool raw = __syncthreads_or(t < 128 && tab[t] != 0) == 0;
  const bool ok = s_ok != 0;
  const uint32_t l = s_len[t];
  if (!raw && ok && l) {
    uint32_t r = 0;
    for (uint32_t u = 0; u < t; ++u) r += s_len[u] == l;
    const uint32_t rc = bitrev(s_cnt[l] + r, l);
    for (uint32_t fill = 0; fill < (1u << (kHuffMaxLen - l)); ++fill)
      s_lut[rc | (fill << l)] = (uint16_t)(t | (l << 8));
  }
  __syncthreads();
  if (!raw && ok) {
    uint32_t *d32 = reinterpret_cast<uint32_t *>(p.lut + (uint64_t)s * kLutSize);
    const uint32_t *l32 = reinterpret_cast<const uint32_t *>(s_lut);
    for (uint32_t k = t; k < kLutSize / 2; k += blockDim.x) d32[k] = l32[k];
  }
  if (t == 0) {
    p.seg_flags[s] = (raw ? 1u : 0u) | (ok ? 0u : 2u);
    if (!ok) set_status(p.status, SPRINTZ_ERR_CORRUPT);
  }
  uint32_t c0, c1;
  seg_chunks(g, s, &c0, &c1);
  for (uint64_t base = c0; base < c1; base += 256) {
    const uint64_t c = base + t;
    const uint32_t v = c < c1 ? le32(p.src + kHdrBytes + c * kEntryBytes + 12) : 0;
    const uint64_t excl = block_scan256(v, s_w, &s_carry);
    const uint32_t ns = c < c1 ? huff_n_sub(v) : 0;
    const uint64_t sub0 = block_scan256(ns, s_w, &s_carry2);
    if (c < c1) {
      p.chunk_poff[c] = excl;
      p.chunk_sub0[c] = sub0;
      // a body larger than any valid one: its sub-blocks have no slots
      if (ns > p.slots) set_status(p.status, SPRINTZ_ERR_CORRUPT);
      uint64_t *m = p.sub_map + (uint64_t)s * p.seg_slots;
      for (uint32_t k = 0; k < ns && sub0 + k < p.seg_slots; ++k) m[sub0 + k] = (c << 32) | k;
    }
  }
  if (t == 0) {
    p.seg_packed[s] = s_carry;
    p.seg_nsub[s] = s_carry2;
  }
}

// Decode `n` symbols of one sub-block's code [in, in + bytes) into out with
// the 11-bit table.  The bit buffer (least significant bit first) holds at
// least 32 bits before every pair of symbols: it is refilled from aligned
// 32-bit words, the next one already loaded (zeros past the code's words,
// bytes only past the end of the stream buffer).  Symbols leave in 8-byte
// stores once out is aligned.  True when every symbol has a code and the
// symbols use exactly the code's bytes.
__device__ __forceinline__ bool huff_decode_sub(const uint8_t *in, uint64_t bytes, uint32_t n, uint8_t *out,
                                                const uint16_t *lut, uintptr_t buf_end) {
  const uintptr_t ia = (uintptr_t)in;
  const uint32_t *w32 = reinterpret_cast<const uint32_t *>(ia & ~(uintptr_t)3);
  const uint32_t lead = (uint32_t)(ia & 3);  // bytes of the first word before the code
  const uint64_t words = (bytes + lead + 3) / 4;
  auto load = [&](uint64_t i) -> uint32_t {
    if (i >= words) return 0u;
    const uintptr_t a = (uintptr_t)(w32 + i);
    if (a + 4 <= buf_end) return __ldg(w32 + i);
    uint32_t v = 0;
    for (uint32_t q = 0; q < 4; ++q)
      if (a + q < buf_end) v |= (uint32_t)*reinterpret_cast<const uint8_t *>(a + q) << (8 * q);
    return v;
  };
  uint64_t buf = ((uint64_t)load(0) | ((uint64_t)load(1) << 32)) >> (8 * lead);
  uint32_t have = 64 - 8 * lead;
  uint32_t nxt = load(2);
  uint64_t wi = 3;  // words loaded (nxt is the last, not yet in buf)
  bool bad = false;
  auto refill = [&]() {
    if (have < 32) {
      buf |= (uint64_t)nxt << have;
      have += 32;
      nxt = load(wi);
      ++wi;
    }
  };
  auto dec1 = [&]() -> uint32_t {
    const uint32_t ent = lut[buf & (kLutSize - 1)];
    const uint32_t l = ent >> 8;
    bad |= l == 0;
    buf >>= l;
    have -= l;
    return ent & 0xFFu;
  };
  const uint32_t head = min((uint32_t)((8 - ((uintptr_t)out & 7)) & 7), n);
  uint32_t k = 0;
  for (; k < head; ++k) {
    refill();
    out[k] = (uint8_t)dec1();
  }
  for (; k + 8 <= n; k += 8) {
    uint64_t o = 0;
#pragma unroll
    for (uint32_t q = 0; q < 8; q += 2) {
      refill();
      o |= (uint64_t)dec1() << (8 * q);
      o |= (uint64_t)dec1() << (8 * q + 8);
    }
    *reinterpret_cast<uint64_t *>(out + k) = o;
  }
  for (; k < n; ++k) {
    refill();
    out[k] = (uint8_t)dec1();
  }
  const uint64_t used = 32ull * (wi - 1) - 8ull * lead - have;  // bits taken from the code
  return !bad && (used + 7) / 8 == bytes;
}

// One thread per sub-block: CTA (segment, part) covers sub-blocks
// [part * blockDim, (part + 1) * blockDim) of its segment; the map built by
// k_huff_dec_prep gives each its chunk and index.  Every sub-block decodes
// into the Huffman-free stream P; the thread of sub-block 0 writes the
// chunk's entry of P's table.
__global__ void __launch_bounds__(kHuffDecThreads, 10) k_huff_decode(HuffDecParams p) {
  __shared__ __align__(16) uint16_t lut[kLutSize];
  const Geom &g = p.g;
  const uint32_t s = blockIdx.x / p.parts, part = blockIdx.x % p.parts, t = threadIdx.x;
  const uint32_t flags = p.seg_flags[s];
  if (flags & 2u) return;
  const bool raw = (flags & 1u) != 0;
  if (!raw) {
    const uint32_t *l32 = reinterpret_cast<const uint32_t *>(p.lut + (uint64_t)s * kLutSize);
    uint32_t *d32 = reinterpret_cast<uint32_t *>(lut);
    for (uint32_t k = t; k < kLutSize / 2; k += blockDim.x) d32[k] = l32[k];
  }
  __syncthreads();
  const uint64_t j = (uint64_t)part * blockDim.x + t;
  if (j >= p.seg_nsub[s] || j >= p.seg_slots) return;
  const uint64_t m = p.sub_map[(uint64_t)s * p.seg_slots + j];
  const uint32_t c = (uint32_t)(m >> 32), k = (uint32_t)m;
  if (c >= g.n_chunks) {  // an entry a corrupt segment left unset
    set_status(p.status, SPRINTZ_ERR_CORRUPT);
    return;
  }
  const uint8_t *e = p.src + kHdrBytes + (uint64_t)c * kEntryBytes;
  const uint64_t off = le64(e);
  const uint32_t nrec = le32(e + 8), packed = le32(e + 12);
  const uint32_t n_sub = huff_n_sub(packed);
  if (k >= n_sub) {
    set_status(p.status, SPRINTZ_ERR_CORRUPT);
    return;
  }
  const uint64_t tail_off = le64(p.src + 48);
  const uint64_t data_bytes = tail_off >= g.data_off && tail_off <= p.src_size ? tail_off - g.data_off : 0;
  const uint64_t end = c + 1 < g.n_chunks ? le64(e + kEntryBytes) : data_bytes;
  const uint64_t poff = p.seg_prefix[s] + p.chunk_poff[c];
  bool bad = off > end || end > data_bytes || p.p_data_off + poff + packed > p.p_cap || n_sub > p.slots;
  const uint64_t coded = bad ? 0 : end - off;
  const uint8_t *in = p.src + g.data_off + off;
  uint64_t i0;
  uint32_t n;
  huff_sub_range(packed, k, &i0, &n);
  uint8_t *out = p.P + p.p_data_off + poff + i0;
  if (!bad && raw) {
    bad = coded != packed;
    if (!bad)
      for (uint32_t i = 0; i < n; ++i) out[i] = in[i0 + i];
  } else if (!bad) {
    const uint64_t jump = 4ull * (n_sub - 1);
    bad = jump > coded;
    if (!bad) {
      const uint64_t span = coded - jump;
      const uint64_t s0 = k ? le32(in + 4ull * (k - 1)) : 0;
      const uint64_t s1 = k + 1 < n_sub ? le32(in + 4ull * k) : span;
      bad = s0 > s1 || s1 > span;
      if (!bad) bad = !huff_decode_sub(in + jump + s0, s1 - s0, n, out, lut, (uintptr_t)p.src + p.src_size);
    }
  }
  if (bad) {
    set_status(p.status, SPRINTZ_ERR_CORRUPT);
    return;
  }
  if (k == 0) {
    uint8_t *pe = p.P + kHdrBytes + (uint64_t)c * kEntryBytes;
    put_le(pe, poff, 8);
    put_le(pe + 8, nrec, 4);
    put_le(pe + 12, packed, 4);
  }
}

// Header and tail of the Huffman-free stream P.
__global__ void k_huff_dec_finish(HuffDecParams p) {
  const Geom &g = p.g;
  const uint64_t packed_total = p.seg_prefix[g.n_segments];
  const uint64_t tail_off_p = p.p_data_off + packed_total;
  const uint64_t tail_bytes = g.tail_rows * g.D * g.wb;
  const uint64_t total_p = tail_off_p + tail_bytes;
  const uint64_t tail_off = le64(p.src + 48);
  if (total_p > p.p_cap || tail_off + tail_bytes > p.src_size) {
    if (threadIdx.x == 0) set_status(p.status, SPRINTZ_ERR_CORRUPT);
    return;
  }
  for (uint64_t k = threadIdx.x; k < tail_bytes; k += blockDim.x) p.P[tail_off_p + k] = p.src[tail_off + k];
  if (threadIdx.x == 0) {
    uint8_t *h = p.P;
    for (int k = 0; k < 64; ++k) h[k] = p.src[k];
    h[7] = 0;                  // no Huffman
    put_le(h + 16, 0, 4);      // huff_chunks field of a Huffman-free stream
    put_le(h + 40, p.p_data_off, 8);
    put_le(h + 48, tail_off_p, 8);
    put_le(h + 56, total_p, 8);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

static uint64_t a256(uint64_t v) { return (v + 255) & ~255ull; }

static Geom plain_geom(const Geom &g) {
  Geom gp = g;
  gp.huffman = 0;
  gp.huff_chunks = 0;
  gp.n_segments = 0;
  gp.data_off = kHdrBytes + (uint64_t)kEntryBytes * g.n_chunks;
  return gp;
}

static uint64_t plain_cap(const Geom &g) {
  uint64_t total = g.data_off;
  if (g.n_chunks) {
    const uint64_t full = g.full_rows / g.chunk_rows;
    const uint64_t last_rows = g.full_rows - full * g.chunk_rows;
    total += full * max_body_bytes(g.chunk_rows / 8, g.D, g.w, g.G);
    if (last_rows) total += max_body_bytes(last_rows / 8, g.D, g.w, g.G);
  }
  return total + g.tail_rows * g.D * g.wb;
}

// Sub-block slots per chunk: the sub-blocks of the largest possible body.
static uint32_t huff_slots(const Geom &g) {
  return (uint32_t)std::max<uint64_t>(1, (g.max_body + kHuffSub - 1) / kHuffSub);
}

constexpr uint64_t kHistSlice = 64 * 1024;  // packed bytes per histogram CTA

struct HuffEncLayout {
  uint64_t P, P_cap, size_word, hist, codes, seg_coded, seg_raw, seg_total, seg_prefix, chunk_coded, chunk_pos,
      sub_off, inner, inner_bytes, total;
  uint32_t slots, slices;
};

static HuffEncLayout huff_enc_layout(const Geom &g, const LaunchCfg &cfg) {
  HuffEncLayout L{};
  const Geom gp = plain_geom(g);
  const uint64_t ns = g.n_segments, nc = g.n_chunks;
  L.slots = huff_slots(g);
  const uint64_t seg_chunks_max = std::min<uint64_t>(g.huff_chunks ? g.huff_chunks : 1, std::max<uint64_t>(nc, 1));
  L.slices = (uint32_t)std::max<uint64_t>(1, (seg_chunks_max * g.max_body + kHistSlice - 1) / kHistSlice);
  L.P = 0;
  L.P_cap = plain_cap(gp);
  L.size_word = a256(L.P_cap + 16);  // P keeps 16 bytes of slack for word reads past its end
  L.hist = L.size_word + 256;
  L.codes = a256(L.hist + 8 * 256 * ns);
  L.seg_coded = a256(L.codes + 4 * 256 * ns);
  L.seg_raw = a256(L.seg_coded + 8 * ns);
  L.seg_total = a256(L.seg_raw + 4 * ns);
  L.seg_prefix = a256(L.seg_total + 8 * ns);
  L.chunk_coded = a256(L.seg_prefix + 8 * (ns + 1));
  L.chunk_pos = a256(L.chunk_coded + 8 * nc);
  L.sub_off = a256(L.chunk_pos + 8 * nc);
  L.inner = a256(L.sub_off + 4 * nc * L.slots);
  L.inner_bytes = encode_workspace_bytes(gp, cfg);
  L.total = L.inner + L.inner_bytes;
  return L;
}

uint64_t huff_encode_workspace_bytes(const Geom &g, const LaunchCfg &cfg) {
  return huff_enc_layout(g, cfg).total;
}

int launch_encode_huffman(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint8_t *dst,
                          uint64_t dst_cap, uint64_t *d_out_size, uint8_t *ws, uint64_t ws_bytes,
                          int *d_status, cudaStream_t stream) {
  // no full block: header (with the Huffman flag) and raw tail only
  if (g.n_chunks == 0) return launch_encode(g, cfg, src, dst, dst_cap, d_out_size, ws, ws_bytes, d_status, stream);
  const HuffEncLayout L = huff_enc_layout(g, cfg);
  if (ws_bytes < L.total) return SPRINTZ_ERR_WS_TOO_SMALL;
  const uint64_t hist_grid = (uint64_t)g.n_segments * L.slices;
  // the encoder's persistent warps: as many as fit, each over an equal
  // contiguous range of sub-block slots
  int enc_occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&enc_occ, k_huff_encode, kHuffEncWarps * 32, 0) != cudaSuccess ||
      enc_occ < 1)
    enc_occ = 1;
  const uint64_t enc_slots = std::max<uint64_t>(1, (uint64_t)g.n_chunks * L.slots);
  const uint64_t enc_warps = std::min<uint64_t>(enc_slots, (uint64_t)cfg.sm_count * enc_occ * kHuffEncWarps);
  const uint64_t enc_per_warp = (enc_slots + enc_warps - 1) / enc_warps;
  const uint64_t enc_grid = ((enc_slots + enc_per_warp - 1) / enc_per_warp + kHuffEncWarps - 1) / kHuffEncWarps;
  if (hist_grid > 0x7FFFFFFFull || enc_grid > 0x7FFFFFFFull) return SPRINTZ_ERR_UNSUPPORTED;
  const Geom gp = plain_geom(g);
  uint8_t *P = ws + L.P;
  int rc = launch_encode_fast(gp, cfg, src, P, L.P_cap, reinterpret_cast<uint64_t *>(ws + L.size_word),
                              ws + L.inner, L.inner_bytes, d_status, stream);
  if (rc != SPRINTZ_OK) return rc;
  HuffEncParams hp{};
  hp.P = P;
  hp.dst = dst;
  hp.dst_cap = dst_cap;
  hp.out_size = d_out_size;
  hp.src = src;
  hp.status = d_status;
  hp.g = g;
  hp.p_data_off = gp.data_off;
  hp.p_body_cap = L.P_cap - gp.data_off;
  hp.slots = L.slots;
  hp.slices = L.slices;
  hp.slice_bytes = kHistSlice;
  hp.hist = reinterpret_cast<unsigned long long *>(ws + L.hist);
  hp.codes = reinterpret_cast<uint32_t *>(ws + L.codes);
  hp.seg_coded = reinterpret_cast<unsigned long long *>(ws + L.seg_coded);
  hp.seg_raw = reinterpret_cast<uint32_t *>(ws + L.seg_raw);
  hp.seg_total = reinterpret_cast<uint64_t *>(ws + L.seg_total);
  hp.seg_prefix = reinterpret_cast<uint64_t *>(ws + L.seg_prefix);
  hp.chunk_coded = reinterpret_cast<uint64_t *>(ws + L.chunk_coded);
  hp.chunk_pos = reinterpret_cast<uint64_t *>(ws + L.chunk_pos);
  hp.sub_off = reinterpret_cast<uint32_t *>(ws + L.sub_off);
  if (cudaMemsetAsync(hp.hist, 0, 8ull * 256 * g.n_segments, stream) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  k_huff_hist<<<(uint32_t)hist_grid, kHuffWarps * 32, 0, stream>>>(hp);
  k_huff_lengths<<<g.n_segments, kHuffThreads, 0, stream>>>(hp);
  k_huff_sizes<<<(g.n_chunks + kHuffWarps - 1) / kHuffWarps, kHuffWarps * 32, 0, stream>>>(hp);
  k_huff_decide<<<g.n_segments, 256, 0, stream>>>(hp);
  k_huff_scan<<<1, 1024, 0, stream>>>(hp.seg_total, hp.seg_prefix, g.n_segments);
  k_huff_encode<<<(uint32_t)enc_grid, kHuffEncWarps * 32, 0, stream>>>(hp, enc_per_warp);
  k_huff_enc_finish<<<1, 256, 0, stream>>>(hp);
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

struct HuffDecLayout {
  uint64_t P, P_cap, lut, seg_flags, seg_packed, seg_prefix, chunk_poff, chunk_sub0, seg_nsub, sub_map, inner,
      inner_bytes, total, seg_slots;
  uint32_t slots, threads, parts;
};

static HuffDecLayout huff_dec_layout(const Geom &g, const LaunchCfg &cfg) {
  HuffDecLayout L{};
  const Geom gp = plain_geom(g);
  const uint64_t ns = g.n_segments, nc = g.n_chunks;
  L.slots = huff_slots(g);
  const uint64_t seg_slots =
      std::min<uint64_t>(g.huff_chunks ? g.huff_chunks : 1, std::max<uint64_t>(nc, 1)) * L.slots;
  L.seg_slots = seg_slots;
  L.threads = (uint32_t)std::min<uint64_t>(kHuffDecThreads, (seg_slots + 31) & ~31ull);
  L.parts = (uint32_t)((seg_slots + L.threads - 1) / L.threads);
  L.P = 0;
  L.P_cap = plain_cap(gp);
  L.lut = a256(L.P_cap + 16);
  L.seg_flags = a256(L.lut + 2ull * kLutSize * ns);
  L.seg_packed = a256(L.seg_flags + 4 * ns);
  L.seg_prefix = a256(L.seg_packed + 8 * ns);
  L.chunk_poff = a256(L.seg_prefix + 8 * (ns + 1));
  L.chunk_sub0 = a256(L.chunk_poff + 8 * nc);
  L.seg_nsub = a256(L.chunk_sub0 + 8 * nc);
  L.sub_map = a256(L.seg_nsub + 8 * ns);
  L.inner = a256(L.sub_map + 8 * ns * seg_slots);
  L.inner_bytes = decode_workspace_bytes(gp, cfg);
  L.total = L.inner + L.inner_bytes;
  return L;
}

uint64_t huff_decode_workspace_bytes(const Geom &g, const LaunchCfg &cfg) {
  return huff_dec_layout(g, cfg).total;
}

int launch_decode_huffman(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint64_t src_size,
                          uint8_t *dst, uint64_t dst_cap, uint8_t *ws, uint64_t ws_bytes, int *d_status,
                          cudaStream_t stream) {
  const HuffDecLayout L = huff_dec_layout(g, cfg);
  if (ws_bytes < L.total) return SPRINTZ_ERR_WS_TOO_SMALL;
  const uint64_t dec_grid = (uint64_t)g.n_segments * L.parts;
  if (dec_grid > 0x7FFFFFFFull) return SPRINTZ_ERR_UNSUPPORTED;
  const Geom gp = plain_geom(g);
  HuffDecParams hp{};
  hp.src = src;
  hp.src_size = src_size;
  hp.P = ws + L.P;
  hp.p_cap = L.P_cap;
  hp.status = d_status;
  hp.g = g;
  hp.p_data_off = gp.data_off;
  hp.slots = L.slots;
  hp.parts = L.parts;
  hp.lut = reinterpret_cast<uint16_t *>(ws + L.lut);
  hp.seg_flags = reinterpret_cast<uint32_t *>(ws + L.seg_flags);
  hp.seg_packed = reinterpret_cast<uint64_t *>(ws + L.seg_packed);
  hp.seg_prefix = reinterpret_cast<uint64_t *>(ws + L.seg_prefix);
  hp.chunk_poff = reinterpret_cast<uint64_t *>(ws + L.chunk_poff);
  hp.chunk_sub0 = reinterpret_cast<uint64_t *>(ws + L.chunk_sub0);
  hp.seg_nsub = reinterpret_cast<uint64_t *>(ws + L.seg_nsub);
  hp.seg_slots = L.seg_slots;
  hp.sub_map = reinterpret_cast<uint64_t *>(ws + L.sub_map);
  if (g.n_chunks) {
    k_huff_dec_prep<<<g.n_segments, 256, 0, stream>>>(hp);
    k_huff_scan<<<1, 1024, 0, stream>>>(hp.seg_packed, hp.seg_prefix, g.n_segments);
    k_huff_decode<<<(uint32_t)dec_grid, L.threads, 0, stream>>>(hp);
  } else {
    cudaMemsetAsync(hp.seg_prefix, 0, 8, stream);
  }
  k_huff_dec_finish<<<1, 128, 0, stream>>>(hp);
  if (cudaGetLastError() != cudaSuccess) return SPRINTZ_ERR_CUDA;
  return launch_decode(gp, cfg, hp.P, L.P_cap, dst, dst_cap, ws + L.inner, L.inner_bytes, d_status, stream);
}

}  // namespace spz
