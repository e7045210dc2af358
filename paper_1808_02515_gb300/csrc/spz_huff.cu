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
// Encode: the regular encoder writes the Huffman-free stream P into the
// workspace; k_huff_build (one CTA per segment) histograms the segment's
// packed bytes, builds its lengths and table and sizes every chunk's code;
// k_huff_scan places the segments; k_huff_encode (one CTA per segment) writes
// the coded chunks, the chunk table and, in the last segment, header and tail.
// Decode: k_huff_decode (one CTA per segment, one thread per chunk) decodes
// each chunk's bitstream with an 11-bit lookup table into a Huffman-free
// stream in the workspace, which the regular decoder then decodes.
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
  uint32_t hist[256];
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
  const uint32_t f = sm.hist[t];
  if (f) atomicAdd(&sm.n_used, 1u);
  sm.len[t] = 0;
  __syncthreads();
  const uint32_t n = sm.n_used;
  // rank among used symbols by (frequency, symbol)
  if (f) {
    uint32_t r = 0;
    for (uint32_t u = 0; u < 256; ++u) {
      const uint32_t fu = sm.hist[u];
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
// Encode
// ---------------------------------------------------------------------------

struct HuffEncParams {
  const uint8_t *P;      // Huffman-free stream (regular encoder output)
  uint8_t *dst;
  uint64_t dst_cap;
  uint64_t *out_size;
  const uint8_t *src;    // raw samples (for the tail)
  int *status;
  Geom g;                // the Huffman stream's geometry
  uint64_t p_data_off;   // data offset of P
  uint32_t *chunk_coded; // [n_chunks] coded bytes of each chunk
  uint64_t *seg_total;   // [n_segments] coded bytes of each segment
  uint64_t *seg_prefix;  // [n_segments + 1]
  uint32_t *gbuf;        // per-segment code buffers in global memory when a chunk's code
  uint64_t gbuf_words;   // does not fit shared memory (else null)
};

// Chunk c of P: body offset (from P's data), records, packed bytes.
__device__ __forceinline__ void p_entry(const HuffEncParams &p, uint32_t c, uint64_t *off, uint32_t *nrec,
                                        uint32_t *packed) {
  const uint8_t *e = p.P + kHdrBytes + (uint64_t)c * kEntryBytes;
  *off = le64(e);
  *nrec = le32(e + 8);
  *packed = le32(e + 12);
}

__global__ void __launch_bounds__(kHuffThreads) k_huff_build(HuffEncParams p) {
  __shared__ HuffSmem sm;
  __shared__ uint64_t s_bits[kHuffThreads / 32];
  const Geom &g = p.g;
  const uint32_t s = blockIdx.x;
  const uint32_t c0 = s * g.huff_chunks;
  const uint32_t c1 = min(g.n_chunks, c0 + g.huff_chunks);
  const uint32_t t = threadIdx.x;
  // histogram of the segment's packed bytes (its bodies are contiguous in P)
  uint64_t o0, o1;
  uint32_t nr, pk;
  p_entry(p, c0, &o0, &nr, &pk);
  p_entry(p, c1 - 1, &o1, &nr, &pk);
  o1 += pk;
  sm.hist[t] = 0;
  __syncthreads();
  const uint8_t *bytes = p.P + p.p_data_off;
  for (uint64_t k = o0 + t; k < o1; k += blockDim.x) atomicAdd(&sm.hist[bytes[k]], 1u);
  __syncthreads();
  huff_lengths(sm);
  // coded size of every chunk of the segment: one warp per chunk
  {
    const uint32_t lane = t & 31, wid = t >> 5;
    uint64_t mine = 0;
    for (uint32_t c = c0 + wid; c < c1; c += kHuffThreads / 32) {
      uint64_t off;
      uint32_t nrec, packed;
      p_entry(p, c, &off, &nrec, &packed);
      uint64_t bits = 0;
      for (uint64_t k = off + lane; k < off + packed; k += 32) bits += sm.len[bytes[k]];
      for (int o = 16; o > 0; o >>= 1) bits += __shfl_xor_sync(0xFFFFFFFFu, bits, o);
      const uint32_t cb = (uint32_t)((bits + 7) / 8);
      if (lane == 0) p.chunk_coded[c] = cb;
      mine += cb;
    }
    if (lane == 0) s_bits[wid] = mine;
    __syncthreads();
  }
  uint64_t coded_total = 0;
  for (int w = 0; w < kHuffThreads / 32; ++w) coded_total += s_bits[w];
  const uint64_t packed_total = o1 - o0;
  const bool raw = packed_total == 0 || coded_total >= packed_total;
  if (raw) {
    sm.len[t] = 0;
    __syncthreads();
    for (uint32_t c = c0 + t; c < c1; c += blockDim.x) {
      uint64_t off;
      uint32_t nrec, packed;
      p_entry(p, c, &off, &nrec, &packed);
      p.chunk_coded[c] = packed;
    }
  }
  // the segment's table: 256 lengths, 4 bits each, symbol 2k in the low nibble
  uint8_t *tab = p.dst + kHdrBytes + (uint64_t)kEntryBytes * g.n_chunks + (uint64_t)kHuffTableBytes * s;
  if (t < 128) tab[t] = (uint8_t)(sm.len[2 * t] | (sm.len[2 * t + 1] << 4));
  if (t == 0) p.seg_total[s] = raw ? packed_total : coded_total;
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

__global__ void __launch_bounds__(kHuffThreads) k_huff_encode(HuffEncParams p) {
  __shared__ HuffSmem sm;
  __shared__ uint32_t s_bits[kHuffThreads];
  extern __shared__ __align__(16) uint32_t obuf[];  // one chunk's code, bit-packed
  const Geom &g = p.g;
  const uint32_t s = blockIdx.x;
  const uint32_t c0 = s * g.huff_chunks;
  const uint32_t c1 = min(g.n_chunks, c0 + g.huff_chunks);
  const uint32_t t = threadIdx.x;
  // the table this segment was given
  const uint8_t *tab = p.dst + kHdrBytes + (uint64_t)kEntryBytes * g.n_chunks + (uint64_t)kHuffTableBytes * s;
  sm.len[t] = (tab[t >> 1] >> ((t & 1) * 4)) & 15u;
  __syncthreads();
  huff_codes(sm);
  // codes bit-reversed once: the stream is least significant bit first
  sm.code[t] = bitrev(sm.code[t], sm.len[t]);
  const bool raw = __syncthreads_or(sm.len[t] != 0) == 0;
  const uint8_t *bytes = p.P + p.p_data_off;
  uint64_t pos = p.seg_prefix[s];
  for (uint32_t c = c0; c < c1; ++c) {
    uint64_t off;
    uint32_t nrec, packed;
    p_entry(p, c, &off, &nrec, &packed);
    const uint32_t coded = p.chunk_coded[c];
    uint8_t *d = p.dst + g.data_off + pos;
    if (t == 0) {
      uint8_t *e = p.dst + kHdrBytes + (uint64_t)c * kEntryBytes;
      put_le(e, pos, 8);
      put_le(e + 8, nrec, 4);
      put_le(e + 12, packed, 4);
    }
    if (raw) {
      for (uint32_t k = t; k < packed; k += blockDim.x) d[k] = bytes[off + k];
    } else {
      // each thread codes a contiguous run of the chunk's bytes; a block scan
      // of the runs' bit counts places them
      const uint32_t per = (packed + blockDim.x - 1) / blockDim.x;
      const uint32_t k0 = min(packed, t * per), k1 = min(packed, k0 + per);
      uint32_t nb = 0;
      for (uint32_t k = k0; k < k1; ++k) nb += sm.len[bytes[off + k]];
      s_bits[t] = nb;
      const uint32_t words = (coded + 3) / 4;
      uint32_t *ob32 = p.gbuf ? p.gbuf + (uint64_t)s * p.gbuf_words : obuf;
      for (uint32_t k = t; k < words; k += blockDim.x) ob32[k] = 0;
      __syncthreads();
      // exclusive scan of s_bits (Hillis-Steele in place)
      for (uint32_t o = 1; o < blockDim.x; o <<= 1) {
        const uint32_t v = t >= o ? s_bits[t - o] : 0;
        __syncthreads();
        s_bits[t] += v;
        __syncthreads();
      }
      uint32_t bit = s_bits[t] - nb;
      for (uint32_t k = k0; k < k1; ++k) {
        const uint32_t sym = bytes[off + k];
        const uint32_t l = sm.len[sym];
        const uint32_t v = sm.code[sym];
        const uint32_t wi = bit >> 5, sh = bit & 31;
        atomicOr(&ob32[wi], v << sh);
        if (sh + l > 32) atomicOr(&ob32[wi + 1], v >> (32 - sh));
        bit += l;
      }
      __syncthreads();
      const uint8_t *ob = reinterpret_cast<const uint8_t *>(ob32);
      for (uint32_t k = t; k < coded; k += blockDim.x) d[k] = ob[k];
    }
    __syncthreads();
    pos += coded;
  }
  if (s == g.n_segments - 1 && t == 0) {
    const uint64_t tail_off = g.data_off + p.seg_prefix[g.n_segments];
    const uint64_t tail_bytes = g.tail_rows * g.D * g.wb;
    const uint64_t total = tail_off + tail_bytes;
    if (total <= p.dst_cap) {
      for (uint64_t k = 0; k < tail_bytes; ++k) p.dst[tail_off + k] = p.src[g.full_rows * g.D * g.wb + k];
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
    } else {
      set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
    }
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
  uint64_t *seg_packed;  // [n_segments] packed bytes per segment, then its prefix
  uint64_t *seg_prefix;  // [n_segments + 1]
};

// Packed bytes of every segment (one thread per segment).
__global__ void k_huff_seg_packed(HuffDecParams p) {
  const Geom &g = p.g;
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.n_segments) return;
  const uint32_t c0 = s * g.huff_chunks, c1 = min(g.n_chunks, c0 + g.huff_chunks);
  uint64_t sum = 0;
  for (uint32_t c = c0; c < c1; ++c) sum += le32(p.src + kHdrBytes + (uint64_t)c * kEntryBytes + 12);
  p.seg_packed[s] = sum;
}

// One CTA per segment, one thread per chunk: decode each chunk's bitstream
// into the Huffman-free stream P (its body and its chunk-table entry).
__global__ void __launch_bounds__(64) k_huff_decode(HuffDecParams p) {
  __shared__ uint8_t s_len[256];
  __shared__ uint32_t s_code[256];
  __shared__ uint32_t s_cnt[16];
  __shared__ uint16_t lut[1u << kHuffMaxLen];  // symbol | length << 8
  __shared__ uint32_t s_packed[64];
  __shared__ uint32_t s_ok;
  const Geom &g = p.g;
  const uint32_t s = blockIdx.x;
  const uint32_t t = threadIdx.x;
  const uint8_t *tab = p.src + kHdrBytes + (uint64_t)kEntryBytes * g.n_chunks + (uint64_t)kHuffTableBytes * s;
  for (uint32_t k = t; k < 256; k += blockDim.x) s_len[k] = (tab[k >> 1] >> ((k & 1) * 4)) & 15u;
  if (t < 16) s_cnt[t] = 0;
  if (t == 0) s_ok = 1;
  __syncthreads();
  for (uint32_t k = t; k < 256; k += blockDim.x)
    if (s_len[k]) atomicAdd(&s_cnt[s_len[k]], 1u);
  __syncthreads();
  // lengths above 11 are invalid; the code must not be over-subscribed (Kraft)
  if (t == 0) {
    for (uint32_t l = kHuffMaxLen + 1; l < 16; ++l)
      if (s_cnt[l]) s_ok = 0;
    uint64_t kraft = 0;
    for (uint32_t l = 1; l <= kHuffMaxLen; ++l) kraft += (uint64_t)s_cnt[l] << (kHuffMaxLen - l);
    if (kraft > (1ull << kHuffMaxLen)) s_ok = 0;
    uint32_t code = 0;
    uint32_t prev = 0;
    for (uint32_t bits = 1; bits <= kHuffMaxLen; ++bits) {
      code = (code + prev) << 1;
      prev = s_cnt[bits];
      s_cnt[bits] = code;  // first code of this length
    }
  }
  const bool raw = __syncthreads_or((t < 128 && tab[t] != 0) || (t + 64 < 128 && tab[t + 64] != 0)) == 0;
  for (uint32_t k = t; k < 256; k += blockDim.x) {
    const uint32_t l = s_len[k];
    uint32_t r = 0;
    if (l)
      for (uint32_t u = 0; u < k; ++u) r += s_len[u] == l;
    s_code[k] = l ? s_cnt[l] + r : 0;
  }
  for (uint32_t k = t; k < (1u << kHuffMaxLen); k += blockDim.x) lut[k] = 0;
  __syncthreads();
  if (!raw && s_ok) {
    for (uint32_t k = t; k < 256; k += blockDim.x) {
      const uint32_t l = s_len[k];
      if (!l) continue;
      const uint32_t rc = bitrev(s_code[k], l);
      for (uint32_t fill = 0; fill < (1u << (kHuffMaxLen - l)); ++fill)
        lut[rc | (fill << l)] = (uint16_t)(k | (l << 8));
    }
  }
  __syncthreads();
  if (!s_ok) {
    if (t == 0) set_status(p.status, SPRINTZ_ERR_CORRUPT);
    return;
  }
  const uint32_t c0 = s * g.huff_chunks, c1 = min(g.n_chunks, c0 + g.huff_chunks);
  const uint64_t tail_off = le64(p.src + 48);
  const uint64_t data_bytes = tail_off >= g.data_off && tail_off <= p.src_size ? tail_off - g.data_off : 0;
  for (uint32_t cb = c0; cb < c1; cb += 64) {
    const uint32_t c = cb + t;
    const bool mine = c < c1;
    uint32_t packed = 0;
    if (mine) packed = le32(p.src + kHdrBytes + (uint64_t)c * kEntryBytes + 12);
    s_packed[t] = packed;
    __syncthreads();
    uint64_t poff = p.seg_prefix[s];
    for (uint32_t k = c0; k < c; ++k)
      poff += k < cb ? le32(p.src + kHdrBytes + (uint64_t)k * kEntryBytes + 12) : s_packed[k - cb];
    __syncthreads();
    if (!mine) continue;
    const uint8_t *e = p.src + kHdrBytes + (uint64_t)c * kEntryBytes;
    const uint64_t off = le64(e);
    const uint32_t nrec = le32(e + 8);
    const uint64_t end = c + 1 < g.n_chunks ? le64(e + kEntryBytes) : data_bytes;
    uint8_t *out = p.P + p.p_data_off + poff;
    bool bad = off > end || end > data_bytes || p.p_data_off + poff + packed > p.p_cap;
    const uint64_t coded = bad ? 0 : end - off;
    const uint8_t *in = p.src + g.data_off + off;
    if (!bad && raw) {
      bad = coded != packed;
      if (!bad)
        for (uint32_t k = 0; k < packed; ++k) out[k] = in[k];
    } else if (!bad) {
      // bit buffer, least significant bit first, refilled with aligned
      // 32-bit loads (bytes only past the end of the buffer); symbols leave
      // in 8-byte stores once the output is aligned
      const uintptr_t ia = (uintptr_t)in;
      const uint32_t *w32 = reinterpret_cast<const uint32_t *>(ia & ~(uintptr_t)3);
      const uint32_t lead = (uint32_t)(ia & 3);  // bytes of the first word before the chunk
      const uint64_t words = (coded + lead + 3) / 4;
      const uintptr_t buf_end = (uintptr_t)p.src + p.src_size;
      uint64_t buf = 0;
      uint32_t have = 0;
      uint64_t wi = 0;
      uint64_t used = 0;  // bits consumed
      auto refill = [&]() {
        while (have <= 32 && wi < words) {
          const uintptr_t a = (uintptr_t)(w32 + wi);
          uint32_t v = 0;
          if (a + 4 <= buf_end) {
            v = __ldg(w32 + wi);
          } else {
            for (uint32_t q = 0; q < 4; ++q)
              if (a + q < buf_end) v |= (uint32_t)*reinterpret_cast<const uint8_t *>(a + q) << (8 * q);
          }
          buf |= (uint64_t)v << have;
          have += 32;
          ++wi;
        }
      };
      refill();
      buf >>= 8 * lead;
      have -= 8 * lead;
      auto next = [&](uint32_t *sym) -> bool {
        refill();
        const uint32_t ent = lut[buf & ((1u << kHuffMaxLen) - 1)];
        const uint32_t l = ent >> 8;
        if (l == 0 || l > have) return false;
        *sym = ent & 0xFFu;
        buf >>= l;
        have -= l;
        used += l;
        return true;
      };
      const uint32_t head = min((uint32_t)((8 - ((uintptr_t)out & 7)) & 7), packed);
      uint32_t k = 0, sym = 0;
      for (; k < head && !bad; ++k) {
        if (!next(&sym)) bad = true;
        else out[k] = (uint8_t)sym;
      }
      for (; k + 8 <= packed && !bad; k += 8) {
        uint64_t o = 0;
#pragma unroll
        for (uint32_t q = 0; q < 8; ++q) {
          if (!next(&sym)) bad = true;
          o |= (uint64_t)sym << (8 * q);
        }
        if (!bad) *reinterpret_cast<uint64_t *>(out + k) = o;
      }
      for (; k < packed && !bad; ++k) {
        if (!next(&sym)) bad = true;
        else out[k] = (uint8_t)sym;
      }
      if (!bad && (used + 7) / 8 != coded) bad = true;
    }
    if (bad) {
      set_status(p.status, SPRINTZ_ERR_CORRUPT);
      continue;
    }
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

struct HuffEncLayout {
  uint64_t P, P_cap, size_word, coded, seg_total, seg_prefix, gbuf, gbuf_bytes, inner, inner_bytes, total;
  uint64_t obytes;  // one chunk's code buffer
  bool global_buf;  // the buffer lives in the workspace (too large for shared memory)
};

// Static shared memory of the Huffman encoder (its per-chunk code buffer is
// dynamic shared memory on top of it).
static uint64_t huff_encode_static_smem() {
  cudaFuncAttributes a{};
  if (cudaFuncGetAttributes(&a, k_huff_encode) != cudaSuccess) return 64 * 1024;
  return a.sharedSizeBytes;
}

static HuffEncLayout huff_enc_layout(const Geom &g, const LaunchCfg &cfg) {
  HuffEncLayout L{};
  const Geom gp = plain_geom(g);
  L.P = 0;
  L.P_cap = plain_cap(gp);
  L.size_word = a256(L.P_cap + 16);
  L.coded = L.size_word + 256;
  L.seg_total = a256(L.coded + 4ull * g.n_chunks);
  L.seg_prefix = a256(L.seg_total + 8ull * g.n_segments);
  L.obytes = ((g.max_body * kHuffMaxLen / 8 + 16) + 15) & ~15ull;
  L.global_buf = L.obytes + huff_encode_static_smem() > (uint64_t)cfg.max_smem_optin;
  L.gbuf = a256(L.seg_prefix + 8ull * (g.n_segments + 1));
  L.gbuf_bytes = L.global_buf ? (uint64_t)g.n_segments * L.obytes : 0;
  L.inner = a256(L.gbuf + L.gbuf_bytes);
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
  hp.chunk_coded = reinterpret_cast<uint32_t *>(ws + L.coded);
  hp.seg_total = reinterpret_cast<uint64_t *>(ws + L.seg_total);
  hp.seg_prefix = reinterpret_cast<uint64_t *>(ws + L.seg_prefix);
  k_huff_build<<<g.n_segments, kHuffThreads, 0, stream>>>(hp);
  k_huff_scan<<<1, 1024, 0, stream>>>(hp.seg_total, hp.seg_prefix, g.n_segments);
  uint64_t obytes = L.obytes;
  if (L.global_buf) {
    hp.gbuf = reinterpret_cast<uint32_t *>(ws + L.gbuf);
    hp.gbuf_words = L.obytes / 4;
    obytes = 0;
  } else if (cudaFuncSetAttribute(k_huff_encode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)obytes) !=
             cudaSuccess) {
    return SPRINTZ_ERR_CUDA;
  }
  k_huff_encode<<<g.n_segments, kHuffThreads, obytes, stream>>>(hp);
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

struct HuffDecLayout {
  uint64_t P, P_cap, seg_packed, seg_prefix, inner, inner_bytes, total;
};

static HuffDecLayout huff_dec_layout(const Geom &g, const LaunchCfg &cfg) {
  HuffDecLayout L{};
  const Geom gp = plain_geom(g);
  L.P = 0;
  L.P_cap = plain_cap(gp);
  L.seg_packed = a256(L.P_cap + 16);
  L.seg_prefix = a256(L.seg_packed + 8ull * g.n_segments);
  L.inner = a256(L.seg_prefix + 8ull * (g.n_segments + 1));
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
  const Geom gp = plain_geom(g);
  HuffDecParams hp{};
  hp.src = src;
  hp.src_size = src_size;
  hp.P = ws + L.P;
  hp.p_cap = L.P_cap;
  hp.status = d_status;
  hp.g = g;
  hp.p_data_off = gp.data_off;
  hp.seg_packed = reinterpret_cast<uint64_t *>(ws + L.seg_packed);
  hp.seg_prefix = reinterpret_cast<uint64_t *>(ws + L.seg_prefix);
  if (g.n_chunks) {
    k_huff_seg_packed<<<(g.n_segments + 127) / 128, 128, 0, stream>>>(hp);
    k_huff_scan<<<1, 1024, 0, stream>>>(hp.seg_packed, hp.seg_prefix, g.n_segments);
    k_huff_decode<<<g.n_segments, 64, 0, stream>>>(hp);
  } else {
    cudaMemsetAsync(hp.seg_prefix, 0, 8, stream);
  }
  k_huff_dec_finish<<<1, 128, 0, stream>>>(hp);
  if (cudaGetLastError() != cudaSuccess) return SPRINTZ_ERR_CUDA;
  return launch_decode(gp, cfg, hp.P, L.P_cap, dst, dst_cap, ws + L.inner, L.inner_bytes, d_status, stream);
}

}  // namespace spz
