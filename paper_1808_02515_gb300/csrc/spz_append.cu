// Appending rows to a compressed stream (sprintz_append).
//
// The stream of a series X followed by rows Y is, byte for byte, what
// compressing X ++ Y from scratch writes.  Chunks restart the forecaster, so
// every chunk of X that is complete (chunk_rows rows) encodes the same in
// both streams and keeps its body; only X's last chunk, if it is partial,
// and X's raw tail rows change, together with Y:
//   1. the rows of X from the first incomplete chunk on are rebuilt in the
//      workspace: that chunk decoded (Algorithm 2), X's raw tail copied,
//      then Y copied after them;
//   2. those rows are encoded (Algorithm 1) into a suffix stream in the
//      workspace;
//   3. one kernel writes the new stream: header, X's kept chunk entries,
//      the suffix's entries with their body offsets moved past X's kept
//      bodies, X's kept bodies, the suffix's bodies and its tail.
// The header check of X and every size the last step needs are read on the
// device; the host knows only the shapes.
#include <algorithm>

#include "spz_common.cuh"

namespace spz {

namespace {

__device__ __forceinline__ uint64_t rd_le(const uint8_t *p, int n) {
  uint64_t v = 0;
  for (int k = 0; k < n; ++k) v |= (uint64_t)p[k] << (8 * k);
  return v;
}
__device__ __forceinline__ void wr_le(uint8_t *p, uint64_t v, int n) {
  for (int k = 0; k < n; ++k) p[k] = (uint8_t)(v >> (8 * k));
}

uint64_t align256a(uint64_t v) { return (v + 255) & ~255ull; }

struct AppendParams {
  const uint8_t *src;     // stream of X
  uint64_t src_size;
  const uint8_t *suffix;  // stream of the rebuilt rows (workspace)
  uint8_t *dst;
  uint64_t dst_cap;
  uint64_t *out_size;
  int *status;
  Geom g_old;             // geometry of X
  uint32_t keep;          // chunks of X kept as they are
  uint32_t n_chunks;      // chunks of the new stream
  uint64_t rows;          // rows of the new stream
  uint64_t data_off;      // data offset of the new stream
  uint64_t sfx_data_off;  // data offset of the suffix stream (its shape fixes it)
  uint64_t sfx_cap;       // bytes the suffix stream may take
};

// X's header agrees with its geometry (the same fields the decoder checks).
__device__ bool old_header_ok(const AppendParams &p, uint64_t *data_bytes) {
  const Geom &g = p.g_old;
  const uint8_t *h = p.src;
  bool ok = p.src_size >= 64 && h[0] == 'S' && h[1] == 'P' && h[2] == 'Z' && h[3] == '1' && h[4] == 1 &&
            h[5] == g.w && h[6] == g.forecaster && h[7] == 0 && rd_le(h + 8, 2) == g.D && h[10] == g.G &&
            h[11] == g.learn_shift && rd_le(h + 12, 4) == g.chunk_rows_opt && rd_le(h + 20, 4) == g.n_chunks &&
            rd_le(h + 24, 8) == g.rows && rd_le(h + 32, 4) == g.tail_rows && rd_le(h + 40, 8) == g.data_off;
  const uint64_t tail_off = rd_le(h + 48, 8), total = rd_le(h + 56, 8);
  ok = ok && tail_off >= g.data_off && total <= p.src_size && total == tail_off + g.tail_rows * g.D * g.wb;
  *data_bytes = ok ? tail_off - g.data_off : 0;
  return ok;
}

// Step 3 (every CTA does its share of each copy; thread 0 of CTA 0 writes the
// header and the size).
__global__ void k_append_assemble(AppendParams p) {
  __shared__ uint32_t s_ok;
  __shared__ uint64_t s_keep_bytes, s_sfx_data_off, s_sfx_tail_off, s_sfx_total, s_total;
  const Geom &g = p.g_old;
  if (threadIdx.x == 0) {
    uint64_t data_bytes = 0;
    bool ok = old_header_ok(p, &data_bytes);
    // bytes of the kept bodies: where chunk `keep` starts, or all of them
    uint64_t keep_bytes = 0;
    if (ok) keep_bytes = p.keep < g.n_chunks ? rd_le(p.src + 64 + 16ull * p.keep, 8) : data_bytes;
    ok = ok && keep_bytes <= data_bytes;
    const uint8_t *h = p.suffix;
    const uint64_t sdo = rd_le(h + 40, 8), sto = rd_le(h + 48, 8), stot = rd_le(h + 56, 8);
    // the suffix's sizes are trusted only if they describe a stream that fits
    // where it was written (after a failed encode, the failure is reported)
    ok = ok && sdo == p.sfx_data_off && sto >= sdo && stot >= sto && stot <= p.sfx_cap;
    const uint64_t total = ok ? p.data_off + keep_bytes + (sto - sdo) + (stot - sto) : 0;
    if (!ok && blockIdx.x == 0) set_status(p.status, SPRINTZ_ERR_CORRUPT);
    if (ok && total > p.dst_cap) {
      ok = false;
      if (blockIdx.x == 0) set_status(p.status, SPRINTZ_ERR_DST_TOO_SMALL);
    }
    s_ok = ok;
    s_keep_bytes = keep_bytes;
    s_sfx_data_off = sdo;
    s_sfx_tail_off = sto;
    s_sfx_total = stot;
    s_total = total;
  }
  __syncthreads();
  if (!s_ok) return;
  const uint64_t keep_bytes = s_keep_bytes, sdo = s_sfx_data_off, sto = s_sfx_tail_off, stot = s_sfx_total;
  const uint32_t n_sfx = p.n_chunks - p.keep;
  // chunk entries: X's first `keep` as they are, then the suffix's with
  // their body offsets moved past X's kept bodies
  grid_copy(p.dst + 64, p.src + 64, 16ull * p.keep);
  const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t c = t0; c < n_sfx; c += nt) {
    const uint8_t *e = p.suffix + 64 + 16 * c;
    uint8_t *d = p.dst + 64 + 16 * ((uint64_t)p.keep + c);
    wr_le(d, rd_le(e, 8) + keep_bytes, 8);
    for (int k = 8; k < 16; ++k) d[k] = e[k];
  }
  // bodies and tail
  grid_copy(p.dst + p.data_off, p.src + g.data_off, keep_bytes);
  grid_copy(p.dst + p.data_off + keep_bytes, p.suffix + sdo, sto - sdo);
  grid_copy(p.dst + p.data_off + keep_bytes + (sto - sdo), p.suffix + sto, stot - sto);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    uint8_t *h = p.dst;
    for (int k = 0; k < 64; ++k) h[k] = p.suffix[k];
    wr_le(h + 20, p.n_chunks, 4);
    wr_le(h + 24, p.rows, 8);
    wr_le(h + 40, p.data_off, 8);
    wr_le(h + 48, p.data_off + keep_bytes + (sto - sdo), 8);
    wr_le(h + 56, s_total, 8);
    *p.out_size = s_total;
  }
}

// Chunks of X kept as they are: all complete chunks before the first partial
// one (chunk_rows = 0: the one chunk is never complete).
uint32_t kept_chunks(const Geom &g) {
  if (g.n_chunks == 0 || g.chunk_rows_opt == 0) return 0;
  return (uint32_t)(g.full_rows / g.chunk_rows);
}

struct AppendLayout {
  Geom g_sfx;
  uint64_t first_row;  // first row of X rebuilt
  uint64_t t_off, sfx_off, size_off, ews_off, total;
};

int append_layout(const Geom &g, const LaunchCfg &cfg, uint64_t n_new, AppendLayout *L) {
  const uint32_t keep = kept_chunks(g);
  L->first_row = (uint64_t)keep * g.chunk_rows;
  const uint64_t t_rows = g.rows - L->first_row + n_new;
  sprintz_opts o{};
  o.forecaster = (uint8_t)g.forecaster;
  o.huffman = 0;
  o.group_blocks = (uint8_t)g.G;
  o.learn_shift = (uint8_t)g.learn_shift;
  o.chunk_rows = g.chunk_rows_opt;
  o.huff_chunks = 0;
  int rc = make_geom(t_rows, g.D, g.w, &o, &L->g_sfx);
  if (rc != SPRINTZ_OK) return rc;
  const uint64_t rb = (uint64_t)g.D * g.wb;
  L->t_off = 0;
  L->sfx_off = align256a(t_rows * rb);
  L->size_off = L->sfx_off + align256a(sprintz_max_compressed_size(t_rows, g.D, g.w, &o));
  L->ews_off = L->size_off + 256;
  L->total = L->ews_off + encode_workspace_bytes(L->g_sfx, cfg);
  return SPRINTZ_OK;
}

}  // namespace

uint64_t append_workspace_bytes(const Geom &g_old, const LaunchCfg &cfg, uint64_t n_new) {
  AppendLayout L;
  if (g_old.huffman || append_layout(g_old, cfg, n_new, &L) != SPRINTZ_OK) return 0;
  return L.total;
}

int launch_append(const Geom &g, const LaunchCfg &cfg, const uint8_t *src, uint64_t src_size, uint64_t old_tail_off,
                  const uint8_t *rows, uint64_t n_new, uint8_t *dst, uint64_t dst_cap, uint64_t *d_out_size,
                  uint8_t *ws, uint64_t ws_bytes, int *d_status, cudaStream_t stream) {
  if (g.huffman) return SPRINTZ_ERR_UNSUPPORTED;
  AppendLayout L;
  int rc = append_layout(g, cfg, n_new, &L);
  if (rc != SPRINTZ_OK) return rc;
  if (ws_bytes < L.total) return SPRINTZ_ERR_WS_TOO_SMALL;
  const uint32_t keep = kept_chunks(g);
  const uint64_t rb = (uint64_t)g.D * g.wb;
  uint8_t *T = ws + L.t_off;
  // 1. X's rows from the first rebuilt chunk on, then Y
  if (keep < g.n_chunks) {
    if (!decode_chunks_supported(g, cfg)) return SPRINTZ_ERR_UNSUPPORTED;
    rc = launch_decode_chunks(g, cfg, src, src_size, keep, g.n_chunks, T, (g.full_rows - L.first_row) * rb, d_status,
                              stream);
    if (rc != SPRINTZ_OK) return rc;
  }
  const uint64_t tail_bytes = g.tail_rows * rb;
  if (tail_bytes) {
    if (old_tail_off + tail_bytes > src_size) return SPRINTZ_ERR_CORRUPT;
    if (cudaMemcpyAsync(T + (g.full_rows - L.first_row) * rb, src + old_tail_off, tail_bytes,
                        cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
      return SPRINTZ_ERR_CUDA;
  }
  if (n_new && cudaMemcpyAsync(T + (g.rows - L.first_row) * rb, rows, n_new * rb, cudaMemcpyDeviceToDevice,
                               stream) != cudaSuccess)
    return SPRINTZ_ERR_CUDA;
  // 2. the suffix stream
  uint64_t *sfx_size = reinterpret_cast<uint64_t *>(ws + L.size_off);
  const uint64_t sfx_cap = L.size_off - L.sfx_off;
  rc = launch_encode_fast(L.g_sfx, cfg, T, ws + L.sfx_off, sfx_cap, sfx_size, ws + L.ews_off, L.total - L.ews_off,
                          d_status, stream);
  if (rc != SPRINTZ_OK) return rc;
  // 3. the new stream
  AppendParams p{};
  p.src = src;
  p.src_size = src_size;
  p.suffix = ws + L.sfx_off;
  p.dst = dst;
  p.dst_cap = dst_cap;
  p.out_size = d_out_size;
  p.status = d_status;
  p.g_old = g;
  p.keep = keep;
  p.n_chunks = keep + L.g_sfx.n_chunks;
  p.rows = g.rows + n_new;
  p.data_off = kHdrBytes + (uint64_t)kEntryBytes * p.n_chunks;
  p.sfx_data_off = L.g_sfx.data_off;
  p.sfx_cap = sfx_cap;
  const uint64_t approx = p.data_off + (g.rows + n_new) * rb;
  const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((approx + 8191) / 8192,
                                                                          (uint64_t)cfg.sm_count * 8));
  k_append_assemble<<<grid, 256, 0, stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

// ---- packing buffers back to back ---------------------------------------------

// Exclusive scan of n sizes with one CTA (1024 threads, chunks of 1024),
// then the capacity check.
__global__ void __launch_bounds__(1024) k_pack_scan(const uint64_t *sizes, uint32_t n, uint64_t *offsets,
                                                    uint64_t cap, int *status, uint32_t *ok) {
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t s_carry;
  const uint32_t t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (t == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += 1024) {
    const uint32_t i = base + t;
    const uint64_t v = i < n ? sizes[i] : 0;
    uint64_t x = v;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint64_t w = s_warp[lane];
#pragma unroll
      for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
        if (lane >= o) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const uint64_t before = s_carry + (wid ? s_warp[wid - 1] : 0) + x - v;
    if (i < n) offsets[i] = before;
    __syncthreads();
    if (t == 1023) s_carry = before + v;
    __syncthreads();
  }
  if (t == 0) {
    offsets[n] = s_carry;
    const bool fits = s_carry <= cap;
    *ok = fits ? 1u : 0u;
    if (!fits) set_status(status, SPRINTZ_ERR_DST_TOO_SMALL);
  }
}

// Every CTA copies the buffers k = blockIdx.x, blockIdx.x + gridDim.x, ...
__global__ void __launch_bounds__(256) k_pack_copy(const uint64_t *srcs, const uint64_t *sizes, uint32_t n,
                                                   uint8_t *dst, const uint64_t *offsets, const uint32_t *ok) {
  if (!*ok) return;
  for (uint32_t k = blockIdx.x; k < n; k += gridDim.x) {
    const uint8_t *src = reinterpret_cast<const uint8_t *>(srcs[k]);
    uint8_t *d = dst + offsets[k];
    const uint64_t len = sizes[k];
    const uintptr_t mis = (uintptr_t)d ^ (uintptr_t)src;
    uint64_t head = (16 - ((uintptr_t)d & 15)) & 15;
    if (head > len) head = len;
    if ((mis & 15) == 0) {
      for (uint64_t q = threadIdx.x; q < head; q += blockDim.x) d[q] = src[q];
      const uint64_t nv = (len - head) / 16;
      const uint4 *s4 = reinterpret_cast<const uint4 *>(src + head);
      uint4 *d4 = reinterpret_cast<uint4 *>(d + head);
      for (uint64_t q = threadIdx.x; q < nv; q += blockDim.x) d4[q] = s4[q];
      for (uint64_t q = head + nv * 16 + threadIdx.x; q < len; q += blockDim.x) d[q] = src[q];
    } else {
      // 16-byte stores built from the source's aligned words
      for (uint64_t q = threadIdx.x; q < head; q += blockDim.x) d[q] = src[q];
      const uint8_t *s1 = src + head;
      const uint32_t sh = (uint32_t)((uintptr_t)s1 & 3) * 8;
      const uint32_t *sw = reinterpret_cast<const uint32_t *>((uintptr_t)s1 & ~(uintptr_t)3);
      const uint64_t nv = (len - head) / 16;
      uint4 *d4 = reinterpret_cast<uint4 *>(d + head);
      // the last unit of a misaligned source reads up to one word past its
      // 16 bytes, inside [src, src + len) only when a whole word remains
      const uint64_t safe = nv && (len - head) - 16 * nv < 4 ? nv - 1 : nv;
      for (uint64_t q = threadIdx.x; q < safe; q += blockDim.x) {
        const uint32_t *w = sw + 4 * q;
        uint4 v;
        v.x = __funnelshift_r(w[0], w[1], sh);
        v.y = __funnelshift_r(w[1], w[2], sh);
        v.z = __funnelshift_r(w[2], w[3], sh);
        v.w = __funnelshift_r(w[3], w[4], sh);
        d4[q] = v;
      }
      for (uint64_t q = head + safe * 16 + threadIdx.x; q < len; q += blockDim.x) d[q] = src[q];
    }
  }
}

int launch_pack(const LaunchCfg &cfg, const uint64_t *srcs, const uint64_t *sizes, uint32_t n, uint8_t *dst,
                uint64_t dst_cap, uint64_t *offsets, int *d_status, uint32_t *d_ok, cudaStream_t stream) {
  k_pack_scan<<<1, 1024, 0, stream>>>(sizes, n, offsets, dst_cap, d_status, d_ok);
  if (n) {
    const uint32_t grid = (uint32_t)std::min<uint64_t>(n, (uint64_t)cfg.sm_count * 8);
    k_pack_copy<<<grid, 256, 0, stream>>>(srcs, sizes, n, dst, offsets, d_ok);
  }
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

}  // namespace spz
