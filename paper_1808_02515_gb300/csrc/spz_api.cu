// C ABI of the CUDA Sprintz codec: argument checks, stream geometry, sizes,
// header parsing and the device status word.  Every compute step runs in the
// kernels of spz_encode.cu and spz_decode.cu; there is no CPU fallback.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <string>

#include "spz_common.cuh"

struct sprintz_ctx {
  int device;
  int *d_status;
  uint32_t *d_pack_ok = nullptr;  // sprintz_pack: the scan's capacity verdict
  int *h_status;  // pinned
  spz::LaunchCfg cfg;
  std::string dev_name;
  // the current batch plan and the host images of its descriptors
  spz::BatchPlan plan{};
  bool has_plan = false;
  std::vector<uint8_t> items_img;
  std::vector<uint64_t> work_img;
  // schedules chosen by the autotuner, by batch kind
  std::map<std::string, sprintz_schedule> schedules;
};

namespace spz {

// Stream geometry from shape and options; the same rules the format states:
// full_rows = rows - rows % 8, chunks of chunk_rows rows (0 = one chunk),
// Huffman segments of huff_chunks chunks, and every chunk body must fit the
// table's 32-bit size field.
int make_geom(uint64_t rows, uint32_t D, uint32_t w, const sprintz_opts *o, Geom *g) {
  if (!o) return SPRINTZ_ERR_INVALID_ARG;
  if (w != 8 && w != 16) return SPRINTZ_ERR_UNSUPPORTED_W;
  if (D < 1 || D > kMaxD) return SPRINTZ_ERR_INVALID_ARG;
  if (o->forecaster > 3 || o->huffman > 1) return SPRINTZ_ERR_INVALID_ARG;
  if (o->group_blocks < 1 || o->group_blocks > 8) return SPRINTZ_ERR_INVALID_ARG;
  if (o->learn_shift > 2 * w - 1) return SPRINTZ_ERR_INVALID_ARG;
  if (o->chunk_rows % kBlockRows) return SPRINTZ_ERR_INVALID_ARG;
  if (o->huffman && o->huff_chunks < 1) return SPRINTZ_ERR_INVALID_ARG;
  memset(g, 0, sizeof(*g));
  g->rows = rows;
  g->tail_rows = rows % kBlockRows;
  g->full_rows = rows - g->tail_rows;
  uint64_t n_chunks =
      g->full_rows == 0 ? 0 : (o->chunk_rows == 0 ? 1 : (g->full_rows + o->chunk_rows - 1) / o->chunk_rows);
  if (n_chunks > 0xFFFFFFFFull) return SPRINTZ_ERR_INVALID_ARG;
  g->n_chunks = (uint32_t)n_chunks;
  g->chunk_rows = o->chunk_rows ? o->chunk_rows : (g->full_rows ? g->full_rows : kBlockRows);
  g->chunk_rows_opt = o->chunk_rows;
  g->D = D;
  g->w = w;
  g->wb = w / 8;
  g->G = o->group_blocks;
  g->hb = w == 8 ? 3 : 4;
  g->hdr_bytes = (g->G * D * g->hb + 7) / 8;
  g->col_major = D * w <= 32;
  g->forecaster = o->forecaster;
  g->learn_shift = o->learn_shift;
  g->huffman = o->huffman;
  g->huff_chunks = o->huffman ? o->huff_chunks : 0;
  g->n_segments = o->huffman ? (uint32_t)((n_chunks + o->huff_chunks - 1) / o->huff_chunks) : 0;
  g->data_off = kHdrBytes + (uint64_t)kEntryBytes * n_chunks + (uint64_t)kHuffTableBytes * g->n_segments;
  uint64_t max_rows = g->full_rows < g->chunk_rows ? g->full_rows : g->chunk_rows;
  g->max_blocks = (uint32_t)(max_rows / kBlockRows);
  g->max_body = max_body_bytes(g->max_blocks, D, w, g->G);
  if (g->max_body > 0xFFFFFFFFull) return SPRINTZ_ERR_INVALID_ARG;
  // Huffman sub-block offsets are u32: at most 11/8 of a body plus its table
  if (g->huffman && g->max_body > (1ull << 31)) return SPRINTZ_ERR_INVALID_ARG;
  return SPRINTZ_OK;
}

}  // namespace spz

using spz::Geom;

static uint64_t le(const uint8_t *p, int n) {
  uint64_t v = 0;
  for (int k = 0; k < n; ++k) v |= (uint64_t)p[k] << (8 * k);
  return v;
}

extern "C" {

int sprintz_ctx_create(sprintz_ctx **out, int device) {
  if (!out) return SPRINTZ_ERR_INVALID_ARG;
  *out = nullptr;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  sprintz_ctx *c = new sprintz_ctx();
  c->device = device;
  int rc = SPRINTZ_OK;
  if (cudaDeviceGetAttribute(&c->cfg.sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->cfg.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
          cudaSuccess ||
      cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->d_pack_ok, sizeof(uint32_t)) != cudaSuccess ||
      cudaMallocHost(&c->h_status, sizeof(int)) != cudaSuccess)
    rc = SPRINTZ_ERR_CUDA;
  cudaDeviceProp prop;
  if (rc == SPRINTZ_OK && cudaGetDeviceProperties(&prop, device) == cudaSuccess) c->dev_name = prop.name;
  cudaSetDevice(prev);
  if (rc != SPRINTZ_OK) {
    sprintz_ctx_destroy(c);
    return rc;
  }
  *out = c;
  return SPRINTZ_OK;
}

void sprintz_ctx_destroy(sprintz_ctx *c) {
  if (!c) return;
  if (c->d_status) cudaFree(c->d_status);
  if (c->d_pack_ok) cudaFree(c->d_pack_ok);
  if (c->h_status) cudaFreeHost(c->h_status);
  delete c;
}

uint64_t sprintz_max_compressed_size(uint64_t rows, uint32_t D, uint32_t w, const sprintz_opts *o) {
  Geom g;
  if (spz::make_geom(rows, D, w, o, &g) != SPRINTZ_OK) return 0;
  uint64_t total = g.data_off;
  if (g.n_chunks) {
    uint64_t full = g.full_rows / g.chunk_rows;  // chunks with chunk_rows rows
    uint64_t last_rows = g.full_rows - full * g.chunk_rows;
    total += full * spz::max_body_bytes(g.chunk_rows / 8, D, w, g.G);
    if (last_rows) total += spz::max_body_bytes(last_rows / 8, D, w, g.G);
  }
  return total + g.tail_rows * D * g.wb;
}

static spz::LaunchCfg default_cfg() {
  spz::LaunchCfg cfg{152, 232448};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaDeviceGetAttribute(&cfg.sm_count, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&cfg.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  return cfg;
}

uint64_t sprintz_compress_workspace_size(uint64_t rows, uint32_t D, uint32_t w, const sprintz_opts *o) {
  Geom g;
  if (spz::make_geom(rows, D, w, o, &g) != SPRINTZ_OK) return 0;
  if (g.huffman) return spz::huff_encode_workspace_bytes(g, default_cfg());
  return spz::encode_workspace_bytes(g, default_cfg());
}

uint64_t sprintz_decompress_workspace_size(const sprintz_info *info) {
  if (!info) return 0;
  Geom g;
  if (spz::make_geom(info->rows, info->D, info->w, &info->opts, &g) != SPRINTZ_OK) return 0;
  if (g.huffman) return spz::huff_decode_workspace_bytes(g, default_cfg());
  return spz::decode_workspace_bytes(g, default_cfg());
}

int sprintz_compress(sprintz_ctx *ctx, const void *src, uint64_t rows, uint32_t D, uint32_t w,
                     const sprintz_opts *opts, void *dst, uint64_t dst_cap, uint64_t *d_out_size,
                     void *workspace, uint64_t ws_bytes, void *stream) {
  if (!ctx || !dst || !d_out_size || (rows && !src)) return SPRINTZ_ERR_INVALID_ARG;
  Geom g;
  int rc = spz::make_geom(rows, D, w, opts, &g);
  if (rc != SPRINTZ_OK) return rc;
  if (dst_cap < sprintz_max_compressed_size(rows, D, w, opts)) return SPRINTZ_ERR_DST_TOO_SMALL;
  if (!workspace && ws_bytes) return SPRINTZ_ERR_INVALID_ARG;
  if (g.huffman) {
    if (ws_bytes < spz::huff_encode_workspace_bytes(g, ctx->cfg)) return SPRINTZ_ERR_WS_TOO_SMALL;
    return spz::launch_encode_huffman(g, ctx->cfg, (const uint8_t *)src, (uint8_t *)dst, dst_cap, d_out_size,
                                      (uint8_t *)workspace, ws_bytes, ctx->d_status, (cudaStream_t)stream);
  }
  if (ws_bytes < spz::encode_workspace_bytes(g, ctx->cfg)) return SPRINTZ_ERR_WS_TOO_SMALL;
  return spz::launch_encode_fast(g, ctx->cfg, (const uint8_t *)src, (uint8_t *)dst, dst_cap, d_out_size,
                                 (uint8_t *)workspace, ws_bytes, ctx->d_status, (cudaStream_t)stream);
}

// The geometry a host-parsed header describes (it must be self-consistent).
static int info_geom(const sprintz_info *info, Geom *g) {
  if (!info) return SPRINTZ_ERR_INVALID_ARG;
  if (spz::make_geom(info->rows, info->D, info->w, &info->opts, g) != SPRINTZ_OK) return SPRINTZ_ERR_INVALID_ARG;
  if (g->n_chunks != info->n_chunks || g->data_off != info->data_off) return SPRINTZ_ERR_INVALID_ARG;
  return SPRINTZ_OK;
}

uint64_t sprintz_decompress_rows_workspace_size(const sprintz_info *info, uint64_t row_begin, uint64_t row_end) {
  Geom g;
  if (info_geom(info, &g) != SPRINTZ_OK || row_end > info->rows) return 0;
  if (row_end <= row_begin) return 0;
  return spz::decode_rows_workspace_bytes(g, default_cfg(), row_begin, row_end);
}

int sprintz_decompress_rows(sprintz_ctx *ctx, const void *src, uint64_t src_size, const sprintz_info *info,
                            uint64_t row_begin, uint64_t row_end, void *dst, uint64_t dst_cap, void *workspace,
                            uint64_t ws_bytes, void *stream) {
  if (!ctx || !src) return SPRINTZ_ERR_INVALID_ARG;
  Geom g;
  int rc = info_geom(info, &g);
  if (rc != SPRINTZ_OK) return rc;
  if (row_end > info->rows) return SPRINTZ_ERR_INVALID_ARG;
  if (row_end <= row_begin) return SPRINTZ_OK;
  if (!dst) return SPRINTZ_ERR_INVALID_ARG;
  if (dst_cap < (row_end - row_begin) * g.D * g.wb) return SPRINTZ_ERR_DST_TOO_SMALL;
  if (src_size < g.data_off) return SPRINTZ_ERR_CORRUPT;
  if (!workspace && ws_bytes) return SPRINTZ_ERR_INVALID_ARG;
  return spz::launch_decode_rows(g, ctx->cfg, (const uint8_t *)src, src_size, row_begin, row_end, (uint8_t *)dst,
                                 (uint8_t *)workspace, ws_bytes, ctx->d_status, (cudaStream_t)stream);
}

uint64_t sprintz_append_workspace_size(const sprintz_info *info, uint64_t n_rows) {
  Geom g;
  if (info_geom(info, &g) != SPRINTZ_OK) return 0;
  return spz::append_workspace_bytes(g, default_cfg(), n_rows);
}

int sprintz_append(sprintz_ctx *ctx, const void *src, uint64_t src_size, const sprintz_info *info, const void *rows,
                   uint64_t n_rows, void *dst, uint64_t dst_cap, uint64_t *d_out_size, void *workspace,
                   uint64_t ws_bytes, void *stream) {
  if (!ctx || !src || !dst || !d_out_size || (n_rows && !rows) || !workspace) return SPRINTZ_ERR_INVALID_ARG;
  Geom g;
  int rc = info_geom(info, &g);
  if (rc != SPRINTZ_OK) return rc;
  if (g.huffman) return SPRINTZ_ERR_UNSUPPORTED;
  if (src_size < g.data_off || info->tail_off < g.data_off || info->tail_off > src_size) return SPRINTZ_ERR_CORRUPT;
  const uint64_t cap = sprintz_max_compressed_size(info->rows + n_rows, info->D, info->w, &info->opts);
  if (cap == 0) return SPRINTZ_ERR_INVALID_ARG;
  if (dst_cap < cap) return SPRINTZ_ERR_DST_TOO_SMALL;
  return spz::launch_append(g, ctx->cfg, (const uint8_t *)src, src_size, info->tail_off, (const uint8_t *)rows,
                            n_rows, (uint8_t *)dst, dst_cap, d_out_size, (uint8_t *)workspace, ws_bytes,
                            ctx->d_status, (cudaStream_t)stream);
}

int sprintz_pack(sprintz_ctx *ctx, const uint64_t *d_src_ptrs, const uint64_t *d_sizes, uint32_t n, void *dst,
                 uint64_t dst_cap, uint64_t *d_offsets, void *stream) {
  if (!ctx || !d_offsets || (n && (!d_src_ptrs || !d_sizes || !dst))) return SPRINTZ_ERR_INVALID_ARG;
  return spz::launch_pack(ctx->cfg, d_src_ptrs, d_sizes, n, (uint8_t *)dst, dst_cap, d_offsets, ctx->d_status,
                          ctx->d_pack_ok, (cudaStream_t)stream);
}

int sprintz_ctx_set_failure_test(sprintz_ctx *ctx, uint32_t wait_limit, uint32_t skip_first_group) {
  if (!ctx || skip_first_group > 1) return SPRINTZ_ERR_INVALID_ARG;
  ctx->cfg.wait_limit = wait_limit;
  ctx->cfg.skip_first_group = skip_first_group;
  return SPRINTZ_OK;
}

int sprintz_forecast(sprintz_ctx *ctx, const void *src, uint64_t rows, uint32_t D, uint32_t w,
                     uint32_t forecaster, uint32_t learn_shift, uint32_t chunk_rows, int inverse, void *dst,
                     void *stream) {
  if (!ctx || (rows && (!src || !dst))) return SPRINTZ_ERR_INVALID_ARG;
  if (w != 8 && w != 16) return SPRINTZ_ERR_UNSUPPORTED_W;
  if (D < 1 || D > 1024 || forecaster > 3 || learn_shift > 2 * w - 1 || chunk_rows % 8 ||
      (inverse != 0 && inverse != 1))
    return SPRINTZ_ERR_INVALID_ARG;
  if (((uintptr_t)src | (uintptr_t)dst) & 7) return SPRINTZ_ERR_UNSUPPORTED;
  if (!rows) return SPRINTZ_OK;
  return spz::launch_forecast(ctx->cfg, (const uint8_t *)src, rows, D, w, forecaster, learn_shift, chunk_rows,
                              inverse != 0, (uint8_t *)dst, (cudaStream_t)stream);
}

uint64_t sprintz_quant_workspace_size(uint32_t D) { return D >= 1 && D <= 1024 ? 32ull * D : 0; }

static int quant_args(sprintz_ctx *ctx, uint64_t rows, uint32_t D, uint32_t w) {
  if (!ctx) return SPRINTZ_ERR_INVALID_ARG;
  if (w != 8 && w != 16) return SPRINTZ_ERR_UNSUPPORTED_W;
  if (D < 1 || D > 1024 || rows > (1ull << 40)) return SPRINTZ_ERR_INVALID_ARG;
  return SPRINTZ_OK;
}

int sprintz_quantize(sprintz_ctx *ctx, const float *src, uint64_t rows, uint32_t D, uint32_t w, void *codes,
                     double *lo_hi, void *workspace, uint64_t ws_bytes, void *stream) {
  int rc = quant_args(ctx, rows, D, w);
  if (rc != SPRINTZ_OK) return rc;
  if (!rows) return SPRINTZ_OK;
  if (!src || !codes || !lo_hi || !workspace) return SPRINTZ_ERR_INVALID_ARG;
  if (ws_bytes < sprintz_quant_workspace_size(D)) return SPRINTZ_ERR_WS_TOO_SMALL;
  return spz::launch_quantize(ctx->cfg, src, rows, D, w, (uint8_t *)codes, lo_hi, (uint8_t *)workspace,
                              (cudaStream_t)stream);
}

int sprintz_dequantize(sprintz_ctx *ctx, const void *codes, uint64_t rows, uint32_t D, uint32_t w,
                       const double *lo_hi, float *dst, void *stream) {
  int rc = quant_args(ctx, rows, D, w);
  if (rc != SPRINTZ_OK) return rc;
  if (!rows) return SPRINTZ_OK;
  if (!codes || !lo_hi || !dst) return SPRINTZ_ERR_INVALID_ARG;
  return spz::launch_dequantize(ctx->cfg, (const uint8_t *)codes, rows, D, w, lo_hi, dst, (cudaStream_t)stream);
}

int sprintz_quant_nmse(sprintz_ctx *ctx, const float *src, const void *codes, uint64_t rows, uint32_t D,
                       uint32_t w, const double *lo_hi, double *nmse, void *workspace, uint64_t ws_bytes,
                       void *stream) {
  int rc = quant_args(ctx, rows, D, w);
  if (rc != SPRINTZ_OK) return rc;
  if (!rows || !src || !codes || !lo_hi || !nmse || !workspace) return SPRINTZ_ERR_INVALID_ARG;
  if (ws_bytes < sprintz_quant_workspace_size(D)) return SPRINTZ_ERR_WS_TOO_SMALL;
  return spz::launch_quant_nmse(ctx->cfg, src, (const uint8_t *)codes, rows, D, w, lo_hi, nmse,
                                (uint8_t *)workspace, (cudaStream_t)stream);
}

int sprintz_query(const void *host_header, uint64_t n, sprintz_info *out) {
  if (!host_header || !out) return SPRINTZ_ERR_INVALID_ARG;
  const uint8_t *h = (const uint8_t *)host_header;
  if (n < spz::kHdrBytes) return SPRINTZ_ERR_CORRUPT;
  if (h[0] != 'S' || h[1] != 'P' || h[2] != 'Z' || h[3] != '1' || h[4] != 1) return SPRINTZ_ERR_CORRUPT;
  if (h[7] & ~1u) return SPRINTZ_ERR_CORRUPT;
  memset(out, 0, sizeof(*out));
  out->w = h[5];
  out->opts.forecaster = h[6];
  out->opts.huffman = h[7] & 1;
  out->D = (uint32_t)le(h + 8, 2);
  out->opts.group_blocks = h[10];
  out->opts.learn_shift = h[11];
  out->opts.chunk_rows = (uint32_t)le(h + 12, 4);
  out->opts.huff_chunks = (uint32_t)le(h + 16, 4);
  out->n_chunks = (uint32_t)le(h + 20, 4);
  out->rows = le(h + 24, 8);
  out->tail_rows = (uint32_t)le(h + 32, 4);
  out->data_off = le(h + 40, 8);
  out->tail_off = le(h + 48, 8);
  out->total_bytes = le(h + 56, 8);
  Geom g;
  if (spz::make_geom(out->rows, out->D, out->w, &out->opts, &g) != SPRINTZ_OK) return SPRINTZ_ERR_CORRUPT;
  if (g.n_chunks != out->n_chunks || g.tail_rows != out->tail_rows || g.data_off != out->data_off ||
      le(h + 36, 4) != 0 || out->tail_off < out->data_off)
    return SPRINTZ_ERR_CORRUPT;
  return SPRINTZ_OK;
}

int sprintz_decompress(sprintz_ctx *ctx, const void *src, uint64_t src_size, const sprintz_info *info,
                       void *dst, uint64_t dst_cap, void *workspace, uint64_t ws_bytes, void *stream) {
  if (!ctx || !src || !info) return SPRINTZ_ERR_INVALID_ARG;
  Geom g;
  if (spz::make_geom(info->rows, info->D, info->w, &info->opts, &g) != SPRINTZ_OK)
    return SPRINTZ_ERR_INVALID_ARG;
  if (g.n_chunks != info->n_chunks || g.data_off != info->data_off) return SPRINTZ_ERR_INVALID_ARG;
  if (src_size < g.data_off) return SPRINTZ_ERR_CORRUPT;
  uint64_t need = info->rows * info->D * g.wb;
  if (need && !dst) return SPRINTZ_ERR_INVALID_ARG;
  if (dst_cap < need) return SPRINTZ_ERR_DST_TOO_SMALL;
  if (g.huffman) {
    if (ws_bytes < spz::huff_decode_workspace_bytes(g, ctx->cfg)) return SPRINTZ_ERR_WS_TOO_SMALL;
    return spz::launch_decode_huffman(g, ctx->cfg, (const uint8_t *)src, src_size, (uint8_t *)dst, dst_cap,
                                      (uint8_t *)workspace, ws_bytes, ctx->d_status, (cudaStream_t)stream);
  }
  if (ws_bytes < spz::decode_workspace_bytes(g, ctx->cfg)) return SPRINTZ_ERR_WS_TOO_SMALL;
  return spz::launch_decode(g, ctx->cfg, (const uint8_t *)src, src_size, (uint8_t *)dst, dst_cap,
                            (uint8_t *)workspace, ws_bytes, ctx->d_status, (cudaStream_t)stream);
}

}  // extern "C"

namespace {

int plan_any(sprintz_ctx *ctx, const sprintz_batch_item *items, uint32_t n, int compress,
             const sprintz_schedule &sched, uint8_t *ws, spz::BatchPlan *pl) {
  if (!ctx || (!items && n)) return SPRINTZ_ERR_INVALID_ARG;
  if (n == 0) return SPRINTZ_ERR_INVALID_ARG;
  return compress ? spz::plan_batch_encode(items, n, ctx->cfg, sched, ctx->d_status, ws, pl, &ctx->items_img,
                                           &ctx->work_img)
                  : spz::plan_batch_decode(items, n, ctx->cfg, sched, ctx->d_status, ws, pl, &ctx->items_img,
                                           &ctx->work_img);
}

// Plan and upload the descriptors and the work list (stream-ordered; the
// host images must outlive the copies, so the call waits for them).
int plan_upload(sprintz_ctx *ctx, const sprintz_batch_item *items, uint32_t n, int compress,
                const sprintz_schedule &sched, void *workspace, uint64_t ws_bytes, cudaStream_t s) {
  if (!workspace) return SPRINTZ_ERR_INVALID_ARG;
  spz::BatchPlan pl;
  if (ctx) ctx->has_plan = false;
  int rc = plan_any(ctx, items, n, compress, sched, (uint8_t *)workspace, &pl);
  if (rc != SPRINTZ_OK) return rc;
  if (ws_bytes < pl.ws_total) return SPRINTZ_ERR_WS_TOO_SMALL;
  pl.ws = workspace;
  uint8_t *ws = (uint8_t *)workspace;
  if (cudaMemcpyAsync(ws + pl.items_off, ctx->items_img.data(), ctx->items_img.size(), cudaMemcpyHostToDevice,
                      s) != cudaSuccess ||
      (ctx->work_img.size() &&
       cudaMemcpyAsync(ws + pl.work_off, ctx->work_img.data(), ctx->work_img.size() * 8, cudaMemcpyHostToDevice,
                       s) != cudaSuccess))
    return SPRINTZ_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  ctx->plan = pl;
  ctx->has_plan = true;
  return SPRINTZ_OK;
}

// The kind of a batch, for the autotuner's memory: device, direction,
// forecasters used, range requests, size (half powers of two) and the share
// of uncompressed bytes in each (w, D bucket) class (tenths).
std::string batch_kind(const sprintz_ctx *ctx, const sprintz_batch_item *items, uint32_t n, int compress) {
  static const uint32_t bucket_hi[] = {1, 2, 3, 4, 8, 16, 32};
  double cls[2][7] = {};
  double total = 0;
  uint32_t fc_mask = 0;
  bool ranged = false;
  for (uint32_t i = 0; i < n; ++i) {
    const sprintz_batch_item &it = items[i];
    const uint64_t rows = (!compress && it.row_end > it.row_begin) ? it.row_end - it.row_begin : it.rows;
    const double u = (double)rows * it.D * (it.w / 8);
    int b = 0;
    while (b < 6 && it.D > bucket_hi[b]) ++b;
    cls[it.w == 16][b] += u;
    total += u;
    fc_mask |= 1u << (it.opts.forecaster & 7);
    ranged |= !compress && it.row_end > it.row_begin;
  }
  char buf[256];
  int len = snprintf(buf, sizeof buf, "%s|%d|%s|fc%x|%s|lg%.1f|", ctx->dev_name.c_str(), ctx->cfg.sm_count,
                     compress ? "enc" : "dec", fc_mask, ranged ? "rng" : "all",
                     total > 0 ? floor(2.0 * log2(total)) / 2.0 : 0.0);
  std::string key(buf, len > 0 ? (size_t)len : 0);
  for (int w = 0; w < 2; ++w)
    for (int b = 0; b < 7; ++b) {
      const int tenth = total > 0 ? (int)lround(10.0 * cls[w][b] / total) : 0;
      key += (char)('0' + tenth % 10 + (tenth == 10 ? 17 : 0));  // 0..9, 'A' for all of it
    }
  return key;
}

const char *schedule_cache_path() { return getenv("SPRINTZ_SCHEDULE_CACHE"); }

void load_schedule_cache(sprintz_ctx *ctx) {
  const char *path = schedule_cache_path();
  if (!path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof line, f)) {
    char key[400];
    sprintz_schedule s{};
    if (sscanf(line, "%399[^\t]\t%u\t%u\t%u\t%u", key, &s.ctas_per_sm, &s.ring_segments, &s.prefetch_bytes,
               &s.order) == 5)
      ctx->schedules[key] = s;
  }
  fclose(f);
}

void save_schedule(const std::string &key, const sprintz_schedule &s, float ms) {
  const char *path = schedule_cache_path();
  if (!path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s\t%u\t%u\t%u\t%u\t%.4f\n", key.c_str(), s.ctas_per_sm, s.ring_segments, s.prefetch_bytes,
          s.order, ms);
  fclose(f);
}

int run_plan(sprintz_ctx *ctx, cudaStream_t s) {
  return ctx->plan.compress ? spz::run_batch_encode(ctx->plan, s) : spz::run_batch_decode(ctx->plan, s);
}

}  // namespace

extern "C" {

uint64_t sprintz_batch_workspace_size(sprintz_ctx *ctx, const sprintz_batch_item *items, uint32_t n,
                                      int compress) {
  spz::BatchPlan pl;
  sprintz_schedule none{};
  if (plan_any(ctx, items, n, compress, none, nullptr, &pl) != SPRINTZ_OK) return 0;
  return pl.ws_total;
}

int sprintz_batch_plan_schedule(sprintz_ctx *ctx, const sprintz_batch_item *items, uint32_t n, int compress,
                                const sprintz_schedule *schedule, void *workspace, uint64_t ws_bytes,
                                void *stream) {
  sprintz_schedule s{};
  if (schedule) s = *schedule;
  return plan_upload(ctx, items, n, compress, s, workspace, ws_bytes, (cudaStream_t)stream);
}

int sprintz_batch_plan(sprintz_ctx *ctx, const sprintz_batch_item *items, uint32_t n, int compress,
                       void *workspace, uint64_t ws_bytes, void *stream) {
  if (!ctx || (!items && n) || n == 0) return SPRINTZ_ERR_INVALID_ARG;
  if (ctx->schedules.empty()) load_schedule_cache(ctx);
  sprintz_schedule s{};
  auto hit = ctx->schedules.find(batch_kind(ctx, items, n, compress));
  if (hit != ctx->schedules.end()) s = hit->second;
  return plan_upload(ctx, items, n, compress, s, workspace, ws_bytes, (cudaStream_t)stream);
}

int sprintz_batch_run(sprintz_ctx *ctx, void *workspace, uint64_t ws_bytes, void *stream) {
  if (!ctx || !ctx->has_plan || ctx->plan.ws != workspace || ws_bytes < ctx->plan.ws_total)
    return SPRINTZ_ERR_INVALID_ARG;
  return run_plan(ctx, (cudaStream_t)stream);
}

int sprintz_batch_schedule(sprintz_ctx *ctx, sprintz_schedule *out) {
  if (!ctx || !out || !ctx->has_plan) return SPRINTZ_ERR_INVALID_ARG;
  *out = ctx->plan.sched;
  return SPRINTZ_OK;
}

int sprintz_batch_autotune(sprintz_ctx *ctx, const sprintz_batch_item *items, uint32_t n, int compress,
                           void *workspace, uint64_t ws_bytes, void *stream, sprintz_schedule *chosen,
                           float *ms_out) {
  if (!ctx || !items || n == 0 || !workspace) return SPRINTZ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SPRINTZ_ERR_CUDA;
  }
  int rc = SPRINTZ_OK;
  // time of one run under schedule c (one untimed run, then the mean of two);
  // a schedule that resolves to one already timed is not run again (*t < 0)
  std::vector<sprintz_schedule> seen;
  auto evaluate = [&](const sprintz_schedule &c, float *t, sprintz_schedule *resolved) -> int {
    int r = plan_upload(ctx, items, n, compress, c, workspace, ws_bytes, s);
    if (r != SPRINTZ_OK) return r;
    *resolved = ctx->plan.sched;
    *t = -1.0f;
    for (const sprintz_schedule &q : seen)
      if (memcmp(&q, resolved, sizeof q) == 0) return SPRINTZ_OK;
    seen.push_back(*resolved);
    if ((r = run_plan(ctx, s)) != SPRINTZ_OK) return r;
    if (cudaEventRecord(e0, s) != cudaSuccess) return SPRINTZ_ERR_CUDA;
    for (int k = 0; k < 2; ++k)
      if ((r = run_plan(ctx, s)) != SPRINTZ_OK) return r;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(t, e0, e1) != cudaSuccess)
      return SPRINTZ_ERR_CUDA;
    *t *= 0.5f;
    return SPRINTZ_OK;
  };
  sprintz_schedule best{}, res{};
  float best_ms = 0;
  rc = evaluate(best, &best_ms, &res);
  if (rc == SPRINTZ_OK) {
    best = res;
    // one knob at a time, from the defaults
    std::vector<std::vector<sprintz_schedule>> knobs;
    std::vector<sprintz_schedule> k_ctas, k_pf, k_order, k_seg;
    for (uint32_t v : {2u, 3u, 4u, 5u, 6u, 8u}) {
      sprintz_schedule c{};
      c.ctas_per_sm = v;
      k_ctas.push_back(c);
    }
    for (uint32_t v : {1u, 1024u, 2048u, 4096u, 8192u}) {
      sprintz_schedule c{};
      c.prefetch_bytes = v;
      k_pf.push_back(c);
    }
    for (uint32_t v : {1u, 2u, 3u}) {
      sprintz_schedule c{};
      c.order = v;
      k_order.push_back(c);
    }
    for (uint32_t v : {2u, 4u}) {
      sprintz_schedule c{};
      c.ring_segments = v;
      k_seg.push_back(c);
    }
    knobs = {k_ctas, k_pf, k_order};
    if (!compress) knobs.push_back(k_seg);
    for (size_t kn = 0; kn < knobs.size() && rc == SPRINTZ_OK; ++kn) {
      const sprintz_schedule base = best;
      for (const sprintz_schedule &delta : knobs[kn]) {
        sprintz_schedule c = base;
        if (kn == 0) c.ctas_per_sm = delta.ctas_per_sm;
        if (kn == 1) c.prefetch_bytes = delta.prefetch_bytes;
        if (kn == 2) c.order = delta.order;
        if (kn == 3) c.ring_segments = delta.ring_segments;
        float t = 0;
        rc = evaluate(c, &t, &res);
        if (rc != SPRINTZ_OK) break;
        if (t >= 0 && t < best_ms) {
          best = res;
          best_ms = t;
        }
      }
    }
  }
  if (rc == SPRINTZ_OK) {
    rc = plan_upload(ctx, items, n, compress, best, workspace, ws_bytes, s);
    if (rc == SPRINTZ_OK) {
      const std::string key = batch_kind(ctx, items, n, compress);
      ctx->schedules[key] = best;
      save_schedule(key, best, best_ms);
      if (chosen) *chosen = best;
      if (ms_out) *ms_out = best_ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int sprintz_get_status(sprintz_ctx *ctx, void *stream) {
  if (!ctx) return SPRINTZ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SPRINTZ_ERR_CUDA;
  if (cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  return *ctx->h_status;
}

const char *sprintz_strerror(int code) {
  switch (code) {
    case SPRINTZ_OK: return "ok";
    case SPRINTZ_ERR_INVALID_ARG: return "invalid argument";
    case SPRINTZ_ERR_UNSUPPORTED_W: return "bit width must be 8 or 16";
    case SPRINTZ_ERR_DST_TOO_SMALL: return "destination buffer too small";
    case SPRINTZ_ERR_WS_TOO_SMALL: return "workspace too small";
    case SPRINTZ_ERR_CORRUPT: return "corrupt stream";
    case SPRINTZ_ERR_TIMEOUT: return "a bounded device wait timed out";
    case SPRINTZ_ERR_CUDA: return "CUDA runtime error";
    case SPRINTZ_ERR_UNSUPPORTED: return "option not supported by this build";
    default: return "unknown error";
  }
}

}  // extern "C"
