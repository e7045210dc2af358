// The forecasting step alone: samples -> forecast errors and back.
//
// This is the subroutine that the FIRE Speed experiment of Sec. 5.6 times on
// its own ("encode" turns raw samples into errors, "decode" rebuilds the
// samples; neither changes the data size).  The four forecasters are the
// codec's (Sec. 4.2.1 delta coding, Sec. 4.2.2 FIRE in its block form, the
// double-delta member of the same family, and Algorithm 3 literally, with an
// update at every sample).  The forecaster restarts every chunk_rows rows,
// exactly as in the codec, so that chunks run in parallel.
//
// A CTA owns `cpc` consecutive chunks.  Per step it stages R rows of each of
// its chunks in shared memory with 8-byte asynchronous copies (cp.async; the
// next step's rows load while this step computes, two tiles in turn), one
// thread per (chunk, column) pair runs that column's recurrence over the
// staged rows in place, and the tile goes back out with 8-byte stores.  Errors are stored as
// w-bit two's complement in the samples' own layout.  dst may equal src: a
// CTA reads and writes only its own chunks' rows.
#include <algorithm>

#include "spz_common.cuh"

namespace spz {

// A w-bit sample in the shared-memory tile (2-byte aligned for w = 16).
template <int W>
__device__ __forceinline__ uint32_t tile_ld(const uint8_t *p) {
  return W == 8 ? (uint32_t)*p : (uint32_t)*reinterpret_cast<const uint16_t *>(p);
}
template <int W>
__device__ __forceinline__ void tile_st(uint8_t *p, uint32_t v) {
  if (W == 8)
    *p = (uint8_t)v;
  else
    *reinterpret_cast<uint16_t *>(p) = (uint16_t)v;
}

constexpr int kFcThreads = 256;
constexpr int kFcMaxPairs = 4;  // (chunk, column) pairs per thread: cpc * D <= 1024

struct FcParams {
  const uint8_t *src;
  uint8_t *dst;
  uint64_t full_rows;  // rows in whole 8-row blocks
  uint64_t n_chunks;
  uint32_t D;
  uint32_t chunk_rows;  // > 0, multiple of 8
  uint32_t learn_shift;
  uint32_t cpc;  // chunks per CTA
  uint32_t R;    // rows per step, multiple of 8
};

template <int W, int FC, bool INV>
__global__ void __launch_bounds__(kFcThreads) k_forecast(FcParams p) {
  extern __shared__ __align__(16) uint8_t tile[];
  constexpr uint32_t wb = W / 8;
  const uint32_t D = p.D, rowb = D * wb, R = p.R;
  const uint64_t c0 = (uint64_t)blockIdx.x * p.cpc;
  const uint32_t nch = (uint32_t)min((uint64_t)p.cpc, p.n_chunks - c0);
  const uint32_t pairs = nch * D;
  uint32_t xp[kFcMaxPairs];
  int32_t dp[kFcMaxPairs], acc[kFcMaxPairs];
#pragma unroll
  for (int q = 0; q < kFcMaxPairs; ++q) {
    xp[q] = 0;
    dp[q] = 0;
    acc[q] = 0;
  }
  auto chunk_len = [&](uint32_t k) -> uint32_t {
    const uint64_t r = (c0 + k) * p.chunk_rows;
    return (uint32_t)min((uint64_t)p.chunk_rows, p.full_rows - r);
  };
  const uint32_t seg_bytes = R * rowb;  // one chunk's slot in a tile
  const uint32_t units_per = seg_bytes / 8;
  const uint64_t tile_bytes = (uint64_t)p.cpc * seg_bytes;
  // 8-byte units of step r0 still inside their chunk
  auto issue = [&](uint64_t r0, uint8_t *buf) {
    for (uint32_t idx = threadIdx.x; idx < nch * units_per; idx += kFcThreads) {
      const uint32_t k = idx / units_per, u = idx % units_per;
      const uint32_t len = chunk_len(k);
      if (r0 >= len || (uint64_t)u * 8 >= (uint64_t)(len - r0) * rowb) continue;
      const uint8_t *g = p.src + ((c0 + k) * p.chunk_rows + r0) * rowb + (uint64_t)u * 8;
      const uint32_t sa = (uint32_t)__cvta_generic_to_shared(buf + (uint64_t)k * seg_bytes + (uint64_t)u * 8);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(g) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  issue(0, tile);
  uint32_t cur = 0;
  for (uint64_t r0 = 0; r0 < p.chunk_rows; r0 += R, cur ^= 1) {
    uint8_t *tl = tile + cur * tile_bytes;
    // the next step's rows load into the other tile while this one computes
    if (r0 + R < p.chunk_rows) {
      issue(r0 + R, tile + (cur ^ 1) * tile_bytes);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    // block by block, the thread's pairs interleaved; a block's 8 samples are
    // read before any is written
    for (uint32_t b = 0; b < R; b += kBlockRows) {
#pragma unroll
      for (int q = 0; q < kFcMaxPairs; ++q) {
        const uint32_t pr = threadIdx.x + q * kFcThreads;
        if (pr >= pairs) continue;
        const uint32_t k = pr / D, j = pr % D;
        if (r0 + b >= chunk_len(k)) continue;
        uint8_t *cell0 = tl + (uint64_t)k * seg_bytes + (uint64_t)b * rowb + j * wb;
        uint32_t v[kBlockRows];
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) v[i] = tile_ld<W>(cell0 + i * rowb);
        const int32_t a = acc[q] >> p.learn_shift;  // block form: alpha fixed for the block
        int32_t gsum = 0;
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) {
          uint32_t x;
          int32_t e;
          if (!INV) {
            x = v[i];
            if (FC == kFcDelta) {
              e = sext<W>(x - xp[q]);
            } else if (FC == kFcDDelta) {
              e = sext<W>(x - xp[q] - (uint32_t)dp[q]);
            } else if (FC == kFcFire) {
              e = sext<W>(x - xp[q] - fire_pred_delta<W>(a, dp[q]));
            } else {
              e = sext<W>(x - xp[q] - fire_pred_delta<W>(acc[q] >> p.learn_shift, dp[q]));
            }
            v[i] = (uint32_t)e;
          } else {
            e = sext<W>(v[i]);
            if (FC == kFcDelta) {
              x = xp[q] + (uint32_t)e;
            } else if (FC == kFcDDelta) {
              x = xp[q] + (uint32_t)dp[q] + (uint32_t)e;
            } else if (FC == kFcFire) {
              x = xp[q] + fire_pred_delta<W>(a, dp[q]) + (uint32_t)e;
            } else {
              x = xp[q] + fire_pred_delta<W>(acc[q] >> p.learn_shift, dp[q]) + (uint32_t)e;
            }
            v[i] = x;
          }
          if (FC == kFcFire && (i & 1) == 0) gsum += sign_of(e) * dp[q];
          if (FC == kFcFireSample)
            acc[q] = wrap_acc<W>((int32_t)((uint32_t)acc[q] + (uint32_t)(sign_of(e) * dp[q])));
          dp[q] = sext<W>(x - xp[q]);
          xp[q] = x & ((1u << W) - 1u);
        }
        if (FC == kFcFire) acc[q] = wrap_acc<W>((int32_t)((uint32_t)acc[q] + (uint32_t)(gsum >> 2)));
#pragma unroll
        for (int i = 0; i < kBlockRows; ++i) tile_st<W>(cell0 + i * rowb, v[i]);
      }
    }
    __syncthreads();
    for (uint32_t k = 0; k < nch; ++k) {
      const uint32_t len = chunk_len(k);
      if (r0 >= len) continue;
      const uint32_t units = (min(R, (uint32_t)(len - r0)) * rowb) / 8;
      uint64_t *d = reinterpret_cast<uint64_t *>(p.dst + ((c0 + k) * p.chunk_rows + r0) * rowb);
      const uint64_t *t = reinterpret_cast<const uint64_t *>(tl + (uint64_t)k * seg_bytes);
      for (uint32_t u = threadIdx.x; u < units; u += kFcThreads) d[u] = t[u];
    }
    __syncthreads();
  }
}

template <int W, bool INV>
static const void *forecast_kernel(uint32_t fc) {
  switch (fc) {
    case kFcDelta: return (const void *)k_forecast<W, kFcDelta, INV>;
    case kFcFire: return (const void *)k_forecast<W, kFcFire, INV>;
    case kFcDDelta: return (const void *)k_forecast<W, kFcDDelta, INV>;
    default: return (const void *)k_forecast<W, kFcFireSample, INV>;
  }
}

int launch_forecast(const LaunchCfg &cfg, const uint8_t *src, uint64_t rows, uint32_t D, uint32_t w,
                    uint32_t forecaster, uint32_t learn_shift, uint32_t chunk_rows, bool inverse, uint8_t *dst,
                    cudaStream_t stream) {
  const uint32_t wb = w / 8, rowb = D * wb;
  const uint64_t full_rows = rows - rows % kBlockRows;
  const uint64_t tail_bytes = (rows - full_rows) * rowb;
  if (tail_bytes && src != dst &&
      cudaMemcpyAsync(dst + full_rows * rowb, src + full_rows * rowb, tail_bytes, cudaMemcpyDeviceToDevice,
                      stream) != cudaSuccess)
    return SPRINTZ_ERR_CUDA;
  if (!full_rows) return SPRINTZ_OK;
  FcParams p{};
  p.src = src;
  p.dst = dst;
  p.full_rows = full_rows;
  p.D = D;
  p.chunk_rows = chunk_rows ? chunk_rows : (uint32_t)std::min<uint64_t>(full_rows, 0xFFFFFFF8u);
  if ((uint64_t)p.chunk_rows < full_rows && !chunk_rows) return SPRINTZ_ERR_UNSUPPORTED;
  p.n_chunks = (full_rows + p.chunk_rows - 1) / p.chunk_rows;
  p.learn_shift = learn_shift;
  // rows per step: whole blocks, at least 512 bytes per chunk segment
  uint32_t R = kBlockRows;
  while (R * rowb < 512 && R < p.chunk_rows) R += kBlockRows;
  p.R = std::min(R, p.chunk_rows);
  const uint32_t seg = p.R * rowb;
  const uint32_t tile_cap = 24 * 1024;  // per tile; two tiles in turn
  uint64_t cpc = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)kFcThreads * kFcMaxPairs / D, tile_cap / seg));
  cpc = std::min<uint64_t>(cpc, p.n_chunks);
  // keep at least two CTAs per SM when there are enough chunks
  while (cpc > 1 && (p.n_chunks + cpc - 1) / cpc < 2ull * (uint64_t)cfg.sm_count) cpc = (cpc + 1) / 2;
  p.cpc = (uint32_t)cpc;
  const uint64_t smem = 2 * cpc * seg;
  if (smem > (uint64_t)cfg.max_smem_optin) return SPRINTZ_ERR_UNSUPPORTED;
  const void *fn = w == 8 ? (inverse ? forecast_kernel<8, true>(forecaster) : forecast_kernel<8, false>(forecaster))
                          : (inverse ? forecast_kernel<16, true>(forecaster) : forecast_kernel<16, false>(forecaster));
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return SPRINTZ_ERR_CUDA;
  const uint64_t grid = (p.n_chunks + cpc - 1) / cpc;
  if (grid > 0x7FFFFFFFull) return SPRINTZ_ERR_UNSUPPORTED;
  void *args[] = {&p};
  if (cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kFcThreads), args, smem, stream) != cudaSuccess)
    return SPRINTZ_ERR_CUDA;
  return SPRINTZ_OK;
}

}  // namespace spz
