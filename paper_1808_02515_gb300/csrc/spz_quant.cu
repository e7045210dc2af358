// Quantizing float data to w-bit integers before compression (Sec. 5.8).
//
// Each column of a row-major float32 series is offset and rescaled so that
// its minimum and maximum map to 0 and 2^w - 1, then floored; the inverse
// maps a code back with the step (max - min) / (2^w - 1).  All arithmetic is
// double precision with every operation rounded on its own (the _rn
// intrinsics: no fused multiply-add), so the integer codes and the rebuilt
// floats are exactly those of a plain sequential implementation.
//
//   k_quant_minmax   per-column extremes: a grid-stride pass keeps each
//                    thread's running min/max, a CTA reduction per column,
//                    then one atomic per column on an order-preserving
//                    integer image of the float (exact, order independent)
//   k_quant_codes    code = min(floor((x - min) * s), 2^w - 1), s per column
//   k_dequant        x = (float)(code * h + min)
//   k_quant_err      per column sum of x, then squared deviations and
//                    squared reconstruction errors (double atomics; only
//                    these sums depend on the order of the additions)
#include <algorithm>

#include "spz_common.cuh"

namespace spz {

constexpr int kQThreads = 256;

// Order-preserving map of a float onto uint32 (and back).  float -> double
// is exact and monotone, so the extremes are found on the floats.
__device__ __forceinline__ uint32_t flt_key(float v) {
  const uint32_t b = __float_as_uint(v);
  return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_flt(uint32_t k) {
  const uint32_t b = (k >> 31) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(b);
}

// Threads of a CTA cover (column, row-lane) pairs: column j = t % D for
// t < D * lanes, row lane = t / D; rows advance by lanes * gridDim.x.
struct QMap {
  uint32_t D, lanes;
};
__device__ __forceinline__ QMap qmap(uint32_t D) {
  QMap m;
  m.D = D;
  m.lanes = D >= kQThreads ? 1u : kQThreads / D;
  return m;
}

__global__ void __launch_bounds__(kQThreads) k_quant_minmax(const float *x, uint64_t rows, uint32_t D,
                                                           uint32_t *keys /* 2 D */) {
  __shared__ uint32_t s_lo[kQThreads], s_hi[kQThreads];
  const QMap m = qmap(D);
  for (uint32_t j0 = 0; j0 < D; j0 += kQThreads / m.lanes) {
    const uint32_t t = threadIdx.x, lane = t / min(D, (uint32_t)kQThreads), jj = t % min(D, (uint32_t)kQThreads);
    const uint32_t j = j0 + jj;
    const bool act = lane < m.lanes && j < D;
    uint32_t lo = ~0u, hi = 0u;
    if (act)
      for (uint64_t r = (uint64_t)blockIdx.x * m.lanes + lane; r < rows; r += (uint64_t)gridDim.x * m.lanes) {
        const uint32_t k = flt_key(x[r * D + j]);
        lo = min(lo, k);
        hi = max(hi, k);
      }
    s_lo[t] = lo;
    s_hi[t] = hi;
    __syncthreads();
    if (act && lane == 0) {
      for (uint32_t l = 1; l < m.lanes; ++l) {
        lo = min(lo, s_lo[l * min(D, (uint32_t)kQThreads) + jj]);
        hi = max(hi, s_hi[l * min(D, (uint32_t)kQThreads) + jj]);
      }
      atomicMin(&keys[2 * j], lo);
      atomicMax(&keys[2 * j + 1], hi);
    }
    __syncthreads();
  }
}

__global__ void k_quant_finish_minmax(const uint32_t *keys, uint32_t D, double *lo_hi) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < D; j += gridDim.x * blockDim.x) {
    lo_hi[2 * j] = (double)key_flt(keys[2 * j]);
    lo_hi[2 * j + 1] = (double)key_flt(keys[2 * j + 1]);
  }
}

// Per-column constants in shared memory: the scale s = (2^w - 1) / (max -
// min) (0 for a constant column) or the step h = (max - min) / (2^w - 1).
template <int W>
__device__ __forceinline__ void column_consts(const double *lo_hi, uint32_t D, double *out, bool step) {
  constexpr double kTop = (double)((1u << W) - 1u);
  for (uint32_t j = threadIdx.x; j < D; j += blockDim.x) {
    const double range = __dsub_rn(lo_hi[2 * j + 1], lo_hi[2 * j]);
    out[j] = step ? __ddiv_rn(range, kTop) : (range > 0.0 ? __ddiv_rn(kTop, range) : 0.0);
  }
  __syncthreads();
}

template <int W>
__global__ void __launch_bounds__(kQThreads) k_quant_codes(const float *x, uint64_t n, uint32_t D,
                                                          const double *lo_hi, uint8_t *codes) {
  extern __shared__ double s_scale[];
  constexpr double kTop = (double)((1u << W) - 1u);
  column_consts<W>(lo_hi, D, s_scale, false);
  const uint64_t step = (uint64_t)gridDim.x * kQThreads;
  const uint32_t jstep = (uint32_t)(step % D);
  uint64_t i = (uint64_t)blockIdx.x * kQThreads + threadIdx.x;
  for (uint32_t j = (uint32_t)(i % D); i < n; i += step, j = j + jstep >= D ? j + jstep - D : j + jstep) {
    double q = floor(__dmul_rn(__dsub_rn((double)x[i], lo_hi[2 * j]), s_scale[j]));
    q = q > kTop ? kTop : (q < 0.0 ? 0.0 : q);
    if (W == 8)
      codes[i] = (uint8_t)q;
    else
      reinterpret_cast<uint16_t *>(codes)[i] = (uint16_t)q;
  }
}

template <int W>
__global__ void __launch_bounds__(kQThreads) k_dequant(const uint8_t *codes, uint64_t n, uint32_t D,
                                                      const double *lo_hi, float *y) {
  extern __shared__ double s_step[];
  column_consts<W>(lo_hi, D, s_step, true);
  const uint64_t step = (uint64_t)gridDim.x * kQThreads;
  const uint32_t jstep = (uint32_t)(step % D);
  uint64_t i = (uint64_t)blockIdx.x * kQThreads + threadIdx.x;
  for (uint32_t j = (uint32_t)(i % D); i < n; i += step, j = j + jstep >= D ? j + jstep - D : j + jstep) {
    const double lo = lo_hi[2 * j], h = s_step[j];
    const double q = W == 8 ? (double)codes[i] : (double)reinterpret_cast<const uint16_t *>(codes)[i];
    y[i] = __double2float_rn(__dadd_rn(__dmul_rn(q, h), lo));
  }
}

// pass 0: sum of x per column; pass 1: squared deviations from the mean and
// squared reconstruction errors per column.
template <int W>
__global__ void __launch_bounds__(kQThreads) k_quant_err(const float *x, const uint8_t *codes, uint64_t rows,
                                                        uint32_t D, const double *lo_hi, double *acc /* 3 D */,
                                                        int pass) {
  __shared__ double s_a[kQThreads], s_b[kQThreads];
  constexpr double kTop = (double)((1u << W) - 1u);
  const QMap m = qmap(D);
  const uint32_t cw = min(D, (uint32_t)kQThreads);
  for (uint32_t j0 = 0; j0 < D; j0 += kQThreads / m.lanes) {
    const uint32_t t = threadIdx.x, lane = t / cw, jj = t % cw, j = j0 + jj;
    const bool act = lane < m.lanes && j < D;
    double a = 0.0, b = 0.0;
    if (act) {
      const double lo = lo_hi[2 * j], h = __ddiv_rn(__dsub_rn(lo_hi[2 * j + 1], lo), kTop);
      const double mean = pass ? __ddiv_rn(acc[3 * j], (double)rows) : 0.0;
      for (uint64_t r = (uint64_t)blockIdx.x * m.lanes + lane; r < rows; r += (uint64_t)gridDim.x * m.lanes) {
        const uint64_t i = r * D + j;
        const double v = (double)x[i];
        if (!pass) {
          a = __dadd_rn(a, v);
        } else {
          const double q = W == 8 ? (double)codes[i] : (double)reinterpret_cast<const uint16_t *>(codes)[i];
          const double xh = (double)__double2float_rn(__dadd_rn(__dmul_rn(q, h), lo));
          const double dv = __dsub_rn(v, mean), de = __dsub_rn(v, xh);
          a = __dadd_rn(a, __dmul_rn(dv, dv));
          b = __dadd_rn(b, __dmul_rn(de, de));
        }
      }
    }
    s_a[t] = a;
    s_b[t] = b;
    __syncthreads();
    if (act && lane == 0) {
      for (uint32_t l = 1; l < m.lanes; ++l) {
        a = __dadd_rn(a, s_a[l * cw + jj]);
        b = __dadd_rn(b, s_b[l * cw + jj]);
      }
      if (!pass) {
        atomicAdd(&acc[3 * j], a);
      } else {
        atomicAdd(&acc[3 * j + 1], a);
        atomicAdd(&acc[3 * j + 2], b);
      }
    }
    __syncthreads();
  }
}

__global__ void k_quant_nmse(const double *acc, uint32_t D, double *nmse) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < D; j += gridDim.x * blockDim.x) {
    const double var = acc[3 * j + 1], mse = acc[3 * j + 2];
    nmse[j] = var > 0.0 ? __ddiv_rn(mse, var) : 0.0;
  }
}

static uint32_t q_grid(const LaunchCfg &cfg, uint64_t work) {
  const uint64_t want = (work + kQThreads - 1) / kQThreads;
  return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)cfg.sm_count * 8));
}

int launch_quantize(const LaunchCfg &cfg, const float *x, uint64_t rows, uint32_t D, uint32_t w, uint8_t *codes,
                    double *lo_hi, uint8_t *ws, cudaStream_t stream) {
  uint32_t *keys = reinterpret_cast<uint32_t *>(ws);
  // keys start at (lo = all ones, hi = zero): an empty min and max
  if (cudaMemsetAsync(keys, 0, 8ull * D, stream) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  if (cudaMemset2DAsync(keys, 8, 0xFF, 4, D, stream) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  k_quant_minmax<<<q_grid(cfg, rows), kQThreads, 0, stream>>>(x, rows, D, keys);
  k_quant_finish_minmax<<<(D + 255) / 256, 256, 0, stream>>>(keys, D, lo_hi);
  const uint64_t n = rows * D;
  const size_t smem = 8ull * D;
  if (w == 8)
    k_quant_codes<8><<<q_grid(cfg, n), kQThreads, smem, stream>>>(x, n, D, lo_hi, codes);
  else
    k_quant_codes<16><<<q_grid(cfg, n), kQThreads, smem, stream>>>(x, n, D, lo_hi, codes);
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

int launch_dequantize(const LaunchCfg &cfg, const uint8_t *codes, uint64_t rows, uint32_t D, uint32_t w,
                      const double *lo_hi, float *y, cudaStream_t stream) {
  const uint64_t n = rows * D;
  const size_t smem = 8ull * D;
  if (w == 8)
    k_dequant<8><<<q_grid(cfg, n), kQThreads, smem, stream>>>(codes, n, D, lo_hi, y);
  else
    k_dequant<16><<<q_grid(cfg, n), kQThreads, smem, stream>>>(codes, n, D, lo_hi, y);
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

int launch_quant_nmse(const LaunchCfg &cfg, const float *x, const uint8_t *codes, uint64_t rows, uint32_t D,
                      uint32_t w, const double *lo_hi, double *nmse, uint8_t *ws, cudaStream_t stream) {
  double *acc = reinterpret_cast<double *>(ws);
  if (cudaMemsetAsync(acc, 0, 24ull * D, stream) != cudaSuccess) return SPRINTZ_ERR_CUDA;
  const uint32_t grid = q_grid(cfg, rows);
  for (int pass = 0; pass < 2; ++pass) {
    if (w == 8)
      k_quant_err<8><<<grid, kQThreads, 0, stream>>>(x, codes, rows, D, lo_hi, acc, pass);
    else
      k_quant_err<16><<<grid, kQThreads, 0, stream>>>(x, codes, rows, D, lo_hi, acc, pass);
  }
  k_quant_nmse<<<(D + 255) / 256, 256, 0, stream>>>(acc, D, nmse);
  return cudaGetLastError() == cudaSuccess ? SPRINTZ_OK : SPRINTZ_ERR_CUDA;
}

}  // namespace spz
