/*
 * Sprintz oracle: a plain, scalar, single-threaded CPU encoder and decoder of
 * the Sprintz codec (Blalock, Madden, Guttag, "Sprintz: Time Series
 * Compression for the Internet of Things", IMWUT 2018, arXiv:1808.02515).
 *
 * TEST INFRASTRUCTURE. This library is the correctness oracle of the CUDA
 * codec. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg load it. The CUDA library never links, loads or calls it, and the two
 * share no source, header, table or helper.
 *
 * Every routine follows the paper step by step (Algorithms 1-3, Sections
 * 3.2-3.4) and writes the stream format that both implementations agree on.
 * Where the paper leaves the byte format open, the reading used is stated at
 * the routine that implements it.
 */
#ifndef SPRINTZ_ORACLE_H
#define SPRINTZ_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPO_OK 0
#define SPO_ERR_INVALID_ARG (-1)
#define SPO_ERR_UNSUPPORTED_W (-2)
#define SPO_ERR_DST_TOO_SMALL (-3)
#define SPO_ERR_CORRUPT (-5)

typedef struct {
  int32_t forecaster;   /* 0 = delta coding (Sec. 4.2.1), 1 = FIRE in its block form
                           (Sec. 4.2.2), 2 = double delta (Sec. 4.2.2, a = 2, b = -1),
                           3 = FIRE per sample (Algorithm 3's per-sample form) */
  int32_t huffman;      /* 1 = Huffman-code the bit-packed bytes (Sec. 4.4) */
  int32_t group_blocks; /* G: records whose headers are stored together (Sec. 4.3) */
  int32_t learn_shift;  /* FIRE: alpha = accumulator >> learn_shift (eta = 2^-shift) */
  uint32_t chunk_rows;  /* rows between forecaster resets; multiple of 8; 0 = one chunk */
  uint32_t huff_chunks; /* chunks that share one Huffman table */
} spo_opts;

/* ---- whole-stream codec ------------------------------------------------ */

/* Upper bound of the compressed size in bytes; 0 for invalid arguments. */
uint64_t spo_max_compressed_size(uint64_t rows, uint32_t D, uint32_t w,
                                 const spo_opts *o);

/* Compress `rows` x `D` row-major little-endian w-bit samples.  Returns the
 * stream size (> 0) or a negative SPO_ERR_* code. */
int64_t spo_compress(const void *src, uint64_t rows, uint32_t D, uint32_t w,
                     const spo_opts *o, uint8_t *dst, uint64_t dst_cap);

/* Parse the 64-byte stream header. */
int spo_query(const uint8_t *src, uint64_t n, uint64_t *rows, uint32_t *D,
              uint32_t *w, spo_opts *o);

/* Decompress a whole stream into `dst` (rows x D samples).  Returns SPO_OK or
 * a negative SPO_ERR_* code. */
int spo_decompress(const uint8_t *src, uint64_t n, void *dst, uint64_t dst_cap);

/* ---- step-level entry points (used by the pin tests) ------------------- */

/* Zigzag code of a signed w-bit error and its inverse (Sec. 4.3). */
uint32_t spo_zigzag(int32_t e, uint32_t w);
int32_t spo_unzigzag(uint32_t z, uint32_t w);

/* Number of bits that hold `v` (0 for 0). */
uint32_t spo_bit_length(uint32_t v);

/* Stored width of one column of one block from its eight zigzagged errors,
 * with the w-1 -> w promotion of Sec. 4.3. */
uint32_t spo_column_width(const uint32_t z[8], uint32_t w);

/* Forecaster-only pass: the prediction errors (signed, w-bit) of `rows` rows
 * (a multiple of 8) starting from the zero state.  `test_mode` selects oracle
 * test variants of FIRE: 0 = normative block form, 1 = learning disabled
 * (accumulator stays 0), 2 = alpha pinned to `pinned_alpha` every block. */
int spo_forecast_errors(const void *src, uint64_t rows, uint32_t D, uint32_t w,
                        int32_t forecaster, int32_t learn_shift, int32_t test_mode,
                        int64_t pinned_alpha, int32_t *err_out);

/* The inverse of spo_forecast_errors: rebuild `rows` x D samples (written
 * as little-endian w-bit values) from their errors. */
int spo_forecast_reconstruct(const int32_t *err_in, uint64_t rows, uint32_t D, uint32_t w,
                             int32_t forecaster, int32_t learn_shift, void *dst);

/* Float data (Sec. 5.8): each column of `rows` x D float32 samples is
 * offset and rescaled linearly so that its minimum and maximum map to 0 and
 * 2^w - 1, then floored.  In double precision, each operation rounded on its
 * own: s = (2^w - 1) / (max - min) (0 for a constant column), code =
 * floor((x - min) * s), capped at 2^w - 1.  lo_hi receives min and max of
 * each column (2 D doubles).  Codes are little-endian w-bit samples. */
int spo_quantize(const float *src, uint64_t rows, uint32_t D, uint32_t w, void *codes, double *lo_hi);

/* The inverse transform: x = (float)(code * h + min) with the step
 * h = (max - min) / (2^w - 1), each operation rounded on its own. */
int spo_dequantize(const void *codes, uint64_t rows, uint32_t D, uint32_t w, const double *lo_hi,
                   float *dst);

/* Per column: mean squared reconstruction error divided by the column's
 * variance (population variance, two-pass), both in double; 0 for a
 * constant column. */
int spo_quant_nmse(const float *src, const void *codes, uint64_t rows, uint32_t D, uint32_t w,
                   const double *lo_hi, double *nmse);

/* FIRE per-block state trace: after each block k, alpha_k used in it and the
 * accumulator after its update (arrays of n_blocks x D). */
int spo_fire_trace(const void *src, uint64_t rows, uint32_t D, uint32_t w,
                   int32_t learn_shift, int64_t *alpha_out, int64_t *acc_out);

/* Length-limited Huffman code lengths (package-merge) for 256 byte symbols. */
int spo_huff_code_lengths(const uint64_t freq[256], uint32_t max_len,
                          uint8_t len_out[256]);

/* Canonical code values (deflate rule) for a set of code lengths. */
int spo_huff_canonical(const uint8_t len[256], uint32_t code_out[256]);

#ifdef __cplusplus
}
#endif
#endif
