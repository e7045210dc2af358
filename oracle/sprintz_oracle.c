/*
 * Sprintz oracle: plain scalar CPU encoder/decoder.  See sprintz_oracle.h.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the CUDA library.
 *
 * Everything here is written for clarity, not speed: samples are read one at
 * a time, bits are written and read one at a time, and every step of
 * Algorithms 1-3 is a separate function.  All arithmetic is two's-complement
 * integer arithmetic with an explicit wrap to the stated bit width.
 *
 * Stream layout (the paper defines the algorithm but not a container; this is
 * the reading both implementations use):
 *   [0, 64)          stream header (field offsets below, little-endian)
 *   [64, 64+16n)     chunk table, one 16-byte entry per chunk:
 *                      u64 body offset from data_off, u32 records, u32 packed bytes
 *   then             Huffman tables (huffman streams only), 128 bytes per segment:
 *                      256 code lengths, 4 bits each, symbol 2k in the low nibble
 *   data_off         chunk bodies, back to back; a Huffman-coded body is a jump
 *                    table of n-1 u32 sub-block offsets followed by n byte-
 *                    aligned sub-block codes (huff_n_sub below)
 *   tail_off         the rows % 8 trailing rows, stored raw (Sec. 5.4: the
 *                    paper memcpy's trailing bytes)
 *   total_bytes      end of stream
 * Parity of this container is unpinned by the paper: it is our format.
 */
#include "sprintz_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAX_D 1024u
#define BLOCK_ROWS 8u          /* B = 8 (Sec. 4.1) */
#define HUFF_MAX_LEN 11u       /* our length limit for the byte Huffman code */
#define MAX_RUN 65535u         /* a zero run's count is stored in 16 bits */
#define HDR_BYTES 64u
#define CHUNK_ENTRY_BYTES 16u
#define HUFF_TABLE_BYTES 128u
#define HUFF_SUB_BYTES 2048u   /* packed bytes per independently decodable sub-block */

/* ------------------------------------------------------------------------ */
/* Integer helpers                                                          */
/* ------------------------------------------------------------------------ */

/* v mod 2^bits, read as a signed two's-complement number. */
static int64_t wrap_signed(int64_t v, uint32_t bits) {
  uint64_t mask = (1ull << bits) - 1ull;
  uint64_t u = (uint64_t)v & mask;
  if ((u >> (bits - 1)) & 1ull) u |= ~mask;
  return (int64_t)u;
}

/* v mod 2^bits, read as unsigned. */
static int64_t wrap_unsigned(int64_t v, uint32_t bits) {
  return (int64_t)((uint64_t)v & ((1ull << bits) - 1ull));
}

/* floor(v / 2^s): the arithmetic right shift of Algorithm 3. */
static int64_t shift_right_floor(int64_t v, uint32_t s) {
  if (v >= 0) return v >> s;
  return -(int64_t)((((uint64_t)(-(v + 1))) >> s) + 1ull);
}

static int64_t sign_of(int64_t v) { return (v > 0) - (v < 0); }

static uint32_t header_bits(uint32_t w) { return w == 8 ? 3u : 4u; } /* log2(w) */

static uint64_t get_le(const uint8_t *p, uint32_t nbytes) {
  uint64_t v = 0;
  for (uint32_t k = 0; k < nbytes; ++k) v |= (uint64_t)p[k] << (8 * k);
  return v;
}

static void put_le(uint8_t *p, uint64_t v, uint32_t nbytes) {
  for (uint32_t k = 0; k < nbytes; ++k) p[k] = (uint8_t)(v >> (8 * k));
}

/* Sample (row r, column j) of a row-major little-endian w-bit array. */
static int64_t get_sample(const uint8_t *base, uint64_t r, uint32_t j, uint32_t D,
                          uint32_t w) {
  uint64_t idx = r * D + j;
  return (int64_t)get_le(base + idx * (w / 8), w / 8);
}

static void put_sample(uint8_t *base, uint64_t r, uint32_t j, uint32_t D, uint32_t w,
                       int64_t v) {
  uint64_t idx = r * D + j;
  put_le(base + idx * (w / 8), (uint64_t)v, w / 8);
}

/* ------------------------------------------------------------------------ */
/* Bit streams: least significant bit first within little-endian bytes.     */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint8_t *buf; /* zero-filled by the caller */
  uint64_t cap_bytes;
  uint64_t pos; /* in bits */
  int overflow;
} bit_writer;

static void bw_bit(bit_writer *b, uint32_t bit) {
  if ((b->pos >> 3) >= b->cap_bytes) {
    b->overflow = 1;
    return;
  }
  if (bit) b->buf[b->pos >> 3] |= (uint8_t)(1u << (b->pos & 7));
  b->pos++;
}

/* The n low bits of v, least significant first. */
static void bw_bits(bit_writer *b, uint64_t v, uint32_t n) {
  for (uint32_t k = 0; k < n; ++k) bw_bit(b, (uint32_t)((v >> k) & 1u));
}

static void bw_align_byte(bit_writer *b) {
  while (b->pos & 7) bw_bit(b, 0);
}

typedef struct {
  const uint8_t *buf;
  uint64_t n_bytes;
  uint64_t pos; /* in bits */
  int overrun;
} bit_reader;

static uint32_t br_bit(bit_reader *b) {
  if ((b->pos >> 3) >= b->n_bytes) {
    b->overrun = 1;
    return 0;
  }
  uint32_t bit = (b->buf[b->pos >> 3] >> (b->pos & 7)) & 1u;
  b->pos++;
  return bit;
}

static uint64_t br_bits(bit_reader *b, uint32_t n) {
  uint64_t v = 0;
  for (uint32_t k = 0; k < n; ++k) v |= (uint64_t)br_bit(b) << k;
  return v;
}

/* ------------------------------------------------------------------------ */
/* Zigzag and bit widths (Sec. 4.3)                                         */
/* ------------------------------------------------------------------------ */

/* Twice |e| for e >= 0, twice |e| minus one for e < 0 (Sec. 4.3). */
uint32_t spo_zigzag(int32_t e, uint32_t w) {
  int64_t v = wrap_signed(e, w);
  int64_t z = v >= 0 ? 2 * v : -2 * v - 1;
  return (uint32_t)z;
}

int32_t spo_unzigzag(uint32_t z, uint32_t w) {
  int64_t v = (z & 1u) ? -(int64_t)((z + 1u) / 2u) : (int64_t)(z / 2u);
  return (int32_t)wrap_signed(v, w);
}

uint32_t spo_bit_length(uint32_t v) {
  uint32_t n = 0;
  while (v) {
    n++;
    v >>= 1;
  }
  return n;
}

/* Width = bits of the OR of the column's zigzagged errors (Sec. 4.3: w minus
 * the fewest leading zeros), and a width of w-1 is stored as w because the
 * log2(w)-bit header holds only w of the w+1 possible widths. */
uint32_t spo_column_width(const uint32_t z[8], uint32_t w) {
  uint32_t all = 0;
  for (uint32_t r = 0; r < BLOCK_ROWS; ++r) all |= z[r];
  uint32_t n = spo_bit_length(all);
  if (n == w - 1) n = w;
  return n;
}

/* Header code of a stored width: widths 0..w-2 are themselves, width w is w-1. */
static uint32_t width_to_code(uint32_t n, uint32_t w) { return n == w ? w - 1 : n; }
static uint32_t code_to_width(uint32_t c, uint32_t w) { return c == w - 1 ? w : c; }

/* ------------------------------------------------------------------------ */
/* Forecasters (Sec. 4.2)                                                   */
/* ------------------------------------------------------------------------ */

/* 0 delta coding (Sec. 4.2.1); 1 FIRE as used in practice: alpha per block,
 * one averaged update per block from every other sample (Sec. 4.2.2, last
 * paragraph); 2 double-delta coding, the a = 2, b = -1 case of the
 * autoregressive model of Sec. 4.2.2 (predict x_{i-1} + delta_{i-1}); 3 FIRE
 * in its per-sample form (Algorithm 3 without the practical changes of
 * Sec. 4.2.2): a fresh alpha and an accumulator step at every sample. */
enum { FC_DELTA = 0, FC_FIRE = 1, FC_DDELTA = 2, FC_FIRE_SAMPLE = 3 };
enum { FIRE_NORMAL = 0, FIRE_NO_LEARNING = 1, FIRE_PINNED_ALPHA = 2 };

typedef struct {
  int32_t kind;
  uint32_t D, w, learn_shift;
  int32_t test_mode;
  int64_t pinned_alpha;
  int64_t prev[MAX_D];   /* x_{i-1}: the previous sample, zeros initially (Sec. 4.2.1) */
  int64_t deltas[MAX_D]; /* FIRE / double delta: x_{i-1} - x_{i-2}, signed w-bit */
  int64_t acc[MAX_D];    /* FIRE accumulator A_j: signed 2w-bit */
  int64_t alpha[MAX_D];  /* FIRE alpha of the current block */
  int64_t grad[MAX_D];   /* FIRE sum of the block's sampled gradients */
} forecaster;

/* Initial state (Sec. 4.2.2): A_j = 0 and delta_{-1} = 0 for every column. */
static void fc_init(forecaster *f, int32_t kind, uint32_t D, uint32_t w,
                    uint32_t learn_shift, int32_t test_mode, int64_t pinned_alpha) {
  memset(f, 0, sizeof(*f));
  f->kind = kind;
  f->D = D;
  f->w = w;
  f->learn_shift = learn_shift;
  f->test_mode = test_mode;
  f->pinned_alpha = pinned_alpha;
}

/* FIRE in practice (last paragraph of Sec. 4.2.2): alpha is computed once at
 * the start of each block as alpha_j = A_j >> s (s = learn_shift, floor). */
static void fc_block_begin(forecaster *f) {
  if (f->kind != FC_FIRE) return;
  for (uint32_t j = 0; j < f->D; ++j) {
    if (f->test_mode == FIRE_PINNED_ALPHA)
      f->alpha[j] = f->pinned_alpha;
    else
      f->alpha[j] = shift_right_floor(f->acc[j], f->learn_shift);
    f->grad[j] = 0;
  }
}

/* Predict column j of sample i from x_{i-1}.
 * Delta: the previous sample.  FIRE (Sec. 4.2.2): x_{i-1} plus the scaled
 * previous delta floor(alpha * delta_{i-1} / 2^w), the product taken in 2w
 * bits. */
static int64_t fc_predict(const forecaster *f, uint32_t j) {
  if (f->kind == FC_DELTA) return f->prev[j];
  /* double delta: linear extrapolation from the last two samples */
  if (f->kind == FC_DDELTA) return wrap_unsigned(f->prev[j] + f->deltas[j], f->w);
  /* per-sample form: alpha_j = A_j >> s taken afresh for every sample */
  int64_t alpha = f->kind == FC_FIRE_SAMPLE ? shift_right_floor(f->acc[j], f->learn_shift) : f->alpha[j];
  int64_t product = wrap_signed(alpha * f->deltas[j], 2 * f->w);
  int64_t predicted_delta = shift_right_floor(product, f->w);
  return wrap_unsigned(f->prev[j] + predicted_delta, f->w);
}

/* Learning step (Sec. 4.2.2) for column j of sample i (0-based row within
 * the block).  The L1 loss |e_i| has gradient -sign(e_i) * delta_{i-1} with
 * respect to alpha, and A_j takes a step against it.  In practice a gradient
 * is taken only on every other sample (rows 0, 2, 4, 6) and summed for one
 * update per block. */
static void fc_train(forecaster *f, uint32_t j, uint32_t i, int64_t x_i, int64_t err) {
  if (f->kind == FC_FIRE) {
    if (i % 2 == 0) f->grad[j] += sign_of(err) * f->deltas[j];
    f->deltas[j] = wrap_signed(x_i - f->prev[j], f->w);
  } else if (f->kind == FC_FIRE_SAMPLE) {
    /* per-sample step: A_j += sign(e_i) * delta_{i-1} (2w-bit wrap), then
     * delta_i = x_i - x_{i-1} */
    f->acc[j] = wrap_signed(f->acc[j] + sign_of(err) * f->deltas[j], 2 * f->w);
    f->deltas[j] = wrap_signed(x_i - f->prev[j], f->w);
  } else if (f->kind == FC_DDELTA) {
    f->deltas[j] = wrap_signed(x_i - f->prev[j], f->w);
  }
  f->prev[j] = x_i;
}

/* One update per block with the average of the four sampled gradients
 * (floor division by 4), wrapped to the accumulator's 2w bits. */
static void fc_block_end(forecaster *f) {
  if (f->kind != FC_FIRE || f->test_mode != FIRE_NORMAL) return;
  for (uint32_t j = 0; j < f->D; ++j)
    f->acc[j] = wrap_signed(f->acc[j] + shift_right_floor(f->grad[j], 2), 2 * f->w);
}

/* Algorithm 1, first loop: predict, take the error, train, for 8 samples. */
static void fc_encode_block(forecaster *f, const int64_t *x /* 8 x D */,
                            int64_t *err /* 8 x D */) {
  fc_block_begin(f);
  for (uint32_t i = 0; i < BLOCK_ROWS; ++i) {
    for (uint32_t j = 0; j < f->D; ++j) {
      int64_t xhat = fc_predict(f, j);
      int64_t e = wrap_signed(x[i * f->D + j] - xhat, f->w);
      err[i * f->D + j] = e;
      fc_train(f, j, i, x[i * f->D + j], e);
    }
  }
  fc_block_end(f);
}

/* Algorithm 2, non-run branch: predict, add the unpacked error, output,
 * train.  With all errors zero this is also the run branch: the forecaster
 * runs on its own predictions (sign(0) = 0 leaves the accumulator as is). */
static void fc_decode_block(forecaster *f, const int64_t *err /* 8 x D */,
                            int64_t *x /* 8 x D */) {
  fc_block_begin(f);
  for (uint32_t i = 0; i < BLOCK_ROWS; ++i) {
    for (uint32_t j = 0; j < f->D; ++j) {
      int64_t xhat = fc_predict(f, j);
      int64_t v = wrap_unsigned(xhat + err[i * f->D + j], f->w);
      x[i * f->D + j] = v;
      fc_train(f, j, i, v, err[i * f->D + j]);
    }
  }
  fc_block_end(f);
}

/* ------------------------------------------------------------------------ */
/* Records, header groups and payloads (Algorithm 1 / Sec. 4.3)             */
/* ------------------------------------------------------------------------ */

typedef struct {
  int is_run;                /* zero run (all headers 0, payload = count) */
  uint32_t run_blocks;       /* 1..65535 */
  uint32_t width[MAX_D];     /* stored widths of a packed block */
  uint32_t z[BLOCK_ROWS * MAX_D]; /* zigzagged errors, row-major 8 x D */
} record;

typedef struct {
  uint32_t D, w, G;
  record *pending; /* G records awaiting their group */
  uint32_t n_pending;
  uint64_t n_records;
  bit_writer out;
} group_writer;

static int column_major(uint32_t D, uint32_t w) { return D * w <= 32; }

/* Payload of one record.  A run stores its block count as 16 bits.  A packed
 * block is column-major when a sample is at most 32 bits wide (each column's
 * 8 values at bits r*n_j, exactly n_j bytes), else row-major (each row's
 * columns at fixed bit offsets, padded to a byte). */
static void write_payload(bit_writer *b, const record *rec, uint32_t D, uint32_t w) {
  if (rec->is_run) {
    bw_bits(b, rec->run_blocks, 16);
    return;
  }
  if (column_major(D, w)) {
    for (uint32_t j = 0; j < D; ++j)
      for (uint32_t r = 0; r < BLOCK_ROWS; ++r) bw_bits(b, rec->z[r * D + j], rec->width[j]);
  } else {
    for (uint32_t r = 0; r < BLOCK_ROWS; ++r) {
      for (uint32_t j = 0; j < D; ++j) bw_bits(b, rec->z[r * D + j], rec->width[j]);
      bw_align_byte(b);
    }
  }
}

/* A group: the headers of its (up to G) records, code of record s column j at
 * bit (s*D + j)*log2(w), padded to a byte, then the records' payloads. */
static void flush_group(group_writer *g) {
  if (g->n_pending == 0) return;
  uint32_t hb = header_bits(g->w);
  for (uint32_t s = 0; s < g->G; ++s) {
    for (uint32_t j = 0; j < g->D; ++j) {
      uint32_t code = 0;
      if (s < g->n_pending && !g->pending[s].is_run)
        code = width_to_code(g->pending[s].width[j], g->w);
      bw_bits(&g->out, code, hb);
    }
  }
  bw_align_byte(&g->out);
  for (uint32_t s = 0; s < g->n_pending; ++s) write_payload(&g->out, &g->pending[s], g->D, g->w);
  g->n_pending = 0;
}

/* Append a finished record; a full group is written out at once. */
static void push_record(group_writer *g, const record *r) {
  memcpy(&g->pending[g->n_pending], r, sizeof(record));
  g->n_pending++;
  g->n_records++;
  if (g->n_pending == g->G) flush_group(g);
}

static void push_run(group_writer *g, record *scratch, uint32_t blocks) {
  scratch->is_run = 1;
  scratch->run_blocks = blocks;
  push_record(g, scratch);
}

/* Encode the chunk of `n_blocks` blocks starting at `src` (Algorithm 1 run
 * over the chunk, the forecaster starting from its zero state).  Writes the
 * body into g->out; returns 0 or an error. */
static int encode_chunk(const uint8_t *src, uint64_t n_blocks, uint32_t D, uint32_t w,
                        const spo_opts *o, group_writer *g) {
  forecaster *f = (forecaster *)malloc(sizeof(forecaster));
  int64_t *x = (int64_t *)malloc(sizeof(int64_t) * BLOCK_ROWS * D);
  int64_t *err = (int64_t *)malloc(sizeof(int64_t) * BLOCK_ROWS * D);
  record *cur = (record *)malloc(sizeof(record));
  record *run_rec = (record *)malloc(sizeof(record));
  if (!f || !x || !err || !cur || !run_rec) {
    free(f); free(x); free(err); free(cur); free(run_rec);
    return SPO_ERR_INVALID_ARG;
  }
  memset(run_rec, 0, sizeof(record));
  fc_init(f, o->forecaster, D, w, (uint32_t)o->learn_shift, FIRE_NORMAL, 0);
  uint32_t run = 0;
  for (uint64_t b = 0; b < n_blocks; ++b) {
    /* Algorithm 1, first step: forecast the block and take the errors. */
    for (uint32_t i = 0; i < BLOCK_ROWS; ++i)
      for (uint32_t j = 0; j < D; ++j)
        x[i * D + j] = get_sample(src, b * BLOCK_ROWS + i, j, D, w);
    fc_encode_block(f, x, err);

    /* Lines 8-11: zigzag, per-column width (bit packing happens when the
     * record's group is written). */
    int all_zero = 1;
    cur->is_run = 0;
    cur->run_blocks = 0;
    for (uint32_t j = 0; j < D; ++j) {
      uint32_t zc[BLOCK_ROWS];
      for (uint32_t i = 0; i < BLOCK_ROWS; ++i) {
        zc[i] = spo_zigzag((int32_t)err[i * D + j], w);
        cur->z[i * D + j] = zc[i];
      }
      cur->width[j] = spo_column_width(zc, w);
      if (cur->width[j] != 0) all_zero = 0;
    }

    /* Lines 12-20: all widths zero -> extend the run of zero blocks; the
     * run's record (zero headers, block count) precedes the block that
     * ends it.  A count is 16 bits, so a run is cut at 65535 blocks. */
    if (all_zero) {
      run++;
      if (run == MAX_RUN) {
        push_run(g, run_rec, run);
        run = 0;
      }
      continue;
    }
    if (run) {
      push_run(g, run_rec, run);
      run = 0;
    }
    /* Lines 21-23: this block's headers and payload. */
    push_record(g, cur);
  }
  if (run) push_run(g, run_rec, run); /* the chunk ends inside a run */
  flush_group(g);                     /* a partial last group */
  free(f);
  free(x);
  free(err);
  free(cur);
  free(run_rec);
  return g->out.overflow ? SPO_ERR_DST_TOO_SMALL : SPO_OK;
}

/* ------------------------------------------------------------------------ */
/* Length-limited Huffman codes (Sec. 4.4; our own coder in place of Huff0) */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t weight;
  uint32_t n_syms;
  uint16_t *syms; /* leaf symbols inside this item, with multiplicity */
} pm_item;

static pm_item pm_leaf(uint64_t weight, uint16_t sym) {
  pm_item it;
  it.weight = weight;
  it.n_syms = 1;
  it.syms = (uint16_t *)malloc(sizeof(uint16_t));
  it.syms[0] = sym;
  return it;
}

static pm_item pm_package(const pm_item *a, const pm_item *b) {
  pm_item it;
  it.weight = a->weight + b->weight;
  it.n_syms = a->n_syms + b->n_syms;
  it.syms = (uint16_t *)malloc(sizeof(uint16_t) * it.n_syms);
  memcpy(it.syms, a->syms, sizeof(uint16_t) * a->n_syms);
  memcpy(it.syms + a->n_syms, b->syms, sizeof(uint16_t) * b->n_syms);
  return it;
}

static pm_item pm_copy(const pm_item *a) {
  pm_item it = *a;
  it.syms = (uint16_t *)malloc(sizeof(uint16_t) * a->n_syms);
  memcpy(it.syms, a->syms, sizeof(uint16_t) * a->n_syms);
  return it;
}

static void pm_free_list(pm_item *list, uint32_t n) {
  for (uint32_t k = 0; k < n; ++k) free(list[k].syms);
  free(list);
}

/* Package-merge (Larmore & Hirschberg 1990), the textbook form:
 *   list <- the leaves sorted by (frequency, symbol);
 *   repeat max_len - 1 times:
 *     package adjacent pairs of list (an odd last item is dropped),
 *     list <- merge(leaves, packages), a leaf before a package of equal weight;
 *   take the first 2n - 2 items; a symbol's code length is the number of
 *   times it occurs in them.
 * A single used symbol gets length 1; unused symbols get length 0. */
int spo_huff_code_lengths(const uint64_t freq[256], uint32_t max_len, uint8_t len_out[256]) {
  memset(len_out, 0, 256);
  uint16_t order[256];
  uint32_t n = 0;
  for (uint32_t s = 0; s < 256; ++s)
    if (freq[s]) order[n++] = (uint16_t)s;
  /* insertion sort by (freq, symbol) */
  for (uint32_t a = 1; a < n; ++a) {
    uint16_t s = order[a];
    uint32_t b = a;
    while (b > 0 && (freq[order[b - 1]] > freq[s] ||
                     (freq[order[b - 1]] == freq[s] && order[b - 1] > s))) {
      order[b] = order[b - 1];
      b--;
    }
    order[b] = s;
  }
  if (n == 0) return SPO_OK;
  if (n == 1) {
    len_out[order[0]] = 1;
    return SPO_OK;
  }
  if (max_len < 1 || max_len > 30 || (uint64_t)n > (1ull << max_len)) return SPO_ERR_INVALID_ARG;

  pm_item *leaves = (pm_item *)malloc(sizeof(pm_item) * n);
  for (uint32_t k = 0; k < n; ++k) leaves[k] = pm_leaf(freq[order[k]], order[k]);

  uint32_t list_n = n;
  pm_item *list = (pm_item *)malloc(sizeof(pm_item) * n);
  for (uint32_t k = 0; k < n; ++k) list[k] = pm_copy(&leaves[k]);

  for (uint32_t level = 1; level < max_len; ++level) {
    uint32_t n_pkg = list_n / 2;
    pm_item *pkg = (pm_item *)malloc(sizeof(pm_item) * (n_pkg ? n_pkg : 1));
    for (uint32_t k = 0; k < n_pkg; ++k) pkg[k] = pm_package(&list[2 * k], &list[2 * k + 1]);
    pm_free_list(list, list_n);

    list_n = n + n_pkg;
    list = (pm_item *)malloc(sizeof(pm_item) * list_n);
    uint32_t a = 0, b = 0;
    for (uint32_t k = 0; k < list_n; ++k) {
      int take_leaf = a < n && (b >= n_pkg || leaves[a].weight <= pkg[b].weight);
      list[k] = take_leaf ? pm_copy(&leaves[a++]) : pm_copy(&pkg[b++]);
    }
    pm_free_list(pkg, n_pkg);
  }

  uint32_t take = 2 * n - 2;
  for (uint32_t k = 0; k < take && k < list_n; ++k)
    for (uint32_t t = 0; t < list[k].n_syms; ++t) len_out[list[k].syms[t]]++;

  pm_free_list(list, list_n);
  pm_free_list(leaves, n);
  return SPO_OK;
}

/* Canonical codes as in RFC 1951 Sec. 3.2.2: shorter codes first, and within
 * one length in symbol order. */
int spo_huff_canonical(const uint8_t len[256], uint32_t code_out[256]) {
  uint32_t bl_count[32] = {0};
  uint32_t next_code[32] = {0};
  for (uint32_t s = 0; s < 256; ++s) {
    if (len[s] > 30) return SPO_ERR_INVALID_ARG;
    if (len[s]) bl_count[len[s]]++;
  }
  uint32_t code = 0;
  for (uint32_t bits = 1; bits < 32; ++bits) {
    code = (code + bl_count[bits - 1]) << 1;
    next_code[bits] = code;
  }
  for (uint32_t s = 0; s < 256; ++s) {
    code_out[s] = 0;
    if (len[s]) code_out[s] = next_code[len[s]]++;
  }
  return SPO_OK;
}

/* Kraft sum check: the code must not be over-subscribed. */
static int huff_lengths_valid(const uint8_t len[256]) {
  uint64_t kraft = 0; /* in units of 2^-HUFF_MAX_LEN */
  for (uint32_t s = 0; s < 256; ++s) {
    if (len[s] > HUFF_MAX_LEN) return 0;
    if (len[s]) kraft += 1ull << (HUFF_MAX_LEN - len[s]);
  }
  return kraft <= (1ull << HUFF_MAX_LEN);
}

/* Write one symbol's code, its most significant bit first, into the
 * least-significant-bit-first stream (the deflate convention). */
static void huff_put(bit_writer *b, uint32_t code, uint32_t len) {
  for (uint32_t k = len; k > 0; --k) bw_bit(b, (code >> (k - 1)) & 1u);
}

/* Canonical decoding one bit at a time: for each length, codes of that length
 * are consecutive starting at `first`. */
static int huff_get(bit_reader *b, const uint8_t len[256], uint32_t *sym) {
  uint32_t count[HUFF_MAX_LEN + 1] = {0};
  uint16_t sorted[256];
  uint32_t n_sorted = 0;
  for (uint32_t l = 1; l <= HUFF_MAX_LEN; ++l)
    for (uint32_t s = 0; s < 256; ++s)
      if (len[s] == l) {
        count[l]++;
        sorted[n_sorted++] = (uint16_t)s;
      }
  uint32_t code = 0, first = 0, index = 0;
  for (uint32_t l = 1; l <= HUFF_MAX_LEN; ++l) {
    code |= br_bit(b);
    if (b->overrun) return SPO_ERR_CORRUPT;
    if (code - first < count[l]) {
      *sym = sorted[index + (code - first)];
      return SPO_OK;
    }
    index += count[l];
    first += count[l];
    first <<= 1;
    code <<= 1;
  }
  return SPO_ERR_CORRUPT;
}

/* ------------------------------------------------------------------------ */
/* Whole stream                                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t rows, full_rows, n_chunks, n_segments, tail_rows;
  uint64_t chunk_rows_eff; /* rows per chunk (the last may be shorter) */
  uint64_t data_off;
} layout;

static int check_opts(uint32_t D, uint32_t w, const spo_opts *o) {
  if (w != 8 && w != 16) return SPO_ERR_UNSUPPORTED_W;
  if (D < 1 || D > MAX_D) return SPO_ERR_INVALID_ARG;
  if (o->forecaster < FC_DELTA || o->forecaster > FC_FIRE_SAMPLE) return SPO_ERR_INVALID_ARG;
  if (o->huffman != 0 && o->huffman != 1) return SPO_ERR_INVALID_ARG;
  if (o->group_blocks < 1 || o->group_blocks > 8) return SPO_ERR_INVALID_ARG;
  if (o->learn_shift < 0 || o->learn_shift > (int32_t)(2 * w - 1)) return SPO_ERR_INVALID_ARG;
  if (o->chunk_rows % BLOCK_ROWS) return SPO_ERR_INVALID_ARG;
  if (o->huffman && o->huff_chunks < 1) return SPO_ERR_INVALID_ARG;
  return SPO_OK;
}

static void make_layout(uint64_t rows, const spo_opts *o, layout *L) {
  L->rows = rows;
  L->tail_rows = rows % BLOCK_ROWS;
  L->full_rows = rows - L->tail_rows;
  if (L->full_rows == 0)
    L->n_chunks = 0;
  else if (o->chunk_rows == 0)
    L->n_chunks = 1;
  else
    L->n_chunks = (L->full_rows + o->chunk_rows - 1) / o->chunk_rows;
  L->chunk_rows_eff = o->chunk_rows ? o->chunk_rows : L->full_rows;
  L->n_segments = o->huffman ? (L->n_chunks + o->huff_chunks - 1) / o->huff_chunks : 0;
  L->data_off = HDR_BYTES + CHUNK_ENTRY_BYTES * L->n_chunks + HUFF_TABLE_BYTES * L->n_segments;
}

static uint64_t chunk_blocks(const layout *L, uint64_t c) {
  uint64_t first = c * L->chunk_rows_eff;
  uint64_t last = first + L->chunk_rows_eff;
  if (last > L->full_rows) last = L->full_rows;
  return (last - first) / BLOCK_ROWS;
}

static uint64_t max_body_bytes(uint64_t n_blocks, uint32_t D, uint32_t w, uint32_t G) {
  uint64_t hdr = ((uint64_t)G * D * header_bits(w) + 7) / 8;
  return (n_blocks + G - 1) / G * hdr + n_blocks * (uint64_t)D * w;
}

/* A chunk body's size is stored in 32 bits and the chunk count in 32 bits. */
static int check_layout(const layout *L, uint32_t D, uint32_t w, uint32_t G, int huffman) {
  if (L->n_chunks > 0xFFFFFFFFull) return SPO_ERR_INVALID_ARG;
  uint64_t limit = huffman ? (1ull << 31) : 0xFFFFFFFFull; /* Huffman: jump-table offsets fit u32 */
  if (L->n_chunks && max_body_bytes(chunk_blocks(L, 0), D, w, G) > limit) return SPO_ERR_INVALID_ARG;
  return SPO_OK;
}

uint64_t spo_max_compressed_size(uint64_t rows, uint32_t D, uint32_t w, const spo_opts *o) {
  if (check_opts(D, w, o) != SPO_OK) return 0;
  layout L;
  make_layout(rows, o, &L);
  if (check_layout(&L, D, w, (uint32_t)o->group_blocks, o->huffman) != SPO_OK) return 0;
  uint64_t total = L.data_off;
  for (uint64_t c = 0; c < L.n_chunks; ++c)
    total += max_body_bytes(chunk_blocks(&L, c), D, w, (uint32_t)o->group_blocks);
  total += L.tail_rows * D * (w / 8);
  return total;
}

static void write_header(uint8_t *dst, const layout *L, uint32_t D, uint32_t w,
                         const spo_opts *o, uint64_t tail_off, uint64_t total) {
  memset(dst, 0, HDR_BYTES);
  dst[0] = 'S';
  dst[1] = 'P';
  dst[2] = 'Z';
  dst[3] = '1';
  dst[4] = 1; /* version */
  dst[5] = (uint8_t)w;
  dst[6] = (uint8_t)o->forecaster;
  dst[7] = (uint8_t)(o->huffman ? 1 : 0);
  put_le(dst + 8, D, 2);
  dst[10] = (uint8_t)o->group_blocks;
  dst[11] = (uint8_t)o->learn_shift;
  put_le(dst + 12, o->chunk_rows, 4);
  put_le(dst + 16, o->huffman ? o->huff_chunks : 0, 4);
  put_le(dst + 20, L->n_chunks, 4);
  put_le(dst + 24, L->rows, 8);
  put_le(dst + 32, L->tail_rows, 4);
  put_le(dst + 40, L->data_off, 8);
  put_le(dst + 48, tail_off, 8);
  put_le(dst + 56, total, 8);
}

/* Sub-blocks of one chunk's code (our container; Huff0, the coder the paper
 * uses, likewise splits a block into separately decodable streams behind a
 * jump table of their sizes, RFC 8878 Sec. 4.2.2).  A body of `packed` bytes
 * has n = ceil(packed / S) sub-blocks of q = ceil(packed / n) bytes each
 * (S = HUFF_SUB_BYTES; the last one may be shorter; an empty body has one
 * empty sub-block): sub-block k holds the packed bytes
 * [min(packed, k*q), min(packed, (k+1)*q)).  The coded body is
 *   n-1 u32 offsets: where sub-blocks 1..n-1 start, counted from the end of
 *                    this table,
 *   n codes:         each sub-block's symbols, padded to a byte. */
static uint64_t huff_n_sub(uint64_t packed) {
  return packed == 0 ? 1 : (packed + HUFF_SUB_BYTES - 1) / HUFF_SUB_BYTES;
}

/* Packed bytes [*i0, *i1) of sub-block k. */
static void huff_sub_range(uint64_t packed, uint64_t k, uint64_t *i0, uint64_t *i1) {
  uint64_t n = huff_n_sub(packed);
  uint64_t q = (packed + n - 1) / n;
  *i0 = k * q < packed ? k * q : packed;
  *i1 = (k + 1) * q < packed ? (k + 1) * q : packed;
}

/* Coded bytes of one chunk body under the code lengths len. */
static uint64_t huff_coded_bytes(const uint8_t *body, uint64_t packed, const uint8_t len[256]) {
  uint64_t n_sub = huff_n_sub(packed);
  uint64_t bytes = 4 * (n_sub - 1);
  for (uint64_t k = 0; k < n_sub; ++k) {
    uint64_t i0, i1, bits = 0;
    huff_sub_range(packed, k, &i0, &i1);
    for (uint64_t i = i0; i < i1; ++i) bits += len[body[i]];
    bytes += (bits + 7) / 8;
  }
  return bytes;
}

/* Huffman-code one segment's packed chunk bodies.  Returns the coded bytes
 * written at out (or a negative error). */
static int64_t huff_encode_segment(uint8_t *const *bodies, const uint64_t *packed,
                                   uint32_t n, uint8_t *table_out, uint8_t *out,
                                   uint64_t out_cap, uint64_t *coded_sizes) {
  uint64_t freq[256] = {0};
  uint64_t total_packed = 0;
  for (uint32_t c = 0; c < n; ++c) {
    for (uint64_t k = 0; k < packed[c]; ++k) freq[bodies[c][k]]++;
    total_packed += packed[c];
  }
  uint8_t len[256];
  spo_huff_code_lengths(freq, HUFF_MAX_LEN, len);
  uint64_t coded_total = 0;
  for (uint32_t c = 0; c < n; ++c) coded_total += huff_coded_bytes(bodies[c], packed[c], len);
  int raw = (total_packed == 0) || (coded_total >= total_packed);
  if (raw) memset(len, 0, sizeof(len));
  for (uint32_t k = 0; k < 128; ++k) table_out[k] = (uint8_t)(len[2 * k] | (len[2 * k + 1] << 4));

  uint32_t code[256];
  spo_huff_canonical(len, code);
  uint64_t pos = 0;
  for (uint32_t c = 0; c < n; ++c) {
    if (raw) {
      if (pos + packed[c] > out_cap) return SPO_ERR_DST_TOO_SMALL;
      memcpy(out + pos, bodies[c], packed[c]);
      coded_sizes[c] = packed[c];
      pos += packed[c];
      continue;
    }
    uint64_t n_sub = huff_n_sub(packed[c]);
    uint64_t jump = 4 * (n_sub - 1);
    if (pos + jump > out_cap) return SPO_ERR_DST_TOO_SMALL;
    bit_writer b = {out + pos + jump, out_cap - pos - jump, 0, 0};
    for (uint64_t k = 0; k < n_sub; ++k) {
      if (k > 0) put_le(out + pos + 4 * (k - 1), b.pos / 8, 4);
      uint64_t i0, i1;
      huff_sub_range(packed[c], k, &i0, &i1);
      for (uint64_t i = i0; i < i1; ++i)
        huff_put(&b, code[bodies[c][i]], len[bodies[c][i]]);
      bw_align_byte(&b);
    }
    if (b.overflow) return SPO_ERR_DST_TOO_SMALL;
    coded_sizes[c] = jump + b.pos / 8;
    pos += coded_sizes[c];
  }
  return (int64_t)pos;
}

int64_t spo_compress(const void *src_v, uint64_t rows, uint32_t D, uint32_t w,
                     const spo_opts *o, uint8_t *dst, uint64_t dst_cap) {
  const uint8_t *src = (const uint8_t *)src_v;
  int rc = check_opts(D, w, o);
  if (rc != SPO_OK) return rc;
  layout L;
  make_layout(rows, o, &L);
  rc = check_layout(&L, D, w, (uint32_t)o->group_blocks, o->huffman);
  if (rc != SPO_OK) return rc;
  if (dst_cap < L.data_off) return SPO_ERR_DST_TOO_SMALL;
  memset(dst, 0, L.data_off);

  uint32_t G = (uint32_t)o->group_blocks;
  group_writer g;
  g.D = D;
  g.w = w;
  g.G = G;
  g.pending = (record *)malloc(sizeof(record) * G);
  if (!g.pending) return SPO_ERR_INVALID_ARG;

  uint64_t sample_bytes = (uint64_t)D * (w / 8);
  uint64_t pos = L.data_off;

  /* Packed bodies are built in scratch buffers; without Huffman they are
   * copied straight to the stream, with Huffman they wait for their segment. */
  uint8_t **bodies = (uint8_t **)calloc(L.n_chunks ? L.n_chunks : 1, sizeof(uint8_t *));
  uint64_t *packed = (uint64_t *)calloc(L.n_chunks ? L.n_chunks : 1, sizeof(uint64_t));
  uint64_t *coded = (uint64_t *)calloc(L.n_chunks ? L.n_chunks : 1, sizeof(uint64_t));
  rc = SPO_OK;
  for (uint64_t c = 0; c < L.n_chunks && rc == SPO_OK; ++c) {
    uint64_t nb = chunk_blocks(&L, c);
    uint64_t cap = max_body_bytes(nb, D, w, G);
    bodies[c] = (uint8_t *)calloc(cap ? cap : 1, 1);
    g.n_pending = 0;
    g.n_records = 0;
    g.out.buf = bodies[c];
    g.out.cap_bytes = cap;
    g.out.pos = 0;
    g.out.overflow = 0;
    rc = encode_chunk(src + c * L.chunk_rows_eff * sample_bytes, nb, D, w, o, &g);
    packed[c] = g.out.pos / 8;
    uint8_t *entry = dst + HDR_BYTES + CHUNK_ENTRY_BYTES * c;
    put_le(entry + 8, g.n_records, 4);
    put_le(entry + 12, packed[c], 4);
    if (!o->huffman && rc == SPO_OK) {
      put_le(entry, pos - L.data_off, 8);
      if (pos + packed[c] > dst_cap) {
        rc = SPO_ERR_DST_TOO_SMALL;
        break;
      }
      memcpy(dst + pos, bodies[c], packed[c]);
      pos += packed[c];
      free(bodies[c]);
      bodies[c] = NULL;
    }
  }
  if (o->huffman && rc == SPO_OK) {
    for (uint64_t s = 0; s < L.n_segments && rc == SPO_OK; ++s) {
      uint64_t c0 = s * o->huff_chunks;
      uint64_t c1 = c0 + o->huff_chunks;
      if (c1 > L.n_chunks) c1 = L.n_chunks;
      uint8_t *table = dst + HDR_BYTES + CHUNK_ENTRY_BYTES * L.n_chunks + HUFF_TABLE_BYTES * s;
      int64_t n = huff_encode_segment(bodies + c0, packed + c0, (uint32_t)(c1 - c0), table,
                                      dst + pos, dst_cap > pos ? dst_cap - pos : 0, coded + c0);
      if (n < 0) {
        rc = (int)n;
        break;
      }
      uint64_t off = pos - L.data_off;
      for (uint64_t c = c0; c < c1; ++c) {
        put_le(dst + HDR_BYTES + CHUNK_ENTRY_BYTES * c, off, 8);
        off += coded[c];
      }
      pos += (uint64_t)n;
    }
  }
  for (uint64_t c = 0; c < L.n_chunks; ++c) free(bodies[c]);
  free(bodies);
  free(packed);
  free(coded);
  free(g.pending);
  if (rc != SPO_OK) return rc;

  /* Trailing rows (rows % 8) are copied as they are. */
  uint64_t tail_off = pos;
  uint64_t tail_bytes = L.tail_rows * sample_bytes;
  if (pos + tail_bytes > dst_cap) return SPO_ERR_DST_TOO_SMALL;
  memcpy(dst + pos, src + L.full_rows * sample_bytes, tail_bytes);
  pos += tail_bytes;
  write_header(dst, &L, D, w, o, tail_off, pos);
  return (int64_t)pos;
}

/* ------------------------------------------------------------------------ */
/* Decoding                                                                 */
/* ------------------------------------------------------------------------ */

int spo_query(const uint8_t *src, uint64_t n, uint64_t *rows, uint32_t *D, uint32_t *w,
              spo_opts *o) {
  if (n < HDR_BYTES) return SPO_ERR_CORRUPT;
  if (src[0] != 'S' || src[1] != 'P' || src[2] != 'Z' || src[3] != '1' || src[4] != 1)
    return SPO_ERR_CORRUPT;
  *w = src[5];
  o->forecaster = src[6];
  o->huffman = src[7] & 1;
  if (src[7] & ~1u) return SPO_ERR_CORRUPT;
  *D = (uint32_t)get_le(src + 8, 2);
  o->group_blocks = src[10];
  o->learn_shift = src[11];
  o->chunk_rows = (uint32_t)get_le(src + 12, 4);
  o->huff_chunks = (uint32_t)get_le(src + 16, 4);
  *rows = get_le(src + 24, 8);
  int rc = check_opts(*D, *w, o);
  if (rc == SPO_ERR_UNSUPPORTED_W) return SPO_ERR_CORRUPT;
  return rc == SPO_OK ? SPO_OK : SPO_ERR_CORRUPT;
}

/* Decode one chunk body (Algorithm 2 applied record by record). */
static int decode_chunk(const uint8_t *body, uint64_t body_bytes, uint64_t n_records,
                        uint64_t n_blocks, uint32_t D, uint32_t w, const spo_opts *o,
                        uint8_t *dst /* chunk's first row */) {
  uint32_t G = (uint32_t)o->group_blocks;
  uint32_t hb = header_bits(w);
  forecaster *f = (forecaster *)malloc(sizeof(forecaster));
  int64_t *err = (int64_t *)malloc(sizeof(int64_t) * BLOCK_ROWS * D);
  int64_t *x = (int64_t *)malloc(sizeof(int64_t) * BLOCK_ROWS * D);
  uint32_t *codes = (uint32_t *)malloc(sizeof(uint32_t) * G * D);
  int rc = SPO_OK;
  if (!f || !err || !x || !codes) rc = SPO_ERR_INVALID_ARG;
  if (rc == SPO_OK) fc_init(f, o->forecaster, D, w, (uint32_t)o->learn_shift, FIRE_NORMAL, 0);

  bit_reader b = {body, body_bytes, 0, 0};
  uint64_t rec = 0, blk = 0;
  while (rc == SPO_OK && rec < n_records) {
    uint64_t k = n_records - rec < G ? n_records - rec : G;
    for (uint32_t s = 0; s < G; ++s)
      for (uint32_t j = 0; j < D; ++j) codes[s * D + j] = (uint32_t)br_bits(&b, hb);
    while (b.pos & 7) br_bit(&b);
    for (uint32_t s = 0; s < G && rc == SPO_OK; ++s) {
      int any = 0;
      for (uint32_t j = 0; j < D; ++j) any |= codes[s * D + j] != 0;
      if (s >= k) {
        if (any) rc = SPO_ERR_CORRUPT; /* unused slots hold zero codes */
        continue;
      }
      if (!any) {
        /* Run branch: the payload is the number of all-zero blocks. */
        uint64_t count = br_bits(&b, 16);
        if (count == 0 || blk + count > n_blocks) {
          rc = SPO_ERR_CORRUPT;
          break;
        }
        for (uint32_t q = 0; q < BLOCK_ROWS * D; ++q) err[q] = 0;
        for (uint64_t r = 0; r < count; ++r) {
          fc_decode_block(f, err, x);
          for (uint32_t i = 0; i < BLOCK_ROWS; ++i)
            for (uint32_t j = 0; j < D; ++j) put_sample(dst, blk * BLOCK_ROWS + i, j, D, w, x[i * D + j]);
          blk++;
        }
        continue;
      }
      if (blk + 1 > n_blocks) {
        rc = SPO_ERR_CORRUPT;
        break;
      }
      uint32_t width[MAX_D];
      for (uint32_t j = 0; j < D; ++j) width[j] = code_to_width(codes[s * D + j], w);
      uint32_t z[BLOCK_ROWS * MAX_D];
      if (column_major(D, w)) {
        for (uint32_t j = 0; j < D; ++j)
          for (uint32_t i = 0; i < BLOCK_ROWS; ++i) z[i * D + j] = (uint32_t)br_bits(&b, width[j]);
      } else {
        for (uint32_t i = 0; i < BLOCK_ROWS; ++i) {
          for (uint32_t j = 0; j < D; ++j) z[i * D + j] = (uint32_t)br_bits(&b, width[j]);
          while (b.pos & 7) br_bit(&b);
        }
      }
      for (uint32_t q = 0; q < BLOCK_ROWS * D; ++q) err[q] = spo_unzigzag(z[q], w);
      fc_decode_block(f, err, x);
      for (uint32_t i = 0; i < BLOCK_ROWS; ++i)
        for (uint32_t j = 0; j < D; ++j) put_sample(dst, blk * BLOCK_ROWS + i, j, D, w, x[i * D + j]);
      blk++;
    }
    rec += k;
    if (b.overrun) rc = SPO_ERR_CORRUPT;
  }
  if (rc == SPO_OK && (blk != n_blocks || b.pos / 8 != body_bytes || b.overrun))
    rc = SPO_ERR_CORRUPT;
  free(f);
  free(err);
  free(x);
  free(codes);
  return rc;
}

int spo_decompress(const uint8_t *src, uint64_t n, void *dst_v, uint64_t dst_cap) {
  uint8_t *dst = (uint8_t *)dst_v;
  uint64_t rows;
  uint32_t D, w;
  spo_opts o;
  int rc = spo_query(src, n, &rows, &D, &w, &o);
  if (rc != SPO_OK) return rc;
  layout L;
  make_layout(rows, &o, &L);
  uint64_t sample_bytes = (uint64_t)D * (w / 8);
  if (rows > (~0ull) / sample_bytes) return SPO_ERR_CORRUPT;
  if (dst_cap < rows * sample_bytes) return SPO_ERR_DST_TOO_SMALL;
  if (get_le(src + 20, 4) != L.n_chunks || get_le(src + 32, 4) != L.tail_rows) return SPO_ERR_CORRUPT;
  if (get_le(src + 36, 4) != 0) return SPO_ERR_CORRUPT;
  uint64_t data_off = get_le(src + 40, 8);
  uint64_t tail_off = get_le(src + 48, 8);
  uint64_t total = get_le(src + 56, 8);
  if (data_off != L.data_off || tail_off < data_off || total > n ||
      total != tail_off + L.tail_rows * sample_bytes)
    return SPO_ERR_CORRUPT;

  uint64_t data_bytes = tail_off - data_off;
  for (uint64_t c = 0; c < L.n_chunks && rc == SPO_OK; ++c) {
    const uint8_t *entry = src + HDR_BYTES + CHUNK_ENTRY_BYTES * c;
    uint64_t off = get_le(entry, 8);
    uint64_t n_records = get_le(entry + 8, 4);
    uint64_t packed = get_le(entry + 12, 4);
    uint64_t end = (c + 1 < L.n_chunks) ? get_le(entry + CHUNK_ENTRY_BYTES, 8) : data_bytes;
    if (off > end || end > data_bytes) return SPO_ERR_CORRUPT;
    uint64_t nb = chunk_blocks(&L, c);
    if (n_records < 1 || n_records > nb) return SPO_ERR_CORRUPT;
    const uint8_t *coded = src + data_off + off;
    uint64_t coded_bytes = end - off;
    uint8_t *chunk_dst = dst + c * L.chunk_rows_eff * sample_bytes;
    if (!o.huffman) {
      if (coded_bytes != packed) return SPO_ERR_CORRUPT;
      rc = decode_chunk(coded, coded_bytes, n_records, nb, D, w, &o, chunk_dst);
      continue;
    }
    /* Huffman: decode the chunk's bitstream back to its packed bytes first. */
    const uint8_t *table =
        src + HDR_BYTES + CHUNK_ENTRY_BYTES * L.n_chunks + HUFF_TABLE_BYTES * (c / o.huff_chunks);
    uint8_t len[256];
    int any = 0;
    for (uint32_t k = 0; k < 128; ++k) {
      len[2 * k] = table[k] & 15u;
      len[2 * k + 1] = table[k] >> 4;
      any |= table[k];
    }
    if (!huff_lengths_valid(len)) return SPO_ERR_CORRUPT;
    uint8_t *body = (uint8_t *)malloc(packed ? packed : 1);
    if (!any) {
      if (coded_bytes != packed) rc = SPO_ERR_CORRUPT;
      else memcpy(body, coded, packed);
    } else {
      /* the jump table, then every sub-block's code on its own */
      uint64_t n_sub = huff_n_sub(packed);
      uint64_t jump = 4 * (n_sub - 1);
      if (jump > coded_bytes) rc = SPO_ERR_CORRUPT;
      uint64_t span = rc == SPO_OK ? coded_bytes - jump : 0;
      for (uint64_t k = 0; k < n_sub && rc == SPO_OK; ++k) {
        uint64_t s0 = k == 0 ? 0 : get_le(coded + 4 * (k - 1), 4);
        uint64_t s1 = k + 1 < n_sub ? get_le(coded + 4 * k, 4) : span;
        if (s0 > s1 || s1 > span) {
          rc = SPO_ERR_CORRUPT;
          break;
        }
        bit_reader b = {coded + jump + s0, s1 - s0, 0, 0};
        uint64_t i0, i1;
        huff_sub_range(packed, k, &i0, &i1);
        for (uint64_t i = i0; i < i1 && rc == SPO_OK; ++i) {
          uint32_t sym;
          rc = huff_get(&b, len, &sym);
          body[i] = (uint8_t)sym;
        }
        if (rc == SPO_OK && (b.pos + 7) / 8 != s1 - s0) rc = SPO_ERR_CORRUPT;
      }
    }
    if (rc == SPO_OK) rc = decode_chunk(body, packed, n_records, nb, D, w, &o, chunk_dst);
    free(body);
  }
  if (rc != SPO_OK) return rc;
  memcpy(dst + L.full_rows * sample_bytes, src + tail_off, L.tail_rows * sample_bytes);
  return SPO_OK;
}

/* ------------------------------------------------------------------------ */
/* Step-level entry points for the pin tests                                */
/* ------------------------------------------------------------------------ */

int spo_forecast_errors(const void *src_v, uint64_t rows, uint32_t D, uint32_t w,
                        int32_t kind, int32_t learn_shift, int32_t test_mode,
                        int64_t pinned_alpha, int32_t *err_out) {
  const uint8_t *src = (const uint8_t *)src_v;
  if ((w != 8 && w != 16) || D < 1 || D > MAX_D || rows % BLOCK_ROWS) return SPO_ERR_INVALID_ARG;
  forecaster *f = (forecaster *)malloc(sizeof(forecaster));
  int64_t *x = (int64_t *)malloc(sizeof(int64_t) * BLOCK_ROWS * D);
  int64_t *err = (int64_t *)malloc(sizeof(int64_t) * BLOCK_ROWS * D);
  fc_init(f, kind, D, w, (uint32_t)learn_shift, test_mode, pinned_alpha);
  for (uint64_t b = 0; b < rows / BLOCK_ROWS; ++b) {
    for (uint32_t i = 0; i < BLOCK_ROWS; ++i)
      for (uint32_t j = 0; j < D; ++j) x[i * D + j] = get_sample(src, b * BLOCK_ROWS + i, j, D, w);
    fc_encode_block(f, x, err);
    for (uint32_t q = 0; q < BLOCK_ROWS * D; ++q) err_out[b * BLOCK_ROWS * D + q] = (int32_t)err[q];
  }
  free(f);
  free(x);
  free(err);
  return SPO_OK;
}

/* The inverse of spo_forecast_errors: the samples rebuilt from their errors
 * (Algorithm 2's non-run branch applied to every block). */
int spo_forecast_reconstruct(const int32_t *err_in, uint64_t rows, uint32_t D, uint32_t w,
                             int32_t kind, int32_t learn_shift, void *dst_v) {
  uint8_t *dst = (uint8_t *)dst_v;
  if ((w != 8 && w != 16) || D < 1 || D > MAX_D || rows % BLOCK_ROWS) return SPO_ERR_INVALID_ARG;
  forecaster *f = (forecaster *)malloc(sizeof(forecaster));
  int64_t *x = (int64_t *)malloc(sizeof(int64_t) * BLOCK_ROWS * D);
  int64_t *err = (int64_t *)malloc(sizeof(int64_t) * BLOCK_ROWS * D);
  fc_init(f, kind, D, w, (uint32_t)learn_shift, FIRE_NORMAL, 0);
  for (uint64_t b = 0; b < rows / BLOCK_ROWS; ++b) {
    for (uint32_t q = 0; q < BLOCK_ROWS * D; ++q) err[q] = err_in[b * BLOCK_ROWS * D + q];
    fc_decode_block(f, err, x);
    for (uint32_t i = 0; i < BLOCK_ROWS; ++i)
      for (uint32_t j = 0; j < D; ++j) put_sample(dst, b * BLOCK_ROWS + i, j, D, w, x[i * D + j]);
  }
  free(f);
  free(x);
  free(err);
  return SPO_OK;
}

/* ------------------------------------------------------------------------ */
/* Quantizing floats (Sec. 5.8)                                             */
/* ------------------------------------------------------------------------ */

static double quant_scale(double lo, double hi, uint32_t w) {
  const double range = hi - lo;
  return range > 0.0 ? (double)((1u << w) - 1u) / range : 0.0;
}

/* The inverse map's step: one code is (max - min) / (2^w - 1) in x. */
static double quant_step(double lo, double hi, uint32_t w) { return (hi - lo) / (double)((1u << w) - 1u); }

int spo_quantize(const float *src, uint64_t rows, uint32_t D, uint32_t w, void *codes, double *lo_hi) {
  if ((w != 8 && w != 16) || D < 1) return SPO_ERR_INVALID_ARG;
  uint8_t *out = (uint8_t *)codes;
  for (uint32_t j = 0; j < D; ++j) {
    /* the column's extremes */
    double lo = 0.0, hi = 0.0;
    for (uint64_t r = 0; r < rows; ++r) {
      const double v = (double)src[r * D + j];
      if (r == 0 || v < lo) lo = v;
      if (r == 0 || v > hi) hi = v;
    }
    lo_hi[2 * j] = lo;
    lo_hi[2 * j + 1] = hi;
    /* linear map of [min, max] onto [0, 2^w - 1], then floor */
    const double s = quant_scale(lo, hi, w);
    const double top = (double)((1u << w) - 1u);
    for (uint64_t r = 0; r < rows; ++r) {
      const double t = ((double)src[r * D + j] - lo) * s;
      double q = floor(t);
      if (q > top) q = top;
      if (q < 0.0) q = 0.0;
      put_sample(out, r, j, D, w, (int64_t)q);
    }
  }
  return SPO_OK;
}

int spo_dequantize(const void *codes, uint64_t rows, uint32_t D, uint32_t w, const double *lo_hi, float *dst) {
  if ((w != 8 && w != 16) || D < 1) return SPO_ERR_INVALID_ARG;
  const uint8_t *in = (const uint8_t *)codes;
  for (uint32_t j = 0; j < D; ++j) {
    const double lo = lo_hi[2 * j], h = quant_step(lo, lo_hi[2 * j + 1], w);
    for (uint64_t r = 0; r < rows; ++r) {
      const double q = (double)get_sample(in, r, j, D, w);
      dst[r * D + j] = (float)(q * h + lo);
    }
  }
  return SPO_OK;
}

int spo_quant_nmse(const float *src, const void *codes, uint64_t rows, uint32_t D, uint32_t w,
                   const double *lo_hi, double *nmse) {
  if ((w != 8 && w != 16) || D < 1 || rows == 0) return SPO_ERR_INVALID_ARG;
  const uint8_t *in = (const uint8_t *)codes;
  for (uint32_t j = 0; j < D; ++j) {
    const double lo = lo_hi[2 * j], h = quant_step(lo, lo_hi[2 * j + 1], w);
    double mean = 0.0;
    for (uint64_t r = 0; r < rows; ++r) mean += (double)src[r * D + j];
    mean /= (double)rows;
    double var = 0.0, mse = 0.0;
    for (uint64_t r = 0; r < rows; ++r) {
      const double x = (double)src[r * D + j];
      const double q = (double)get_sample(in, r, j, D, w);
      const double xh = (double)(float)(q * h + lo);
      var += (x - mean) * (x - mean);
      mse += (x - xh) * (x - xh);
    }
    nmse[j] = var > 0.0 ? mse / var : 0.0;
  }
  return SPO_OK;
}

int spo_fire_trace(const void *src_v, uint64_t rows, uint32_t D, uint32_t w,
                   int32_t learn_shift, int64_t *alpha_out, int64_t *acc_out) {
  const uint8_t *src = (const uint8_t *)src_v;
  if ((w != 8 && w != 16) || D < 1 || D > MAX_D || rows % BLOCK_ROWS) return SPO_ERR_INVALID_ARG;
  forecaster *f = (forecaster *)malloc(sizeof(forecaster));
  int64_t *x = (int64_t *)malloc(sizeof(int64_t) * BLOCK_ROWS * D);
  int64_t *err = (int64_t *)malloc(sizeof(int64_t) * BLOCK_ROWS * D);
  fc_init(f, FC_FIRE, D, w, (uint32_t)learn_shift, FIRE_NORMAL, 0);
  for (uint64_t b = 0; b < rows / BLOCK_ROWS; ++b) {
    for (uint32_t i = 0; i < BLOCK_ROWS; ++i)
      for (uint32_t j = 0; j < D; ++j) x[i * D + j] = get_sample(src, b * BLOCK_ROWS + i, j, D, w);
    fc_encode_block(f, x, err);
    for (uint32_t j = 0; j < D; ++j) {
      alpha_out[b * D + j] = f->alpha[j];
      acc_out[b * D + j] = f->acc[j];
    }
  }
  free(f);
  free(x);
  free(err);
  return SPO_OK;
}
