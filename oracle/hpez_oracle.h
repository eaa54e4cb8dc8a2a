/*
 * hpez_oracle.h -- plain single-threaded CPU oracle of HPEZ (arXiv 2311.12133).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path; the two meet only through the
 * compressed byte stream, whose layout each side writes independently.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math (strict IEEE
 * binary32: one correctly rounded operation per source operator, no FMA).
 */
#ifndef HPEZ_ORACLE_H
#define HPEZ_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORA_MAX_LEVELS 16
#define ORA_RADIUS 32768
#define ORA_HEADER_BYTES 512

/* interpolator kinds (Sec. 5.2): Eq. 2 linear, Eq. 4 not-a-knot cubic,
 * Eq. 6 natural cubic; and, opt in, the natural cubic spline through every
 * known point of the line (a global spline, solved per line; 1D-style
 * paradigm only, without same-level halves or a block map) */
enum { ORA_LINEAR = 0, ORA_CUBIC_NAK = 1, ORA_CUBIC_NAT = 2, ORA_SPLINE_GLOBAL = 3 };
/* paradigms (Sec. 5.3): 1D-style (one direction per pass) or
 * multi-dimensional (Eq. 8) */
enum { ORA_1D = 0, ORA_MD = 1 };
enum { ORA_EB_ABS = 0, ORA_EB_REL = 1 };

enum {
  ORA_OK = 0,
  ORA_ERR_INVALID_ARG = -1,
  ORA_ERR_NONFINITE = -2,
  ORA_ERR_OUT_TOO_SMALL = -3,
  ORA_ERR_CORRUPT = -4,
  ORA_ERR_NO_MEMORY = -5,
  ORA_ERR_SELFCHECK = -6
};

typedef struct {
  int32_t anchor_stride; /* A: power of two in [2, 32768] (Sec. 5.1) */
  int32_t frozen_dim;    /* -1 or the frozen dimension (Sec. 6.3) */
  int32_t chunk_syms;    /* Huffman chunk length, power of two in [256, 32768] */
  int32_t blockwise;     /* 1: per-block interpolator from blockmap (Sec. 6.6) */
  int32_t block_size;    /* block side for the block map (Sec. 6.6: 32) */
  int32_t predictor;     /* 0 interpolation; 1, 2: Lorenzo of that order
                            on blocks of side anchor_stride (Sec. 6.5) */
  double alpha, beta;    /* Eq. 15 */
  double md_inv_var[3];  /* 1/sigma_i^2 per dimension for Eq. 14 weights */
  uint8_t interp[ORA_MAX_LEVELS];     /* per level l (index l-1) */
  uint8_t paradigm[ORA_MAX_LEVELS];
  uint8_t same_level[ORA_MAX_LEVELS]; /* Sec. 5.4.2, cubic only */
  uint8_t order[ORA_MAX_LEVELS][3];   /* 1D-style dimension order */
  const uint8_t* blockmap; /* per block: bits0-1 interp kind, bit2 same-level */
} ora_config;

/* Statistics of the last compress call (diagnostics for the tests). */
typedef struct {
  uint64_t n_points, n_anchors, n_outliers, n_used, total_words, n_chunks;
  uint64_t predicted;    /* points predicted by the level sweep */
  uint64_t bad_reads;    /* neighbour reads of points not known before the sub-pass */
  uint64_t double_visits;/* points predicted more than once */
  uint64_t sum_len_bits; /* sum over symbols of the Huffman code length */
  float e;               /* absolute error bound in use */
  float vmin, vmax;
} ora_stats;

uint64_t ora_compress_bound(int ndim, const uint64_t* dims);

/* Compress x (row-major, dims slowest first).  eb_mode 0 = absolute error
 * bound eb, 1 = value-range relative (e = eb * (max - min), Sec. 7.1.3).
 * cfg == NULL uses ora_default_config(ndim).  codes_out (N entries) and
 * recon_out (N entries) are optional.  Returns 0 or a negative ORA_ERR_*. */
int ora_compress(const float* x, int ndim, const uint64_t* dims, int eb_mode,
                 double eb, const ora_config* cfg, uint8_t* out, uint64_t cap,
                 uint64_t* out_size, uint16_t* codes_out, float* recon_out,
                 ora_stats* stats);

/* Decompress a stream into out (cap_elems floats). */
int ora_decompress(const uint8_t* in, uint64_t size, float* out,
                   uint64_t cap_elems);

/* Read ndim/dims/abs eb from a header. */
int ora_inspect(const uint8_t* in, uint64_t size, int* ndim, uint64_t* dims,
                double* abs_eb);

void ora_default_config(int ndim, ora_config* cfg);

/* ---- building blocks exposed for the pin tests ---- */

/* Prediction of line[pos] along a 1D line of n values spaced 1 apart with
 * stride s (neighbours at pos +- s, +-2s, +-3s).  half_b selects the
 * same-level formula (Eq. 10 / Eq. 11). */
float ora_predict_1d(int kind, int half_b, const float* line, uint64_t n,
                     uint64_t pos, uint64_t s);

/* Linear quantization of x against prediction p (Sec. 4 Step 3). */
uint16_t ora_quantize(float x, float p, float el, float inv2, float twoe,
                      float* recon);

/* Level error bounds (Eq. 15) and the derived quantizer constants. */
int ora_level_params(float e, double alpha, double beta, int L, float* el,
                     float* inv2, float* twoe);

/* Huffman code lengths by the two-queue merge and canonical codes. */
int ora_huffman_lengths(const uint64_t* freq, int nsym, uint8_t* lens);
int ora_canonical_codes(const uint8_t* lens, int nsym, uint64_t* codes);

/* ---- auto-tuning (Sec. 6) ---- */
typedef struct {
  double sample_rate;   /* statistics lattice density (Sec. 6.1: 0.2 %) */
  double block_rate;    /* global tuning: sampled volume fraction (1 %) */
  double sub_frac;      /* block-wise tuning: sub-block fraction (4 %) */
  double lorenzo_coef;  /* multiplier of the Lorenzo bit estimate */
  int32_t block_size;   /* block-wise tuning block side (Sec. 6.6: 32) */
  int32_t tune_levels, tune_eb, tune_freeze, tune_lorenzo, tune_blockwise;
  int32_t allow_natural, allow_same_level;
  int32_t anchor_stride; /* 0: default for ndim */
} ora_tune_params;

typedef struct {
  uint64_t stats_count, mse_lin[3], mse_cub[3]; /* fixed-point sums */
  int32_t nonsmooth_dim, froze, lorenzo_better;
  uint32_t n_sample_blocks;
  uint64_t bits[2];          /* sample estimate without / with freezing */
  uint64_t lorenzo_bits[2];  /* order 1, order 2 */
  uint8_t level_choice[2][ORA_MAX_LEVELS];
  uint64_t level_score[2][ORA_MAX_LEVELS];
} ora_tune_report;

void ora_default_tune_params(ora_tune_params* t);
/* Candidate j of the per-level global tuning; returns 0 past the end. */
int ora_tune_candidate(const ora_tune_params* tp, int ndim, int frozen, int j,
                       int* kind, int* paradigm, uint8_t order[3], int* same);
/* Compression test on a sub-field: anchors, then levels L .. l_stop with
 * config c and absolute bound e.  Adds the per-level error scores, the code
 * histogram (65536 bins), the escapes and the anchors to the non-NULL
 * accumulators. */
int ora_subfield_test(const float* xs, int ndim, const uint64_t* ds,
                      const ora_config* c, float e, int l_stop,
                      uint64_t* score, uint64_t* hist, uint64_t* nout,
                      uint64_t* n_anchors);
uint64_t ora_blockmap_size(int ndim, const uint64_t* dims, int block_size);
/* Tunes theta for x; out->blockmap points at `blockmap` when the block-wise
 * map is produced.  Returns 0 or a negative ORA_ERR_*. */
int ora_tune(const float* x, int ndim, const uint64_t* dims, int eb_mode,
             double eb, const ora_tune_params* tp, ora_config* out,
             uint8_t* blockmap, uint64_t blockmap_cap, ora_tune_report* rep);

/* MD weight of dimension d within the odd-dimension set `mask` (Eq. 14). */
float ora_md_weight(const double* inv_var, unsigned mask, int d);

/* ---- the quality-metric target (Sec. 3.1, Eq. 1) and integer inputs ---- */

/* PSNR of y against x (Sec. 7.1.3): 20 log10(max x - min x) - 10 log10(MSE).
 * The squared errors are summed exactly in the fixed-point unit `unit`:
 * q_i = rint((x_i - y_i) / unit) in double, sse = sum q_i^2 (64-bit
 * integer), MSE = sse unit^2 / n; +inf when sse = 0.  The caller keeps
 * |x_i - y_i| / unit <= 2^16 (unit = e / 2^16 for a bound e) and x finite. */
int ora_psnr(const float* x, const float* y, uint64_t n, double unit,
             double* psnr, uint64_t* sse);

/* Eq. 1 with M = PSNR and target m0 = target_db: the largest absolute bound
 * the search below finds whose auto-tuned round trip keeps PSNR >= m0
 * (the compression ratio grows with the bound).  The search, in double:
 * e_u = range sqrt(3) 10^(-m0/20) (uniform errors on [-e, e] give exactly
 * m0); from e_u, double (or halve) up to 6 times to bracket the target;
 * then 8 geometric bisection steps e = sqrt(lo hi), keeping PSNR(lo) >= m0.
 * Each probe is ora_tune + ora_compress (absolute bound e) + ora_decompress
 * + ora_psnr with unit = (float)e / 2^16.  Writes the stream of the final
 * bound, the bound (eb_out) and its PSNR.  x must be finite. */
int ora_compress_psnr(const float* x, int ndim, const uint64_t* dims,
                      double target_db, const ora_tune_params* tp, uint8_t* out,
                      uint64_t cap, uint64_t* out_size, double* eb_out,
                      double* psnr_out);

/* Integer inputs (the integer datasets of Sec. 7): int16, uint16 or int32
 * values (|v| <= 2^24) are widened to binary32 exactly and compressed with
 * the absolute bound just below floor(e) + 1/2, e the requested bound (REL:
 * eb (max - min)); decompression rounds to the nearest integer (ties to
 * even) and clamps to the type's range, so every integer stays within
 * floor(e) of its input (lossless when e < 1).  The stream records the type
 * at header byte ORA_H_DTYPE.  tune = 1: auto-tuned (ora_tune), else cfg
 * (NULL: default). */
enum { ORA_DTYPE_F32 = 0, ORA_DTYPE_I16 = 1, ORA_DTYPE_U16 = 2, ORA_DTYPE_I32 = 3 };
#define ORA_H_DTYPE 320
int ora_compress_typed(const void* x, int dtype, int ndim, const uint64_t* dims,
                       int eb_mode, double eb, const ora_config* cfg, int tune,
                       const ora_tune_params* tp, uint8_t* out, uint64_t cap,
                       uint64_t* out_size);
/* Decompress an integer (or float) stream into out (cap_elems values of
 * dtype, which must match the stream's). */
int ora_decompress_typed(const uint8_t* in, uint64_t size, void* out, int dtype,
                         uint64_t cap_elems);

/* ---- the lossless stage after Huffman (Sec. 4, Step 5) ----
 * Read as run suppression of repeated 32-bit words over the stream body
 * (the bytes after the 512-byte header, zero-padded to whole words): in
 * every block of 32 words a mask marks the words that differ from the word
 * before them (the word before the first is 0), and only those words are
 * kept; a second mask per group of 32 blocks marks the blocks whose mask is
 * not 0, and only those masks are kept.  The result: the header with flag
 * bit 2 and the raw size at byte ORA_H_RAWSIZE, then the counts (words,
 * literals, masks, 0 as four u64), the group masks, the kept block masks and
 * the kept words.  When that is not smaller than the input, the input is
 * returned unchanged.  ora_decompress accepts either form. */
#define ORA_H_RAWSIZE 328
int ora_lossless_encode(const uint8_t* in, uint64_t size, uint8_t* out, uint64_t cap,
                        uint64_t* out_size);
int ora_lossless_decode(const uint8_t* in, uint64_t size, uint8_t* out, uint64_t cap,
                        uint64_t* out_size);

#ifdef __cplusplus
}
#endif
#endif
