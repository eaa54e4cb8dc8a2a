/*
 * hpez_oracle.c -- plain, slow, single-threaded CPU oracle of the HPEZ
 * interpolation predict-and-quantize path (arXiv 2311.12133).
 *
 * TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
 * benchmark's CPU-baseline leg may call it.  It shares no code with the CUDA
 * path; the two agree only on the compressed stream layout, which each side
 * writes on its own.
 *
 * What it follows, step by step:
 *   Sec. 4 (Steps 2-4)     prediction, linear quantization, Huffman coding
 *   Sec. 5.1               anchor grid + level-wise interpolation, strides
 *                          A/2 .. 1, the grid doubling at every level
 *   Sec. 5.2 Eq. 2, 4, 6   linear, not-a-knot cubic, natural cubic stencils
 *   Sec. 5.3 Eq. 8, 14     multi-dimensional interpolation, weights
 *                          alpha_i proportional to 1/sigma_i^2
 *   Sec. 5.4.2 Eq. 10, 11  same-level cubic interpolation (two halves)
 *   Sec. 6.1-6.6           the auto-tuner (statistics, per-level tests,
 *                          (alpha, beta), freezing, Lorenzo test, block map)
 *   Sec. 6.3               dimension freezing (anchor stride 1 on one dim)
 *   Sec. 6.4 Eq. 15        level error bounds e_l = e / min(alpha^(l-1), beta)
 *   Sec. 6.5               the full-field dynamic-order Lorenzo predictor,
 *                          read as block-local (blocks of side A)
 *   Sec. 6.6               block-wise interpolator choice (block map)
 *   Sec. 7.1.3             value-range relative bound e = eps * (max - min)
 * and, opt in beside Eq. 6, the natural cubic spline through every known
 * point of a pass line (a global spline, Thomas algorithm per line).
 *
 * Readings where the paper is silent (each listed in the design notes):
 * boundary fallbacks of the stencils, the quantizer's exact rounding steps,
 * the outlier escape (code 0), the canonical Huffman tie-breaks and the
 * chunked bit layout, and the stream container.
 *
 * Every binary32 operation below is one correctly rounded IEEE operation in
 * the order written (compiled with -ffp-contract=off, no fast-math).
 */
#include "hpez_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* little-endian byte access                                           */
/* ------------------------------------------------------------------ */
static void put_u8(uint8_t* b, uint64_t o, uint8_t v) { b[o] = v; }
static void put_u16(uint8_t* b, uint64_t o, uint16_t v) {
  b[o] = (uint8_t)(v & 0xff);
  b[o + 1] = (uint8_t)(v >> 8);
}
static void put_u32(uint8_t* b, uint64_t o, uint32_t v) {
  for (int i = 0; i < 4; ++i) b[o + i] = (uint8_t)(v >> (8 * i));
}
static void put_u64(uint8_t* b, uint64_t o, uint64_t v) {
  for (int i = 0; i < 8; ++i) b[o + i] = (uint8_t)(v >> (8 * i));
}
static void put_f32(uint8_t* b, uint64_t o, float v) {
  uint32_t u;
  memcpy(&u, &v, 4);
  put_u32(b, o, u);
}
static void put_f64(uint8_t* b, uint64_t o, double v) {
  uint64_t u;
  memcpy(&u, &v, 8);
  put_u64(b, o, u);
}
static uint16_t get_u16(const uint8_t* b, uint64_t o) {
  return (uint16_t)(b[o] | ((uint16_t)b[o + 1] << 8));
}
static uint32_t get_u32(const uint8_t* b, uint64_t o) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= (uint32_t)b[o + i] << (8 * i);
  return v;
}
static uint64_t get_u64(const uint8_t* b, uint64_t o) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= (uint64_t)b[o + i] << (8 * i);
  return v;
}
static float get_f32(const uint8_t* b, uint64_t o) {
  uint32_t u = get_u32(b, o);
  float v;
  memcpy(&v, &u, 4);
  return v;
}
static double get_f64(const uint8_t* b, uint64_t o) {
  uint64_t u = get_u64(b, o);
  double v;
  memcpy(&v, &u, 8);
  return v;
}
static uint64_t align16(uint64_t v) { return (v + 15) & ~(uint64_t)15; }

/* ------------------------------------------------------------------ */
/* stream container layout (byte offsets inside the 512-byte header)   */
/* ------------------------------------------------------------------ */
#define H_MAGIC 0
#define H_VERSION 4
#define H_FLAGS 8
#define H_NDIM 12
#define H_DIMS 16
#define H_EBMODE 40
#define H_ANCHOR 44
#define H_EBVALUE 48
#define H_E 56
#define H_CONST 60
#define H_FROZEN 64
#define H_CHUNK 68
#define H_ALPHA 72
#define H_BETA 80
#define H_MDIV 88
#define H_INTERP 112
#define H_PARADIGM 128
#define H_SAME 144
#define H_ORDER 160
#define H_PREDICTOR 208
#define H_BLOCKWISE 212
#define H_NANCHORS 216
#define H_NOUTLIERS 224
#define H_NUSED 232
#define H_BLOCKSIZE 236
#define H_NCHUNKS 240
#define H_TOTALWORDS 248
#define H_OFF_ANCHORS 256
#define H_OFF_CHUNKW 264
#define H_OFF_TABLE 272
#define H_OFF_OUTLIERS 280
#define H_OFF_BITS 288
#define H_OFF_BLOCKMAP 296
#define H_TOTAL 304
#define H_NBLOCKS 312
#define MAGIC 0x5A455048u /* "HPEZ" */
#define VERSION 1u
#define FLAG_CONST 1u
#define FLAG_LOSSLESS 2u

/* ------------------------------------------------------------------ */
/* field geometry: every field is held as 3 slots, the real dimensions  */
/* in the last ndim slots; padded slots have extent 1 and are never     */
/* interpolated.                                                        */
/* ------------------------------------------------------------------ */
typedef struct {
  int ndim, off;
  uint64_t n[3], st[3], N;
  int interp[3];
  int k, A, L;
} geom;

static int ilog2(uint64_t v) {
  int l = 0;
  while (((uint64_t)1 << l) < v) ++l;
  return l;
}
static int is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

static int geom_init(geom* g, int ndim, const uint64_t* dims, int A,
                     int frozen) {
  if (ndim < 1 || ndim > 3) return ORA_ERR_INVALID_ARG;
  if (frozen < -1 || frozen >= ndim || (ndim == 1 && frozen != -1))
    return ORA_ERR_INVALID_ARG;
  if (!is_pow2(A) || A < 2 || A > 32768) return ORA_ERR_INVALID_ARG;
  g->ndim = ndim;
  g->off = 3 - ndim;
  g->N = 1;
  for (int s = 0; s < 3; ++s) {
    g->n[s] = 1;
    g->interp[s] = 0;
  }
  for (int d = 0; d < ndim; ++d) {
    if (dims[d] == 0) return ORA_ERR_INVALID_ARG;
    g->n[d + g->off] = dims[d];
    g->interp[d + g->off] = (d != frozen);
    g->N *= dims[d];
    if (g->N > 0xFFFFFFFFull) return ORA_ERR_INVALID_ARG;
  }
  g->st[2] = 1;
  g->st[1] = g->n[2];
  g->st[0] = g->n[1] * g->n[2];
  g->k = 0;
  for (int s = 0; s < 3; ++s) g->k += g->interp[s];
  g->A = A;
  g->L = ilog2((uint64_t)A);
  return ORA_OK;
}

void ora_default_config(int ndim, ora_config* c) {
  memset(c, 0, sizeof(*c));
  c->anchor_stride = ndim == 1 ? 128 : (ndim == 2 ? 64 : 32);
  c->frozen_dim = -1;
  c->chunk_syms = 16384;
  c->blockwise = 0;
  c->block_size = 32;
  c->alpha = 1.0;
  c->beta = 1.0;
  for (int d = 0; d < 3; ++d) c->md_inv_var[d] = 1.0;
  for (int l = 0; l < ORA_MAX_LEVELS; ++l) {
    c->interp[l] = ORA_CUBIC_NAK;
    c->paradigm[l] = ORA_1D;
    c->same_level[l] = 0;
    for (int j = 0; j < 3; ++j) c->order[l][j] = (uint8_t)(j < ndim ? j : 255);
  }
  c->blockmap = NULL;
}

/* Checks a config against the field shape; fills the per-level 1D-style
 * order as slots.  Returns 0 or ORA_ERR_INVALID_ARG. */
static int check_config(const geom* g, const ora_config* c) {
  if (!is_pow2(c->chunk_syms) || c->chunk_syms < 256 || c->chunk_syms > 32768)
    return ORA_ERR_INVALID_ARG;
  if (!(c->alpha >= 1.0) || !(c->beta >= 1.0) || !isfinite(c->alpha) ||
      !isfinite(c->beta))
    return ORA_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d)
    if (!(c->md_inv_var[d] > 0.0) || !isfinite(c->md_inv_var[d]))
      return ORA_ERR_INVALID_ARG;
  if (c->blockwise) {
    if (!c->blockmap || c->block_size < 1) return ORA_ERR_INVALID_ARG;
  }
  if (c->predictor < 0 || c->predictor > 2 || (c->predictor && c->blockwise))
    return ORA_ERR_INVALID_ARG;
  for (int l = 0; l < g->L; ++l) {
    if (c->interp[l] > ORA_SPLINE_GLOBAL || c->paradigm[l] > ORA_MD ||
        c->same_level[l] > 1)
      return ORA_ERR_INVALID_ARG;
    /* the global spline runs along whole lines: one direction per pass */
    if (c->interp[l] == ORA_SPLINE_GLOBAL &&
        (c->paradigm[l] != ORA_1D || c->same_level[l] || c->blockwise))
      return ORA_ERR_INVALID_ARG;
    /* the 1D-style order lists each interpolation dimension exactly once */
    int seen[3] = {0, 0, 0};
    for (int j = 0; j < g->k; ++j) {
      int d = c->order[l][j];
      if (d >= g->ndim || !g->interp[d + g->off] || seen[d])
        return ORA_ERR_INVALID_ARG;
      seen[d] = 1;
    }
  }
  return ORA_OK;
}

/* ------------------------------------------------------------------ */
/* Eq. 15 level error bounds + quantizer constants                     */
/* ------------------------------------------------------------------ */
int ora_level_params(float e, double alpha, double beta, int L, float* el,
                     float* inv2, float* twoe) {
  for (int l = 1; l <= L; ++l) {
    double ap = 1.0; /* alpha^(l-1) by repeated multiplication */
    for (int i = 1; i < l; ++i) ap = ap * alpha;
    double m = ap < beta ? ap : beta;
    float e_l = (float)((double)e / m);
    if (!(e_l > 0.0f) || !isfinite(e_l)) return ORA_ERR_INVALID_ARG;
    float t = 2.0f * e_l;
    if (!isfinite(t)) return ORA_ERR_INVALID_ARG;
    el[l - 1] = e_l;
    twoe[l - 1] = t;
    inv2[l - 1] = (float)(1.0 / (2.0 * (double)e_l));
  }
  return ORA_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 5.2 / 5.4.2 stencils along one line                            */
/* ------------------------------------------------------------------ */
/* formula ids, chosen from which neighbours exist */
enum {
  F_COPY, F_EXTRAP, F_LIN, F_NAK4, F_NAT4, F_NAK3L, F_NAK3R, F_NAT3L,
  F_NAT3R, F_SL_NAK, F_SL_NAT
};

/* have[j+3]: neighbour at offset j*s lies inside the line (j = -3..3).
 * The offset -1 neighbour always exists (the point is at an odd multiple
 * of s >= s). */
static int choose_formula(int kind, int half_b, const int have[7]) {
  const int hm3 = have[0], hm2 = have[1], hp1 = have[4], hp2 = have[5],
            hp3 = have[6];
  if (half_b) {
    /* Eq. 10 (as printed: neighbours +-s, +-2s) and Eq. 11 */
    if (kind == ORA_CUBIC_NAK && hp1 && hm2 && hp2) return F_SL_NAK;
    if (kind == ORA_CUBIC_NAT && hp1 && hm2 && hp2 && hm3 && hp3)
      return F_SL_NAT;
  }
  if (!hp1) return hm3 ? F_EXTRAP : F_COPY;
  if (kind == ORA_LINEAR) return F_LIN;
  if (hm3 && hp3) return kind == ORA_CUBIC_NAK ? F_NAK4 : F_NAT4;
  if (hm3) return kind == ORA_CUBIC_NAK ? F_NAK3L : F_NAT3L;
  if (hp3) return kind == ORA_CUBIC_NAK ? F_NAK3R : F_NAT3R;
  return F_LIN;
}

/* which offsets (-3..3 -> bit j+3) a formula reads */
static unsigned formula_reads(int f) {
  switch (f) {
    case F_COPY: return 1u << 2;
    case F_EXTRAP: return (1u << 0) | (1u << 2);
    case F_LIN: return (1u << 2) | (1u << 4);
    case F_NAK4: case F_NAT4: return (1u << 0) | (1u << 2) | (1u << 4) | (1u << 6);
    case F_NAK3L: case F_NAT3L: return (1u << 0) | (1u << 2) | (1u << 4);
    case F_NAK3R: case F_NAT3R: return (1u << 2) | (1u << 4) | (1u << 6);
    case F_SL_NAK: return (1u << 1) | (1u << 2) | (1u << 4) | (1u << 5);
    case F_SL_NAT: return 0x77u; /* all but the centre */
  }
  return 0;
}

/* v[j+3] = neighbour value at offset j*s (only the ones read are set) */
static float eval_formula(int f, const float v[7]) {
  const float m3 = v[0], m2 = v[1], m1 = v[2], p1 = v[4], p2 = v[5],
              p3 = v[6];
  switch (f) {
    case F_COPY: /* no right neighbour and no d-3: repeat d-1 */
      return m1;
    case F_EXTRAP: /* line through d-3, d-1 evaluated at 0 */
      return (m1 * 3.0f - m3) / 2.0f;
    case F_LIN: /* Eq. 2 */
      return (m1 + p1) * 0.5f;
    case F_NAK4: /* Eq. 4: (-1, 9, 9, -1) / 16 */
      return ((m1 + p1) * 9.0f - (m3 + p3)) / 16.0f;
    case F_NAT4: /* Eq. 6: (-3, 23, 23, -3) / 40 */
      return ((m1 + p1) * 23.0f - (m3 + p3) * 3.0f) / 40.0f;
    case F_NAK3L: /* quadratic through d-3, d-1, d+1: (-1, 6, 3) / 8 */
      return ((m1 * 6.0f + p1 * 3.0f) - m3) / 8.0f;
    case F_NAK3R: /* mirror: (3, 6, -1) / 8 on d-1, d+1, d+3 */
      return ((m1 * 3.0f + p1 * 6.0f) - p3) / 8.0f;
    case F_NAT3L: /* natural spline on knots -3, -1, 1: (-3, 22, 13) / 32 */
      return ((m1 * 22.0f + p1 * 13.0f) - m3 * 3.0f) / 32.0f;
    case F_NAT3R: /* mirror: (13, 22, -3) / 32 on d-1, d+1, d+3 */
      return ((m1 * 13.0f + p1 * 22.0f) - p3 * 3.0f) / 32.0f;
    case F_SL_NAK: /* Eq. 10: (-1, 4, 4, -1) / 6 on d-2, d-1, d+1, d+2 */
      return ((m1 + p1) * 4.0f - (m2 + p2)) / 6.0f;
    case F_SL_NAT: /* Eq. 11: (3, -18, 46, 46, -18, 3) / 62 */
      return (((m1 + p1) * 46.0f - (m2 + p2) * 18.0f) + (m3 + p3) * 3.0f) /
             62.0f;
  }
  return 0.0f;
}

static void line_have(uint64_t c, uint64_t n, uint64_t s, int have[7]) {
  for (int j = -3; j <= 3; ++j) {
    if (j == 0) {
      have[3] = 1;
      continue;
    }
    uint64_t a = (uint64_t)(j < 0 ? -j : j) * s;
    have[j + 3] = j < 0 ? (c >= a) : (c + a <= n - 1);
  }
}

float ora_predict_1d(int kind, int half_b, const float* line, uint64_t n,
                     uint64_t pos, uint64_t s) {
  int have[7];
  float v[7] = {0, 0, 0, 0, 0, 0, 0};
  line_have(pos, n, s, have);
  int f = choose_formula(kind, half_b, have);
  unsigned rd = formula_reads(f);
  for (int j = 0; j < 7; ++j)
    if (rd & (1u << j)) v[j] = line[pos + (uint64_t)(j - 3) * s];
  return eval_formula(f, v);
}

/* ------------------------------------------------------------------ */
/* Sec. 4 Step 3: linear quantization with an exact bound check        */
/* ------------------------------------------------------------------ */
/* |r - x| <= e decided exactly: d = rn(r - x) plus its TwoSum residual. */
static int within_bound(float r, float x, float e) {
  float nx = -x;
  float d = r + nx;
  float bb = d - r;
  float res = (r - (d - bb)) + (nx - bb);
  float ad = fabsf(d);
  if (ad < e) return 1;
  if (ad == e) {
    if (d > 0.0f) return res <= 0.0f;
    if (d < 0.0f) return res >= 0.0f;
  }
  return 0; /* also NaN */
}

uint16_t ora_quantize(float x, float p, float el, float inv2, float twoe,
                      float* recon) {
  float diff = x - p;
  float m = fabsf(diff) * inv2 + 0.5f;
  if (m < 32768.0f) { /* false for NaN */
    int k = (int)m;
    int q = diff < 0.0f ? -k : k;
    float r = p + (float)q * twoe;
    if (within_bound(r, x, el)) {
      *recon = r;
      return (uint16_t)(q + ORA_RADIUS);
    }
  }
  *recon = x; /* unpredictable: stored verbatim in the outlier list */
  return 0;
}

/* ------------------------------------------------------------------ */
/* Eq. 14 weights                                                      */
/* ------------------------------------------------------------------ */
float ora_md_weight(const double* inv_var, unsigned mask, int d) {
  double sum = 0.0;
  for (int j = 0; j < 3; ++j)
    if (mask & (1u << j)) sum = sum + inv_var[j];
  return (float)(inv_var[d] / sum);
}

/* ------------------------------------------------------------------ */
/* the level-wise sweep                                                */
/* ------------------------------------------------------------------ */
typedef struct {
  const geom* g;
  const ora_config* c;
  const float* x;      /* compress: input; decompress: NULL */
  float* recon;        /* N */
  uint16_t* codes;     /* N */
  uint32_t* stamp;     /* N: 0 unknown, else the sub-pass that set it */
  uint32_t cur;        /* current sub-pass stamp */
  float el[ORA_MAX_LEVELS], inv2[ORA_MAX_LEVELS], twoe[ORA_MAX_LEVELS];
  uint64_t bad_reads, double_visits, predicted;
  int decompress;
  uint64_t nb[3];      /* blocks per real dim (block map) */
  /* tuning hooks (compress only; NULL when unused) */
  uint64_t* score;     /* [level]: sum of fixed-point |x - p| / e_l */
  uint64_t* chist;     /* [65536]: codes of predicted points */
  uint64_t nout;       /* escapes among predicted points */
} sweep;

/* Fixed-point error measure of the tuner: |d| * (1/e_l) in binary32 (the
 * reciprocal rounded once from double), capped at 2^24 - 1, in units of
 * 1/256 (exact scaling), floored: a 32-bit value per point.  Integer sums
 * of it do not depend on the summation order. */
static uint64_t err_fixed(float d, float inv_el) {
  float v = fabsf(d) * inv_el;
  v = fminf(v, 16777215.0f);
  return (uint64_t)(uint32_t)floorf(v * 256.0f);
}

static float load_known(sweep* w, uint64_t idx) {
  uint32_t st = w->stamp[idx];
  if (st == 0 || st >= w->cur) w->bad_reads++;
  return w->recon[idx];
}

/* per-point interpolator kind and same-level flag */
static void point_cfg(const sweep* w, int l, const uint64_t c[3], int* kind,
                      int* same) {
  const geom* g = w->g;
  if (w->c->blockwise) {
    uint64_t b = 0;
    for (int d = 0; d < g->ndim; ++d) {
      uint64_t bd = c[d + g->off] / (uint64_t)w->c->block_size;
      b = b * w->nb[d] + bd;
    }
    uint8_t v = w->c->blockmap[b];
    *kind = v & 3;
    *same = (v >> 2) & 1;
    if (*kind > ORA_CUBIC_NAT) *kind = ORA_CUBIC_NAT;
  } else {
    *kind = w->c->interp[l - 1];
    *same = w->c->same_level[l - 1];
  }
  if (*kind == ORA_LINEAR) *same = 0;
}

/* prediction along slot d for the point at linear index i */
static float predict_dim(sweep* w, uint64_t i, const uint64_t c[3], int d,
                         uint64_t s, int kind, int half_b) {
  const geom* g = w->g;
  int have[7];
  float v[7] = {0, 0, 0, 0, 0, 0, 0};
  line_have(c[d], g->n[d], s, have);
  int f = choose_formula(kind, half_b, have);
  unsigned rd = formula_reads(f);
  for (int j = 0; j < 7; ++j) {
    if (!(rd & (1u << j))) continue;
    int64_t o = (int64_t)(j - 3) * (int64_t)s * (int64_t)g->st[d];
    v[j] = load_known(w, (uint64_t)((int64_t)i + o));
  }
  return eval_formula(f, v);
}

/* The natural cubic spline through every known point of the line along
 * slot d (the knots at the multiples of h = 2s), evaluated halfway between
 * the two knots around the point.  With N_k = h^2 M_k / 6 (M: the spline's
 * second derivative at knot k) its conditions read
 *   N_{k-1} + 4 N_k + N_{k+1} = y_{k-1} - 2 y_k + y_{k+1},  k = 1..K-1,
 *   N_0 = N_K = 0 (natural ends),
 * and halfway between knots j and j+1 the cubic piece is
 *   (y_j + y_{j+1}) / 2 - 3/8 (N_j + N_{j+1}).
 * The system is solved by the Thomas algorithm: c'_1 = 1/4, c'_k =
 * 1 / (4 - c'_{k-1}); D_1 = r_1 c'_1, D_k = (r_k - D_{k-1}) c'_k;
 * N_{K-1} = D_{K-1}, N_k = D_k - c'_k N_{k+1}.  Everything in binary32 in
 * the order written.  A point with no knot to its right takes the
 * boundary rule of the other interpolators. */
static float spline_global(sweep* w, uint64_t i, const uint64_t c[3], int d, uint64_t s) {
  const geom* g = w->g;
  const uint64_t h = 2 * s;
  const uint64_t K = (g->n[d] - 1) / h; /* knots 0..K at k h */
  const uint64_t j = (c[d] - s) / h;    /* between knots j and j + 1 */
  if (j + 1 > K) return predict_dim(w, i, c, d, s, ORA_LINEAR, 0);
  float* y = (float*)malloc(sizeof(float) * (K + 1));
  float* cp = (float*)calloc(K + 1, sizeof(float));
  float* D = (float*)calloc(K + 1, sizeof(float));
  float* N = (float*)calloc(K + 1, sizeof(float));
  const uint64_t line0 = i - c[d] * g->st[d];
  for (uint64_t k = 0; k <= K; ++k) y[k] = load_known(w, line0 + k * h * g->st[d]);
  if (K >= 2) {
    for (uint64_t k = 1; k <= K - 1; ++k) {
      const float r = (y[k - 1] + y[k + 1]) - 2.0f * y[k];
      if (k == 1) {
        cp[k] = 0.25f;
        D[k] = r * cp[k];
      } else {
        cp[k] = 1.0f / (4.0f - cp[k - 1]);
        D[k] = (r - D[k - 1]) * cp[k];
      }
    }
    N[K - 1] = D[K - 1];
    for (uint64_t k = K - 2; k >= 1; --k) N[k] = D[k] - cp[k] * N[k + 1];
  }
  const float p = (y[j] + y[j + 1]) * 0.5f - 0.375f * (N[j] + N[j + 1]);
  free(y);
  free(cp);
  free(D);
  free(N);
  return p;
}

static void process_point(sweep* w, int l, uint64_t i, const uint64_t c[3],
                          int md, int pass_slot, unsigned odd_mask,
                          int half_b, int kind) {
  const geom* g = w->g;
  uint64_t s = (uint64_t)1 << (l - 1);
  float p;
  if (!md) {
    p = kind == ORA_SPLINE_GLOBAL ? spline_global(w, i, c, pass_slot, s)
                                  : predict_dim(w, i, c, pass_slot, s, kind, half_b);
  } else {
    /* Eq. 8: weighted sum over all odd dimensions, ascending, with the
     * Eq. 14 weights of this odd-dimension set */
    unsigned real_mask = 0;
    for (int d = 0; d < 3; ++d)
      if (odd_mask & (1u << d)) real_mask |= 1u << (d - g->off);
    float acc = 0.0f;
    int first = 1;
    for (int d = 0; d < 3; ++d) {
      if (!(odd_mask & (1u << d))) continue;
      float pd = predict_dim(w, i, c, d, s, kind, half_b);
      float wd = ora_md_weight(w->c->md_inv_var, real_mask, d - g->off);
      float t = wd * pd;
      if (first) {
        acc = t;
        first = 0;
      } else {
        acc = acc + t;
      }
    }
    p = acc;
  }
  if (w->stamp[i] != 0) w->double_visits++;
  w->predicted++;
  if (!w->decompress) {
    float r;
    w->codes[i] = ora_quantize(w->x[i], p, w->el[l - 1], w->inv2[l - 1],
                               w->twoe[l - 1], &r);
    w->recon[i] = r;
    if (w->score)
      w->score[l - 1] +=
          err_fixed(w->x[i] - p, (float)(1.0 / (double)w->el[l - 1]));
    if (w->chist) w->chist[w->codes[i]]++;
    if (w->codes[i] == 0) w->nout++;
  } else {
    uint16_t code = w->codes[i];
    if (code != 0) {
      int q = (int)code - ORA_RADIUS;
      w->recon[i] = p + (float)q * w->twoe[l - 1];
    } /* else: the outlier value is already in recon[i] */
  }
  w->stamp[i] = w->cur;
}

/* One level (stride s = 2^(l-1)), Sec. 5.1: the new points are the points
 * of the stride-s grid that are not on the stride-2s grid. */
static void run_level(sweep* w, int l) {
  const geom* g = w->g;
  const ora_config* c = w->c;
  uint64_t s = (uint64_t)1 << (l - 1);
  uint64_t step[3];
  for (int d = 0; d < 3; ++d) step[d] = g->interp[d] ? s : 1;
  int md = c->paradigm[l - 1] == ORA_MD;
  int npass = g->k;
  for (int pj = 0; pj < npass; ++pj) {
    int pass_slot = -1;
    if (!md) pass_slot = c->order[l - 1][pj] + g->off;
    for (int half = 0; half < 2; ++half) {
      w->cur++;
      uint64_t cc[3];
      for (cc[0] = 0; cc[0] < g->n[0]; cc[0] += step[0])
        for (cc[1] = 0; cc[1] < g->n[1]; cc[1] += step[1])
          for (cc[2] = 0; cc[2] < g->n[2]; cc[2] += step[2]) {
            /* classify: u_d = c_d / s on interpolation slots */
            unsigned odd = 0;
            int nodd = 0;
            for (int d = 0; d < 3; ++d)
              if (g->interp[d] && ((cc[d] / s) & 1)) {
                odd |= 1u << d;
                nodd++;
              }
            if (nodd == 0) continue; /* on the stride-2s grid: known */
            unsigned S;
            if (!md) {
              /* 1D-style pass j along order[j]: odd on that dim, any
               * parity on earlier dims of the order, even on later ones */
              if (!(odd & (1u << pass_slot))) continue;
              int ok = 1;
              for (int m = pj + 1; m < g->k; ++m) {
                int sl = c->order[l - 1][m] + g->off;
                if (odd & (1u << sl)) ok = 0;
              }
              if (!ok) continue;
              S = 1u << pass_slot;
            } else {
              /* MD sub-pass pj+1: exactly pj+1 odd coordinates */
              if (nodd != pj + 1) continue;
              S = odd;
            }
            int kind, same;
            point_cfg(w, l, cc, &kind, &same);
            /* same-level split (Sec. 5.4.2): parity of sum (u_d - 1)/2 */
            unsigned par = 0;
            for (int d = 0; d < 3; ++d)
              if (S & (1u << d)) par += (unsigned)(((cc[d] / s) - 1) / 2);
            int in_b = same && (par & 1u);
            if (in_b != half) continue;
            uint64_t i = cc[0] * g->st[0] + cc[1] * g->st[1] + cc[2];
            process_point(w, l, i, cc, md, pass_slot, S, in_b, kind);
          }
    }
  }
}

static int is_anchor(const geom* g, const uint64_t c[3]) {
  for (int d = 0; d < 3; ++d)
    if (g->interp[d] && (c[d] % (uint64_t)g->A) != 0) return 0;
  return 1;
}

/* ------------------------------------------------------------------ */
/* Huffman (Sec. 4 Step 4)                                             */
/* ------------------------------------------------------------------ */
typedef struct {
  uint64_t f;
  uint32_t sym;
} leaf_t;

static int leaf_cmp(const void* a, const void* b) {
  const leaf_t* x = (const leaf_t*)a;
  const leaf_t* y = (const leaf_t*)b;
  if (x->f != y->f) return x->f < y->f ? -1 : 1;
  return x->sym < y->sym ? -1 : (x->sym > y->sym ? 1 : 0);
}

/* Two-queue Huffman merge: leaves sorted by (frequency, symbol); the
 * internal nodes form a FIFO in creation order; each pick takes the
 * smaller weight and, on a tie, the leaf.  Lengths are leaf depths. */
int ora_huffman_lengths(const uint64_t* freq, int nsym, uint8_t* lens) {
  int n = 0;
  for (int i = 0; i < nsym; ++i) {
    lens[i] = 0;
    if (freq[i]) n++;
  }
  if (n <= 1) return ORA_OK; /* a lone symbol gets the empty code */
  leaf_t* lv = (leaf_t*)malloc(sizeof(leaf_t) * (size_t)n);
  uint64_t* iw = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  uint32_t* parent = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(2 * n));
  uint32_t* depth = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(2 * n));
  if (!lv || !iw || !parent || !depth) {
    free(lv); free(iw); free(parent); free(depth);
    return ORA_ERR_NO_MEMORY;
  }
  int j = 0;
  for (int i = 0; i < nsym; ++i)
    if (freq[i]) {
      lv[j].f = freq[i];
      lv[j].sym = (uint32_t)i;
      j++;
    }
  qsort(lv, (size_t)n, sizeof(leaf_t), leaf_cmp);
  int a = 0, b = 0, m = 0; /* leaf head, internal head, internal count */
  for (int t = 0; t < n - 1; ++t) {
    uint32_t pick[2];
    uint64_t wsum = 0;
    for (int r = 0; r < 2; ++r) {
      if (a < n && (b >= m || lv[a].f <= iw[b])) {
        pick[r] = (uint32_t)a;
        wsum += lv[a].f;
        a++;
      } else {
        pick[r] = (uint32_t)(n + b);
        wsum += iw[b];
        b++;
      }
    }
    iw[m] = wsum;
    parent[pick[0]] = (uint32_t)(n + m);
    parent[pick[1]] = (uint32_t)(n + m);
    m++;
  }
  int root = 2 * n - 2;
  depth[root] = 0;
  for (int id = root - 1; id >= 0; --id) depth[id] = depth[parent[id]] + 1;
  int rc = ORA_OK;
  for (int i = 0; i < n; ++i) {
    if (depth[i] > 63) rc = ORA_ERR_INVALID_ARG;
    lens[lv[i].sym] = (uint8_t)depth[i];
  }
  free(lv); free(iw); free(parent); free(depth);
  return rc;
}

/* Canonical codes: symbols ordered by (length, symbol); the first code is
 * 0 and each next code is (previous + 1) shifted left by the length step. */
int ora_canonical_codes(const uint8_t* lens, int nsym, uint64_t* codes) {
  uint64_t bl_count[65] = {0};
  uint64_t next[65] = {0};
  int maxlen = 0;
  for (int i = 0; i < nsym; ++i) {
    codes[i] = 0;
    if (lens[i] > 63) return ORA_ERR_INVALID_ARG;
    if (lens[i]) {
      bl_count[lens[i]]++;
      if (lens[i] > maxlen) maxlen = lens[i];
    }
  }
  uint64_t code = 0;
  for (int bits = 1; bits <= maxlen; ++bits) {
    code = (code + bl_count[bits - 1]) << 1;
    next[bits] = code;
  }
  for (int i = 0; i < nsym; ++i)
    if (lens[i]) codes[i] = next[lens[i]]++;
  return ORA_OK;
}

/* ------------------------------------------------------------------ */
/* compress                                                            */
/* ------------------------------------------------------------------ */
static uint64_t count_anchors(const geom* g) {
  uint64_t na = 1;
  for (int d = 0; d < 3; ++d)
    na *= g->interp[d] ? (g->n[d] + (uint64_t)g->A - 1) / (uint64_t)g->A
                       : g->n[d];
  return na;
}

static uint64_t count_blocks(const geom* g, int bs, uint64_t nb[3]) {
  uint64_t t = 1;
  for (int d = 0; d < g->ndim; ++d) {
    nb[d] = (g->n[d + g->off] + (uint64_t)bs - 1) / (uint64_t)bs;
    t *= nb[d];
  }
  return t;
}

uint64_t ora_compress_bound(int ndim, const uint64_t* dims) {
  uint64_t N = 1;
  for (int d = 0; d < ndim; ++d) N *= dims[d];
  uint64_t nch = (N + 255) / 256;
  /* header + anchors/outliers (<= N floats each) + block map + lane bit
   * counts + table + bitstream (<= 17 bits per symbol + one pad word per
   * chunk) */
  return 512 + 16 * 8 + 4 * N + 4 * N + N + 64 * nch + 3 * 65536 + 4 +
         (17 * N) / 8 + 4 * nch + 64;
}

/* The Lorenzo predictor over the whole field (Sec. 6.5, the dynamic-order
 * predictor of sz-auto, read here as block-local): the field is cut into
 * blocks of side A along every dimension (the last ones ragged); inside a
 * block, in row-major order, a point is predicted from the reconstructed
 * points of its block by the order-1 or order-2 Lorenzo stencil, a
 * neighbour outside the block reading 0 -- the recurrence the tuner's
 * Lorenzo test runs on its sample blocks.  Terms in the order of the
 * offsets (a, b, c) along dims 0, 1, 2, a outermost; each weight is minus
 * the product of the per-dimension coefficients (1, -1) or (1, -2, 1).
 * The error bound is the global e.  compress: codes and recon from x;
 * decompress: recon from the codes, recon already holding the outliers. */
static void lorenzo_field(const geom* g, int order, float e, const float* x,
                          uint16_t* codes, float* recon, int decompress) {
  const float inv2 = (float)(1.0 / (2.0 * (double)e));
  const float twoe = 2.0f * e;
  const float co[2][3] = {{1.0f, -1.0f, 0.0f}, {1.0f, -2.0f, 1.0f}};
  int lim[3];
  for (int d = 0; d < 3; ++d) lim[d] = d < g->off ? 0 : order;
  const uint64_t B = (uint64_t)g->A;
  uint64_t o[3];
  for (o[0] = 0; o[0] < g->n[0]; o[0] += (g->off > 0 ? 1 : B))
    for (o[1] = 0; o[1] < g->n[1]; o[1] += (g->off > 1 ? 1 : B))
      for (o[2] = 0; o[2] < g->n[2]; o[2] += B) {
        uint64_t m[3];
        for (int d = 0; d < 3; ++d) {
          const uint64_t side = d < g->off ? 1 : B;
          m[d] = g->n[d] - o[d] < side ? g->n[d] - o[d] : side;
        }
        for (uint64_t i0 = 0; i0 < m[0]; ++i0)
          for (uint64_t i1 = 0; i1 < m[1]; ++i1)
            for (uint64_t i2 = 0; i2 < m[2]; ++i2) {
              float acc = 0.0f;
              for (int a = 0; a <= lim[0]; ++a)
                for (int b = 0; b <= lim[1]; ++b)
                  for (int c = 0; c <= lim[2]; ++c) {
                    if (a == 0 && b == 0 && c == 0) continue;
                    const float wgt = -(co[order - 1][a] * co[order - 1][b] * co[order - 1][c]);
                    float v = 0.0f;
                    if ((uint64_t)a <= i0 && (uint64_t)b <= i1 && (uint64_t)c <= i2)
                      v = recon[(o[0] + i0 - a) * g->st[0] + (o[1] + i1 - b) * g->st[1] +
                                (o[2] + i2 - c)];
                    acc = acc + wgt * v;
                  }
              const uint64_t i = (o[0] + i0) * g->st[0] + (o[1] + i1) * g->st[1] + (o[2] + i2);
              if (!decompress) {
                float rec;
                codes[i] = ora_quantize(x[i], acc, e, inv2, twoe, &rec);
                recon[i] = rec;
              } else if (codes[i] != 0) {
                const int q = (int)codes[i] - ORA_RADIUS;
                recon[i] = acc + (float)q * twoe;
              } /* else: the outlier value is already in recon[i] */
            }
      }
}

static int write_const(uint8_t* out, uint64_t cap, uint64_t* out_size,
                       int ndim, const uint64_t* dims, int eb_mode, double eb,
                       float v, const ora_config* c) {
  if (cap < ORA_HEADER_BYTES) return ORA_ERR_OUT_TOO_SMALL;
  memset(out, 0, ORA_HEADER_BYTES);
  put_u32(out, H_MAGIC, MAGIC);
  put_u32(out, H_VERSION, VERSION);
  put_u32(out, H_FLAGS, FLAG_CONST);
  put_u32(out, H_NDIM, (uint32_t)ndim);
  for (int d = 0; d < 3; ++d) put_u64(out, H_DIMS + 8 * d, d < ndim ? dims[d] : 1);
  put_u32(out, H_EBMODE, (uint32_t)eb_mode);
  put_u32(out, H_ANCHOR, (uint32_t)c->anchor_stride);
  put_f64(out, H_EBVALUE, eb);
  put_f32(out, H_E, 0.0f);
  put_f32(out, H_CONST, v);
  put_u32(out, H_FROZEN, (uint32_t)(int32_t)-1);
  put_u32(out, H_CHUNK, (uint32_t)c->chunk_syms);
  for (int s = H_OFF_ANCHORS; s <= H_OFF_BLOCKMAP; s += 8)
    put_u64(out, (uint64_t)s, ORA_HEADER_BYTES);
  put_u64(out, H_TOTAL, ORA_HEADER_BYTES);
  *out_size = ORA_HEADER_BYTES;
  return ORA_OK;
}

int ora_compress(const float* x, int ndim, const uint64_t* dims, int eb_mode,
                 double eb, const ora_config* cfg_in, uint8_t* out,
                 uint64_t cap, uint64_t* out_size, uint16_t* codes_out,
                 float* recon_out, ora_stats* stats) {
  ora_config defc;
  if (!x || !dims || !out || !out_size) return ORA_ERR_INVALID_ARG;
  if (ndim < 1 || ndim > 3) return ORA_ERR_INVALID_ARG;
  if (!cfg_in) {
    ora_default_config(ndim, &defc);
    cfg_in = &defc;
  }
  const ora_config* c = cfg_in;
  geom g;
  int rc = geom_init(&g, ndim, dims, c->anchor_stride, c->frozen_dim);
  if (rc) return rc;
  rc = check_config(&g, c);
  if (rc) return rc;
  if (eb_mode != ORA_EB_ABS && eb_mode != ORA_EB_REL) return ORA_ERR_INVALID_ARG;
  if (!(eb > 0.0) || !isfinite(eb)) return ORA_ERR_INVALID_ARG;
  const uint64_t N = g.N;
  if (stats) memset(stats, 0, sizeof(*stats));

  /* error bound: absolute, or eps * value range (Sec. 7.1.3) */
  float e;
  float vmin = x[0], vmax = x[0];
  if (eb_mode == ORA_EB_REL) {
    for (uint64_t i = 0; i < N; ++i) {
      float v = x[i];
      if (!isfinite(v)) return ORA_ERR_NONFINITE;
      if (v < vmin) vmin = v;
      if (v > vmax) vmax = v;
    }
    double range = (double)vmax - (double)vmin;
    if (range == 0.0)
      return write_const(out, cap, out_size, ndim, dims, eb_mode, eb, x[0], c);
    e = (float)(eb * range);
  } else {
    e = (float)eb;
  }
  if (!(e > 0.0f) || !isfinite(e)) return ORA_ERR_INVALID_ARG;

  sweep w;
  memset(&w, 0, sizeof(w));
  w.g = &g;
  w.c = c;
  rc = ora_level_params(e, c->alpha, c->beta, g.L, w.el, w.inv2, w.twoe);
  if (rc) return rc;
  uint64_t nblocks = 0;
  if (c->blockwise) nblocks = count_blocks(&g, c->block_size, w.nb);

  w.x = x;
  w.recon = (float*)malloc(sizeof(float) * N);
  w.codes = (uint16_t*)malloc(sizeof(uint16_t) * N);
  w.stamp = (uint32_t*)calloc(N, sizeof(uint32_t));
  if (!w.recon || !w.codes || !w.stamp) {
    free(w.recon); free(w.codes); free(w.stamp);
    return ORA_ERR_NO_MEMORY;
  }

  /* anchors (Sec. 5.1): stored losslessly, code = radius (zero error);
   * the Lorenzo predictor has none */
  uint64_t na = c->predictor ? 0 : count_anchors(&g);
  float* anchors = (float*)malloc(sizeof(float) * (na ? na : 1));
  uint64_t ai = 0;
  uint64_t missing = 0;
  if (c->predictor) {
    lorenzo_field(&g, c->predictor, e, x, w.codes, w.recon, 0);
    w.predicted = N;
  } else {
    uint64_t cc[3];
    for (cc[0] = 0; cc[0] < g.n[0]; ++cc[0])
      for (cc[1] = 0; cc[1] < g.n[1]; ++cc[1])
        for (cc[2] = 0; cc[2] < g.n[2]; ++cc[2]) {
          uint64_t i = cc[0] * g.st[0] + cc[1] * g.st[1] + cc[2];
          if (is_anchor(&g, cc)) {
            anchors[ai++] = x[i];
            w.recon[i] = x[i];
            w.codes[i] = ORA_RADIUS;
            w.stamp[i] = 1;
          }
        }
    w.cur = 1;

    /* the level sweep, coarse to fine */
    for (int l = g.L; l >= 1; --l) run_level(&w, l);

    /* every point is either an anchor or predicted exactly once */
    for (uint64_t i = 0; i < N; ++i)
      if (w.stamp[i] == 0) missing++;
  }

  /* outliers in row-major order */
  uint64_t nout = 0;
  for (uint64_t i = 0; i < N; ++i)
    if (w.codes[i] == 0) nout++;
  float* outl = (float*)malloc(sizeof(float) * (nout ? nout : 1));
  {
    uint64_t k = 0;
    for (uint64_t i = 0; i < N; ++i)
      if (w.codes[i] == 0) outl[k++] = x[i];
  }

  /* Huffman over the row-major code array */
  uint64_t* hist = (uint64_t*)calloc(65536, sizeof(uint64_t));
  uint8_t* lens = (uint8_t*)malloc(65536);
  uint64_t* code64 = (uint64_t*)malloc(sizeof(uint64_t) * 65536);
  for (uint64_t i = 0; i < N; ++i) hist[w.codes[i]]++;
  rc = ora_huffman_lengths(hist, 65536, lens);
  if (!rc) rc = ora_canonical_codes(lens, 65536, code64);
  uint32_t nused = 0;
  for (int i = 0; i < 65536; ++i)
    if (hist[i]) nused++;
  /* chunked bit layout: a chunk of C symbols is coded as 32 lanes, lane l
   * holding the chunk's symbols l, l+32, l+64, ... in order; the lanes'
   * bits follow one another (lane 0 first), MSB first in 32-bit words;
   * each chunk starts on a word; the bit count of every lane is stored */
  const uint64_t C = (uint64_t)c->chunk_syms;
  const uint64_t nch = (N + C - 1) / C;
  uint16_t* lanebits = (uint16_t*)calloc(nch * 32, sizeof(uint16_t));
  uint64_t sumlen = 0;
  for (uint64_t i = 0; i < N; ++i) sumlen += lens[w.codes[i]];
  uint64_t maxwords = sumlen / 32 + nch + 1;
  uint32_t* bits = (uint32_t*)calloc(maxwords, sizeof(uint32_t));
  uint64_t wpos = 0;
  for (uint64_t ch = 0; ch < nch && !rc; ++ch) {
    uint32_t cur = 0;
    int nb = 0;
    const uint64_t beg = ch * C;
    const uint64_t nc = (beg + C < N ? beg + C : N) - beg;
    for (uint64_t lane = 0; lane < 32; ++lane) {
      uint64_t lb = 0;
      for (uint64_t j = lane; j < nc; j += 32) {
        uint16_t sy = w.codes[beg + j];
        int L_ = lens[sy];
        uint64_t cw = code64[sy];
        lb += (uint64_t)L_;
        for (int b = L_ - 1; b >= 0; --b) { /* MSB first */
          cur = (cur << 1) | (uint32_t)((cw >> b) & 1u);
          nb++;
          if (nb == 32) {
            bits[wpos++] = cur;
            cur = 0;
            nb = 0;
          }
        }
      }
      lanebits[ch * 32 + lane] = (uint16_t)lb;
    }
    if (nb) bits[wpos++] = cur << (32 - nb);
  }

  /* container */
  uint64_t off_anchors = ORA_HEADER_BYTES;
  uint64_t off_blockmap = align16(off_anchors + 4 * na);
  uint64_t off_chunkw = align16(off_blockmap + nblocks);
  uint64_t off_table = align16(off_chunkw + 64 * nch);
  uint64_t off_outl = align16(off_table + 3 * (uint64_t)nused);
  uint64_t off_bits = align16(off_outl + 4 * nout);
  uint64_t total = off_bits + 4 * wpos;
  if (!rc && total > cap) rc = ORA_ERR_OUT_TOO_SMALL;
  if (!rc && (missing || w.bad_reads || w.double_visits)) rc = ORA_ERR_SELFCHECK;
  if (!rc) {
    memset(out, 0, total);
    put_u32(out, H_MAGIC, MAGIC);
    put_u32(out, H_VERSION, VERSION);
    put_u32(out, H_FLAGS, 0);
    put_u32(out, H_NDIM, (uint32_t)ndim);
    for (int d = 0; d < 3; ++d) put_u64(out, H_DIMS + 8 * d, d < ndim ? dims[d] : 1);
    put_u32(out, H_EBMODE, (uint32_t)eb_mode);
    put_u32(out, H_ANCHOR, (uint32_t)c->anchor_stride);
    put_f64(out, H_EBVALUE, eb);
    put_f32(out, H_E, e);
    put_f32(out, H_CONST, 0.0f);
    put_u32(out, H_FROZEN, (uint32_t)c->frozen_dim);
    put_u32(out, H_CHUNK, (uint32_t)c->chunk_syms);
    put_f64(out, H_ALPHA, c->alpha);
    put_f64(out, H_BETA, c->beta);
    for (int d = 0; d < 3; ++d) put_f64(out, H_MDIV + 8 * d, c->md_inv_var[d]);
    for (int l = 0; l < ORA_MAX_LEVELS; ++l) {
      int used = l < g.L;
      put_u8(out, H_INTERP + l, used ? c->interp[l] : 0);
      put_u8(out, H_PARADIGM + l, used ? c->paradigm[l] : 0);
      put_u8(out, H_SAME + l, used ? c->same_level[l] : 0);
      for (int j = 0; j < 3; ++j)
        put_u8(out, H_ORDER + 3 * l + j,
               (used && j < g.k) ? c->order[l][j] : 255);
    }
    put_u32(out, H_PREDICTOR, (uint32_t)c->predictor);
    put_u32(out, H_BLOCKWISE, (uint32_t)c->blockwise);
    put_u64(out, H_NANCHORS, na);
    put_u64(out, H_NOUTLIERS, nout);
    put_u32(out, H_NUSED, nused);
    put_u32(out, H_BLOCKSIZE, (uint32_t)c->block_size);
    put_u64(out, H_NCHUNKS, nch);
    put_u64(out, H_TOTALWORDS, wpos);
    put_u64(out, H_OFF_ANCHORS, off_anchors);
    put_u64(out, H_OFF_CHUNKW, off_chunkw);
    put_u64(out, H_OFF_TABLE, off_table);
    put_u64(out, H_OFF_OUTLIERS, off_outl);
    put_u64(out, H_OFF_BITS, off_bits);
    put_u64(out, H_OFF_BLOCKMAP, off_blockmap);
    put_u64(out, H_TOTAL, total);
    put_u64(out, H_NBLOCKS, nblocks);
    for (uint64_t i = 0; i < na; ++i) put_f32(out, off_anchors + 4 * i, anchors[i]);
    for (uint64_t i = 0; i < nblocks; ++i) put_u8(out, off_blockmap + i, c->blockmap[i]);
    for (uint64_t i = 0; i < 32 * nch; ++i) put_u16(out, off_chunkw + 2 * i, lanebits[i]);
    {
      uint64_t k = 0;
      for (int sy = 0; sy < 65536; ++sy)
        if (hist[sy]) {
          put_u16(out, off_table + 2 * k, (uint16_t)sy);
          put_u8(out, off_table + 2 * (uint64_t)nused + k, lens[sy]);
          k++;
        }
    }
    for (uint64_t i = 0; i < nout; ++i) put_f32(out, off_outl + 4 * i, outl[i]);
    for (uint64_t i = 0; i < wpos; ++i) put_u32(out, off_bits + 4 * i, bits[i]);
    *out_size = total;
  }
  if (stats) {
    stats->n_points = N;
    stats->n_anchors = na;
    stats->n_outliers = nout;
    stats->n_used = nused;
    stats->total_words = wpos;
    stats->n_chunks = nch;
    stats->predicted = w.predicted;
    stats->bad_reads = w.bad_reads + missing;
    stats->double_visits = w.double_visits;
    stats->sum_len_bits = sumlen;
    stats->e = e;
    stats->vmin = vmin;
    stats->vmax = vmax;
  }
  if (codes_out) memcpy(codes_out, w.codes, sizeof(uint16_t) * N);
  if (recon_out) memcpy(recon_out, w.recon, sizeof(float) * N);
  free(w.recon); free(w.codes); free(w.stamp); free(anchors); free(outl);
  free(hist); free(lens); free(code64); free(lanebits); free(bits);
  return rc;
}

/* ------------------------------------------------------------------ */
/* decompress                                                          */
/* ------------------------------------------------------------------ */
int ora_inspect(const uint8_t* in, uint64_t size, int* ndim, uint64_t* dims,
                double* abs_eb) {
  if (!in || size < ORA_HEADER_BYTES) return ORA_ERR_CORRUPT;
  if (get_u32(in, H_MAGIC) != MAGIC || get_u32(in, H_VERSION) != VERSION)
    return ORA_ERR_CORRUPT;
  int nd = (int)get_u32(in, H_NDIM);
  if (nd < 1 || nd > 3) return ORA_ERR_CORRUPT;
  if (ndim) *ndim = nd;
  if (dims)
    for (int d = 0; d < nd; ++d) dims[d] = get_u64(in, H_DIMS + 8 * d);
  if (abs_eb) *abs_eb = (double)get_f32(in, H_E);
  return ORA_OK;
}

int ora_decompress(const uint8_t* in, uint64_t size, float* out,
                   uint64_t cap_elems) {
  int ndim;
  uint64_t dims[3];
  int rc = ora_inspect(in, size, &ndim, dims, NULL);
  if (rc) return rc;
  if (get_u32(in, H_FLAGS) & FLAG_LOSSLESS) {
    /* undo the lossless stage first */
    const uint64_t raw = get_u64(in, ORA_H_RAWSIZE);
    if (raw < ORA_HEADER_BYTES || raw > ((uint64_t)1 << 40)) return ORA_ERR_CORRUPT;
    uint8_t* tmp = (uint8_t*)malloc(raw);
    uint64_t got = 0;
    rc = ora_lossless_decode(in, size, tmp, raw, &got);
    if (!rc && got != raw) rc = ORA_ERR_CORRUPT;
    if (!rc) rc = ora_decompress(tmp, raw, out, cap_elems);
    free(tmp);
    return rc;
  }
  if (!out) return ORA_ERR_INVALID_ARG;
  uint64_t N = 1;
  for (int d = 0; d < ndim; ++d) {
    if (dims[d] == 0) return ORA_ERR_CORRUPT;
    N *= dims[d];
    if (N > 0xFFFFFFFFull) return ORA_ERR_CORRUPT;
  }
  if (N > cap_elems) return ORA_ERR_OUT_TOO_SMALL;
  if (get_u64(in, H_TOTAL) > size) return ORA_ERR_CORRUPT;
  if (get_u32(in, H_FLAGS) & FLAG_CONST) {
    float v = get_f32(in, H_CONST);
    for (uint64_t i = 0; i < N; ++i) out[i] = v;
    return ORA_OK;
  }
  ora_config c;
  memset(&c, 0, sizeof(c));
  c.anchor_stride = (int32_t)get_u32(in, H_ANCHOR);
  c.frozen_dim = (int32_t)get_u32(in, H_FROZEN);
  c.chunk_syms = (int32_t)get_u32(in, H_CHUNK);
  c.alpha = get_f64(in, H_ALPHA);
  c.beta = get_f64(in, H_BETA);
  for (int d = 0; d < 3; ++d) c.md_inv_var[d] = get_f64(in, H_MDIV + 8 * d);
  for (int l = 0; l < ORA_MAX_LEVELS; ++l) {
    c.interp[l] = in[H_INTERP + l];
    c.paradigm[l] = in[H_PARADIGM + l];
    c.same_level[l] = in[H_SAME + l];
    for (int j = 0; j < 3; ++j) c.order[l][j] = in[H_ORDER + 3 * l + j];
  }
  c.blockwise = (int32_t)get_u32(in, H_BLOCKWISE);
  c.block_size = (int32_t)get_u32(in, H_BLOCKSIZE);
  c.predictor = (int32_t)get_u32(in, H_PREDICTOR);
  geom g;
  rc = geom_init(&g, ndim, dims, c.anchor_stride, c.frozen_dim);
  if (rc) return ORA_ERR_CORRUPT;
  uint64_t nb[3] = {1, 1, 1};
  uint64_t nblocks = 0;
  if (c.blockwise) {
    if (c.block_size < 1) return ORA_ERR_CORRUPT;
    nblocks = count_blocks(&g, c.block_size, nb);
    if (get_u64(in, H_NBLOCKS) != nblocks) return ORA_ERR_CORRUPT;
    uint64_t ob = get_u64(in, H_OFF_BLOCKMAP);
    if (ob + nblocks > size) return ORA_ERR_CORRUPT;
    c.blockmap = in + ob;
  }
  if (check_config(&g, &c)) return ORA_ERR_CORRUPT;
  float e = get_f32(in, H_E);
  if (!(e > 0.0f) || !isfinite(e)) return ORA_ERR_CORRUPT;

  sweep w;
  memset(&w, 0, sizeof(w));
  w.g = &g;
  w.c = &c;
  w.decompress = 1;
  for (int d = 0; d < 3; ++d) w.nb[d] = nb[d];
  if (ora_level_params(e, c.alpha, c.beta, g.L, w.el, w.inv2, w.twoe))
    return ORA_ERR_CORRUPT;

  uint64_t na = get_u64(in, H_NANCHORS);
  uint64_t nout = get_u64(in, H_NOUTLIERS);
  uint32_t nused = get_u32(in, H_NUSED);
  uint64_t nch = get_u64(in, H_NCHUNKS);
  uint64_t twords = get_u64(in, H_TOTALWORDS);
  const uint64_t C = (uint64_t)c.chunk_syms;
  if (na != (c.predictor ? 0 : count_anchors(&g)) || nch != (N + C - 1) / C || nused == 0 ||
      nused > 65536 || nout > N)
    return ORA_ERR_CORRUPT;
  uint64_t oa = get_u64(in, H_OFF_ANCHORS), ocw = get_u64(in, H_OFF_CHUNKW),
           ot = get_u64(in, H_OFF_TABLE), oo = get_u64(in, H_OFF_OUTLIERS),
           obits = get_u64(in, H_OFF_BITS);
  if (oa + 4 * na > size || ocw + 64 * nch > size ||
      ot + 3 * (uint64_t)nused > size || oo + 4 * nout > size ||
      obits + 4 * twords > size)
    return ORA_ERR_CORRUPT;

  /* canonical decode tables */
  uint16_t* syms = (uint16_t*)malloc(sizeof(uint16_t) * nused);
  uint8_t* lns = (uint8_t*)malloc(nused);
  uint64_t cnt[65] = {0};
  int maxlen = 0;
  for (uint32_t k = 0; k < nused; ++k) {
    syms[k] = get_u16(in, ot + 2 * (uint64_t)k);
    lns[k] = in[ot + 2 * (uint64_t)nused + k];
    if ((k > 0 && syms[k] <= syms[k - 1]) || lns[k] > 63 ||
        (nused > 1 && lns[k] == 0) || (nused == 1 && lns[k] != 0)) {
      free(syms); free(lns);
      return ORA_ERR_CORRUPT;
    }
    cnt[lns[k]]++;
    if (lns[k] > maxlen) maxlen = lns[k];
  }
  /* symbols sorted by (length, symbol): stable counting order */
  uint64_t first[65] = {0}, offs[65] = {0};
  uint16_t* sorted = (uint16_t*)malloc(sizeof(uint16_t) * nused);
  {
    uint64_t code = 0, pos = 0;
    for (int b = 1; b <= maxlen; ++b) {
      code = (code + cnt[b - 1]) << 1;
      first[b] = code;
      offs[b] = pos;
      pos += cnt[b];
    }
    uint64_t fill[65];
    memcpy(fill, offs, sizeof(fill));
    for (uint32_t k = 0; k < nused; ++k)
      if (lns[k]) sorted[fill[lns[k]]++] = syms[k];
  }
  uint16_t* codes = (uint16_t*)malloc(sizeof(uint16_t) * N);
  w.codes = codes;
  w.recon = out;
  w.stamp = (uint32_t*)calloc(N, sizeof(uint32_t));
  rc = ORA_OK;
  uint64_t wbase = 0;
  for (uint64_t ch = 0; ch < nch && !rc; ++ch) {
    uint64_t lb[32], sum = 0;
    for (int l = 0; l < 32; ++l) {
      lb[l] = get_u16(in, ocw + 64 * ch + 2 * (uint64_t)l);
      sum += lb[l];
    }
    const uint64_t nw = (sum + 31) / 32;
    if (wbase + nw > twords) {
      rc = ORA_ERR_CORRUPT;
      break;
    }
    const uint64_t beg = ch * C;
    const uint64_t nc = (beg + C < N ? beg + C : N) - beg;
    uint64_t bitpos = 0;
    for (int lane = 0; lane < 32 && !rc; ++lane) {
      const uint64_t lane_end = bitpos + lb[lane];
      for (uint64_t j = (uint64_t)lane; j < nc; j += 32) {
        if (nused == 1) {
          codes[beg + j] = syms[0];
          continue;
        }
        uint64_t code = 0;
        int len = 0, found = 0;
        while (len < maxlen && bitpos < lane_end) {
          uint32_t word = get_u32(in, obits + 4 * (wbase + bitpos / 32));
          uint32_t bit = (word >> (31 - (bitpos % 32))) & 1u;
          bitpos++;
          code = (code << 1) | bit;
          len++;
          if (cnt[len] && code >= first[len] && code - first[len] < cnt[len]) {
            codes[beg + j] = sorted[offs[len] + (code - first[len])];
            found = 1;
            break;
          }
        }
        if (!found) {
          rc = ORA_ERR_CORRUPT;
          break;
        }
      }
      if (bitpos != lane_end) rc = ORA_ERR_CORRUPT;
    }
    wbase += nw;
  }
  if (!rc && wbase != twords) rc = ORA_ERR_CORRUPT;

  if (!rc) {
    /* anchors, then outliers scattered in row-major order */
    uint64_t ai = 0, oi = 0;
    uint64_t cc[3];
    for (cc[0] = 0; cc[0] < g.n[0]; ++cc[0])
      for (cc[1] = 0; cc[1] < g.n[1]; ++cc[1])
        for (cc[2] = 0; cc[2] < g.n[2]; ++cc[2]) {
          uint64_t i = cc[0] * g.st[0] + cc[1] * g.st[1] + cc[2];
          if (!c.predictor && is_anchor(&g, cc)) {
            out[i] = get_f32(in, oa + 4 * ai);
            ai++;
            w.stamp[i] = 1;
          } else if (codes[i] == 0) {
            if (oi < nout) out[i] = get_f32(in, oo + 4 * oi);
            oi++;
          }
        }
    if (oi != nout) rc = ORA_ERR_CORRUPT;
  }
  if (!rc && c.predictor) {
    lorenzo_field(&g, c.predictor, e, NULL, codes, out, 1);
  } else if (!rc) {
    w.cur = 1;
    for (int l = g.L; l >= 1; --l) run_level(&w, l);
    if (w.bad_reads || w.double_visits) rc = ORA_ERR_SELFCHECK;
  }
  free(syms); free(lns); free(sorted); free(codes); free(w.stamp);
  return rc;
}

/* ================================================================== */
/* Auto-tuning (Sec. 6): statistics on a sample (6.1), per-level global  */
/* interpolation tuning on sampled blocks (6.2), level error bounds      */
/* alpha/beta (6.4), dimension freezing (6.3), Lorenzo test (6.5),       */
/* block-wise interpolator choice (6.6).  Every score is an integer     */
/* (fixed-point errors, Huffman bit counts), so decisions do not depend  */
/* on summation order.                                                   */
/* ================================================================== */

void ora_default_tune_params(ora_tune_params* t) {
  memset(t, 0, sizeof(*t));
  t->sample_rate = 0.002;
  t->block_rate = 0.01;
  t->sub_frac = 0.04;
  t->lorenzo_coef = 1.0;
  t->block_size = 32;
  t->tune_levels = 1;
  t->tune_eb = 1;
  t->tune_freeze = 1;
  t->tune_lorenzo = 1;
  t->tune_blockwise = 1;
  t->allow_natural = 1;
  t->allow_same_level = 1;
  t->anchor_stride = 0;
}

/* squared error in units of e^2 / 256 (|d| / e capped at 2^16) */
static uint64_t sq_fixed(float d, double inv_e) {
  double v = fabs((double)d) * inv_e;
  v = fmin(v, 65536.0);
  return (uint64_t)floor(v * v * 256.0);
}

/* number of bits of a Huffman code for these counts (sum of freq * len) */
static uint64_t huff_cost(const uint64_t* hist) {
  uint8_t* lens = (uint8_t*)malloc(65536);
  uint64_t c = 0;
  if (ora_huffman_lengths(hist, 65536, lens) == ORA_OK)
    for (int i = 0; i < 65536; ++i) c += hist[i] * (uint64_t)lens[i];
  free(lens);
  return c;
}

/* Runs the sweep on an extracted sub-field from the coarsest level down to
 * level l_stop: per-level scores, code histogram and escapes of the
 * predicted points.  *n_anchors receives the anchor count. */
int ora_subfield_test(const float* xs, int ndim, const uint64_t* ds,
                         const ora_config* c, float e, int l_stop,
                         uint64_t* score, uint64_t* chist, uint64_t* nout,
                         uint64_t* n_anchors) {
  geom g;
  int rc = geom_init(&g, ndim, ds, c->anchor_stride, c->frozen_dim);
  if (rc) return rc;
  sweep w;
  memset(&w, 0, sizeof(w));
  w.g = &g;
  w.c = c;
  if (ora_level_params(e, c->alpha, c->beta, g.L, w.el, w.inv2, w.twoe))
    return ORA_ERR_INVALID_ARG;
  const uint64_t N = g.N;
  w.x = xs;
  w.recon = (float*)malloc(sizeof(float) * N);
  w.codes = (uint16_t*)malloc(sizeof(uint16_t) * N);
  w.stamp = (uint32_t*)calloc(N, sizeof(uint32_t));
  w.score = score;
  w.chist = chist;
  uint64_t na = 0;
  uint64_t cc[3];
  for (cc[0] = 0; cc[0] < g.n[0]; ++cc[0])
    for (cc[1] = 0; cc[1] < g.n[1]; ++cc[1])
      for (cc[2] = 0; cc[2] < g.n[2]; ++cc[2]) {
        uint64_t i = cc[0] * g.st[0] + cc[1] * g.st[1] + cc[2];
        if (is_anchor(&g, cc)) {
          w.recon[i] = xs[i];
          w.codes[i] = ORA_RADIUS;
          w.stamp[i] = 1;
          na++;
        }
      }
  w.cur = 1;
  for (int l = g.L; l >= l_stop && l >= 1; --l) run_level(&w, l);
  if (nout) *nout += w.nout;
  if (n_anchors) *n_anchors += na;
  free(w.recon);
  free(w.codes);
  free(w.stamp);
  return ORA_OK;
}

/* region [start, start + ext) of the field, row-major */
static float* extract(const float* x, int ndim, const uint64_t* dims,
                      const uint64_t* start, const uint64_t* ext) {
  uint64_t n[3] = {1, 1, 1}, st[3] = {0, 0, 0}, e3[3] = {1, 1, 1};
  int off = 3 - ndim;
  for (int d = 0; d < ndim; ++d) {
    n[d + off] = dims[d];
    st[d + off] = start[d];
    e3[d + off] = ext[d];
  }
  float* out = (float*)malloc(sizeof(float) * e3[0] * e3[1] * e3[2]);
  uint64_t k = 0;
  for (uint64_t a = 0; a < e3[0]; ++a)
    for (uint64_t b = 0; b < e3[1]; ++b)
      for (uint64_t c = 0; c < e3[2]; ++c)
        out[k++] = x[((st[0] + a) * n[1] + (st[1] + b)) * n[2] + st[2] + c];
  return out;
}

/* Candidate j of the global per-level tuning (Sec. 6.2): interpolator
 * (linear, not-a-knot, natural) x paradigm (each 1D-style order of the
 * interpolation dims in lexicographic order, then multi-dimensional) x
 * same-level (cubic only).  Returns 0 past the end of the list. */
int ora_tune_candidate(const ora_tune_params* tp, int ndim, int frozen, int j,
                       int* kind, int* paradigm, uint8_t order[3], int* same) {
  int dims[3], k = 0;
  for (int d = 0; d < ndim; ++d)
    if (d != frozen) dims[k++] = d;
  /* orders of the k dims, lexicographic */
  int perms[6][3], np = 0;
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b)
      for (int c = 0; c < k; ++c) {
        if (k >= 2 && b == a) continue;
        if (k >= 3 && (c == a || c == b)) continue;
        if (k < 2 && b != 0) continue;
        if (k < 3 && c != 0) continue;
        perms[np][0] = dims[a];
        perms[np][1] = k > 1 ? dims[b] : 255;
        perms[np][2] = k > 2 ? dims[c] : 255;
        np++;
      }
  const int nvar = np + (k >= 2 ? 1 : 0);
  int idx = 0;
  for (int kd = 0; kd < 3; ++kd) {
    if (kd == ORA_CUBIC_NAT && !tp->allow_natural) continue;
    const int nsl = (kd == ORA_LINEAR || !tp->allow_same_level) ? 1 : 2;
    for (int v = 0; v < nvar; ++v)
      for (int sl = 0; sl < nsl; ++sl) {
        if (idx == j) {
          *kind = kd;
          *same = sl;
          if (v < np) {
            *paradigm = ORA_1D;
            for (int q = 0; q < 3; ++q) order[q] = (uint8_t)perms[v][q];
          } else {
            *paradigm = ORA_MD;
            for (int q = 0; q < 3; ++q) order[q] = (uint8_t)(q < k ? dims[q] : 255);
          }
          return 1;
        }
        idx++;
      }
  }
  return 0;
}

static void set_level(ora_config* c, int l, int kind, int paradigm,
                      const uint8_t order[3], int same) {
  c->interp[l - 1] = (uint8_t)kind;
  c->paradigm[l - 1] = (uint8_t)paradigm;
  c->same_level[l - 1] = (uint8_t)same;
  for (int q = 0; q < 3; ++q) c->order[l - 1][q] = order[q];
}

typedef struct {
  int nblk;
  float** xs;
  uint64_t (*ds)[3];
} blockset;

/* Sample blocks of the global tuning: blocks of B + 1 points (B = the
 * anchor stride) on a lattice of block indices, every tau-th block per
 * dim, tau the smallest stride giving at most block_rate * N / B^ndim
 * blocks (at least one). */
static void sample_blocks(const float* x, int ndim, const uint64_t* dims,
                          int B, double rate, blockset* bs) {
  uint64_t nb[3], N = 1, vol = 1;
  for (int d = 0; d < ndim; ++d) {
    nb[d] = (dims[d] - 1) / (uint64_t)B;
    N *= dims[d];
    vol *= (uint64_t)B;
  }
  double tgt = floor(rate * (double)N / (double)vol + 0.5);
  uint64_t target = tgt < 1.0 ? 1 : (uint64_t)tgt;
  uint64_t tau = 1;
  for (;;) {
    uint64_t cnt = 1;
    for (int d = 0; d < ndim; ++d) {
      uint64_t m = nb[d] ? nb[d] : 1;
      cnt *= (m + tau - 1) / tau;
    }
    if (cnt <= target) break;
    tau++;
  }
  uint64_t cntd[3] = {1, 1, 1};
  int total = 1;
  for (int d = 0; d < ndim; ++d) {
    uint64_t m = nb[d] ? nb[d] : 1;
    cntd[d] = (m + tau - 1) / tau;
    total *= (int)cntd[d];
  }
  bs->nblk = total;
  bs->xs = (float**)malloc(sizeof(float*) * (size_t)total);
  bs->ds = (uint64_t(*)[3])malloc(sizeof(uint64_t[3]) * (size_t)total);
  for (int t = 0; t < total; ++t) {
    uint64_t r = (uint64_t)t, start[3], ext[3];
    for (int d = ndim - 1; d >= 0; --d) {
      uint64_t j = r % cntd[d];
      r /= cntd[d];
      if (nb[d]) {
        start[d] = j * tau * (uint64_t)B;
        ext[d] = (uint64_t)B + 1;
      } else {
        start[d] = 0;
        ext[d] = dims[d];
      }
      bs->ds[t][d] = ext[d];
    }
    bs->xs[t] = extract(x, ndim, dims, start, ext);
  }
}

static void free_blocks(blockset* bs) {
  for (int t = 0; t < bs->nblk; ++t) free(bs->xs[t]);
  free(bs->xs);
  free(bs->ds);
}

/* bits of compressing the sample blocks with c: Huffman bits of the codes
 * + 32 per escape + 32 per anchor */
static uint64_t blocks_bits(const blockset* bs, int ndim, const ora_config* c,
                            float e, uint64_t* anchors_out) {
  uint64_t* hist = (uint64_t*)calloc(65536, sizeof(uint64_t));
  uint64_t nout = 0, na = 0;
  for (int t = 0; t < bs->nblk; ++t)
    ora_subfield_test(bs->xs[t], ndim, bs->ds[t], c, e, 1, NULL, hist, &nout, &na);
  uint64_t bits = huff_cost(hist) + 32 * nout + 32 * na;
  free(hist);
  if (anchors_out) *anchors_out = na;
  return bits;
}

static const double kAlpha[5] = {1.0, 1.25, 1.5, 1.75, 2.0};
static const double kBeta[4] = {2.0, 4.0, 8.0, 16.0};

/* a12 + a13 for one frozen-dim choice; returns the sample bits estimate */
static uint64_t tune_global(const float* x, int ndim, const uint64_t* dims,
                            float e, const ora_tune_params* tp, int frozen,
                            const double* inv_var, ora_config* cfg,
                            ora_tune_report* rep, int slot) {
  ora_default_config(ndim, cfg);
  if (tp->anchor_stride) cfg->anchor_stride = tp->anchor_stride;
  cfg->frozen_dim = frozen;
  for (int d = 0; d < 3; ++d) cfg->md_inv_var[d] = inv_var[d];
  const int A = cfg->anchor_stride;
  const int L = ilog2((uint64_t)A);
  /* default order lists the interpolation dims only */
  for (int l = 0; l < ORA_MAX_LEVELS; ++l) {
    int k = 0;
    for (int d = 0; d < ndim; ++d)
      if (d != frozen) cfg->order[l][k++] = (uint8_t)d;
    for (; k < 3; ++k) cfg->order[l][k] = 255;
  }
  blockset bs;
  sample_blocks(x, ndim, dims, A, tp->block_rate, &bs);
  if (rep && slot == 0) rep->n_sample_blocks = (uint32_t)bs.nblk;
  if (tp->tune_levels) {
    for (int l = L; l >= 1; --l) {
      uint64_t best = UINT64_MAX;
      int bj = 0;
      int kind, par, same;
      uint8_t ord[3];
      for (int j = 0; ora_tune_candidate(tp, ndim, frozen, j, &kind, &par, ord, &same); ++j) {
        ora_config c2 = *cfg;
        set_level(&c2, l, kind, par, ord, same);
        uint64_t sc[ORA_MAX_LEVELS] = {0};
        for (int t = 0; t < bs.nblk; ++t)
          ora_subfield_test(bs.xs[t], ndim, bs.ds[t], &c2, e, l, sc, NULL, NULL, NULL);
        if (sc[l - 1] < best) {
          best = sc[l - 1];
          bj = j;
        }
      }
      ora_tune_candidate(tp, ndim, frozen, bj, &kind, &par, ord, &same);
      set_level(cfg, l, kind, par, ord, same);
      if (rep) {
        rep->level_choice[slot][l - 1] = (uint8_t)bj;
        rep->level_score[slot][l - 1] = best;
      }
    }
  }
  if (tp->tune_eb) {
    uint64_t best = UINT64_MAX;
    double ba = 1.0, bb = 1.0;
    for (int ia = 0; ia < 5; ++ia)
      for (int ib = 0; ib < (ia == 0 ? 1 : 4); ++ib) {
        ora_config c2 = *cfg;
        c2.alpha = kAlpha[ia];
        c2.beta = ia == 0 ? 1.0 : kBeta[ib];
        uint64_t bits = blocks_bits(&bs, ndim, &c2, e, NULL);
        if (bits < best) {
          best = bits;
          ba = c2.alpha;
          bb = c2.beta;
        }
      }
    cfg->alpha = ba;
    cfg->beta = bb;
  }
  uint64_t na = 0;
  uint64_t bits = blocks_bits(&bs, ndim, cfg, e, &na);
  if (rep) rep->bits[slot] = bits;
  free_blocks(&bs);
  return bits;
}

/* Lorenzo prediction test on a sub-field (Sec. 6.5): order 1 or 2,
 * neighbours outside the block read as 0, quantized with the global bound */
static void lorenzo_test(const float* xs, int ndim, const uint64_t* ds, int order,
                         float e, uint64_t* hist, uint64_t* nout) {
  uint64_t n[3] = {1, 1, 1};
  int off = 3 - ndim;
  for (int d = 0; d < ndim; ++d) n[d + off] = ds[d];
  const uint64_t N = n[0] * n[1] * n[2];
  float* r = (float*)malloc(sizeof(float) * N);
  const float inv2 = (float)(1.0 / (2.0 * (double)e));
  const float twoe = 2.0f * e;
  const float co[2][3] = {{1.0f, -1.0f, 0.0f}, {1.0f, -2.0f, 1.0f}};
  const int lim[3] = {off > 0 ? 0 : order, off > 1 ? 0 : order, order};
  for (uint64_t i0 = 0; i0 < n[0]; ++i0)
    for (uint64_t i1 = 0; i1 < n[1]; ++i1)
      for (uint64_t i2 = 0; i2 < n[2]; ++i2) {
        float acc = 0.0f;
        for (int a = 0; a <= lim[0]; ++a)
          for (int b = 0; b <= lim[1]; ++b)
            for (int c = 0; c <= lim[2]; ++c) {
              if (a == 0 && b == 0 && c == 0) continue;
              const float wgt = -(co[order - 1][a] * co[order - 1][b] * co[order - 1][c]);
              float v = 0.0f;
              if ((uint64_t)a <= i0 && (uint64_t)b <= i1 && (uint64_t)c <= i2)
                v = r[((i0 - a) * n[1] + (i1 - b)) * n[2] + (i2 - c)];
              acc = acc + wgt * v;
            }
        const uint64_t i = (i0 * n[1] + i1) * n[2] + i2;
        float rec;
        uint16_t code = ora_quantize(xs[i], acc, e, inv2, twoe, &rec);
        r[i] = rec;
        hist[code]++;
        if (code == 0) (*nout)++;
      }
  free(r);
}

uint64_t ora_blockmap_size(int ndim, const uint64_t* dims, int bs) {
  if (bs < 1 || ndim < 1 || ndim > 3) return 0;
  uint64_t t = 1;
  for (int d = 0; d < ndim; ++d) t *= (dims[d] + (uint64_t)bs - 1) / (uint64_t)bs;
  return t;
}

int ora_tune(const float* x, int ndim, const uint64_t* dims, int eb_mode,
             double eb, const ora_tune_params* tp_in, ora_config* out,
             uint8_t* blockmap, uint64_t blockmap_cap, ora_tune_report* rep) {
  ora_tune_params tpd;
  if (!tp_in) {
    ora_default_tune_params(&tpd);
    tp_in = &tpd;
  }
  const ora_tune_params* tp = tp_in;
  if (!x || !dims || !out || ndim < 1 || ndim > 3) return ORA_ERR_INVALID_ARG;
  if (eb_mode != ORA_EB_ABS && eb_mode != ORA_EB_REL) return ORA_ERR_INVALID_ARG;
  if (!(eb > 0.0) || !isfinite(eb)) return ORA_ERR_INVALID_ARG;
  if (tp->block_size < 1 || !(tp->sample_rate > 0.0) || !(tp->block_rate > 0.0) ||
      !(tp->sub_frac > 0.0) || tp->sub_frac > 1.0)
    return ORA_ERR_INVALID_ARG;
  if (tp->tune_blockwise &&
      (!blockmap || blockmap_cap < ora_blockmap_size(ndim, dims, tp->block_size)))
    return ORA_ERR_OUT_TOO_SMALL;
  if (rep) memset(rep, 0, sizeof(*rep));
  ora_default_config(ndim, out);
  if (tp->anchor_stride) out->anchor_stride = tp->anchor_stride;
  geom g0;
  int rc = geom_init(&g0, ndim, dims, out->anchor_stride, -1);
  if (rc) return rc;
  const uint64_t N = g0.N;
  /* absolute bound exactly as compress derives it */
  float e;
  if (eb_mode == ORA_EB_REL) {
    float vmin = x[0], vmax = x[0];
    for (uint64_t i = 0; i < N; ++i) {
      if (!isfinite(x[i])) return ORA_ERR_NONFINITE;
      if (x[i] < vmin) vmin = x[i];
      if (x[i] > vmax) vmax = x[i];
    }
    double range = (double)vmax - (double)vmin;
    if (range == 0.0) return ORA_OK; /* constant field: nothing to tune */
    e = (float)(eb * range);
  } else {
    e = (float)eb;
  }
  if (!(e > 0.0f) || !isfinite(e)) return ORA_ERR_INVALID_ARG;
  const double inv_e = 1.0 / (double)e;

  /* a11: statistics on a uniform lattice (Sec. 6.1): MSE of linear and
   * cubic interpolation along every dim at points with all +-3 neighbours */
  int t = 1;
  for (;;) {
    double p = 1.0;
    for (int d = 0; d < ndim; ++d) p *= (double)t;
    if (p * tp->sample_rate >= 1.0) break;
    t++;
  }
  uint64_t cnt = 0, lin[3] = {0, 0, 0}, cub[3] = {0, 0, 0};
  {
    uint64_t n[3] = {1, 1, 1}, st[3];
    const int off = 3 - ndim;
    for (int d = 0; d < ndim; ++d) n[d + off] = dims[d];
    st[2] = 1;
    st[1] = n[2];
    st[0] = n[1] * n[2];
    int ok = 1;
    for (int d = 0; d < ndim; ++d)
      if (dims[d] < 7) ok = 0;
    if (ok) {
      uint64_t c[3];
      uint64_t lo[3], step[3];
      for (int sl = 0; sl < 3; ++sl) {
        lo[sl] = sl < off ? 0 : 3;
        step[sl] = sl < off ? 1 : (uint64_t)t;
      }
      for (c[0] = lo[0]; c[0] + (off > 0 ? 0 : 3) < n[0]; c[0] += step[0])
        for (c[1] = lo[1]; c[1] + (off > 1 ? 0 : 3) < n[1]; c[1] += step[1])
          for (c[2] = lo[2]; c[2] + 3 < n[2]; c[2] += step[2]) {
            const uint64_t i = c[0] * st[0] + c[1] * st[1] + c[2];
            cnt++;
            for (int d = 0; d < ndim; ++d) {
              const uint64_t s = st[d + off];
              float v[7] = {0, 0, 0, 0, 0, 0, 0};
              v[0] = x[i - 3 * s];
              v[2] = x[i - s];
              v[4] = x[i + s];
              v[6] = x[i + 3 * s];
              const float pc = eval_formula(F_NAK4, v);
              const float pl = eval_formula(F_LIN, v);
              cub[d] += sq_fixed(x[i] - pc, inv_e);
              lin[d] += sq_fixed(x[i] - pl, inv_e);
            }
          }
    }
  }
  double inv_var[3] = {1.0, 1.0, 1.0};
  int nonsmooth = -1;
  if (cnt) {
    uint64_t mx = 0;
    for (int d = 0; d < ndim; ++d) {
      inv_var[d] = (double)cnt * 256.0 / (double)(cub[d] ? cub[d] : 1);
      if (nonsmooth < 0 || cub[d] > mx) {
        mx = cub[d];
        nonsmooth = d;
      }
    }
  }
  if (rep) {
    rep->stats_count = cnt;
    for (int d = 0; d < 3; ++d) {
      rep->mse_lin[d] = lin[d];
      rep->mse_cub[d] = cub[d];
    }
    rep->nonsmooth_dim = nonsmooth;
    rep->froze = 0;
  }

  /* a12 + a13 without freezing, and (a14) with the most non-smooth dim
   * frozen; the smaller sample estimate wins */
  ora_config cfg_nf, cfg_f;
  uint64_t bits_nf = tune_global(x, ndim, dims, e, tp, -1, inv_var, &cfg_nf, rep, 0);
  *out = cfg_nf;
  uint64_t bits_best = bits_nf;
  if (tp->tune_freeze && cnt && ndim >= 2) {
    uint64_t bits_f = tune_global(x, ndim, dims, e, tp, nonsmooth, inv_var, &cfg_f, rep, 1);
    if (bits_f < bits_nf) {
      *out = cfg_f;
      bits_best = bits_f;
      if (rep) rep->froze = 1;
    }
  }

  /* a15: Lorenzo test on the same sample blocks */
  if (tp->tune_lorenzo) {
    blockset bs;
    sample_blocks(x, ndim, dims, out->anchor_stride, tp->block_rate, &bs);
    uint64_t lb[2];
    for (int o = 1; o <= 2; ++o) {
      uint64_t* hist = (uint64_t*)calloc(65536, sizeof(uint64_t));
      uint64_t nout = 0;
      for (int b = 0; b < bs.nblk; ++b)
        lorenzo_test(bs.xs[b], ndim, bs.ds[b], o, e, hist, &nout);
      lb[o - 1] = huff_cost(hist) + 32 * nout;
      free(hist);
    }
    free_blocks(&bs);
    const uint64_t m = lb[0] <= lb[1] ? lb[0] : lb[1];
    const int better = (double)m * tp->lorenzo_coef < (double)bits_best;
    if (rep) {
      rep->lorenzo_bits[0] = lb[0];
      rep->lorenzo_bits[1] = lb[1];
      rep->lorenzo_better = better;
    }
    /* the selection (Sec. 6.5): the Lorenzo predictor of the order with
     * the smaller estimate (order 1 on a tie) when it beats interpolation;
     * the block-wise interpolation tuning then does not apply */
    if (better) {
      out->predictor = lb[0] <= lb[1] ? 1 : 2;
      return ORA_OK;
    }
  }

  /* a16: block-wise interpolator choice on a centred sub-block per block */
  if (tp->tune_blockwise) {
    const int bsz = tp->block_size;
    const uint64_t nbt = ora_blockmap_size(ndim, dims, bsz);
    double q0 = 32.0 * pow(tp->sub_frac, 1.0 / (double)ndim);
    int Q = (int)floor((double)bsz / 32.0 * q0 + 0.5);
    if (Q < 5) Q = 5;
    uint64_t nb[3];
    for (int d = 0; d < ndim; ++d) nb[d] = (dims[d] + (uint64_t)bsz - 1) / (uint64_t)bsz;
    static const uint8_t cand_code[5] = {0, 1, 5, 2, 6};
    for (uint64_t b = 0; b < nbt; ++b) {
      uint64_t r = b, start[3], ext[3];
      uint64_t qmin = UINT64_MAX;
      for (int d = ndim - 1; d >= 0; --d) {
        const uint64_t j = r % nb[d];
        r /= nb[d];
        const uint64_t bstart = j * (uint64_t)bsz;
        const uint64_t bext = dims[d] - bstart < (uint64_t)bsz ? dims[d] - bstart : (uint64_t)bsz;
        const uint64_t q = bext < (uint64_t)Q ? bext : (uint64_t)Q;
        start[d] = bstart + (bext - q) / 2;
        ext[d] = q;
        if (d != out->frozen_dim && q < qmin) qmin = q;
      }
      int As = 2;
      while ((uint64_t)(As * 2) <= (qmin > 1 ? qmin - 1 : 1)) As *= 2;
      float* xs = extract(x, ndim, dims, start, ext);
      uint64_t best = UINT64_MAX;
      int bj = 0;
      for (int j = 0; j < 5; ++j) {
        const uint8_t v = cand_code[j];
        if ((v & 3) == ORA_CUBIC_NAT && !tp->allow_natural) continue;
        if ((v & 4) && !tp->allow_same_level) continue;
        ora_config c2 = *out;
        c2.anchor_stride = As;
        c2.blockwise = 0;
        for (int l = 0; l < ORA_MAX_LEVELS; ++l) {
          c2.interp[l] = v & 3;
          c2.same_level[l] = (v >> 2) & 1;
        }
        uint64_t sc[ORA_MAX_LEVELS] = {0};
        ora_subfield_test(xs, ndim, ext, &c2, e, 1, sc, NULL, NULL, NULL);
        uint64_t tot = 0;
        for (int l = 0; l < ORA_MAX_LEVELS; ++l) tot += sc[l];
        if (tot < best) {
          best = tot;
          bj = j;
        }
      }
      blockmap[b] = cand_code[bj];
      free(xs);
    }
    out->blockwise = 1;
    out->block_size = bsz;
    out->blockmap = blockmap;
  }
  return ORA_OK;
}

/* ================================================================== */
/* Quality-metric target (Sec. 3.1, Eq. 1 with M = PSNR) and integer    */
/* inputs.  Both wrap the method above; the arithmetic they add is the  */
/* metric and the bound search (in double), and the integer widening    */
/* and rounding.                                                        */
/* ================================================================== */

int ora_psnr(const float* x, const float* y, uint64_t n, double unit,
             double* psnr, uint64_t* sse) {
  if (!x || !y || n == 0 || !(unit > 0.0) || !isfinite(unit)) return ORA_ERR_INVALID_ARG;
  double vmin = (double)x[0], vmax = (double)x[0];
  uint64_t acc = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const double xv = (double)x[i];
    if (!isfinite(xv)) return ORA_ERR_NONFINITE;
    if (xv < vmin) vmin = xv;
    if (xv > vmax) vmax = xv;
    const double q = rint((xv - (double)y[i]) / unit);
    if (!(fabs(q) <= 65536.0)) return ORA_ERR_INVALID_ARG;
    const int64_t iq = (int64_t)q;
    acc += (uint64_t)(iq * iq);
  }
  if (sse) *sse = acc;
  if (psnr) {
    if (acc == 0) {
      *psnr = INFINITY;
    } else {
      const double mse = (double)acc * unit * unit / (double)n;
      *psnr = 20.0 * log10(vmax - vmin) - 10.0 * log10(mse);
    }
  }
  return ORA_OK;
}

typedef struct {
  const float* x;
  int ndim;
  const uint64_t* dims;
  const ora_tune_params* tp;
  uint64_t n, cap;
  uint8_t* buf;
  float* y;
} psnr_probe;

/* one probe of the search: tune + compress at absolute bound e, decompress,
 * PSNR; the stream stays in p->buf */
static int probe_psnr(psnr_probe* p, double e, uint64_t* size, double* psnr) {
  ora_config cfg;
  uint8_t* bm = (uint8_t*)malloc(ora_blockmap_size(p->ndim, p->dims,
                                                   p->tp ? p->tp->block_size : 32) + 1);
  int rc = ora_tune(p->x, p->ndim, p->dims, ORA_EB_ABS, e, p->tp, &cfg, bm,
                    ora_blockmap_size(p->ndim, p->dims, p->tp ? p->tp->block_size : 32) + 1,
                    NULL);
  ora_stats st;
  if (!rc)
    rc = ora_compress(p->x, p->ndim, p->dims, ORA_EB_ABS, e, &cfg, p->buf, p->cap, size,
                      NULL, NULL, &st);
  free(bm);
  if (!rc) rc = ora_decompress(p->buf, *size, p->y, p->n);
  if (!rc) rc = ora_psnr(p->x, p->y, p->n, (double)st.e / 65536.0, psnr, NULL);
  return rc;
}

int ora_compress_psnr(const float* x, int ndim, const uint64_t* dims,
                      double target_db, const ora_tune_params* tp, uint8_t* out,
                      uint64_t cap, uint64_t* out_size, double* eb_out,
                      double* psnr_out) {
  if (!x || !dims || !out || !out_size || ndim < 1 || ndim > 3 || !isfinite(target_db))
    return ORA_ERR_INVALID_ARG;
  uint64_t n = 1;
  for (int d = 0; d < ndim; ++d) n *= dims[d];
  if (n == 0) return ORA_ERR_INVALID_ARG;
  double vmin = (double)x[0], vmax = (double)x[0];
  for (uint64_t i = 0; i < n; ++i) {
    if (!isfinite(x[i])) return ORA_ERR_NONFINITE;
    if ((double)x[i] < vmin) vmin = (double)x[i];
    if ((double)x[i] > vmax) vmax = (double)x[i];
  }
  psnr_probe p = {x, ndim, dims, tp, n, ora_compress_bound(ndim, dims), NULL, NULL};
  p.buf = (uint8_t*)malloc(p.cap);
  p.y = (float*)malloc(sizeof(float) * n);
  int rc = ORA_OK;
  uint64_t size = 0;
  double ps = 0.0;
  double lo, hi;
  const double range = vmax - vmin;
  /* a constant field: any bound keeps it exact */
  double e = range > 0.0 ? range * sqrt(3.0) * pow(10.0, -target_db / 20.0) : 1.0;
  if (!(e > 0.0) || !isfinite(e)) rc = ORA_ERR_INVALID_ARG;
  int found = 0;
  if (!rc) rc = probe_psnr(&p, e, &size, &ps);
  if (!rc && ps >= target_db) {
    lo = e;
    hi = 2.0 * e;
    found = 1;
    int g;
    for (g = 0; g < 6 && !rc; ++g) {
      rc = probe_psnr(&p, hi, &size, &ps);
      if (rc || ps < target_db) break;
      lo = hi;
      hi = 2.0 * hi;
    }
    if (!rc && g == 6) hi = 0.0; /* the target holds at every bound tried */
  } else if (!rc) {
    hi = e;
    lo = 0.5 * e;
    int g;
    for (g = 0; g < 6 && !rc; ++g) {
      rc = probe_psnr(&p, lo, &size, &ps);
      if (rc || ps >= target_db) break;
      hi = lo;
      lo = 0.5 * lo;
    }
    found = !rc && g < 6;
    if (!found) hi = 0.0;
  }
  if (!rc && hi > 0.0) {
    for (int it = 0; it < 8 && !rc; ++it) {
      const double mid = sqrt(lo * hi);
      rc = probe_psnr(&p, mid, &size, &ps);
      if (rc) break;
      if (ps >= target_db)
        lo = mid;
      else
        hi = mid;
    }
  }
  if (!rc) {
    if (!found) lo = lo * 2.0; /* the smallest bound tried */
    rc = probe_psnr(&p, lo, &size, &ps);
  }
  if (!rc) {
    if (size > cap) {
      rc = ORA_ERR_OUT_TOO_SMALL;
    } else {
      memcpy(out, p.buf, size);
      *out_size = size;
      if (eb_out) *eb_out = lo;
      if (psnr_out) *psnr_out = ps;
    }
  }
  free(p.buf);
  free(p.y);
  return rc;
}

static int dtype_ok(int dtype) {
  return dtype == ORA_DTYPE_F32 || dtype == ORA_DTYPE_I16 || dtype == ORA_DTYPE_U16 ||
         dtype == ORA_DTYPE_I32;
}

int ora_compress_typed(const void* x, int dtype, int ndim, const uint64_t* dims,
                       int eb_mode, double eb, const ora_config* cfg, int tune,
                       const ora_tune_params* tp, uint8_t* out, uint64_t cap,
                       uint64_t* out_size) {
  if (!x || !dims || !out || !out_size || ndim < 1 || ndim > 3 || !dtype_ok(dtype))
    return ORA_ERR_INVALID_ARG;
  if (eb_mode != ORA_EB_ABS && eb_mode != ORA_EB_REL) return ORA_ERR_INVALID_ARG;
  uint64_t n = 1;
  for (int d = 0; d < ndim; ++d) n *= dims[d];
  if (n == 0) return ORA_ERR_INVALID_ARG;
  float* xf = (float*)malloc(sizeof(float) * n);
  double vmin = 0.0, vmax = 0.0;
  int rc = ORA_OK;
  for (uint64_t i = 0; i < n && !rc; ++i) {
    double v;
    switch (dtype) {
      case ORA_DTYPE_I16: v = (double)((const int16_t*)x)[i]; break;
      case ORA_DTYPE_U16: v = (double)((const uint16_t*)x)[i]; break;
      case ORA_DTYPE_I32:
        v = (double)((const int32_t*)x)[i];
        if (fabs(v) > 16777216.0) rc = ORA_ERR_INVALID_ARG;
        break;
      default: v = (double)((const float*)x)[i]; break;
    }
    xf[i] = (float)v;
    if (i == 0 || v < vmin) vmin = v;
    if (i == 0 || v > vmax) vmax = v;
  }
  int mode = eb_mode;
  double e = eb;
  if (!rc && dtype != ORA_DTYPE_F32) {
    /* the integer bound and the float bound that keeps the rounded
     * reconstruction within it */
    const double ei = eb_mode == ORA_EB_REL ? eb * (vmax - vmin) : eb;
    if (!(ei >= 0.0) || !isfinite(ei) || ei > 4194304.0) {
      rc = ORA_ERR_INVALID_ARG;
    } else {
      e = (double)nextafterf((float)(floor(ei) + 0.5), 0.0f);
      mode = ORA_EB_ABS;
    }
  }
  ora_config tc;
  uint8_t* bm = NULL;
  if (!rc && tune) {
    const uint64_t nbm = ora_blockmap_size(ndim, dims, tp ? tp->block_size : 32) + 1;
    bm = (uint8_t*)malloc(nbm);
    rc = ora_tune(xf, ndim, dims, mode, e, tp, &tc, bm, nbm, NULL);
    cfg = &tc;
  }
  if (!rc) rc = ora_compress(xf, ndim, dims, mode, e, cfg, out, cap, out_size, NULL, NULL, NULL);
  if (!rc) put_u32(out, ORA_H_DTYPE, (uint32_t)dtype);
  free(bm);
  free(xf);
  return rc;
}

int ora_decompress_typed(const uint8_t* in, uint64_t size, void* out, int dtype,
                         uint64_t cap_elems) {
  if (!in || !out || !dtype_ok(dtype) || size < ORA_HEADER_BYTES) return ORA_ERR_INVALID_ARG;
  if ((int)get_u32(in, ORA_H_DTYPE) != dtype) return ORA_ERR_INVALID_ARG;
  int ndim;
  uint64_t dims[3];
  int rc = ora_inspect(in, size, &ndim, dims, NULL);
  if (rc) return rc;
  uint64_t n = 1;
  for (int d = 0; d < ndim; ++d) n *= dims[d];
  if (n > cap_elems) return ORA_ERR_OUT_TOO_SMALL;
  float* y = (float*)malloc(sizeof(float) * (n ? n : 1));
  rc = ora_decompress(in, size, y, n);
  for (uint64_t i = 0; i < n && !rc; ++i) {
    float r = rintf(y[i]);
    switch (dtype) {
      case ORA_DTYPE_I16:
        r = fminf(fmaxf(r, -32768.0f), 32767.0f);
        ((int16_t*)out)[i] = (int16_t)r;
        break;
      case ORA_DTYPE_U16:
        r = fminf(fmaxf(r, 0.0f), 65535.0f);
        ((uint16_t*)out)[i] = (uint16_t)r;
        break;
      case ORA_DTYPE_I32:
        ((int32_t*)out)[i] = (int32_t)r;
        break;
      default:
        ((float*)out)[i] = y[i];
        break;
    }
  }
  free(y);
  return rc;
}

/* ================================================================== */
/* The lossless stage (Sec. 4, Step 5): run suppression of repeated     */
/* 32-bit words of the stream body, two levels of masks.                */
/* ================================================================== */

static uint32_t body_word(const uint8_t* b, uint64_t nbytes, uint64_t i) {
  uint32_t v = 0;
  for (int k = 0; k < 4; ++k) {
    const uint64_t o = 4 * i + (uint64_t)k;
    if (o < nbytes) v |= (uint32_t)b[o] << (8 * k);
  }
  return v;
}

int ora_lossless_encode(const uint8_t* in, uint64_t size, uint8_t* out, uint64_t cap,
                        uint64_t* out_size) {
  if (!in || !out || !out_size || size < ORA_HEADER_BYTES) return ORA_ERR_INVALID_ARG;
  if (get_u32(in, H_FLAGS) & FLAG_LOSSLESS) return ORA_ERR_INVALID_ARG;
  const uint8_t* body = in + ORA_HEADER_BYTES;
  const uint64_t nbytes = size - ORA_HEADER_BYTES;
  const uint64_t nw = (nbytes + 3) / 4, nb = (nw + 31) / 32, ng = (nb + 31) / 32;
  uint32_t* m1 = (uint32_t*)calloc(nb ? nb : 1, 4);
  uint32_t* m2 = (uint32_t*)calloc(ng ? ng : 1, 4);
  uint64_t nlit = 0, nmask = 0;
  uint32_t prev = 0;
  for (uint64_t i = 0; i < nw; ++i) {
    const uint32_t w = body_word(body, nbytes, i);
    if (w != prev) {
      m1[i / 32] |= 1u << (i % 32);
      ++nlit;
    }
    prev = w;
  }
  for (uint64_t b = 0; b < nb; ++b)
    if (m1[b]) {
      m2[b / 32] |= 1u << (b % 32);
      ++nmask;
    }
  const uint64_t zsize = ORA_HEADER_BYTES + 32 + 4 * (ng + nmask + nlit);
  int rc = ORA_OK;
  if (zsize >= size) {
    /* no gain: the stream stays as it is */
    if (size > cap) {
      rc = ORA_ERR_OUT_TOO_SMALL;
    } else {
      memmove(out, in, size);
      *out_size = size;
    }
  } else if (zsize > cap) {
    rc = ORA_ERR_OUT_TOO_SMALL;
  } else {
    uint8_t* hdr = (uint8_t*)malloc(ORA_HEADER_BYTES);
    memcpy(hdr, in, ORA_HEADER_BYTES);
    put_u32(hdr, H_FLAGS, get_u32(hdr, H_FLAGS) | FLAG_LOSSLESS);
    put_u64(hdr, ORA_H_RAWSIZE, size);
    uint64_t o = ORA_HEADER_BYTES;
    uint8_t* z = out;
    /* literals first into a scratch (the output may alias nothing) */
    uint32_t* lits = (uint32_t*)malloc(4 * (nlit ? nlit : 1));
    uint64_t k = 0;
    prev = 0;
    for (uint64_t i = 0; i < nw; ++i) {
      const uint32_t w = body_word(body, nbytes, i);
      if (w != prev) lits[k++] = w;
      prev = w;
    }
    memcpy(z, hdr, ORA_HEADER_BYTES);
    put_u64(z, o, nw);
    put_u64(z, o + 8, nlit);
    put_u64(z, o + 16, nmask);
    put_u64(z, o + 24, 0);
    o += 32;
    for (uint64_t g = 0; g < ng; ++g, o += 4) put_u32(z, o, m2[g]);
    for (uint64_t b = 0; b < nb; ++b)
      if (m1[b]) {
        put_u32(z, o, m1[b]);
        o += 4;
      }
    for (uint64_t i = 0; i < nlit; ++i, o += 4) put_u32(z, o, lits[i]);
    *out_size = o;
    free(lits);
    free(hdr);
  }
  free(m1);
  free(m2);
  return rc;
}

int ora_lossless_decode(const uint8_t* in, uint64_t size, uint8_t* out, uint64_t cap,
                        uint64_t* out_size) {
  if (!in || !out || !out_size || size < ORA_HEADER_BYTES + 32) return ORA_ERR_INVALID_ARG;
  if (!(get_u32(in, H_FLAGS) & FLAG_LOSSLESS)) return ORA_ERR_INVALID_ARG;
  const uint64_t raw = get_u64(in, ORA_H_RAWSIZE);
  if (raw < ORA_HEADER_BYTES) return ORA_ERR_CORRUPT;
  if (raw > cap) return ORA_ERR_OUT_TOO_SMALL;
  uint64_t o = ORA_HEADER_BYTES;
  const uint64_t nw = get_u64(in, o), nlit = get_u64(in, o + 8), nmask = get_u64(in, o + 16);
  const uint64_t nbytes = raw - ORA_HEADER_BYTES;
  if (nw != (nbytes + 3) / 4 || get_u64(in, o + 24) != 0) return ORA_ERR_CORRUPT;
  const uint64_t nb = (nw + 31) / 32, ng = (nb + 31) / 32;
  if (nmask > nb || nlit > nw || size != ORA_HEADER_BYTES + 32 + 4 * (ng + nmask + nlit))
    return ORA_ERR_CORRUPT;
  o += 32;
  const uint64_t om = o + 4 * ng, ol = om + 4 * nmask;
  uint64_t km = 0, kl = 0;
  uint32_t prev = 0;
  memcpy(out, in, ORA_HEADER_BYTES);
  put_u32(out, H_FLAGS, get_u32(in, H_FLAGS) & ~FLAG_LOSSLESS);
  put_u64(out, ORA_H_RAWSIZE, 0);
  for (uint64_t b = 0; b < nb; ++b) {
    const uint32_t g = get_u32(in, o + 4 * (b / 32));
    uint32_t m = 0;
    if ((g >> (b % 32)) & 1u) {
      if (km >= nmask) return ORA_ERR_CORRUPT;
      m = get_u32(in, om + 4 * km++);
      if (!m) return ORA_ERR_CORRUPT;
    }
    for (uint64_t j = 0; j < 32 && 32 * b + j < nw; ++j) {
      if ((m >> j) & 1u) {
        if (kl >= nlit) return ORA_ERR_CORRUPT;
        prev = get_u32(in, ol + 4 * kl++);
      }
      const uint64_t i = 32 * b + j;
      for (int q = 0; q < 4; ++q) {
        const uint64_t ob = 4 * i + (uint64_t)q;
        if (ob < nbytes) out[ORA_HEADER_BYTES + ob] = (uint8_t)(prev >> (8 * q));
      }
    }
  }
  if (km != nmask || kl != nlit) return ORA_ERR_CORRUPT;
  *out_size = raw;
  return ORA_OK;
}
