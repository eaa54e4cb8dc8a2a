// hpez_internal.cuh -- device-side building blocks of the HPEZ sweep.
//
// Every binary32 operation of the prediction and quantization runs through
// an explicit round-to-nearest intrinsic (__fadd_rn, __fmul_rn, ...), which
// the compiler never contracts into FMA, so the results are reproducible
// bit for bit on any IEEE-754 machine that performs the same operations in
// the same order.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hpez {

constexpr int kMaxLevels = 16;
constexpr int kRadius = 32768;
constexpr int kHeaderBytes = 512;

enum Interp { LINEAR = 0, CUBIC_NAK = 1, CUBIC_NAT = 2 };

// status codes written by kernels (mirror the C-ABI error codes)
enum DevStatus {
  ST_OK = 0,
  ST_INVALID = -1,
  ST_NONFINITE = -2,
  ST_OUT_TOO_SMALL = -3,
  ST_CORRUPT = -4,
  ST_TIMEOUT = -9,
};

// Per-call control block in device memory.
struct Ctl {
  unsigned int vmin_key, vmax_key;  // order-preserving float keys
  int nonfinite;
  int is_const;
  int status;
  int pad0;
  float e;
  float const_value;
  float el[kMaxLevels], inv2[kMaxLevels], twoe[kMaxLevels];
  unsigned long long n_out;
  unsigned long long total_words;
  unsigned long long off_table, off_outliers, off_bits, total_size;
  unsigned int n_used;
  unsigned int max_len;
  unsigned long long dbg[4];
};

// ---------------------------------------------------------------------
// order-preserving float <-> uint key (for atomic min/max)
// ---------------------------------------------------------------------
__device__ __forceinline__ unsigned int f2key(float f) {
  unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(unsigned int k) {
  unsigned int u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

// ---------------------------------------------------------------------
// Stencils along one line (Sec. 5.2 Eq. 2/4/6, Sec. 5.4.2 Eq. 10/11) and
// the boundary fallbacks (spline through the available knots, linear
// extrapolation with no right neighbour, copy as the last resort).
// Neighbour offsets are in units of the level stride; slot j+3 of the
// value array holds offset j.
// ---------------------------------------------------------------------
enum Formula {
  F_COPY, F_EXTRAP, F_LIN, F_NAK4, F_NAT4, F_NAK3L, F_NAK3R, F_NAT3L,
  F_NAT3R, F_SL_NAK, F_SL_NAT
};

// Chooses the stencil from which neighbours exist along the line.
// u: position (in stride units) of the point, m: number of grid points on
// the line, so offset j exists iff 0 <= u + j <= m - 1.  u is odd >= 1,
// hence offset -1 always exists.
__device__ __forceinline__ int choose_formula(int kind, bool half_b, int u,
                                              int m) {
  const bool hm3 = u >= 3, hm2 = u >= 2;
  const bool hp1 = u + 1 <= m - 1, hp2 = u + 2 <= m - 1,
             hp3 = u + 3 <= m - 1;
  if (half_b) {
    if (kind == CUBIC_NAK && hp1 && hm2 && hp2) return F_SL_NAK;
    if (kind == CUBIC_NAT && hp1 && hm2 && hp2 && hm3 && hp3) return F_SL_NAT;
  }
  if (!hp1) return hm3 ? F_EXTRAP : F_COPY;
  if (kind == LINEAR) return F_LIN;
  if (hm3 && hp3) return kind == CUBIC_NAK ? F_NAK4 : F_NAT4;
  if (hm3) return kind == CUBIC_NAK ? F_NAK3L : F_NAT3L;
  if (hp3) return kind == CUBIC_NAK ? F_NAK3R : F_NAT3R;
  return F_LIN;
}

// Division by a power of two is exact scaling, so multiplying by the exact
// reciprocal rounds to the same value as the division.
__device__ __forceinline__ float eval_formula(int f, float m3, float m2,
                                              float m1, float p1, float p2,
                                              float p3) {
  switch (f) {
    case F_COPY:
      return m1;
    case F_EXTRAP:  // (3 d-1 - d-3) / 2
      return __fmul_rn(__fsub_rn(__fmul_rn(m1, 3.0f), m3), 0.5f);
    case F_LIN:  // Eq. 2
      return __fmul_rn(__fadd_rn(m1, p1), 0.5f);
    case F_NAK4:  // Eq. 4
      return __fmul_rn(
          __fsub_rn(__fmul_rn(__fadd_rn(m1, p1), 9.0f), __fadd_rn(m3, p3)),
          0.0625f);
    case F_NAT4:  // Eq. 6
      return __fdiv_rn(__fsub_rn(__fmul_rn(__fadd_rn(m1, p1), 23.0f),
                                 __fmul_rn(__fadd_rn(m3, p3), 3.0f)),
                       40.0f);
    case F_NAK3L:  // (-1, 6, 3) / 8
      return __fmul_rn(
          __fsub_rn(__fadd_rn(__fmul_rn(m1, 6.0f), __fmul_rn(p1, 3.0f)), m3),
          0.125f);
    case F_NAK3R:  // (3, 6, -1) / 8
      return __fmul_rn(
          __fsub_rn(__fadd_rn(__fmul_rn(m1, 3.0f), __fmul_rn(p1, 6.0f)), p3),
          0.125f);
    case F_NAT3L:  // (-3, 22, 13) / 32
      return __fmul_rn(
          __fsub_rn(__fadd_rn(__fmul_rn(m1, 22.0f), __fmul_rn(p1, 13.0f)),
                    __fmul_rn(m3, 3.0f)),
          0.03125f);
    case F_NAT3R:  // (13, 22, -3) / 32
      return __fmul_rn(
          __fsub_rn(__fadd_rn(__fmul_rn(m1, 13.0f), __fmul_rn(p1, 22.0f)),
                    __fmul_rn(p3, 3.0f)),
          0.03125f);
    case F_SL_NAK:  // Eq. 10
      return __fdiv_rn(
          __fsub_rn(__fmul_rn(__fadd_rn(m1, p1), 4.0f), __fadd_rn(m2, p2)),
          6.0f);
    case F_SL_NAT:  // Eq. 11
      return __fdiv_rn(
          __fadd_rn(__fsub_rn(__fmul_rn(__fadd_rn(m1, p1), 46.0f),
                              __fmul_rn(__fadd_rn(m2, p2), 18.0f)),
                    __fmul_rn(__fadd_rn(m3, p3), 3.0f)),
          62.0f);
  }
  return 0.0f;
}

// Prediction along one line of a compact grid: `base` points at the
// point's own entry, `st` is the stride of the line in elements.
__device__ __forceinline__ float predict_line(const float* __restrict__ base,
                                              long long st, int u, int m,
                                              int kind, bool half_b) {
  const int f = choose_formula(kind, half_b, u, m);
  float m3 = 0.f, m2 = 0.f, m1 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
  m1 = __ldg(base - st);
  switch (f) {
    case F_COPY:
      break;
    case F_EXTRAP:
      m3 = __ldg(base - 3 * st);
      break;
    case F_LIN:
      p1 = __ldg(base + st);
      break;
    case F_NAK4:
    case F_NAT4:
      m3 = __ldg(base - 3 * st);
      p1 = __ldg(base + st);
      p3 = __ldg(base + 3 * st);
      break;
    case F_NAK3L:
    case F_NAT3L:
      m3 = __ldg(base - 3 * st);
      p1 = __ldg(base + st);
      break;
    case F_NAK3R:
    case F_NAT3R:
      p1 = __ldg(base + st);
      p3 = __ldg(base + 3 * st);
      break;
    case F_SL_NAK:
      m2 = __ldg(base - 2 * st);
      p1 = __ldg(base + st);
      p2 = __ldg(base + 2 * st);
      break;
    case F_SL_NAT:
      m3 = __ldg(base - 3 * st);
      m2 = __ldg(base - 2 * st);
      p1 = __ldg(base + st);
      p2 = __ldg(base + 2 * st);
      p3 = __ldg(base + 3 * st);
      break;
  }
  return eval_formula(f, m3, m2, m1, p1, p2, p3);
}

// ---------------------------------------------------------------------
// Linear quantization (Sec. 4 Step 3) with the exact bound check:
// |r - x| <= e decided from rn(r - x) and its TwoSum residual.
// ---------------------------------------------------------------------
__device__ __forceinline__ bool within_bound(float r, float x, float e) {
  const float nx = -x;
  const float d = __fadd_rn(r, nx);
  const float bb = __fsub_rn(d, r);
  const float res = __fadd_rn(__fsub_rn(r, __fsub_rn(d, bb)), __fsub_rn(nx, bb));
  const float ad = fabsf(d);
  if (ad < e) return true;
  if (ad == e) {
    if (d > 0.0f) return res <= 0.0f;
    if (d < 0.0f) return res >= 0.0f;
  }
  return false;
}

// Returns the code word (q + radius, or 0 = unpredictable) and the
// reconstructed value.
__device__ __forceinline__ unsigned quantize(float x, float p, float el,
                                             float inv2, float twoe,
                                             float& recon) {
  const float diff = __fsub_rn(x, p);
  const float m = __fadd_rn(__fmul_rn(fabsf(diff), inv2), 0.5f);
  if (m < 32768.0f) {
    const int k = __float2int_rz(m);
    const int q = diff < 0.0f ? -k : k;
    const float r = __fadd_rn(p, __fmul_rn(__int2float_rn(q), twoe));
    if (within_bound(r, x, el)) {
      recon = r;
      return (unsigned)(q + kRadius);
    }
  }
  recon = x;
  return 0u;
}

// quantize() with a fast accept: rn(r - x) strictly inside the bound
// implies the exact difference is inside too (rounding is monotonic), so
// the TwoSum residual of within_bound is only needed near the bound
__device__ __forceinline__ unsigned quantize_fast(float x, float p, float el, float inv2,
                                                  float twoe, float& recon) {
  const float diff = __fsub_rn(x, p);
  const float m = __fadd_rn(__fmul_rn(fabsf(diff), inv2), 0.5f);
  if (m < 32768.0f) {
    const int k = __float2int_rz(m);
    const int q = diff < 0.0f ? -k : k;
    const float r = __fadd_rn(p, __fmul_rn(__int2float_rn(q), twoe));
    if (fabsf(__fsub_rn(r, x)) < el || within_bound(r, x, el)) {
      recon = r;
      return (unsigned)(q + kRadius);
    }
  }
  recon = x;
  return 0u;
}

__device__ __forceinline__ float dequantize(unsigned code, float p,
                                            float twoe) {
  const int q = (int)code - kRadius;
  return __fadd_rn(p, __fmul_rn(__int2float_rn(q), twoe));
}

// ---------------------------------------------------------------------
// Sweep geometry: every field is 3 slots (real dims in the last ndim
// slots).  A level's compact grid G_s keeps the points whose coordinate is
// a multiple of s on every interpolation slot.
// ---------------------------------------------------------------------
struct LevelGeom {
  uint32_t m[3];     // G_s extent per slot
  uint32_t gst[3];   // G_s element strides
  uint32_t step[3];  // full-field coordinate step per G_s index (s or 1)
  uint32_t fst[3];   // full-field element strides
};

// One launch of the sweep: a box of G_s indices u_d = a_d + b_d * t_d.
struct PassBox {
  uint32_t a[3], b[3], cnt[3];
  uint32_t total;
  uint32_t S;        // slots predicted along (bit per slot)
  float w[3];        // multi-dimensional weights per slot (Eq. 8 / Eq. 14)
  int md;            // 1: weighted sum over S, 0: single slot in S
  int half;          // same-level half processed by this launch
  int level;         // l >= 1
  int write_recon;   // compress: store the reconstruction
};

struct SweepBufs {
  const float* x;              // compress: full input
  float* R;                    // G_s reconstruction
  uint16_t* C;                 // compress: G_s codes
  const uint16_t* codes_full;  // decompress: full-field codes
  const float* outl_full;      // decompress: outliers scattered (full)
  const uint8_t* blockmap;     // per-block interpolator (or null)
  uint32_t bs;                 // block side
  uint32_t nb[3];              // blocks per slot
  int kind, same;              // level interpolator when no block map
  const Ctl* ctl;
};

// One step of the fused level kernel: a pass (or one same-level half of
// it) over a box of the level grid given relative to the tile origin.
struct FusedStep {
  int8_t par[3];   // per slot: 0 any parity, 1 odd, 2 even
  int8_t dim;      // slot predicted along
  int8_t half;     // same-level half processed
  int8_t pad_[3];  // pad_[0]: every neighbour read lies in the region
  int16_t lo[3], hi[3];
};

struct FusedLevel {
  LevelGeom g, gc;      // this level's grid and the coarse grid
  uint32_t E[3];        // tile extents
  int32_t rlo[3], rhi[3];  // shared-memory region relative to the tile
  uint32_t RX[3];       // region extents (rhi - rlo)
  uint32_t ntile[3];
  uint32_t ntiles;
  int interp[3];        // slot is an interpolation dimension
  int nsteps;
  FusedStep st[6];
  int level;
  int write_recon;
  int stage_x;   // compress: 1 = 4-byte async copies of the input, 2 = 16-byte;
                 // decompress: 1 = 16-byte async copies of the codes; 0 = none
};

// The dedicated 3D level kernel (direction order 0,1,2, one interpolator,
// no same-level halves): tiles of 2 planes x E1 rows x whole rows.
struct Level3D {
  int m[3];          // level grid extents
  int E1;            // tile rows
  int W;             // shared-memory row length (m[2] rounded up to 8)
  int nt0, nt1;      // tiles along dims 0 and 1
  uint32_t fs0, fs1, fs2;  // full-field element strides of level-grid steps
  uint32_t cst0, cst1;     // coarse-grid strides
  int level;
  int write_recon;
  int stage16;       // compress: input rows staged with 16-byte copies
  int stage_codes;   // decompress: code rows staged (16-byte copies)
  int vec_out;       // rows of the output grids start 16-byte aligned
};

// One level of the multi-dimensional paradigm (one launch per sub-pass).
struct LevelMD {
  LevelGeom g, gc;     // level grid, coarse grid
  uint32_t nc[3];      // cells per slot (coarse extent; the extent on a
                       // non-interpolation slot)
  uint32_t fst[3];     // full-field strides
  int interp[3];
  int k;               // interpolation slots = sub-passes
  int level, write_recon;
  int nmask[3];        // odd sets of sub-pass k' (index k'-1)
  uint8_t masks[3][3];
  float w[8][3];       // Eq. 14 weight per odd set and slot
};

// ---------------------------------------------------------------------
// Auto-tuner (Sec. 6): one theta of a compression test, and the geometry
// of the sub-fields the tests run on.
// ---------------------------------------------------------------------
// one candidate of a level's tests: the level's fields of a theta (the
// 1D-style order as slots)
struct TuneCand {
  uint8_t kind, md, same, ord[3];
};

struct TuneCfg {
  uint8_t kind[kMaxLevels];   // interpolator per level (l-1)
  uint8_t md[kMaxLevels];     // 1: multi-dimensional paradigm
  uint8_t same[kMaxLevels];   // same-level interpolation
  uint8_t ord[kMaxLevels][3]; // 1D-style order as slots
  double alpha, beta;         // Eq. 15 (the device fills el/inv2/twoe)
  float el[kMaxLevels], inv2[kMaxLevels], twoe[kMaxLevels];
  float inv_el[kMaxLevels];   // (float)(1 / e_l) for the error scores
  float mdw[8][3];            // Eq. 14 weight per odd-slot mask and slot
};

struct TuneGeom {
  uint32_t n[3];     // field extents per slot (padded slots 1)
  uint32_t fst[3];   // field strides
  int interp[3];     // interpolation slots
  int k;             // number of interpolation slots
  int off;           // padded slots (3 - ndim)
  int A, L;          // anchor stride, levels
  uint32_t ext[3];   // sample-block extents
  uint32_t cnt[3];   // sample blocks per slot
  uint32_t step[3];  // start offset between sample blocks per slot
};

// ---------------------------------------------------------------------
// Batched work lists.  A batched launch runs one stage for many fields:
// job j owns the launch's blocks [off[j], off[j+1]), and its block
// blockIdx.x - off[j] plays the role the block index plays in the
// single-field launch.  Single-CTA stages run one block per job.
// ---------------------------------------------------------------------
__device__ __forceinline__ int batch_job_of(const uint32_t* __restrict__ off,
                                            int nj, uint32_t b) {
  int lo = 0, hi = nj - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int batch_job(const uint32_t* __restrict__ off,
                                         int nj) {
  return batch_job_of(off, nj, blockIdx.x);
}

// Persistent batched launch: the grid holds at most the CTAs resident on
// the GPU at once, and CTA c walks the launch's virtual blocks c,
// c + gridDim.x, ... (job j owns virtual blocks [off[j], off[j+1])).  The
// barrier between two virtual blocks keeps the next one from overwriting
// shared memory the previous one still reads; every thread of a CTA walks
// the same sequence, so the barrier is reached by all.
template <class Body>
__device__ __forceinline__ void for_each_batch_block(const uint32_t* __restrict__ off,
                                                     int nj, Body body) {
  const uint32_t total = __ldg(off + nj);
  for (uint32_t v = blockIdx.x; v < total; v += gridDim.x) {
    if (v != blockIdx.x) __syncthreads();
    const int j = batch_job_of(off, nj, v);
    body(j, v - __ldg(off + j));
  }
}

struct InitJob { Ctl* ctl; };
struct RangeJob { const float* x; uint32_t N; Ctl* ctl; };
struct ParamsJob {
  Ctl* ctl; int eb_mode; int L; double eb, alpha, beta; const float* x;
};
struct AnchorJob {
  const float* x; LevelGeom ga; uint32_t total; float* RA; uint16_t* CA;
  const Ctl* ctl;
};
struct FillJob { float* out; uint32_t N; float v; };
struct ZeroJob { void* ptr; unsigned long long bytes; };
struct UpsampleJob {
  LevelGeom gc; uint32_t total_c; LevelGeom gs; const float* Rc;
  const uint16_t* Cc; float* Rs; uint16_t* Cs; const Ctl* ctl;
};
struct PassJob { LevelGeom g; PassBox pb; SweepBufs B; };
// a request's outcome: status (0 or a negative error) and stream size
struct ResultJob {
  const Ctl* ctl; const unsigned long long* tot;  // decompress: counters
  unsigned long long twords, nout;                // decompress: expected
  unsigned long long* size_out; int* status_out; int decomp;
};
struct Level3DJob {
  Level3D P; const float* X; const uint16_t* codes_full; const float* outl_full;
  const float* Rc; const uint16_t* Cc; float* Rs; uint16_t* Cs; const Ctl* ctl;
};
struct LevelJob {
  FusedLevel P; SweepBufs B; const float* Rc; const uint16_t* Cc; float* Rs;
  uint16_t* Cs;
};
// a 3D multi-dimensional level: even planes, then odd planes, in tiles of
// E1 rows (nt1 tiles per plane)
struct MD3Job {
  LevelMD P; int E1, nt1; const float* X; const uint16_t* codes_full;
  const float* outl_full; const float* Rc; const uint16_t* Cc; float* Rs;
  uint16_t* Cs; const Ctl* ctl;
};
// the Lorenzo pass (Sec. 6.5) over one field of blocks of side A
struct LorGeom {
  uint32_t n[3];     // field extents per slot (padded slots 1)
  uint32_t st[3];    // field strides
  uint32_t B[3];     // block side per slot (1 on padded slots)
  uint32_t nb[3];    // blocks per slot
  uint32_t nblocks;  // nb[0] nb[1] nb[2]
  uint32_t g[3];     // the grid size in the radix of nb
  uint32_t W;        // ring row width in floats (B[1] + 2 padded for banks)
  uint32_t slot;     // floats per ring slot: (B[0] + 2) W
  int logP;          // log2 B[2]
};
struct LorenzoJob {
  LorGeom G; const float* x; uint16_t* codes; float* out; const Ctl* ctl;
};
// the finest 3D multi-dimensional level as warp strips: n1 x n2 strips per
// chunk of K even planes
struct MD3WJob {
  LevelMD P; int n1, n2, K; const void* in; const float* outl; const float* Rc;
  const uint16_t* Cc; float* Rs; uint16_t* Cs; const Ctl* ctl;
};
struct HistJob {
  const uint16_t* codes; uint32_t N, C, nch; uint32_t* hist; uint32_t* zc;
  const Ctl* ctl;
};
struct ScanJob {
  const uint32_t* in; unsigned long long* out; uint32_t n;
  unsigned long long* total; const Ctl* ctl;
};
struct CodebookJob {
  const uint32_t* hist; unsigned long long* enc; uint16_t* tsyms; uint8_t* tlens;
  unsigned long long* gkeys; unsigned long long* giw; uint32_t* gpar;
  uint8_t* lens_by_sym; Ctl* ctl;
};
struct EncLenJob {
  const uint16_t* codes; uint32_t N, C, nch; const unsigned long long* enc;
  uint16_t* lanebits; uint32_t* chw; const Ctl* ctl;
};
struct LayoutJob { Ctl* ctl; unsigned long long off_table, cap; };
struct PackJob {
  const uint16_t* codes; uint32_t N, C, nch; const unsigned long long* enc;
  const uint16_t* lanebits; const uint32_t* chw; const unsigned long long* woff;
  uint8_t* out; const Ctl* ctl;
};
struct OutlierJob {
  const uint16_t* codes; uint32_t N, C, nch; const uint32_t* zc;
  const unsigned long long* zoff; const float* src; float* dst; uint8_t* stream;
  unsigned long long max_out; Ctl* ctl; int gather;
};
struct FinalizeJob {
  const uint8_t* hdr; const uint8_t* hdr_const; uint8_t* out; const float* RA;
  uint32_t na; unsigned long long off_anchors; const uint8_t* bmap;
  uint32_t nblocks; unsigned long long off_bmap; const uint16_t* lanebits;
  uint32_t nch; unsigned long long off_chw; const uint16_t* tsyms;
  const uint8_t* tlens; const Ctl* ctl;
};
struct ChunkWordsJob { const uint8_t* lanebits_bytes; uint32_t nch; uint32_t* chw; };
struct DecTablesJob {
  const uint8_t* stream; uint32_t n_used; unsigned long long off_table;
  uint32_t* lut; uint32_t* cnt; unsigned long long* first; uint32_t* offs;
  uint16_t* sorted; unsigned long long* gkeys; Ctl* ctl;
};
struct DecodeJob {
  const uint8_t* stream; unsigned long long off_bits, total_words;
  const uint8_t* lanebits_bytes; const unsigned long long* woff; uint32_t N, C,
      nch, n_used;
  const uint8_t* single_src;  // the lone symbol of a one-symbol table
  const uint32_t* lut; const uint32_t* cnt; const unsigned long long* first;
  const uint32_t* offs; const uint16_t* sorted; uint16_t* codes; uint32_t* zc;
  Ctl* ctl;
};

}  // namespace hpez
