// k_tune.cu -- the auto-tuner's data-parallel work (Sec. 6): the sampling
// statistics (Sec. 6.1), compression tests of candidate thetas on sample
// blocks (Sec. 6.2 / 6.4), the Lorenzo test (Sec. 6.5), the block-wise
// tests (Sec. 6.6), and the Huffman bit count of a code histogram.
//
// A test runs one sub-field in one CTA: its reconstruction lives in shared
// memory, its input is read from the field in place.  Every score is an
// integer (fixed-point errors, code counts), so the sums do not depend on
// the order in which threads add them; the floating-point steps follow the
// compressor's operation order with explicit round-to-nearest intrinsics.
#include <algorithm>
#include <cfloat>

#include "hpez_internal.cuh"
#include "hpez_launch.h"

namespace hpez {
namespace {

constexpr int kTuneThreads = 1024;  // Lorenzo wavefront
// candidate tests and level advances: 512 threads leave each 128 registers
constexpr int kTestThreads = 512;
// block-map codes of the block-wise candidates, in test order: linear,
// not-a-knot, not-a-knot + same-level, natural, natural + same-level
__constant__ uint8_t kBlockCodes[5] = {0, 1, 5, 2, 6};
constexpr int kBlockThreads = 64;  // two warps per (block, group of candidates)
constexpr size_t kTuneSmemMax = 200 * 1024;

// floor(min(|d| * (1/e_l), 2^24 - 1) * 256) in binary32: the per-point
// error score (the scaling by 256 is exact, the result fits 32 bits)
__device__ __forceinline__ unsigned err_fixed(float d, float inv_el) {
  float v = __fmul_rn(fabsf(d), inv_el);
  v = fminf(v, 16777215.0f);
  return (unsigned)floorf(__fmul_rn(v, 256.0f));
}

// r / n for r * n < 2^32 with a precomputed m = ceil(2^32 / n) (m = 0: n = 1)
__device__ __forceinline__ unsigned fdiv(unsigned r, unsigned m) {
  return m ? __umulhi(r, m) : r;
}
__host__ __device__ __forceinline__ unsigned fdiv_magic(unsigned n) {
  // ceil(2^32 / n) = floor((2^32 - 1) / n) + 1 for n >= 2 (32-bit division)
  return n <= 1 ? 0u : 0xFFFFFFFFu / n + 1u;
}

// floor(min(|d| / e, 2^16)^2 * 256): the statistics' squared error
__device__ __forceinline__ unsigned long long sq_fixed(float d,
                                                       double inv_e) {
  double v = __dmul_rn(fabs((double)d), inv_e);
  v = fmin(v, 65536.0);
  return (unsigned long long)floor(__dmul_rn(__dmul_rn(v, v), 256.0));
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA-wide sum, valid in thread 0.  `red` holds 32 entries.
__device__ unsigned long long block_sum(unsigned long long v,
                                        unsigned long long* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  unsigned long long t = 0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
    t = warp_sum(t);
  }
  return t;
}

// ---------------------------------------------------------------------
// Sec. 6.1 statistics: lattice points with +-3 neighbours on every dim
// ---------------------------------------------------------------------
struct StatsGeom {
  uint32_t fst[3];
  uint32_t lo[3], step[3], cnt[3];
  int real[3];
};

__global__ void __launch_bounds__(256)
    k_tune_stats(const float* __restrict__ x, StatsGeom g,
                 unsigned long long total, const Ctl* __restrict__ ctl,
                 unsigned long long* acc) {
  __shared__ unsigned long long red[32];
  const double inv_e = __ddiv_rn(1.0, (double)ctl->e);
  unsigned long long cnt = 0, lin[3] = {0, 0, 0}, cub[3] = {0, 0, 0};
  const unsigned long long nthr = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x +
                              threadIdx.x;
       q < total; q += nthr) {
    const uint32_t u2 = (uint32_t)(q % g.cnt[2]);
    const unsigned long long r = q / g.cnt[2];
    const uint32_t u1 = (uint32_t)(r % g.cnt[1]);
    const uint32_t u0 = (uint32_t)(r / g.cnt[1]);
    const size_t i = (size_t)(g.lo[0] + g.step[0] * u0) * g.fst[0] +
                     (size_t)(g.lo[1] + g.step[1] * u1) * g.fst[1] +
                     (size_t)(g.lo[2] + g.step[2] * u2);
    ++cnt;
    const float xv = x[i];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      if (!g.real[s]) continue;
      const size_t st = g.fst[s];
      const float m3 = x[i - 3 * st], m1 = x[i - st], p1 = x[i + st],
                  p3 = x[i + 3 * st];
      const float pc = eval_formula(F_NAK4, m3, 0.f, m1, p1, 0.f, p3);
      const float pl = eval_formula(F_LIN, 0.f, 0.f, m1, p1, 0.f, 0.f);
      cub[s] += sq_fixed(__fsub_rn(xv, pc), inv_e);
      lin[s] += sq_fixed(__fsub_rn(xv, pl), inv_e);
    }
  }
  unsigned long long v[7] = {cnt, lin[0], lin[1], lin[2], cub[0], cub[1], cub[2]};
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const unsigned long long t = block_sum(v[j], red);
    if (threadIdx.x == 0 && t) atomicAdd(acc + j, t);
  }
}

// ---------------------------------------------------------------------
// level error bounds of every variant (Eq. 15), as the compressor does
// ---------------------------------------------------------------------
// one thread per (variant, level)
__global__ void k_tune_params(TuneCfg* cfgs, int nvar, int L,
                              const Ctl* __restrict__ ctl) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = t / L, l = t % L + 1;
  if (v >= nvar) return;
  TuneCfg& c = cfgs[v];
  const float e = ctl->e;
  double ap = 1.0;
  for (int i = 1; i < l; ++i) ap = __dmul_rn(ap, c.alpha);
  const double m = ap < c.beta ? ap : c.beta;
  const float el = __double2float_rn(__ddiv_rn((double)e, m));
  c.el[l - 1] = el;
  c.twoe[l - 1] = __fmul_rn(2.0f, el);
  c.inv2[l - 1] = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(2.0, (double)el)));
  c.inv_el[l - 1] = __double2float_rn(__ddiv_rn(1.0, (double)el));
}

__global__ void k_tune_expand(const TuneCfg* __restrict__ base,
                              const TuneCand* __restrict__ cands, int n0, int l,
                              TuneCfg* __restrict__ cfgs) {
  const int t = blockIdx.x;
  const uint32_t* s = reinterpret_cast<const uint32_t*>(base + (t < n0 ? 0 : 1));
  uint32_t* d = reinterpret_cast<uint32_t*>(cfgs + t);
  for (int i = threadIdx.x; i < (int)(sizeof(TuneCfg) / 4); i += blockDim.x) d[i] = s[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    const TuneCand c = cands[t];
    TuneCfg& o = cfgs[t];
    o.kind[l - 1] = c.kind;
    o.md[l - 1] = c.md;
    o.same[l - 1] = c.same;
    for (int j = 0; j < 3; ++j) o.ord[l - 1][j] = c.ord[j];
  }
}

__global__ void k_tune_select(const unsigned long long* __restrict__ score,
                              const TuneCand* __restrict__ cands, int n0, int n1, int nv,
                              int l, TuneCfg* base, uint8_t* choice,
                              unsigned long long* best_score) {
  const int v = threadIdx.x;
  if (v >= nv) return;
  const int b0 = v == 0 ? 0 : n0, n = v == 0 ? n0 : n1;
  int best = 0;
  for (int j = 1; j < n; ++j)
    if (score[b0 + j] < score[b0 + best]) best = j;
  const TuneCand c = cands[b0 + best];
  TuneCfg& o = base[v];
  o.kind[l - 1] = c.kind;
  o.md[l - 1] = c.md;
  o.same[l - 1] = c.same;
  for (int j = 0; j < 3; ++j) o.ord[l - 1][j] = c.ord[j];
  choice[v * kMaxLevels + l - 1] = (uint8_t)best;
  best_score[v * kMaxLevels + l - 1] = score[b0 + best];
}

// ---------------------------------------------------------------------
// one sub-field in shared memory
// ---------------------------------------------------------------------
struct Sub {
  int n[3];          // extents per slot
  int st[3];         // shared-memory strides
  const float* x;    // input at the sub-field origin
  uint32_t xst[3];   // input strides (a field has fewer than 2^32 points)
};

__device__ __forceinline__ void set_strides(Sub& f) {
  f.st[2] = 1;
  f.st[1] = f.n[2];
  f.st[0] = f.n[1] * f.n[2];
}

// sample block b of the lattice of blocks
__device__ Sub sample_block(const float* x, const TuneGeom& g, unsigned b) {
  Sub f;
  uint32_t off = 0;
  for (int d = 2; d >= 0; --d) {
    const unsigned j = b % g.cnt[d];
    b /= g.cnt[d];
    off += j * g.step[d] * g.fst[d];
    f.n[d] = (int)g.ext[d];
    f.xst[d] = g.fst[d];
  }
  f.x = x + off;
  set_strides(f);
  return f;
}

__device__ __forceinline__ float xval(const Sub& f, const int c[3]) {
  return f.x[(uint32_t)c[0] * f.xst[0] + (uint32_t)c[1] * f.xst[1] +
             (uint32_t)c[2] * f.xst[2]];
}

// anchors (every interpolation coordinate a multiple of A) from the input,
// enumerated on their own lattice; every other entry is written by the
// sweep before it is read
__device__ void init_anchors(float* R, const Sub& f, const int interp[3],
                             int A) {
  int m[3], st[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    st[d] = interp[d] ? A : 1;
    m[d] = (f.n[d] + st[d] - 1) / st[d];
  }
  const int tot = m[0] * m[1] * m[2];
  for (int q = threadIdx.x; q < tot; q += blockDim.x) {
    int c[3];
    c[2] = (q % m[2]) * st[2];
    const int r = q / m[2];
    c[1] = (r % m[1]) * st[1];
    c[0] = (r / m[1]) * st[0];
    R[c[0] * f.st[0] + c[1] * f.st[1] + c[2]] = xval(f, c);
  }
  __syncthreads();
}

// Every point of a sub-field with a dense shared layout (set_strides) from
// the input, sixteen loads in flight per thread (a CTA alone on its SM has
// nothing else to overlap them with).  The sweeps then read a point's
// input value from its own entry, just before they overwrite it with the
// reconstruction: a pass reads only points of earlier passes (or of its
// own half A), never one it has still to visit, so an entry holds the
// input until its point is visited.
__device__ void fill_x(float* R, const Sub& f) {
  const unsigned n2 = (unsigned)f.n[2], n1 = (unsigned)f.n[1];
  const unsigned mg2 = fdiv_magic(n2), mg1 = fdiv_magic(n1);
  const int tot = f.n[0] * f.n[1] * f.n[2];
  constexpr int U = 16;
  for (int q0 = threadIdx.x; q0 < tot; q0 += U * blockDim.x) {
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + u * (int)blockDim.x;
      if (q < tot) {
        const unsigned r1 = fdiv((unsigned)q, mg2), c2 = (unsigned)q - r1 * n2;
        const unsigned c0 = fdiv(r1, mg1), c1 = r1 - c0 * n1;
        v[u] = f.x[c0 * f.xst[0] + c1 * f.xst[1] + c2 * f.xst[2]];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + u * (int)blockDim.x;
      if (q < tot) R[q] = v[u];
    }
  }
  __syncthreads();
}

// Over the inputs of a compact level-s grid fc: the coarser levels'
// reconstruction at its points with even interpolation coordinates, from
// the state (the sample-block layout of f), eight loads in flight per
// thread.
__device__ void overlay_state(float* R, const float* __restrict__ state, const Sub& f,
                              const Sub& fc, const int interp[3], int s) {
  int m[3], sp[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    sp[d] = interp[d] ? 2 : 1;
    m[d] = (fc.n[d] + sp[d] - 1) / sp[d];
  }
  const unsigned mg2 = fdiv_magic((unsigned)m[2]), mg1 = fdiv_magic((unsigned)m[1]);
  const int tot = m[0] * m[1] * m[2];
  constexpr int U = 8;
  for (int q0 = threadIdx.x; q0 < tot; q0 += U * blockDim.x) {
    float v[U];
    int dst[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + u * (int)blockDim.x;
      dst[u] = -1;
      if (q < tot) {
        const unsigned r1 = fdiv((unsigned)q, mg2);
        const unsigned r0 = fdiv(r1, mg1);
        const int c[3] = {(int)r0 * sp[0], ((int)r1 - (int)r0 * m[1]) * sp[1],
                          (q - (int)r1 * m[2]) * sp[2]};
        int full = 0, comp = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          full += c[d] * (interp[d] ? s : 1) * f.st[d];
          comp += c[d] * fc.st[d];
        }
        v[u] = state[full];
        dst[u] = comp;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (dst[u] >= 0) R[dst[u]] = v[u];
  }
  __syncthreads();
}

// prediction along one slot from shared memory (same stencil choice and
// operation order as the compressor)
__device__ __forceinline__ float predict_smem(const float* R, int i, int st,
                                              int u, int m, int kind,
                                              bool half_b) {
  const int f = choose_formula(kind, half_b, u, m);
  float m3 = 0.f, m2 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
  const float m1 = R[i - st];
  switch (f) {
    case F_COPY:
      break;
    case F_EXTRAP:
      m3 = R[i - 3 * st];
      break;
    case F_LIN:
      p1 = R[i + st];
      break;
    case F_NAK4:
    case F_NAT4:
      m3 = R[i - 3 * st];
      p1 = R[i + st];
      p3 = R[i + 3 * st];
      break;
    case F_NAK3L:
    case F_NAT3L:
      m3 = R[i - 3 * st];
      p1 = R[i + st];
      break;
    case F_NAK3R:
    case F_NAT3R:
      p1 = R[i + st];
      p3 = R[i + 3 * st];
      break;
    case F_SL_NAK:
      m2 = R[i - 2 * st];
      p1 = R[i + st];
      p2 = R[i + 2 * st];
      break;
    case F_SL_NAT:
      m3 = R[i - 3 * st];
      m2 = R[i - 2 * st];
      p1 = R[i + st];
      p2 = R[i + 2 * st];
      p3 = R[i + 3 * st];
      break;
  }
  return eval_formula(f, m3, m2, m1, p1, p2, p3);
}

// One level (stride s = 2^(l-1)) of the sweep on the sub-field: passes
// and same-level halves in the compressor's order, a barrier after each.
// The points of a pass (or of one same-level half of it) are a few boxes
// of the stride-s lattice, enumerated directly: a 1D-style pass is one box
// (odd along its direction, any multiple of s on earlier directions, even
// on later ones), a multi-dimensional sub-pass one box per set of odd
// directions of its size.  A same-level half keeps the points whose odd
// indices t_d (coordinate s (2 t_d + 1)) have a sum of that parity: per
// parity pattern of the t_d, a box of step 4s along the odd directions.
// Adds the error scores (when score_on), the code counts (kHist) and the
// escapes of the level's points to the thread's accumulators.
struct Box {
  int a[3], b[3], cnt[3];
  unsigned mg[3];  // division magic of cnt
  int total;
  unsigned S;
};

// odd: directions odd at stride s; any: directions at any multiple of s;
// split: restrict the odd directions to index parities par (same-level)
__device__ __forceinline__ void make_box(Box& bx, const Sub& f,
                                         const int interp[3], int s,
                                         unsigned odd, unsigned any,
                                         bool split, unsigned par) {
  bx.total = 1;
  bx.S = odd;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int n = f.n[d];
    if (!interp[d]) {
      bx.a[d] = 0;
      bx.b[d] = 1;
      bx.cnt[d] = n;
    } else if (odd & (1u << d)) {
      const int a = split ? s * (2 * (int)((par >> d) & 1u) + 1) : s;
      const int b = split ? 4 * s : 2 * s;
      bx.a[d] = a;
      bx.b[d] = b;
      bx.cnt[d] = n - 1 >= a ? (n - 1 - a) / b + 1 : 0;
    } else if (any & (1u << d)) {
      bx.a[d] = 0;
      bx.b[d] = s;
      bx.cnt[d] = (n - 1) / s + 1;
    } else {
      bx.a[d] = 0;
      bx.b[d] = 2 * s;
      bx.cnt[d] = (n - 1) / (2 * s) + 1;
    }
    bx.total *= bx.cnt[d];
    bx.mg[d] = fdiv_magic((unsigned)bx.cnt[d]);
  }
}

// what make_box needs for one box of a pass
struct BoxDesc {
  unsigned S, any, par;
};

// the boxes of odd set S (and any) for half `half` of a same-level pass
// (split), or of the whole pass
__device__ __forceinline__ void add_boxes(BoxDesc* bd, int& nb, unsigned S, unsigned any,
                                          bool split, int half) {
  if (!split) {
    bd[nb++] = BoxDesc{S, any, 0u};
    return;
  }
  for (unsigned par = 0; par < 8; ++par)
    if ((par & ~S) == 0 && (int)(__popc(par) & 1) == half) bd[nb++] = BoxDesc{S, any, par};
}

// codes within kWin/2 of the zero-error code are counted in shared memory
constexpr int kWin = 2048;

// the histogram a point's code goes to: the shared window, or global
// memory beyond it
struct HistSink {
  uint32_t* win;   // shared, kWin bins centred on the zero-error code
  uint32_t* glob;  // global, 65536 bins
  __device__ __forceinline__ void add(unsigned code) const {
    const unsigned o = code - (unsigned)(kRadius - kWin / 2);
    if (o < (unsigned)kWin)
      atomicAdd(win + o, 1u);
    else
      atomicAdd(glob + code, 1u);
  }
};

// exact bound check with a fast accept: rn(r - x) strictly inside the
// bound implies the exact difference is inside (rounding is monotonic)
__device__ __forceinline__ unsigned quantize_t(float x, float p, float el,
                                               float inv2, float twoe,
                                               float& recon) {
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

// prediction along one slot from shared memory: the stencil of an
// interior point directly (the one choose_formula selects there), else the
// general choice
template <int KIND>
__device__ __forceinline__ float predict_t(const float* R, int i, int st, int u, int m,
                                           bool hb) {
  if (!hb) {
    if (KIND == LINEAR) {
      if (u + 1 <= m - 1) return eval_formula(F_LIN, 0.f, 0.f, R[i - st], R[i + st], 0.f, 0.f);
    } else if (u >= 3 && u + 3 <= m - 1) {
      return eval_formula(KIND == CUBIC_NAK ? F_NAK4 : F_NAT4, R[i - 3 * st], 0.f,
                          R[i - st], R[i + st], 0.f, R[i + 3 * st]);
    }
  } else if (KIND == CUBIC_NAK) {
    if (u >= 2 && u + 2 <= m - 1)
      return eval_formula(F_SL_NAK, 0.f, R[i - 2 * st], R[i - st], R[i + st],
                          R[i + 2 * st], 0.f);
  } else if (KIND == CUBIC_NAT) {
    if (u >= 3 && u + 3 <= m - 1)
      return eval_formula(F_SL_NAT, R[i - 3 * st], R[i - 2 * st], R[i - st], R[i + st],
                          R[i + 2 * st], R[i + 3 * st]);
  }
  return predict_smem(R, i, st, u, m, KIND, hb);
}

// The points of one box of a pass (or same-level half), specialized on the
// interpolator and the paradigm, which are uniform within a level; hb: the
// box is in half B of a same-level pass.
// REC false: the points' reconstructions are never read again (the last
// pass, or its same-level half B, of a score-only test): only the
// prediction and its score are needed, so the point is not quantized.
template <int KIND, bool MD, int PS, bool kHist, bool REC>
__device__ __forceinline__ void sweep_box(float* R, const Sub& f, const Box B, bool hb,
                                          int sh, const int line[3], const TuneCfg& c,
                                          int l, bool score_on, unsigned long long& score,
                                          const HistSink& hist, unsigned long long& nout) {
  const int s = 1 << sh;
  const float el = c.el[l - 1], inv2 = c.inv2[l - 1], twoe = c.twoe[l - 1];
  const float inv_el = c.inv_el[l - 1];
  const unsigned S = B.S;
  float w[3] = {0.f, 0.f, 0.f};
  int sst[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    sst[d] = s * f.st[d];
    if (MD) w[d] = c.mdw[S][d];
  }
  for (int t = threadIdx.x; t < B.total; t += blockDim.x) {
    const unsigned r1 = fdiv((unsigned)t, B.mg[2]);
    int cc[3];
    cc[2] = B.a[2] + B.b[2] * (t - (int)r1 * B.cnt[2]);
    const unsigned r0 = fdiv(r1, B.mg[1]);
    cc[1] = B.a[1] + B.b[1] * ((int)r1 - (int)r0 * B.cnt[1]);
    cc[0] = B.a[0] + B.b[0] * (int)r0;
    const int i = cc[0] * f.st[0] + cc[1] * f.st[1] + cc[2];
    const float xv = R[i];  // the input, until the point is visited
    float p;
    if (!MD) {
      p = predict_t<KIND>(R, i, sst[PS], cc[PS] >> sh, line[PS], hb);
    } else {
      float acc = 0.0f;
      bool first = true;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (!(S & (1u << d))) continue;
        const float pd = predict_t<KIND>(R, i, sst[d], cc[d] >> sh, line[d], hb);
        const float tw = __fmul_rn(w[d], pd);
        acc = first ? tw : __fadd_rn(acc, tw);
        first = false;
      }
      p = acc;
    }
    if (REC) {
      float rv;
      const unsigned code = quantize_t(xv, p, el, inv2, twoe, rv);
      R[i] = rv;
      if (kHist) hist.add(code);
      if (code == 0u) ++nout;
    }
    if (score_on) score += err_fixed(__fsub_rn(xv, p), inv_el);
  }
}

// KIND < 0: the level's interpolator read from the config; KIND >= 0:
// fixed (the config's value is that kind)
// sbox: shared memory for the boxes of a pass (at most 6), each built by
// one thread
// sh: the level's stride as a shift in the coordinates of f (l - 1 on the
// sample block, 0 on its compact level-l grid)
// free_last: a score-only test of this level alone (no histogram, the
// level's state not kept), whose last pass (its half B with same-level
// halves) is not quantized
// the boxes of every pass and same-level half of one level: slot
// pj * halves + half holds nb[slot] boxes at b[6 * slot]
struct LevelBoxes {
  Box b[36];
  int nb[6];
};

template <int KIND, bool kHist>
__device__ void sweep_level_k(float* R, const Sub& f, const int interp[3],
                              int k, int l, int sh, const TuneCfg& c, bool score_on,
                              unsigned long long& score, const HistSink& hist,
                              unsigned long long& nout, LevelBoxes* lb, bool free_last) {
  const int s = 1 << sh;
  int line[3];
  unsigned imask = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    line[d] = (f.n[d] - 1) / s + 1;
    if (interp[d]) imask |= 1u << d;
  }
  const int kind = c.kind[l - 1];
  const bool md = c.md[l - 1] != 0;
  const bool same = c.same[l - 1] != 0 && kind != LINEAR;
  const int halves = same ? 2 : 1;
  // every box of the level at once, one thread each (the barrier that
  // ended the previous level's last pass freed the array)
  if ((int)threadIdx.x < 6 * k * halves) {
    const int slot = (int)threadIdx.x / 6, q = (int)threadIdx.x % 6;
    const int pj = slot / halves, half = slot % halves;
    BoxDesc bd[6];
    int nb = 0;
    if (!md) {
      unsigned any = 0;  // directions earlier in the order: any parity
      for (int r = 0; r < pj; ++r) any |= 1u << c.ord[l - 1][r];
      add_boxes(bd, nb, 1u << c.ord[l - 1][pj], any, same, half);
    } else {
      for (unsigned S = 1; S < 8; ++S)
        if ((S & imask) == S && __popc(S) == pj + 1) add_boxes(bd, nb, S, 0u, same, half);
    }
    if (q < nb) make_box(lb->b[6 * slot + q], f, interp, s, bd[q].S, bd[q].any, same, bd[q].par);
    if (q == 0) lb->nb[slot] = nb;
  }
  __syncthreads();
  for (int pj = 0; pj < k; ++pj) {
    for (int half = 0; half < halves; ++half) {
      const int slot = pj * halves + half;
      const int nb = lb->nb[slot];
      const Box* sbox = lb->b + 6 * slot;
      const bool hb = half == 1;
      const bool rec = kHist || !free_last || pj != k - 1 || (same && half == 0);
      for (int q = 0; q < nb; ++q) {
        const Box B = sbox[q];
        if (B.total == 0) continue;
#define HPEZ_SWEEP(K, M, P)                                                   \
  do {                                                                        \
    if (rec)                                                                  \
      sweep_box<K, M, P, kHist, true>(R, f, B, hb, sh, line, c, l, score_on,  \
                                      score, hist, nout);                    \
    else                                                                      \
      sweep_box<K, M, P, kHist, false>(R, f, B, hb, sh, line, c, l, score_on, \
                                       score, hist, nout);                   \
  } while (0)
#define HPEZ_SWEEP_1D(K)                                                      \
  do {                                                                        \
    const int ps = c.ord[l - 1][pj];                                          \
    if (ps == 0) HPEZ_SWEEP(K, false, 0);                                     \
    else if (ps == 1) HPEZ_SWEEP(K, false, 1);                                \
    else HPEZ_SWEEP(K, false, 2);                                             \
  } while (0)
        if (KIND >= 0) {
          if (md) HPEZ_SWEEP(KIND < 0 ? 0 : KIND, true, 0);
          else HPEZ_SWEEP_1D(KIND < 0 ? 0 : KIND);
        } else if (md) {
          if (kind == LINEAR) HPEZ_SWEEP(LINEAR, true, 0);
          else if (kind == CUBIC_NAK) HPEZ_SWEEP(CUBIC_NAK, true, 0);
          else HPEZ_SWEEP(CUBIC_NAT, true, 0);
        } else {
          if (kind == LINEAR) HPEZ_SWEEP_1D(LINEAR);
          else if (kind == CUBIC_NAK) HPEZ_SWEEP_1D(CUBIC_NAK);
          else HPEZ_SWEEP_1D(CUBIC_NAT);
        }
#undef HPEZ_SWEEP_1D
#undef HPEZ_SWEEP
      }
      __syncthreads();
    }
  }
}

// The same sweep for small sub-fields (the block-wise tests, one warp
// each), for NK interpolators K0, K1, K2 at once: their passes have the
// same points (one paradigm and order per level, from the global theta;
// same-level halves for all of them or none), so the enumeration, the
// input value and the index are shared and only the prediction, the
// quantization and the score are per interpolator, each on its own
// reconstruction (R + k * vol).  The boxes of a pass (or of a same-level
// half: boxes of step 4s along the odd directions, one per parity pattern)
// are one enumeration -- fewer partial iterations than a loop per box when
// the boxes hold a few points each.
template <int NK, int K0, int K1, int K2, bool SAME, bool MD, int PS, bool REC>
__device__ void sweep_pass_multi(float* R, int vol, const Sub& f, const Box* bx, int nb,
                                 int tot, int half, int sh, const int line[3],
                                 const TuneCfg& c, int l, unsigned long long (&score)[NK]) {
  const int s = 1 << sh;
  const float el = c.el[l - 1], inv2 = c.inv2[l - 1], twoe = c.twoe[l - 1];
  const float inv_el = c.inv_el[l - 1];
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    int q = 0, r = t;
    while (q + 1 < nb && r >= bx[q].total) r -= bx[q++].total;
    const Box& B = bx[q];
    const unsigned r1 = fdiv((unsigned)r, B.mg[2]);
    int cc[3];
    cc[2] = B.a[2] + B.b[2] * (r - (int)r1 * B.cnt[2]);
    const unsigned r0 = fdiv(r1, B.mg[1]);
    cc[1] = B.a[1] + B.b[1] * ((int)r1 - (int)r0 * B.cnt[1]);
    cc[0] = B.a[0] + B.b[0] * (int)r0;
    const unsigned S = B.S;
    const bool in_b = SAME && half == 1;
    const int i = cc[0] * f.st[0] + cc[1] * f.st[1] + cc[2];
    const float xv = R[i];  // copy 0 holds the input until the point is visited
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      const int kind = k == 0 ? K0 : (k == 1 ? K1 : K2);
      float* Rk = R + k * vol;
      float p;
      if (!MD) {
        p = predict_smem(Rk, i, s * f.st[PS], cc[PS] >> sh, line[PS], kind, in_b);
      } else {
        float acc = 0.0f;
        bool first = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (!(S & (1u << d))) continue;
          const float pd = predict_smem(Rk, i, s * f.st[d], cc[d] >> sh, line[d], kind, in_b);
          const float tw = __fmul_rn(c.mdw[S][d], pd);
          acc = first ? tw : __fadd_rn(acc, tw);
          first = false;
        }
        p = acc;
      }
      if (REC) {
        float rv;
        quantize_t(xv, p, el, inv2, twoe, rv);
        Rk[i] = rv;
      }
      score[k] += err_fixed(__fsub_rn(xv, p), inv_el);
    }
  }
}

// One level of the block-wise sweep for the NK interpolators of
// sweep_pass_multi: passes (and same-level halves) in the compressor's
// order, a barrier after each.
template <int NK, int K0, int K1, int K2, bool SAME>
__device__ void sweep_level_multi(float* R, int vol, const Sub& f, const int interp[3],
                                  int k, int l, const TuneCfg& c,
                                  unsigned long long (&score)[NK], Box* bx) {
  const int sh = l - 1, s = 1 << sh;
  int line[3];
  unsigned imask = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    line[d] = (f.n[d] - 1) / s + 1;
    if (interp[d]) imask |= 1u << d;
  }
  const bool md = c.md[l - 1] != 0;
  for (int pj = 0; pj < k; ++pj) {
    for (int half = 0; half < (SAME ? 2 : 1); ++half) {
      // the boxes of the pass or half (at most 6) in shared memory, one
      // thread each
      BoxDesc bd[6];
      int nb = 0;
      if (!md) {
        unsigned any = 0;  // directions earlier in the order: any parity
        for (int q = 0; q < pj; ++q) any |= 1u << c.ord[l - 1][q];
        add_boxes(bd, nb, 1u << c.ord[l - 1][pj], any, SAME, half);
      } else {
        for (unsigned S = 1; S < 8; ++S)
          if ((S & imask) == S && __popc(S) == pj + 1) add_boxes(bd, nb, S, 0u, SAME, half);
      }
      __syncthreads();  // the previous pass or half is done with bx
      if ((int)threadIdx.x < nb)
        make_box(bx[threadIdx.x], f, interp, s, bd[threadIdx.x].S, bd[threadIdx.x].any, SAME,
                 bd[threadIdx.x].par);
      __syncthreads();
      int tot = 0;
      for (int q = 0; q < nb; ++q) tot += bx[q].total;
      // the finest level's last pass (half B with same-level halves) is
      // read by nothing: scored, not quantized
      const bool rec = l != 1 || pj != k - 1 || (SAME && half == 0);
#define HPEZ_SWEEP(M, P)                                                      \
  do {                                                                        \
    if (rec)                                                                  \
      sweep_pass_multi<NK, K0, K1, K2, SAME, M, P, true>(R, vol, f, bx, nb, tot, half, sh, \
                                                         line, c, l, score);  \
    else                                                                      \
      sweep_pass_multi<NK, K0, K1, K2, SAME, M, P, false>(R, vol, f, bx, nb, tot, half, \
                                                          sh, line, c, l, score); \
  } while (0)
      if (md) {
        HPEZ_SWEEP(true, 0);
      } else {
        const int ps = c.ord[l - 1][pj];
        if (ps == 0) HPEZ_SWEEP(false, 0);
        else if (ps == 1) HPEZ_SWEEP(false, 1);
        else HPEZ_SWEEP(false, 2);
      }
#undef HPEZ_SWEEP
      __syncthreads();
    }
  }
}

template <bool kHist>
__device__ __forceinline__ void sweep_level(float* R, const Sub& f,
                                            const int interp[3], int k, int l,
                                            const TuneCfg& c, bool score_on,
                                            unsigned long long& score,
                                            const HistSink& hist,
                                            unsigned long long& nout, LevelBoxes* lb,
                                            int sh, bool free_last = false) {
  sweep_level_k<-1, kHist>(R, f, interp, k, l, sh, c, score_on, score, hist, nout, lb,
                           free_last);
}

__device__ __forceinline__ void load_cfg(TuneCfg* dst, const TuneCfg* src) {
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(TuneCfg) / 4); i += blockDim.x)
    d[i] = s[i];
  __syncthreads();
}

// ---------------------------------------------------------------------
// Sec. 6.2 / 6.4: CTA (sample block, variant): anchors, levels L..l_stop
// ---------------------------------------------------------------------
// the points of the sub-field whose interpolation coordinates are multiples
// of st, copied between shared memory and a state buffer of the same layout
template <bool kLoad>
__device__ void copy_lattice(float* R, float* __restrict__ state, const Sub& f,
                             const int interp[3], int st) {
  int m[3], sp[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    sp[d] = interp[d] ? st : 1;
    m[d] = (f.n[d] + sp[d] - 1) / sp[d];
  }
  const unsigned mg2 = fdiv_magic((unsigned)m[2]), mg1 = fdiv_magic((unsigned)m[1]);
  const int tot = m[0] * m[1] * m[2];
  for (int q = threadIdx.x; q < tot; q += blockDim.x) {
    const unsigned r1 = fdiv((unsigned)q, mg2);
    const unsigned r0 = fdiv(r1, mg1);
    const int c2 = (q - (int)r1 * m[2]) * sp[2];
    const int c1 = ((int)r1 - (int)r0 * m[1]) * sp[1];
    const int c0 = (int)r0 * sp[0];
    const int i = c0 * f.st[0] + c1 * f.st[1] + c2;
    if (kLoad)
      R[i] = state[i];
    else
      state[i] = R[i];
  }
  __syncthreads();
}

// The level-s grid of a sample block (the points whose interpolation
// coordinates are multiples of s) as a sub-field of its own: compact in
// shared memory, its input strides scaled by s.  A level's passes read and
// write only points of its grid, with neighbours at s, 2s, 3s (1, 2, 3 on
// the compact grid), so the level runs on the compact grid unchanged.
__device__ __forceinline__ Sub compact_sub(const Sub& f, const int interp[3], int s) {
  Sub c = f;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (interp[d]) {
      c.n[d] = (f.n[d] - 1) / s + 1;
      c.xst[d] = f.xst[d] * (uint32_t)s;
    }
  set_strides(c);
  return c;
}

// Variants y < ny0 use geometry g0, the others g1 (two frozen-dimension
// choices in one launch).  With a state buffer (candidate tests of level
// l_stop), a CTA starts from its block's reconstruction after the coarser
// levels, kept there by k_tune_advance, and runs level l_stop only;
// without one it starts from the anchors and runs levels L..l_stop.
template <bool kHist>
__global__ void __launch_bounds__(kTestThreads, 1)
    k_tune_test(const float* __restrict__ x, TuneGeom g0, TuneGeom g1, int ny0,
                const TuneCfg* __restrict__ cfgs, int l_stop,
                unsigned long long* score, uint32_t* hists,
                unsigned long long* nout, float* __restrict__ state,
                unsigned vol) {
  const bool second = (int)blockIdx.y >= ny0;
  const TuneGeom& g = second ? g1 : g0;
  extern __shared__ float R[];
  __shared__ TuneCfg c;
  __shared__ unsigned long long red[32];
  __shared__ uint32_t win[kHist ? kWin : 1];
  __shared__ LevelBoxes sbox;
  const int v = blockIdx.y;
  if (kHist)
    for (int i = threadIdx.x; i < kWin; i += blockDim.x) win[i] = 0;
  load_cfg(&c, cfgs + v);
  const Sub f = sample_block(x, g, blockIdx.x);
  unsigned long long sc = 0, no = 0;
  HistSink h{win, kHist ? hists + (size_t)v * 65536 : nullptr};
  if (state) {
    // level l_stop alone, on the compact level grid, from the state after
    // the levels above it (the anchors at the coarsest level)
    const int s = 1 << (l_stop - 1);
    const Sub fc = compact_sub(f, g.interp, s);
    // the input at the level's points, the coarser levels' reconstruction
    // at the others (the anchors, from the input, at the coarsest level)
    fill_x(R, fc);
    if (l_stop < g.L)
      overlay_state(R, state + ((size_t)(second ? 1 : 0) * gridDim.x + blockIdx.x) * vol, f,
                    fc, g.interp, s);
    sweep_level<kHist>(R, fc, g.interp, g.k, l_stop, c, true, sc, h, no, &sbox, 0, !kHist);
  } else {
    fill_x(R, f);  // the input everywhere, the anchors among it
    for (int l = g.L; l >= l_stop; --l)
      sweep_level<kHist>(R, f, g.interp, g.k, l, c, l == l_stop, sc, h, no, &sbox, l - 1);
  }
  if (kHist)
    for (int i = threadIdx.x; i < kWin; i += blockDim.x)
      if (win[i]) atomicAdd(h.glob + (kRadius - kWin / 2) + i, win[i]);
  sc = block_sum(sc, red);
  if (threadIdx.x == 0 && sc) atomicAdd(score + v, sc);
  if (nout) {  // escapes: counted by the (alpha, beta) tests only
    no = block_sum(no, red);
    if (threadIdx.x == 0 && no) atomicAdd(nout + v, no);
  }
}

// After level l's choice: CTA (sample block, variant w) runs level l with
// the chosen config cfgs[w] from the block's state (the anchors at the
// coarsest level) and stores the stride-2^(l-1) lattice back.
__global__ void __launch_bounds__(kTestThreads, 1)
    k_tune_advance(const float* __restrict__ x, TuneGeom g0, TuneGeom g1,
                   const TuneCfg* __restrict__ cfgs, int l,
                   float* __restrict__ state, unsigned vol) {
  const int w = blockIdx.y;
  const TuneGeom& g = w ? g1 : g0;
  extern __shared__ float R[];
  __shared__ TuneCfg c;
  __shared__ LevelBoxes sbox;
  load_cfg(&c, cfgs + w);
  const Sub f = sample_block(x, g, blockIdx.x);
  float* st = state + ((size_t)w * gridDim.x + blockIdx.x) * vol;
  // the input on the level's lattice (the anchors at the coarsest level),
  // then the coarser points' reconstruction over it
  init_anchors(R, f, g.interp, 1 << (l - 1));
  if (l < g.L) copy_lattice<true>(R, st, f, g.interp, 2 << (l - 1));
  unsigned long long sc = 0, no = 0;
  const HistSink none{nullptr, nullptr};
  sweep_level<false>(R, f, g.interp, g.k, l, c, false, sc, none, no, &sbox, l - 1);
  copy_lattice<false>(R, st, f, g.interp, 1 << (l - 1));
}

// ---------------------------------------------------------------------
// Sec. 6.5: Lorenzo test, CTA (sample block, order).  The recurrence runs
// as a wavefront over the planes i0 + i1 + i2 = t: every neighbour a point
// reads lies on an earlier plane.  Neighbours outside the block read 0.
// ---------------------------------------------------------------------
// Lorenzo coefficient of offset a (0..ORDER) along one direction: order 1
// (1, -1), order 2 (1, -2, 1); a point's weight is minus the product over
// the three directions (small integers, so every product is exact)
template <int ORDER>
__device__ __forceinline__ float lorenzo_coef(int a) {
  return ORDER == 1 ? (a == 0 ? 1.0f : -1.0f) : (a == 1 ? -2.0f : 1.0f);
}

// row length of the Lorenzo block in shared memory: even, so that the
// points of a wavefront plane taken by consecutive lanes (i1 + 1, i2 - 1:
// a step of n2p - 1 words) fall in distinct banks
__host__ __device__ __forceinline__ int lorenzo_row(int n2) { return n2 + (n2 & 1); }

template <int ORDER>
__device__ __forceinline__ void lorenzo_body(const Sub& f, const int lim[3], float e,
                                             float inv2, float twoe, float* R,
                                             uint32_t* h, unsigned long long& no) {
  const int n0 = f.n[0], n1 = f.n[1], n2 = f.n[2], n2p = lorenzo_row(n2);
  const int T = (n0 - 1) + (n1 - 1) + (n2 - 1);
  const int npair = n0 * n1;
  const unsigned mg1 = fdiv_magic((unsigned)n1);
  // a thread's pairs (i0, i1) are q = tid + k * blockDim (at most kP); the
  // input values of plane t + 1 are loaded while plane t is computed
  constexpr int kP = 4;
  float xcur[kP], xnext[kP];
  auto load_plane = [&](int t, float* xv) {
#pragma unroll
    for (int k = 0; k < kP; ++k) {
      const int q = threadIdx.x + k * blockDim.x;
      xv[k] = 0.0f;
      if (q >= npair) continue;
      const int i0 = (int)fdiv((unsigned)q, mg1), i1 = q - i0 * n1, i2 = t - i0 - i1;
      if (i2 < 0 || i2 >= n2) continue;
      const int cc[3] = {i0, i1, i2};
      xv[k] = xval(f, cc);
    }
  };
  load_plane(0, xcur);
  for (int t = 0; t <= T; ++t) {
    if (t < T) load_plane(t + 1, xnext);
#pragma unroll
    for (int k = 0; k < kP; ++k) {
      const int q = threadIdx.x + k * blockDim.x;
      if (q >= npair) continue;
      const int i0 = (int)fdiv((unsigned)q, mg1), i1 = q - i0 * n1, i2 = t - i0 - i1;
      if (i2 < 0 || i2 >= n2) continue;
      const int base = (i0 * n1 + i1) * n2p + i2;
      // terms in the order a (dim 0), b (dim 1), cz (dim 2); neighbours
      // outside the block read 0
      float acc = 0.0f;
#pragma unroll
      for (int a = 0; a <= ORDER; ++a)
#pragma unroll
        for (int b = 0; b <= ORDER; ++b)
#pragma unroll
          for (int cz = 0; cz <= ORDER; ++cz) {
            if (a == 0 && b == 0 && cz == 0) continue;
            if (a > lim[0] || b > lim[1] || cz > lim[2]) continue;
            const float wgt = -__fmul_rn(__fmul_rn(lorenzo_coef<ORDER>(a), lorenzo_coef<ORDER>(b)),
                                         lorenzo_coef<ORDER>(cz));
            float v = 0.0f;
            if (a <= i0 && b <= i1 && cz <= i2) v = R[base - (a * n1 + b) * n2p - cz];
            acc = __fadd_rn(acc, __fmul_rn(wgt, v));
          }
      float rv;
      const unsigned code = quantize(xcur[k], acc, e, inv2, twoe, rv);
      R[base] = rv;
      atomicAdd(h + code, 1u);
      if (code == 0u) ++no;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kP; ++k) xcur[k] = xnext[k];
  }
}

__global__ void __launch_bounds__(kTuneThreads)
    k_tune_lorenzo(const float* __restrict__ x, TuneGeom g,
                   const Ctl* __restrict__ ctl, uint32_t* hists,
                   unsigned long long* nout) {
  extern __shared__ float R[];
  __shared__ unsigned long long red[32];
  const int order = blockIdx.y + 1;
  const Sub f = sample_block(x, g, blockIdx.x);
  const float e = ctl->e;
  const float inv2 = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(2.0, (double)e)));
  const float twoe = __fmul_rn(2.0f, e);
  int lim[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) lim[d] = d < g.off ? 0 : order;
  uint32_t* h = hists + (size_t)blockIdx.y * 65536;
  unsigned long long no = 0;
  if (order == 1)
    lorenzo_body<1>(f, lim, e, inv2, twoe, R, h, no);
  else
    lorenzo_body<2>(f, lim, e, inv2, twoe, R, h, no);
  no = block_sum(no, red);
  if (threadIdx.x == 0 && no) atomicAdd(nout + blockIdx.y, no);
}

// ---------------------------------------------------------------------
// Sec. 6.6: CTA per field block: the centred sub-block, every candidate
// interpolator for all levels, the smallest summed score wins
// ---------------------------------------------------------------------
struct BlockGeom {
  uint32_t nb[3];
  int bs, Q, frozen_slot;
};

// CTA (field block) of one launch: the summed level scores of the centred
// sub-block with each of the launch's NK interpolators at every level,
// written to the candidates' slots (kBlockCodes[j] for j in slots, 8 bits
// each)
template <int NK, int K0, int K1, int K2, bool SAME>
__global__ void __launch_bounds__(kBlockThreads)
    k_tune_blockwise(const float* __restrict__ x, TuneGeom g, BlockGeom bg,
                     const TuneCfg* __restrict__ base, uint32_t slots,
                     unsigned long long* scores) {
  extern __shared__ float R[];
  __shared__ TuneCfg c;
  __shared__ unsigned long long red[32];
  __shared__ Box sbx[6];
  load_cfg(&c, base);
  unsigned b = blockIdx.x;
  Sub f;
  uint32_t off = 0;
  int qmin = 0x7fffffff;
  for (int d = 2; d >= 0; --d) {
    const unsigned j = b % bg.nb[d];
    b /= bg.nb[d];
    f.xst[d] = g.fst[d];
    if (d < g.off) {
      f.n[d] = 1;
      continue;
    }
    const int b0 = (int)j * bg.bs;
    const int bext = min(bg.bs, (int)g.n[d] - b0);
    const int q = min(bext, bg.Q);
    off += (uint32_t)(b0 + (bext - q) / 2) * g.fst[d];
    f.n[d] = q;
    if (d != bg.frozen_slot) qmin = min(qmin, q);
  }
  f.x = x + off;
  set_strides(f);
  const int vol = f.n[0] * f.n[1] * f.n[2];
  int As = 2;
  const int lim = qmin > 1 ? qmin - 1 : 1;
  while (As * 2 <= lim) As *= 2;
  int L = 0;
  while ((1 << L) < As) ++L;
  // the input everywhere in copy 0, the anchors in the others
  fill_x(R, f);
  if (NK > 1) {
    int m[3], st[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      st[d] = g.interp[d] ? As : 1;
      m[d] = (f.n[d] + st[d] - 1) / st[d];
    }
    const int tot = m[0] * m[1] * m[2];
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
      int cc[3];
      cc[2] = (q % m[2]) * st[2];
      const int r = q / m[2];
      cc[1] = (r % m[1]) * st[1];
      cc[0] = (r / m[1]) * st[0];
      const int i = cc[0] * f.st[0] + cc[1] * f.st[1] + cc[2];
      const float v = xval(f, cc);
#pragma unroll
      for (int k = 1; k < NK; ++k) R[k * vol + i] = v;
    }
    __syncthreads();
  }
  unsigned long long sc[NK];
#pragma unroll
  for (int k = 0; k < NK; ++k) sc[k] = 0;
  for (int l = L; l >= 1; --l)
    sweep_level_multi<NK, K0, K1, K2, SAME>(R, vol, f, g.interp, g.k, l, c, sc, sbx);
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    const unsigned long long t = block_sum(sc[k], red);
    if (threadIdx.x == 0)
      scores[(size_t)blockIdx.x * 5 + ((slots >> (8 * k)) & 0xFFu)] = t;
    __syncthreads();
  }
}

// the block map: per block the first candidate with the smallest score
// among the allowed ones (natural: slots 3, 4; same-level: slots 2, 4)
__global__ void k_tune_block_argmin(const unsigned long long* __restrict__ scores,
                                    uint32_t nblocks, unsigned allow, uint8_t* bmap) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  unsigned long long best = scores[(size_t)b * 5];
  int bj = 0;
  for (int j = 1; j < 5; ++j) {
    if ((j >= 3 && !(allow & 1u)) || ((j == 2 || j == 4) && !(allow & 2u))) continue;
    const unsigned long long v = scores[(size_t)b * 5 + j];
    if (v < best) {
      best = v;
      bj = j;
    }
  }
  bmap[b] = kBlockCodes[bj];
}

void set_smem_attr() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_tune_test<true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kTuneSmemMax);
  cudaFuncSetAttribute(k_tune_test<false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kTuneSmemMax);
  cudaFuncSetAttribute(k_tune_lorenzo,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kTuneSmemMax);
  cudaFuncSetAttribute(k_tune_advance,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kTuneSmemMax);
#define HPEZ_BW_ATTR(...)                                                     \
  cudaFuncSetAttribute(k_tune_blockwise<__VA_ARGS__>,                         \
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTuneSmemMax)
  HPEZ_BW_ATTR(3, LINEAR, CUBIC_NAK, CUBIC_NAT, false);
  HPEZ_BW_ATTR(2, LINEAR, CUBIC_NAK, 0, false);
  HPEZ_BW_ATTR(2, CUBIC_NAK, CUBIC_NAT, 0, true);
  HPEZ_BW_ATTR(1, LINEAR, 0, 0, false);
  HPEZ_BW_ATTR(1, CUBIC_NAK, 0, 0, false);
  HPEZ_BW_ATTR(1, CUBIC_NAT, 0, 0, false);
  HPEZ_BW_ATTR(1, CUBIC_NAK, 0, 0, true);
  HPEZ_BW_ATTR(1, CUBIC_NAT, 0, 0, true);
#undef HPEZ_BW_ATTR
  done = true;
}

}  // namespace

void launch_tune_stats(const float* x, const uint32_t n[3],
                       const uint32_t fst[3], const int real[3], int t,
                       const Ctl* ctl, unsigned long long* acc, int num_sms,
                       cudaStream_t s) {
  StatsGeom g;
  unsigned long long total = 1;
  for (int d = 0; d < 3; ++d) {
    g.fst[d] = fst[d];
    g.real[d] = real[d];
    if (real[d]) {
      g.lo[d] = 3;
      g.step[d] = (uint32_t)t;
      g.cnt[d] = n[d] >= 7 ? (n[d] - 7) / (uint32_t)t + 1 : 0;
    } else {
      g.lo[d] = 0;
      g.step[d] = 1;
      g.cnt[d] = 1;
    }
    total *= g.cnt[d];
  }
  if (total == 0) return;
  unsigned long long blocks = (total + 255) / 256;
  if (blocks > (unsigned long long)num_sms * 8) blocks = (unsigned long long)num_sms * 8;
  k_tune_stats<<<(unsigned)blocks, 256, 0, s>>>(x, g, total, ctl, acc);
}

void launch_tune_params(TuneCfg* cfgs, int nvar, int L, const Ctl* ctl,
                        cudaStream_t s) {
  const int n = nvar * L;
  k_tune_params<<<(n + 127) / 128, 128, 0, s>>>(cfgs, nvar, L, ctl);
}

void launch_tune_expand(const TuneCfg* base, const TuneCand* cands, int n0, int n1, int l,
                        TuneCfg* cfgs, cudaStream_t s) {
  if (n0 + n1 > 0) k_tune_expand<<<n0 + n1, 64, 0, s>>>(base, cands, n0, l, cfgs);
}

void launch_tune_select(const unsigned long long* score, const TuneCand* cands, int n0,
                        int n1, int nv, int l, TuneCfg* base, uint8_t* choice,
                        unsigned long long* best, cudaStream_t s) {
  k_tune_select<<<1, 32, 0, s>>>(score, cands, n0, n1, nv, l, base, choice, best);
}

size_t tune_test_smem(const TuneGeom& g) {
  return (size_t)g.ext[0] * g.ext[1] * g.ext[2] * sizeof(float);
}

// the compact level-l grid of a sample block
size_t tune_level_smem(const TuneGeom& g, int l) {
  const uint32_t st = 1u << (l - 1);
  size_t n = sizeof(float);
  for (int d = 0; d < 3; ++d) n *= g.interp[d] ? (g.ext[d] - 1) / st + 1 : g.ext[d];
  return n;
}

size_t tune_lorenzo_smem(const TuneGeom& g) {
  return (size_t)g.ext[0] * g.ext[1] * lorenzo_row((int)g.ext[2]) * sizeof(float);
}

void launch_tune_test(const float* x, const TuneGeom& g0, const TuneGeom& g1,
                      int ny0, const TuneCfg* cfgs, int nvar, int nblk,
                      int l_stop, bool hist, unsigned long long* score,
                      uint32_t* hists, unsigned long long* nout, float* state,
                      cudaStream_t s) {
  set_smem_attr();
  const dim3 grid((unsigned)nblk, (unsigned)nvar);
  const size_t sm = state ? std::max(tune_level_smem(g0, l_stop), tune_level_smem(g1, l_stop))
                          : std::max(tune_test_smem(g0), tune_test_smem(g1));
  const unsigned vol = (unsigned)(tune_test_smem(g0) / sizeof(float));
  // a coarse level's compact grid holds a few hundred or thousand points: a
  // smaller CTA per (block, candidate) lets every CTA of the launch be
  // resident at once (their fixed costs then overlap)
  int tpb = kTestThreads;
  if (state) {
    const size_t pts = sm / sizeof(float);
    tpb = pts <= 1024 ? 128 : pts <= 8192 ? 256 : kTestThreads;
  }
  if (hist)
    k_tune_test<true><<<grid, tpb, sm, s>>>(x, g0, g1, ny0, cfgs, l_stop, score, hists, nout,
                                            state, vol);
  else
    k_tune_test<false><<<grid, tpb, sm, s>>>(x, g0, g1, ny0, cfgs, l_stop, score, hists,
                                             nout, state, vol);
}

void launch_tune_advance(const float* x, const TuneGeom& g0, const TuneGeom& g1,
                         int nv, int nblk, const TuneCfg* cfgs, int l, float* state,
                         cudaStream_t s) {
  set_smem_attr();
  const size_t sm = std::max(tune_test_smem(g0), tune_test_smem(g1));
  const unsigned vol = (unsigned)(tune_test_smem(g0) / sizeof(float));
  k_tune_advance<<<dim3((unsigned)nblk, (unsigned)nv), kTestThreads, sm, s>>>(
      x, g0, g1, cfgs, l, state, vol);
}

void launch_tune_lorenzo(const float* x, const TuneGeom& g, int nblk,
                         const Ctl* ctl, uint32_t* hists,
                         unsigned long long* nout, cudaStream_t s) {
  set_smem_attr();
  k_tune_lorenzo<<<dim3((unsigned)nblk, 2), kTuneThreads, tune_lorenzo_smem(g), s>>>(
      x, g, ctl, hists, nout);
}

int launch_tune_blockwise(const float* x, const TuneGeom& g, int bs, int Q,
                           int frozen_slot, const uint32_t nb[3],
                           uint32_t nblocks, const TuneCfg* base,
                           unsigned allow, unsigned long long* scores,
                           uint8_t* bmap, cudaStream_t s, cudaStream_t s2,
                           cudaEvent_t fork, cudaEvent_t join) {
  set_smem_attr();
  BlockGeom bg;
  size_t vol = 1;
  for (int d = 0; d < 3; ++d) {
    bg.nb[d] = nb[d];
    if (d >= g.off) vol *= (size_t)(Q < bs ? Q : bs);
  }
  bg.bs = bs;
  bg.Q = Q;
  bg.frozen_slot = frozen_slot;
  // slots j (kBlockCodes[j]): 0 linear, 1 not-a-knot, 2 not-a-knot with
  // same-level halves, 3 natural, 4 natural with same-level halves.  A
  // launch scores the interpolators whose passes have the same points, as
  // many as fit next to each other in shared memory.
  const size_t bytes = vol * sizeof(float);
  const int per = (int)(kTuneSmemMax / bytes);  // >= 1 (checked by the caller)
  const bool nat = (allow & 1u) != 0, sl = (allow & 2u) != 0;
  const dim3 grid(nblocks);
  int n = 1;
#define HPEZ_BW(NK, K0, K1, K2, SAME, SLOTS)                                  \
  do {                                                                        \
    ++n;                                                                      \
    k_tune_blockwise<NK, K0, K1, K2, SAME><<<grid, kBlockThreads, NK * bytes, s>>>( \
        x, g, bg, base, SLOTS, scores);                                       \
  } while (0)
  if (nat && per >= 3) {
    HPEZ_BW(3, LINEAR, CUBIC_NAK, CUBIC_NAT, false, 0u | (1u << 8) | (3u << 16));
  } else if (per >= 2) {
    HPEZ_BW(2, LINEAR, CUBIC_NAK, 0, false, 0u | (1u << 8));
    if (nat) HPEZ_BW(1, CUBIC_NAT, 0, 0, false, 3u);
  } else {
    HPEZ_BW(1, LINEAR, 0, 0, false, 0u);
    HPEZ_BW(1, CUBIC_NAK, 0, 0, false, 1u);
    if (nat) HPEZ_BW(1, CUBIC_NAT, 0, 0, false, 3u);
  }
  if (sl) {
    // the same-level candidates on the second stream, so that their CTAs
    // fill the SMs the first launch's last wave leaves idle
    cudaEventRecord(fork, s);
    cudaStreamWaitEvent(s2, fork, 0);
    cudaStream_t s1 = s;
    s = s2;
    if (nat && per >= 2) {
      HPEZ_BW(2, CUBIC_NAK, CUBIC_NAT, 0, true, 2u | (4u << 8));
    } else {
      HPEZ_BW(1, CUBIC_NAK, 0, 0, true, 2u);
      if (nat) HPEZ_BW(1, CUBIC_NAT, 0, 0, true, 4u);
    }
    cudaEventRecord(join, s2);
    s = s1;
    cudaStreamWaitEvent(s, join, 0);
  }
#undef HPEZ_BW
  k_tune_block_argmin<<<(nblocks + 255) / 256, 256, 0, s>>>(scores, nblocks, allow, bmap);
  return n;
}


}  // namespace hpez
