// k_level_md3.cu -- a 3D level of the multi-dimensional paradigm (Sec. 5.3,
// Eq. 8): the finest level streamed in one launch (below), other levels in
// two launches: even planes, then odd planes.
//
// The paradigm's sub-pass k' predicts the points with exactly k' odd
// coordinates from points with k'-1 odd coordinates, so any order that
// computes a point after the points it reads gives the same values.  This
// kernel groups the points by the parity of their plane:
//   even planes: (0,1,0) and (0,0,1) from coarse points, then (0,1,1)
//                from those -- everything a 2D level of the plane needs;
//   odd planes:  (1,0,0) from coarse planes, then (1,0,1) and (1,1,0),
//                then (1,1,1); their predictions along dim 0 read the even
//                planes, which the first launch has finished.
// A CTA owns E1 rows of one plane (full rows) and recomputes the points of
// the 3 rows on either side that its own points read along dim 1; the
// plane's values it builds stay in shared memory, values of other planes
// come from the level grid (global memory, L2-resident for neighbouring
// planes).  Row-major warps keep every global access a contiguous row.
#include <cuda.h>

#include <type_traits>

#include "hpez_internal.cuh"
#include "hpez_launch.h"

namespace hpez {
namespace {

// the neighbours of a point along a line, j = -3..3 (j != 0), through a
// functor; prediction with the stencil its position selects
template <int KIND, class F>
__device__ __forceinline__ float predict_by(const F& at, int u, int m) {
  const int f = choose_formula(KIND, false, u, m);
  float m3 = 0.f, p1 = 0.f, p3 = 0.f;
  const float m1 = at(-1);
  switch (f) {
    case F_COPY:
      break;
    case F_EXTRAP:
      m3 = at(-3);
      break;
    case F_LIN:
      p1 = at(1);
      break;
    case F_NAK4:
    case F_NAT4:
      m3 = at(-3);
      p1 = at(1);
      p3 = at(3);
      break;
    case F_NAK3L:
    case F_NAT3L:
      m3 = at(-3);
      p1 = at(1);
      break;
    case F_NAK3R:
    case F_NAT3R:
      p1 = at(1);
      p3 = at(3);
      break;
  }
  return eval_formula(f, m3, 0.f, m1, p1, 0.f, p3);
}

struct Tile {
  int u0;          // plane (level grid)
  int R0, Rlo, Rhi, Thi;  // tile rows [R0, Thi), region rows [Rlo, Rhi)
  int W;           // shared row length
};

__device__ __forceinline__ Tile make_tile(const LevelMD& P, int u0, int t1,
                                          int E1) {
  Tile T;
  T.u0 = u0;
  T.R0 = t1 * E1;
  T.Thi = min(T.R0 + E1, (int)P.g.m[1]);
  T.Rlo = max(T.R0 - 3, 0);
  T.Rhi = min(T.Thi + 3, (int)P.g.m[1]);
  T.W = (int)P.g.m[2];
  return T;
}

// One point: quantize (compress) or reconstruct (decompress), write the
// code / reconstruction when the point is the CTA's own, keep the value in
// shared memory.
template <bool kDecomp>
__device__ __forceinline__ void finish(const LevelMD& P, const Tile& T, int r,
                                       int c, float p, float* sm,
                                       const float* __restrict__ X,
                                       const uint16_t* __restrict__ codes_full,
                                       const float* __restrict__ outl_full,
                                       float* __restrict__ Rs,
                                       uint16_t* __restrict__ Cs, float el,
                                       float inv2, float twoe, bool keep_recon) {
  const LevelGeom& g = P.g;
  const uint32_t fi = (uint32_t)T.u0 * g.step[0] * P.fst[0] +
                      (uint32_t)r * g.step[1] * P.fst[1] + (uint32_t)c * g.step[2];
  const uint32_t gi = (uint32_t)T.u0 * g.gst[0] + (uint32_t)r * g.gst[1] + (uint32_t)c;
  const bool own = r >= T.R0 && r < T.Thi;
  float rec;
  if (!kDecomp) {
    const unsigned code = quantize(X[fi], p, el, inv2, twoe, rec);
    if (own) {
      Cs[gi] = (uint16_t)code;
      if (keep_recon) Rs[gi] = rec;
    }
  } else {
    const unsigned code = codes_full[fi];
    rec = code ? dequantize(code, p, twoe) : outl_full[fi];
    if (own) Rs[gi] = rec;
  }
  sm[(r - T.Rlo) * T.W + c] = rec;
}

// ---------------------------------------------------------------------
// even planes: coarse copy, (0,1,0), (0,0,1), (0,1,1)
// ---------------------------------------------------------------------
template <bool kDecomp, int KIND>
__device__ __forceinline__ void md3_even_body(
    const LevelMD& P, int E1, int nt1, const float* __restrict__ X,
    const uint16_t* __restrict__ codes_full, const float* __restrict__ outl_full,
    const float* __restrict__ Rc, const uint16_t* __restrict__ Cc, float* __restrict__ Rs,
    uint16_t* __restrict__ Cs, const Ctl* __restrict__ ctl, unsigned bid) {
  if (ctl->status || ctl->is_const) return;
  extern __shared__ float sm[];
  const int li = P.level - 1;
  const float el = ctl->el[li], inv2 = ctl->inv2[li], twoe = ctl->twoe[li];
  const LevelGeom& g = P.g;
  const int c0 = (int)(bid / (unsigned)nt1);
  const Tile T = make_tile(P, 2 * c0, (int)(bid % (unsigned)nt1), E1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int m1 = (int)g.m[1], m2 = (int)g.m[2];
  // even planes hold every value the odd planes read along dim 0
  const bool keep = true;
  // coarse points of the region's even rows
  const int r_even0 = T.Rlo + (T.Rlo & 1);
  for (int r = r_even0 + 2 * warp; r < T.Rhi; r += 2 * nw) {
    const uint32_t cb = (uint32_t)c0 * P.gc.gst[0] + (uint32_t)(r >> 1) * P.gc.gst[1];
    const uint32_t gb = (uint32_t)T.u0 * g.gst[0] + (uint32_t)r * g.gst[1];
    const bool own = r >= T.R0 && r < T.Thi;
    for (int c = 2 * lane; c < m2; c += 64) {
      const float v = __ldg(Rc + cb + (c >> 1));
      sm[(r - T.Rlo) * T.W + c] = v;
      if (own) {
        if (!kDecomp) Cs[gb + c] = Cc[cb + (c >> 1)];
        if (kDecomp || P.write_recon) Rs[gb + c] = v;
      }
    }
  }
  __syncthreads();
  // (0,0,1): even rows of the region, odd columns, along dim 2
  for (int r = r_even0 + 2 * warp; r < T.Rhi; r += 2 * nw) {
    const float* row = sm + (r - T.Rlo) * T.W;
    for (int c = 2 * lane + 1; c < m2; c += 64) {
      const float pd = predict_by<KIND>([&](int j) { return row[c + j]; }, c, m2);
      finish<kDecomp>(P, T, r, c, __fmul_rn(P.w[4][2], pd), sm, X, codes_full,
                      outl_full, Rs, Cs, el, inv2, twoe, keep);
    }
  }
  // (0,1,0): odd rows of the tile, even columns, along dim 1 (coarse rows)
  const int r_odd0 = T.R0 + ((T.R0 & 1) ^ 1);
  for (int r = r_odd0 + 2 * warp; r < T.Thi; r += 2 * nw) {
    for (int c = 2 * lane; c < m2; c += 64) {
      const float pd = predict_by<KIND>(
          [&](int j) { return sm[(r + j - T.Rlo) * T.W + c]; }, r, m1);
      finish<kDecomp>(P, T, r, c, __fmul_rn(P.w[2][1], pd), sm, X, codes_full,
                      outl_full, Rs, Cs, el, inv2, twoe, keep);
    }
  }
  __syncthreads();
  // (0,1,1): odd rows of the tile, odd columns, along dims 1 and 2
  for (int r = r_odd0 + 2 * warp; r < T.Thi; r += 2 * nw) {
    const float* row = sm + (r - T.Rlo) * T.W;
    for (int c = 2 * lane + 1; c < m2; c += 64) {
      const float p1 = predict_by<KIND>(
          [&](int j) { return sm[(r + j - T.Rlo) * T.W + c]; }, r, m1);
      const float p2 = predict_by<KIND>([&](int j) { return row[c + j]; }, c, m2);
      const float p = __fadd_rn(__fmul_rn(P.w[6][1], p1), __fmul_rn(P.w[6][2], p2));
      finish<kDecomp>(P, T, r, c, p, sm, X, codes_full, outl_full, Rs, Cs, el,
                      inv2, twoe, keep);
    }
  }
}

// ---------------------------------------------------------------------
// odd planes: (1,0,0), (1,0,1), (1,1,0), (1,1,1)
// ---------------------------------------------------------------------
template <bool kDecomp, int KIND>
__device__ __forceinline__ void md3_odd_body(
    const LevelMD& P, int E1, int nt1, const float* __restrict__ X,
    const uint16_t* __restrict__ codes_full, const float* __restrict__ outl_full,
    const float* __restrict__ Rc, float* __restrict__ Rs, uint16_t* __restrict__ Cs,
    const Ctl* __restrict__ ctl, unsigned bid) {
  if (ctl->status || ctl->is_const) return;
  extern __shared__ float sm[];
  const int li = P.level - 1;
  const float el = ctl->el[li], inv2 = ctl->inv2[li], twoe = ctl->twoe[li];
  const LevelGeom& g = P.g;
  const int c0 = (int)(bid / (unsigned)nt1);
  const Tile T = make_tile(P, 2 * c0 + 1, (int)(bid % (unsigned)nt1), E1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int m0 = (int)g.m[0], m1 = (int)g.m[1], m2 = (int)g.m[2];
  const bool keep = kDecomp || P.write_recon;
  const uint32_t gst0 = g.gst[0], gst1 = g.gst[1];
  const int u0 = T.u0;
  // along dim 0: the point's column in the even planes u0 + j of the level
  // grid, which the first launch has finished
  auto plane_at = [=](int r, int c) {
    return [=](int j) {
      return __ldg(Rs + (uint32_t)(u0 + j) * gst0 + (uint32_t)r * gst1 + c);
    };
  };
  const int r_even0 = T.Rlo + (T.Rlo & 1);
  // (1,0,0): even rows of the region, even columns, from coarse planes
  for (int r = r_even0 + 2 * warp; r < T.Rhi; r += 2 * nw) {
    const uint32_t cb = (uint32_t)(r >> 1) * P.gc.gst[1];
    for (int c = 2 * lane; c < m2; c += 64) {
      const float pd = predict_by<KIND>(
          [&](int j) {
            return __ldg(Rc + (uint32_t)((T.u0 + j) >> 1) * P.gc.gst[0] + cb + (c >> 1));
          },
          T.u0, m0);
      finish<kDecomp>(P, T, r, c, __fmul_rn(P.w[1][0], pd), sm, X, codes_full,
                      outl_full, Rs, Cs, el, inv2, twoe, keep);
    }
  }
  __syncthreads();
  // (1,0,1): even rows of the region, odd columns, along dims 0 and 2
  for (int r = r_even0 + 2 * warp; r < T.Rhi; r += 2 * nw) {
    const float* row = sm + (r - T.Rlo) * T.W;
    for (int c = 2 * lane + 1; c < m2; c += 64) {
      const float p0 = predict_by<KIND>(plane_at(r, c), T.u0, m0);
      const float p2 = predict_by<KIND>([&](int j) { return row[c + j]; }, c, m2);
      const float p = __fadd_rn(__fmul_rn(P.w[5][0], p0), __fmul_rn(P.w[5][2], p2));
      finish<kDecomp>(P, T, r, c, p, sm, X, codes_full, outl_full, Rs, Cs, el,
                      inv2, twoe, keep);
    }
  }
  // (1,1,0): odd rows of the tile, even columns, along dims 0 and 1
  const int r_odd0 = T.R0 + ((T.R0 & 1) ^ 1);
  for (int r = r_odd0 + 2 * warp; r < T.Thi; r += 2 * nw) {
    for (int c = 2 * lane; c < m2; c += 64) {
      const float p0 = predict_by<KIND>(plane_at(r, c), T.u0, m0);
      const float p1 = predict_by<KIND>(
          [&](int j) { return sm[(r + j - T.Rlo) * T.W + c]; }, r, m1);
      const float p = __fadd_rn(__fmul_rn(P.w[3][0], p0), __fmul_rn(P.w[3][1], p1));
      finish<kDecomp>(P, T, r, c, p, sm, X, codes_full, outl_full, Rs, Cs, el,
                      inv2, twoe, keep);
    }
  }
  __syncthreads();
  // (1,1,1): odd rows of the tile, odd columns, along dims 0, 1 and 2
  for (int r = r_odd0 + 2 * warp; r < T.Thi; r += 2 * nw) {
    const float* row = sm + (r - T.Rlo) * T.W;
    for (int c = 2 * lane + 1; c < m2; c += 64) {
      const float p0 = predict_by<KIND>(plane_at(r, c), T.u0, m0);
      const float p1 = predict_by<KIND>(
          [&](int j) { return sm[(r + j - T.Rlo) * T.W + c]; }, r, m1);
      const float p2 = predict_by<KIND>([&](int j) { return row[c + j]; }, c, m2);
      float p = __fmul_rn(P.w[7][0], p0);
      p = __fadd_rn(p, __fmul_rn(P.w[7][1], p1));
      p = __fadd_rn(p, __fmul_rn(P.w[7][2], p2));
      finish<kDecomp>(P, T, r, c, p, sm, X, codes_full, outl_full, Rs, Cs, el,
                      inv2, twoe, keep);
    }
  }
}

template <bool kDecomp, int KIND>
__global__ void __launch_bounds__(256)
    k_md3_even(LevelMD P, int E1, int nt1, const float* __restrict__ X,
               const uint16_t* __restrict__ codes_full,
               const float* __restrict__ outl_full, const float* __restrict__ Rc,
               const uint16_t* __restrict__ Cc, float* __restrict__ Rs,
               uint16_t* __restrict__ Cs, const Ctl* __restrict__ ctl) {
  md3_even_body<kDecomp, KIND>(P, E1, nt1, X, codes_full, outl_full, Rc, Cc, Rs, Cs, ctl,
                               blockIdx.x);
}

template <bool kDecomp, int KIND>
__global__ void __launch_bounds__(256)
    k_md3_odd(LevelMD P, int E1, int nt1, const float* __restrict__ X,
              const uint16_t* __restrict__ codes_full,
              const float* __restrict__ outl_full, const float* __restrict__ Rc,
              float* __restrict__ Rs, uint16_t* __restrict__ Cs,
              const Ctl* __restrict__ ctl) {
  md3_odd_body<kDecomp, KIND>(P, E1, nt1, X, codes_full, outl_full, Rc, Rs, Cs, ctl,
                              blockIdx.x);
}

// batched, persistent: job j owns the tiles [off[j], off[j+1]) of the
// launch (even planes in one launch, odd planes in the next)
template <bool kDecomp, int KIND, bool kOdd>
__global__ void __launch_bounds__(256)
    k_md3_batch(const MD3Job* __restrict__ J, const uint32_t* __restrict__ off, int nj) {
  // the job's level geometry, read in every inner loop, in shared memory
  // (the single-field kernel reads it from its parameters)
  __shared__ LevelMD sP;
  static_assert(sizeof(LevelMD) % 4 == 0, "word copy");
  for_each_batch_block(off, nj, [&](int j, uint32_t t) {
    const MD3Job& q = J[j];
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&q.P);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sP);
    for (int i = threadIdx.x; i < (int)(sizeof(LevelMD) / 4); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    if (kOdd)
      md3_odd_body<kDecomp, KIND>(sP, q.E1, q.nt1, q.X, q.codes_full, q.outl_full, q.Rc,
                                  q.Rs, q.Cs, q.ctl, t);
    else
      md3_even_body<kDecomp, KIND>(sP, q.E1, q.nt1, q.X, q.codes_full, q.outl_full, q.Rc,
                                   q.Cc, q.Rs, q.Cs, q.ctl, t);
  });
}

template <bool kDecomp, int KIND, bool kOdd>
void launch_md3_b(const MD3Job* J, const uint32_t* off, int nj, uint32_t nblk, size_t smem,
                  int num_sms, int max_ctas, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_md3_batch<kDecomp, KIND, kOdd>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const unsigned grid =
      persistent_grid(k_md3_batch<kDecomp, KIND, kOdd>, 256, smem, nblk, num_sms, max_ctas);
  k_md3_batch<kDecomp, KIND, kOdd><<<grid, 256, smem, s>>>(J, off, nj);
}

template <bool kDecomp, int KIND>
void launch_md3_k(const LevelMD& P, int E1, const SweepBufs& B, const float* Rc,
                  const uint16_t* Cc, float* Rs, uint16_t* Cs, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_md3_even<kDecomp, KIND>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_md3_odd<kDecomp, KIND>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const int m0 = (int)P.g.m[0], m1 = (int)P.g.m[1];
  const int nt1 = (m1 + E1 - 1) / E1;
  const size_t smem = md3_smem_bytes(P, E1);
  const unsigned ge = (unsigned)(((m0 + 1) / 2) * nt1), go = (unsigned)((m0 / 2) * nt1);
  if (ge)
    k_md3_even<kDecomp, KIND><<<ge, 256, smem, s>>>(P, E1, nt1, B.x, B.codes_full,
                                                   B.outl_full, Rc, Cc, Rs, Cs, B.ctl);
  if (go)
    k_md3_odd<kDecomp, KIND><<<go, 256, smem, s>>>(P, E1, nt1, B.x, B.codes_full,
                                                  B.outl_full, Rc, Rs, Cs, B.ctl);
}


// ---------------------------------------------------------------------
// The finest level streamed through shared memory, one launch.
//
// A CTA owns a tile of kS1 x kS2 points (dims 1, 2) of the planes of a
// chunk and walks them in an order that computes every plane after the
// planes it reads: even plane k (a 2D level of the plane from its coarse
// points), then odd plane k as soon as the even planes it reads along dim 0
// (k-1 .. k+2, as its stencil selects) are done.  The even planes live in a
// ring of shared-memory buffers until no odd plane reads them, so the
// level's values never round-trip through HBM; the even planes just
// outside the chunk that its odd planes read are recomputed, not written.
// Each buffer holds the tile and a 3-point halo on every side; a point of
// the halo is computed when a point of the tile reads it (the same value
// the owning CTA computes).  The input of each plane -- the field values
// (compress) or codes (decompress) of the tile and halo, and for an even
// plane its coarse points and (compress) their codes -- arrives by TMA
// tensor copies issued kNB planes
// ahead on one mbarrier per buffer, so the copies of later planes overlap
// the arithmetic of this one.  Every wait is bounded: on expiry the CTA
// records a timeout, waits (bounded) for its copies in flight and returns.
// ---------------------------------------------------------------------
constexpr int kS1 = 16, kS2 = 128;                 // tile rows, columns
constexpr int kBR = kS1 + 6, kBC = kS2 + 6;        // plane buffer, halo 3
// TMA boxes start every row on a 16-byte boundary: the input box at column
// C0 - kXOff, the coarse boxes (values f32, codes u16) at C0/2 - kCOff; both
// offsets and C0/2 are multiples of 8 elements, and every box row is a
// whole number of 16-byte units
constexpr int kXOff = 8, kCOff = 8;
constexpr int kXR = kS1 + 6, kXC = kS2 + 2 * kXOff;  // rows from R0-3
constexpr int kCR = kS1 / 2 + 3, kCC = kS2 / 2 + 2 * kCOff;  // rows from R0/2-1
static_assert(kS2 % 16 == 0 && kXOff % 8 == 0 && kCOff % 8 == 0,
              "TMA x coordinates of every tile are multiples of 8 elements");
static_assert((kXC * 2) % 16 == 0 && (kCC * 2) % 16 == 0,
              "TMA box rows are whole 16-byte units");
static_assert(kXOff >= 3 && kCOff >= 2, "boxes cover the halo");
constexpr int kNB = 3;                             // input boxes in flight
constexpr int kStreamThreads = 512;
constexpr int kWaitLimit = 1 << 24;
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s

__host__ __device__ constexpr int round128(int v) { return (v + 127) & ~127; }

template <bool kDecomp>
struct StreamLayout {
  using In = typename std::conditional<kDecomp, uint16_t, float>::type;
  static constexpr int kInBytes = kXR * kXC * (int)sizeof(In);
  static constexpr int kCBytes = kCR * kCC * 4;
  static constexpr int kCCBytes = kDecomp ? 0 : kCR * kCC * 2;  // coarse codes
  static constexpr int kBufBytes = kBR * kBC * 4;
  static constexpr int kOffIn = 128;
  static constexpr int kOffC = kOffIn + kNB * round128(kInBytes);
  static constexpr int kOffCC = kOffC + kNB * round128(kCBytes);
  static constexpr int kOffBuf = kOffCC + kNB * round128(kCCBytes);
  static constexpr int bytes(int ring) { return kOffBuf + (ring + 1) * round128(kBufBytes); }
};

template <int KIND>
struct Ring {
  static constexpr int n = KIND == LINEAR ? 3 : 4;   // live even planes
  static constexpr int ahead = KIND == LINEAR ? 1 : 2;  // planes read past k
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

// A wait ends after kWaitNs of wall time (the nanosecond global timer) or
// kWaitLimit polls, whichever comes first; false: the copy did not land.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (int it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// 3D tiled tensor copy global -> shared, completing on bar
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// prediction with the interior stencil when every neighbour it reads
// exists (the choice choose_formula makes there), else the general path
template <int KIND, class F>
__device__ __forceinline__ float predict_fast(const F& at, int u, int m) {
  if (KIND == LINEAR) {
    if (u + 1 <= m - 1) return eval_formula(F_LIN, 0.f, 0.f, at(-1), at(1), 0.f, 0.f);
  } else if (u >= 3 && u + 3 <= m - 1) {
    return eval_formula(KIND == CUBIC_NAK ? F_NAK4 : F_NAT4, at(-3), 0.f, at(-1), at(1), 0.f,
                        at(3));
  }
  return predict_by<KIND>(at, u, m);
}

// the plane schedule of one CTA: even planes [next_e, e_end], odd planes
// [k_odd, k_odd_end); an odd plane k follows the even planes up to k+ahead
struct Sched {
  int k_odd, k_odd_end, next_e, e_end, ahead, ke;
  __device__ bool next(bool& odd, int& k) {
    if (k_odd < k_odd_end) {
      const int need = min(ke - 1, k_odd + ahead);
      if (next_e <= need) {
        odd = false;
        k = next_e++;
        return true;
      }
      odd = true;
      k = k_odd++;
      return true;
    }
    if (next_e <= e_end) {
      odd = false;
      k = next_e++;
      return true;
    }
    return false;
  }
};

struct StreamCtx {
  int R0, C0, m0, m1, m2;
  uint32_t gst0, gst1;
  float el, inv2, twoe;
};

// quantize (compress) or reconstruct (decompress) one point, keep it in
// the plane buffer, write the code / reconstruction of an owned point
template <bool kDecomp, class In>
__device__ __forceinline__ void stream_finish(const StreamCtx& S, const LevelMD& P, int u0,
                                              int r, int c, int br, int bc, int xc, float p,
                                              bool own, float* B, const In* xb,
                                              const float* __restrict__ outl,
                                              float* __restrict__ Rs,
                                              uint16_t* __restrict__ Cs) {
  const uint32_t fi = (uint32_t)u0 * S.gst0 + (uint32_t)r * S.gst1 + (uint32_t)c;
  float rec;
  if (!kDecomp) {
    const unsigned code = quantize_fast((float)xb[br * kXC + xc], p, S.el, S.inv2, S.twoe, rec);
    if (own) Cs[fi] = (uint16_t)code;
  } else {
    const unsigned code = (unsigned)xb[br * kXC + xc];
    rec = code ? dequantize(code, p, S.twoe) : outl[fi];
    if (own) Rs[fi] = rec;
  }
  B[br * kBC + bc] = rec;
}

// even plane k: coarse points, (0,0,1) and (0,1,0), then (0,1,1)
// HR: the region's extra even rows / columns beyond the tile's (2 for
// the cubic stencils' +-3 reads, 0 when only +-1 is read)
template <bool kDecomp, int KIND, int HR, class In>
__device__ __forceinline__ void stream_even(const StreamCtx& S, const LevelMD& P, int k,
                                            bool own_e, float* B, const In* xb,
                                            const float* cb, const uint16_t* ccb,
                                            const float* __restrict__ outl,
                                            float* __restrict__ Rs,
                                            uint16_t* __restrict__ Cs) {
  constexpr int RR = kS1 / 2 + 1 + HR, RC = kS2 / 2 + 1 + HR;
  const int tid = threadIdx.x;
  const int u0 = 2 * k;
  const int r_hi = min(S.R0 + kS1, S.m1), c_hi = min(S.C0 + kS2, S.m2);
  for (int i = tid; i < RR * RC; i += kStreamThreads) {
    const int ii = i / RC, jj = i - ii * RC;
    const int r = S.R0 - HR + 2 * ii, c = S.C0 - HR + 2 * jj;
    if (r < 0 || r >= S.m1 || c < 0 || c >= S.m2) continue;
    const float v = cb[(ii + 1 - HR / 2) * kCC + jj + kCOff - HR / 2];
    B[(3 - HR + 2 * ii) * kBC + 3 - HR + 2 * jj] = v;
    if (own_e && r >= S.R0 && r < r_hi && c >= S.C0 && c < c_hi) {
      const uint32_t fi = (uint32_t)u0 * S.gst0 + (uint32_t)r * S.gst1 + (uint32_t)c;
      if (!kDecomp) {
        Cs[fi] = ccb[(ii + 1 - HR / 2) * kCC + jj + kCOff - HR / 2];
      } else {
        Rs[fi] = v;
      }
    }
  }
  __syncthreads();
  // (0,0,1): even rows of the region, odd columns of the tile, along dim 2;
  // (0,1,0): odd rows of the tile, even columns of the region, along dim 1
  constexpr int n1 = RR * (kS2 / 2), n2 = (kS1 / 2) * RC;
  for (int i = tid; i < n1 + n2; i += kStreamThreads) {
    if (i < n1) {
      const int ii = i / (kS2 / 2), jj = i - ii * (kS2 / 2);
      const int r = S.R0 - HR + 2 * ii, c = S.C0 + 1 + 2 * jj;
      if (r < 0 || r >= S.m1 || c >= S.m2) continue;
      const int br = 3 - HR + 2 * ii, bc = 4 + 2 * jj;
      const float* row = B + br * kBC + bc;
      const float pd = predict_fast<KIND>([&](int j) { return row[j]; }, c, S.m2);
      stream_finish<kDecomp>(S, P, u0, r, c, br, bc, kXOff + 1 + 2 * jj, __fmul_rn(P.w[4][2], pd),
                             own_e && r >= S.R0 && r < r_hi, B, xb, outl, Rs, Cs);
    } else {
      const int i2 = i - n1;
      const int ii = i2 / RC, jj = i2 - ii * RC;
      const int r = S.R0 + 1 + 2 * ii, c = S.C0 - HR + 2 * jj;
      if (r >= S.m1 || c < 0 || c >= S.m2) continue;
      const int br = 4 + 2 * ii, bc = 3 - HR + 2 * jj;
      const float* col = B + br * kBC + bc;
      const float pd = predict_fast<KIND>([&](int j) { return col[j * kBC]; }, r, S.m1);
      stream_finish<kDecomp>(S, P, u0, r, c, br, bc, kXOff - HR + 2 * jj, __fmul_rn(P.w[2][1], pd),
                             own_e && c >= S.C0 && c < c_hi, B, xb, outl, Rs, Cs);
    }
  }
  __syncthreads();
  // (0,1,1): odd rows and odd columns of the tile, along dims 1 and 2
  for (int i = tid; i < (kS1 / 2) * (kS2 / 2); i += kStreamThreads) {
    const int ii = i / (kS2 / 2), jj = i - ii * (kS2 / 2);
    const int r = S.R0 + 1 + 2 * ii, c = S.C0 + 1 + 2 * jj;
    if (r >= S.m1 || c >= S.m2) continue;
    const int br = 4 + 2 * ii, bc = 4 + 2 * jj;
    const float* pt = B + br * kBC + bc;
    const float p1 = predict_fast<KIND>([&](int j) { return pt[j * kBC]; }, r, S.m1);
    const float p2 = predict_fast<KIND>([&](int j) { return pt[j]; }, c, S.m2);
    const float p = __fadd_rn(__fmul_rn(P.w[6][1], p1), __fmul_rn(P.w[6][2], p2));
    stream_finish<kDecomp>(S, P, u0, r, c, br, bc, kXOff + 1 + 2 * jj, p, own_e, B, xb, outl, Rs,
                           Cs);
  }
}

// prediction along dim 0 of odd plane u0 from the even planes' buffers
// (E[0..3] = planes u0-3, u0-1, u0+1, u0+3) with the plane's stencil f0;
// FZ >= 0: f0 is known to be FZ (the interior stencil of the plane)
template <int FZ>
__device__ __forceinline__ float pred_dim0(int f0, const float* const E[4], int idx) {
  if (FZ == F_LIN) return eval_formula(F_LIN, 0.f, 0.f, E[1][idx], E[2][idx], 0.f, 0.f);
  if (FZ == F_NAK4 || FZ == F_NAT4)
    return eval_formula(FZ, E[0][idx], 0.f, E[1][idx], E[2][idx], 0.f, E[3][idx]);
  float m3 = 0.f, p1 = 0.f, p3 = 0.f;
  const float m1 = E[1][idx];
  switch (f0) {
    case F_COPY:
      break;
    case F_EXTRAP:
      m3 = E[0][idx];
      break;
    case F_LIN:
      p1 = E[2][idx];
      break;
    case F_NAK4:
    case F_NAT4:
      m3 = E[0][idx];
      p1 = E[2][idx];
      p3 = E[3][idx];
      break;
    case F_NAK3L:
    case F_NAT3L:
      m3 = E[0][idx];
      p1 = E[2][idx];
      break;
    case F_NAK3R:
    case F_NAT3R:
      p1 = E[2][idx];
      p3 = E[3][idx];
      break;
  }
  return eval_formula(f0, m3, 0.f, m1, p1, 0.f, p3);
}

// odd plane k: (1,0,0), then (1,0,1) and (1,1,0), then (1,1,1); FZ as
// for pred_dim0
template <bool kDecomp, int KIND, int FZ, int HR, class In>
__device__ __forceinline__ void stream_odd(const StreamCtx& S, const LevelMD& P, int k,
                                           int f0, float* O, const float* ring, const In* xb,
                                           const float* __restrict__ outl,
                                           float* __restrict__ Rs,
                                           uint16_t* __restrict__ Cs) {
  constexpr int RN = Ring<KIND>::n;
  constexpr int PB = round128(kBR * kBC * 4) / 4;
  constexpr int RR = kS1 / 2 + 1 + HR, RC = kS2 / 2 + 1 + HR;
  const int tid = threadIdx.x;
  const int u0 = 2 * k + 1;
  const float* E[4] = {ring + ((k + RN - 1) % RN) * PB, ring + (k % RN) * PB,
                       ring + ((k + 1) % RN) * PB, ring + ((k + 2) % RN) * PB};
  const int r_hi = min(S.R0 + kS1, S.m1), c_hi = min(S.C0 + kS2, S.m2);
  for (int i = tid; i < RR * RC; i += kStreamThreads) {
    const int ii = i / RC, jj = i - ii * RC;
    const int r = S.R0 - HR + 2 * ii, c = S.C0 - HR + 2 * jj;
    if (r < 0 || r >= S.m1 || c < 0 || c >= S.m2) continue;
    const int br = 3 - HR + 2 * ii, bc = 3 - HR + 2 * jj;
    const float pd = pred_dim0<FZ>(f0, E, br * kBC + bc);
    stream_finish<kDecomp>(S, P, u0, r, c, br, bc, kXOff - HR + 2 * jj, __fmul_rn(P.w[1][0], pd),
                           r >= S.R0 && r < r_hi && c >= S.C0 && c < c_hi, O, xb, outl, Rs,
                           Cs);
  }
  __syncthreads();
  constexpr int n1 = RR * (kS2 / 2), n2 = (kS1 / 2) * RC;
  for (int i = tid; i < n1 + n2; i += kStreamThreads) {
    if (i < n1) {
      // (1,0,1): even rows of the region, odd columns of the tile
      const int ii = i / (kS2 / 2), jj = i - ii * (kS2 / 2);
      const int r = S.R0 - HR + 2 * ii, c = S.C0 + 1 + 2 * jj;
      if (r < 0 || r >= S.m1 || c >= S.m2) continue;
      const int br = 3 - HR + 2 * ii, bc = 4 + 2 * jj;
      const float* pt = O + br * kBC + bc;
      const float p0 = pred_dim0<FZ>(f0, E, br * kBC + bc);
      const float p2 = predict_fast<KIND>([&](int j) { return pt[j]; }, c, S.m2);
      const float p = __fadd_rn(__fmul_rn(P.w[5][0], p0), __fmul_rn(P.w[5][2], p2));
      stream_finish<kDecomp>(S, P, u0, r, c, br, bc, kXOff + 1 + 2 * jj, p,
                             r >= S.R0 && r < r_hi, O, xb, outl, Rs, Cs);
    } else {
      // (1,1,0): odd rows of the tile, even columns of the region
      const int i2 = i - n1;
      const int ii = i2 / RC, jj = i2 - ii * RC;
      const int r = S.R0 + 1 + 2 * ii, c = S.C0 - HR + 2 * jj;
      if (r >= S.m1 || c < 0 || c >= S.m2) continue;
      const int br = 4 + 2 * ii, bc = 3 - HR + 2 * jj;
      const float* pt = O + br * kBC + bc;
      const float p0 = pred_dim0<FZ>(f0, E, br * kBC + bc);
      const float p1 = predict_fast<KIND>([&](int j) { return pt[j * kBC]; }, r, S.m1);
      const float p = __fadd_rn(__fmul_rn(P.w[3][0], p0), __fmul_rn(P.w[3][1], p1));
      stream_finish<kDecomp>(S, P, u0, r, c, br, bc, kXOff - HR + 2 * jj, p,
                             c >= S.C0 && c < c_hi, O, xb, outl, Rs, Cs);
    }
  }
  __syncthreads();
  // (1,1,1): odd rows and odd columns of the tile, along dims 0, 1 and 2
  for (int i = tid; i < (kS1 / 2) * (kS2 / 2); i += kStreamThreads) {
    const int ii = i / (kS2 / 2), jj = i - ii * (kS2 / 2);
    const int r = S.R0 + 1 + 2 * ii, c = S.C0 + 1 + 2 * jj;
    if (r >= S.m1 || c >= S.m2) continue;
    const int br = 4 + 2 * ii, bc = 4 + 2 * jj;
    const float* pt = O + br * kBC + bc;
    const float p0 = pred_dim0<FZ>(f0, E, br * kBC + bc);
    const float p1 = predict_fast<KIND>([&](int j) { return pt[j * kBC]; }, r, S.m1);
    const float p2 = predict_fast<KIND>([&](int j) { return pt[j]; }, c, S.m2);
    float p = __fmul_rn(P.w[7][0], p0);
    p = __fadd_rn(p, __fmul_rn(P.w[7][1], p1));
    p = __fadd_rn(p, __fmul_rn(P.w[7][2], p2));
    stream_finish<kDecomp>(S, P, u0, r, c, br, bc, kXOff + 1 + 2 * jj, p, true, O, xb, outl, Rs, Cs);
  }
}

template <bool kDecomp, int KIND>
__global__ void __launch_bounds__(kStreamThreads, 2)
    k_md3_stream(const __grid_constant__ CUtensorMap tm_in,
                 const __grid_constant__ CUtensorMap tm_c,
                 const __grid_constant__ CUtensorMap tm_cc, LevelMD P, int nt2,
                 int ntiles, int K, const float* __restrict__ outl, float* __restrict__ Rs,
                 uint16_t* __restrict__ Cs, Ctl* ctl, int drop_copy) {
  using L = StreamLayout<kDecomp>;
  using In = typename L::In;
  constexpr int RN = Ring<KIND>::n;
  if (ctl->status || ctl->is_const) return;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  float* ring = reinterpret_cast<float*>(smem + L::kOffBuf);
  float* O = ring + RN * (round128(L::kBufBytes) / 4);
  const int tid = threadIdx.x;
  const int li = P.level - 1;
  StreamCtx S;
  S.m0 = (int)P.g.m[0];
  S.m1 = (int)P.g.m[1];
  S.m2 = (int)P.g.m[2];
  S.gst0 = P.g.gst[0];
  S.gst1 = P.g.gst[1];
  S.el = ctl->el[li];
  S.inv2 = ctl->inv2[li];
  S.twoe = ctl->twoe[li];
  const int tile = (int)(blockIdx.x % (unsigned)ntiles);
  const int chunk = (int)(blockIdx.x / (unsigned)ntiles);
  S.R0 = (tile / nt2) * kS1;
  S.C0 = (tile % nt2) * kS2;
  // the region beyond the tile: +-3 reads need two more even rows and
  // columns on each side; linear reads +-1 (within the tile and one row /
  // column past it), except extrapolation at the field's end, which reads
  // 3 back and leaves the tile only when the last tile has under 4 rows or
  // columns
  const bool wide = KIND != LINEAR || S.m1 - S.R0 < 4 || S.m2 - S.C0 < 4;
  const int ke = (S.m0 + 1) / 2, ko = S.m0 / 2;
  const int K0 = chunk * K;
  const int K1o = min(K0 + K, ko), K1e = min(K0 + K, ke);
  if (K0 >= ke) return;
  // the first odd plane reads even plane K0-1 with a cubic stencil, or
  // when it is the last plane (extrapolation)
  const bool need_lo = KIND != LINEAR || (S.m0 % 2 == 0 && K0 == ko - 1);
  Sched sp;
  sp.k_odd = K0;
  sp.k_odd_end = K1o;
  sp.next_e = need_lo && K0 > 0 ? K0 - 1 : K0;
  sp.ahead = Ring<KIND>::ahead;
  sp.ke = ke;
  sp.e_end = max(K1e - 1, min(ke - 1, K1o - 1 + sp.ahead));
  Sched si = sp;  // issue cursor, kNB planes ahead

  // drop_copy > 0 (a test of the bounded waits): CTA 0 does not issue the
  // copies of its plane drop_copy - 1, so the wait for them expires
  auto issue = [&](int slot, bool odd, int k, int item) {
    if (blockIdx.x == 0 && item + 1 == drop_copy) return;
    uint64_t* b = bar + slot;
    mbar_expect_tx(b, (uint32_t)(L::kInBytes + (odd ? 0 : L::kCBytes + L::kCCBytes)));
    tma_load_3d(smem + L::kOffIn + slot * round128(L::kInBytes), &tm_in, b, S.C0 - kXOff,
                S.R0 - 3, odd ? 2 * k + 1 : 2 * k);
    if (!odd) {
      tma_load_3d(smem + L::kOffC + slot * round128(L::kCBytes), &tm_c, b, S.C0 / 2 - kCOff,
                  S.R0 / 2 - 1, k);
      if (!kDecomp)
        tma_load_3d(smem + L::kOffCC + slot * round128(L::kCCBytes), &tm_cc, b,
                    S.C0 / 2 - kCOff, S.R0 / 2 - 1, k);
    }
  };
  if (tid == 0) {
    for (int b = 0; b < kNB; ++b) mbar_init(bar + b);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  int issued = 0;
  {
    bool odd;
    int k;
    for (int b = 0; b < kNB && si.next(odd, k); ++b) {
      if (tid == 0) issue(b, odd, k, issued);
      ++issued;
    }
  }
  uint32_t phase = 0;  // parity bit per slot
  int done = 0;
  bool odd;
  int k;
  while (sp.next(odd, k)) {
    const int slot = done % kNB;
    const bool ok = mbar_wait(bar + slot, (phase >> slot) & 1u);
    if (__syncthreads_or(!ok)) {
      // a copy did not land: record it, let the copies in flight finish
      if (tid == 0) atomicCAS(&ctl->status, 0, ST_TIMEOUT);
      for (int d = done; d < issued; ++d) {  // at most kNB, distinct slots
        const int sl = d % kNB;
        mbar_wait(bar + sl, (phase >> sl) & 1u);
      }
      return;
    }
    phase ^= 1u << slot;
    const In* xb = reinterpret_cast<const In*>(smem + L::kOffIn + slot * round128(L::kInBytes));
    if (!odd) {
      const float* cb =
          reinterpret_cast<const float*>(smem + L::kOffC + slot * round128(L::kCBytes));
      const uint16_t* ccb =
          reinterpret_cast<const uint16_t*>(smem + L::kOffCC + slot * round128(L::kCCBytes));
      float* B = ring + (k % RN) * (round128(L::kBufBytes) / 4);
      if (wide)
        stream_even<kDecomp, KIND, 2>(S, P, k, k >= K0 && k < K1e, B, xb, cb, ccb, outl, Rs,
                                      Cs);
      else
        stream_even<kDecomp, KIND, 0>(S, P, k, k >= K0 && k < K1e, B, xb, cb, ccb, outl, Rs,
                                      Cs);
    } else {
      constexpr int FZ = KIND == LINEAR ? F_LIN : (KIND == CUBIC_NAK ? F_NAK4 : F_NAT4);
      const int f0 = choose_formula(KIND, false, 2 * k + 1, S.m0);
      if (f0 == FZ) {
        if (wide)
          stream_odd<kDecomp, KIND, FZ, 2>(S, P, k, f0, O, ring, xb, outl, Rs, Cs);
        else
          stream_odd<kDecomp, KIND, FZ, 0>(S, P, k, f0, O, ring, xb, outl, Rs, Cs);
      } else if (wide) {
        stream_odd<kDecomp, KIND, -1, 2>(S, P, k, f0, O, ring, xb, outl, Rs, Cs);
      } else {
        stream_odd<kDecomp, KIND, -1, 0>(S, P, k, f0, O, ring, xb, outl, Rs, Cs);
      }
    }
    ++done;
    __syncthreads();  // the slot and the plane buffers are free again
    bool odd2;
    int k2;
    if (si.next(odd2, k2)) {
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        issue(slot, odd2, k2, issued);
      }
      ++issued;
    }
  }
}

template <bool kDecomp, int KIND>
int launch_md3s_k(const CUtensorMap& tin, const CUtensorMap& tc, const CUtensorMap& tcc,
                  const LevelMD& P, const float* outl, float* Rs, uint16_t* Cs, Ctl* ctl,
                  int num_sms, int drop_copy, int chunks, cudaStream_t s) {
  const int smem = StreamLayout<kDecomp>::bytes(Ring<KIND>::n);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_md3_stream<kDecomp, KIND>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_md3_stream<kDecomp, KIND>,
                                                kStreamThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const int m0 = (int)P.g.m[0], m1 = (int)P.g.m[1], m2 = (int)P.g.m[2];
  const int nt1 = (m1 + kS1 - 1) / kS1, nt2 = (m2 + kS2 - 1) / kS2;
  const int ntiles = nt1 * nt2;
  const int ke = (m0 + 1) / 2;
  // chunks > 0 (an execution option) sets the chunk count; the default
  // fills the resident CTAs
  int nch = chunks > 0 ? chunks : (num_sms * per_sm) / ntiles;
  nch = std::max(1, std::min(nch, ke));
  const int K = (ke + nch - 1) / nch;
  nch = (ke + K - 1) / K;
  k_md3_stream<kDecomp, KIND><<<(unsigned)(ntiles * nch), kStreamThreads, smem, s>>>(
      tin, tc, tcc, P, nt2, ntiles, K, outl, Rs, Cs, ctl, drop_copy);
  return nch;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 3D tensor map over a compact grid (dims m2 fastest), box {bx, by, 1}
bool make_map(CUtensorMap* map, const void* base, bool u16, const uint32_t m[3], int bx,
              int by) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t es = u16 ? 2 : 4;
  const cuuint64_t dim[3] = {m[2], m[1], m[0]};
  const cuuint64_t stride[2] = {m[2] * es, (cuuint64_t)m[1] * m[2] * es};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, u16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
            const_cast<void*>(base), dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t md3_smem_bytes(const LevelMD& P, int E1) {
  return (size_t)(E1 + 6) * P.g.m[2] * sizeof(float);
}

// A 3D level of the multi-dimensional paradigm (no frozen dimension, one
// interpolator, no same-level halves): even planes, then odd planes.
void launch_level_md3(bool decomp, int kind, const LevelMD& P, int E1,
                      const SweepBufs& B, const float* Rc, const uint16_t* Cc,
                      float* Rs, uint16_t* Cs, cudaStream_t s) {
  if (decomp) {
    if (kind == LINEAR) launch_md3_k<true, LINEAR>(P, E1, B, Rc, Cc, Rs, Cs, s);
    else if (kind == CUBIC_NAK) launch_md3_k<true, CUBIC_NAK>(P, E1, B, Rc, Cc, Rs, Cs, s);
    else launch_md3_k<true, CUBIC_NAT>(P, E1, B, Rc, Cc, Rs, Cs, s);
  } else {
    if (kind == LINEAR) launch_md3_k<false, LINEAR>(P, E1, B, Rc, Cc, Rs, Cs, s);
    else if (kind == CUBIC_NAK) launch_md3_k<false, CUBIC_NAK>(P, E1, B, Rc, Cc, Rs, Cs, s);
    else launch_md3_k<false, CUBIC_NAT>(P, E1, B, Rc, Cc, Rs, Cs, s);
  }
}

}  // namespace hpez

namespace hpez {

// The finest level in one streamed launch: level-1 grid (unit steps, the
// grid is the field), rows of whole 16-byte units for the TMA copies of
// the input (codes need 8 columns), of the coarse grid and (compress) of
// its codes (16 columns), aligned bases.
bool md3s_supported(const LevelMD& P, bool decomp, const void* in, const float* Rc,
                    const uint16_t* Cc) {
  // the finest level: compress keeps no reconstruction, decompress writes it
  if (P.level != 1 || P.write_recon != (decomp ? 1 : 0)) return false;
  for (int d = 0; d < 3; ++d)
    if (P.g.step[d] != 1 || P.g.gst[d] != P.fst[d]) return false;
  if (P.g.m[0] < 2 || P.g.m[1] < 2 || P.g.m[2] < 2) return false;
  if (P.g.m[2] % 8 || P.gc.m[2] % 4) return false;
  if (!decomp && (P.gc.m[2] % 8 || ((uintptr_t)Cc & 15))) return false;
  if (P.g.gst[1] != P.g.m[2] || P.gc.gst[1] != P.gc.m[2] ||
      P.gc.gst[0] != P.gc.m[1] * P.gc.m[2])
    return false;
  if (((uintptr_t)in & 15) || ((uintptr_t)Rc & 15)) return false;
  return encode_tiled() != nullptr;
}

// Returns the chunks along dim 0 (0 when the tensor maps could not be
// made; nothing was launched then).
void launch_md3_batch(bool decomp, bool odd, int kind, const MD3Job* J, const uint32_t* off,
                      int nj, uint32_t nblk, size_t smem, int num_sms, int max_ctas,
                      cudaStream_t s) {
  if (!nblk) return;
#define HPEZ_MD3B(D, K, O) launch_md3_b<D, K, O>(J, off, nj, nblk, smem, num_sms, max_ctas, s)
  if (decomp) {
    if (odd) {
      if (kind == LINEAR) HPEZ_MD3B(true, LINEAR, true);
      else if (kind == CUBIC_NAK) HPEZ_MD3B(true, CUBIC_NAK, true);
      else HPEZ_MD3B(true, CUBIC_NAT, true);
    } else {
      if (kind == LINEAR) HPEZ_MD3B(true, LINEAR, false);
      else if (kind == CUBIC_NAK) HPEZ_MD3B(true, CUBIC_NAK, false);
      else HPEZ_MD3B(true, CUBIC_NAT, false);
    }
  } else {
    if (odd) {
      if (kind == LINEAR) HPEZ_MD3B(false, LINEAR, true);
      else if (kind == CUBIC_NAK) HPEZ_MD3B(false, CUBIC_NAK, true);
      else HPEZ_MD3B(false, CUBIC_NAT, true);
    } else {
      if (kind == LINEAR) HPEZ_MD3B(false, LINEAR, false);
      else if (kind == CUBIC_NAK) HPEZ_MD3B(false, CUBIC_NAK, false);
      else HPEZ_MD3B(false, CUBIC_NAT, false);
    }
  }
#undef HPEZ_MD3B
}

int launch_level_md3s(bool decomp, int kind, const LevelMD& P, const SweepBufs& B,
                      const float* Rc, const uint16_t* Cc, float* Rs, uint16_t* Cs,
                      Ctl* ctl, int num_sms, int drop_copy, int chunks, cudaStream_t s) {
  CUtensorMap tin, tc, tcc;
  const void* in = decomp ? (const void*)B.codes_full : (const void*)B.x;
  if (!make_map(&tin, in, decomp, P.g.m, kXC, kXR)) return 0;
  if (!make_map(&tc, Rc, false, P.gc.m, kCC, kCR)) return 0;
  if (decomp) {
    tcc = tc;  // unused
  } else if (!make_map(&tcc, Cc, true, P.gc.m, kCC, kCR)) {
    return 0;
  }
  const float* outl = B.outl_full;
  if (decomp) {
    if (kind == LINEAR)
      return launch_md3s_k<true, LINEAR>(tin, tc, tcc, P, outl, Rs, Cs, ctl, num_sms, drop_copy, chunks, s);
    if (kind == CUBIC_NAK)
      return launch_md3s_k<true, CUBIC_NAK>(tin, tc, tcc, P, outl, Rs, Cs, ctl, num_sms, drop_copy, chunks, s);
    return launch_md3s_k<true, CUBIC_NAT>(tin, tc, tcc, P, outl, Rs, Cs, ctl, num_sms, drop_copy, chunks, s);
  }
  if (kind == LINEAR)
    return launch_md3s_k<false, LINEAR>(tin, tc, tcc, P, outl, Rs, Cs, ctl, num_sms, drop_copy, chunks, s);
  if (kind == CUBIC_NAK)
    return launch_md3s_k<false, CUBIC_NAK>(tin, tc, tcc, P, outl, Rs, Cs, ctl, num_sms, drop_copy, chunks, s);
  return launch_md3s_k<false, CUBIC_NAT>(tin, tc, tcc, P, outl, Rs, Cs, ctl, num_sms, drop_copy, chunks, s);
}

}  // namespace hpez
