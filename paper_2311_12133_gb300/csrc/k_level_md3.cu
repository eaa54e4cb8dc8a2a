// k_level_md3.cu -- a 3D level of the multi-dimensional paradigm (Sec. 5.3,
// Eq. 8) in two launches: even planes, then odd planes.
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
__global__ void __launch_bounds__(256)
    k_md3_even(LevelMD P, int E1, int nt1, const float* __restrict__ X,
               const uint16_t* __restrict__ codes_full,
               const float* __restrict__ outl_full, const float* __restrict__ Rc,
               const uint16_t* __restrict__ Cc, float* __restrict__ Rs,
               uint16_t* __restrict__ Cs, const Ctl* __restrict__ ctl) {
  if (ctl->status || ctl->is_const) return;
  extern __shared__ float sm[];
  const int li = P.level - 1;
  const float el = ctl->el[li], inv2 = ctl->inv2[li], twoe = ctl->twoe[li];
  const LevelGeom& g = P.g;
  const int c0 = (int)(blockIdx.x / (unsigned)nt1);
  const Tile T = make_tile(P, 2 * c0, (int)(blockIdx.x % (unsigned)nt1), E1);
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
__global__ void __launch_bounds__(256)
    k_md3_odd(LevelMD P, int E1, int nt1, const float* __restrict__ X,
              const uint16_t* __restrict__ codes_full,
              const float* __restrict__ outl_full, const float* __restrict__ Rc,
              float* __restrict__ Rs, uint16_t* __restrict__ Cs,
              const Ctl* __restrict__ ctl) {
  if (ctl->status || ctl->is_const) return;
  extern __shared__ float sm[];
  const int li = P.level - 1;
  const float el = ctl->el[li], inv2 = ctl->inv2[li], twoe = ctl->twoe[li];
  const LevelGeom& g = P.g;
  const int c0 = (int)(blockIdx.x / (unsigned)nt1);
  const Tile T = make_tile(P, 2 * c0 + 1, (int)(blockIdx.x % (unsigned)nt1), E1);
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
