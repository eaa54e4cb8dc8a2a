// k_level_md.cu -- a level of the multi-dimensional paradigm (Sec. 5.3,
// Eq. 8) in three launches, one per sub-pass.
//
// Sub-pass k' predicts the points of the stride-s grid with exactly k' odd
// coordinates (in units of s) as the weighted sum, in ascending direction
// order, of the 1D predictions along each odd direction (Eq. 8 with the
// Eq. 14 weights of that odd set).  Its neighbours along an odd direction
// have that coordinate even, so they belong to sub-pass k'-1 (or are coarse
// points for k' = 1): the points of one sub-pass are independent, and a
// grid-wide barrier between sub-passes (the launch boundary) is all the
// ordering the level needs.  A thread owns one 2x2x2 cell of the level
// grid (the coarse point at its even corner and the new points around it)
// and handles the cell's points of its sub-pass; neighbouring threads own
// neighbouring cells along the fastest direction, so loads and stores of a
// warp cover contiguous rows.  The first launch also copies the coarse
// points (and, in compress, their codes) into the level grid.
#include "hpez_internal.cuh"
#include "hpez_launch.h"

namespace hpez {
namespace {

template <int KIND>
__device__ __forceinline__ float predict_line_k(const float* __restrict__ base,
                                                long long st, int u, int m) {
  return predict_line(base, st, u, m, KIND, false);
}

// the coarse point at coordinate v (even along direction d, so v/2 on the
// coarse grid) of direction d
__device__ __forceinline__ float coarse_at(const float* __restrict__ Rc,
                                           const LevelMD& P, const int c[3],
                                           int d, int v) {
  uint32_t i = 0;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int ue = e == d ? (v >> 1) : c[e];
    i += (uint32_t)ue * P.gc.gst[e];
  }
  return __ldg(Rc + i);
}

// 1D prediction along direction d of the sub-pass-1 point u from the
// coarse grid (the point's other interpolation coordinates are even; c is
// its coarse cell)
template <int KIND>
__device__ __forceinline__ float predict_coarse(const float* __restrict__ Rc,
                                                const LevelMD& P, const int c[3],
                                                int d, int u, int m) {
  const int f = choose_formula(KIND, false, u, m);
  float m3 = 0.f, p1 = 0.f, p3 = 0.f;
  const float m1 = coarse_at(Rc, P, c, d, u - 1);
  switch (f) {
    case F_COPY:
      break;
    case F_EXTRAP:
      m3 = coarse_at(Rc, P, c, d, u - 3);
      break;
    case F_LIN:
      p1 = coarse_at(Rc, P, c, d, u + 1);
      break;
    case F_NAK4:
    case F_NAT4:
      m3 = coarse_at(Rc, P, c, d, u - 3);
      p1 = coarse_at(Rc, P, c, d, u + 1);
      p3 = coarse_at(Rc, P, c, d, u + 3);
      break;
    case F_NAK3L:
    case F_NAT3L:
      m3 = coarse_at(Rc, P, c, d, u - 3);
      p1 = coarse_at(Rc, P, c, d, u + 1);
      break;
    case F_NAK3R:
    case F_NAT3R:
      p1 = coarse_at(Rc, P, c, d, u + 1);
      p3 = coarse_at(Rc, P, c, d, u + 3);
      break;
  }
  return eval_formula(f, m3, 0.f, m1, p1, 0.f, p3);
}

template <bool kDecomp, int KIND, int SUB>
__global__ void __launch_bounds__(256)
    k_level_md(LevelMD P, const float* __restrict__ X,
               const uint16_t* __restrict__ codes_full,
               const float* __restrict__ outl_full, const float* __restrict__ Rc,
               const uint16_t* __restrict__ Cc, float* __restrict__ Rs,
               uint16_t* __restrict__ Cs, const Ctl* __restrict__ ctl) {
  if (ctl->status || ctl->is_const) return;
  const int li = P.level - 1;
  const float el = ctl->el[li], inv2 = ctl->inv2[li], twoe = ctl->twoe[li];
  const LevelGeom& g = P.g;
  const unsigned long long ncell =
      (unsigned long long)P.nc[0] * P.nc[1] * P.nc[2];
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x +
                              threadIdx.x;
       t < ncell; t += (unsigned long long)gridDim.x * blockDim.x) {
    int c[3];
    c[2] = (int)(t % P.nc[2]);
    const unsigned long long r = t / P.nc[2];
    c[1] = (int)(r % P.nc[1]);
    c[0] = (int)(r / P.nc[1]);
    if (SUB == 1) {
      // the coarse point at the cell's even corner: its code, and its
      // reconstruction where the level grid is read later
      uint32_t ci = 0, fi = 0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        ci += (uint32_t)c[d] * P.gc.gst[d];
        fi += (uint32_t)(P.interp[d] ? 2 * c[d] : c[d]) * g.gst[d];
      }
      if (kDecomp || P.write_recon) Rs[fi] = Rc[ci];
      if (!kDecomp) Cs[fi] = Cc[ci];
    }
    for (int q = 0; q < P.nmask[SUB - 1]; ++q) {
      const unsigned S = P.masks[SUB - 1][q];
      int u[3];
      bool inside = true;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        u[d] = P.interp[d] ? 2 * c[d] + (int)((S >> d) & 1u) : c[d];
        inside = inside && u[d] < (int)g.m[d];
      }
      if (!inside) continue;
      const uint32_t gi = (uint32_t)u[0] * g.gst[0] + (uint32_t)u[1] * g.gst[1] +
                          (uint32_t)u[2];
      float p = 0.0f;
      bool first = true;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (!(S & (1u << d))) continue;
        float pd;
        if (SUB == 1)
          pd = predict_coarse<KIND>(Rc, P, c, d, u[d], (int)g.m[d]);
        else
          pd = predict_line_k<KIND>(Rs + gi, (long long)g.gst[d], u[d], (int)g.m[d]);
        const float tw = __fmul_rn(P.w[S][d], pd);
        p = first ? tw : __fadd_rn(p, tw);
        first = false;
      }
      const uint32_t fi = (uint32_t)u[0] * g.step[0] * P.fst[0] +
                          (uint32_t)u[1] * g.step[1] * P.fst[1] +
                          (uint32_t)u[2] * g.step[2];
      if (!kDecomp) {
        float rec;
        const unsigned code = quantize(X[fi], p, el, inv2, twoe, rec);
        Cs[gi] = (uint16_t)code;
        if (P.write_recon || SUB < P.k) Rs[gi] = rec;
      } else {
        const unsigned code = codes_full[fi];
        Rs[gi] = code ? dequantize(code, p, twoe) : outl_full[fi];
      }
    }
  }
}

template <bool kDecomp, int KIND>
void launch_md_k(const LevelMD& P, const SweepBufs& B, const float* Rc,
                 const uint16_t* Cc, float* Rs, uint16_t* Cs, int num_sms,
                 cudaStream_t s) {
  const unsigned long long ncell = (unsigned long long)P.nc[0] * P.nc[1] * P.nc[2];
  unsigned long long grid = (ncell + 255) / 256;
  const unsigned long long cap = (unsigned long long)num_sms * 16;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  k_level_md<kDecomp, KIND, 1><<<(unsigned)grid, 256, 0, s>>>(
      P, B.x, B.codes_full, B.outl_full, Rc, Cc, Rs, Cs, B.ctl);
  if (P.k >= 2)
    k_level_md<kDecomp, KIND, 2><<<(unsigned)grid, 256, 0, s>>>(
        P, B.x, B.codes_full, B.outl_full, Rc, Cc, Rs, Cs, B.ctl);
  if (P.k >= 3)
    k_level_md<kDecomp, KIND, 3><<<(unsigned)grid, 256, 0, s>>>(
        P, B.x, B.codes_full, B.outl_full, Rc, Cc, Rs, Cs, B.ctl);
}

}  // namespace

// One level of the multi-dimensional paradigm: P.k launches.
void launch_level_md(bool decomp, int kind, const LevelMD& P, const SweepBufs& B,
                     const float* Rc, const uint16_t* Cc, float* Rs, uint16_t* Cs,
                     int num_sms, cudaStream_t s) {
  if (decomp) {
    if (kind == LINEAR) launch_md_k<true, LINEAR>(P, B, Rc, Cc, Rs, Cs, num_sms, s);
    else if (kind == CUBIC_NAK) launch_md_k<true, CUBIC_NAK>(P, B, Rc, Cc, Rs, Cs, num_sms, s);
    else launch_md_k<true, CUBIC_NAT>(P, B, Rc, Cc, Rs, Cs, num_sms, s);
  } else {
    if (kind == LINEAR) launch_md_k<false, LINEAR>(P, B, Rc, Cc, Rs, Cs, num_sms, s);
    else if (kind == CUBIC_NAK) launch_md_k<false, CUBIC_NAK>(P, B, Rc, Cc, Rs, Cs, num_sms, s);
    else launch_md_k<false, CUBIC_NAT>(P, B, Rc, Cc, Rs, Cs, num_sms, s);
  }
}

}  // namespace hpez
