// k_level.cu -- one launch per level for the 1D-style paradigm.
//
// Within a level (stride s, Sec. 5.1) the 1D-style passes run one direction
// after the other (Sec. 5.3): pass j predicts along pi_j the points that
// are odd on pi_j, of any parity on the earlier directions and even on the
// later ones, from neighbours at +-s, +-3s (and +-2s for the second
// same-level half, Sec. 5.4.2).  A CTA owns a tile of the level's compact
// grid and recomputes, in shared memory, the few points of earlier passes
// that its later passes need from just outside the tile (a halo of 3 along
// the later directions, 5 with same-level halves).  Every value it writes
// is the same one the neighbouring tile computes, because both run the same
// IEEE operations on the same inputs.  The level's coarse points come from
// the compact coarse grid; the tile's codes and reconstruction are written
// out once, coalesced along the fastest dimension.
#include "hpez_internal.cuh"
#include "hpez_launch.h"

namespace hpez {

// Exact bound test with a fast accept: rn(r - x) strictly inside the bound
// implies the exact difference is inside too (rounding is monotonic), so
// the TwoSum residual is only needed near the bound.
__device__ __forceinline__ unsigned quantize_fast(float x, float p, float el,
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

// Prediction at a point from neighbours along one slot: smem[idx + j*st]
// when the neighbour lies in the CTA's region, else (first pass only) the
// compact coarse grid.
struct Line {
  const float* sm;
  int idx, st;     // region index of the point, region stride along the slot
  int u, lo, hi;   // grid coordinate along the slot, region bounds
  bool in_smem;    // every existing neighbour is in the region
  const float* Rc;
  uint32_t cbase, cst;
  __device__ __forceinline__ float at(int j) const {
    if (in_smem) return sm[idx + j * st];
    const int v = u + j;
    if (v >= lo && v < hi) return sm[idx + j * st];
    return __ldg(Rc + cbase + (uint32_t)(v >> 1) * cst);
  }
};

__device__ __forceinline__ float predict_at(const Line& L, int m, int kind,
                                            bool half_b) {
  const int u = L.u;
  // interior fast path: all four inter-level knots present
  if (!half_b && u >= 3 && u + 3 <= m - 1) {
    const float m1 = L.at(-1), p1 = L.at(1);
    if (kind == LINEAR) return eval_formula(F_LIN, 0.f, 0.f, m1, p1, 0.f, 0.f);
    const float m3 = L.at(-3), p3 = L.at(3);
    return eval_formula(kind == CUBIC_NAK ? F_NAK4 : F_NAT4, m3, 0.f, m1, p1,
                        0.f, p3);
  }
  const int f = choose_formula(kind, half_b, u, m);
  float m3 = 0.f, m2 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
  const float m1 = L.at(-1);
  switch (f) {
    case F_COPY:
      break;
    case F_EXTRAP:
      m3 = L.at(-3);
      break;
    case F_LIN:
      p1 = L.at(1);
      break;
    case F_NAK4:
    case F_NAT4:
      m3 = L.at(-3);
      p1 = L.at(1);
      p3 = L.at(3);
      break;
    case F_NAK3L:
    case F_NAT3L:
      m3 = L.at(-3);
      p1 = L.at(1);
      break;
    case F_NAK3R:
    case F_NAT3R:
      p1 = L.at(1);
      p3 = L.at(3);
      break;
    case F_SL_NAK:
      m2 = L.at(-2);
      p1 = L.at(1);
      p2 = L.at(2);
      break;
    case F_SL_NAT:
      m3 = L.at(-3);
      m2 = L.at(-2);
      p1 = L.at(1);
      p2 = L.at(2);
      p3 = L.at(3);
      break;
  }
  return eval_formula(f, m3, m2, m1, p1, p2, p3);
}

// Rows of a box are (slot 0, slot 1) index pairs handed to warps; lanes
// walk the fastest slot.  One division per row, none per point.
template <bool kDecomp>
__global__ void __launch_bounds__(256)
    k_level(FusedLevel P, SweepBufs B, const float* __restrict__ Rc,
            const uint16_t* __restrict__ Cc, float* __restrict__ Rs,
            uint16_t* __restrict__ Cs) {
  const Ctl* ctl = B.ctl;
  if (ctl->status || ctl->is_const) return;
  extern __shared__ float sm[];
  const LevelGeom& g = P.g;
  const LevelGeom& gc = P.gc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  uint32_t tb = blockIdx.x;
  int o[3];
  {
    const uint32_t t2 = tb % P.ntile[2];
    tb /= P.ntile[2];
    const uint32_t t1 = tb % P.ntile[1];
    const uint32_t t0 = tb / P.ntile[1];
    o[0] = (int)(t0 * P.E[0]);
    o[1] = (int)(t1 * P.E[1]);
    o[2] = (int)(t2 * P.E[2]);
  }
  int base[3], lo[3], hi[3], te[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    base[d] = o[d] + P.rlo[d];
    lo[d] = max(base[d], 0);
    hi[d] = min(o[d] + P.rhi[d], (int)g.m[d]);
    te[d] = min(o[d] + (int)P.E[d], (int)g.m[d]);
  }
  const int RX1 = (int)P.RX[1], RX2 = (int)P.RX[2];
  const int sst[3] = {RX1 * RX2, RX2, 1};
  uint16_t* ctile = reinterpret_cast<uint16_t*>(sm + P.RX[0] * P.RX[1] * P.RX[2]);
  const int E1 = (int)P.E[1], E2 = (int)P.E[2];
  const int li = P.level - 1;
  const float el = ctl->el[li], inv2 = ctl->inv2[li], twoe = ctl->twoe[li];
  const uint32_t fst0 = g.step[0] * g.fst[0], fst1 = g.step[1] * g.fst[1],
                 fst2 = g.step[2];

  // 1. coarse points of the region
  {
    int st0[3], cn[3], stp[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      stp[d] = P.interp[d] ? 2 : 1;
      st0[d] = P.interp[d] ? ((lo[d] + 1) & ~1) : lo[d];
      cn[d] = hi[d] > st0[d] ? (hi[d] - st0[d] + stp[d] - 1) / stp[d] : 0;
    }
    const int rows = cn[0] * cn[1];
    for (int r = warp; r < rows; r += nwarps) {
      const int a0 = r / cn[1], a1 = r - a0 * cn[1];
      const int u0 = st0[0] + a0 * stp[0], u1 = st0[1] + a1 * stp[1];
      const uint32_t crow = (uint32_t)(u0 / stp[0]) * gc.gst[0] +
                            (uint32_t)(u1 / stp[1]) * gc.gst[1] +
                            (uint32_t)(st0[2] / stp[2]);
      float* srow = sm + (u0 - base[0]) * sst[0] + (u1 - base[1]) * RX2 +
                    (st0[2] - base[2]);
      for (int a2 = lane; a2 < cn[2]; a2 += 32)
        srow[a2 * stp[2]] = __ldg(Rc + crow + a2);
    }
  }
  __syncthreads();

  // 2. the passes, each half a step
  for (int si = 0; si < P.nsteps; ++si) {
    const FusedStep& S = P.st[si];
    int st0[3], cn[3], stp[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int a = max(o[d] + S.lo[d], lo[d]);
      const int b = min(o[d] + S.hi[d], hi[d]);
      if (S.par[d] == 0) {
        st0[d] = a;
        stp[d] = 1;
      } else {
        const int want = S.par[d] == 1 ? 1 : 0;
        st0[d] = a + ((a & 1) != want ? 1 : 0);
        stp[d] = 2;
      }
      cn[d] = b > st0[d] ? (b - st0[d] + stp[d] - 1) / stp[d] : 0;
    }
    const int d = S.dim;
    const bool in_smem = S.pad_[0] != 0;
    const int md = (int)g.m[d];
    const int rows = cn[0] * cn[1];
    for (int r = warp; r < rows; r += nwarps) {
      const int a0 = r / cn[1], a1 = r - a0 * cn[1];
      const int u0 = st0[0] + a0 * stp[0], u1 = st0[1] + a1 * stp[1];
      const int rsm = (u0 - base[0]) * sst[0] + (u1 - base[1]) * RX2 - base[2];
      const uint32_t rfull = (uint32_t)u0 * fst0 + (uint32_t)u1 * fst1;
      const bool row_in_tile = u0 >= o[0] && u0 < te[0] && u1 >= o[1] && u1 < te[1];
      const int rtile = ((u0 - o[0]) * E1 + (u1 - o[1])) * E2 - o[2];
      uint32_t brow = 0;
      if (B.blockmap)
        brow = (((uint32_t)u0 * g.step[0]) / B.bs * B.nb[1] +
                ((uint32_t)u1 * g.step[1]) / B.bs) * B.nb[2];
      // coarse index of the row with slot d left out (first pass only)
      uint32_t cb_row = 0;
      if (!in_smem) {
        if (d != 0) cb_row += (uint32_t)(P.interp[0] ? (u0 >> 1) : u0) * gc.gst[0];
        if (d != 1) cb_row += (uint32_t)(P.interp[1] ? (u1 >> 1) : u1) * gc.gst[1];
      }
      for (int a2 = lane; a2 < cn[2]; a2 += 32) {
        const int u2 = st0[2] + a2 * stp[2];
        int kind = B.kind, same = B.same;
        if (B.blockmap) {
          const unsigned v = B.blockmap[brow + ((uint32_t)u2 * g.step[2]) / B.bs];
          kind = (int)(v & 3u);
          if (kind > CUBIC_NAT) kind = CUBIC_NAT;
          same = (int)((v >> 2) & 1u);
        }
        if (kind == LINEAR) same = 0;
        const int ud = d == 0 ? u0 : (d == 1 ? u1 : u2);
        const int in_b = same && (((ud - 1) >> 1) & 1);
        if (in_b != S.half) continue;
        const int idx = rsm + u2;
        Line L;
        L.sm = sm;
        L.idx = idx;
        L.st = sst[d];
        L.u = ud;
        L.lo = lo[d];
        L.hi = hi[d];
        L.in_smem = in_smem;
        L.Rc = Rc;
        L.cbase = cb_row + (d != 2 ? (uint32_t)(P.interp[2] ? (u2 >> 1) : u2) : 0u);
        L.cst = gc.gst[d];
        const float p = predict_at(L, md, kind, in_b);
        const uint32_t fi = rfull + (uint32_t)u2 * fst2;
        float rec;
        if (!kDecomp) {
          const unsigned code = quantize_fast(__ldg(B.x + fi), p, el, inv2, twoe, rec);
          if (row_in_tile && u2 >= o[2] && u2 < te[2]) ctile[rtile + u2] = (uint16_t)code;
        } else {
          const unsigned code = B.codes_full[fi];
          rec = code ? dequantize(code, p, twoe) : B.outl_full[fi];
        }
        sm[idx] = rec;
      }
    }
    __syncthreads();
  }

  // 3. write the tile out, rows to warps, consecutive elements to lanes
  {
    const int n0 = te[0] - o[0], n1 = te[1] - o[1], n2 = te[2] - o[2];
    const int rows = n0 * n1;
    for (int r = warp; r < rows; r += nwarps) {
      const int a0 = r / n1, a1 = r - a0 * n1;
      const int u0 = o[0] + a0, u1 = o[1] + a1;
      const uint32_t grow = (uint32_t)u0 * g.gst[0] + (uint32_t)u1 * g.gst[1] + (uint32_t)o[2];
      const float* srow = sm + (u0 - base[0]) * sst[0] + (u1 - base[1]) * RX2 + (o[2] - base[2]);
      if (!kDecomp) {
        const bool crow = (!P.interp[0] || !(u0 & 1)) && (!P.interp[1] || !(u1 & 1));
        const uint32_t ccrow = (uint32_t)(P.interp[0] ? u0 >> 1 : u0) * gc.gst[0] +
                               (uint32_t)(P.interp[1] ? u1 >> 1 : u1) * gc.gst[1];
        const uint16_t* trow = ctile + (a0 * E1 + a1) * E2;
        for (int a2 = lane; a2 < n2; a2 += 32) {
          const int u2 = o[2] + a2;
          uint16_t code;
          if (crow && (!P.interp[2] || !(u2 & 1)))
            code = Cc[ccrow + (uint32_t)(P.interp[2] ? u2 >> 1 : u2)];
          else
            code = trow[a2];
          Cs[grow + a2] = code;
          if (P.write_recon) Rs[grow + a2] = srow[a2];
        }
      } else {
        for (int a2 = lane; a2 < n2; a2 += 32) Rs[grow + a2] = srow[a2];
      }
    }
  }
}

size_t fused_smem_bytes(const FusedLevel& P, bool decomp) {
  size_t b = (size_t)P.RX[0] * P.RX[1] * P.RX[2] * sizeof(float);
  if (!decomp) b += (size_t)P.E[0] * P.E[1] * P.E[2] * sizeof(uint16_t);
  return b;
}

void launch_level(bool decomp, const FusedLevel& P, const SweepBufs& B,
                  const float* Rc, const uint16_t* Cc, float* Rs, uint16_t* Cs,
                  cudaStream_t s) {
  const size_t smem = fused_smem_bytes(P, decomp);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_level<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(k_level<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr = true;
  }
  if (decomp)
    k_level<true><<<P.ntiles, 256, smem, s>>>(P, B, Rc, Cc, Rs, Cs);
  else
    k_level<false><<<P.ntiles, 256, smem, s>>>(P, B, Rc, Cc, Rs, Cs);
}

}  // namespace hpez
