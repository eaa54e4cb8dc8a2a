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

// fetch of a neighbour along slot d at offset j: from shared memory when
// it lies inside the CTA's region, else from the compact coarse grid (only
// happens for the first pass, whose neighbours are all coarse points)
struct NeighbourCtx {
  const float* sm;        // region values
  const float* Rc;        // compact coarse grid
  int idx;                // the point's region index
  int st;                 // region stride along d
  int u;                  // the point's grid coordinate along d
  int lo, hi;             // region bounds along d (grid coordinates)
  uint32_t cbase;         // coarse index of the point with u_d removed
  uint32_t cst;           // coarse stride along d
  __device__ float at(int j) const {
    const int v = u + j;
    if (v >= lo && v < hi) return sm[idx + j * st];
    return __ldg(Rc + cbase + (uint32_t)(v >> 1) * cst);
  }
};

__device__ __forceinline__ float predict_fused(const NeighbourCtx& n, int m,
                                               int kind, bool half_b) {
  const int f = choose_formula(kind, half_b, n.u, m);
  float m3 = 0.f, m2 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
  const float m1 = n.at(-1);
  switch (f) {
    case F_COPY:
      break;
    case F_EXTRAP:
      m3 = n.at(-3);
      break;
    case F_LIN:
      p1 = n.at(1);
      break;
    case F_NAK4:
    case F_NAT4:
      m3 = n.at(-3);
      p1 = n.at(1);
      p3 = n.at(3);
      break;
    case F_NAK3L:
    case F_NAT3L:
      m3 = n.at(-3);
      p1 = n.at(1);
      break;
    case F_NAK3R:
    case F_NAT3R:
      p1 = n.at(1);
      p3 = n.at(3);
      break;
    case F_SL_NAK:
      m2 = n.at(-2);
      p1 = n.at(1);
      p2 = n.at(2);
      break;
    case F_SL_NAT:
      m3 = n.at(-3);
      m2 = n.at(-2);
      p1 = n.at(1);
      p2 = n.at(2);
      p3 = n.at(3);
      break;
  }
  return eval_formula(f, m3, m2, m1, p1, p2, p3);
}

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
  // tile origin and region bounds (grid coordinates)
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
    te[d] = min(o[d] + (int)P.E[d], (int)g.m[d]);  // tile end
  }
  const int RX1 = (int)P.RX[1], RX2 = (int)P.RX[2];
  const int sst[3] = {RX1 * RX2, RX2, 1};
  uint16_t* ctile = reinterpret_cast<uint16_t*>(sm + P.RX[0] * P.RX[1] * P.RX[2]);
  const int E1 = (int)P.E[1], E2 = (int)P.E[2];
  const int li = P.level - 1;
  const float el = ctl->el[li], inv2 = ctl->inv2[li], twoe = ctl->twoe[li];

  // 1. coarse points of the region (every interpolation coordinate even)
  {
    int st0[3], cn[3], stp[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      stp[d] = P.interp[d] ? 2 : 1;
      st0[d] = P.interp[d] ? ((lo[d] + 1) & ~1) : lo[d];
      cn[d] = hi[d] > st0[d] ? (hi[d] - st0[d] + stp[d] - 1) / stp[d] : 0;
    }
    const uint32_t tot = (uint32_t)(cn[0] * cn[1] * cn[2]);
    for (uint32_t t = threadIdx.x; t < tot; t += blockDim.x) {
      const int a2 = (int)(t % (uint32_t)cn[2]);
      const uint32_t r = t / (uint32_t)cn[2];
      const int a1 = (int)(r % (uint32_t)cn[1]);
      const int a0 = (int)(r / (uint32_t)cn[1]);
      const int u0 = st0[0] + a0 * stp[0], u1 = st0[1] + a1 * stp[1],
                u2 = st0[2] + a2 * stp[2];
      const uint32_t ci = (uint32_t)(u0 / stp[0]) * gc.gst[0] +
                          (uint32_t)(u1 / stp[1]) * gc.gst[1] +
                          (uint32_t)(u2 / stp[2]);
      sm[(u0 - base[0]) * sst[0] + (u1 - base[1]) * RX2 + (u2 - base[2])] =
          __ldg(Rc + ci);
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
    const uint32_t tot = (uint32_t)(cn[0] * cn[1] * cn[2]);
    for (uint32_t t = threadIdx.x; t < tot; t += blockDim.x) {
      const int a2 = (int)(t % (uint32_t)cn[2]);
      const uint32_t r = t / (uint32_t)cn[2];
      const int a1 = (int)(r % (uint32_t)cn[1]);
      const int a0 = (int)(r / (uint32_t)cn[1]);
      const int u[3] = {st0[0] + a0 * stp[0], st0[1] + a1 * stp[1],
                        st0[2] + a2 * stp[2]};
      int kind = B.kind, same = B.same;
      if (B.blockmap) {
        uint32_t bi = 0;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          bi = bi * B.nb[q] + ((uint32_t)u[q] * g.step[q]) / B.bs;
        const unsigned v = B.blockmap[bi];
        kind = (int)(v & 3u);
        if (kind > CUBIC_NAT) kind = CUBIC_NAT;
        same = (int)((v >> 2) & 1u);
      }
      if (kind == LINEAR) same = 0;
      const int in_b = same && (((u[d] - 1) >> 1) & 1);
      if (in_b != S.half) continue;
      const int idx = (u[0] - base[0]) * sst[0] + (u[1] - base[1]) * RX2 +
                      (u[2] - base[2]);
      NeighbourCtx nc;
      nc.sm = sm;
      nc.Rc = Rc;
      nc.idx = idx;
      nc.st = sst[d];
      nc.u = u[d];
      nc.lo = lo[d];
      nc.hi = hi[d];
      {
        // coarse index with slot d left out (only used by the first pass)
        uint32_t cb = 0;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (q != d) cb += (uint32_t)(P.interp[q] ? (u[q] >> 1) : u[q]) * gc.gst[q];
        nc.cbase = cb;
        nc.cst = gc.gst[d];
      }
      const float p = predict_fused(nc, (int)g.m[d], kind, in_b);
      const uint32_t fi = (uint32_t)u[0] * g.step[0] * g.fst[0] +
                          (uint32_t)u[1] * g.step[1] * g.fst[1] +
                          (uint32_t)u[2] * g.step[2];
      float rec;
      if (!kDecomp) {
        const unsigned code = quantize(__ldg(B.x + fi), p, el, inv2, twoe, rec);
        if (u[0] >= o[0] && u[0] < te[0] && u[1] >= o[1] && u[1] < te[1] &&
            u[2] >= o[2] && u[2] < te[2])
          ctile[((u[0] - o[0]) * E1 + (u[1] - o[1])) * E2 + (u[2] - o[2])] =
              (uint16_t)code;
      } else {
        const unsigned code = B.codes_full[fi];
        rec = code ? dequantize(code, p, twoe) : B.outl_full[fi];
      }
      sm[idx] = rec;
    }
    __syncthreads();
  }

  // 3. write the tile: codes (coarse ones copied from the coarse grid) and
  //    the reconstruction when the next level reads it
  {
    const int n0 = te[0] - o[0], n1 = te[1] - o[1], n2 = te[2] - o[2];
    const uint32_t tot = (uint32_t)(n0 * n1 * n2);
    for (uint32_t t = threadIdx.x; t < tot; t += blockDim.x) {
      const int a2 = (int)(t % (uint32_t)n2);
      const uint32_t r = t / (uint32_t)n2;
      const int a1 = (int)(r % (uint32_t)n1);
      const int a0 = (int)(r / (uint32_t)n1);
      const int u0 = o[0] + a0, u1 = o[1] + a1, u2 = o[2] + a2;
      const uint32_t gi = (uint32_t)u0 * g.gst[0] + (uint32_t)u1 * g.gst[1] + (uint32_t)u2;
      const int idx = (u0 - base[0]) * sst[0] + (u1 - base[1]) * RX2 + (u2 - base[2]);
      if (!kDecomp) {
        const bool coarse = (!P.interp[0] || !(u0 & 1)) && (!P.interp[1] || !(u1 & 1)) &&
                            (!P.interp[2] || !(u2 & 1));
        uint16_t code;
        if (coarse) {
          const uint32_t ci = (uint32_t)(P.interp[0] ? u0 >> 1 : u0) * gc.gst[0] +
                              (uint32_t)(P.interp[1] ? u1 >> 1 : u1) * gc.gst[1] +
                              (uint32_t)(P.interp[2] ? u2 >> 1 : u2);
          code = Cc[ci];
        } else {
          code = ctile[(a0 * E1 + a1) * E2 + a2];
        }
        Cs[gi] = code;
        if (P.write_recon) Rs[gi] = sm[idx];
      } else {
        Rs[gi] = sm[idx];
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
