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

// ---------------------------------------------------------------------
// Shared-memory layout of the CTA's region: rows (slot 0, slot 1) of RX2
// columns in grid order.  Before the passes the region holds the input
// values (staged with asynchronous copies); the coarse points are then
// overwritten with their reconstruction, and each pass replaces a point's
// input value by its reconstruction, which later passes read.
// ---------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
}
struct Region {
  int o[3], base[3], lo[3], hi[3], te[3];
  int RX1, RX2, HX;        // row length, half-row length
  int rst0, rst1;          // element stride of a step along slot 0 / 1
  __device__ __forceinline__ int col(int u2) const { return u2 - base[2]; }
  __device__ __forceinline__ int row(int u0, int u1) const {
    return (u0 - base[0]) * rst0 + (u1 - base[1]) * rst1;
  }
};

template <int KIND>
__device__ __forceinline__ float interior_k(float m3, float m1, float p1,
                                            float p3) {
  if (KIND == LINEAR) return eval_formula(F_LIN, 0.f, 0.f, m1, p1, 0.f, 0.f);
  if (KIND == CUBIC_NAK) return eval_formula(F_NAK4, m3, 0.f, m1, p1, 0.f, p3);
  return eval_formula(F_NAT4, m3, 0.f, m1, p1, 0.f, p3);
}

// Neighbour access along slot D of the point (u0, u1, u2): shared memory
// inside the region, the compact coarse grid outside (first pass only).
template <int D>
struct Nbr {
  const float* sm;
  const Region* R;
  int r, u0, u1, u2;   // row offset and coordinates of the point
  bool in_smem;
  const float* Rc;
  uint32_t cbase, cst;
  __device__ __forceinline__ float at(int j) const {
    const int u = D == 0 ? u0 : (D == 1 ? u1 : u2);
    const int v = u + j;
    if (!in_smem && (v < R->lo[D] || v >= R->hi[D]))
      return __ldg(Rc + cbase + (uint32_t)(v >> 1) * cst);
    if (D == 2) return sm[r + R->col(v)];
    if (D == 1) return sm[r + j * R->rst1 + R->col(u2)];
    return sm[r + j * R->rst0 + R->col(u2)];
  }
};

template <int KIND, int D>
__device__ __forceinline__ float predict_nbr(const Nbr<D>& n, int u, int m,
                                             int kind, bool half_b) {
  if (!half_b && u >= 3 && u + 3 <= m - 1) {
    const float m1 = n.at(-1), p1 = n.at(1);
    if (KIND != 3) {
      if (KIND == LINEAR) return interior_k<LINEAR>(0.f, m1, p1, 0.f);
      return interior_k<KIND>(n.at(-3), m1, p1, n.at(3));
    }
    if (kind == LINEAR) return interior_k<LINEAR>(0.f, m1, p1, 0.f);
    const float m3 = n.at(-3), p3 = n.at(3);
    return kind == CUBIC_NAK ? interior_k<CUBIC_NAK>(m3, m1, p1, p3)
                             : interior_k<CUBIC_NAT>(m3, m1, p1, p3);
  }
  const int f = choose_formula(kind, half_b, u, m);
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

struct LevelConsts {
  float el, inv2, twoe;
  uint32_t fst0, fst1, fst2;
};

// One pass half over its box: rows to warps, the fastest slot to lanes.
// Interior points of a fixed interpolator whose neighbours are all in
// shared memory take a straight-line path with precomputed indices; all
// other points (boundaries, same-level halves, block map, first pass)
// take the general one.  Codes (and reconstructions the next level reads)
// of points inside the tile go straight to global memory.
template <bool kDecomp, int KIND, int D>
__device__ __forceinline__ void run_step(const FusedLevel& P, const SweepBufs& B,
                                         const FusedStep& S, const Region& R,
                                         const LevelConsts& K, float* sm,
                                         const uint16_t* scodes,
                                         const float* __restrict__ Rc,
                                         float* __restrict__ Rs,
                                         uint16_t* __restrict__ Cs) {
  const LevelGeom& g = P.g;
  const LevelGeom& gc = P.gc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  int st0[3], cn[3], stp[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int a = max(R.o[d] + S.lo[d], R.lo[d]);
    const int b = min(R.o[d] + S.hi[d], R.hi[d]);
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
  const bool in_smem = S.pad_[0] != 0;
  const bool fast_ok = in_smem && KIND != 3;
  const int md = (int)g.m[D];
  const int rows = cn[0] * cn[1];
  const int nst = D == 2 ? 0 : (D == 1 ? R.rst1 : R.rst0);  // neighbour stride
  for (int rr = warp; rr < rows; rr += nwarps) {
    const int a0 = rr / cn[1], a1 = rr - a0 * cn[1];
    const int u0 = st0[0] + a0 * stp[0], u1 = st0[1] + a1 * stp[1];
    const int rsm = R.row(u0, u1);
    const uint32_t rfull = (uint32_t)u0 * K.fst0 + (uint32_t)u1 * K.fst1;
    const uint32_t rgrid = (uint32_t)u0 * g.gst[0] + (uint32_t)u1 * g.gst[1];
    const bool row_in_tile =
        u0 >= R.o[0] && u0 < R.te[0] && u1 >= R.o[1] && u1 < R.te[1];
    // along slot 0/1 the stencil depends on the row only
    const int urow = D == 0 ? u0 : u1;
    const bool row_interior = D == 2 || (urow >= 3 && urow + 3 <= md - 1);
    uint32_t brow = 0;
    if (KIND == 3 && B.blockmap)
      brow = (((uint32_t)u0 * g.step[0]) / B.bs * B.nb[1] +
              ((uint32_t)u1 * g.step[1]) / B.bs) * B.nb[2];
    uint32_t cb_row = 0;
    if (!in_smem) {
      if (D != 0) cb_row += (uint32_t)(P.interp[0] ? (u0 >> 1) : u0) * gc.gst[0];
      if (D != 1) cb_row += (uint32_t)(P.interp[1] ? (u1 >> 1) : u1) * gc.gst[1];
    }
    // batches of kBatch points per lane: all their global loads (input
    // value or code) are issued before any of them is computed, so each
    // lane keeps several memory requests in flight
    constexpr int kBatch = 4;
    for (int a2b = lane; a2b < cn[2]; a2b += 32 * kBatch) {
      float xin[kBatch];
      unsigned cin[kBatch];
#pragma unroll
      for (int k = 0; k < kBatch; ++k) {
        const int a2 = a2b + 32 * k;
        xin[k] = 0.f;
        cin[k] = 0u;
        if (a2 < cn[2]) {
          const int u2 = st0[2] + a2 * stp[2];
          if (!kDecomp) {
            xin[k] = P.stage_x ? sm[rsm + (u2 - R.base[2])]
                               : __ldg(B.x + rfull + (uint32_t)u2 * K.fst2);
          } else {
            cin[k] = P.stage_x ? scodes[rsm + (u2 - R.base[2])]
                               : B.codes_full[rfull + (uint32_t)u2 * K.fst2];
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kBatch; ++k) {
        const int a2 = a2b + 32 * k;
        if (a2 >= cn[2]) break;
        const int u2 = st0[2] + a2 * stp[2];
        const int sidx = rsm + (u2 - R.base[2]);
        float p;
        const bool interior =
            fast_ok && !B.same && row_interior && (D != 2 || (u2 >= 3 && u2 + 3 <= md - 1));
        if (interior) {
          float m3, m1, p1, p3;
          if (D == 2) {
            m3 = sm[sidx - 3];
            m1 = sm[sidx - 1];
            p1 = sm[sidx + 1];
            p3 = sm[sidx + 3];
          } else {
            m3 = sm[sidx - 3 * nst];
            m1 = sm[sidx - nst];
            p1 = sm[sidx + nst];
            p3 = sm[sidx + 3 * nst];
          }
          p = interior_k<KIND>(m3, m1, p1, p3);
        } else {
          int kind = KIND == 3 ? B.kind : KIND, same = B.same;
          if (KIND == 3 && B.blockmap) {
            const unsigned v = B.blockmap[brow + ((uint32_t)u2 * g.step[2]) / B.bs];
            kind = (int)(v & 3u);
            if (kind > CUBIC_NAT) kind = CUBIC_NAT;
            same = (int)((v >> 2) & 1u);
          }
          if (kind == LINEAR) same = 0;
          const int ud = D == 0 ? u0 : (D == 1 ? u1 : u2);
          const int in_b = same && (((ud - 1) >> 1) & 1);
          if (in_b != S.half) continue;
          Nbr<D> n;
          n.sm = sm;
          n.R = &R;
          n.r = rsm;
          n.u0 = u0;
          n.u1 = u1;
          n.u2 = u2;
          n.in_smem = in_smem;
          n.Rc = Rc;
          n.cbase = cb_row + (D != 2 ? (uint32_t)(P.interp[2] ? (u2 >> 1) : u2) : 0u);
          n.cst = gc.gst[D];
          p = predict_nbr<KIND, D>(n, ud, md, kind, in_b);
        }
        const bool in_tile = row_in_tile && u2 >= R.o[2] && u2 < R.te[2];
        float rec;
        if (!kDecomp) {
          const unsigned code = quantize_fast(xin[k], p, K.el, K.inv2, K.twoe, rec);
          if (in_tile) {
            Cs[rgrid + (uint32_t)u2] = (uint16_t)code;
            if (P.write_recon) Rs[rgrid + (uint32_t)u2] = rec;
          }
        } else {
          const unsigned code = cin[k];
          rec = code ? dequantize(code, p, K.twoe)
                     : B.outl_full[rfull + (uint32_t)u2 * K.fst2];
          if (in_tile) Rs[rgrid + (uint32_t)u2] = rec;
        }
        sm[sidx] = rec;
      }
    }
  }
}

template <bool kDecomp, int KIND>
__device__ __forceinline__ void level_body(const FusedLevel& P,
                                           const SweepBufs& B,
                                           const float* __restrict__ Rc,
                                           const uint16_t* __restrict__ Cc,
                                           float* __restrict__ Rs,
                                           uint16_t* __restrict__ Cs,
                                           unsigned bid) {
  const Ctl* ctl = B.ctl;
  if (ctl->status || ctl->is_const) return;
  extern __shared__ float sm[];
  const LevelGeom& g = P.g;
  const LevelGeom& gc = P.gc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  Region R;
  {
    uint32_t tb = bid;
    const uint32_t t2 = tb % P.ntile[2];
    tb /= P.ntile[2];
    const uint32_t t1 = tb % P.ntile[1];
    const uint32_t t0 = tb / P.ntile[1];
    R.o[0] = (int)(t0 * P.E[0]);
    R.o[1] = (int)(t1 * P.E[1]);
    R.o[2] = (int)(t2 * P.E[2]);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R.base[d] = R.o[d] + P.rlo[d];
    R.lo[d] = max(R.base[d], 0);
    R.hi[d] = min(R.o[d] + P.rhi[d], (int)g.m[d]);
    R.te[d] = min(R.o[d] + (int)P.E[d], (int)g.m[d]);
  }
  R.RX1 = (int)P.RX[1];
  R.RX2 = (int)P.RX[2];
  R.HX = R.RX2 >> 1;
  R.rst1 = R.RX2;
  R.rst0 = R.RX1 * R.RX2;
  const int li = P.level - 1;
  LevelConsts K;
  K.el = ctl->el[li];
  K.inv2 = ctl->inv2[li];
  K.twoe = ctl->twoe[li];
  K.fst0 = g.step[0] * g.fst[0];
  K.fst1 = g.step[1] * g.fst[1];
  K.fst2 = g.step[2];

  // 0. stage the region's input values (compress) or codes (decompress)
  uint16_t* scodes = reinterpret_cast<uint16_t*>(sm + P.RX[0] * P.RX[1] * P.RX[2]);
  if (P.stage_x) {
    const int ncol = R.hi[2] - R.lo[2];
    const int rows = (R.hi[0] - R.lo[0]) * (R.hi[1] - R.lo[1]);
    const int n1 = R.hi[1] - R.lo[1];
    for (int r = warp; r < rows; r += nwarps) {
      const int u0 = R.lo[0] + r / n1, u1 = R.lo[1] + r % n1;
      const int rsm = R.row(u0, u1) + (R.lo[2] - R.base[2]);
      const uint32_t rfull = (uint32_t)u0 * K.fst0 + (uint32_t)u1 * K.fst1 +
                             (uint32_t)R.lo[2] * K.fst2;
      if (!kDecomp) {
        if (P.stage_x == 2) {  // 16-byte copies, rows 16-byte aligned
          for (int c4 = lane * 4; c4 < ncol; c4 += 128)
            cp_async16(sm + rsm + c4, B.x + rfull + c4);
        } else {
          for (int c = lane; c < ncol; c += 32)
            cp_async4(sm + rsm + c, B.x + rfull + (uint32_t)c * K.fst2);
        }
      } else {
        for (int c8 = lane * 8; c8 < ncol; c8 += 256)
          cp_async16(scodes + rsm + c8, B.codes_full + rfull + c8);
      }
    }
    cp_async_wait_all();
    __syncthreads();
  }

  // 1. coarse points of the region (all interpolation coordinates even)
  {
    int st0[3], cn[3], stp[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      stp[d] = P.interp[d] ? 2 : 1;
      st0[d] = P.interp[d] ? ((R.lo[d] + 1) & ~1) : R.lo[d];
      cn[d] = R.hi[d] > st0[d] ? (R.hi[d] - st0[d] + stp[d] - 1) / stp[d] : 0;
    }
    const int rows = cn[0] * cn[1];
    for (int r = warp; r < rows; r += nwarps) {
      const int a0 = r / cn[1], a1 = r - a0 * cn[1];
      const int u0 = st0[0] + a0 * stp[0], u1 = st0[1] + a1 * stp[1];
      const uint32_t crow = (uint32_t)(u0 / stp[0]) * gc.gst[0] +
                            (uint32_t)(u1 / stp[1]) * gc.gst[1] +
                            (uint32_t)(st0[2] / stp[2]);
      const int rsm = R.row(u0, u1);
#pragma unroll 4
      for (int a2 = lane; a2 < cn[2]; a2 += 32)
        sm[rsm + R.col(st0[2] + a2 * stp[2])] = __ldg(Rc + crow + a2);
    }
  }
  __syncthreads();

  // 2. the passes, each half a step
  for (int si = 0; si < P.nsteps; ++si) {
    const FusedStep& S = P.st[si];
    if (S.dim == 2)
      run_step<kDecomp, KIND, 2>(P, B, S, R, K, sm, scodes, Rc, Rs, Cs);
    else if (S.dim == 1)
      run_step<kDecomp, KIND, 1>(P, B, S, R, K, sm, scodes, Rc, Rs, Cs);
    else
      run_step<kDecomp, KIND, 0>(P, B, S, R, K, sm, scodes, Rc, Rs, Cs);
    __syncthreads();
  }

  // 3. the tile's coarse points: codes copied from the coarse grid, and the
  //    reconstruction where this level's output is read again
  {
    int st0[3], cn[3], stp[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      stp[d] = P.interp[d] ? 2 : 1;
      st0[d] = P.interp[d] ? ((R.o[d] + 1) & ~1) : R.o[d];
      cn[d] = R.te[d] > st0[d] ? (R.te[d] - st0[d] + stp[d] - 1) / stp[d] : 0;
    }
    const int rows = cn[0] * cn[1];
    for (int r = warp; r < rows; r += nwarps) {
      const int a0 = r / cn[1], a1 = r - a0 * cn[1];
      const int u0 = st0[0] + a0 * stp[0], u1 = st0[1] + a1 * stp[1];
      const uint32_t grow = (uint32_t)u0 * g.gst[0] + (uint32_t)u1 * g.gst[1];
      const uint32_t crow = (uint32_t)(u0 / stp[0]) * gc.gst[0] +
                            (uint32_t)(u1 / stp[1]) * gc.gst[1] +
                            (uint32_t)(st0[2] / stp[2]);
      const int rsm = R.row(u0, u1);
#pragma unroll 4
      for (int a2 = lane; a2 < cn[2]; a2 += 32) {
        const int u2 = st0[2] + a2 * stp[2];
        if (!kDecomp) {
          Cs[grow + (uint32_t)u2] = Cc[crow + a2];
          if (P.write_recon) Rs[grow + (uint32_t)u2] = sm[rsm + R.col(u2)];
        } else {
          Rs[grow + (uint32_t)u2] = sm[rsm + R.col(u2)];
        }
      }
    }
  }
}

template <bool kDecomp, int KIND>
__global__ void __launch_bounds__(256)
    k_level(FusedLevel P, SweepBufs B, const float* __restrict__ Rc,
            const uint16_t* __restrict__ Cc, float* __restrict__ Rs,
            uint16_t* __restrict__ Cs) {
  level_body<kDecomp, KIND>(P, B, Rc, Cc, Rs, Cs, blockIdx.x);
}

// batched, persistent: job j owns tiles [off[j], off[j+1]) of the launch
template <bool kDecomp, int KIND>
__global__ void __launch_bounds__(256)
    k_level_batch(const LevelJob* __restrict__ J, const uint32_t* __restrict__ off,
                  int nj) {
  for_each_batch_block(off, nj, [&](int j, uint32_t t) {
    const LevelJob& q = J[j];
    level_body<kDecomp, KIND>(q.P, q.B, q.Rc, q.Cc, q.Rs, q.Cs, t);
  });
}

size_t fused_smem_bytes(const FusedLevel& P, bool decomp) {
  size_t b = (size_t)P.RX[0] * P.RX[1] * P.RX[2] * sizeof(float);
  if (decomp && P.stage_x) b += (size_t)P.RX[0] * P.RX[1] * P.RX[2] * sizeof(uint16_t);
  return b;
}

template <bool kDecomp, int KIND>
static void launch_kind(const FusedLevel& P, const SweepBufs& B, size_t smem,
                        const float* Rc, const uint16_t* Cc, float* Rs,
                        uint16_t* Cs, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_level<kDecomp, KIND>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_level<kDecomp, KIND><<<P.ntiles, 256, smem, s>>>(P, B, Rc, Cc, Rs, Cs);
}

template <bool kDecomp>
static void launch_dec(const FusedLevel& P, const SweepBufs& B, size_t smem,
                       const float* Rc, const uint16_t* Cc, float* Rs,
                       uint16_t* Cs, cudaStream_t s) {
  // a fixed interpolator compiles to straight-line code; a block map (or
  // a same-level level) takes the per-point path
  const int kind = (B.blockmap || B.same) ? 3 : B.kind;
  switch (kind) {
    case LINEAR: launch_kind<kDecomp, LINEAR>(P, B, smem, Rc, Cc, Rs, Cs, s); break;
    case CUBIC_NAK: launch_kind<kDecomp, CUBIC_NAK>(P, B, smem, Rc, Cc, Rs, Cs, s); break;
    case CUBIC_NAT: launch_kind<kDecomp, CUBIC_NAT>(P, B, smem, Rc, Cc, Rs, Cs, s); break;
    default: launch_kind<kDecomp, 3>(P, B, smem, Rc, Cc, Rs, Cs, s); break;
  }
}

void launch_level(bool decomp, const FusedLevel& P, const SweepBufs& B,
                  const float* Rc, const uint16_t* Cc, float* Rs, uint16_t* Cs,
                  cudaStream_t s) {
  const size_t smem = fused_smem_bytes(P, decomp);
  if (decomp)
    launch_dec<true>(P, B, smem, Rc, Cc, Rs, Cs, s);
  else
    launch_dec<false>(P, B, smem, Rc, Cc, Rs, Cs, s);
}

template <bool kDecomp, int KIND>
static void launch_kind_b(const LevelJob* J, const uint32_t* off, int nj,
                          uint32_t nblk, size_t smem, int num_sms, int max_ctas,
                          cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_level_batch<kDecomp, KIND>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const unsigned grid =
      persistent_grid(k_level_batch<kDecomp, KIND>, 256, smem, nblk, num_sms, max_ctas);
  k_level_batch<kDecomp, KIND><<<grid, 256, smem, s>>>(J, off, nj);
}

// kind: the interpolator of every job, or 3 for the per-point path (block
// map or same-level), the value level_kind() returns
void launch_level_batch(bool decomp, int kind, const LevelJob* J,
                        const uint32_t* off, int nj, uint32_t nblk, size_t smem,
                        int num_sms, int max_ctas, cudaStream_t s) {
  if (!nblk) return;
  const int k = kind == LINEAR || kind == CUBIC_NAK || kind == CUBIC_NAT ? kind : 3;
  if (decomp) {
    switch (k) {
      case LINEAR: launch_kind_b<true, LINEAR>(J, off, nj, nblk, smem, num_sms, max_ctas, s); break;
      case CUBIC_NAK: launch_kind_b<true, CUBIC_NAK>(J, off, nj, nblk, smem, num_sms, max_ctas, s); break;
      case CUBIC_NAT: launch_kind_b<true, CUBIC_NAT>(J, off, nj, nblk, smem, num_sms, max_ctas, s); break;
      default: launch_kind_b<true, 3>(J, off, nj, nblk, smem, num_sms, max_ctas, s); break;
    }
  } else {
    switch (k) {
      case LINEAR: launch_kind_b<false, LINEAR>(J, off, nj, nblk, smem, num_sms, max_ctas, s); break;
      case CUBIC_NAK: launch_kind_b<false, CUBIC_NAK>(J, off, nj, nblk, smem, num_sms, max_ctas, s); break;
      case CUBIC_NAT: launch_kind_b<false, CUBIC_NAT>(J, off, nj, nblk, smem, num_sms, max_ctas, s); break;
      default: launch_kind_b<false, 3>(J, off, nj, nblk, smem, num_sms, max_ctas, s); break;
    }
  }
}

int level_kind(const SweepBufs& B) { return (B.blockmap || B.same) ? 3 : B.kind; }

}  // namespace hpez
