// k_level3d.cu -- one level of the 1D-style sweep for the common 3D layout:
// direction order (0, 1, 2) (slowest dimension first, fastest last), one
// interpolator for the whole level, no same-level halves, no block map.
//
// A CTA owns two consecutive planes (an even plane P0 and the odd plane
// P0+1) and E1 rows of the level grid, whole rows along the fastest
// dimension.  Pass 1 (along dim 0) predicts the odd plane's even-row,
// even-column points from the coarse grid; pass 2 (along dim 1) the odd
// rows' even columns from rows +-1, +-3; pass 3 (along dim 2) every odd
// column from columns +-1, +-3 (Sec. 5.3, 1D-style).  Pass 2 needs pass 1
// on 3 rows beyond the tile, so those are recomputed (the same operations
// on the same inputs as in the neighbouring CTA).  The CTA's input rows
// are staged in shared memory with asynchronous copies and overwritten in
// place by the reconstruction.
#include "hpez_internal.cuh"
#include "hpez_launch.h"

namespace hpez {

namespace {

__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
}

template <int KIND>
__device__ __forceinline__ float stencil4(float m3, float m1, float p1, float p3) {
  if (KIND == LINEAR) return eval_formula(F_LIN, 0.f, 0.f, m1, p1, 0.f, 0.f);
  if (KIND == CUBIC_NAK) return eval_formula(F_NAK4, m3, 0.f, m1, p1, 0.f, p3);
  return eval_formula(F_NAT4, m3, 0.f, m1, p1, 0.f, p3);
}

// Boundary stencil from which of the neighbours at -3, -1, +1, +3 exist.
template <int KIND>
__device__ __forceinline__ float stencil_edge(int f, float m3, float m1, float p1,
                                              float p3) {
  return eval_formula(f, m3, 0.f, m1, p1, 0.f, p3);
}

__device__ __forceinline__ unsigned quant(float x, float p, float el, float inv2,
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

}  // namespace

template <bool kDecomp, int KIND>
__global__ void __launch_bounds__(256)
    k_level3d(Level3D P, const float* __restrict__ X,
              const uint16_t* __restrict__ codes_full,
              const float* __restrict__ outl_full, const float* __restrict__ Rc,
              const uint16_t* __restrict__ Cc, float* __restrict__ Rs,
              uint16_t* __restrict__ Cs, const Ctl* __restrict__ ctl) {
  if (ctl->status || ctl->is_const) return;
  extern __shared__ float sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = 8;
  const int m0 = P.m[0], m1 = P.m[1], m2 = P.m[2];
  const int RR = P.E1 + 6;          // region rows: tile rows + 3 on each side
  const int W = P.W;                // shared-memory row length (>= m2)
  const int t1 = blockIdx.x % P.nt1;
  const int t0 = blockIdx.x / P.nt1;
  const int P0 = 2 * t0;
  const bool odd_plane = P0 + 1 < m0;
  const int R0 = t1 * P.E1;
  const int Rlo = max(R0 - 3, 0), Rhi = min(R0 + P.E1 + 3, m1);
  const int Tlo = R0, Thi = min(R0 + P.E1, m1);
  const int li = P.level - 1;
  const float el = ctl->el[li], inv2 = ctl->inv2[li], twoe = ctl->twoe[li];
  uint16_t* scode = reinterpret_cast<uint16_t*>(sm + 2 * RR * W);
  auto srow = [&](int plane, int row) { return plane * RR * W + (row - (R0 - 3)) * W; };
  const uint32_t gst0 = (uint32_t)m1 * (uint32_t)m2, gst1 = (uint32_t)m2;

  // 0. stage the region rows: input values (compress) or codes (decompress)
  {
    const int nrows = (Rhi - Rlo) * (odd_plane ? 2 : 1);
    const int nr = Rhi - Rlo;
    for (int r = warp; r < nrows; r += NW) {
      const int pl = r / nr, row = Rlo + (r - pl * nr);
      const uint32_t fr = (uint32_t)(P0 + pl) * P.fs0 + (uint32_t)row * P.fs1;
      const int so = srow(pl, row);
      if (!kDecomp) {
        if (P.stage16)
          for (int c = lane * 4; c < m2; c += 128) cp16(sm + so + c, X + fr + c);
        else
          for (int c = lane; c < m2; c += 32) cp4(sm + so + c, X + fr + (uint32_t)c * P.fs2);
      } else if (P.stage_codes) {
        for (int c = lane * 8; c < m2; c += 256) cp16(scode + so + c, codes_full + fr + c);
      }
    }
    cp_wait();
    __syncthreads();
  }

  // 1. coarse points: plane P0, even rows, even columns
  {
    const int r0 = (Rlo + 1) & ~1;
    const int nr = (Rhi - r0 + 1) >> 1, nc = (m2 + 1) >> 1;
    for (int r = warp; r < nr; r += NW) {
      const int row = r0 + 2 * r;
      const uint32_t crow = (uint32_t)(P0 >> 1) * P.cst0 + (uint32_t)(row >> 1) * P.cst1;
      const int so = srow(0, row);
#pragma unroll 4
      for (int c = lane; c < nc; c += 32) sm[so + 2 * c] = __ldg(Rc + crow + c);
    }
  }
  __syncthreads();

  // 2. pass 1 (along dim 0): odd plane, even rows of the region, even columns
  if (odd_plane) {
    const int u0 = P0 + 1;
    const bool hm3 = u0 >= 3, hp1 = u0 + 1 <= m0 - 1, hp3 = u0 + 3 <= m0 - 1;
    int f;  // the same stencil for the whole plane
    if (!hp1) f = hm3 ? F_EXTRAP : F_COPY;
    else if (KIND == LINEAR) f = F_LIN;
    else if (hm3 && hp3) f = KIND == CUBIC_NAK ? F_NAK4 : F_NAT4;
    else if (hm3) f = KIND == CUBIC_NAK ? F_NAK3L : F_NAT3L;
    else if (hp3) f = KIND == CUBIC_NAK ? F_NAK3R : F_NAT3R;
    else f = F_LIN;
    const int k0 = P0 >> 1;  // coarse plane of u0 - 1
    const int r0 = (Rlo + 1) & ~1;
    const int nr = (Rhi - r0 + 1) >> 1, nc = (m2 + 1) >> 1;
    for (int r = warp; r < nr; r += NW) {
      const int row = r0 + 2 * r;
      const bool in_tile = row >= Tlo && row < Thi;
      const uint32_t crow = (uint32_t)(row >> 1) * P.cst1;
      const int so = srow(1, row);
      const uint32_t grow = (uint32_t)u0 * gst0 + (uint32_t)row * gst1;
      const uint32_t fr = (uint32_t)u0 * P.fs0 + (uint32_t)row * P.fs1;
#pragma unroll 2
      for (int c = lane; c < nc; c += 32) {
        const int col = 2 * c;
        const uint32_t cc = crow + (uint32_t)c;
        const float m1v = __ldg(Rc + (uint32_t)k0 * P.cst0 + cc);
        const float p1v = hp1 ? __ldg(Rc + (uint32_t)(k0 + 1) * P.cst0 + cc) : 0.f;
        const float m3v = hm3 ? __ldg(Rc + (uint32_t)(k0 - 1) * P.cst0 + cc) : 0.f;
        const float p3v = hp3 ? __ldg(Rc + (uint32_t)(k0 + 2) * P.cst0 + cc) : 0.f;
        const float p = eval_formula(f, m3v, 0.f, m1v, p1v, 0.f, p3v);
        float rec;
        if (!kDecomp) {
          const unsigned code = quant(sm[so + col], p, el, inv2, twoe, rec);
          if (in_tile) {
            Cs[grow + (uint32_t)col] = (uint16_t)code;
            if (P.write_recon) Rs[grow + (uint32_t)col] = rec;
          }
        } else {
          const unsigned code = P.stage_codes ? scode[so + col]
                                              : codes_full[fr + (uint32_t)col * P.fs2];
          rec = code ? dequantize(code, p, twoe) : outl_full[fr + (uint32_t)col * P.fs2];
          if (in_tile) Rs[grow + (uint32_t)col] = rec;
        }
        sm[so + col] = rec;
      }
    }
  }
  __syncthreads();

  // 3. pass 2 (along dim 1): both planes, odd rows of the tile, even columns
  {
    const int np = odd_plane ? 2 : 1;
    const int r0 = Tlo | 1;
    const int nr = Thi > r0 ? (Thi - r0 + 1) >> 1 : 0, nc = (m2 + 1) >> 1;
    for (int r = warp; r < nr * np; r += NW) {
      const int pl = r / nr, row = r0 + 2 * (r - pl * nr);
      const int u0 = P0 + pl;
      const bool hm3 = row >= 3, hp1 = row + 1 <= m1 - 1, hp3 = row + 3 <= m1 - 1;
      int f;
      if (!hp1) f = hm3 ? F_EXTRAP : F_COPY;
      else if (KIND == LINEAR) f = F_LIN;
      else if (hm3 && hp3) f = KIND == CUBIC_NAK ? F_NAK4 : F_NAT4;
      else if (hm3) f = KIND == CUBIC_NAK ? F_NAK3L : F_NAT3L;
      else if (hp3) f = KIND == CUBIC_NAK ? F_NAK3R : F_NAT3R;
      else f = F_LIN;
      const int so = srow(pl, row);
      const uint32_t grow = (uint32_t)u0 * gst0 + (uint32_t)row * gst1;
      const uint32_t fr = (uint32_t)u0 * P.fs0 + (uint32_t)row * P.fs1;
      const bool interior = KIND == LINEAR ? f == F_LIN : (f == F_NAK4 || f == F_NAT4);
#pragma unroll 2
      for (int c = lane; c < nc; c += 32) {
        const int col = 2 * c;
        const int s = so + col;
        float p;
        if (interior) {
          // only the knots the stencil uses are read (rows +-3 may not exist
          // for the linear stencil)
          if (KIND == LINEAR)
            p = eval_formula(F_LIN, 0.f, 0.f, sm[s - W], sm[s + W], 0.f, 0.f);
          else
            p = stencil4<KIND>(sm[s - 3 * W], sm[s - W], sm[s + W], sm[s + 3 * W]);
        } else {
          const float m1v = sm[s - W];
          const float p1v = hp1 ? sm[s + W] : 0.f;
          const float m3v = hm3 ? sm[s - 3 * W] : 0.f;
          const float p3v = hp3 ? sm[s + 3 * W] : 0.f;
          p = eval_formula(f, m3v, 0.f, m1v, p1v, 0.f, p3v);
        }
        float rec;
        if (!kDecomp) {
          const unsigned code = quant(sm[s], p, el, inv2, twoe, rec);
          Cs[grow + (uint32_t)col] = (uint16_t)code;
          if (P.write_recon) Rs[grow + (uint32_t)col] = rec;
        } else {
          const unsigned code = P.stage_codes ? scode[s]
                                              : codes_full[fr + (uint32_t)col * P.fs2];
          rec = code ? dequantize(code, p, twoe) : outl_full[fr + (uint32_t)col * P.fs2];
          Rs[grow + (uint32_t)col] = rec;
        }
        sm[s] = rec;
      }
    }
  }
  __syncthreads();

  // 4. pass 3 (along dim 2): both planes, every row of the tile, odd columns
  {
    const int np = odd_plane ? 2 : 1;
    const int nr = Thi - Tlo, nc = m2 >> 1;
    for (int r = warp; r < nr * np; r += NW) {
      const int pl = r / nr, row = Tlo + (r - pl * nr);
      const int u0 = P0 + pl;
      const int so = srow(pl, row);
      const uint32_t grow = (uint32_t)u0 * gst0 + (uint32_t)row * gst1;
      const uint32_t fr = (uint32_t)u0 * P.fs0 + (uint32_t)row * P.fs1;
#pragma unroll 4
      for (int c = lane; c < nc; c += 32) {
        const int col = 2 * c + 1;
        const int s = so + col;
        float p;
        if (col >= 3 && col + 3 <= m2 - 1) {
          if (KIND == LINEAR)
            p = eval_formula(F_LIN, 0.f, 0.f, sm[s - 1], sm[s + 1], 0.f, 0.f);
          else
            p = stencil4<KIND>(sm[s - 3], sm[s - 1], sm[s + 1], sm[s + 3]);
        } else {
          const bool hm3 = col >= 3, hp1 = col + 1 <= m2 - 1, hp3 = col + 3 <= m2 - 1;
          int f;
          if (!hp1) f = hm3 ? F_EXTRAP : F_COPY;
          else if (KIND == LINEAR) f = F_LIN;
          else if (hm3) f = KIND == CUBIC_NAK ? F_NAK3L : F_NAT3L;
          else if (hp3) f = KIND == CUBIC_NAK ? F_NAK3R : F_NAT3R;
          else f = F_LIN;
          const float m1v = sm[s - 1];
          const float p1v = hp1 ? sm[s + 1] : 0.f;
          const float m3v = hm3 ? sm[s - 3] : 0.f;
          const float p3v = hp3 ? sm[s + 3] : 0.f;
          p = eval_formula(f, m3v, 0.f, m1v, p1v, 0.f, p3v);
        }
        float rec;
        if (!kDecomp) {
          const unsigned code = quant(sm[s], p, el, inv2, twoe, rec);
          Cs[grow + (uint32_t)col] = (uint16_t)code;
          if (P.write_recon) Rs[grow + (uint32_t)col] = rec;
        } else {
          const unsigned code = P.stage_codes ? scode[s]
                                              : codes_full[fr + (uint32_t)col * P.fs2];
          rec = code ? dequantize(code, p, twoe) : outl_full[fr + (uint32_t)col * P.fs2];
          Rs[grow + (uint32_t)col] = rec;
        }
      }
    }
  }

  // 5. the tile's coarse points: codes from the coarse grid, reconstruction
  {
    const int r0 = (Tlo + 1) & ~1;
    const int nr = Thi > r0 ? (Thi - r0 + 1) >> 1 : 0, nc = (m2 + 1) >> 1;
    for (int r = warp; r < nr; r += NW) {
      const int row = r0 + 2 * r;
      const uint32_t grow = (uint32_t)P0 * gst0 + (uint32_t)row * gst1;
      const uint32_t crow = (uint32_t)(P0 >> 1) * P.cst0 + (uint32_t)(row >> 1) * P.cst1;
      const int so = srow(0, row);
#pragma unroll 4
      for (int c = lane; c < nc; c += 32) {
        if (!kDecomp) {
          Cs[grow + 2u * c] = Cc[crow + c];
          if (P.write_recon) Rs[grow + 2u * c] = sm[so + 2 * c];
        } else {
          Rs[grow + 2u * c] = sm[so + 2 * c];
        }
      }
    }
  }
}

size_t level3d_smem_bytes(const Level3D& P, bool decomp) {
  size_t b = 2ull * (P.E1 + 6) * P.W * sizeof(float);
  if (decomp && P.stage_codes) b += 2ull * (P.E1 + 6) * P.W * sizeof(uint16_t);
  return b;
}

template <bool kDecomp, int KIND>
static void launch3(const Level3D& P, const SweepBufs& B, const float* Rc,
                    const uint16_t* Cc, float* Rs, uint16_t* Cs, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_level3d<kDecomp, KIND>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const unsigned grid = (unsigned)(P.nt0 * P.nt1);
  k_level3d<kDecomp, KIND><<<grid, 256, level3d_smem_bytes(P, kDecomp), s>>>(
      P, B.x, B.codes_full, B.outl_full, Rc, Cc, Rs, Cs, B.ctl);
}

void launch_level3d(bool decomp, const Level3D& P, const SweepBufs& B,
                    const float* Rc, const uint16_t* Cc, float* Rs, uint16_t* Cs,
                    cudaStream_t s) {
  if (decomp) {
    if (B.kind == LINEAR) launch3<true, LINEAR>(P, B, Rc, Cc, Rs, Cs, s);
    else if (B.kind == CUBIC_NAK) launch3<true, CUBIC_NAK>(P, B, Rc, Cc, Rs, Cs, s);
    else launch3<true, CUBIC_NAT>(P, B, Rc, Cc, Rs, Cs, s);
  } else {
    if (B.kind == LINEAR) launch3<false, LINEAR>(P, B, Rc, Cc, Rs, Cs, s);
    else if (B.kind == CUBIC_NAK) launch3<false, CUBIC_NAK>(P, B, Rc, Cc, Rs, Cs, s);
    else launch3<false, CUBIC_NAT>(P, B, Rc, Cc, Rs, Cs, s);
  }
}

}  // namespace hpez
