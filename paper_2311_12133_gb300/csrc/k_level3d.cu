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

// The stencil of a point from which neighbours exist along its line.
template <int KIND>
__device__ __forceinline__ int edge_formula(bool hm3, bool hp1, bool hp3) {
  if (!hp1) return hm3 ? F_EXTRAP : F_COPY;
  if (KIND == LINEAR) return F_LIN;
  if (hm3 && hp3) return KIND == CUBIC_NAK ? F_NAK4 : F_NAT4;
  if (hm3) return KIND == CUBIC_NAK ? F_NAK3L : F_NAT3L;
  if (hp3) return KIND == CUBIC_NAK ? F_NAK3R : F_NAT3R;
  return F_LIN;
}

// Shared-memory layout: region values [2 planes][RR rows][W] (input values
// first, reconstructions once computed); compress adds the tile's codes
// [2][E1][W]; decompress stages the region's codes [2][RR][W].  A lane
// works on 4 consecutive columns through float4 accesses (conflict-free),
// and pass 3 writes whole rows of codes / reconstructions to global memory.
template <bool kDecomp, int KIND>
__device__ __forceinline__ void level3d_body(
    const Level3D& P, const float* __restrict__ X,
    const uint16_t* __restrict__ codes_full, const float* __restrict__ outl_full,
    const float* __restrict__ Rc, const uint16_t* __restrict__ Cc,
    float* __restrict__ Rs, uint16_t* __restrict__ Cs,
    const Ctl* __restrict__ ctl, unsigned bid) {
  if (ctl->status || ctl->is_const) return;
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = 8;
  const int m0 = P.m[0], m1 = P.m[1], m2 = P.m[2];
  const int RR = P.E1 + 6;
  const int W = P.W, W4 = W >> 2;
  const int t1 = (int)(bid % (unsigned)P.nt1);
  const int t0 = (int)(bid / (unsigned)P.nt1);
  const int P0 = 2 * t0;
  const bool odd_plane = P0 + 1 < m0;
  const int R0 = t1 * P.E1;
  const int Rlo = max(R0 - 3, 0), Rhi = min(R0 + P.E1 + 3, m1);
  const int Tlo = R0, Thi = min(R0 + P.E1, m1);
  const int li = P.level - 1;
  const float el = ctl->el[li], inv2 = ctl->inv2[li], twoe = ctl->twoe[li];
  // region row (plane, row) starts at float index srow(); code tile rows
  auto srow = [&](int plane, int row) { return (plane * RR + (row - (R0 - 3))) * W; };
  uint16_t* ctile = reinterpret_cast<uint16_t*>(sm + 2 * RR * W);  // compress
  uint16_t* scode = ctile;                                            // decompress
  auto trow = [&](int plane, int row) { return (plane * P.E1 + (row - R0)) * W; };
  const uint32_t gst0 = (uint32_t)m1 * (uint32_t)m2, gst1 = (uint32_t)m2;
  const int nc4 = (m2 + 3) >> 2;  // float4 groups per row

  // 0. stage the region rows: input values (compress) or codes (decompress)
  {
    const int nr = Rhi - Rlo;
    const int nrows = nr * (odd_plane ? 2 : 1);
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
  }
  __syncthreads();

  // 1. coarse points of plane P0 (even rows, even columns): reconstruction
  //    for the region, codes for the tile
  {
    const int r0 = (Rlo + 1) & ~1;
    const int nr = (Rhi - r0 + 1) >> 1, nc = (m2 + 1) >> 1;
    for (int r = warp; r < nr; r += NW) {
      const int row = r0 + 2 * r;
      const uint32_t crow = (uint32_t)(P0 >> 1) * P.cst0 + (uint32_t)(row >> 1) * P.cst1;
      const int so = srow(0, row);
      const bool in_tile = row >= Tlo && row < Thi;
      const int to = in_tile ? trow(0, row) : 0;
#pragma unroll 4
      for (int c = lane; c < nc; c += 32) {
        sm[so + 2 * c] = __ldg(Rc + crow + c);
        if (!kDecomp && in_tile) ctile[to + 2 * c] = Cc[crow + c];
      }
    }
  }
  __syncthreads();

  // 2. pass 1 (along dim 0): the odd plane's even rows (region), even columns
  if (odd_plane) {
    const int u0 = P0 + 1;
    const bool hm3 = u0 >= 3, hp1 = u0 + 1 <= m0 - 1, hp3 = u0 + 3 <= m0 - 1;
    const int f = edge_formula<KIND>(hm3, hp1, hp3);  // one stencil per plane
    const int k0 = P0 >> 1;  // coarse plane of u0 - 1
    const int r0 = (Rlo + 1) & ~1;
    const int nr = (Rhi - r0 + 1) >> 1;
    for (int r = warp; r < nr; r += NW) {
      const int row = r0 + 2 * r;
      const bool in_tile = row >= Tlo && row < Thi;
      const uint32_t crow = (uint32_t)(row >> 1) * P.cst1;
      const int so = srow(1, row);
      const int to = in_tile ? trow(1, row) : 0;
      const uint32_t fr = (uint32_t)u0 * P.fs0 + (uint32_t)row * P.fs1;
      for (int g = lane; g < nc4; g += 32) {
        float4 v = sm4[(so >> 2) + g];
        const int col0 = 4 * g;
        float vin[2] = {v.x, v.z};
        float rec[2];
        unsigned code[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = col0 + 2 * h;
          if (col >= m2) break;
          const uint32_t cc = crow + (uint32_t)(col >> 1);
          const float m1v = __ldg(Rc + (uint32_t)k0 * P.cst0 + cc);
          const float p1v = hp1 ? __ldg(Rc + (uint32_t)(k0 + 1) * P.cst0 + cc) : 0.f;
          const float m3v = hm3 ? __ldg(Rc + (uint32_t)(k0 - 1) * P.cst0 + cc) : 0.f;
          const float p3v = hp3 ? __ldg(Rc + (uint32_t)(k0 + 2) * P.cst0 + cc) : 0.f;
          const float p = eval_formula(f, m3v, 0.f, m1v, p1v, 0.f, p3v);
          if (!kDecomp) {
            code[h] = quant(vin[h], p, el, inv2, twoe, rec[h]);
          } else {
            const unsigned cd = P.stage_codes ? scode[so + col]
                                              : codes_full[fr + (uint32_t)col * P.fs2];
            rec[h] = cd ? dequantize(cd, p, twoe) : outl_full[fr + (uint32_t)col * P.fs2];
          }
        }
        v.x = rec[0];
        if (col0 + 2 < m2) v.z = rec[1];
        sm4[(so >> 2) + g] = v;
        if (!kDecomp && in_tile) {
          ctile[to + col0] = (uint16_t)code[0];
          if (col0 + 2 < m2) ctile[to + col0 + 2] = (uint16_t)code[1];
        }
      }
    }
  }
  __syncthreads();

  // 3. pass 2 (along dim 1): both planes, odd rows of the tile, even columns
  {
    const int np = odd_plane ? 2 : 1;
    const int r0 = Tlo | 1;
    const int nr = Thi > r0 ? (Thi - r0 + 1) >> 1 : 0;
    for (int r = warp; r < nr * np; r += NW) {
      const int pl = r / nr, row = r0 + 2 * (r - pl * nr);
      const bool hm3 = row >= 3, hp1 = row + 1 <= m1 - 1, hp3 = row + 3 <= m1 - 1;
      const int f = edge_formula<KIND>(hm3, hp1, hp3);  // one stencil per row
      const int so = srow(pl, row) >> 2, W4r = W4;
      const int to = trow(pl, row);
      const uint32_t fr = (uint32_t)(P0 + pl) * P.fs0 + (uint32_t)row * P.fs1;
      for (int g = lane; g < nc4; g += 32) {
        float4 v = sm4[so + g];
        const float4 a1 = sm4[so - W4r + g];
        const float4 b1 = hp1 ? sm4[so + W4r + g] : a1;
        const float4 a3 = hm3 ? sm4[so - 3 * W4r + g] : a1;
        const float4 b3 = hp3 ? sm4[so + 3 * W4r + g] : a1;
        const int col0 = 4 * g;
        float vin[2] = {v.x, v.z};
        float m3s[2] = {a3.x, a3.z}, m1s[2] = {a1.x, a1.z}, p1s[2] = {b1.x, b1.z},
              p3s[2] = {b3.x, b3.z};
        float rec[2];
        unsigned code[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = col0 + 2 * h;
          if (col >= m2) break;
          const float p = eval_formula(f, m3s[h], 0.f, m1s[h], p1s[h], 0.f, p3s[h]);
          if (!kDecomp) {
            code[h] = quant(vin[h], p, el, inv2, twoe, rec[h]);
          } else {
            const unsigned cd = P.stage_codes ? scode[4 * so + col]
                                              : codes_full[fr + (uint32_t)col * P.fs2];
            rec[h] = cd ? dequantize(cd, p, twoe) : outl_full[fr + (uint32_t)col * P.fs2];
          }
        }
        v.x = rec[0];
        if (col0 + 2 < m2) v.z = rec[1];
        sm4[so + g] = v;
        if (!kDecomp) {
          ctile[to + col0] = (uint16_t)code[0];
          if (col0 + 2 < m2) ctile[to + col0 + 2] = (uint16_t)code[1];
        }
      }
    }
  }
  __syncthreads();

  // 4. pass 3 (along dim 2): both planes, every tile row, odd columns; the
  //    finished rows (codes, reconstruction) go to global memory
  {
    const int np = odd_plane ? 2 : 1;
    const int nr = Thi - Tlo;
    for (int r = warp; r < nr * np; r += NW) {
      const int pl = r / nr, row = Tlo + (r - pl * nr);
      const int u0 = P0 + pl;
      const int so = srow(pl, row) >> 2;
      const int to = trow(pl, row);
      const uint32_t grow = (uint32_t)u0 * gst0 + (uint32_t)row * gst1;
      const uint32_t fr = (uint32_t)u0 * P.fs0 + (uint32_t)row * P.fs1;
      for (int g = lane; g < nc4; g += 32) {
        const float4 v = sm4[so + g];
        const float4 prev = g > 0 ? sm4[so + g - 1] : v;
        const float4 next = g + 1 < W4 ? sm4[so + g + 1] : v;
        const int col0 = 4 * g;
        // odd columns col0+1 and col0+3
        const float vin[2] = {v.y, v.w};
        const float m3s[2] = {prev.z, v.x}, m1s[2] = {v.x, v.z}, p1s[2] = {v.z, next.x},
                    p3s[2] = {next.x, next.z};
        float rec[2] = {v.y, v.w};
        unsigned code[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = col0 + 1 + 2 * h;
          if (col >= m2) break;
          float p;
          if (col >= 3 && col + 3 <= m2 - 1) {
            p = KIND == LINEAR ? eval_formula(F_LIN, 0.f, 0.f, m1s[h], p1s[h], 0.f, 0.f)
                               : stencil4<KIND>(m3s[h], m1s[h], p1s[h], p3s[h]);
          } else {
            const int f = edge_formula<KIND>(col >= 3, col + 1 <= m2 - 1, col + 3 <= m2 - 1);
            p = eval_formula(f, m3s[h], 0.f, m1s[h], p1s[h], 0.f, p3s[h]);
          }
          if (!kDecomp) {
            code[h] = quant(vin[h], p, el, inv2, twoe, rec[h]);
          } else {
            const unsigned cd = P.stage_codes ? scode[4 * so + col]
                                              : codes_full[fr + (uint32_t)col * P.fs2];
            rec[h] = cd ? dequantize(cd, p, twoe) : outl_full[fr + (uint32_t)col * P.fs2];
          }
        }
        const float4 out = make_float4(v.x, rec[0], v.z, rec[1]);
        const bool full = col0 + 4 <= m2 && P.vec_out;
        if (!kDecomp) {
          const uint16_t c0 = ctile[to + col0];
          const uint16_t c2 = col0 + 2 < m2 ? ctile[to + col0 + 2] : 0;
          if (full) {
            *reinterpret_cast<uint2*>(Cs + grow + col0) =
                make_uint2((uint32_t)c0 | (code[0] << 16), (uint32_t)c2 | (code[1] << 16));
            if (P.write_recon) *reinterpret_cast<float4*>(Rs + grow + col0) = out;
          } else {
            const uint16_t cv[4] = {c0, (uint16_t)code[0], c2, (uint16_t)code[1]};
            const float ov[4] = {out.x, out.y, out.z, out.w};
            for (int q = 0; q < 4 && col0 + q < m2; ++q) {
              Cs[grow + col0 + q] = cv[q];
              if (P.write_recon) Rs[grow + col0 + q] = ov[q];
            }
          }
        } else {
          if (full) {
            *reinterpret_cast<float4*>(Rs + grow + col0) = out;
          } else {
            const float ov[4] = {out.x, out.y, out.z, out.w};
            for (int q = 0; q < 4 && col0 + q < m2; ++q) Rs[grow + col0 + q] = ov[q];
          }
        }
      }
    }
  }
}

template <bool kDecomp, int KIND>
__global__ void __launch_bounds__(256)
    k_level3d(Level3D P, const float* __restrict__ X,
              const uint16_t* __restrict__ codes_full,
              const float* __restrict__ outl_full, const float* __restrict__ Rc,
              const uint16_t* __restrict__ Cc, float* __restrict__ Rs,
              uint16_t* __restrict__ Cs, const Ctl* __restrict__ ctl) {
  level3d_body<kDecomp, KIND>(P, X, codes_full, outl_full, Rc, Cc, Rs, Cs, ctl,
                              blockIdx.x);
}

// batched, persistent: job j owns tiles [off[j], off[j+1]) of the launch
template <bool kDecomp, int KIND>
__global__ void __launch_bounds__(256)
    k_level3d_batch(const Level3DJob* __restrict__ J,
                    const uint32_t* __restrict__ off, int nj) {
  for_each_batch_block(off, nj, [&](int j, uint32_t t) {
    const Level3DJob& q = J[j];
    const Level3D P = q.P;
    level3d_body<kDecomp, KIND>(P, q.X, q.codes_full, q.outl_full, q.Rc, q.Cc,
                                q.Rs, q.Cs, q.ctl, t);
  });
}

size_t level3d_smem_bytes(const Level3D& P, bool decomp) {
  size_t b = 2ull * (P.E1 + 6) * P.W * sizeof(float);
  if (decomp && P.stage_codes) b += 2ull * (P.E1 + 6) * P.W * sizeof(uint16_t);
  if (!decomp) b += 2ull * P.E1 * P.W * sizeof(uint16_t);
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

template <bool kDecomp, int KIND>
static void launch3b(const Level3DJob* J, const uint32_t* off, int nj,
                     uint32_t nblk, size_t smem, int num_sms, int max_ctas,
                     cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_level3d_batch<kDecomp, KIND>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const unsigned grid =
      persistent_grid(k_level3d_batch<kDecomp, KIND>, 256, smem, nblk, num_sms, max_ctas);
  k_level3d_batch<kDecomp, KIND><<<grid, 256, smem, s>>>(J, off, nj);
}

void launch_level3d_batch(bool decomp, int kind, const Level3DJob* J,
                          const uint32_t* off, int nj, uint32_t nblk,
                          size_t smem, int num_sms, int max_ctas, cudaStream_t s) {
  if (!nblk) return;
  if (decomp) {
    if (kind == LINEAR) launch3b<true, LINEAR>(J, off, nj, nblk, smem, num_sms, max_ctas, s);
    else if (kind == CUBIC_NAK)
      launch3b<true, CUBIC_NAK>(J, off, nj, nblk, smem, num_sms, max_ctas, s);
    else launch3b<true, CUBIC_NAT>(J, off, nj, nblk, smem, num_sms, max_ctas, s);
  } else {
    if (kind == LINEAR) launch3b<false, LINEAR>(J, off, nj, nblk, smem, num_sms, max_ctas, s);
    else if (kind == CUBIC_NAK)
      launch3b<false, CUBIC_NAK>(J, off, nj, nblk, smem, num_sms, max_ctas, s);
    else launch3b<false, CUBIC_NAT>(J, off, nj, nblk, smem, num_sms, max_ctas, s);
  }
}

}  // namespace hpez
