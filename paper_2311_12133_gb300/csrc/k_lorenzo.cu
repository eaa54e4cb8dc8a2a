// k_lorenzo.cu -- the Lorenzo predictor over the whole field (Sec. 6.5:
// the dynamic-order predictor, order 1 or 2, that the tuner selects when
// its estimate beats interpolation), read as block-local: the field is cut
// into blocks of side A along every dimension, and inside a block a point
// is predicted from the reconstructed points of its block (a neighbour
// outside the block reads 0) -- the recurrence the tuner's Lorenzo test
// runs on its sample blocks.
//
// The recurrence is sequential inside a block: point (i0, i1, i2) needs
// every neighbour (i0 - a, i1 - b, i2 - c), so the points of one wavefront
// plane i0 + i1 + i2 = t are independent.  A thread owns one (i0, i1)
// column of a block and walks it along i2 one step per barrier; a column
// with s = i0 + i1 starts s steps after column (0, 0).  A CTA does not
// wait for a block to drain: it streams its blocks back to back, column
// (i0, i1) working on its j-th block at steps P j + s .. P j + s + P - 1
// (P = the block side along i2), so past the first s steps every column
// thread has a point at every step.
//
// The value a neighbour column wrote for the same i2 is on the ring slot
// of the step it was written in: column (i0 - a, i1 - b) reaches i2 at
// step tau - a - b, one slot per step, a ring of more slots than the
// stencil's reach (4 for order 1, 8 for order 2).  Values for i2 - c, c >
// 0, were loaded at the thread's previous steps and stay in registers, so
// a step reads one value per neighbour column from shared memory.  Rows
// and columns -1, -2 of the ring are zero, the neighbours outside the
// block; the i2 history is zeroed when a column starts a block.  The
// input of the next eight steps (the field values, or the codes and the
// escaped values) is loaded eight steps ahead, one 32-byte sector of a
// field row per thread.
//
// For 32 x 32 columns (3D, A = 32) lane l of warp w owns column (l,
// (w - l) mod 32): its s is w or w + 32, so every lane of a warp is at the
// same i2 at every step and the segment work does not diverge; the ring
// row width 34 keeps the lanes' shared-memory words in distinct banks.
// Order 1 on rows of 16-byte multiples takes k_lorenzo_tma instead: the
// input of a warp's 32 columns arrives as one TMA tensor box per segment.
#include <cuda.h>

#include <cstdio>
#include <cstdlib>
#include "hpez.h"
#include "hpez_internal.cuh"
#include "hpez_launch.h"

namespace hpez {
namespace {

constexpr int kSeg = 8;  // input / output segment along i2


template <int ORDER>
__host__ __device__ constexpr int lor_ring() { return ORDER == 1 ? 4 : 8; }

// per-dimension coefficient of offset a: order 1 (1, -1), order 2
// (1, -2, 1); the weight of term (a, b, c) is minus their product
template <int ORDER>
__host__ __device__ constexpr float lor_coef(int a) {
  return ORDER == 1 ? (a == 0 ? 1.0f : -1.0f) : (a == 1 ? -2.0f : 1.0f);
}

// acc + w v in binary32 for the constant weight w: +-1 as an add or a
// subtract (w v is exact), otherwise the product rounded, then the sum
template <int ORDER>
__device__ __forceinline__ float lor_term(float acc, int a, int b, int c, float v) {
  const float w = -(lor_coef<ORDER>(a) * lor_coef<ORDER>(b) * lor_coef<ORDER>(c));
  if (w == 1.0f) return __fadd_rn(acc, v);
  if (w == -1.0f) return __fsub_rn(acc, v);
  return __fadd_rn(acc, __fmul_rn(w, v));
}

// A thread's view of one block: the field index of its column's first
// point and the column's points inside the block (0 when the column lies
// outside it)
struct ColGeo {
  uint32_t col;
  int m2;
};

// The blocks a CTA streams, blockIdx.x + j gridDim.x, walked as a mixed-
// radix counter over (nb[0], nb[1], nb[2]) whose step is the grid size's
// digits g: no division per block.
struct Walk {
  uint32_t b0, b1, b2;
};

__device__ __forceinline__ Walk walk_start(const LorGeom& G, uint32_t bid) {
  uint32_t b = bid;
  Walk w;
  w.b2 = b % G.nb[2];
  b /= G.nb[2];
  w.b1 = b % G.nb[1];
  w.b0 = b / G.nb[1];
  return w;
}

__device__ __forceinline__ void walk_next(const LorGeom& G, Walk& w) {
  w.b2 += G.g[2];
  uint32_t c = w.b2 >= G.nb[2] ? 1u : 0u;
  w.b2 -= c ? G.nb[2] : 0u;
  w.b1 += G.g[1] + c;
  c = w.b1 >= G.nb[1] ? 1u : 0u;
  w.b1 -= c ? G.nb[1] : 0u;
  w.b0 += G.g[0] + c;
}

__device__ __forceinline__ ColGeo col_geo(const LorGeom& G, const Walk& w, int i0, int i1) {
  const uint32_t o0 = w.b0 * G.B[0] + (uint32_t)i0, o1 = w.b1 * G.B[1] + (uint32_t)i1,
                 o2 = w.b2 * G.B[2];
  const bool in = o0 < G.n[0] && o1 < G.n[1] && o2 < G.n[2];
  ColGeo g;
  g.m2 = in ? (int)min(G.B[2], G.n[2] - o2) : 0;
  g.col = in ? o0 * G.st[0] + o1 * G.st[1] + o2 : 0u;
  return g;
}

// The loads of a segment go straight into the registers that hold it
// until it is used a segment later: the index is clamped to 0 (an
// in-bounds read whose values are not used) instead of branching, so no
// instruction waits on a load at the time it is issued.  They are volatile
// asm so that the compiler keeps them where they are issued, a segment
// ahead, rather than moving them next to their first use.
//   vec: one 32-byte sector (8 floats or 8 codes) per row; the rows start
//   on 16-byte boundaries.  Otherwise sl <= 8 scalar loads.
__device__ __forceinline__ float4 ld_f4(const float* p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_f1(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ uint4 ld_u4(const uint16_t* p) {
  uint4 v;
  asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ uint32_t ld_u16(const uint16_t* p) {
  unsigned short v;
  asm volatile("ld.global.nc.u16 %0, [%1];" : "=h"(v) : "l"(p));
  return (uint32_t)v;
}

template <bool kVec>
__device__ __forceinline__ void load_x(float4& a, float4& b, const float* x, const ColGeo& g,
                                       int i2, int sl) {
  if (kVec) {
    const float* p = x + (i2 < g.m2 ? g.col + (uint32_t)i2 : 0u);
    a = ld_f4(p);
    b = ld_f4(p + 4);
  } else {
    float t[kSeg];
#pragma unroll
    for (int k = 0; k < kSeg; ++k)
      t[k] = ld_f1(x + (k < sl && i2 + k < g.m2 ? g.col + (uint32_t)(i2 + k) : 0u));
    a = make_float4(t[0], t[1], t[2], t[3]);
    b = make_float4(t[4], t[5], t[6], t[7]);
  }
}

// codes of a segment: vec, one 16-byte load (8 codes, two per word);
// otherwise 8 scalar loads kept unpacked until the segment is promoted
struct RawCodes {
  uint32_t w[kSeg];
};

template <bool kVec>
__device__ __forceinline__ void load_codes(uint4& v, RawCodes& r, const uint16_t* codes,
                                           const ColGeo& g, int i2, int sl) {
  if (kVec) {
    v = ld_u4(codes + (i2 < g.m2 ? g.col + (uint32_t)i2 : 0u));
  } else {
#pragma unroll
    for (int k = 0; k < kSeg; ++k) {
      const bool ok = k < sl && i2 + k < g.m2;
      r.w[k] = ld_u16(codes + (ok ? g.col + (uint32_t)(i2 + k) : 0u));
      r.w[k] = ok ? r.w[k] : 1u;
    }
  }
}

template <bool kVec>
__device__ __forceinline__ uint4 pack_codes(const uint4& v, const RawCodes& r) {
  if (kVec) return v;
  return make_uint4(r.w[0] | (r.w[1] << 16), r.w[2] | (r.w[3] << 16), r.w[4] | (r.w[5] << 16),
                    r.w[6] | (r.w[7] << 16));
}

__device__ __forceinline__ void prefetch_l1(const float* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// --- TMA tensor boxes and their mbarriers (the box-fed kernel) ---
constexpr int kWaitLimit = 1 << 24;
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
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
// ends after kWaitNs of wall time or kWaitLimit polls; false: not landed
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

// The prediction of the point at i2 of this column at step tau: the
// stencil's terms in the order of the offsets (a, b, c); c = 0 from the
// ring slot written a + b steps ago, c > 0 from the history h (c <= HD on
// the neighbour columns) or the ring.  v0 receives the c = 0 values.
template <int ORDER, int L0, int L1, int HD, int RING>
__device__ __forceinline__ float lor_predict(const float* mine, int tau, int slot, int W, int i2,
                                             const float (&h)[L0 + 1][L1 + 1][ORDER],
                                             float (&v0)[L0 + 1][L1 + 1]) {
#pragma unroll
  for (int a = 0; a <= L0; ++a)
#pragma unroll
    for (int b = 0; b <= L1; ++b)
      if (a + b > 0) v0[a][b] = mine[((tau - a - b) & (RING - 1)) * slot - a * W - b];
  float acc = 0.0f;
#pragma unroll
  for (int a = 0; a <= L0; ++a)
#pragma unroll
    for (int b = 0; b <= L1; ++b)
#pragma unroll
      for (int c = 0; c <= ORDER; ++c) {
        if (a + b + c == 0) continue;
        float v;
        if (c == 0)
          v = v0[a][b];
        else if (c <= HD || a + b == 0)
          v = h[a][b][c - 1];
        else
          v = i2 >= c ? mine[((tau - a - b - c) & (RING - 1)) * slot - a * W - b] : 0.0f;
        acc = lor_term<ORDER>(acc, a, b, c, v);
      }
  return acc;
}

// the histories after the point: c = 1 becomes this step's c = 0 value
template <int ORDER, int L0, int L1, int HD>
__device__ __forceinline__ void lor_shift(float (&h)[L0 + 1][L1 + 1][ORDER],
                                          const float (&v0)[L0 + 1][L1 + 1], float rec) {
#pragma unroll
  for (int a = 0; a <= L0; ++a)
#pragma unroll
    for (int b = 0; b <= L1; ++b) {
#pragma unroll
      for (int c = ORDER - 1; c > 0; --c)
        if (a + b == 0 || c < HD) h[a][b][c] = h[a][b][c - 1];
      h[a][b][0] = a + b > 0 ? v0[a][b] : rec;
    }
}

template <int ORDER, int L0, int L1>
__device__ __forceinline__ void lor_zero(float (&h)[L0 + 1][L1 + 1][ORDER]) {
#pragma unroll
  for (int a = 0; a <= L0; ++a)
#pragma unroll
    for (int b = 0; b <= L1; ++b)
#pragma unroll
      for (int c = 0; c < ORDER; ++c) h[a][b][c] = 0.0f;
}

// A CTA of the Lorenzo pass: block index bid of a grid of `grid` CTAs over
// the field of G (G.g: that grid size in the radix of G.nb).
template <bool kDecomp, int ORDER, int NDR, bool kVec, bool kSkew>
__device__ __forceinline__ void lor_body(const LorGeom& G, const float* __restrict__ x,
                                         uint16_t* __restrict__ codes, float* __restrict__ out,
                                         const Ctl* __restrict__ ctl, uint32_t bid,
                                         uint32_t grid) {
  if (ctl->status || ctl->is_const) return;
  constexpr int RING = lor_ring<ORDER>();
  constexpr int L0 = NDR >= 3 ? ORDER : 0;  // stencil reach along slot 0
  constexpr int L1 = NDR >= 2 ? ORDER : 0;  // along slot 1
  extern __shared__ float ring[];
  for (uint32_t i = threadIdx.x; i < RING * G.slot; i += blockDim.x) ring[i] = 0.0f;

  const int B1 = (int)G.B[1];
  const int q = (int)threadIdx.x;
  const bool real = q < (int)(G.B[0] * G.B[1]);
  int i0, i1;
  if (kSkew) {
    i0 = q & 31;
    i1 = ((q >> 5) - i0) & 31;
  } else {
    i0 = real ? q / B1 : 0;
    i1 = real ? q - i0 * B1 : 0;
  }
  const int P = (int)G.B[2];
  const int sl = kVec ? kSeg : min(kSeg, P);
  const uint32_t J = (G.nblocks - 1u - bid) / grid + 1u;
  const int span = P * (int)J;  // steps a column is busy
  const int T = span + (int)G.B[0] + B1 - 2;
  const int W = (int)G.W;
  float* const mine = ring + (i0 + 2) * W + i1 + 2;
  const float e = ctl->e;
  // 1 / (2 e) in double, rounded once: one thread divides (fp64 is slow)
  __shared__ float s_inv2;
  if (threadIdx.x == 0) s_inv2 = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(2.0, (double)e)));
  const float twoe = __fmul_rn(2.0f, e);

  // h[a][b][c - 1]: column (i0 - a, i1 - b) at i2 - c, for c <= HD on the
  // neighbour columns (the rest is read from the ring: in 3D order 2 the
  // registers hold one step of history), all c on the own column
  constexpr int HD = (ORDER == 2 && NDR == 3) ? 1 : ORDER;
  float h[L0 + 1][L1 + 1][ORDER];

  // input pipeline.  compress: the field values of the next segment (n0,
  // n1) and of the current one (cv).  decompress: the codes two segments
  // ahead (cA), of the next segment (cB, whose escaped values are being
  // prefetched into L1) and of the current one (cc); ov collects the
  // reconstructions of the segment for one vector store.
  Walk wk = walk_start(G, bid);
  ColGeo cg = col_geo(G, wk, i0, i1);
  ColGeo gB = cg, gA = cg;
  float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
  float cv[kSeg];
  uint4 cA = make_uint4(0u, 0u, 0u, 0u), cB = cA, cc = cA;
  RawCodes rA;
  float ov[kSeg];
  uint32_t pk[kSeg / 2];  // compress: codes of the segment
#pragma unroll
  for (int k = 0; k < kSeg; ++k) {
    cv[k] = ov[k] = 0.0f;
    rA.w[k] = 1u;
  }
#pragma unroll
  for (int k = 0; k < kSeg / 2; ++k) pk[k] = 0u;
  if (real) {
    if (!kDecomp) {
      load_x<kVec>(n0, n1, x, cg, 0, sl);
    } else {
      load_codes<kVec>(cA, rA, codes, gB, 0, sl);
      cB = pack_codes<kVec>(cA, rA);
#pragma unroll
      for (int k = 0; k < kSeg; ++k)
        if (k < gB.m2 && ((((k & 1) ? (&cB.x)[k / 2] >> 16 : (&cB.x)[k / 2]) & 0xFFFFu) == 0u))
          prefetch_l1(out + gB.col + (uint32_t)k);
      if (sl < span) {
        const int i2a = sl & (P - 1);
        if (i2a == 0) {
          walk_next(G, wk);
          gA = col_geo(G, wk, i0, i1);
        }
        load_codes<kVec>(cA, rA, codes, gA, i2a, sl);
      }
    }
  }
  __syncthreads();
  const float inv2 = s_inv2;

  int u = -(i0 + i1);  // this column's step within its block stream
  for (int tau = 0; tau < T; ++tau, ++u) {
    if (real && u >= 0 && u < span) {
      const int i2 = u & (P - 1);
      const int ks = i2 & (sl - 1);
      if (ks == 0) {
        if (i2 == 0) lor_zero<ORDER, L0, L1>(h);
        if (!kDecomp) {
          if (i2 == 0) cg = gB;
          cv[0] = n0.x;
          cv[1] = n0.y;
          cv[2] = n0.z;
          cv[3] = n0.w;
          cv[4] = n1.x;
          cv[5] = n1.y;
          cv[6] = n1.z;
          cv[7] = n1.w;
          if (u + sl < span) {
            const int i2f = (u + sl) & (P - 1);
            if (i2f == 0) {
              walk_next(G, wk);
              gB = col_geo(G, wk, i0, i1);
            }
            load_x<kVec>(n0, n1, x, gB, i2f, sl);
          }
        } else {
          if (i2 == 0) cg = gB;
          cc = cB;
          if (u + sl < span) {
            const int i2b = (u + sl) & (P - 1);
            gB = gA;
            cB = pack_codes<kVec>(cA, rA);
#pragma unroll
            for (int k = 0; k < kSeg; ++k)
              if (i2b + k < gB.m2 &&
                  ((((k & 1) ? (&cB.x)[k / 2] >> 16 : (&cB.x)[k / 2]) & 0xFFFFu) == 0u))
                prefetch_l1(out + gB.col + (uint32_t)(i2b + k));
            if (u + 2 * sl < span) {
              const int i2a = (u + 2 * sl) & (P - 1);
              if (i2a == 0) {
                walk_next(G, wk);
                gA = col_geo(G, wk, i0, i1);
              }
              load_codes<kVec>(cA, rA, codes, gA, i2a, sl);
            }
          }
        }
      }
      const bool act = i2 < cg.m2;
      float rec = 0.0f;
      if (act) {
        float v0[L0 + 1][L1 + 1];
        const float acc =
            lor_predict<ORDER, L0, L1, HD, RING>(mine, tau, (int)G.slot, W, i2, h, v0);
        const uint32_t fi = cg.col + (uint32_t)i2;
        if (!kDecomp) {
          const unsigned code = quantize_fast(cv[0], acc, e, inv2, twoe, rec);
          if (kVec) {
#pragma unroll
            for (int k = 0; k < kSeg / 2 - 1; ++k) pk[k] = __funnelshift_r(pk[k], pk[k + 1], 16);
            pk[kSeg / 2 - 1] = (pk[kSeg / 2 - 1] >> 16) | (code << 16);
            if (ks == kSeg - 1)
              *reinterpret_cast<uint4*>(codes + fi - (kSeg - 1)) =
                  make_uint4(pk[0], pk[1], pk[2], pk[3]);
          } else {
            codes[fi] = (uint16_t)code;
          }
        } else {
          const unsigned code = cc.x & 0xFFFFu;
          rec = code ? dequantize(code, acc, twoe) : out[fi];
          if (!kVec) out[fi] = rec;
        }
        mine[(tau & (RING - 1)) * (int)G.slot] = rec;
        lor_shift<ORDER, L0, L1, HD>(h, v0, rec);
      }
      // advance the segment cursor
      if (!kDecomp) {
#pragma unroll
        for (int k = 0; k < kSeg - 1; ++k) cv[k] = cv[k + 1];
      } else {
        cc.x = __funnelshift_r(cc.x, cc.y, 16);
        cc.y = __funnelshift_r(cc.y, cc.z, 16);
        cc.z = __funnelshift_r(cc.z, cc.w, 16);
        cc.w >>= 16;
        if (kVec) {
#pragma unroll
          for (int k = 0; k < kSeg - 1; ++k) ov[k] = ov[k + 1];
          ov[kSeg - 1] = rec;
          if (act && ks == kSeg - 1) {
            float4* o4 = reinterpret_cast<float4*>(out + cg.col + (uint32_t)(i2 - (kSeg - 1)));
            o4[0] = make_float4(ov[0], ov[1], ov[2], ov[3]);
            o4[1] = make_float4(ov[4], ov[5], ov[6], ov[7]);
          }
        }
      }
    }
    __syncthreads();
  }
}

template <bool kDecomp, int ORDER, int NDR, bool kVec, bool kSkew>
__global__ void __launch_bounds__(1024, 1)
    k_lorenzo(LorGeom G, const float* __restrict__ x, uint16_t* __restrict__ codes,
              float* __restrict__ out, const Ctl* __restrict__ ctl) {
  lor_body<kDecomp, ORDER, NDR, kVec, kSkew>(G, x, codes, out, ctl, blockIdx.x, gridDim.x);
}

// batched: job j owns the persistent CTAs [off[j], off[j+1]) of the launch
// (its G.g is that CTA count in the radix of its blocks)
template <bool kDecomp, int ORDER, int NDR, bool kVec, bool kSkew>
__global__ void __launch_bounds__(1024, 1)
    k_lorenzo_batch(const LorenzoJob* __restrict__ J, const uint32_t* __restrict__ off, int nj) {
  const int j = batch_job(off, nj);
  const LorenzoJob& q = J[j];
  const uint32_t o = __ldg(off + j);
  lor_body<kDecomp, ORDER, NDR, kVec, kSkew>(q.G, q.x, q.codes, q.out, q.ctl, blockIdx.x - o,
                                             __ldg(off + j + 1) - o);
}

// The 3D, A = 32 form fed by TMA.  Warp w owns the columns (w, 0..31) of
// its CTA's blocks (lane l: i1 = l, so s = w + l) and reads its input from
// tensor boxes of 8 columns x 32 rows of plane w (segment m of its stream:
// block m / 4, columns 8 (m mod 4)..+8): one copy per warp and segment
// instead of a load per row.  Lane l uses segment m at steps w + 8m + l ..
// +7, so a box lives for 39 steps: the warp keeps kNB boxes in a ring and
// fetches kLead segments ahead (compress: 6 boxes, the next segment;
// decompress: 7 boxes of codes, two segments ahead, so that the escaped
// values of a segment are prefetched into L1 from its landed codes).  At
// step w + 8m the warp waits for the box it fetched at the previous
// event and fetches the next into the buffer of segment m + kLead - kNB,
// which its last lane left two steps before.
template <bool kDecomp>
struct LorBox {
  static constexpr int kNB = kDecomp ? 7 : 6;
  static constexpr int kLead = kDecomp ? 2 : 1;
  static constexpr uint32_t kBytes = 32u * kSeg * (kDecomp ? 2u : 4u);
  static constexpr uint32_t kStride = kBytes;  // 128-byte aligned (tensor copy destinations)
  static constexpr uint32_t kWarp = kNB * kStride;
  static_assert(kStride % 128u == 0u, "box buffers must stay 128-byte aligned");
};

template <bool kDecomp, int ORDER>
__global__ void __launch_bounds__(1024, 1)
    k_lorenzo_tma(const __grid_constant__ CUtensorMap tm, LorGeom G, uint16_t* __restrict__ codes,
                  float* __restrict__ out, Ctl* __restrict__ ctl, uint32_t ring_bytes,
                  int drop) {
  using BX = LorBox<kDecomp>;
  __shared__ int s_skip;
  __shared__ float s_inv2;
  if (threadIdx.x == 0) s_skip = ctl->status || ctl->is_const;
  __syncthreads();
  if (s_skip) return;  // read once: another CTA may set the status meanwhile
  constexpr int RING = lor_ring<ORDER>();
  constexpr int L0 = ORDER, L1 = ORDER;
  constexpr int HD = ORDER == 2 ? 1 : ORDER;
  extern __shared__ __align__(128) unsigned char lsm[];
  float* const ring = reinterpret_cast<float*>(lsm);
  for (uint32_t i = threadIdx.x; i < RING * G.slot; i += blockDim.x) ring[i] = 0.0f;
  const int q = (int)threadIdx.x, lane = q & 31, w = q >> 5;
  const int i0 = w, i1 = lane, s = i0 + i1;
  unsigned char* const boxes = lsm + ring_bytes + (uint32_t)w * BX::kWarp;
  uint64_t* const bar = reinterpret_cast<uint64_t*>(lsm + ring_bytes + 32u * BX::kWarp) + w;
  // the warp's last two blocks: field index of (o0, o1, o2) and the
  // extents m0, m1, m2, written when the warp fetches a block's first box
  // (a lane reaches that block at least 8 steps later, and the entry is
  // rewritten only after every lane has left the block)
  __shared__ uint4 s_blk[32][2];
  if (lane == 0) mbar_init(bar);
  const uint32_t J = (G.nblocks - 1u - blockIdx.x) / gridDim.x + 1u;
  const int span = 32 * (int)J, nseg = 4 * (int)J;
  const int T = span + 62;
  const int W = (int)G.W;
  float* const mine = ring + (i0 + 2) * W + i1 + 2;
  const float e = ctl->e;
  if (threadIdx.x == 0) s_inv2 = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(2.0, (double)e)));
  const float twoe = __fmul_rn(2.0f, e);
  __syncthreads();
  const float inv2 = s_inv2;

  // the warp's box walk (block of the next segment to fetch)
  Walk wb = walk_start(G, blockIdx.x);
  const uint32_t lane_off = (uint32_t)i0 * G.st[0] + (uint32_t)i1 * G.st[1];
  ColGeo cg;
  cg.col = 0u;
  cg.m2 = 0;
  int nf = 0;        // segments fetched by this warp
  uint32_t nw = 0;   // fetches waited for
  bool fail = false;
  auto fetch = [&]() {  // warp-uniform: the next segment nf into its buffer
    if (nf >= nseg) return false;
    if (nf > 0 && (nf & 3) == 0) walk_next(G, wb);
    if (lane == 0 && (nf & 3) == 0) {
      const uint32_t o0 = wb.b0 * 32u, o1 = wb.b1 * 32u, o2 = wb.b2 * 32u;
      s_blk[w][(nf >> 2) & 1] =
          make_uint4(o0 * G.st[0] + o1 * G.st[1] + o2, min(32u, G.n[0] - o0),
                     min(32u, G.n[1] - o1), min(32u, G.n[2] - o2));
    }
    // drop > 0 (a test of the bounded waits): warp 0 of CTA 0 leaves out its
    // fetch drop - 1, whose wait then expires
    if (lane == 0 && !(drop > 0 && blockIdx.x == 0 && w == 0 && nf + 1 == drop)) {
      unsigned char* dst = boxes + (uint32_t)(nf % BX::kNB) * BX::kStride;
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_expect_tx(bar, BX::kBytes);
      tma_load_3d(dst, &tm, bar, (int)(wb.b2 * 32u) + 8 * (nf & 3), (int)(wb.b1 * 32u),
                  (int)(wb.b0 * 32u) + w);
    }
    ++nf;
    return true;
  };
  // this lane's column in the block of table entry t
  auto geo_of = [&](int t) {
    __syncwarp();
    const uint4 b = s_blk[w][t];
    ColGeo g;
    const bool in = (uint32_t)i0 < b.y && (uint32_t)i1 < b.z;
    g.m2 = in ? (int)b.w : 0;
    g.col = b.x + lane_off;
    return g;
  };
  // decompress: L1 prefetch of the escaped values of segment m (landed)
  auto escapes = [&](int m) {
    if (m >= nseg) return;
    const uint4 v = *reinterpret_cast<const uint4*>(
        boxes + (uint32_t)(m % BX::kNB) * BX::kStride + (uint32_t)lane * 16u);
    const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
    const ColGeo g = geo_of((m >> 2) & 1);
    const int c0 = 8 * (m & 3);
#pragma unroll
    for (int k = 0; k < kSeg; ++k)
      if (((wd[k >> 1] >> (16 * (k & 1))) & 0xFFFFu) == 0u && c0 + k < g.m2)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(out + g.col + (uint32_t)(c0 + k)));
  };
  if (fetch()) {
    if (kDecomp) {
      fail = !mbar_wait(bar, nw & 1u);
      ++nw;
      if (!fail) {
        escapes(0);
        fetch();
      }
    }
  }
  float h[L0 + 1][L1 + 1][ORDER];
  float ov[kSeg];
  uint32_t pk[kSeg / 2];
#pragma unroll
  for (int k = 0; k < kSeg; ++k) ov[k] = 0.0f;
#pragma unroll
  for (int k = 0; k < kSeg / 2; ++k) pk[k] = 0u;

  int u = -s;
  int bi = 0;  // this lane's box buffer (its segment mod kNB)
  for (int tau = 0; tau < T; ++tau, ++u) {
    const int ev = tau - w;  // lane 0's stream position
    if (!fail && ev >= 0 && (ev & (kSeg - 1)) == 0) {
      const int m = ev >> 3;  // lane 0 starts segment m now
      // the fetch of the previous event (or the prologue) must have landed
      if (m + BX::kLead - 1 < nseg) {
        fail = !mbar_wait(bar, nw & 1u);
        ++nw;
      }
      if (!fail) {
        if (kDecomp) escapes(m + 1);
        fetch();
      }
    }
    if (!fail && u >= 0 && u < span) {
      const int i2 = u & 31, ks = i2 & (kSeg - 1);
      if (ks == 0 && u > 0) bi = bi + 1 == BX::kNB ? 0 : bi + 1;
      if (i2 == 0) {
        const uint4 b = s_blk[w][(u >> 5) & 1];
        const bool in = (uint32_t)i0 < b.y && (uint32_t)i1 < b.z;
        cg.m2 = in ? (int)b.w : 0;
        cg.col = b.x + lane_off;
        lor_zero<ORDER, L0, L1>(h);
      }
      const unsigned char* bp =
          boxes + (uint32_t)bi * BX::kStride + (uint32_t)lane * (BX::kBytes / 32u);
      const bool act = i2 < cg.m2;
      float rec = 0.0f;
      if (act) {
        float v0[L0 + 1][L1 + 1];
        const float acc =
            lor_predict<ORDER, L0, L1, HD, RING>(mine, tau, (int)G.slot, W, i2, h, v0);
        const uint32_t fi = cg.col + (uint32_t)i2;
        if (!kDecomp) {
          const float xv = reinterpret_cast<const float*>(bp)[ks];
          const unsigned code = quantize_fast(xv, acc, e, inv2, twoe, rec);
#pragma unroll
          for (int k = 0; k < kSeg / 2 - 1; ++k) pk[k] = __funnelshift_r(pk[k], pk[k + 1], 16);
          pk[kSeg / 2 - 1] = (pk[kSeg / 2 - 1] >> 16) | (code << 16);
          if (ks == kSeg - 1)
            *reinterpret_cast<uint4*>(codes + fi - (kSeg - 1)) =
                make_uint4(pk[0], pk[1], pk[2], pk[3]);
        } else {
          const unsigned code = reinterpret_cast<const uint16_t*>(bp)[ks];
          rec = code ? dequantize(code, acc, twoe) : out[fi];
        }
        mine[(tau & (RING - 1)) * (int)G.slot] = rec;
        lor_shift<ORDER, L0, L1, HD>(h, v0, rec);
      }
      if (kDecomp) {
#pragma unroll
        for (int k = 0; k < kSeg - 1; ++k) ov[k] = ov[k + 1];
        ov[kSeg - 1] = rec;
        if (act && ks == kSeg - 1) {
          float4* o4 = reinterpret_cast<float4*>(out + cg.col + (uint32_t)(i2 - (kSeg - 1)));
          o4[0] = make_float4(ov[0], ov[1], ov[2], ov[3]);
          o4[1] = make_float4(ov[4], ov[5], ov[6], ov[7]);
        }
      }
    }
    if (__syncthreads_or(fail)) break;
  }
  if (__syncthreads_or(fail)) {
    // a box did not land: record it, then wait (bounded) for this warp's
    // fetch still in flight before leaving
    if (threadIdx.x == 0) atomicCAS(&ctl->status, 0, ST_TIMEOUT);
    if (fail)
      mbar_wait(bar, (nw - 1u) & 1u);
    else if ((uint32_t)nf > nw)
      mbar_wait(bar, nw & 1u);
  }
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

// the field (or its codes) as a 3D tensor, slot 2 fastest, boxes of 8
// columns x 32 rows x 1 plane; out-of-range box elements read 0
bool lor_map(CUtensorMap* map, const void* base, bool u16, const uint32_t n[3]) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t es = u16 ? 2 : 4;
  const cuuint64_t dim[3] = {n[2], n[1], n[0]};
  const cuuint64_t stride[2] = {n[2] * es, (cuuint64_t)n[1] * n[2] * es};
  const cuuint32_t box[3] = {(cuuint32_t)kSeg, 32, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, u16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
            const_cast<void*>(base), dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool lor_geom(const uint32_t n[3], const uint32_t fst[3], int off, int A, int order,
              LorGeom& G, size_t& smem, unsigned& threads) {
  uint64_t nbl = 1;
  for (int d = 0; d < 3; ++d) {
    G.n[d] = n[d];
    G.st[d] = fst[d];
    G.B[d] = d < off ? 1u : (uint32_t)A;
    G.nb[d] = (G.n[d] + G.B[d] - 1) / G.B[d];
    nbl *= G.nb[d];
  }
  if (A < 2 || (A & (A - 1)) != 0 || nbl == 0 || nbl > 0x7FFFFFFFull) return false;
  G.nblocks = (uint32_t)nbl;
  G.logP = 0;
  while ((1 << G.logP) < A) ++G.logP;
  const uint64_t cols = (uint64_t)G.B[0] * G.B[1];
  G.W = G.B[1] >= 32 ? G.B[1] + 2 : G.B[1] + 32;
  G.slot = (G.B[0] + 2) * G.W;
  const int ring = order == 1 ? lor_ring<1>() : lor_ring<2>();
  smem = (size_t)ring * G.slot * sizeof(float);
  if (cols > 1024 || smem > 200 * 1024) return false;
  // the step count P J + B0 + B1 stays far inside int
  if ((uint64_t)A * nbl + cols > 0x3FFFFFFFull) return false;
  threads = (unsigned)((cols + 31) / 32 * 32);
  return true;
}

template <bool kDecomp, int ORDER, int NDR, bool kVec, bool kSkew = false>
int launch_lor_k(const LorGeom& G, size_t smem, unsigned threads, int num_sms,
                 int max_ctas, const float* x, uint16_t* codes, float* out, const Ctl* ctl,
                 cudaStream_t s) {
  auto kern = k_lorenzo<kDecomp, ORDER, NDR, kVec, kSkew>;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  const cudaError_t oe =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)threads, smem);
  if (oe != cudaSuccess || per_sm < 1) {
    if (std::getenv("HPEZ_DEBUG_CUDA"))
      std::fprintf(stderr, "hpez: Lorenzo occupancy %s, %d CTAs per SM (%u threads, %zu B)\n",
                   cudaGetErrorName(oe), per_sm, threads, smem);
    return HPEZ_ERR_CUDA;
  }
  // persistent CTAs, the blocks dealt round robin; the grid shrunk to the
  // fewest CTAs that keep the most loaded one's block count
  uint64_t cap = (uint64_t)per_sm * (uint64_t)(num_sms > 0 ? num_sms : 1);
  if (max_ctas > 0 && cap > (uint64_t)max_ctas) cap = (uint64_t)max_ctas;
  uint64_t grid = G.nblocks < cap ? G.nblocks : cap;
  const uint64_t J = (G.nblocks + grid - 1) / grid;
  grid = (G.nblocks + J - 1) / J;
  LorGeom Gk = G;
  Gk.g[2] = (uint32_t)(grid % G.nb[2]);
  Gk.g[1] = (uint32_t)(grid / G.nb[2] % G.nb[1]);
  Gk.g[0] = (uint32_t)(grid / G.nb[2] / G.nb[1]);
  kern<<<(unsigned)grid, threads, smem, s>>>(Gk, x, codes, out, ctl);
  return HPEZ_OK;
}

// The box-fed kernel when its shared memory fits and the tensor map can be
// made; 1: launched, 0: not taken (use the register-fed kernel), < 0: error.
template <bool kDecomp, int ORDER>
int launch_lor_tma(const LorGeom& G, int num_sms, int max_ctas, const float* x, uint16_t* codes,
                   float* out, Ctl* ctl, int drop, cudaStream_t s) {
  using BX = LorBox<kDecomp>;
  auto kern = k_lorenzo_tma<kDecomp, ORDER>;
  const uint32_t ring_bytes =
      (uint32_t)(((size_t)lor_ring<ORDER>() * G.slot * sizeof(float) + 127) / 128 * 128);
  const size_t smem = ring_bytes + 32u * BX::kWarp + 32u * sizeof(uint64_t);
  if (smem > 220u * 1024u) return 0;
  CUtensorMap tm;
  if (!lor_map(&tm, kDecomp ? static_cast<const void*>(codes) : static_cast<const void*>(x),
               kDecomp, G.n))
    return 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return HPEZ_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 1024, smem) != cudaSuccess ||
      per_sm < 1)
    return HPEZ_ERR_CUDA;
  uint64_t cap = (uint64_t)per_sm * (uint64_t)(num_sms > 0 ? num_sms : 1);
  if (max_ctas > 0 && cap > (uint64_t)max_ctas) cap = (uint64_t)max_ctas;
  uint64_t grid = G.nblocks < cap ? G.nblocks : cap;
  const uint64_t J = (G.nblocks + grid - 1) / grid;
  grid = (G.nblocks + J - 1) / J;
  LorGeom Gk = G;
  Gk.g[2] = (uint32_t)(grid % G.nb[2]);
  Gk.g[1] = (uint32_t)(grid / G.nb[2] % G.nb[1]);
  Gk.g[0] = (uint32_t)(grid / G.nb[2] / G.nb[1]);
  kern<<<(unsigned)grid, 1024, smem, s>>>(tm, Gk, codes, out, ctl, ring_bytes, drop);
  return 1;
}

template <bool kDecomp, int ORDER>
int launch_lor_nd(int ndr, bool vec, const LorGeom& G, size_t smem, unsigned threads,
                  int num_sms, int max_ctas, const float* x, uint16_t* codes, float* out,
                  const Ctl* ctl, int drop, cudaStream_t s) {
  // order 1 takes the box-fed kernel (order 2: no faster measured, and the
  // compressor's shared memory would not fit)
  if (ORDER == 1 && ndr == 3 && G.B[0] == 32 && G.B[1] == 32 && vec) {
    const int r =
        launch_lor_tma<kDecomp, ORDER>(G, num_sms, max_ctas, x, codes, out, const_cast<Ctl*>(ctl), drop, s);
    if (r != 0) return r < 0 ? r : HPEZ_OK;
  }
  if (ndr == 3 && G.B[0] == 32 && G.B[1] == 32)
    return vec ? launch_lor_k<kDecomp, ORDER, 3, true, true>(G, smem, threads, num_sms, max_ctas, x, codes, out, ctl, s)
               : launch_lor_k<kDecomp, ORDER, 3, false, true>(G, smem, threads, num_sms, max_ctas, x, codes, out, ctl, s);
  if (ndr == 3)
    return vec ? launch_lor_k<kDecomp, ORDER, 3, true>(G, smem, threads, num_sms, max_ctas, x, codes, out, ctl, s)
               : launch_lor_k<kDecomp, ORDER, 3, false>(G, smem, threads, num_sms, max_ctas, x, codes, out, ctl, s);
  if (ndr == 2)
    return vec ? launch_lor_k<kDecomp, ORDER, 2, true>(G, smem, threads, num_sms, max_ctas, x, codes, out, ctl, s)
               : launch_lor_k<kDecomp, ORDER, 2, false>(G, smem, threads, num_sms, max_ctas, x, codes, out, ctl, s);
  return vec ? launch_lor_k<kDecomp, ORDER, 1, true>(G, smem, threads, num_sms, max_ctas, x, codes, out, ctl, s)
             : launch_lor_k<kDecomp, ORDER, 1, false>(G, smem, threads, num_sms, max_ctas, x, codes, out, ctl, s);
}

}  // namespace

bool lorenzo_supported(const uint32_t n[3], const uint32_t fst[3], int off, int A) {
  LorGeom G;
  size_t smem;
  unsigned threads;
  return lor_geom(n, fst, off, A, 2, G, smem, threads);
}

// The Lorenzo pass over the field (slots n, strides fst, off padded slots,
// block side A): compress (x -> codes) or decompress (codes, the escaped
// values already scattered into out -> out).  vec: rows start on 16-byte
// boundaries (n[2] a multiple of 8 and the float buffer 16-byte aligned;
// taken when A >= 8).
// drop_copy: see HPEZ_OPT_DROP_COPY (0 in normal use); max_ctas > 0 caps
// the persistent grid (HPEZ_OPT_LORENZO_CTAS), so each CTA streams more
// blocks.  Returns
// HPEZ_ERR_UNSUPPORTED for geometries the kernel does not take.
int launch_lorenzo(bool decomp, int order, const uint32_t n[3], const uint32_t fst[3],
                   int off, int A, bool vec, const float* x, uint16_t* codes, float* out,
                   const Ctl* ctl, int num_sms, int drop_copy, int max_ctas,
                   cudaStream_t s) {
  LorGeom G;
  size_t smem;
  unsigned threads;
  if (order < 1 || order > 2 || !lor_geom(n, fst, off, A, order, G, smem, threads))
    return HPEZ_ERR_UNSUPPORTED;
  vec = vec && (n[2] % kSeg) == 0 && A >= kSeg;
  const int ndr = 3 - off;
  if (decomp)
    return order == 1 ? launch_lor_nd<true, 1>(ndr, vec, G, smem, threads, num_sms, max_ctas, x, codes, out, ctl, drop_copy, s)
                      : launch_lor_nd<true, 2>(ndr, vec, G, smem, threads, num_sms, max_ctas, x, codes, out, ctl, drop_copy, s);
  return order == 1 ? launch_lor_nd<false, 1>(ndr, vec, G, smem, threads, num_sms, max_ctas, x, codes, out, ctl, drop_copy, s)
                    : launch_lor_nd<false, 2>(ndr, vec, G, smem, threads, num_sms, max_ctas, x, codes, out, ctl, drop_copy, s);
}

// ---------------------------------------------------------------------
// batched form: the register-fed kernel with one job table per launch.  A
// launch's jobs share the template (direction, order, real dimensions, row
// vectors, skewed lane map) and the CTA size, which the op variant encodes:
// variant = ((((decomp 2 + order - 1) 3 + ndr - 1) 2 + vec) 2 + skew) 6 +
// log2(threads / 32).
// ---------------------------------------------------------------------
namespace {

template <class F>
struct LorDispatch {
  template <bool D, int O>
  static void by_shape(int ndr, bool vec, bool skew, F& f) {
    if (ndr == 3 && skew) {
      if (vec) f.template run<D, O, 3, true, true>(); else f.template run<D, O, 3, false, true>();
    } else if (ndr == 3) {
      if (vec) f.template run<D, O, 3, true, false>(); else f.template run<D, O, 3, false, false>();
    } else if (ndr == 2) {
      if (vec) f.template run<D, O, 2, true, false>(); else f.template run<D, O, 2, false, false>();
    } else {
      if (vec) f.template run<D, O, 1, true, false>(); else f.template run<D, O, 1, false, false>();
    }
  }
  static void go(bool decomp, int order, int ndr, bool vec, bool skew, F& f) {
    if (decomp) {
      if (order == 1) by_shape<true, 1>(ndr, vec, skew, f); else by_shape<true, 2>(ndr, vec, skew, f);
    } else {
      if (order == 1) by_shape<false, 1>(ndr, vec, skew, f); else by_shape<false, 2>(ndr, vec, skew, f);
    }
  }
};

struct LorOcc {
  unsigned threads;
  size_t smem;
  int per_sm = 0;
  template <bool D, int O, int N, bool V, bool S>
  void run() {
    auto k = k_lorenzo_batch<D, O, N, V, S>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)threads, smem) !=
        cudaSuccess) {
      cudaGetLastError();
      per_sm = 0;
    }
  }
};

struct LorLaunch {
  const LorenzoJob* J;
  const uint32_t* off;
  int nj;
  uint32_t nblk;
  unsigned threads;
  size_t smem;
  cudaStream_t s;
  template <bool D, int O, int N, bool V, bool S>
  void run() {
    auto k = k_lorenzo_batch<D, O, N, V, S>;
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr = true;
    }
    k<<<nblk, threads, smem, s>>>(J, off, nj);
  }
};

}  // namespace

bool lorenzo_batch_job(bool decomp, int order, const uint32_t n[3], const uint32_t fst[3],
                       int off, int A, bool vec, int num_sms, int max_ctas, LorGeom* Gout,
                       int* variant, uint32_t* ctas, size_t* smem_out) {
  LorGeom G;
  size_t smem;
  unsigned threads;
  if (order < 1 || order > 2 || !lor_geom(n, fst, off, A, order, G, smem, threads)) return false;
  vec = vec && (n[2] % kSeg) == 0 && A >= kSeg;
  const int ndr = 3 - off;
  const bool skew = ndr == 3 && G.B[0] == 32 && G.B[1] == 32;
  LorOcc occ;
  occ.threads = threads;
  occ.smem = smem;
  LorDispatch<LorOcc>::go(decomp, order, ndr, vec, skew, occ);
  if (occ.per_sm < 1) return false;
  uint64_t cap = (uint64_t)occ.per_sm * (uint64_t)(num_sms > 0 ? num_sms : 1);
  if (max_ctas > 0 && cap > (uint64_t)max_ctas) cap = (uint64_t)max_ctas;
  uint64_t grid = G.nblocks < cap ? G.nblocks : cap;
  const uint64_t J = (G.nblocks + grid - 1) / grid;
  grid = (G.nblocks + J - 1) / J;
  G.g[2] = (uint32_t)(grid % G.nb[2]);
  G.g[1] = (uint32_t)(grid / G.nb[2] % G.nb[1]);
  G.g[0] = (uint32_t)(grid / G.nb[2] / G.nb[1]);
  int tcls = 0;
  while ((32u << tcls) < threads) ++tcls;
  *Gout = G;
  *variant = (((((decomp ? 1 : 0) * 2 + order - 1) * 3 + ndr - 1) * 2 + (vec ? 1 : 0)) * 2 +
              (skew ? 1 : 0)) * 6 + tcls;
  *ctas = (uint32_t)grid;
  *smem_out = smem;
  return true;
}

void launch_lorenzo_batch(int variant, const LorenzoJob* J, const uint32_t* off, int nj,
                          uint32_t nblk, size_t smem, cudaStream_t s) {
  if (!nblk || variant < 0 || variant >= kLorVariants) return;
  int v = variant;
  const int tcls = v % 6;
  v /= 6;
  const bool skew = v % 2;
  v /= 2;
  const bool vec = v % 2;
  v /= 2;
  const int ndr = v % 3 + 1;
  v /= 3;
  const int order = v % 2 + 1;
  const bool decomp = v / 2;
  LorLaunch L{J, off, nj, nblk, 32u << tcls, smem, s};
  LorDispatch<LorLaunch>::go(decomp, order, ndr, vec, skew, L);
}

}  // namespace hpez
