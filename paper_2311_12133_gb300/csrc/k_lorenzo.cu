// k_lorenzo.cu -- the Lorenzo predictor over the whole field (Sec. 6.5:
// the dynamic-order predictor, order 1 or 2, that the tuner selects when
// its estimate beats interpolation), read as block-local: the field is cut
// into blocks of side A along every dimension, and inside a block a point
// is predicted from the reconstructed points of its block (a neighbour
// outside the block reads 0) -- the recurrence the tuner's Lorenzo test
// runs on its sample blocks.
//
// A CTA owns one block with the block's reconstruction in shared memory
// and runs the recurrence as a wavefront over the planes i0 + i1 + i2 = t:
// every neighbour a point reads lies on an earlier plane.  A thread owns
// one (i0, i1) column of the block; the input of its next point (the field
// value, or the code) is loaded while the current plane is computed.
#include "hpez.h"
#include "hpez_internal.cuh"
#include "hpez_launch.h"

namespace hpez {
namespace {

struct LorGeom {
  uint32_t n[3];    // field extents per slot (padded slots 1)
  uint32_t st[3];   // field strides
  uint32_t B[3];    // block side per slot (1 on padded slots)
  uint32_t nb[3];   // blocks per slot
  int lim[3];       // stencil reach per slot: the order, 0 on padded slots
};

// per-dimension coefficient of offset a: order 1 (1, -1), order 2
// (1, -2, 1); a term's weight is minus the product over the three slots
template <int ORDER>
__device__ __forceinline__ float lor_coef(int a) {
  return ORDER == 1 ? (a == 0 ? 1.0f : -1.0f) : (a == 1 ? -2.0f : 1.0f);
}

__host__ __device__ __forceinline__ uint32_t lor_row(uint32_t m2) { return m2 + (m2 & 1u); }

template <bool kDecomp, int ORDER>
__global__ void __launch_bounds__(1024)
    k_lorenzo(LorGeom G, const float* __restrict__ x, uint16_t* __restrict__ codes,
              float* __restrict__ out, const Ctl* __restrict__ ctl) {
  if (ctl->status || ctl->is_const) return;
  extern __shared__ float R[];
  unsigned b = blockIdx.x;
  uint32_t o[3], m[3];
  for (int d = 2; d >= 0; --d) {
    const uint32_t j = b % G.nb[d];
    b /= G.nb[d];
    o[d] = j * G.B[d];
    m[d] = min(G.B[d], G.n[d] - o[d]);
  }
  const uint32_t m2p = lor_row(m[2]);
  const float e = ctl->e;
  const float inv2 = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(2.0, (double)e)));
  const float twoe = __fmul_rn(2.0f, e);
  const int q = (int)threadIdx.x;
  const bool mine = (uint32_t)q < m[0] * m[1];
  const int i0 = mine ? q / (int)m[1] : 0, i1 = mine ? q - i0 * (int)m[1] : 0;
  const uint32_t col = (o[0] + (uint32_t)i0) * G.st[0] + (o[1] + (uint32_t)i1) * G.st[1] + o[2];
  const int T = (int)(m[0] - 1) + (int)(m[1] - 1) + (int)(m[2] - 1);
  auto load = [&](int t) -> float {
    const int i2 = t - i0 - i1;
    if (!mine || i2 < 0 || i2 >= (int)m[2]) return 0.0f;
    if (kDecomp) return __uint_as_float((uint32_t)codes[col + (uint32_t)i2]);
    return __ldg(x + col + (uint32_t)i2);
  };
  float cur = load(0);
  for (int t = 0; t <= T; ++t) {
    const float nxt = t < T ? load(t + 1) : 0.0f;
    const int i2 = t - i0 - i1;
    if (mine && i2 >= 0 && i2 < (int)m[2]) {
      const int base = (i0 * (int)m[1] + i1) * (int)m2p + i2;
      float acc = 0.0f;
#pragma unroll
      for (int a = 0; a <= ORDER; ++a)
#pragma unroll
        for (int bb = 0; bb <= ORDER; ++bb)
#pragma unroll
          for (int c = 0; c <= ORDER; ++c) {
            if (a == 0 && bb == 0 && c == 0) continue;
            if (a > G.lim[0] || bb > G.lim[1] || c > G.lim[2]) continue;
            const float w = -__fmul_rn(__fmul_rn(lor_coef<ORDER>(a), lor_coef<ORDER>(bb)),
                                       lor_coef<ORDER>(c));
            float v = 0.0f;
            if (a <= i0 && bb <= i1 && c <= i2) v = R[base - (a * (int)m[1] + bb) * (int)m2p - c];
            acc = __fadd_rn(acc, __fmul_rn(w, v));
          }
      const uint32_t fi = col + (uint32_t)i2;
      float rec;
      if (!kDecomp) {
        const unsigned code = quantize(cur, acc, e, inv2, twoe, rec);
        codes[fi] = (uint16_t)code;
      } else {
        const unsigned code = __float_as_uint(cur);
        rec = code ? dequantize(code, acc, twoe) : out[fi];
        out[fi] = rec;
      }
      R[base] = rec;
    }
    __syncthreads();
    cur = nxt;
  }
}

bool lor_geom(const uint32_t n[3], const uint32_t fst[3], int off, int A, LorGeom& G,
              size_t& smem, unsigned& threads) {
  for (int d = 0; d < 3; ++d) {
    G.n[d] = n[d];
    G.st[d] = fst[d];
    G.B[d] = d < off ? 1u : (uint32_t)A;
    G.nb[d] = (G.n[d] + G.B[d] - 1) / G.B[d];
    G.lim[d] = 0;
  }
  const uint64_t pairs = (uint64_t)G.B[0] * G.B[1];
  smem = (size_t)G.B[0] * G.B[1] * lor_row(G.B[2]) * sizeof(float);
  if (pairs > 1024 || smem > 200 * 1024) return false;
  threads = (unsigned)((pairs + 31) / 32 * 32);
  return true;
}

template <bool kDecomp, int ORDER>
void launch_lor_k(const LorGeom& G, size_t smem, unsigned threads, const float* x,
                  uint16_t* codes, float* out, const Ctl* ctl, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_lorenzo<kDecomp, ORDER>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const unsigned nblk = G.nb[0] * G.nb[1] * G.nb[2];
  k_lorenzo<kDecomp, ORDER><<<nblk, threads, smem, s>>>(G, x, codes, out, ctl);
}

}  // namespace

bool lorenzo_supported(const uint32_t n[3], const uint32_t fst[3], int off, int A) {
  LorGeom G;
  size_t smem;
  unsigned threads;
  return lor_geom(n, fst, off, A, G, smem, threads);
}

// The Lorenzo pass over the field (slots n, strides fst, off padded slots,
// block side A): compress (x -> codes) or decompress (codes, the outliers
// already scattered into out -> out).  Returns HPEZ_ERR_UNSUPPORTED when a
// block's shared-memory image or its columns do not fit a CTA.
int launch_lorenzo(bool decomp, int order, const uint32_t n[3], const uint32_t fst[3],
                   int off, int A, const float* x, uint16_t* codes, float* out,
                   const Ctl* ctl, cudaStream_t s) {
  LorGeom G;
  size_t smem;
  unsigned threads;
  if (!lor_geom(n, fst, off, A, G, smem, threads) || order < 1 || order > 2)
    return HPEZ_ERR_UNSUPPORTED;
  for (int d = 0; d < 3; ++d) G.lim[d] = d < off ? 0 : order;
  if (decomp) {
    if (order == 1) launch_lor_k<true, 1>(G, smem, threads, x, codes, out, ctl, s);
    else launch_lor_k<true, 2>(G, smem, threads, x, codes, out, ctl, s);
  } else {
    if (order == 1) launch_lor_k<false, 1>(G, smem, threads, x, codes, out, ctl, s);
    else launch_lor_k<false, 2>(G, smem, threads, x, codes, out, ctl, s);
  }
  return HPEZ_OK;
}

}  // namespace hpez
