// k_sweep.cu -- value range, level parameters, anchors and the level-wise
// interpolation predict-and-quantize sweep (compress and decompress).
//
// Sec. 5.1: anchors at stride A are stored verbatim; levels l = L..1 use
// stride s = 2^(l-1) and predict the points of the stride-s grid that are
// not on the stride-2s grid from already reconstructed points.  Each level
// works on a compact copy of its grid (G_s), so every level -- not only the
// finest -- reads and writes densely packed memory.
#include "hpez_internal.cuh"
#include "hpez_launch.h"

#include <cfloat>

namespace hpez {

// ---------------------------------------------------------------------
// control block init + value range (Sec. 7.1.3: e = eps * (max - min))
// ---------------------------------------------------------------------
__device__ __forceinline__ void init_ctl_body(Ctl* ctl) {
  unsigned* p = reinterpret_cast<unsigned*>(ctl);
  for (int i = threadIdx.x; i < (int)(sizeof(Ctl) / 4); i += blockDim.x)
    p[i] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->vmin_key = 0xFFFFFFFFu;
    ctl->vmax_key = 0u;
  }
}

__global__ void k_init_ctl(Ctl* ctl) { init_ctl_body(ctl); }

// the value range found by an earlier pass over the same input
__global__ void k_set_range(Ctl* ctl, unsigned kmin, unsigned kmax) {
  ctl->vmin_key = kmin;
  ctl->vmax_key = kmax;
}

__device__ __forceinline__ void range_body(const float* __restrict__ x,
                                           uint32_t N, Ctl* ctl, unsigned bid,
                                           unsigned nblk) {
  float mn = FLT_MAX, mx = -FLT_MAX;
  int bad = 0;
  const uint32_t tid = bid * blockDim.x + threadIdx.x;
  const uint32_t nthr = nblk * blockDim.x;
  const bool vec = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
  uint32_t done = 0;
  if (vec) {
    const uint32_t n4 = N / 4;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (uint32_t i = tid; i < n4; i += nthr) {
      float4 v = __ldcs(x4 + i);
      bad |= !isfinite(v.x) | !isfinite(v.y) | !isfinite(v.z) | !isfinite(v.w);
      mn = fminf(fminf(mn, v.x), fminf(v.y, fminf(v.z, v.w)));
      mx = fmaxf(fmaxf(mx, v.x), fmaxf(v.y, fmaxf(v.z, v.w)));
    }
    done = n4 * 4;
  }
  for (uint32_t i = done + tid; i < N; i += nthr) {
    float v = x[i];
    bad |= !isfinite(v);
    mn = fminf(mn, v);
    mx = fmaxf(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  __shared__ float smn[32], smx[32];
  __shared__ int sbad[32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    smn[w] = mn;
    smx[w] = mx;
    sbad[w] = bad;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    mn = lane < nw ? smn[lane] : FLT_MAX;
    mx = lane < nw ? smx[lane] : -FLT_MAX;
    bad = lane < nw ? sbad[lane] : 0;
    for (int o = 16; o > 0; o >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
      atomicMin(&ctl->vmin_key, f2key(mn));
      atomicMax(&ctl->vmax_key, f2key(mx));
      if (bad) atomicOr(&ctl->nonfinite, 1);
    }
  }
}

__global__ void __launch_bounds__(256) k_range(const float* __restrict__ x,
                                               uint32_t N, Ctl* ctl) {
  range_body(x, N, ctl, blockIdx.x, gridDim.x);
}

// Level parameters in IEEE double, one rounding to binary32 each (Eq. 15):
// e_l = e / min(alpha^(l-1), beta), alpha^(l-1) by repeated multiplication;
// inv2_l = 1 / (2 e_l); twoe_l = 2 e_l.
__device__ __forceinline__ void params_body(Ctl* ctl, int eb_mode, double eb,
                                            double alpha, double beta, int L,
                                            const float* __restrict__ x) {
  if (threadIdx.x != 0) return;
  float e;
  if (eb_mode == 1) {
    if (ctl->nonfinite) {
      ctl->status = ST_NONFINITE;
      return;
    }
    const float vmin = key2f(ctl->vmin_key), vmax = key2f(ctl->vmax_key);
    const double range = __dsub_rn((double)vmax, (double)vmin);
    if (range == 0.0) {
      ctl->is_const = 1;
      ctl->const_value = x[0];
      return;
    }
    e = __double2float_rn(__dmul_rn(eb, range));
  } else {
    e = __double2float_rn(eb);
  }
  if (!(e > 0.0f) || !isfinite(e)) {
    ctl->status = ST_INVALID;
    return;
  }
  ctl->e = e;
  for (int l = 1; l <= L; ++l) {
    double ap = 1.0;
    for (int i = 1; i < l; ++i) ap = __dmul_rn(ap, alpha);
    const double m = ap < beta ? ap : beta;
    const float el = __double2float_rn(__ddiv_rn((double)e, m));
    const float t = __fmul_rn(2.0f, el);
    if (!(el > 0.0f) || !isfinite(el) || !isfinite(t)) {
      ctl->status = ST_INVALID;
      return;
    }
    ctl->el[l - 1] = el;
    ctl->twoe[l - 1] = t;
    ctl->inv2[l - 1] = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(2.0, (double)el)));
  }
}

__global__ void k_params(Ctl* ctl, int eb_mode, double eb, double alpha,
                         double beta, int L, const float* __restrict__ x) {
  if (blockIdx.x != 0) return;
  params_body(ctl, eb_mode, eb, alpha, beta, L, x);
}

// ---------------------------------------------------------------------
// anchors: G_A <- x (compress) ; G_A <- stored anchors (decompress)
// ---------------------------------------------------------------------
__device__ __forceinline__ void anchor_body(const float* __restrict__ x,
                                            const LevelGeom& ga, uint32_t total,
                                            float* __restrict__ RA,
                                            uint16_t* __restrict__ CA,
                                            const Ctl* __restrict__ ctl,
                                            unsigned bid, unsigned nblk) {
  if (ctl->status || ctl->is_const) return;
  for (uint32_t t = bid * blockDim.x + threadIdx.x; t < total;
       t += nblk * blockDim.x) {
    const uint32_t u2 = t % ga.m[2];
    const uint32_t r = t / ga.m[2];
    const uint32_t u1 = r % ga.m[1];
    const uint32_t u0 = r / ga.m[1];
    const uint32_t fi = u0 * ga.step[0] * ga.fst[0] +
                        u1 * ga.step[1] * ga.fst[1] + u2 * ga.step[2];
    RA[t] = x[fi];
    if (CA) CA[t] = (uint16_t)kRadius;
  }
}

__global__ void k_anchor_gather(const float* __restrict__ x, LevelGeom ga,
                                uint32_t total, float* __restrict__ RA,
                                uint16_t* __restrict__ CA,
                                const Ctl* __restrict__ ctl) {
  anchor_body(x, ga, total, RA, CA, ctl, blockIdx.x, gridDim.x);
}

// G_2s -> G_s: coarse points keep their reconstruction (and code).
__device__ __forceinline__ void upsample_body(
    const LevelGeom& gc, uint32_t total_c, const LevelGeom& gs,
    const float* __restrict__ Rc, const uint16_t* __restrict__ Cc,
    float* __restrict__ Rs, uint16_t* __restrict__ Cs,
    const Ctl* __restrict__ ctl, unsigned bid, unsigned nblk) {
  if (ctl->status || ctl->is_const) return;
  for (uint32_t t = bid * blockDim.x + threadIdx.x; t < total_c;
       t += nblk * blockDim.x) {
    const uint32_t v2 = t % gc.m[2];
    const uint32_t r = t / gc.m[2];
    const uint32_t v1 = r % gc.m[1];
    const uint32_t v0 = r / gc.m[1];
    // a slot with step change 2 (interpolation slot) doubles its index
    const uint32_t f0 = gc.step[0] / gs.step[0], f1 = gc.step[1] / gs.step[1],
                   f2 = gc.step[2] / gs.step[2];
    const uint32_t i = v0 * f0 * gs.gst[0] + v1 * f1 * gs.gst[1] + v2 * f2;
    Rs[i] = Rc[t];
    if (Cc) Cs[i] = Cc[t];
  }
}

__global__ void k_upsample(LevelGeom gc, uint32_t total_c, LevelGeom gs,
                           const float* __restrict__ Rc,
                           const uint16_t* __restrict__ Cc,
                           float* __restrict__ Rs, uint16_t* __restrict__ Cs,
                           const Ctl* __restrict__ ctl) {
  upsample_body(gc, total_c, gs, Rc, Cc, Rs, Cs, ctl, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------
// the predict-and-quantize pass (one launch per (pass, half))
// ---------------------------------------------------------------------
template <bool kDecomp>
__device__ __forceinline__ void pass_body(const LevelGeom& g, const PassBox& pb,
                                          const SweepBufs& B, unsigned bid,
                                          unsigned nblk) {
  const Ctl* ctl = B.ctl;
  if (ctl->status || ctl->is_const) return;
  const int li = pb.level - 1;
  const float el = ctl->el[li], inv2 = ctl->inv2[li], twoe = ctl->twoe[li];
  for (uint32_t t = bid * blockDim.x + threadIdx.x; t < pb.total;
       t += nblk * blockDim.x) {
    const uint32_t t2 = t % pb.cnt[2];
    const uint32_t r = t / pb.cnt[2];
    const uint32_t t1 = r % pb.cnt[1];
    const uint32_t t0 = r / pb.cnt[1];
    const uint32_t u[3] = {pb.a[0] + pb.b[0] * t0, pb.a[1] + pb.b[1] * t1,
                           pb.a[2] + pb.b[2] * t2};
    int kind = B.kind, same = B.same;
    if (B.blockmap) {
      uint32_t bi = 0;
      for (int d = 0; d < 3; ++d)
        bi = bi * B.nb[d] + (u[d] * g.step[d]) / B.bs;
      const unsigned v = B.blockmap[bi];
      kind = (int)(v & 3u);
      if (kind > CUBIC_NAT) kind = CUBIC_NAT;
      same = (int)((v >> 2) & 1u);
    }
    if (kind == LINEAR) same = 0;
    // same-level split (Sec. 5.4.2): parity of sum over S of (u_d - 1) / 2
    unsigned par = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (pb.S & (1u << d)) par += (u[d] - 1u) >> 1;
    const int in_b = same && (par & 1u);
    if (in_b != pb.half) continue;
    const uint32_t ci = u[0] * g.gst[0] + u[1] * g.gst[1] + u[2];
    const float* base = B.R + ci;
    float p;
    if (!pb.md) {
      const int d = (pb.S & 1u) ? 0 : ((pb.S & 2u) ? 1 : 2);
      p = predict_line(base, (long long)g.gst[d], (int)u[d], (int)g.m[d],
                       kind, in_b);
    } else {
      // Eq. 8: weighted sum over the odd slots, ascending
      bool first = true;
      p = 0.0f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (!(pb.S & (1u << d))) continue;
        const float pd = predict_line(base, (long long)g.gst[d], (int)u[d],
                                      (int)g.m[d], kind, in_b);
        const float tw = __fmul_rn(pb.w[d], pd);
        p = first ? tw : __fadd_rn(p, tw);
        first = false;
      }
    }
    const uint32_t fi = u[0] * g.step[0] * g.fst[0] +
                        u[1] * g.step[1] * g.fst[1] + u[2] * g.step[2];
    if (!kDecomp) {
      float rec;
      const unsigned code = quantize(B.x[fi], p, el, inv2, twoe, rec);
      B.C[ci] = (uint16_t)code;
      if (pb.write_recon) B.R[ci] = rec;
    } else {
      const unsigned code = B.codes_full[fi];
      B.R[ci] = code ? dequantize(code, p, twoe) : B.outl_full[fi];
    }
  }
}

template <bool kDecomp>
__global__ void __launch_bounds__(256)
    k_pass(LevelGeom g, PassBox pb, SweepBufs B) {
  pass_body<kDecomp>(g, pb, B, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void fill_body(float* __restrict__ out, uint32_t N,
                                          float v, unsigned bid, unsigned nblk) {
  for (uint32_t i = bid * blockDim.x + threadIdx.x; i < N; i += nblk * blockDim.x)
    out[i] = v;
}

__global__ void k_fill(float* __restrict__ out, uint32_t N, float v) {
  fill_body(out, N, v, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------
// batched forms: one launch over the concatenated work of many fields
// ---------------------------------------------------------------------
__global__ void k_init_ctl_batch(const InitJob* __restrict__ J) {
  init_ctl_body(J[blockIdx.x].ctl);
}

__global__ void __launch_bounds__(256)
    k_range_batch(const RangeJob* __restrict__ J, const uint32_t* __restrict__ off,
                  int nj) {
  const int j = batch_job(off, nj);
  range_body(J[j].x, J[j].N, J[j].ctl, blockIdx.x - off[j], off[j + 1] - off[j]);
}

__global__ void k_params_batch(const ParamsJob* __restrict__ J) {
  const ParamsJob& q = J[blockIdx.x];
  params_body(q.ctl, q.eb_mode, q.eb, q.alpha, q.beta, q.L, q.x);
}

__global__ void k_anchor_batch(const AnchorJob* __restrict__ J,
                               const uint32_t* __restrict__ off, int nj) {
  const int j = batch_job(off, nj);
  const AnchorJob& q = J[j];
  anchor_body(q.x, q.ga, q.total, q.RA, q.CA, q.ctl, blockIdx.x - off[j],
              off[j + 1] - off[j]);
}

__global__ void k_upsample_batch(const UpsampleJob* __restrict__ J,
                                 const uint32_t* __restrict__ off, int nj) {
  const int j = batch_job(off, nj);
  const UpsampleJob& q = J[j];
  upsample_body(q.gc, q.total_c, q.gs, q.Rc, q.Cc, q.Rs, q.Cs, q.ctl,
                blockIdx.x - off[j], off[j + 1] - off[j]);
}

template <bool kDecomp>
__global__ void __launch_bounds__(256)
    k_pass_batch(const PassJob* __restrict__ J, const uint32_t* __restrict__ off,
                 int nj) {
  const int j = batch_job(off, nj);
  const PassJob& q = J[j];
  pass_body<kDecomp>(q.g, q.pb, q.B, blockIdx.x - off[j], off[j + 1] - off[j]);
}

// zero-fill of byte ranges (16-byte multiples, 16-byte aligned)
__global__ void k_zero_batch(const ZeroJob* __restrict__ J,
                             const uint32_t* __restrict__ off, int nj) {
  const int j = batch_job(off, nj);
  uint4* p = reinterpret_cast<uint4*>(J[j].ptr);
  const unsigned long long n = J[j].bytes >> 4;
  const unsigned b = blockIdx.x - off[j], nb = off[j + 1] - off[j];
  for (unsigned long long i = (unsigned long long)b * blockDim.x + threadIdx.x;
       i < n; i += (unsigned long long)nb * blockDim.x)
    p[i] = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void k_fill_batch(const FillJob* __restrict__ J,
                             const uint32_t* __restrict__ off, int nj) {
  const int j = batch_job(off, nj);
  fill_body(J[j].out, J[j].N, J[j].v, blockIdx.x - off[j], off[j + 1] - off[j]);
}

// ---------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------
static inline unsigned grid_for(uint64_t n, int threads, unsigned cap) {
  uint64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

void launch_init_ctl(Ctl* ctl, cudaStream_t s) {
  k_init_ctl<<<1, 256, 0, s>>>(ctl);
}

void launch_fill(float* out, uint32_t N, float v, int num_sms,
                 cudaStream_t s) {
  k_fill<<<grid_for(N, 256, num_sms * 16), 256, 0, s>>>(out, N, v);
}

void launch_range(const float* x, uint32_t N, Ctl* ctl, int num_sms,
                  cudaStream_t s) {
  k_range<<<grid_for(N / 4 + 1, 256, num_sms * 8), 256, 0, s>>>(x, N, ctl);
}

void launch_set_range(Ctl* ctl, unsigned kmin, unsigned kmax, cudaStream_t s) {
  k_set_range<<<1, 1, 0, s>>>(ctl, kmin, kmax);
}

void launch_params(Ctl* ctl, int eb_mode, double eb, double alpha,
                   double beta, int L, const float* x, cudaStream_t s) {
  k_params<<<1, 32, 0, s>>>(ctl, eb_mode, eb, alpha, beta, L, x);
}

void launch_anchor_gather(const float* x, const LevelGeom& ga, uint32_t total,
                          float* RA, uint16_t* CA, const Ctl* ctl,
                          cudaStream_t s) {
  k_anchor_gather<<<grid_for(total, 256, 65535), 256, 0, s>>>(x, ga, total,
                                                              RA, CA, ctl);
}

void launch_upsample(const LevelGeom& gc, uint32_t total_c,
                     const LevelGeom& gs, const float* Rc, const uint16_t* Cc,
                     float* Rs, uint16_t* Cs, const Ctl* ctl, cudaStream_t s) {
  k_upsample<<<grid_for(total_c, 256, 65535), 256, 0, s>>>(gc, total_c, gs, Rc,
                                                           Cc, Rs, Cs, ctl);
}

void launch_pass(bool decomp, const LevelGeom& g, const PassBox& pb,
                 const SweepBufs& B, int num_sms, cudaStream_t s) {
  if (pb.total == 0) return;
  const unsigned grid = grid_for(pb.total, 256, (unsigned)num_sms * 16);
  if (decomp)
    k_pass<true><<<grid, 256, 0, s>>>(g, pb, B);
  else
    k_pass<false><<<grid, 256, 0, s>>>(g, pb, B);
}

void launch_init_ctl_batch(const InitJob* J, int nj, cudaStream_t s) {
  if (nj > 0) k_init_ctl_batch<<<nj, 256, 0, s>>>(J);
}
void launch_range_batch(const RangeJob* J, const uint32_t* off, int nj,
                        uint32_t nblk, cudaStream_t s) {
  if (nblk) k_range_batch<<<nblk, 256, 0, s>>>(J, off, nj);
}
void launch_params_batch(const ParamsJob* J, int nj, cudaStream_t s) {
  if (nj > 0) k_params_batch<<<nj, 32, 0, s>>>(J);
}
void launch_anchor_batch(const AnchorJob* J, const uint32_t* off, int nj,
                         uint32_t nblk, cudaStream_t s) {
  if (nblk) k_anchor_batch<<<nblk, 256, 0, s>>>(J, off, nj);
}
void launch_fill_batch(const FillJob* J, const uint32_t* off, int nj,
                       uint32_t nblk, cudaStream_t s) {
  if (nblk) k_fill_batch<<<nblk, 256, 0, s>>>(J, off, nj);
}

void launch_upsample_batch(const UpsampleJob* J, const uint32_t* off, int nj,
                           uint32_t nblk, cudaStream_t s) {
  if (nblk) k_upsample_batch<<<nblk, 256, 0, s>>>(J, off, nj);
}
void launch_pass_batch(bool decomp, const PassJob* J, const uint32_t* off,
                       int nj, uint32_t nblk, cudaStream_t s) {
  if (!nblk) return;
  if (decomp)
    k_pass_batch<true><<<nblk, 256, 0, s>>>(J, off, nj);
  else
    k_pass_batch<false><<<nblk, 256, 0, s>>>(J, off, nj);
}
void launch_zero_batch(const ZeroJob* J, const uint32_t* off, int nj,
                       uint32_t nblk, cudaStream_t s) {
  if (nblk) k_zero_batch<<<nblk, 256, 0, s>>>(J, off, nj);
}
uint32_t grid_blocks(uint64_t n, unsigned cap) { return grid_for(n, 256, cap); }
uint32_t pass_blocks(uint32_t total, int num_sms) {
  return grid_for(total, 256, (unsigned)num_sms * 16);
}

}  // namespace hpez
