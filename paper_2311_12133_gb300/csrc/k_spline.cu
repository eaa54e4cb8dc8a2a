// k_spline.cu -- the global natural-spline interpolator (interp 3) for one
// 1D-style pass: along each line of the pass dimension, the natural cubic
// spline through every known point of the line (the knots at the even
// level-grid indices 0, 2, .., 2K) is evaluated halfway between knots, at
// the odd indices.  The paper's Eq. 6 is a local four-knot spline; this is
// the whole-line form, solved per line.
//
// With N_k = h^2 M_k / 6 (M: second derivative at knot k, h the knot
// spacing) the spline's conditions are N_{k-1} + 4 N_k + N_{k+1} = r_k,
// r_k = y_{k-1} - 2 y_k + y_{k+1} (k = 1..K-1), N_0 = N_K = 0, and halfway
// between knots k and k+1 the cubic piece is (y_k + y_{k+1}) / 2 -
// 3/8 (N_k + N_{k+1}).  A thread owns a line and runs the Thomas algorithm:
// the forward sweep keeps D_k in the slot of midpoint k (not predicted yet),
// the backward sweep forms N_k and finishes midpoint k (quantize or
// reconstruct).  The Thomas coefficients c'_1 = 1/4, c'_k = 1/(4 - c'_{k-1})
// in binary32 are stationary from k = 7 on, so a 16-entry table gives every
// c'_k exactly.  A point with no knot to its right takes the boundary rule
// of the other interpolators.  Lines of a launch are independent; threads
// run along the fastest other slot, so a pass along slot 0 or 1 reads and
// writes coalesced rows.
#include "hpez.h"
#include "hpez_internal.cuh"
#include "hpez_launch.h"

namespace hpez {
namespace {

constexpr int kCT = 16;

// the lines of one pass: line t has the level-grid index v_a = a_a + b_a
// (t / n_b) on the slower other slot and v_b = a_b + b_b (t % n_b) on the
// faster one; its first point sits at level-grid index v_a g_a + v_b g_b
// and field index v_a f_a + v_b f_b
struct SplineLines {
  uint32_t aa, ba, ab, bb, nb, nl;
  uint32_t ga, gb, fa, fb;  // level-grid / field strides of the two slots
  uint32_t st, fsd;         // along the line: level-grid and field strides
  int m;                    // level-grid extent along the line
};

template <bool kDecomp>
__global__ void __launch_bounds__(256)
    k_spline_pass(SplineLines Ln, int level, SweepBufs B, float* __restrict__ dscr) {
  __shared__ float ct[kCT];
  if (threadIdx.x == 0) {
    float c = 0.25f;
    ct[0] = 0.0f;
    ct[1] = c;
    for (int k = 2; k < kCT; ++k) {
      c = __fdiv_rn(1.0f, __fsub_rn(4.0f, c));
      ct[k] = c;
    }
  }
  __syncthreads();
  const Ctl* ctl = B.ctl;
  if (ctl->status || ctl->is_const) return;
  const int li = level - 1;
  const float el = ctl->el[li], inv2 = ctl->inv2[li], twoe = ctl->twoe[li];
  const int m = Ln.m;
  const int K = (m - 1) / 2;
  const uint32_t st = Ln.st, fsd = Ln.fsd;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < Ln.nl;
       t += gridDim.x * blockDim.x) {
    const uint32_t va = Ln.aa + Ln.ba * (t / Ln.nb), vb = Ln.ab + Ln.bb * (t % Ln.nb);
    const uint32_t ci0 = va * Ln.ga + vb * Ln.gb;
    const uint32_t fi0 = va * Ln.fa + vb * Ln.fb;
    float* const R = B.R + ci0;
    // D_k goes to the slot of midpoint k: in the level grid itself, or in
    // dscr when the level grid is the output that holds the escaped values
    float* const Dv = dscr ? dscr + ci0 : R;
    auto finish = [&](int uq, float p) {
      const uint32_t ci = ci0 + (uint32_t)uq * st, fi = fi0 + (uint32_t)uq * fsd;
      if (!kDecomp) {
        float rec;
        const unsigned code = quantize(B.x[fi], p, el, inv2, twoe, rec);
        B.C[ci] = (uint16_t)code;
        B.R[ci] = rec;
      } else {
        const unsigned code = B.codes_full[fi];
        B.R[ci] = code ? dequantize(code, p, twoe) : B.outl_full[fi];
      }
    };
    if (K >= 2) {
      float ym = R[0], y0 = R[2u * st], Dp = 0.0f;
#pragma unroll 4
      for (int k = 1; k <= K - 1; ++k) {
        const float yp = R[(uint32_t)(2 * k + 2) * st];
        const float r = __fsub_rn(__fadd_rn(ym, yp), __fmul_rn(2.0f, y0));
        const float c = ct[min(k, kCT - 1)];
        const float D = k == 1 ? __fmul_rn(r, c) : __fmul_rn(__fsub_rn(r, Dp), c);
        Dv[(uint32_t)(2 * k + 1) * st] = D;
        Dp = D;
        ym = y0;
        y0 = yp;
      }
    }
    float Nn = 0.0f;                          // N_{k+1}
    float yr = R[(uint32_t)(2 * K) * st];     // y_{k+1}
#pragma unroll 4
    for (int k = K - 1; k >= 0; --k) {
      const float yl = R[(uint32_t)(2 * k) * st];
      float Nk = 0.0f;
      if (k >= 1)
        Nk = __fsub_rn(Dv[(uint32_t)(2 * k + 1) * st], __fmul_rn(ct[min(k, kCT - 1)], Nn));
      const float p =
          __fsub_rn(__fmul_rn(__fadd_rn(yl, yr), 0.5f), __fmul_rn(0.375f, __fadd_rn(Nk, Nn)));
      finish(2 * k + 1, p);
      Nn = Nk;
      yr = yl;
    }
    if ((m & 1) == 0) {  // the odd index m - 1 has no knot to its right
      const int uq = m - 1;
      finish(uq, predict_line(R + (uint32_t)uq * st, (long long)st, uq, m, LINEAR, 0));
    }
  }
}

}  // namespace

// One 1D-style pass of the global spline (pb: the pass box, one slot in
// pb.S).  dscr: null, or a level-grid-sized scratch for the forward sweep
// when the level grid aliases the escaped values (decompress, level 1).
void launch_spline_pass(bool decomp, const LevelGeom& g, const PassBox& pb, const SweepBufs& B,
                        float* dscr, int num_sms, cudaStream_t s) {
  const int d = (pb.S & 1u) ? 0 : ((pb.S & 2u) ? 1 : 2);
  const int ea = d == 0 ? 1 : 0, eb = d == 2 ? 1 : 2;  // the other slots, ea < eb
  const uint64_t nl = (uint64_t)pb.cnt[ea] * pb.cnt[eb];
  if (nl == 0 || pb.cnt[d] == 0) return;
  SplineLines Ln;
  Ln.aa = pb.a[ea];
  Ln.ba = pb.b[ea];
  Ln.ab = pb.a[eb];
  Ln.bb = pb.b[eb];
  Ln.nb = pb.cnt[eb];
  Ln.nl = (uint32_t)nl;
  Ln.ga = g.gst[ea];
  Ln.gb = eb == 2 ? 1u : g.gst[eb];
  Ln.fa = g.step[ea] * g.fst[ea];
  Ln.fb = eb == 2 ? g.step[2] : g.step[eb] * g.fst[eb];
  Ln.st = d == 2 ? 1u : g.gst[d];
  Ln.fsd = d == 2 ? g.step[2] : g.step[d] * g.fst[d];
  Ln.m = (int)g.m[d];
  uint64_t grid = (nl + 255) / 256;
  const uint64_t cap = (uint64_t)(num_sms > 0 ? num_sms : 1) * 16;
  if (grid > cap) grid = cap;
  if (decomp)
    k_spline_pass<true><<<(unsigned)grid, 256, 0, s>>>(Ln, pb.level, B, dscr);
  else
    k_spline_pass<false><<<(unsigned)grid, 256, 0, s>>>(Ln, pb.level, B, dscr);
}

}  // namespace hpez
