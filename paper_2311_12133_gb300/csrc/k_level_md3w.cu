// k_level_md3w.cu -- the finest 3D level of the multi-dimensional paradigm
// (Sec. 5.3, Eq. 8) with one warp per strip of the field and no CTA
// barriers.
//
// A point with odd-coordinate set S is predicted from points with one odd
// coordinate fewer, along each direction of S (Eq. 8), so the level can be
// swept in any order that visits a point after the points it reads.  Here
// each lane owns a pair of columns (c even, c + 1) of a strip of rows and
// walks the strip row by row:
//   - along dim 2 (columns) the neighbours of the odd column c + 1 are the
//     even columns of the lanes around it (warp shuffles);
//   - along dim 1 (rows) an odd row trails the even rows it reads by one
//     (linear) or three (cubic) rows; the last four even rows of the lane's
//     columns stay in registers;
//   - along dim 0 (planes) a step runs the same rows of two planes: even
//     plane k + a and odd plane 2k + 1, which reads the even planes 2k - 2
//     .. 2k + 4 at those rows -- the newest from the registers of this
//     step, the older ones from a ring of per-lane history rows in shared
//     memory, where the new even plane then replaces the one no odd plane
//     reads again.
// So no value crosses warps: a strip recomputes the columns (halo lanes)
// and even rows just outside it that its own points read, and stores only
// its own points.  Each lane stages its inputs a few steps ahead with
// asynchronous copies into its own shared-memory slots (8-byte copies of
// its two columns: a warp reads 256 contiguous bytes of a row); codes leave
// as 4-byte pairs, reconstructions as 8-byte pairs.  A step away from the
// field's edges runs the interior stencils without the boundary choices.
#include <cuda.h>

#include "hpez_internal.cuh"
#include "hpez_launch.h"

namespace hpez {
namespace {

constexpr int kWRows = 16;  // owned rows of a strip
constexpr int kWWarps = 4;  // warps (strips) per CTA
// steps staged ahead (ring slots): compress loads more per step and stages
// deeper; decompress keeps more warps resident
template <bool kDecomp>
__host__ __device__ constexpr int wdepth() {
  return kDecomp ? 3 : 4;
}

template <int KIND>
struct WK {
  static constexpr int lag = KIND == LINEAR ? 0 : 1;   // odd row = newest even row - 1 - 2 lag
  static constexpr int ahead = KIND == LINEAR ? 1 : 2;  // even planes read past an odd plane
  // even planes kept in shared memory: linear 2k (2k + 2 comes from the
  // step's registers), cubic 2k - 2 .. 2k + 2 (2k + 4 from the registers)
  static constexpr int ring = KIND == LINEAR ? 1 : 3;
  static constexpr int hd = KIND == LINEAR ? 1 : 2;    // even halo rows below the strip
  static constexpr int hr = KIND == LINEAR ? 1 : 2;    // halo lanes on the right
  // history rows per plane: rows E_lo .. R1 - 2 + 2 hd, E_lo >= R0 - 2
  static constexpr int hist = KIND == LINEAR ? kWRows + 1 : kWRows + 5;
  static constexpr int fz = KIND == LINEAR ? F_LIN : (KIND == CUBIC_NAK ? F_NAK4 : F_NAT4);
};

// owned columns per strip (even)
template <int KIND>
__host__ __device__ constexpr int wcols() {
  return 2 * (32 - WK<KIND>::hr - (KIND == LINEAR ? 0 : 1));
}

// staged inputs of one step, per lane (lane-major arrays: a warp's access
// is contiguous): x (compress) or code pairs (decompress) of the even
// plane's and the odd plane's even and odd row, the even plane's coarse
// value and (compress) the 4-byte word holding its coarse code
struct WSlot {
  float2 ee[32], eo[32], oe[32], oo[32];  // [plane][row]: e = even, o = odd
  float cv[32];
  unsigned cc[32];
};
static_assert(sizeof(WSlot) == 32 * 40, "slot layout");

template <bool kDecomp, int KIND>
__host__ __device__ constexpr int wsmem_per_warp() {
  return wdepth<kDecomp>() * (int)sizeof(WSlot) + WK<KIND>::ring * WK<KIND>::hist * 32 * 8;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// asynchronous global -> shared copy of kBytes (4 or 8), zero-filled when
// !valid (nothing is read then)
template <int kBytes>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid) {
  const int n = valid ? kBytes : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_addr(dst)),
               "l"(src), "n"(kBytes), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The plane groups of a chunk: first the even planes the chunk's first odd
// plane reads, one group each; then for every odd plane k of the chunk the
// group (even plane k + ahead, odd plane k).  Where that even plane lies
// beyond the field, a linear odd plane that extrapolates from planes 2k and
// 2k - 2 gets plane k - 1 recomputed in its group instead (rec: not stored,
// not kept); otherwise the group has no even plane.  ke_ < 0 / ko_ < 0: no
// plane of that parity.
struct WSched {
  int lead, lead_end;  // lead-in even planes [lead, lead_end)
  int k, k_end;        // odd planes [k, k_end)
  int ahead, ke;
  bool lin;
  __device__ bool next(int& ke_, int& ko_, bool& rec_) {
    rec_ = false;
    if (lead < lead_end) {
      ke_ = lead++;
      ko_ = -1;
      return true;
    }
    if (k < k_end) {
      ko_ = k;
      if (k + ahead < ke) {
        ke_ = k + ahead;
      } else if (lin && k >= 1) {
        ke_ = k - 1;
        rec_ = true;
      } else {
        ke_ = -1;
      }
      ++k;
      return true;
    }
    return false;
  }
};

struct WCursor {
  WSched sc;
  int ke, ko, t;
  bool rec, valid;
  __device__ void init(const WSched& s) {
    sc = s;
    t = 0;
    valid = sc.next(ke, ko, rec);
  }
  __device__ void advance(int T) {
    if (++t == T) {
      t = 0;
      valid = sc.next(ke, ko, rec);
    }
  }
};

// the strip a warp works on: rows [R0, R1), owned columns [O0, O1), lane
// columns c = C0 + 2 lane; even rows E_lo .. re_last, T steps per group
struct WStrip {
  int R0, R1, O0, O1, C0;
  int E_lo, re_last, T;
  int m0, m1, m2;
};

// the stencil f, or (FAST) the interior stencil of the kind
template <int KIND, bool FAST>
__device__ __forceinline__ float wpred(int f, float m3, float m1, float p1, float p3) {
  constexpr int FZ = WK<KIND>::fz;
  if (FAST) return eval_formula(FZ, m3, 0.f, m1, p1, 0.f, p3);
  return eval_formula(f, m3, 0.f, m1, p1, 0.f, p3);
}

// stage the inputs of the group step at cursor `cu` into slot `sl`
template <bool kDecomp, int LAG>
__device__ __forceinline__ void w_stage(WSlot* sl, int lane, const WCursor& cu, const WStrip& S,
                                        int c, bool lane_in, const void* __restrict__ in,
                                        const float* __restrict__ Rc,
                                        const uint16_t* __restrict__ Cc, uint32_t gst0,
                                        uint32_t gst1, uint32_t cgst0, uint32_t cgst1) {
  const bool ok = cu.valid && lane_in;
  const int re = S.E_lo + 2 * cu.t;
  const int ro = re - 1 - 2 * LAG;
  const bool ve = ok && re <= S.re_last;
  const bool vo = ok && ro > S.R0 && ro < S.R1 && ro < S.m1;
  const bool he = cu.ke >= 0, ho = cu.ko >= 0;
  const uint32_t rb = (uint32_t)c + (uint32_t)re * gst1;  // even row, plane 0
  const uint32_t rbo = (uint32_t)c + (uint32_t)ro * gst1;
  const uint32_t pe = he ? (uint32_t)(2 * cu.ke) * gst0 : 0u;
  const uint32_t po = ho ? (uint32_t)(2 * cu.ko + 1) * gst0 : 0u;
  // invalid copies read nothing; their source is any valid address
  const uint32_t i_ee = ve && he ? pe + rb : 0u, i_eo = vo && he ? pe + rbo : 0u;
  const uint32_t i_oe = ve && ho ? po + rb : 0u, i_oo = vo && ho ? po + rbo : 0u;
  const bool vc = ve && he;
  const uint32_t ci =
      vc ? (uint32_t)cu.ke * cgst0 + (uint32_t)(re >> 1) * cgst1 + (uint32_t)(c >> 1) : 0u;
  cp_async<4>(&sl->cv[lane], Rc + ci, vc);
  if (!kDecomp) {
    const float* X = static_cast<const float*>(in);
    cp_async<8>(&sl->ee[lane], X + i_ee, ve && he);
    cp_async<8>(&sl->eo[lane], X + i_eo, vo && he);
    cp_async<8>(&sl->oe[lane], X + i_oe, ve && ho);
    cp_async<8>(&sl->oo[lane], X + i_oo, vo && ho);
    cp_async<4>(&sl->cc[lane], Cc + (ci & ~1u), vc);  // the aligned word holding the code
  } else {
    const uint16_t* Cf = static_cast<const uint16_t*>(in);
    cp_async<4>(&sl->ee[lane], Cf + i_ee, ve && he);
    cp_async<4>(&sl->eo[lane], Cf + i_eo, vo && he);
    cp_async<4>(&sl->oe[lane], Cf + i_oe, ve && ho);
    cp_async<4>(&sl->oo[lane], Cf + i_oo, vo && ho);
  }
}

// Quantize (compress): the code word and the reconstruction, with the
// exact bound check of quantize() taken only near the bound or out of
// range.  Reconstruct (decompress): p + 2 e_l q, or the escaped value
// (lane_in: the lane's columns lie in the field; other lanes only fill
// shuffles and read nothing).
template <bool kDecomp>
__device__ __forceinline__ float w_point(float p, float x, unsigned code, uint32_t fi,
                                         bool lane_in, const float* __restrict__ outl, float el,
                                         float inv2, float twoe, unsigned& code_out) {
  if (!kDecomp) {
    const float diff = __fsub_rn(x, p);
    const float m = __fadd_rn(__fmul_rn(fabsf(diff), inv2), 0.5f);
    const int kq = __float2int_rz(fminf(m, 32767.0f));
    const int q = diff < 0.0f ? -kq : kq;
    const float r = __fadd_rn(p, __fmul_rn(__int2float_rn(q), twoe));
    if (m < 32768.0f && fabsf(__fsub_rn(r, x)) < el) {
      code_out = (unsigned)(q + kRadius);
      return r;
    }
    float rec;
    code_out = quantize(x, p, el, inv2, twoe, rec);
    return rec;
  }
  if (code) return dequantize(code, p, twoe);
  return lane_in ? __ldg(outl + fi) : 0.f;
}

struct WConst {
  float el, inv2, twoe;
  float w001, w010, w100, w011a, w011b, w101a, w101b, w110a, w110b, w111a, w111b, w111c;
  uint32_t gst0, gst1, cgst0, cgst1, chalf;  // chalf: coarse column c / 2
  int c, f2;
  bool lane_in, own_c;
};

struct WRow {
  float2 e, o;  // values of the step's even row (re) and odd row (ro)
};

__device__ __forceinline__ void win_push(float2 (&w)[4], float2 v) {
  w[0] = w[1];
  w[1] = w[2];
  w[2] = w[3];
  w[3] = v;
}

// the even plane ke at rows re (coarse point, (0,0,1)) and ro ((0,1,0),
// (0,1,1)); returns the values for the odd plane and the history
template <bool kDecomp, int KIND, bool FAST>
__device__ __forceinline__ WRow w_even(const WConst& K, const WStrip& S, const WSlot* sl, int lane,
                                       int k, bool own_e, int re, int ro, bool ve, bool vo,
                                       float2 (&win)[4], const float* __restrict__ outl,
                                       float* __restrict__ Rs, uint16_t* __restrict__ Cs) {
  using W = WK<KIND>;
  constexpr unsigned FULL = 0xFFFFFFFFu;
  WRow out;
  out.e = out.o = make_float2(0.f, 0.f);
  const uint32_t pb = (uint32_t)(2 * k) * K.gst0 + (uint32_t)K.c;
  if (ve) {
    const uint32_t fi = pb + (uint32_t)re * K.gst1;
    const float2 xe = sl->ee[lane];
    const unsigned ce = kDecomp ? __float_as_uint(xe.x) : 0u;
    const float ee = sl->cv[lane];
    unsigned code_ee = 0u, code_eo = 0u;
    if (!kDecomp) {
      // the code's half of the aligned word staged for it
      const unsigned wcc = sl->cc[lane];
      const uint32_t ci = (uint32_t)k * K.cgst0 + (uint32_t)(re >> 1) * K.cgst1 + K.chalf;
      code_ee = (ci & 1u) ? wcc >> 16 : wcc & 0xFFFFu;
    }
    const float vp1 = __shfl_down_sync(FULL, ee, 1);
    const float vm3 = __shfl_up_sync(FULL, ee, 1);
    const float vp3 = KIND != LINEAR ? __shfl_down_sync(FULL, ee, 2) : 0.f;
    const float q2 = wpred<KIND, FAST>(K.f2, vm3, ee, vp1, vp3);
    const float eo = w_point<kDecomp>(__fmul_rn(K.w001, q2), xe.y, ce >> 16, fi + 1, K.lane_in,
                                      outl, K.el, K.inv2, K.twoe, code_eo);
    if (K.own_c && own_e && re >= S.R0 && re < S.R1) {
      if (!kDecomp)
        *reinterpret_cast<unsigned*>(Cs + fi) = code_ee | (code_eo << 16);
      else
        *reinterpret_cast<float2*>(Rs + fi) = make_float2(ee, eo);
    }
    out.e = make_float2(ee, eo);
  }
  win_push(win, out.e);
  if (vo) {
    const uint32_t fi = pb + (uint32_t)ro * K.gst1;
    const int f1 = FAST ? W::fz : choose_formula(KIND, false, ro, S.m1);
    const float2 rm3 = W::lag ? win[0] : win[1];
    const float2 rm1 = W::lag ? win[1] : win[2];
    const float2 rp1 = W::lag ? win[2] : win[3];
    const float2 rp3 = W::lag ? win[3] : make_float2(0.f, 0.f);
    const float2 xo = sl->eo[lane];
    const unsigned co = kDecomp ? __float_as_uint(xo.x) : 0u;
    unsigned code_oe = 0u, code_oo = 0u;
    const float p1e = wpred<KIND, FAST>(f1, rm3.x, rm1.x, rp1.x, rp3.x);
    const float p1o = wpred<KIND, FAST>(f1, rm3.y, rm1.y, rp1.y, rp3.y);
    // (0,1,0) along dim 1, then (0,1,1) along dims 1 and 2
    const float oe = w_point<kDecomp>(__fmul_rn(K.w010, p1e), xo.x, co & 0xFFFFu, fi, K.lane_in,
                                      outl, K.el, K.inv2, K.twoe, code_oe);
    const float vp1 = __shfl_down_sync(FULL, oe, 1);
    const float vm3 = __shfl_up_sync(FULL, oe, 1);
    const float vp3 = KIND != LINEAR ? __shfl_down_sync(FULL, oe, 2) : 0.f;
    const float p2 = wpred<KIND, FAST>(K.f2, vm3, oe, vp1, vp3);
    const float p = __fadd_rn(__fmul_rn(K.w011a, p1o), __fmul_rn(K.w011b, p2));
    const float oo = w_point<kDecomp>(p, xo.y, co >> 16, fi + 1, K.lane_in, outl, K.el, K.inv2,
                                      K.twoe, code_oo);
    if (K.own_c && own_e) {
      if (!kDecomp)
        *reinterpret_cast<unsigned*>(Cs + fi) = code_oe | (code_oo << 16);
      else
        *reinterpret_cast<float2*>(Rs + fi) = make_float2(oe, oo);
    }
    out.o = make_float2(oe, oo);
  }
  return out;
}

// the odd plane 2k + 1 at rows re ((1,0,0), (1,0,1)) and ro ((1,1,0),
// (1,1,1)); d0e / d0o: the even planes 2k - 2, 2k, 2k + 2, 2k + 4 at the
// two rows
template <bool kDecomp, int KIND, bool FAST>
__device__ __forceinline__ void w_odd(const WConst& K, const WStrip& S, const WSlot* sl, int lane,
                                      int k, int f0, int re, int ro, bool ve, bool vo,
                                      const float2 (&d0e)[4], const float2 (&d0o)[4],
                                      float2 (&win)[4], const float* __restrict__ outl,
                                      float* __restrict__ Rs, uint16_t* __restrict__ Cs) {
  using W = WK<KIND>;
  constexpr unsigned FULL = 0xFFFFFFFFu;
  const uint32_t pb = (uint32_t)(2 * k + 1) * K.gst0 + (uint32_t)K.c;
  float2 ve_val = make_float2(0.f, 0.f);
  if (ve) {
    const uint32_t fi = pb + (uint32_t)re * K.gst1;
    const float2 xe = sl->oe[lane];
    const unsigned ce = kDecomp ? __float_as_uint(xe.x) : 0u;
    unsigned code_ee = 0u, code_eo = 0u;
    // (1,0,0) along dim 0, then (1,0,1) along dims 0 and 2
    const float p0 = wpred<KIND, FAST>(f0, d0e[0].x, d0e[1].x, d0e[2].x, d0e[3].x);
    const float ee = w_point<kDecomp>(__fmul_rn(K.w100, p0), xe.x, ce & 0xFFFFu, fi, K.lane_in,
                                      outl, K.el, K.inv2, K.twoe, code_ee);
    const float q0 = wpred<KIND, FAST>(f0, d0e[0].y, d0e[1].y, d0e[2].y, d0e[3].y);
    const float vp1 = __shfl_down_sync(FULL, ee, 1);
    const float vm3 = __shfl_up_sync(FULL, ee, 1);
    const float vp3 = KIND != LINEAR ? __shfl_down_sync(FULL, ee, 2) : 0.f;
    const float q2 = wpred<KIND, FAST>(K.f2, vm3, ee, vp1, vp3);
    const float p = __fadd_rn(__fmul_rn(K.w101a, q0), __fmul_rn(K.w101b, q2));
    const float eo = w_point<kDecomp>(p, xe.y, ce >> 16, fi + 1, K.lane_in, outl, K.el, K.inv2,
                                      K.twoe, code_eo);
    if (K.own_c && re >= S.R0 && re < S.R1) {
      if (!kDecomp)
        *reinterpret_cast<unsigned*>(Cs + fi) = code_ee | (code_eo << 16);
      else
        *reinterpret_cast<float2*>(Rs + fi) = make_float2(ee, eo);
    }
    ve_val = make_float2(ee, eo);
  }
  win_push(win, ve_val);
  if (vo) {
    const uint32_t fi = pb + (uint32_t)ro * K.gst1;
    const int f1 = FAST ? W::fz : choose_formula(KIND, false, ro, S.m1);
    const float2 rm3 = W::lag ? win[0] : win[1];
    const float2 rm1 = W::lag ? win[1] : win[2];
    const float2 rp1 = W::lag ? win[2] : win[3];
    const float2 rp3 = W::lag ? win[3] : make_float2(0.f, 0.f);
    const float2 xo = sl->oo[lane];
    const unsigned co = kDecomp ? __float_as_uint(xo.x) : 0u;
    unsigned code_oe = 0u, code_oo = 0u;
    const float p1e = wpred<KIND, FAST>(f1, rm3.x, rm1.x, rp1.x, rp3.x);
    const float p1o = wpred<KIND, FAST>(f1, rm3.y, rm1.y, rp1.y, rp3.y);
    // (1,1,0) along dims 0 and 1
    const float p0 = wpred<KIND, FAST>(f0, d0o[0].x, d0o[1].x, d0o[2].x, d0o[3].x);
    const float pa = __fadd_rn(__fmul_rn(K.w110a, p0), __fmul_rn(K.w110b, p1e));
    const float oe = w_point<kDecomp>(pa, xo.x, co & 0xFFFFu, fi, K.lane_in, outl, K.el, K.inv2,
                                      K.twoe, code_oe);
    // (1,1,1) along dims 0, 1 and 2
    const float vp1 = __shfl_down_sync(FULL, oe, 1);
    const float vm3 = __shfl_up_sync(FULL, oe, 1);
    const float vp3 = KIND != LINEAR ? __shfl_down_sync(FULL, oe, 2) : 0.f;
    const float p2 = wpred<KIND, FAST>(K.f2, vm3, oe, vp1, vp3);
    const float q0 = wpred<KIND, FAST>(f0, d0o[0].y, d0o[1].y, d0o[2].y, d0o[3].y);
    float p = __fmul_rn(K.w111a, q0);
    p = __fadd_rn(p, __fmul_rn(K.w111b, p1o));
    p = __fadd_rn(p, __fmul_rn(K.w111c, p2));
    const float oo = w_point<kDecomp>(p, xo.y, co >> 16, fi + 1, K.lane_in, outl, K.el, K.inv2,
                                      K.twoe, code_oo);
    if (K.own_c) {
      if (!kDecomp)
        *reinterpret_cast<unsigned*>(Cs + fi) = code_oe | (code_oo << 16);
      else
        *reinterpret_cast<float2*>(Rs + fi) = make_float2(oe, oo);
    }
  }
}

// one group step: the even plane (if any), then the odd plane (if any),
// then the even plane's rows replace the oldest plane of the history ring
template <bool kDecomp, int KIND, bool FAST>
__device__ __forceinline__ void w_group(const WConst& K, const WStrip& S, const WSlot* sl,
                                        int lane, int ke, int ko, bool rec, bool own_e, int f0,
                                        int re, int ro, bool ve, bool vo, float2* hist,
                                        float2 (&win_e)[4], float2 (&win_o)[4],
                                        const float* __restrict__ outl, float* __restrict__ Rs,
                                        uint16_t* __restrict__ Cs) {
  using W = WK<KIND>;
  constexpr int RN = W::ring;
  constexpr int HS = W::hist * 32;
  const int he = (re - S.E_lo) * 32, ho = (ro - S.E_lo) * 32;
  WRow nw;
  nw.e = nw.o = make_float2(0.f, 0.f);
  if (ke >= 0)
    nw = w_even<kDecomp, KIND, FAST>(K, S, sl, lane, ke, own_e, re, ro, ve, vo, win_e, outl, Rs,
                                     Cs);
  if (ko >= 0) {
    // the even planes 2k-2, 2k, 2k+2, 2k+4 (even-plane indices k-1 .. k+2)
    // at rows re and ro: this step's even plane from the registers, the
    // others from the ring (linear: only plane k)
    float2 d0e[4], d0o[4];
    const float2 z = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int kk = ko - 1 + j;
      const bool in_ring = KIND == LINEAR ? j == 1 : j < 3;
      if (ke >= 0 && kk == ke) {
        d0e[j] = nw.e;
        d0o[j] = nw.o;
      } else if (!in_ring) {
        d0e[j] = d0o[j] = z;  // not read
      } else {
        const float2* h = hist + ((kk + RN) % RN) * HS;
        d0e[j] = ve ? h[he] : z;
        d0o[j] = vo ? h[ho] : z;
      }
    }
    w_odd<kDecomp, KIND, FAST>(K, S, sl, lane, ko, f0, re, ro, ve, vo, d0e, d0o, win_o, outl, Rs,
                               Cs);
  }
  if (ke >= 0 && !rec) {
    float2* h = hist + (ke % RN) * HS;
    if (ve) h[he] = nw.e;
    if (vo) h[ho] = nw.o;
  }
}

template <bool kDecomp, int KIND>
__device__ __forceinline__ void md3w_body(const LevelMD& P, int n1, int n2, int K,
                                          const void* __restrict__ in,
                                          const float* __restrict__ outl,
                                          const float* __restrict__ Rc,
                                          const uint16_t* __restrict__ Cc,
                                          float* __restrict__ Rs, uint16_t* __restrict__ Cs,
                                          const Ctl* __restrict__ ctl, unsigned bid) {
  using W = WK<KIND>;
  constexpr int kWD = wdepth<kDecomp>();
  if (ctl->status || ctl->is_const) return;
  extern __shared__ __align__(16) unsigned char wsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wid = (int)bid * kWWarps + warp;
  const int s2 = wid % n2, s1 = (wid / n2) % n1, chunk = wid / (n1 * n2);
  WStrip S;
  S.m0 = (int)P.g.m[0];
  S.m1 = (int)P.g.m[1];
  S.m2 = (int)P.g.m[2];
  const int ke = (S.m0 + 1) / 2, ko = S.m0 / 2;
  const int K0 = chunk * K;
  if (K0 >= ke) return;  // warp-uniform
  const int K1o = min(K0 + K, ko), K1e = min(K0 + K, ke);
  // columns: a cubic strip reads one lane to its left; a linear strip only
  // when its last odd column extrapolates from three columns back
  constexpr int WC = wcols<KIND>();
  S.O0 = s2 * WC;
  S.O1 = min(S.O0 + WC, S.m2);
  const int hl = (KIND != LINEAR || S.O1 - S.O0 < 4) ? 1 : 0;
  S.C0 = S.O0 - 2 * hl;
  WConst Kc;
  Kc.c = S.C0 + 2 * lane;
  Kc.lane_in = Kc.c >= 0 && Kc.c < S.m2;
  Kc.own_c = Kc.c >= S.O0 && Kc.c < S.O1;
  Kc.chalf = (uint32_t)(Kc.c >> 1);
  // rows: even halo rows above (cubic, or a short last strip that
  // extrapolates) and below
  S.R0 = s1 * kWRows;
  S.R1 = min(S.R0 + kWRows, S.m1);
  const int hu = (KIND != LINEAR || (S.R1 == S.m1 && S.R1 - S.R0 < 4)) ? 1 : 0;
  S.E_lo = max(S.R0 - 2 * hu, 0);
  const int last_even = (S.m1 - 1) & ~1;
  S.re_last = min(S.R1 < S.m1 ? S.R1 - 2 + 2 * W::hd : last_even, last_even);
  {
    const int ro_last = ((S.R1 - 1) & 1) ? S.R1 - 1 : S.R1 - 2;  // largest odd row < R1
    const int T_e = (S.re_last - S.E_lo) / 2 + 1;
    const int T_o = ro_last > S.R0 ? (ro_last + 1 + 2 * W::lag - S.E_lo) / 2 + 1 : 0;
    S.T = max(T_e, T_o);
  }
  // the plane groups (the even planes just outside the chunk that its odd
  // planes read are recomputed, not stored): lead-in even planes up to
  // K0 + ahead - 1 (cubic: from K0 - 1, which its stencils read), then one
  // group per odd plane
  WSched sched;
  sched.lin = KIND == LINEAR;
  sched.lead = KIND != LINEAR && K0 > 0 ? K0 - 1 : K0;
  sched.lead_end = K1o > K0 ? min(K0 + W::ahead, ke) : K1e;
  sched.k = K0;
  sched.k_end = K1o;
  sched.ahead = W::ahead;
  sched.ke = ke;

  const int li = P.level - 1;
  Kc.el = ctl->el[li];
  Kc.inv2 = ctl->inv2[li];
  Kc.twoe = ctl->twoe[li];
  Kc.gst0 = P.g.gst[0];
  Kc.gst1 = P.g.gst[1];
  Kc.cgst0 = P.gc.gst[0];
  Kc.cgst1 = P.gc.gst[1];
  Kc.w001 = P.w[4][2];
  Kc.w010 = P.w[2][1];
  Kc.w100 = P.w[1][0];
  Kc.w011a = P.w[6][1];
  Kc.w011b = P.w[6][2];
  Kc.w101a = P.w[5][0];
  Kc.w101b = P.w[5][2];
  Kc.w110a = P.w[3][0];
  Kc.w110b = P.w[3][1];
  Kc.w111a = P.w[7][0];
  Kc.w111b = P.w[7][1];
  Kc.w111c = P.w[7][2];
  // the stencil along dim 2 at this lane's odd column; the strip is
  // interior when every owned lane takes the interior stencil
  Kc.f2 = choose_formula(KIND, false, Kc.c + 1, S.m2);
  const bool strip_fast = __all_sync(0xFFFFFFFFu, !Kc.own_c || Kc.f2 == W::fz);

  WSlot* slots = reinterpret_cast<WSlot*>(wsm + (size_t)warp * wsmem_per_warp<kDecomp, KIND>());
  float2* hist = reinterpret_cast<float2*>(wsm + (size_t)warp * wsmem_per_warp<kDecomp, KIND>() +
                                           kWD * sizeof(WSlot)) + lane;

  WCursor ci, cc;
  ci.init(sched);
  cc = ci;
  // stage the first kWD - 1 steps
#pragma unroll
  for (int i = 0; i < kWD - 1; ++i) {
    w_stage<kDecomp, W::lag>(slots + i, lane, ci, S, Kc.c, Kc.lane_in, in, Rc, Cc, Kc.gst0,
                             Kc.gst1, Kc.cgst0, Kc.cgst1);
    cp_commit();
    ci.advance(S.T);
  }
  float2 win_e[4], win_o[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) win_e[j] = win_o[j] = make_float2(0.f, 0.f);
  int f0 = W::fz;
  bool own_e = true, group_fast = true;
  int slot = 0;
  while (cc.valid) {
    // stage the step kWD - 1 ahead into the slot the last step used
    w_stage<kDecomp, W::lag>(slots + (slot + kWD - 1) % kWD, lane, ci, S, Kc.c,
                             Kc.lane_in, in, Rc, Cc, Kc.gst0, Kc.gst1, Kc.cgst0, Kc.cgst1);
    cp_commit();
    ci.advance(S.T);
    if (cc.t == 0) {
      // a new group
      own_e = !cc.rec && cc.ke >= K0 && cc.ke < K1e;
      f0 = cc.ko >= 0 ? choose_formula(KIND, false, 2 * cc.ko + 1, S.m0) : W::fz;
      group_fast = strip_fast && f0 == W::fz;
    }
    const int re = S.E_lo + 2 * cc.t;
    const int ro = re - 1 - 2 * W::lag;
    const bool ve = re <= S.re_last;
    const bool vo = ro > S.R0 && ro < S.R1 && ro < S.m1;
    const bool row_fast = !vo || (KIND == LINEAR ? ro + 1 < S.m1 : (ro >= 3 && ro + 3 < S.m1));
    cp_wait<kWD - 1>();
    const WSlot* sl = slots + slot;
    if (group_fast && row_fast)
      w_group<kDecomp, KIND, true>(Kc, S, sl, lane, cc.ke, cc.ko, cc.rec, own_e, f0, re, ro, ve, vo,
                                   hist, win_e, win_o, outl, Rs, Cs);
    else
      w_group<kDecomp, KIND, false>(Kc, S, sl, lane, cc.ke, cc.ko, cc.rec, own_e, f0, re, ro, ve,
                                    vo,
                                    hist, win_e, win_o, outl, Rs, Cs);
    slot = slot + 1 == kWD ? 0 : slot + 1;
    cc.advance(S.T);
  }
  cp_wait<0>();
}

template <bool kDecomp, int KIND>
__global__ void __launch_bounds__(32 * kWWarps, kDecomp ? 7 : 5)
    k_md3w(LevelMD P, int n1, int n2, int K, const void* __restrict__ in,
           const float* __restrict__ outl, const float* __restrict__ Rc,
           const uint16_t* __restrict__ Cc, float* __restrict__ Rs, uint16_t* __restrict__ Cs,
           const Ctl* __restrict__ ctl) {
  md3w_body<kDecomp, KIND>(P, n1, n2, K, in, outl, Rc, Cc, Rs, Cs, ctl, blockIdx.x);
}

// batched: job j owns the CTAs (groups of kWWarps strips) [off[j], off[j+1])
// of the launch.  The kernel is persistent by construction: each warp
// streams the K even planes of its chunk (and the odd planes between them)
// through its own staging slots, and the planner sizes the chunks so that
// the launch holds about the CTAs resident at once.
template <bool kDecomp, int KIND>
__global__ void __launch_bounds__(32 * kWWarps, kDecomp ? 7 : 5)
    k_md3w_batch(const MD3WJob* __restrict__ J, const uint32_t* __restrict__ off, int nj) {
  const int j = batch_job(off, nj);
  const MD3WJob& q = J[j];
  md3w_body<kDecomp, KIND>(q.P, q.n1, q.n2, q.K, q.in, q.outl, q.Rc, q.Cc, q.Rs, q.Cs, q.ctl,
                           blockIdx.x - __ldg(off + j));
}

template <bool kDecomp, int KIND>
void launch_md3w_b(const MD3WJob* J, const uint32_t* off, int nj, uint32_t nblk,
                   int num_sms, int max_ctas, cudaStream_t s) {
  const int smem = kWWarps * wsmem_per_warp<kDecomp, KIND>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_md3w_batch<kDecomp, KIND>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  (void)num_sms;
  (void)max_ctas;
  k_md3w_batch<kDecomp, KIND><<<nblk, 32 * kWWarps, smem, s>>>(J, off, nj);
}

template <bool kDecomp, int KIND>
int md3w_occupancy() {
  const int smem = kWWarps * wsmem_per_warp<kDecomp, KIND>();
  static int per_sm = 0;
  if (!per_sm) {
    cudaFuncSetAttribute(k_md3w<kDecomp, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_md3w<kDecomp, KIND>,
                                                  32 * kWWarps, smem);
    if (per_sm < 1) per_sm = 1;
  }
  return per_sm;
}

template <bool kDecomp, int KIND>
int launch_md3w_k(const LevelMD& P, const void* in, const float* outl, const float* Rc,
                  const uint16_t* Cc, float* Rs, uint16_t* Cs, const Ctl* ctl, int num_sms,
                  int chunks, cudaStream_t s) {
  const int smem = kWWarps * wsmem_per_warp<kDecomp, KIND>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_md3w<kDecomp, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    attr = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_md3w<kDecomp, KIND>, 32 * kWWarps,
                                                smem);
  if (per_sm < 1) per_sm = 1;
  const int m0 = (int)P.g.m[0], m1 = (int)P.g.m[1], m2 = (int)P.g.m[2];
  const int n1 = (m1 + kWRows - 1) / kWRows;
  const int n2 = (m2 + wcols<KIND>() - 1) / wcols<KIND>();
  const int ke = (m0 + 1) / 2;
  const int strips = n1 * n2;
  int nch = chunks > 0 ? chunks : (num_sms * per_sm * kWWarps) / strips;
  nch = std::max(1, std::min(nch, ke));
  const int K = (ke + nch - 1) / nch;
  nch = (ke + K - 1) / K;
  const long long warps = (long long)strips * nch;
  const unsigned grid = (unsigned)((warps + kWWarps - 1) / kWWarps);
  k_md3w<kDecomp, KIND><<<grid, 32 * kWWarps, smem, s>>>(P, n1, n2, K, in, outl, Rc, Cc, Rs,
                                                          Cs, ctl);
  return nch;
}

}  // namespace

// The finest level, warp strips: level-1 grid (the grid is the field),
// rows of an even number of points (8-byte pairs), 8-byte aligned input and
// (decompress) output, 4-byte aligned codes (compress), the coarse grid
// compact.
bool md3w_supported(const LevelMD& P, bool decomp, const void* in, const float* Rc,
                    const uint16_t* Cc, const float* Rs, const uint16_t* Cs) {
  if (P.level != 1 || P.write_recon != (decomp ? 1 : 0)) return false;
  for (int d = 0; d < 3; ++d)
    if (P.g.step[d] != 1 || P.g.gst[d] != P.fst[d]) return false;
  if (P.g.m[0] < 2 || P.g.m[1] < 2 || P.g.m[2] < 2) return false;
  if (P.g.m[2] % 2) return false;
  if (P.g.gst[1] != P.g.m[2] || P.gc.gst[1] != P.gc.m[2] ||
      P.gc.gst[0] != P.gc.m[1] * P.gc.m[2])
    return false;
  if ((uint64_t)P.g.m[0] * P.g.m[1] * P.g.m[2] >= (1ull << 32)) return false;
  if (((uintptr_t)in & 7) || ((uintptr_t)Rc & 3)) return false;
  if (!decomp && (((uintptr_t)Cc & 3) || ((uintptr_t)Cs & 3))) return false;
  if (decomp && ((uintptr_t)Rs & 7)) return false;
  return true;
}

// Returns the chunks along dim 0.
int launch_level_md3w(bool decomp, int kind, const LevelMD& P, const SweepBufs& B,
                      const float* Rc, const uint16_t* Cc, float* Rs, uint16_t* Cs,
                      const Ctl* ctl, int num_sms, int chunks, cudaStream_t s) {
  const void* in = decomp ? (const void*)B.codes_full : (const void*)B.x;
  const float* outl = B.outl_full;
  if (decomp) {
    if (kind == LINEAR)
      return launch_md3w_k<true, LINEAR>(P, in, outl, Rc, Cc, Rs, Cs, ctl, num_sms, chunks, s);
    if (kind == CUBIC_NAK)
      return launch_md3w_k<true, CUBIC_NAK>(P, in, outl, Rc, Cc, Rs, Cs, ctl, num_sms, chunks, s);
    return launch_md3w_k<true, CUBIC_NAT>(P, in, outl, Rc, Cc, Rs, Cs, ctl, num_sms, chunks, s);
  }
  if (kind == LINEAR)
    return launch_md3w_k<false, LINEAR>(P, in, outl, Rc, Cc, Rs, Cs, ctl, num_sms, chunks, s);
  if (kind == CUBIC_NAK)
    return launch_md3w_k<false, CUBIC_NAK>(P, in, outl, Rc, Cc, Rs, Cs, ctl, num_sms, chunks, s);
  return launch_md3w_k<false, CUBIC_NAT>(P, in, outl, Rc, Cc, Rs, Cs, ctl, num_sms, chunks, s);
}

// The geometry of a warp-strip level: strips per chunk (n1 x n2), even
// planes per chunk K, CTAs.  chunks <= 0: as many chunks as fill the GPU
// with this field alone.
void md3w_geometry(bool decomp, int kind, const LevelMD& P, int num_sms, int chunks, int* n1,
                   int* n2, int* K, uint32_t* ctas) {
  int per_sm;
  int wc;
  if (decomp) {
    per_sm = kind == LINEAR ? md3w_occupancy<true, LINEAR>()
                            : (kind == CUBIC_NAK ? md3w_occupancy<true, CUBIC_NAK>()
                                                 : md3w_occupancy<true, CUBIC_NAT>());
  } else {
    per_sm = kind == LINEAR ? md3w_occupancy<false, LINEAR>()
                            : (kind == CUBIC_NAK ? md3w_occupancy<false, CUBIC_NAK>()
                                                 : md3w_occupancy<false, CUBIC_NAT>());
  }
  wc = kind == LINEAR ? wcols<LINEAR>()
                      : (kind == CUBIC_NAK ? wcols<CUBIC_NAK>() : wcols<CUBIC_NAT>());
  const int m0 = (int)P.g.m[0], m1 = (int)P.g.m[1], m2 = (int)P.g.m[2];
  *n1 = (m1 + kWRows - 1) / kWRows;
  *n2 = (m2 + wc - 1) / wc;
  const int ke = (m0 + 1) / 2;
  const int strips = *n1 * *n2;
  int nch = chunks > 0 ? chunks : (num_sms * per_sm * kWWarps) / strips;
  nch = std::max(1, std::min(nch, ke));
  *K = (ke + nch - 1) / nch;
  nch = (ke + *K - 1) / *K;
  const long long warps = (long long)strips * nch;
  *ctas = (uint32_t)((warps + kWWarps - 1) / kWWarps);
}

void launch_md3w_batch(bool decomp, int kind, const MD3WJob* J, const uint32_t* off, int nj,
                       uint32_t nblk, int num_sms, int max_ctas, cudaStream_t s) {
  if (!nblk) return;
  if (decomp) {
    if (kind == LINEAR) launch_md3w_b<true, LINEAR>(J, off, nj, nblk, num_sms, max_ctas, s);
    else if (kind == CUBIC_NAK)
      launch_md3w_b<true, CUBIC_NAK>(J, off, nj, nblk, num_sms, max_ctas, s);
    else launch_md3w_b<true, CUBIC_NAT>(J, off, nj, nblk, num_sms, max_ctas, s);
  } else {
    if (kind == LINEAR) launch_md3w_b<false, LINEAR>(J, off, nj, nblk, num_sms, max_ctas, s);
    else if (kind == CUBIC_NAK)
      launch_md3w_b<false, CUBIC_NAK>(J, off, nj, nblk, num_sms, max_ctas, s);
    else launch_md3w_b<false, CUBIC_NAT>(J, off, nj, nblk, num_sms, max_ctas, s);
  }
}

}  // namespace hpez
