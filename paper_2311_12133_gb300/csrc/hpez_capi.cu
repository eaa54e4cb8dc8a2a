// hpez_capi.cu -- the C-ABI entry points of libhpez.so (declared in
// include/hpez.h): argument validation, the level/pass schedule, the device
// scratch arena, and the launch sequence of compress and decompress.
#include "hpez.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "hpez_internal.cuh"
#include "hpez_launch.h"
#include "hpez_ctx.h"

using namespace hpez;



namespace hpez {
namespace host {


void wr32(uint8_t* b, int o, uint32_t v) { std::memcpy(b + o, &v, 4); }
void wr64(uint8_t* b, int o, uint64_t v) { std::memcpy(b + o, &v, 8); }
void wrf64(uint8_t* b, int o, double v) { std::memcpy(b + o, &v, 8); }
uint32_t rd32(const uint8_t* b, int o) {
  uint32_t v;
  std::memcpy(&v, b + o, 4);
  return v;
}
uint64_t rd64(const uint8_t* b, int o) {
  uint64_t v;
  std::memcpy(&v, b + o, 8);
  return v;
}
double rdf64(const uint8_t* b, int o) {
  double v;
  std::memcpy(&v, b + o, 8);
  return v;
}
float rdf32(const uint8_t* b, int o) {
  float v;
  std::memcpy(&v, b + o, 4);
  return v;
}

uint64_t a16(uint64_t v) { return (v + 15) & ~(uint64_t)15; }
bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// ---------------------------------------------------------------------
// geometry plan
// ---------------------------------------------------------------------

int plan_geometry(Plan& p, int ndim, const uint64_t* dims, int A,
                  int frozen) {
  if (ndim < 1 || ndim > 3 || !dims) return HPEZ_ERR_INVALID_ARG;
  if (frozen < -1 || frozen >= ndim || (ndim == 1 && frozen != -1))
    return HPEZ_ERR_INVALID_ARG;
  if (!pow2(A) || A < 2 || A > 32768) return HPEZ_ERR_INVALID_ARG;
  p.ndim = ndim;
  p.off = 3 - ndim;
  uint64_t N = 1;
  for (int d = 0; d < ndim; ++d) {
    if (dims[d] == 0) return HPEZ_ERR_INVALID_ARG;
    N *= dims[d];
    if (N > 0xFFFFFFFFull) return HPEZ_ERR_INVALID_ARG;
    p.n[d + p.off] = (uint32_t)dims[d];
    p.interp[d + p.off] = d != frozen;
  }
  p.N = (uint32_t)N;
  p.fst[2] = 1;
  p.fst[1] = p.n[2];
  p.fst[0] = p.n[1] * p.n[2];
  p.k = 0;
  for (int s = 0; s < 3; ++s) p.k += p.interp[s];
  p.A = A;
  p.L = 0;
  while ((1 << p.L) < A) ++p.L;
  for (int g = 0; g <= p.L; ++g) {
    const uint32_t S = 1u << g;
    LevelGeom& lg = p.grid[g];
    for (int s = 0; s < 3; ++s) {
      lg.m[s] = p.interp[s] ? (p.n[s] + S - 1) / S : p.n[s];
      lg.step[s] = p.interp[s] ? S : 1u;
      lg.fst[s] = p.fst[s];
    }
    lg.gst[2] = 1;
    lg.gst[1] = lg.m[2];
    lg.gst[0] = lg.m[1] * lg.m[2];
    p.gsize[g] = lg.m[0] * lg.m[1] * lg.m[2];
  }
  return HPEZ_OK;
}

int check_config(const Plan& p, const hpez_config& c) {
  if (!pow2(c.chunk_syms) || c.chunk_syms < 256 || c.chunk_syms > 32768)
    return HPEZ_ERR_INVALID_ARG;
  if (!(c.alpha >= 1.0) || !(c.beta >= 1.0) || !std::isfinite(c.alpha) ||
      !std::isfinite(c.beta))
    return HPEZ_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d)
    if (!(c.md_inv_var[d] > 0.0) || !std::isfinite(c.md_inv_var[d]))
      return HPEZ_ERR_INVALID_ARG;
  if (c.blockwise && c.block_size < 1) return HPEZ_ERR_INVALID_ARG;
  if (c.predictor < 0 || c.predictor > 2 || (c.predictor && c.blockwise))
    return HPEZ_ERR_INVALID_ARG;
  for (int l = 0; l < p.L; ++l) {
    if (c.interp[l] > HPEZ_SPLINE_GLOBAL || c.paradigm[l] > HPEZ_PARADIGM_MD ||
        c.same_level[l] > 1)
      return HPEZ_ERR_INVALID_ARG;
    // the global spline runs along whole lines: one direction per pass
    if (c.interp[l] == HPEZ_SPLINE_GLOBAL &&
        (c.paradigm[l] != HPEZ_PARADIGM_1D || c.same_level[l] || c.blockwise))
      return HPEZ_ERR_INVALID_ARG;
    bool seen[3] = {false, false, false};
    for (int j = 0; j < p.k; ++j) {
      const int d = c.order[l][j];
      if (d >= p.ndim || !p.interp[d + p.off] || seen[d])
        return HPEZ_ERR_INVALID_ARG;
      seen[d] = true;
    }
  }
  return HPEZ_OK;
}

void plan_chunks_blocks(Plan& p, const hpez_config& c) {
  p.C = (uint32_t)c.chunk_syms;
  p.nch = (uint32_t)(((uint64_t)p.N + p.C - 1) / p.C);
  p.nblocks = 0;
  for (int s = 0; s < 3; ++s) p.nb[s] = 1;
  if (c.blockwise) {
    uint64_t t = 1;
    for (int s = 0; s < 3; ++s) {
      p.nb[s] = (p.n[s] + (uint32_t)c.block_size - 1) / (uint32_t)c.block_size;
      t *= p.nb[s];
    }
    p.nblocks = (uint32_t)t;
  }
}

// Eq. 14 weight of slot d within the slot mask S (sum over ascending dims
// in double, one rounding)
float md_weight(const Plan& p, const hpez_config& c, unsigned S, int slot) {
  double sum = 0.0;
  for (int s = 0; s < 3; ++s)
    if (S & (1u << s)) sum = sum + c.md_inv_var[s - p.off];
  return (float)(c.md_inv_var[slot - p.off] / sum);
}

// The launches of one level: for the 1D-style paradigm one box per pass
// (order pi: odd on pi_j, any parity on earlier dims, even on later ones);
// for the multi-dimensional paradigm one box per odd-slot set S, grouped by
// |S|.  Each (pass, half) is a launch; launches run in list order.

std::vector<Launch> level_schedule(const Plan& p, const hpez_config& c,
                                   int l) {
  std::vector<Launch> out;
  const LevelGeom& g = p.grid[l - 1];
  const bool halves =
      c.blockwise || (c.interp[l - 1] != HPEZ_LINEAR && c.same_level[l - 1]);
  const bool md = c.paradigm[l - 1] == HPEZ_PARADIGM_MD;
  std::vector<std::vector<unsigned>> groups;  // odd-slot masks per group
  if (!md) {
    for (int j = 0; j < p.k; ++j) groups.push_back({1u << (c.order[l - 1][j] + p.off)});
  } else {
    for (int kp = 1; kp <= p.k; ++kp) {
      std::vector<unsigned> gs;
      for (unsigned S = 1; S < 8; ++S) {
        bool ok = true;
        int cnt = 0;
        for (int s = 0; s < 3; ++s)
          if (S & (1u << s)) {
            if (!p.interp[s]) ok = false;
            ++cnt;
          }
        if (ok && cnt == kp) gs.push_back(S);
      }
      groups.push_back(gs);
    }
  }
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    for (int half = 0; half < (halves ? 2 : 1); ++half) {
      for (unsigned S : groups[gi]) {
        PassBox pb;
        std::memset(&pb, 0, sizeof(pb));
        uint64_t tot = 1;
        for (int s = 0; s < 3; ++s) {
          const uint32_t m = g.m[s];
          int kind;  // 0 any, 1 odd, 2 even
          if (!p.interp[s]) {
            kind = 0;
          } else if (S & (1u << s)) {
            kind = 1;
          } else if (md) {
            kind = 2;
          } else {
            // 1D-style: earlier dims of the order any, later ones even
            int pos_s = -1, pos_j = -1;
            for (int j = 0; j < p.k; ++j) {
              if (c.order[l - 1][j] + p.off == s) pos_s = j;
              if ((1u << (c.order[l - 1][j] + p.off)) == S) pos_j = j;
            }
            kind = pos_s < pos_j ? 0 : 2;
          }
          if (kind == 0) {
            pb.a[s] = 0; pb.b[s] = 1; pb.cnt[s] = m;
          } else if (kind == 1) {
            pb.a[s] = 1; pb.b[s] = 2; pb.cnt[s] = m / 2;
          } else {
            pb.a[s] = 0; pb.b[s] = 2; pb.cnt[s] = (m + 1) / 2;
          }
          tot *= pb.cnt[s];
        }
        pb.total = (uint32_t)tot;
        pb.S = S;
        pb.md = md ? 1 : 0;
        for (int s = 0; s < 3; ++s)
          pb.w[s] = (md && (S & (1u << s))) ? md_weight(p, c, S, s) : 0.0f;
        pb.half = half;
        pb.level = l;
        pb.write_recon = 1;
        out.push_back({pb, (int)(gi * 2 + half)});
      }
    }
  }
  if (l == 1 && !out.empty()) {
    // the last group of the finest level is never read again
    const int last = out.back().group;
    for (auto& L : out)
      if (L.group == last) L.pb.write_recon = 0;
  }
  return out;
}

// ---------------------------------------------------------------------
// fused level plan (1D-style paradigm): tile extents and, per pass and
// half, the box of points to compute relative to the tile.  Working back
// from the last pass: pass j's half B is needed on R_B(j), its half A on
// R_A(j) = R_B(j) grown by 2 along pi_j (same-level neighbours at +-2s),
// and every earlier pass on R_B(j-1) = R_A(j) grown by 3 along pi_j
// (neighbours at +-s, +-3s).
// ---------------------------------------------------------------------
bool plan_fused(const hpez_ctx* ctx, const Plan& p, const hpez_config& c,
                int l, bool decomp, FusedLevel& F) {
  if (c.paradigm[l - 1] == HPEZ_PARADIGM_MD || p.k == 0) return false;
  std::memset(&F, 0, sizeof(F));
  F.g = p.grid[l - 1];
  F.gc = p.grid[l];
  const bool sl =
      c.blockwise || (c.interp[l - 1] != HPEZ_LINEAR && c.same_level[l - 1]);
  int pi[3];
  for (int j = 0; j < p.k; ++j) pi[j] = c.order[l - 1][j] + p.off;
  int hA[3][3], hB[3][3];  // halo per pass j and slot
  for (int s = 0; s < 3; ++s) hB[p.k - 1][s] = 0;
  for (int j = p.k - 1; j >= 0; --j) {
    for (int s = 0; s < 3; ++s) hA[j][s] = hB[j][s];
    if (sl) hA[j][pi[j]] += 2;
    if (j > 0) {
      for (int s = 0; s < 3; ++s) hB[j - 1][s] = hA[j][s];
      hB[j - 1][pi[j]] += 3;
    }
  }
  const uint32_t* m = F.g.m;
  for (int s = 0; s < 3; ++s) F.interp[s] = p.interp[s] ? 1 : 0;
  // tile extents: long along the fastest slot, thin along the slowest
  uint32_t E[3];
  const bool one_d = m[0] == 1 && m[1] == 1;
  E[2] = one_d ? std::min<uint32_t>(m[2], 4096) : (m[2] <= 512 ? m[2] : 256);
  E[1] = std::min<uint32_t>(m[1], 8);
  E[0] = std::min<uint32_t>(m[0], 2);
  for (int s = 0; s < 3; ++s)
    if (ctx->tile_e[s] > 0) E[s] = std::min<uint32_t>(m[s], (uint32_t)ctx->tile_e[s]);
  auto fix_even = [&](int s) {
    if (p.interp[s] && E[s] < m[s] && (E[s] & 1)) E[s] += 1;
    if (E[s] < 1) E[s] = 1;
  };
  for (int s = 0; s < 3; ++s) fix_even(s);
  // a slot the tile covers whole needs no halo
  auto halo = [&](int s) { return E[s] >= m[s] ? 0 : hA[0][s]; };
  auto smem = [&]() {
    size_t b = decomp ? 6 : 4;  // decompress stages the codes as well
    for (int s = 0; s < 3; ++s)
      b *= (size_t)(E[s] + 2 * halo(s) + (s == 2 ? 14 : 0));
    return b;
  };
  while (smem() > ctx->fused_smem_cap) {
    int big = 2;
    for (int s = 0; s < 3; ++s)
      if (E[s] > E[big]) big = s;
    if (E[big] <= 2) return false;
    E[big] = (E[big] / 2) & ~1u;
    if (E[big] < 2) E[big] = 2;
    fix_even(big);
  }
  uint64_t nt = 1;
  for (int s = 0; s < 3; ++s) {
    F.E[s] = E[s];
    // along the fastest slot the region is padded to multiples of 8
    // columns, so staged rows start on 16-byte (8-code) boundaries
    const int h = s == 2 ? ((halo(s) + 7) & ~7) : halo(s);
    F.rlo[s] = -h;
    F.rhi[s] = (int)E[s] + h;
    if (s == 2) F.rhi[s] = F.rlo[s] + (((F.rhi[s] - F.rlo[s]) + 7) & ~7);
    F.RX[s] = (uint32_t)(F.rhi[s] - F.rlo[s]);
    F.ntile[s] = (m[s] + E[s] - 1) / E[s];
    nt *= F.ntile[s];
  }
  if (nt > 0x7FFFFFFFull) return false;
  F.ntiles = (uint32_t)nt;
  F.nsteps = 0;
  for (int j = 0; j < p.k; ++j) {
    for (int half = 0; half < (sl ? 2 : 1); ++half) {
      FusedStep& S = F.st[F.nsteps++];
      std::memset(&S, 0, sizeof(S));
      S.dim = (int8_t)pi[j];
      S.half = (int8_t)half;
      for (int s = 0; s < 3; ++s) {
        const int h = half == 0 ? hA[j][s] : hB[j][s];
        S.lo[s] = (int16_t)(-h);
        S.hi[s] = (int16_t)((int)E[s] + h);
        S.par[s] = 0;  // non-interpolation slots and earlier directions
      }
      S.par[pi[j]] = 1;
      for (int m2 = j + 1; m2 < p.k; ++m2) S.par[pi[m2]] = 2;
      // passes after the first read only points computed in the region;
      // the first pass's +-s, +-3s neighbours may be coarse points outside
      S.pad_[0] = (int8_t)(j > 0 ? 1 : 0);
    }
  }
  F.level = l;
  F.write_recon = (decomp || l > 1) ? 1 : 0;
  // staging: rows of the level grid are contiguous in the full field only
  // at stride 1 along the fastest slot; 16-byte copies need rows, the tile
  // and the region to start on 16-byte boundaries
  F.stage_x = 0;
  const bool contig = F.g.step[2] == 1;
  const bool al4 = (p.n[2] % 4 == 0) && (F.g.m[2] == p.n[2]) && (F.E[2] % 4 == 0 || F.E[2] >= m[2]);
  const bool al8 = (p.n[2] % 8 == 0) && (F.g.m[2] == p.n[2]) && (F.E[2] % 8 == 0 || F.E[2] >= m[2]);
  if (!decomp) {
    F.stage_x = (contig && al4 && ctx->x_aligned16) ? 2 : 1;
  } else {
    F.stage_x = (contig && al8 && ctx->codes_aligned16) ? 1 : 0;
  }
  return true;
}

// The dedicated 3D kernel applies to levels of a 3D field with no frozen
// dimension, the 1D-style order (0, 1, 2), one interpolator and no
// same-level halves; whole rows along dim 2 must fit shared memory.
bool plan_level3d(const hpez_ctx* ctx, const Plan& p, const hpez_config& c,
                  int l, bool decomp, Level3D& F) {
  if (!ctx->level3d || p.ndim != 3 || p.k != 3 || c.blockwise) return false;
  if (c.paradigm[l - 1] != HPEZ_PARADIGM_1D) return false;
  if (c.order[l - 1][0] != 0 || c.order[l - 1][1] != 1 || c.order[l - 1][2] != 2)
    return false;
  if (c.interp[l - 1] != HPEZ_LINEAR && c.same_level[l - 1]) return false;
  const LevelGeom& g = p.grid[l - 1];
  const LevelGeom& gc = p.grid[l];
  if (g.m[2] < 8) return false;
  std::memset(&F, 0, sizeof(F));
  for (int s = 0; s < 3; ++s) F.m[s] = (int)g.m[s];
  // whole rows of the level grids start on 16-byte boundaries when the
  // row length is a multiple of 4 (the arena aligns every grid to 256 B)
  F.vec_out = (g.m[2] % 4 == 0 && (l > 1 || !decomp || ctx->out_aligned16)) ? 1 : 0;
  F.E1 = ctx->tile_e[1] > 0 ? ctx->tile_e[1] : 8;
  if (F.E1 & 1) F.E1 += 1;
  F.W = (F.m[2] + 7) & ~7;
  F.fs0 = g.step[0] * g.fst[0];
  F.fs1 = g.step[1] * g.fst[1];
  F.fs2 = g.step[2];
  F.cst0 = gc.gst[0];
  F.cst1 = gc.gst[1];
  F.level = l;
  F.write_recon = (decomp || l > 1) ? 1 : 0;
  const bool contig = g.step[2] == 1;
  F.stage16 = (!decomp && contig && (p.n[2] % 4 == 0) && ctx->x_aligned16) ? 1 : 0;
  F.stage_codes = (decomp && contig && (p.n[2] % 8 == 0) && ctx->codes_aligned16) ? 1 : 0;
  while (level3d_smem_bytes(F, decomp) > ctx->fused_smem_cap && F.E1 > 2) F.E1 -= 2;
  if (level3d_smem_bytes(F, decomp) > ctx->fused_smem_cap) return false;
  F.nt0 = (F.m[0] + 1) / 2;
  F.nt1 = (F.m[1] + F.E1 - 1) / F.E1;
  if ((uint64_t)F.nt0 * (uint64_t)F.nt1 > 0x7FFFFFFFull) return false;
  return true;
}

// ---------------------------------------------------------------------
// scratch arena
// ---------------------------------------------------------------------

int ensure_scratch(hpez_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->scratch_cap) return HPEZ_OK;
  if (ctx->scratch) {
    cudaDeviceSynchronize();
    cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_cap = 0;
  }
  size_t want = bytes + bytes / 8;
  if (cudaMalloc(&ctx->scratch, want) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&ctx->scratch, bytes) != cudaSuccess) {
      cudaGetLastError();
      ctx->scratch = nullptr;
      return HPEZ_ERR_NO_MEMORY;
    }
    want = bytes;
  }
  ctx->scratch_cap = want;
  return HPEZ_OK;
}

int map_status(int st) {
  switch (st) {
    case ST_OK: return HPEZ_OK;
    case ST_INVALID: return HPEZ_ERR_INVALID_ARG;
    case ST_NONFINITE: return HPEZ_ERR_NONFINITE_INPUT;
    case ST_OUT_TOO_SMALL: return HPEZ_ERR_OUT_TOO_SMALL;
    case ST_CORRUPT: return HPEZ_ERR_CORRUPT_STREAM;
    case ST_TIMEOUT: return HPEZ_ERR_TIMEOUT;
  }
  return HPEZ_ERR_CUDA;
}

int cuda_check(cudaError_t e) {
  if (e == cudaSuccess) return HPEZ_OK;
  // HPEZ_DEBUG_CUDA=1 in the environment names the runtime error on stderr
  static const bool dbg = std::getenv("HPEZ_DEBUG_CUDA") != nullptr;
  if (dbg) std::fprintf(stderr, "hpez: CUDA runtime error %s\n", cudaGetErrorName(e));
  if (e == cudaErrorMemoryAllocation) return HPEZ_ERR_NO_MEMORY;
  return HPEZ_ERR_CUDA;
}

void default_config(int ndim, hpez_config* c) {
  std::memset(c, 0, sizeof(*c));
  c->anchor_stride = ndim == 1 ? 128 : (ndim == 2 ? 64 : 32);
  c->frozen_dim = -1;
  c->chunk_syms = 16384;
  c->blockwise = 0;
  c->block_size = 32;
  c->alpha = 1.0;
  c->beta = 1.0;
  for (int d = 0; d < 3; ++d) c->md_inv_var[d] = 1.0;
  for (int l = 0; l < HPEZ_MAX_LEVELS; ++l) {
    c->interp[l] = HPEZ_CUBIC_NAK;
    c->paradigm[l] = HPEZ_PARADIGM_1D;
    c->same_level[l] = 0;
    for (int j = 0; j < 3; ++j) c->order[l][j] = (uint8_t)(j < ndim ? j : 255);
  }
}

// A level of the multi-dimensional paradigm with one interpolator for every
// point and no same-level halves runs as one launch per sub-pass.
bool plan_md(const hpez_ctx* ctx, const Plan& p, const hpez_config& c, int l,
             bool decomp, LevelMD& F) {
  if (!ctx->fused_levels || c.paradigm[l - 1] != HPEZ_PARADIGM_MD || p.k == 0)
    return false;
  if (c.blockwise) return false;
  if (c.same_level[l - 1] && c.interp[l - 1] != HPEZ_LINEAR) return false;
  std::memset(&F, 0, sizeof(F));
  F.g = p.grid[l - 1];
  F.gc = p.grid[l];
  unsigned imask = 0;
  for (int s = 0; s < 3; ++s) {
    F.interp[s] = p.interp[s] ? 1 : 0;
    F.nc[s] = F.gc.m[s];
    F.fst[s] = p.fst[s];
    if (p.interp[s]) imask |= 1u << s;
  }
  F.k = p.k;
  F.level = l;
  F.write_recon = (decomp || l > 1) ? 1 : 0;
  for (unsigned S = 1; S < 8; ++S) {
    if ((S & imask) != S) continue;
    const int kk = __builtin_popcount(S);
    F.masks[kk - 1][F.nmask[kk - 1]++] = (uint8_t)S;
    for (int s = 0; s < 3; ++s)
      if (S & (1u << s)) F.w[S][s] = md_weight(p, c, S, s);
  }
  return true;
}

// A 3D multi-dimensional level with every dimension interpolated runs as
// two launches (even planes, odd planes) of row tiles E1 rows high.
bool plan_md3(const hpez_ctx* ctx, const Plan& p, const hpez_config& c, int l,
              bool decomp, LevelMD& F, int& E1) {
  if (p.ndim != 3 || p.k != 3) return false;
  if (!plan_md(ctx, p, c, l, decomp, F)) return false;
  if (F.g.m[0] < 2 || F.g.m[1] < 2 || F.g.m[2] < 2) return false;
  E1 = ctx->tile_e[1] > 0 ? ((ctx->tile_e[1] + 1) & ~1) : 16;
  while (E1 > 2 && md3_smem_bytes(F, E1) > 96 * 1024) E1 /= 2;
  return md3_smem_bytes(F, E1) <= 160 * 1024;
}

// A block map whose blocks all carry the same interpolator is the same
// predictor as that interpolator (and same-level flag) at every level.
bool uniform_blockmap(const uint8_t* bm, uint32_t n, uint8_t* v) {
  if (!bm || n == 0) return false;
  for (uint32_t i = 1; i < n; ++i)
    if (bm[i] != bm[0]) return false;
  *v = bm[0];
  return true;
}

hpez_config sweep_config(const hpez_config& c, const uint8_t* h_bmap,
                         uint32_t nblocks) {
  hpez_config r = c;
  uint8_t v;
  if (c.blockwise && uniform_blockmap(h_bmap, nblocks, &v)) {
    r.blockwise = 0;
    for (int l = 0; l < HPEZ_MAX_LEVELS; ++l) {
      r.interp[l] = (uint8_t)((v & 3u) > HPEZ_CUBIC_NAT ? HPEZ_CUBIC_NAT : (v & 3u));
      r.same_level[l] = (uint8_t)((v >> 2) & 1u);
    }
  }
  return r;
}

uint64_t n_anchors(const Plan& p) { return p.gsize[p.L]; }

void header_templates(const Plan& p, const hpez_config& c, int eb_mode,
                      double eb, uint64_t off_anchors, uint64_t off_bmap,
                      uint64_t off_chw, uint8_t* h, uint8_t* hc) {
  std::memset(h, 0, kHeaderBytes);
  std::memset(hc, 0, kHeaderBytes);
  for (uint8_t* b : {h, hc}) {
    wr32(b, H_MAGIC, kMagic);
    wr32(b, H_VERSION, kVersion);
    wr32(b, H_NDIM, (uint32_t)p.ndim);
    for (int d = 0; d < 3; ++d)
      wr64(b, H_DIMS + 8 * d, d < p.ndim ? p.n[d + p.off] : 1);
    wr32(b, H_EBMODE, (uint32_t)eb_mode);
    wr32(b, H_ANCHOR, (uint32_t)c.anchor_stride);
    wrf64(b, H_EBVALUE, eb);
    wr32(b, H_CHUNK, (uint32_t)c.chunk_syms);
  }
  // constant field: no sections
  wr32(hc, H_FLAGS, 1u);
  wr32(hc, H_FROZEN, 0xFFFFFFFFu);
  for (int o = H_OFF_ANCHORS; o <= H_OFF_BLOCKMAP; o += 8) wr64(hc, o, kHeaderBytes);
  wr64(hc, H_TOTAL, kHeaderBytes);
  // regular stream: static fields (the device patches e, counts, offsets)
  wr32(h, H_FROZEN, (uint32_t)c.frozen_dim);
  wrf64(h, H_ALPHA, c.alpha);
  wrf64(h, H_BETA, c.beta);
  for (int d = 0; d < 3; ++d) wrf64(h, H_MDIV + 8 * d, c.md_inv_var[d]);
  for (int l = 0; l < kMaxLevels; ++l) {
    const bool used = l < p.L;
    h[H_INTERP + l] = used ? c.interp[l] : 0;
    h[H_PARADIGM + l] = used ? c.paradigm[l] : 0;
    h[H_SAME + l] = used ? c.same_level[l] : 0;
    for (int j = 0; j < 3; ++j)
      h[H_ORDER + 3 * l + j] = (used && j < p.k) ? c.order[l][j] : 255;
  }
  wr32(h, H_PREDICTOR, (uint32_t)c.predictor);
  wr32(h, H_BLOCKWISE, (uint32_t)c.blockwise);
  wr64(h, H_NANCHORS, c.predictor ? 0 : n_anchors(p));
  wr32(h, H_BLOCKSIZE, (uint32_t)c.block_size);
  wr64(h, H_NCHUNKS, p.nch);
  wr64(h, H_OFF_ANCHORS, off_anchors);
  wr64(h, H_OFF_CHUNKW, off_chw);
  wr64(h, H_OFF_BLOCKMAP, off_bmap);
  wr64(h, H_NBLOCKS, p.nblocks);
}

struct CompressBufs {
  Ctl* ctl;
  uint32_t* hist;
  unsigned long long* enc;
  uint16_t* tsyms;
  uint8_t* tlens;
  uint8_t* lens_by_sym;
  unsigned long long* gkeys;
  unsigned long long* giw;
  uint32_t* gpar;
  float* R[kMaxLevels + 1];
  uint16_t* Cg[kMaxLevels + 1];
  uint32_t* zc;
  unsigned long long* zoff;
  uint32_t* chw;
  unsigned long long* woff;
  uint16_t* lbits;
  uint8_t* bmap;
  unsigned long long* flags;  // the one-pass encode's chunk flags + counter
};


// Reads and validates a stream header (host copy of its first 512 bytes).
int parse_stream_header(const uint8_t* h, uint64_t in_size, StreamInfo& si) {
  si = StreamInfo();  // value-initialized: the plan keeps its defaults
  int nd;
  uint64_t dims[3];
  int rc = hpez_inspect(h, kHeaderBytes, &nd, dims, nullptr);
  if (rc) return rc;
  if (rd64(h, H_TOTAL) > in_size) return HPEZ_ERR_CORRUPT_STREAM;
  uint64_t N = 1;
  for (int d = 0; d < nd; ++d) {
    if (dims[d] == 0) return HPEZ_ERR_CORRUPT_STREAM;
    N *= dims[d];
    if (N > 0xFFFFFFFFull) return HPEZ_ERR_CORRUPT_STREAM;
  }
  si.nd = nd;
  for (int d = 0; d < 3; ++d) si.dims[d] = d < nd ? dims[d] : 1;
  si.N = N;
  hpez_config& cfg = si.cfg;
  cfg.anchor_stride = (int32_t)rd32(h, H_ANCHOR);
  cfg.frozen_dim = (int32_t)rd32(h, H_FROZEN);
  cfg.chunk_syms = (int32_t)rd32(h, H_CHUNK);
  cfg.blockwise = (int32_t)rd32(h, H_BLOCKWISE);
  cfg.block_size = (int32_t)rd32(h, H_BLOCKSIZE);
  cfg.predictor = (int32_t)rd32(h, H_PREDICTOR);
  cfg.alpha = rdf64(h, H_ALPHA);
  cfg.beta = rdf64(h, H_BETA);
  for (int d = 0; d < 3; ++d) cfg.md_inv_var[d] = rdf64(h, H_MDIV + 8 * d);
  for (int l = 0; l < HPEZ_MAX_LEVELS; ++l) {
    cfg.interp[l] = h[H_INTERP + l];
    cfg.paradigm[l] = h[H_PARADIGM + l];
    cfg.same_level[l] = h[H_SAME + l];
    for (int j = 0; j < 3; ++j) cfg.order[l][j] = h[H_ORDER + 3 * l + j];
  }
  if (rd32(h, H_FLAGS) & 1u) {
    // constant field
    if (plan_geometry(si.p, nd, dims, 2, -1)) return HPEZ_ERR_CORRUPT_STREAM;
    si.is_const = true;
    si.const_value = rdf32(h, H_CONST);
    return HPEZ_OK;
  }
  Plan& p = si.p;
  if (plan_geometry(p, nd, dims, cfg.anchor_stride, cfg.frozen_dim))
    return HPEZ_ERR_CORRUPT_STREAM;
  if (check_config(p, cfg)) return HPEZ_ERR_CORRUPT_STREAM;
  plan_chunks_blocks(p, cfg);
  const float e = rdf32(h, H_E);
  if (!(e > 0.0f) || !std::isfinite(e)) return HPEZ_ERR_CORRUPT_STREAM;
  si.e = e;
  const uint64_t na = rd64(h, H_NANCHORS), nout = rd64(h, H_NOUTLIERS),
                 nch = rd64(h, H_NCHUNKS), twords = rd64(h, H_TOTALWORDS);
  const uint32_t nused = rd32(h, H_NUSED);
  const uint64_t oa = rd64(h, H_OFF_ANCHORS), ocw = rd64(h, H_OFF_CHUNKW),
                 ot = rd64(h, H_OFF_TABLE), oo = rd64(h, H_OFF_OUTLIERS),
                 ob = rd64(h, H_OFF_BITS), obm = rd64(h, H_OFF_BLOCKMAP);
  if (na != (cfg.predictor ? 0 : n_anchors(p)) || nch != p.nch || nused == 0 ||
      nused > 65536 || nout > N || (cfg.blockwise && rd64(h, H_NBLOCKS) != p.nblocks))
    return HPEZ_ERR_CORRUPT_STREAM;
  if (oa + 4 * na > in_size || ocw + 64 * nch > in_size ||
      ot + 3ull * nused > in_size || oo + 4 * nout > in_size ||
      ob + 4 * twords > in_size || (cfg.blockwise && obm + p.nblocks > in_size) ||
      (oa & 15) || (ocw & 15) || (oo & 15) || (ob & 15))
    return HPEZ_ERR_CORRUPT_STREAM;
  si.na = na;
  si.nout = nout;
  si.nch = nch;
  si.twords = twords;
  si.nused = nused;
  si.oa = oa;
  si.ocw = ocw;
  si.ot = ot;
  si.oo = oo;
  si.ob = ob;
  si.obm = obm;
  return HPEZ_OK;
}
int ensure_io(void** buf, size_t* cap, size_t bytes) {
  if (bytes <= *cap) return HPEZ_OK;
  if (*buf) {
    cudaDeviceSynchronize();
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
  }
  if (cudaMalloc(buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return HPEZ_ERR_NO_MEMORY;
  }
  *cap = bytes;
  return HPEZ_OK;
}

}  // namespace host
}  // namespace hpez

using namespace hpez::host;

// =====================================================================
// C-ABI
// =====================================================================
extern "C" {

const char* hpez_strerror(int code) {
  switch (code) {
    case HPEZ_OK: return "ok";
    case HPEZ_ERR_INVALID_ARG: return "invalid argument";
    case HPEZ_ERR_NONFINITE_INPUT: return "non-finite input with a relative bound";
    case HPEZ_ERR_OUT_TOO_SMALL: return "output buffer too small";
    case HPEZ_ERR_CORRUPT_STREAM: return "corrupt or unsupported stream";
    case HPEZ_ERR_NO_MEMORY: return "device allocation failed";
    case HPEZ_ERR_CUDA: return "CUDA runtime error";
    case HPEZ_ERR_UNSUPPORTED: return "unsupported configuration";
    case HPEZ_ERR_TIMEOUT: return "bounded device wait timed out";
    case HPEZ_ERR_TOO_LARGE:
      return "field larger than the fixed scratch of the no-allocation entry point";
  }
  return "unknown error";
}

int hpez_profile_enable(hpez_ctx* ctx, int enable) {
  if (!ctx) return HPEZ_ERR_INVALID_ARG;
  ctx->prof.reset();
  ctx->prof.on = enable != 0;
  ctx->launches = 0;
  return HPEZ_OK;
}

int hpez_profile_get(hpez_ctx* ctx, int phase, double* total_ms,
                     uint64_t* count) {
  if (!ctx || phase < 0 || phase >= HPEZ_PROFILE_PHASES) return HPEZ_ERR_INVALID_ARG;
  if (total_ms) *total_ms = ctx->prof.total_ms[phase];
  if (count) *count = ctx->prof.count[phase];
  return HPEZ_OK;
}

int hpez_set_option(hpez_ctx* ctx, int option, int64_t value) {
  if (!ctx) return HPEZ_ERR_INVALID_ARG;
  switch (option) {
    case HPEZ_OPT_FUSED_LEVELS:
      ctx->fused_levels = value != 0;
      return HPEZ_OK;
    case HPEZ_OPT_TILE_E0:
    case HPEZ_OPT_TILE_E1:
    case HPEZ_OPT_TILE_E2:
      if (value < 0 || value > 4096) return HPEZ_ERR_INVALID_ARG;
      ctx->tile_e[option - HPEZ_OPT_TILE_E0] = (int)value;
      return HPEZ_OK;
    case HPEZ_OPT_LEVEL3D:
      ctx->level3d = value != 0;
      return HPEZ_OK;
    case HPEZ_OPT_STREAM_LEVELS:
      ctx->stream_levels = value != 0;
      return HPEZ_OK;
    case HPEZ_OPT_DROP_COPY:
      if (value < 0 || value > 1000000) return HPEZ_ERR_INVALID_ARG;
      ctx->drop_copy = (int)value;
      return HPEZ_OK;
    case HPEZ_OPT_WARP_LEVELS:
      ctx->warp_levels = value != 0;
      return HPEZ_OK;
    case HPEZ_OPT_STREAM_CHUNKS:
      if (value < 0 || value > 1000000) return HPEZ_ERR_INVALID_ARG;
      ctx->stream_chunks = (int)value;
      return HPEZ_OK;
    case HPEZ_OPT_LORENZO_CTAS:
      if (value < 0 || value > 1000000) return HPEZ_ERR_INVALID_ARG;
      ctx->lorenzo_ctas = (int)value;
      return HPEZ_OK;
    case HPEZ_OPT_BATCH_CTAS:
      if (value < 0 || value > 1000000) return HPEZ_ERR_INVALID_ARG;
      ctx->batch_ctas = (int)value;
      return HPEZ_OK;
    case HPEZ_OPT_FUSED_SMEM:
      if (value < 4096 || value > 200 * 1024) return HPEZ_ERR_INVALID_ARG;
      ctx->fused_smem_cap = (size_t)value;
      return HPEZ_OK;
  }
  return HPEZ_ERR_INVALID_ARG;
}

int hpez_launch_count(hpez_ctx* ctx, uint64_t* launches) {
  if (!ctx || !launches) return HPEZ_ERR_INVALID_ARG;
  *launches = ctx->launches;
  return HPEZ_OK;
}

const char* hpez_profile_phase_name(int phase) {
  static const char* fixed[] = {"range", "anchors", "hist", "codebook",
                                "encode_len", "pack", "outliers", "finalize",
                                "dec_prep", "decode", "scatter"};
  static char names[HPEZ_PROFILE_PHASES][24];
  if (phase < 0 || phase >= HPEZ_PROFILE_PHASES) return "";
  if (phase < HPEZ_PH_LEVEL) return fixed[phase];
  if (phase >= HPEZ_PH_TUNE_STATS) {
    static const char* tune[] = {"tune_stats", "tune_levels", "tune_eb",
                                 "tune_lorenzo", "tune_blocks"};
    return tune[phase - HPEZ_PH_TUNE_STATS];
  }
  if (phase < HPEZ_PH_DLEVEL)
    std::snprintf(names[phase], 24, "level%d", phase - HPEZ_PH_LEVEL + 1);
  else
    std::snprintf(names[phase], 24, "dlevel%d", phase - HPEZ_PH_DLEVEL + 1);
  return names[phase];
}

int hpez_default_config(int ndim, hpez_config* out) {
  if (!out || ndim < 1 || ndim > 3) return HPEZ_ERR_INVALID_ARG;
  default_config(ndim, out);
  return HPEZ_OK;
}

int hpez_create(hpez_ctx** out, int device) {
  if (!out) return HPEZ_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return HPEZ_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return HPEZ_ERR_CUDA;
  hpez_ctx* c = new hpez_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMallocHost(&c->h_ctl, sizeof(Ctl)) != cudaSuccess ||
      cudaMallocHost(&c->h_hdr, kHeaderBytes) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return HPEZ_ERR_NO_MEMORY;
  }
  *out = c;
  return HPEZ_OK;
}

int hpez_destroy(hpez_ctx* ctx) {
  if (!ctx) return HPEZ_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->io_in) cudaFree(ctx->io_in);
  if (ctx->io_out) cudaFree(ctx->io_out);
  if (ctx->typed_buf) cudaFree(ctx->typed_buf);
  if (ctx->typed_red) cudaFree(ctx->typed_red);
  if (ctx->lz_buf) cudaFree(ctx->lz_buf);
  if (ctx->lz_stream) cudaFree(ctx->lz_stream);
  if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
  if (ctx->h_hdr) cudaFreeHost(ctx->h_hdr);
  if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
  for (int i = 0; i < 2; ++i)
    if (ctx->aux_ev[i]) cudaEventDestroy(ctx->aux_ev[i]);
  delete ctx;
  return HPEZ_OK;
}

int hpez_compress_bound(int ndim, const uint64_t* dims, uint64_t* out_bytes) {
  if (!dims || !out_bytes || ndim < 1 || ndim > 3) return HPEZ_ERR_INVALID_ARG;
  uint64_t N = 1;
  for (int d = 0; d < ndim; ++d) {
    if (dims[d] == 0) return HPEZ_ERR_INVALID_ARG;
    N *= dims[d];
  }
  const uint64_t nch = (N + 255) / 256;
  *out_bytes = 512 + 16 * 8 + 4 * N + 4 * N + N + 64 * nch + 3 * 65536 + 4 +
               (17 * N) / 8 + 4 * nch + 64;
  return HPEZ_OK;
}

// A level's chunk count for the warp-strip kernel from the context's
// schedule table (searched offline), unless HPEZ_OPT_STREAM_CHUNKS is set.
// The single-field calls take only that from the table: the batched
// form's persistent launches of the other families favour other tile
// shapes than one CTA per tile.  A decompress level without a warp-strip
// entry takes the compress level's.
struct LevelSchedScope {
  int chunks;
  LevelSchedScope(const hpez_ctx* c, const Plan& p, const hpez_config& kc, int l, bool decomp)
      : chunks(c->stream_chunks) {
    if (c->stream_chunks || c->sched.m.empty()) return;
    for (int d = decomp ? 1 : 0; d >= 0; --d) {
      std::array<int32_t, 8> k = sched_key(p, kc, l, decomp);
      k[7] = d;
      const auto it = c->sched.m.find(k);
      if (it != c->sched.m.end() && it->second.family == HPEZ_FAM_MD3W) {
        chunks = it->second.chunks;
        return;
      }
    }
  }
};

// The compress launch sequence.  Synchronous (d_status null): the size
// comes back in *h_out_size.  Asynchronous: a last kernel writes the size
// and the status to *d_size / *d_status and nothing waits.
static int compress_impl(hpez_ctx* ctx, const float* d_in, int ndim, const uint64_t* dims,
                         int eb_mode, double eb, const hpez_config* cfg_in, void* d_out,
                         uint64_t out_cap, uint64_t* h_out_size, unsigned long long* d_size,
                         int* d_status, void* stream) {
  if (!ctx || !d_in || !d_out || (!h_out_size && !d_status)) return HPEZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_out) & 15u) != 0) return HPEZ_ERR_INVALID_ARG;
  if (eb_mode != HPEZ_EB_ABS && eb_mode != HPEZ_EB_REL) return HPEZ_ERR_INVALID_ARG;
  if (!(eb > 0.0) || !std::isfinite(eb)) return HPEZ_ERR_INVALID_ARG;
  hpez_config cfg;
  if (cfg_in)
    cfg = *cfg_in;
  else if (ndim >= 1 && ndim <= 3)
    default_config(ndim, &cfg);
  else
    return HPEZ_ERR_INVALID_ARG;
  Plan p;
  int rc = plan_geometry(p, ndim, dims, cfg.anchor_stride, cfg.frozen_dim);
  if (rc) return rc;
  rc = check_config(p, cfg);
  if (rc) return rc;
  if (cfg.blockwise && !cfg.h_blockmap) return HPEZ_ERR_INVALID_ARG;
  if (cfg.predictor && !lorenzo_supported(p.n, p.fst, p.off, p.A))
    return HPEZ_ERR_UNSUPPORTED;
  // the asynchronous form takes no host memory but the arguments
  if (d_status && cfg.blockwise) return HPEZ_ERR_UNSUPPORTED;
  plan_chunks_blocks(p, cfg);
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ctx->x_aligned16 = (reinterpret_cast<uintptr_t>(d_in) & 15u) == 0;

  // scratch layout
  Arena ar;
  const size_t o_ctl = ar.take<Ctl>(1);
  const size_t o_hist = ar.take<uint32_t>(65536);
  const size_t o_enc = ar.take<unsigned long long>(65536);
  const size_t o_tsyms = ar.take<uint16_t>(65536);
  const size_t o_tlens = ar.take<uint8_t>(65536);
  const size_t o_lbs = ar.take<uint8_t>(65536);
  const size_t o_gkeys = ar.take<unsigned long long>(65536);
  const size_t o_giw = ar.take<unsigned long long>(65536);
  const size_t o_gpar = ar.take<uint32_t>(131072);
  size_t o_R[kMaxLevels + 1], o_C[kMaxLevels + 1];
  for (int g = 0; g <= p.L; ++g) {
    o_R[g] = ar.take<float>(p.gsize[g]);
    // two spare codes: kernels may read a code as the aligned 4-byte word
    // that holds it
    o_C[g] = ar.take<uint16_t>(p.gsize[g] + 2);
  }
  const size_t o_zc = ar.take<uint32_t>(p.nch);
  const size_t o_zoff = ar.take<unsigned long long>(p.nch);
  const size_t o_chw = ar.take<uint32_t>(p.nch);
  const size_t o_woff = ar.take<unsigned long long>(p.nch);
  const size_t o_lbits = ar.take<uint16_t>((size_t)p.nch * 32);
  const size_t o_bmap = ar.take<uint8_t>(p.nblocks + 1);
  const size_t o_flags = ar.take<unsigned long long>((size_t)p.nch + 1);
  rc = ensure_scratch(ctx, ar.off);
  if (rc) return rc;
  char* S = ctx->scratch;
  CompressBufs b;
  b.ctl = reinterpret_cast<Ctl*>(S + o_ctl);
  b.hist = reinterpret_cast<uint32_t*>(S + o_hist);
  b.enc = reinterpret_cast<unsigned long long*>(S + o_enc);
  b.tsyms = reinterpret_cast<uint16_t*>(S + o_tsyms);
  b.tlens = reinterpret_cast<uint8_t*>(S + o_tlens);
  b.lens_by_sym = reinterpret_cast<uint8_t*>(S + o_lbs);
  b.gkeys = reinterpret_cast<unsigned long long*>(S + o_gkeys);
  b.giw = reinterpret_cast<unsigned long long*>(S + o_giw);
  b.gpar = reinterpret_cast<uint32_t*>(S + o_gpar);
  for (int g = 0; g <= p.L; ++g) {
    b.R[g] = reinterpret_cast<float*>(S + o_R[g]);
    b.Cg[g] = reinterpret_cast<uint16_t*>(S + o_C[g]);
  }
  b.zc = reinterpret_cast<uint32_t*>(S + o_zc);
  b.zoff = reinterpret_cast<unsigned long long*>(S + o_zoff);
  b.chw = reinterpret_cast<uint32_t*>(S + o_chw);
  b.woff = reinterpret_cast<unsigned long long*>(S + o_woff);
  b.lbits = reinterpret_cast<uint16_t*>(S + o_lbits);
  b.bmap = reinterpret_cast<uint8_t*>(S + o_bmap);
  b.flags = reinterpret_cast<unsigned long long*>(S + o_flags);

  // stream layout (static part)
  const uint64_t na = cfg.predictor ? 0 : n_anchors(p);
  const uint64_t off_anchors = kHeaderBytes;
  const uint64_t off_bmap = a16(off_anchors + 4 * na);
  const uint64_t off_chw = a16(off_bmap + p.nblocks);
  const uint64_t off_table = a16(off_chw + 64ull * p.nch);
  uint8_t hdr[kHeaderBytes], hdrc[kHeaderBytes];
  header_templates(p, cfg, eb_mode, eb, off_anchors, off_bmap, off_chw, hdr, hdrc);

  // ---- launch sequence ----
  PhaseProfiler& pf = ctx->prof;
  uint64_t& nl = ctx->launches;
  launch_init_ctl(b.ctl, s);
  ++nl;
  if (eb_mode == HPEZ_EB_REL) {
    if (ctx->range_hint_on && ctx->range_x == d_in && ctx->range_n == p.N) {
      launch_set_range(b.ctl, ctx->range_kmin, ctx->range_kmax, s);
    } else {
      pf.begin(HPEZ_PH_RANGE, s);
      launch_range(d_in, p.N, b.ctl, ctx->num_sms, s);
      pf.end(s);
    }
    ++nl;
  }
  launch_params(b.ctl, eb_mode, eb, cfg.alpha, cfg.beta, p.L, d_in, s);
  ++nl;
  if (cfg.blockwise)
    cudaMemcpyAsync(b.bmap, cfg.h_blockmap, p.nblocks, cudaMemcpyHostToDevice, s);
  if (cfg.predictor) {
    // Sec. 6.5: the Lorenzo predictor over the field, codes into the
    // finest grid's code array
    pf.begin(HPEZ_PH_LEVEL, s);
    rc = launch_lorenzo(false, cfg.predictor, p.n, p.fst, p.off, p.A, ctx->x_aligned16,
                        d_in, b.Cg[0], nullptr, b.ctl, ctx->num_sms, ctx->drop_copy,
                        ctx->lorenzo_ctas, s);
    pf.end(s);
    if (rc) return rc;
    ++nl;
  } else {
  pf.begin(HPEZ_PH_ANCHORS, s);
  launch_anchor_gather(d_in, p.grid[p.L], p.gsize[p.L], b.R[p.L], b.Cg[p.L],
                       b.ctl, s);
  pf.end(s);
  ++nl;
  // the predictor the sweep runs (a uniform block map becomes its
  // interpolator); the header keeps the configuration as given
  const hpez_config sc = sweep_config(cfg, cfg.h_blockmap, p.nblocks);
  SweepBufs sb;
  std::memset(&sb, 0, sizeof(sb));
  sb.x = d_in;
  sb.blockmap = sc.blockwise ? b.bmap : nullptr;
  sb.bs = (uint32_t)(cfg.block_size > 0 ? cfg.block_size : 1);
  for (int s3 = 0; s3 < 3; ++s3) sb.nb[s3] = p.nb[s3];
  sb.ctl = b.ctl;
  for (int l = p.L; l >= 1; --l) {
    const int g = l - 1;
    const LevelSchedScope ls(ctx, p, sc, l, false);
    pf.begin(HPEZ_PH_LEVEL + g, s);
    sb.R = b.R[g];
    sb.C = b.Cg[g];
    sb.kind = sc.interp[l - 1];
    sb.same = sc.same_level[l - 1];
    FusedLevel F;
    Level3D F3;
    LevelMD FM;
    int E1 = 0;
    const bool spline = sc.interp[l - 1] == HPEZ_SPLINE_GLOBAL;
    if (!spline && ctx->fused_levels && plan_level3d(ctx, p, sc, l, false, F3)) {
      launch_level3d(false, F3, sb, b.R[l], b.Cg[l], b.R[g], b.Cg[g], s);
      ++nl;
    } else if (!spline && plan_md3(ctx, p, sc, l, false, FM, E1)) {
      if (ctx->warp_levels &&
          md3w_supported(FM, false, d_in, b.R[l], b.Cg[l], b.R[g], b.Cg[g])) {
        launch_level_md3w(false, sb.kind, FM, sb, b.R[l], b.Cg[l], b.R[g], b.Cg[g], b.ctl,
                          ctx->num_sms, ls.chunks, s);
        ++nl;
      } else if (ctx->stream_levels && md3s_supported(FM, false, d_in, b.R[l], b.Cg[l]) &&
          launch_level_md3s(false, sb.kind, FM, sb, b.R[l], b.Cg[l], b.R[g], b.Cg[g],
                            b.ctl, ctx->num_sms, ctx->drop_copy, ctx->stream_chunks, s)) {
        ++nl;
      } else {
        launch_level_md3(false, sb.kind, FM, E1, sb, b.R[l], b.Cg[l], b.R[g],
                         b.Cg[g], s);
        nl += 2;
      }
    } else if (!spline && plan_md(ctx, p, sc, l, false, FM)) {
      launch_level_md(false, sb.kind, FM, sb, b.R[l], b.Cg[l], b.R[g], b.Cg[g],
                      ctx->num_sms, s);
      nl += FM.k;
    } else if (!spline && ctx->fused_levels && plan_fused(ctx, p, sc, l, false, F)) {
      launch_level(false, F, sb, b.R[l], b.Cg[l], b.R[g], b.Cg[g], s);
      ++nl;
    } else {
      launch_upsample(p.grid[l], p.gsize[l], p.grid[g], b.R[l], b.Cg[l], b.R[g],
                      b.Cg[g], b.ctl, s);
      ++nl;
      for (const Launch& L : level_schedule(p, sc, l)) {
        if (spline)
          launch_spline_pass(false, p.grid[g], L.pb, sb, nullptr, ctx->num_sms, s);
        else
          launch_pass(false, p.grid[g], L.pb, sb, ctx->num_sms, s);
        nl += L.pb.total ? 1 : 0;
      }
    }
    pf.end(s);
  }
  }  // interpolation
  uint16_t* codes = b.Cg[0];
  pf.begin(HPEZ_PH_HIST, s);
  cudaMemsetAsync(b.hist, 0, 65536 * sizeof(uint32_t), s);
  launch_hist(codes, p.N, p.C, p.nch, b.hist, b.zc, b.ctl, ctx->num_sms, s);
  launch_scan(b.zc, b.zoff, p.nch, &b.ctl->n_out, b.ctl, s);
  pf.end(s);
  pf.begin(HPEZ_PH_CODEBOOK, s);
  launch_codebook(b.hist, b.enc, b.tsyms, b.tlens, b.gkeys, b.giw, b.gpar,
                  b.lens_by_sym, b.ctl, s);
  pf.end(s);
  // the stream's section offsets (their capacity check comes with the
  // bit count, inside the one-pass encode)
  pf.begin(HPEZ_PH_ENCODE, s);
  launch_layout(b.ctl, off_table, ~0ull, s);
  pf.end(s);
  uint8_t* out = static_cast<uint8_t*>(d_out);
  pf.begin(HPEZ_PH_PACK, s);
  launch_encode(codes, p.N, p.C, p.nch, b.enc, b.lbits, b.flags, out, b.ctl, out_cap,
                ctx->num_sms, s);
  pf.end(s);
  pf.begin(HPEZ_PH_OUTLIERS, s);
  launch_outliers(true, codes, p.N, p.C, p.nch, b.zc, b.zoff, d_in, nullptr,
                  out, ~0ull, b.ctl, ctx->num_sms, s);
  pf.end(s);
  pf.begin(HPEZ_PH_FINALIZE, s);
  launch_finalize(hdr, hdrc, out, b.R[p.L], (uint32_t)na, off_anchors, b.bmap,
                  p.nblocks, off_bmap, b.lbits, p.nch, off_chw, b.tsyms, b.tlens,
                  b.ctl, ctx->num_sms, s);
  pf.end(s);
  nl += 10;
  if (d_status) {
    launch_result_one(ResultJob{b.ctl, nullptr, 0, 0, d_size, d_status, 0}, s);
    ++nl;
    return cuda_check(cudaGetLastError());
  }
  rc = cuda_check(cudaGetLastError());
  if (rc) return rc;
  rc = cuda_check(cudaMemcpyAsync(ctx->h_ctl, b.ctl, sizeof(Ctl),
                                  cudaMemcpyDeviceToHost, s));
  if (rc) return rc;
  rc = cuda_check(cudaStreamSynchronize(s));
  if (rc) return rc;
  ctx->prof.collect();
  if (ctx->h_ctl->status) return map_status(ctx->h_ctl->status);
  *h_out_size = ctx->h_ctl->total_size;
  return HPEZ_OK;
}

int hpez_compress(hpez_ctx* ctx, const float* d_in, int ndim, const uint64_t* dims,
                  int eb_mode, double eb, const hpez_config* cfg_in, void* d_out,
                  uint64_t out_cap, uint64_t* h_out_size, void* stream) {
  if (!h_out_size) return HPEZ_ERR_INVALID_ARG;
  return compress_impl(ctx, d_in, ndim, dims, eb_mode, eb, cfg_in, d_out, out_cap, h_out_size,
                       nullptr, nullptr, stream);
}

int hpez_compress_async(hpez_ctx* ctx, const float* d_in, int ndim, const uint64_t* dims,
                        int eb_mode, double eb, const hpez_config* cfg, void* d_out,
                        uint64_t out_cap, uint64_t* d_size, int32_t* d_status, void* stream) {
  if (!d_size || !d_status) return HPEZ_ERR_INVALID_ARG;
  return compress_impl(ctx, d_in, ndim, dims, eb_mode, eb, cfg, d_out, out_cap, nullptr,
                       reinterpret_cast<unsigned long long*>(d_size), d_status, stream);
}

int hpez_inspect(const void* h_header, uint64_t n, int* ndim, uint64_t* dims,
                 double* abs_eb) {
  if (!h_header || n < (uint64_t)kHeaderBytes) return HPEZ_ERR_INVALID_ARG;
  const uint8_t* h = static_cast<const uint8_t*>(h_header);
  if (rd32(h, H_MAGIC) != kMagic || rd32(h, H_VERSION) != kVersion)
    return HPEZ_ERR_CORRUPT_STREAM;
  const int nd = (int)rd32(h, H_NDIM);
  if (nd < 1 || nd > 3) return HPEZ_ERR_CORRUPT_STREAM;
  if (ndim) *ndim = nd;
  if (dims)
    for (int d = 0; d < 3; ++d) dims[d] = d < nd ? rd64(h, H_DIMS + 8 * d) : 1;
  if (abs_eb) *abs_eb = (double)rdf32(h, H_E);
  return HPEZ_OK;
}

// The decompress launch sequence.  Synchronous (d_status null): the
// header is read back first.  Asynchronous: the caller's host copy of the
// header plans the launches, the one-symbol table's symbol and a block map
// are read on the device, and a last kernel writes the status.
static int decompress_impl(hpez_ctx* ctx, const void* d_in, uint64_t in_size,
                           const void* h_header, float* d_out, uint64_t out_cap_elems,
                           int* d_status, void* stream) {
  if (!ctx || !d_in || !d_out) return HPEZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_in) & 15u) != 0) return HPEZ_ERR_INVALID_ARG;
  if (in_size < (uint64_t)kHeaderBytes) return HPEZ_ERR_CORRUPT_STREAM;
  if ((reinterpret_cast<uintptr_t>(d_out) & 3u) != 0) return HPEZ_ERR_INVALID_ARG;
  if (d_status && !h_header) return HPEZ_ERR_INVALID_ARG;
  ctx->out_aligned16 = (reinterpret_cast<uintptr_t>(d_out) & 15u) == 0;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc;
  uint8_t hdr_local[kHeaderBytes];
  const uint8_t* hh = hdr_local;
  if (d_status) {
    std::memcpy(hdr_local, h_header, kHeaderBytes);
  } else {
    rc = cuda_check(cudaMemcpyAsync(ctx->h_hdr, d_in, kHeaderBytes, cudaMemcpyDeviceToHost, s));
    if (rc) return rc;
    rc = cuda_check(cudaStreamSynchronize(s));
    if (rc) return rc;
    hh = ctx->h_hdr;
  }
  uint64_t raw = 0;
  if (lossless_flagged(hh, &raw)) {
    if (d_status) return HPEZ_ERR_UNSUPPORTED;  // undoing the stage needs its sizes
    // the lossless stage (Sec. 4, Step 5) first, into the context's buffer
    if (raw < (uint64_t)kHeaderBytes || raw > (1ull << 40)) return HPEZ_ERR_CORRUPT_STREAM;
    if ((rc = ensure_io(&ctx->lz_stream, &ctx->lz_stream_cap, raw))) return rc;
    uint64_t got = 0;
    rc = hpez_lossless_decode(ctx, d_in, in_size, ctx->lz_stream, raw, &got, stream);
    if (rc) return rc;
    return hpez_decompress(ctx, ctx->lz_stream, got, d_out, out_cap_elems, stream);
  }
  StreamInfo si;
  rc = parse_stream_header(hh, in_size, si);
  if (rc) return rc;
  const uint64_t N = si.N;
  if (N > out_cap_elems) return HPEZ_ERR_OUT_TOO_SMALL;
  const uint8_t* in = static_cast<const uint8_t*>(d_in);
  if (si.is_const) {
    launch_fill(d_out, (uint32_t)N, si.const_value, ctx->num_sms, s);
    if (d_status) {
      rc = cuda_check(cudaMemsetAsync(d_status, 0, sizeof(int), s));
      if (rc) return rc;
      return cuda_check(cudaGetLastError());
    }
    rc = cuda_check(cudaGetLastError());
    if (rc) return rc;
    return cuda_check(cudaStreamSynchronize(s));
  }
  const hpez_config& cfg = si.cfg;
  const Plan& p = si.p;
  const float e = si.e;
  const uint64_t nout = si.nout, twords = si.twords;
  const uint32_t nused = si.nused;
  const uint64_t oa = si.oa, ocw = si.ocw, ot = si.ot, oo = si.oo, ob = si.ob,
                 obm = si.obm;
  uint16_t single_sym = 0;
  if (nused == 1 && !d_status) {
    // the lone symbol of a single-symbol code table
    rc = cuda_check(cudaMemcpyAsync(ctx->h_hdr, in + ot, 2,
                                    cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
    if (rc) return rc;
    single_sym = (uint16_t)(ctx->h_hdr[0] | (ctx->h_hdr[1] << 8));
  }
  Arena ar;
  const size_t o_ctl = ar.take<Ctl>(1);
  const size_t o_lut = ar.take<uint32_t>(4096);
  const size_t o_cnt = ar.take<uint32_t>(64);
  const size_t o_first = ar.take<unsigned long long>(64);
  const size_t o_offs = ar.take<uint32_t>(64);
  const size_t o_sorted = ar.take<uint16_t>(65536);
  const size_t o_gkeys = ar.take<unsigned long long>(65536);
  size_t o_R[kMaxLevels + 1];
  for (int g = 1; g < p.L; ++g) o_R[g] = ar.take<float>(p.gsize[g]);
  const size_t o_codes = ar.take<uint16_t>(N);
  const size_t o_zc = ar.take<uint32_t>(p.nch);
  const size_t o_zoff = ar.take<unsigned long long>(p.nch);
  const size_t o_woff = ar.take<unsigned long long>(p.nch);
  const size_t o_dchw = ar.take<uint32_t>(p.nch);
  const size_t o_tot = ar.take<unsigned long long>(2);
  // level 1 of the global spline: its forward sweep must not overwrite the
  // escaped values already in the output
  const bool spline1 = !cfg.predictor && !cfg.blockwise && cfg.interp[0] == HPEZ_SPLINE_GLOBAL;
  const size_t o_dscr = spline1 ? ar.take<float>(p.gsize[0]) : 0;
  rc = ensure_scratch(ctx, ar.off);
  if (rc) return rc;
  char* S = ctx->scratch;
  Ctl* ctl = reinterpret_cast<Ctl*>(S + o_ctl);
  uint32_t* lut = reinterpret_cast<uint32_t*>(S + o_lut);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(S + o_cnt);
  unsigned long long* first = reinterpret_cast<unsigned long long*>(S + o_first);
  uint32_t* offs = reinterpret_cast<uint32_t*>(S + o_offs);
  uint16_t* sorted = reinterpret_cast<uint16_t*>(S + o_sorted);
  unsigned long long* gkeys = reinterpret_cast<unsigned long long*>(S + o_gkeys);
  uint16_t* codes = reinterpret_cast<uint16_t*>(S + o_codes);
  uint32_t* zc = reinterpret_cast<uint32_t*>(S + o_zc);
  unsigned long long* zoff = reinterpret_cast<unsigned long long*>(S + o_zoff);
  unsigned long long* woff = reinterpret_cast<unsigned long long*>(S + o_woff);
  unsigned long long* tot = reinterpret_cast<unsigned long long*>(S + o_tot);
  uint32_t* dchw = reinterpret_cast<uint32_t*>(S + o_dchw);
  float* R[kMaxLevels + 1];
  for (int g = 1; g < p.L; ++g) R[g] = reinterpret_cast<float*>(S + o_R[g]);
  R[0] = d_out;
  R[p.L] = const_cast<float*>(reinterpret_cast<const float*>(in + oa));
  float* const dscr = spline1 ? reinterpret_cast<float*>(S + o_dscr) : nullptr;

  PhaseProfiler& pf = ctx->prof;
  uint64_t& nl = ctx->launches;
  launch_init_ctl(ctl, s);
  launch_params(ctl, HPEZ_EB_ABS, (double)e, cfg.alpha, cfg.beta, p.L, d_out, s);
  const uint8_t* lbits_stream = in + ocw;
  pf.begin(HPEZ_PH_DEC_PREP, s);
  launch_chunk_words(lbits_stream, p.nch, dchw, ctx->num_sms, s);
  launch_scan(dchw, woff, p.nch, &tot[0], ctl, s);
  launch_dec_tables(in, nused, ot, lut, cnt, first, offs, sorted, gkeys, ctl, s);
  pf.end(s);
  pf.begin(HPEZ_PH_DECODE, s);
  launch_decode(in, ob, twords, lbits_stream, woff, p.N, p.C, p.nch, nused,
                single_sym, lut, cnt, first, offs, sorted, codes, zc, ctl,
                ctx->num_sms, s, d_status && nused == 1 ? in + ot : nullptr);
  pf.end(s);
  pf.begin(HPEZ_PH_SCATTER, s);
  launch_scan(zc, zoff, p.nch, &tot[1], ctl, s);
  launch_outliers(false, codes, p.N, p.C, p.nch, zc, zoff, nullptr, d_out,
                  const_cast<uint8_t*>(in) + oo, nout, ctl, ctx->num_sms, s);
  pf.end(s);
  nl += 8;
  if (cfg.predictor) {
    // Sec. 6.5: the Lorenzo recurrence over the decoded codes; outliers
    // are already in place
    if (!lorenzo_supported(p.n, p.fst, p.off, p.A)) return HPEZ_ERR_UNSUPPORTED;
    pf.begin(HPEZ_PH_DLEVEL, s);
    rc = launch_lorenzo(true, cfg.predictor, p.n, p.fst, p.off, p.A, ctx->out_aligned16,
                        nullptr, codes, d_out, ctl, ctx->num_sms, ctx->drop_copy,
                        ctx->lorenzo_ctas, s);
    pf.end(s);
    if (rc) return rc;
    ++nl;
  }
  // a uniform block map runs as its interpolator (the map is read back)
  std::vector<uint8_t> hmap;
  if (cfg.blockwise && !d_status) {
    hmap.resize(p.nblocks);
    rc = cuda_check(cudaMemcpyAsync(hmap.data(), in + obm, p.nblocks,
                                    cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
    if (rc) return rc;
  }
  const hpez_config sc = sweep_config(cfg, hmap.data(), p.nblocks);
  SweepBufs sb;
  std::memset(&sb, 0, sizeof(sb));
  sb.codes_full = codes;
  sb.outl_full = d_out;
  sb.blockmap = sc.blockwise ? in + obm : nullptr;
  sb.bs = (uint32_t)(cfg.block_size > 0 ? cfg.block_size : 1);
  for (int s3 = 0; s3 < 3; ++s3) sb.nb[s3] = p.nb[s3];
  sb.ctl = ctl;
  for (int l = cfg.predictor ? 0 : p.L; l >= 1; --l) {
    const int g = l - 1;
    // keyed by the config this sweep runs (a uniform block map read back
    // is its interpolator)
    const LevelSchedScope ls(ctx, p, sc, l, true);
    pf.begin(HPEZ_PH_DLEVEL + g, s);
    sb.R = R[g];
    sb.kind = sc.interp[l - 1];
    sb.same = sc.same_level[l - 1];
    FusedLevel F;
    Level3D F3;
    LevelMD FM;
    int E1 = 0;
    const bool spline = sc.interp[l - 1] == HPEZ_SPLINE_GLOBAL;
    if (!spline && ctx->fused_levels && plan_level3d(ctx, p, sc, l, true, F3)) {
      launch_level3d(true, F3, sb, R[l], nullptr, R[g], nullptr, s);
      ++nl;
    } else if (!spline && plan_md3(ctx, p, sc, l, true, FM, E1)) {
      if (ctx->warp_levels && md3w_supported(FM, true, codes, R[l], nullptr, R[g], nullptr)) {
        launch_level_md3w(true, sb.kind, FM, sb, R[l], nullptr, R[g], nullptr, ctl,
                          ctx->num_sms, ls.chunks, s);
        ++nl;
      } else if (ctx->stream_levels && md3s_supported(FM, true, codes, R[l], nullptr) &&
          launch_level_md3s(true, sb.kind, FM, sb, R[l], nullptr, R[g], nullptr, ctl,
                            ctx->num_sms, ctx->drop_copy, ctx->stream_chunks, s)) {
        ++nl;
      } else {
        launch_level_md3(true, sb.kind, FM, E1, sb, R[l], nullptr, R[g], nullptr, s);
        nl += 2;
      }
    } else if (!spline && plan_md(ctx, p, sc, l, true, FM)) {
      launch_level_md(true, sb.kind, FM, sb, R[l], nullptr, R[g], nullptr,
                      ctx->num_sms, s);
      nl += FM.k;
    } else if (!spline && ctx->fused_levels && plan_fused(ctx, p, sc, l, true, F)) {
      launch_level(true, F, sb, R[l], nullptr, R[g], nullptr, s);
      ++nl;
    } else {
      launch_upsample(p.grid[l], p.gsize[l], p.grid[g], R[l], nullptr, R[g],
                      nullptr, ctl, s);
      ++nl;
      for (const Launch& L : level_schedule(p, sc, l)) {
        if (spline)
          launch_spline_pass(true, p.grid[g], L.pb, sb, g == 0 ? dscr : nullptr,
                             ctx->num_sms, s);
        else
          launch_pass(true, p.grid[g], L.pb, sb, ctx->num_sms, s);
        nl += L.pb.total ? 1 : 0;
      }
    }
    pf.end(s);
  }
  if (d_status) {
    launch_result_one(ResultJob{ctl, tot, twords, nout, nullptr, d_status, 1}, s);
    ++nl;
    return cuda_check(cudaGetLastError());
  }
  rc = cuda_check(cudaGetLastError());
  if (rc) return rc;
  unsigned long long h_tot[2];
  rc = cuda_check(cudaMemcpyAsync(ctx->h_ctl, ctl, sizeof(Ctl),
                                  cudaMemcpyDeviceToHost, s));
  if (rc) return rc;
  rc = cuda_check(cudaMemcpyAsync(h_tot, tot, sizeof(h_tot),
                                  cudaMemcpyDeviceToHost, s));
  if (rc) return rc;
  rc = cuda_check(cudaStreamSynchronize(s));
  if (rc) return rc;
  ctx->prof.collect();
  if (ctx->h_ctl->status) return map_status(ctx->h_ctl->status);
  if (h_tot[0] != twords || h_tot[1] != nout) return HPEZ_ERR_CORRUPT_STREAM;
  return HPEZ_OK;
}

int hpez_decompress(hpez_ctx* ctx, const void* d_in, uint64_t in_size, float* d_out,
                    uint64_t out_cap_elems, void* stream) {
  return decompress_impl(ctx, d_in, in_size, nullptr, d_out, out_cap_elems, nullptr, stream);
}

int hpez_decompress_async(hpez_ctx* ctx, const void* d_in, uint64_t in_size,
                          const void* h_header, float* d_out, uint64_t out_cap_elems,
                          int32_t* d_status, void* stream) {
  if (!d_status || !h_header) return HPEZ_ERR_INVALID_ARG;
  return decompress_impl(ctx, d_in, in_size, h_header, d_out, out_cap_elems, d_status, stream);
}


int hpez_compress_host(hpez_ctx* ctx, const float* h_in, int ndim,
                       const uint64_t* dims, int eb_mode, double eb,
                       const hpez_config* cfg, void* h_out, uint64_t out_cap,
                       uint64_t* h_out_size, void* stream) {
  if (!ctx || !h_in || !h_out || !h_out_size || !dims || ndim < 1 || ndim > 3)
    return HPEZ_ERR_INVALID_ARG;
  uint64_t N = 1;
  for (int d = 0; d < ndim; ++d) N *= dims[d];
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = ensure_io(&ctx->io_in, &ctx->io_in_cap, N * sizeof(float));
  if (rc) return rc;
  rc = ensure_io(&ctx->io_out, &ctx->io_out_cap, out_cap);
  if (rc) return rc;
  rc = cuda_check(cudaMemcpyAsync(ctx->io_in, h_in, N * sizeof(float),
                                  cudaMemcpyHostToDevice, s));
  if (rc) return rc;
  rc = hpez_compress(ctx, static_cast<const float*>(ctx->io_in), ndim, dims,
                     eb_mode, eb, cfg, ctx->io_out, out_cap, h_out_size, stream);
  if (rc) return rc;
  rc = cuda_check(cudaMemcpyAsync(h_out, ctx->io_out, *h_out_size,
                                  cudaMemcpyDeviceToHost, s));
  if (rc) return rc;
  return cuda_check(cudaStreamSynchronize(s));
}

int hpez_decompress_host(hpez_ctx* ctx, const void* h_in, uint64_t in_size,
                         float* h_out, uint64_t out_cap_elems, void* stream) {
  if (!ctx || !h_in || !h_out) return HPEZ_ERR_INVALID_ARG;
  int nd;
  uint64_t dims[3];
  int rc = hpez_inspect(h_in, in_size, &nd, dims, nullptr);
  if (rc) return rc;
  uint64_t N = 1;
  for (int d = 0; d < nd; ++d) N *= dims[d];
  if (N > out_cap_elems) return HPEZ_ERR_OUT_TOO_SMALL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = ensure_io(&ctx->io_in, &ctx->io_in_cap, in_size);
  if (rc) return rc;
  rc = ensure_io(&ctx->io_out, &ctx->io_out_cap, N * sizeof(float));
  if (rc) return rc;
  rc = cuda_check(cudaMemcpyAsync(ctx->io_in, h_in, in_size,
                                  cudaMemcpyHostToDevice, s));
  if (rc) return rc;
  rc = hpez_decompress(ctx, ctx->io_in, in_size, static_cast<float*>(ctx->io_out),
                       N, stream);
  if (rc) return rc;
  rc = cuda_check(cudaMemcpyAsync(h_out, ctx->io_out, N * sizeof(float),
                                  cudaMemcpyDeviceToHost, s));
  if (rc) return rc;
  return cuda_check(cudaStreamSynchronize(s));
}

}  // extern "C"

// =====================================================================
// Decompression without any allocation, for callers that cannot allocate
// device or pinned host memory (for example code running under an external
// memory manager that forbids cudaMalloc, or inside a pre-sized real-time
// loop).  Its scratch is this fixed device array; the caller still passes
// the stream and the output.
// =====================================================================
namespace {

static __device__ __align__(256) unsigned char
    g_noalloc_scratch[HPEZ_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[128] = {};  // per device: address of g_noalloc_scratch

// Device address of the array on the current device, looked up once per
// device (a host-side reference to the symbol is not a device address).
int noalloc_scratch(int dev, char** out) {
  if (dev < 0 || dev >= 128) return HPEZ_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return HPEZ_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = ptr;
  }
  *out = static_cast<char*>(g_noalloc_ptr[dev]);
  return HPEZ_OK;
}

}  // namespace

extern "C" int hpez_decompress_noalloc(const void* d_in, uint64_t in_size,
                                       float* d_out, uint64_t out_cap_elems,
                                       void* stream) {
  if (!d_in || !d_out) return HPEZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_in) & 15u) != 0) return HPEZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_out) & 3u) != 0) return HPEZ_ERR_INVALID_ARG;
  if (in_size < (uint64_t)kHeaderBytes) return HPEZ_ERR_CORRUPT_STREAM;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HPEZ_ERR_CUDA;
  char* S = nullptr;
  int rc = noalloc_scratch(dev, &S);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // execution settings of a default context, built on the stack (nothing
  // in it allocates)
  hpez_ctx opt;
  opt.device = dev;
  cudaDeviceGetAttribute(&opt.num_sms, cudaDevAttrMultiProcessorCount, dev);
  opt.out_aligned16 = (reinterpret_cast<uintptr_t>(d_out) & 15u) == 0;
  uint8_t h[kHeaderBytes];
  rc = cuda_check(cudaMemcpyAsync(h, d_in, kHeaderBytes, cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc) return rc;
  uint64_t raw = 0;
  if (lossless_flagged(h, &raw)) return HPEZ_ERR_UNSUPPORTED;  // hpez_decompress undoes it
  // the same header validation as hpez_decompress (dims, offsets, counts,
  // alignment of the sections)
  StreamInfo si;
  rc = parse_stream_header(h, in_size, si);
  if (rc) return rc;
  const uint64_t N = si.N;
  if (N > HPEZ_NOALLOC_MAX_POINTS) return HPEZ_ERR_TOO_LARGE;
  if (N > out_cap_elems) return HPEZ_ERR_OUT_TOO_SMALL;
  const uint8_t* in = static_cast<const uint8_t*>(d_in);
  if (si.is_const) {
    launch_fill(d_out, (uint32_t)N, si.const_value, opt.num_sms, s);
    rc = cuda_check(cudaGetLastError());
    if (rc) return rc;
    return cuda_check(cudaStreamSynchronize(s));
  }
  const hpez_config& cfg = si.cfg;
  const Plan& p = si.p;
  if (cfg.predictor) return HPEZ_ERR_UNSUPPORTED;  // Lorenzo streams: hpez_decompress
  for (int l = 0; l < p.L; ++l)  // global-spline streams: hpez_decompress
    if (cfg.interp[l] == HPEZ_SPLINE_GLOBAL) return HPEZ_ERR_UNSUPPORTED;
  const float e = si.e;
  const uint64_t nout = si.nout, twords = si.twords;
  const uint32_t nused = si.nused;
  const uint64_t oa = si.oa, ocw = si.ocw, ot = si.ot, oo = si.oo, ob = si.ob,
                 obm = si.obm;
  uint16_t single_sym = 0;
  if (nused == 1) {
    uint8_t tb[2];
    rc = cuda_check(cudaMemcpyAsync(tb, in + ot, 2, cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
    if (rc) return rc;
    single_sym = (uint16_t)(tb[0] | (tb[1] << 8));
  }
  // carve the scratch out of the fixed array
  Arena ar;
  const size_t o_ctl = ar.take<Ctl>(1);
  const size_t o_lut = ar.take<uint32_t>(4096);
  const size_t o_cnt = ar.take<uint32_t>(64);
  const size_t o_first = ar.take<unsigned long long>(64);
  const size_t o_offs = ar.take<uint32_t>(64);
  const size_t o_sorted = ar.take<uint16_t>(65536);
  const size_t o_gkeys = ar.take<unsigned long long>(65536);
  size_t o_R[kMaxLevels + 1];
  for (int g = 1; g < p.L; ++g) o_R[g] = ar.take<float>(p.gsize[g]);
  const size_t o_codes = ar.take<uint16_t>(N);
  const size_t o_zc = ar.take<uint32_t>(p.nch);
  const size_t o_zoff = ar.take<unsigned long long>(p.nch);
  const size_t o_woff = ar.take<unsigned long long>(p.nch);
  const size_t o_dchw = ar.take<uint32_t>(p.nch);
  const size_t o_tot = ar.take<unsigned long long>(2);
  if (ar.off > (size_t)HPEZ_NOALLOC_SCRATCH_BYTES) return HPEZ_ERR_TOO_LARGE;
  Ctl* ctl = reinterpret_cast<Ctl*>(S + o_ctl);
  uint32_t* lut = reinterpret_cast<uint32_t*>(S + o_lut);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(S + o_cnt);
  unsigned long long* first = reinterpret_cast<unsigned long long*>(S + o_first);
  uint32_t* offs = reinterpret_cast<uint32_t*>(S + o_offs);
  uint16_t* sorted = reinterpret_cast<uint16_t*>(S + o_sorted);
  unsigned long long* gkeys = reinterpret_cast<unsigned long long*>(S + o_gkeys);
  uint16_t* codes = reinterpret_cast<uint16_t*>(S + o_codes);
  uint32_t* zc = reinterpret_cast<uint32_t*>(S + o_zc);
  unsigned long long* zoff = reinterpret_cast<unsigned long long*>(S + o_zoff);
  unsigned long long* woff = reinterpret_cast<unsigned long long*>(S + o_woff);
  unsigned long long* tot = reinterpret_cast<unsigned long long*>(S + o_tot);
  uint32_t* dchw = reinterpret_cast<uint32_t*>(S + o_dchw);
  float* R[kMaxLevels + 1];
  for (int g = 1; g < p.L; ++g) R[g] = reinterpret_cast<float*>(S + o_R[g]);
  R[0] = d_out;
  R[p.L] = const_cast<float*>(reinterpret_cast<const float*>(in + oa));
  // the control block is cleared by its first kernel; every other buffer is
  // written in full before it is read
  launch_init_ctl(ctl, s);
  launch_params(ctl, HPEZ_EB_ABS, (double)e, cfg.alpha, cfg.beta, p.L, d_out, s);
  const uint8_t* lbits_stream = in + ocw;
  launch_chunk_words(lbits_stream, p.nch, dchw, opt.num_sms, s);
  launch_scan(dchw, woff, p.nch, &tot[0], ctl, s);
  launch_dec_tables(in, nused, ot, lut, cnt, first, offs, sorted, gkeys, ctl, s);
  launch_decode(in, ob, twords, lbits_stream, woff, p.N, p.C, p.nch, nused,
                single_sym, lut, cnt, first, offs, sorted, codes, zc, ctl,
                opt.num_sms, s);
  launch_scan(zc, zoff, p.nch, &tot[1], ctl, s);
  launch_outliers(false, codes, p.N, p.C, p.nch, zc, zoff, nullptr, d_out,
                  const_cast<uint8_t*>(in) + oo, nout, ctl, opt.num_sms, s);
  SweepBufs sb;
  std::memset(&sb, 0, sizeof(sb));
  sb.codes_full = codes;
  sb.outl_full = d_out;
  sb.blockmap = cfg.blockwise ? in + obm : nullptr;
  sb.bs = (uint32_t)(cfg.block_size > 0 ? cfg.block_size : 1);
  for (int s3 = 0; s3 < 3; ++s3) sb.nb[s3] = p.nb[s3];
  sb.ctl = ctl;
  for (int l = p.L; l >= 1; --l) {
    const int g = l - 1;
    sb.R = R[g];
    sb.kind = cfg.interp[l - 1];
    sb.same = cfg.same_level[l - 1];
    FusedLevel F;
    Level3D F3;
    if (plan_level3d(&opt, p, cfg, l, true, F3)) {
      launch_level3d(true, F3, sb, R[l], nullptr, R[g], nullptr, s);
    } else if (plan_fused(&opt, p, cfg, l, true, F)) {
      launch_level(true, F, sb, R[l], nullptr, R[g], nullptr, s);
    } else {
      launch_upsample(p.grid[l], p.gsize[l], p.grid[g], R[l], nullptr, R[g],
                      nullptr, ctl, s);
      for (const Launch& L : level_schedule(p, cfg, l))
        launch_pass(true, p.grid[g], L.pb, sb, opt.num_sms, s);
    }
  }
  rc = cuda_check(cudaGetLastError());
  if (rc) return rc;
  Ctl hc;
  unsigned long long h_tot[2];
  rc = cuda_check(cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_check(cudaMemcpyAsync(h_tot, tot, sizeof(h_tot),
                                           cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc) return rc;
  if (hc.status) return map_status(hc.status);
  if (h_tot[0] != twords || h_tot[1] != nout) return HPEZ_ERR_CORRUPT_STREAM;
  return HPEZ_OK;
}
