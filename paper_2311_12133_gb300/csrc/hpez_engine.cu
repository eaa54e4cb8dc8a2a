// hpez_engine.cu -- the batched and the served forms of compress and
// decompress (declared in include/hpez.h).
//
// A request (one field to compress, or one stream to decompress) is planned
// into a list of operations -- the same kernels, in the same order, as the
// single-field path -- with all its buffers in one device workspace.  A
// "tick" advances every active request by one operation, and launches one
// batched kernel per operation kind present: job j of a batched launch owns
// blocks [off[j], off[j+1]).  Requests at different points of their work
// (other levels, other stages) share a tick, which is what lets new requests
// join while others are running.
//
//   hpez_batch_*   all requests start together; the tick sequence is fixed
//                  at creation, its job tables are uploaded once, and a run
//                  is kernel launches only (capturable in a CUDA graph).
//   hpez_server_*  a request loop: admission by a device-memory budget and
//                  free slots, one tick per step over whatever is active,
//                  host<->device copies of the requests' data inside.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "hpez.h"
#include "hpez_ctx.h"
#include "hpez_internal.cuh"
#include "hpez_launch.h"

using namespace hpez;
using namespace hpez::host;

namespace {

// operation kinds; kinds with one CTA per job need no offset table
enum OpType : int {
  OP_INIT, OP_RANGE, OP_PARAMS, OP_ANCHOR,
  OP_L3D_C,               // + interpolator (0..2): compress, 3D level kernel
  OP_L3D_D = OP_L3D_C + 3,
  OP_LVL_C = OP_L3D_D + 3,  // + kind (0..3): fused level kernel
  OP_LVL_D = OP_LVL_C + 4,
  OP_UPS = OP_LVL_D + 4, OP_PASS_C, OP_PASS_D,
  OP_ZERO, OP_HIST, OP_SCAN, OP_CODEBOOK, OP_ENCLEN, OP_LAYOUT, OP_PACK,
  OP_OUTL, OP_FINAL, OP_CWORDS, OP_DECTAB, OP_DECODE, OP_FILL, OP_RESULT,
  OP_MD3E_C,              // + interpolator (0..2): 3D multi-dimensional level,
  OP_MD3E_D = OP_MD3E_C + 3,  // even planes
  OP_MD3O_C = OP_MD3E_D + 3,  // odd planes
  OP_MD3O_D = OP_MD3O_C + 3,
  OP_MD3W_C = OP_MD3O_D + 3,  // finest level as warp strips
  OP_MD3W_D = OP_MD3W_C + 3,
  OP_LOR = OP_MD3W_D + 3,     // + variant: the Lorenzo pass (Sec. 6.5)
  OP_COUNT = OP_LOR + kLorVariants
};

// The batched form runs ops of equal key in one tick: the ops before the
// sweep by position, a level's ops by (level, position within the level),
// so that every field's level l runs in the same launches, and the ops
// after the sweep by position.
constexpr uint32_t kKeyLevel = 1u << 16, kKeyPost = 2u << 16;
uint32_t level_key(int l, int sub) {
  return kKeyLevel + ((uint32_t)(kMaxLevels + 1 - l) << 8) + (uint32_t)sub;
}

bool one_cta_per_job(int t) {
  return t == OP_INIT || t == OP_PARAMS || t == OP_SCAN || t == OP_CODEBOOK ||
         t == OP_LAYOUT || t == OP_DECTAB || t == OP_RESULT;
}

struct Op {
  int type;
  uint32_t nblk;  // blocks of this job
  uint32_t smem;  // dynamic shared memory
  uint32_t key;   // tick of the batched form
  std::vector<unsigned char> job;
};

template <class J>
Op make_op(int type, const J& j, uint32_t nblk = 1, uint32_t smem = 0) {
  Op o;
  o.type = type;
  o.nblk = nblk < 1 ? 1 : nblk;
  o.smem = smem;
  o.key = 0;
  o.job.resize(sizeof(J));
  std::memcpy(o.job.data(), &j, sizeof(J));
  return o;
}

struct Upload {
  void* dst;
  std::vector<unsigned char> bytes;
};

struct Request {
  int decomp = 0;
  std::vector<Op> ops;
  std::vector<Upload> uploads;  // host -> device at admission
  size_t ws_bytes = 0;
  uint64_t N = 0;               // points
  uint64_t in_bytes = 0, out_cap = 0;
};

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------
// the kernel family of one level (the same order of preference as the
// single-field call, without the TMA-streamed level)
// ---------------------------------------------------------------------
enum LevelFamily { FAM_LEVEL3D, FAM_MD3W, FAM_MD3, FAM_FUSED, FAM_PASS };

struct LevelPick {
  int fam = FAM_PASS;
  Level3D F3;
  FusedLevel F;
  LevelMD FM;
  int E1 = 0;
  int n1 = 0, n2 = 0, K = 0;
  uint32_t ctas = 0;
};

// The schedule `want` (HPEZ_FAM_*) for level l when the level can run it.
bool pick_family(hpez_ctx* ctx, const Plan& p, const hpez_config& sc, int l, bool decomp,
                 const void* in, const void* rs, int want, const int tile[3], int chunks,
                 LevelPick& k) {
  const void* al = reinterpret_cast<const void*>((uintptr_t)256);
  int saved[3];
  for (int s = 0; s < 3; ++s) {
    saved[s] = ctx->tile_e[s];
    if (tile[s] > 0) ctx->tile_e[s] = tile[s];
  }
  bool ok = false;
  switch (want) {
    case HPEZ_FAM_LEVEL3D:
      ok = ctx->fused_levels && plan_level3d(ctx, p, sc, l, decomp, k.F3);
      if (ok) k.fam = FAM_LEVEL3D;
      break;
    case HPEZ_FAM_MD3W:
    case HPEZ_FAM_MD3:
      ok = plan_md3(ctx, p, sc, l, decomp, k.FM, k.E1);
      if (ok && want == HPEZ_FAM_MD3W) {
        const float* Rs = l == 1 && decomp ? static_cast<const float*>(rs)
                                           : static_cast<const float*>(al);
        ok = md3w_supported(k.FM, decomp, in, static_cast<const float*>(al),
                            static_cast<const uint16_t*>(al), const_cast<float*>(Rs),
                            static_cast<const uint16_t*>(al));
        if (ok) {
          k.fam = FAM_MD3W;
          md3w_geometry(decomp, sc.interp[l - 1], k.FM, ctx->num_sms, chunks, &k.n1, &k.n2,
                        &k.K, &k.ctas);
        }
      } else if (ok) {
        k.fam = FAM_MD3;
      }
      break;
    case HPEZ_FAM_FUSED:
      ok = ctx->fused_levels && plan_fused(ctx, p, sc, l, decomp, k.F);
      if (ok) k.fam = FAM_FUSED;
      break;
    case HPEZ_FAM_PASS:
      ok = true;
      k.fam = FAM_PASS;
      break;
  }
  for (int s = 0; s < 3; ++s) ctx->tile_e[s] = saved[s];
  return ok;
}

// in: the field (compress) or the code array (decompress); rs: the level's
// reconstruction (decompress level 1: the caller's output).  Arena buffers
// are 256-byte aligned.  The context's schedule table first, then the
// fixed rules.
LevelPick pick_level(hpez_ctx* ctx, const Plan& p, const hpez_config& sc, int l, bool decomp,
                     const void* in, const void* rs) {
  LevelPick k;
  if (sc.interp[l - 1] == HPEZ_SPLINE_GLOBAL) return k;
  const int none[3] = {0, 0, 0};
  if (!ctx->sched.m.empty()) {
    const auto it = ctx->sched.m.find(sched_key(p, sc, l, decomp));
    if (it != ctx->sched.m.end()) {
      const hpez_level_sched& v = it->second;
      LevelPick t;
      if (pick_family(ctx, p, sc, l, decomp, in, rs, v.family, v.tile, v.chunks, t)) return t;
    }
  }
  if (pick_family(ctx, p, sc, l, decomp, in, rs, HPEZ_FAM_LEVEL3D, none, 0, k)) return k;
  if (ctx->warp_levels &&
      pick_family(ctx, p, sc, l, decomp, in, rs, HPEZ_FAM_MD3W, none, ctx->stream_chunks, k))
    return k;
  if (pick_family(ctx, p, sc, l, decomp, in, rs, HPEZ_FAM_MD3, none, 0, k)) return k;
  if (pick_family(ctx, p, sc, l, decomp, in, rs, HPEZ_FAM_FUSED, none, 0, k)) return k;
  k = LevelPick();
  return k;
}

// The ops of level l, keyed (l, position).  Compress: in = the field;
// decompress: in = the code array and Rs of level 1 = the caller's output.
void add_level_ops(hpez_ctx* ctx, const Plan& p, const hpez_config& sc, int l,
                   bool decomp, const SweepBufs& sb, const float* Rc, const uint16_t* Cc,
                   float* Rs, uint16_t* Cs, const void* in, Ctl* ctl, std::vector<Op>& ops) {
  const int g = l - 1;
  const int kind = sc.interp[l - 1];
  const int sms = ctx->num_sms;
  int sub = 0;
  auto add = [&](Op o) {
    o.key = level_key(l, sub++);
    ops.push_back(std::move(o));
  };
  const LevelPick k = pick_level(ctx, p, sc, l, decomp, in, Rs);
  const float* X = decomp ? nullptr : static_cast<const float*>(in);
  const uint16_t* codes = decomp ? static_cast<const uint16_t*>(in) : nullptr;
  const float* outl = decomp ? sb.outl_full : nullptr;
  switch (k.fam) {
    case FAM_LEVEL3D: {
      Level3DJob j{k.F3, X, codes, outl, Rc, decomp ? nullptr : Cc, Rs,
                   decomp ? nullptr : Cs, ctl};
      add(make_op((decomp ? OP_L3D_D : OP_L3D_C) + kind, j, (uint32_t)(k.F3.nt0 * k.F3.nt1),
                  (uint32_t)level3d_smem_bytes(k.F3, decomp)));
      return;
    }
    case FAM_MD3W: {
      MD3WJob j{k.FM, k.n1, k.n2, k.K, in, outl, Rc, decomp ? nullptr : Cc, Rs,
                decomp ? nullptr : Cs, ctl};
      add(make_op((decomp ? OP_MD3W_D : OP_MD3W_C) + kind, j, k.ctas));
      return;
    }
    case FAM_MD3: {
      const int m0 = (int)k.FM.g.m[0], m1 = (int)k.FM.g.m[1];
      const int nt1 = (m1 + k.E1 - 1) / k.E1;
      MD3Job j{k.FM, k.E1, nt1, X, codes, outl, Rc, decomp ? nullptr : Cc, Rs,
               decomp ? nullptr : Cs, ctl};
      const uint32_t smem = (uint32_t)md3_smem_bytes(k.FM, k.E1);
      add(make_op((decomp ? OP_MD3E_D : OP_MD3E_C) + kind, j,
                  (uint32_t)(((m0 + 1) / 2) * nt1), smem));
      if (m0 / 2 > 0)
        add(make_op((decomp ? OP_MD3O_D : OP_MD3O_C) + kind, j, (uint32_t)((m0 / 2) * nt1),
                    smem));
      return;
    }
    case FAM_FUSED: {
      LevelJob j{k.F, sb, Rc, decomp ? nullptr : Cc, Rs, decomp ? nullptr : Cs};
      add(make_op((decomp ? OP_LVL_D : OP_LVL_C) + level_kind(sb), j, k.F.ntiles,
                  (uint32_t)fused_smem_bytes(k.F, decomp)));
      return;
    }
    default:
      break;
  }
  add(make_op(OP_UPS,
              UpsampleJob{p.grid[l], p.gsize[l], p.grid[g], Rc, decomp ? nullptr : Cc, Rs,
                          decomp ? nullptr : Cs, ctl},
              grid_blocks(p.gsize[l], 65535)));
  for (const Launch& L : level_schedule(p, sc, l))
    if (L.pb.total)
      add(make_op(decomp ? OP_PASS_D : OP_PASS_C, PassJob{p.grid[g], L.pb, sb},
                  pass_blocks(L.pb.total, sms)));
}

// ---------------------------------------------------------------------
// planning: with base == nullptr only the workspace size is computed
// ---------------------------------------------------------------------
int plan_compress(hpez_ctx* ctx, const float* d_in, int ndim,
                  const uint64_t* dims, int eb_mode, double eb,
                  const hpez_config* cfg_in, void* d_out, uint64_t out_cap,
                  char* base, Request& r, unsigned long long* d_size,
                  int* d_status) {
  if (!d_in || !d_out || !dims) return HPEZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_out) & 15u) != 0) return HPEZ_ERR_INVALID_ARG;
  if (eb_mode != HPEZ_EB_ABS && eb_mode != HPEZ_EB_REL) return HPEZ_ERR_INVALID_ARG;
  if (!(eb > 0.0) || !std::isfinite(eb)) return HPEZ_ERR_INVALID_ARG;
  if (ndim < 1 || ndim > 3) return HPEZ_ERR_INVALID_ARG;
  hpez_config cfg;
  if (cfg_in)
    cfg = *cfg_in;
  else
    default_config(ndim, &cfg);
  Plan p;
  int rc = plan_geometry(p, ndim, dims, cfg.anchor_stride, cfg.frozen_dim);
  if (rc) return rc;
  if ((rc = check_config(p, cfg))) return rc;
  if (cfg.blockwise && !cfg.h_blockmap) return HPEZ_ERR_INVALID_ARG;
  const bool lor = cfg.predictor != 0;
  LorenzoJob lj;
  int lor_var = 0;
  uint32_t lor_ctas = 0;
  size_t lor_smem = 0;
  if (lor && !lorenzo_batch_job(false, cfg.predictor, p.n, p.fst, p.off, p.A,
                                (reinterpret_cast<uintptr_t>(d_in) & 15u) == 0, ctx->num_sms,
                                ctx->lorenzo_ctas, &lj.G, &lor_var, &lor_ctas, &lor_smem))
    return HPEZ_ERR_UNSUPPORTED;
  for (int l = 0; l < p.L && !lor; ++l)  // global spline: hpez_compress
    if (cfg.interp[l] == HPEZ_SPLINE_GLOBAL) return HPEZ_ERR_UNSUPPORTED;
  plan_chunks_blocks(p, cfg);
  r.decomp = 0;
  r.N = p.N;
  // the predictor the sweep runs (a uniform block map becomes its
  // interpolator); the header keeps the configuration as given
  const hpez_config sc = sweep_config(cfg, cfg.h_blockmap, p.nblocks);
  ctx->x_aligned16 = (reinterpret_cast<uintptr_t>(d_in) & 15u) == 0;
  // the finest level's fused kernels write no reconstruction in compress:
  // its grid is then not allocated
  // the Lorenzo pass needs the finest code array only
  const LevelPick pick1 = lor ? LevelPick() : pick_level(ctx, p, sc, 1, false, d_in, nullptr);
  const bool need_r0 = !lor && (pick1.fam == FAM_MD3 || pick1.fam == FAM_PASS);

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
    o_R[g] = ((g > 0 && !lor) || need_r0) ? ar.take<float>(p.gsize[g]) : 0;
    // two spare codes: kernels may read a code as the aligned 4-byte word
    // that holds it
    o_C[g] = (g == 0 || !lor) ? ar.take<uint16_t>(p.gsize[g] + 2) : 0;
  }
  const size_t o_zc = ar.take<uint32_t>(p.nch);
  const size_t o_zoff = ar.take<unsigned long long>(p.nch);
  const size_t o_chw = ar.take<uint32_t>(p.nch);
  const size_t o_woff = ar.take<unsigned long long>(p.nch);
  const size_t o_lbits = ar.take<uint16_t>((size_t)p.nch * 32);
  const size_t o_bmap = ar.take<uint8_t>(p.nblocks + 1);
  const size_t o_hdr = ar.take<uint8_t>(kHeaderBytes);
  const size_t o_hdrc = ar.take<uint8_t>(kHeaderBytes);
  r.ws_bytes = al256(ar.off);
  if (!base) return HPEZ_OK;

  Ctl* ctl = reinterpret_cast<Ctl*>(base + o_ctl);
  uint32_t* hist = reinterpret_cast<uint32_t*>(base + o_hist);
  unsigned long long* enc = reinterpret_cast<unsigned long long*>(base + o_enc);
  uint16_t* tsyms = reinterpret_cast<uint16_t*>(base + o_tsyms);
  uint8_t* tlens = reinterpret_cast<uint8_t*>(base + o_tlens);
  uint8_t* lbs = reinterpret_cast<uint8_t*>(base + o_lbs);
  unsigned long long* gkeys = reinterpret_cast<unsigned long long*>(base + o_gkeys);
  unsigned long long* giw = reinterpret_cast<unsigned long long*>(base + o_giw);
  uint32_t* gpar = reinterpret_cast<uint32_t*>(base + o_gpar);
  float* R[kMaxLevels + 1];
  uint16_t* Cg[kMaxLevels + 1];
  for (int g = 0; g <= p.L; ++g) {
    R[g] = ((g > 0 && !lor) || need_r0) ? reinterpret_cast<float*>(base + o_R[g]) : nullptr;
    Cg[g] = (g == 0 || !lor) ? reinterpret_cast<uint16_t*>(base + o_C[g]) : nullptr;
  }
  uint32_t* zc = reinterpret_cast<uint32_t*>(base + o_zc);
  unsigned long long* zoff = reinterpret_cast<unsigned long long*>(base + o_zoff);
  uint32_t* chw = reinterpret_cast<uint32_t*>(base + o_chw);
  unsigned long long* woff = reinterpret_cast<unsigned long long*>(base + o_woff);
  uint16_t* lbits = reinterpret_cast<uint16_t*>(base + o_lbits);
  uint8_t* bmap = reinterpret_cast<uint8_t*>(base + o_bmap);
  uint8_t* hdr_d = reinterpret_cast<uint8_t*>(base + o_hdr);
  uint8_t* hdrc_d = reinterpret_cast<uint8_t*>(base + o_hdrc);

  const uint64_t na = lor ? 0 : n_anchors(p);
  const uint64_t off_anchors = kHeaderBytes;
  const uint64_t off_bmap = a16(off_anchors + 4 * na);
  const uint64_t off_chw = a16(off_bmap + p.nblocks);
  const uint64_t off_table = a16(off_chw + 64ull * p.nch);
  Upload uh, uc;
  uh.dst = hdr_d;
  uh.bytes.resize(kHeaderBytes);
  uc.dst = hdrc_d;
  uc.bytes.resize(kHeaderBytes);
  header_templates(p, cfg, eb_mode, eb, off_anchors, off_bmap, off_chw,
                   uh.bytes.data(), uc.bytes.data());
  r.uploads.push_back(std::move(uh));
  r.uploads.push_back(std::move(uc));
  if (cfg.blockwise) {
    Upload ub;
    ub.dst = bmap;
    ub.bytes.assign(cfg.h_blockmap, cfg.h_blockmap + p.nblocks);
    r.uploads.push_back(std::move(ub));
  }

  const int sms = ctx->num_sms;
  uint8_t* out = static_cast<uint8_t*>(d_out);
  auto& ops = r.ops;
  uint32_t kpre = 0, kpost = kKeyPost;
  auto pre = [&](Op o) { o.key = kpre++; ops.push_back(std::move(o)); };
  auto post = [&](Op o) { o.key = kpost++; ops.push_back(std::move(o)); };
  pre(make_op(OP_INIT, InitJob{ctl}));
  if (eb_mode == HPEZ_EB_REL)
    pre(make_op(OP_RANGE, RangeJob{d_in, p.N, ctl},
                grid_blocks(p.N / 4 + 1, (unsigned)sms * 8)));
  else
    ++kpre;
  ParamsJob pj;
  pj.ctl = ctl;
  pj.eb_mode = eb_mode;
  pj.L = p.L;
  pj.eb = eb;
  pj.alpha = cfg.alpha;
  pj.beta = cfg.beta;
  pj.x = d_in;
  pre(make_op(OP_PARAMS, pj));
  if (lor) {
    // the Lorenzo pass in the place of the sweep (at level 1's tick)
    lj.x = d_in;
    lj.codes = Cg[0];
    lj.out = nullptr;
    lj.ctl = ctl;
    Op o = make_op(OP_LOR + lor_var, lj, lor_ctas, (uint32_t)lor_smem);
    o.key = level_key(1, 0);
    ops.push_back(std::move(o));
  } else {
    pre(make_op(OP_ANCHOR, AnchorJob{d_in, p.grid[p.L], p.gsize[p.L], R[p.L], Cg[p.L], ctl},
                grid_blocks(p.gsize[p.L], 65535)));
  }
  SweepBufs sb;
  std::memset(&sb, 0, sizeof(sb));
  sb.x = d_in;
  sb.blockmap = sc.blockwise ? bmap : nullptr;
  sb.bs = (uint32_t)(cfg.block_size > 0 ? cfg.block_size : 1);
  for (int s3 = 0; s3 < 3; ++s3) sb.nb[s3] = p.nb[s3];
  sb.ctl = ctl;
  for (int l = lor ? 0 : p.L; l >= 1; --l) {
    const int g = l - 1;
    sb.R = R[g];
    sb.C = Cg[g];
    sb.kind = sc.interp[l - 1];
    sb.same = sc.same_level[l - 1];
    add_level_ops(ctx, p, sc, l, false, sb, R[l], Cg[l], R[g], Cg[g], d_in, ctl, ops);
  }
  uint16_t* codes = Cg[0];
  post(make_op(OP_ZERO, ZeroJob{hist, 65536ull * 4}, 16));
  post(make_op(OP_HIST, HistJob{codes, p.N, p.C, p.nch, hist, zc, ctl},
               hist_blocks(p.nch, sms)));
  post(make_op(OP_SCAN, ScanJob{zc, zoff, p.nch, &ctl->n_out, ctl}));
  post(make_op(OP_CODEBOOK, CodebookJob{hist, enc, tsyms, tlens, gkeys, giw, gpar, lbs, ctl}));
  post(make_op(OP_ENCLEN, EncLenJob{codes, p.N, p.C, p.nch, enc, lbits, chw, ctl},
               enc_blocks(p.nch, sms)));
  post(make_op(OP_SCAN, ScanJob{chw, woff, p.nch, &ctl->total_words, ctl}));
  post(make_op(OP_LAYOUT, LayoutJob{ctl, off_table, out_cap}));
  post(make_op(OP_PACK, PackJob{codes, p.N, p.C, p.nch, enc, lbits, chw, woff, out, ctl},
               enc_blocks(p.nch, sms)));
  OutlierJob oj;
  oj.codes = codes;
  oj.N = p.N;
  oj.C = p.C;
  oj.nch = p.nch;
  oj.zc = zc;
  oj.zoff = zoff;
  oj.src = d_in;
  oj.dst = nullptr;
  oj.stream = out;
  oj.max_out = ~0ull;
  oj.ctl = ctl;
  oj.gather = 1;
  post(make_op(OP_OUTL, oj, p.nch));
  FinalizeJob fj{hdr_d, hdrc_d, out, R[p.L], (uint32_t)na, off_anchors, bmap,
                 p.nblocks, off_bmap, lbits, p.nch, off_chw, tsyms, tlens, ctl};
  post(make_op(OP_FINAL, fj, finalize_blocks((uint32_t)na, p.nch, sms)));
  post(make_op(OP_RESULT, ResultJob{ctl, nullptr, 0, 0, d_size, d_status, 0}));
  return HPEZ_OK;
}

int plan_decompress(hpez_ctx* ctx, const void* d_in, uint64_t in_size,
                    const void* h_header, float* d_out, uint64_t out_cap_elems,
                    char* base, Request& r, int* d_status) {
  if (!d_in || !d_out || !h_header) return HPEZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_in) & 15u) != 0) return HPEZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_out) & 3u) != 0) return HPEZ_ERR_INVALID_ARG;
  if (in_size < (uint64_t)kHeaderBytes) return HPEZ_ERR_CORRUPT_STREAM;
  StreamInfo si;
  int rc = parse_stream_header(static_cast<const uint8_t*>(h_header), in_size, si);
  if (rc) return rc;
  if (si.N > out_cap_elems) return HPEZ_ERR_OUT_TOO_SMALL;
  const bool lor = !si.is_const && si.cfg.predictor != 0;
  LorenzoJob lj;
  int lor_var = 0;
  uint32_t lor_ctas = 0;
  size_t lor_smem = 0;
  if (lor && !lorenzo_batch_job(true, si.cfg.predictor, si.p.n, si.p.fst, si.p.off, si.p.A,
                                (reinterpret_cast<uintptr_t>(d_out) & 15u) == 0, ctx->num_sms,
                                ctx->lorenzo_ctas, &lj.G, &lor_var, &lor_ctas, &lor_smem))
    return HPEZ_ERR_UNSUPPORTED;
  if (!si.is_const && !lor)
    for (int l = 0; l < si.p.L; ++l)
      if (si.cfg.interp[l] == HPEZ_SPLINE_GLOBAL) return HPEZ_ERR_UNSUPPORTED;
  r.decomp = 1;
  r.N = si.N;
  const Plan& p = si.p;
  const hpez_config& cfg = si.cfg;
  const int sms = ctx->num_sms;
  const uint8_t* in = static_cast<const uint8_t*>(d_in);
  auto& ops = r.ops;
  if (si.is_const) {
    Arena ar;
    const size_t o_ctl = ar.take<Ctl>(1);
    r.ws_bytes = al256(ar.off);
    if (!base) return HPEZ_OK;
    Ctl* ctl = reinterpret_cast<Ctl*>(base + o_ctl);
    ops.push_back(make_op(OP_INIT, InitJob{ctl}));
    ops.back().key = 0;
    ops.push_back(make_op(OP_FILL, FillJob{d_out, (uint32_t)si.N, si.const_value},
                          grid_blocks(si.N, (unsigned)sms * 16)));
    ops.back().key = 1;
    ops.push_back(make_op(OP_RESULT, ResultJob{ctl, nullptr, 0, 0, nullptr, d_status, 1}));
    ops.back().key = kKeyPost;
    return HPEZ_OK;
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
  for (int g = 1; g < p.L; ++g) o_R[g] = lor ? 0 : ar.take<float>(p.gsize[g]);
  const size_t o_codes = ar.take<uint16_t>(si.N + 2);  // 2 spare: 4-byte code reads
  const size_t o_zc = ar.take<uint32_t>(p.nch);
  const size_t o_zoff = ar.take<unsigned long long>(p.nch);
  const size_t o_woff = ar.take<unsigned long long>(p.nch);
  const size_t o_dchw = ar.take<uint32_t>(p.nch);
  const size_t o_tot = ar.take<unsigned long long>(2);
  r.ws_bytes = al256(ar.off);
  if (!base) return HPEZ_OK;

  Ctl* ctl = reinterpret_cast<Ctl*>(base + o_ctl);
  uint32_t* lut = reinterpret_cast<uint32_t*>(base + o_lut);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(base + o_cnt);
  unsigned long long* first = reinterpret_cast<unsigned long long*>(base + o_first);
  uint32_t* offs = reinterpret_cast<uint32_t*>(base + o_offs);
  uint16_t* sorted = reinterpret_cast<uint16_t*>(base + o_sorted);
  unsigned long long* gkeys = reinterpret_cast<unsigned long long*>(base + o_gkeys);
  uint16_t* codes = reinterpret_cast<uint16_t*>(base + o_codes);
  uint32_t* zc = reinterpret_cast<uint32_t*>(base + o_zc);
  unsigned long long* zoff = reinterpret_cast<unsigned long long*>(base + o_zoff);
  unsigned long long* woff = reinterpret_cast<unsigned long long*>(base + o_woff);
  uint32_t* dchw = reinterpret_cast<uint32_t*>(base + o_dchw);
  unsigned long long* tot = reinterpret_cast<unsigned long long*>(base + o_tot);
  float* R[kMaxLevels + 1];
  for (int g = 1; g < p.L; ++g) R[g] = lor ? nullptr : reinterpret_cast<float*>(base + o_R[g]);
  R[0] = d_out;
  R[p.L] = const_cast<float*>(reinterpret_cast<const float*>(in + si.oa));

  uint32_t kpre = 0;
  auto pre = [&](Op o) { o.key = kpre++; ops.push_back(std::move(o)); };
  pre(make_op(OP_INIT, InitJob{ctl}));
  ParamsJob pj;
  pj.ctl = ctl;
  pj.eb_mode = HPEZ_EB_ABS;
  pj.L = p.L;
  pj.eb = (double)si.e;
  pj.alpha = cfg.alpha;
  pj.beta = cfg.beta;
  pj.x = d_out;
  pre(make_op(OP_PARAMS, pj));
  const uint8_t* lbits_stream = in + si.ocw;
  pre(make_op(OP_CWORDS, ChunkWordsJob{lbits_stream, p.nch, dchw},
              chunk_words_blocks(p.nch, sms)));
  pre(make_op(OP_SCAN, ScanJob{dchw, woff, p.nch, &tot[0], ctl}));
  pre(make_op(OP_DECTAB,
              DecTablesJob{in, si.nused, si.ot, lut, cnt, first, offs, sorted, gkeys, ctl}));
  DecodeJob dj;
  dj.stream = in;
  dj.off_bits = si.ob;
  dj.total_words = si.twords;
  dj.lanebits_bytes = lbits_stream;
  dj.woff = woff;
  dj.N = p.N;
  dj.C = p.C;
  dj.nch = p.nch;
  dj.n_used = si.nused;
  dj.single_src = si.nused == 1 ? in + si.ot : nullptr;
  dj.lut = lut;
  dj.cnt = cnt;
  dj.first = first;
  dj.offs = offs;
  dj.sorted = sorted;
  dj.codes = codes;
  dj.zc = zc;
  dj.ctl = ctl;
  pre(make_op(OP_DECODE, dj, decode_blocks(p.nch, sms)));
  pre(make_op(OP_SCAN, ScanJob{zc, zoff, p.nch, &tot[1], ctl}));
  OutlierJob oj;
  oj.codes = codes;
  oj.N = p.N;
  oj.C = p.C;
  oj.nch = p.nch;
  oj.zc = zc;
  oj.zoff = zoff;
  oj.src = nullptr;
  oj.dst = d_out;
  oj.stream = const_cast<uint8_t*>(in) + si.oo;
  oj.max_out = si.nout;
  oj.ctl = ctl;
  oj.gather = 0;
  pre(make_op(OP_OUTL, oj, p.nch));
  SweepBufs sb;
  std::memset(&sb, 0, sizeof(sb));
  sb.codes_full = codes;
  sb.outl_full = d_out;
  sb.blockmap = cfg.blockwise ? in + si.obm : nullptr;
  sb.bs = (uint32_t)(cfg.block_size > 0 ? cfg.block_size : 1);
  for (int s3 = 0; s3 < 3; ++s3) sb.nb[s3] = p.nb[s3];
  sb.ctl = ctl;
  ctx->out_aligned16 = (reinterpret_cast<uintptr_t>(d_out) & 15u) == 0;
  ctx->codes_aligned16 = true;
  if (lor) {
    // the Lorenzo recurrence over the decoded codes; the escaped values
    // are already in place
    lj.x = nullptr;
    lj.codes = codes;
    lj.out = d_out;
    lj.ctl = ctl;
    Op o = make_op(OP_LOR + lor_var, lj, lor_ctas, (uint32_t)lor_smem);
    o.key = level_key(1, 0);
    ops.push_back(std::move(o));
  }
  for (int l = lor ? 0 : p.L; l >= 1; --l) {
    const int g = l - 1;
    sb.R = R[g];
    sb.kind = cfg.interp[l - 1];
    sb.same = cfg.same_level[l - 1];
    add_level_ops(ctx, p, cfg, l, true, sb, R[l], nullptr, R[g], nullptr, codes, ctl, ops);
  }
  ops.push_back(make_op(OP_RESULT, ResultJob{ctl, tot, si.twords, si.nout,
                                             nullptr, d_status, 1}));
  ops.back().key = kKeyPost;
  return HPEZ_OK;
}

// ---------------------------------------------------------------------
// ticks
// ---------------------------------------------------------------------
struct Entry {
  int type;
  int nj;
  uint32_t nblk;
  uint32_t smem;
  size_t jobs_off, off_off;  // into the tick table
};

void tab_align(std::vector<unsigned char>& tab) {
  tab.resize(al256(tab.size()));
}

// One tick: one entry per operation kind among `ops`, job structs and
// block offsets appended to `tab`.
void build_tick(const std::vector<const Op*>& ops, std::vector<unsigned char>& tab,
                std::vector<Entry>& out) {
  std::map<int, std::vector<const Op*>> by;
  for (const Op* o : ops) by[o->type].push_back(o);
  for (auto& kv : by) {
    Entry e;
    e.type = kv.first;
    e.nj = (int)kv.second.size();
    e.smem = 0;
    tab_align(tab);
    e.jobs_off = tab.size();
    for (const Op* o : kv.second) {
      tab.insert(tab.end(), o->job.begin(), o->job.end());
      e.smem = std::max(e.smem, o->smem);
    }
    tab_align(tab);
    e.off_off = tab.size();
    uint32_t run = 0;
    std::vector<uint32_t> off;
    off.reserve(kv.second.size() + 1);
    for (const Op* o : kv.second) {
      off.push_back(run);
      run += one_cta_per_job(e.type) ? 1u : o->nblk;
    }
    off.push_back(run);
    e.nblk = run;
    const unsigned char* ob = reinterpret_cast<const unsigned char*>(off.data());
    tab.insert(tab.end(), ob, ob + off.size() * sizeof(uint32_t));
    out.push_back(e);
  }
}

// Level ops run as persistent launches of at most max_ctas CTAs (0: the
// CTAs resident on the GPU at once).
void launch_entry(const Entry& e, const unsigned char* d_tab, int sms, int max_ctas,
                  cudaStream_t s) {
  const void* J = d_tab + e.jobs_off;
  const uint32_t* off = reinterpret_cast<const uint32_t*>(d_tab + e.off_off);
  const int t = e.type;
  if (t >= OP_L3D_C && t < OP_L3D_C + 3) {
    launch_level3d_batch(false, t - OP_L3D_C, (const Level3DJob*)J, off, e.nj,
                         e.nblk, e.smem, sms, max_ctas, s);
    return;
  }
  if (t >= OP_L3D_D && t < OP_L3D_D + 3) {
    launch_level3d_batch(true, t - OP_L3D_D, (const Level3DJob*)J, off, e.nj,
                         e.nblk, e.smem, sms, max_ctas, s);
    return;
  }
  if (t >= OP_LVL_C && t < OP_LVL_C + 4) {
    launch_level_batch(false, t - OP_LVL_C, (const LevelJob*)J, off, e.nj, e.nblk,
                       e.smem, sms, max_ctas, s);
    return;
  }
  if (t >= OP_LVL_D && t < OP_LVL_D + 4) {
    launch_level_batch(true, t - OP_LVL_D, (const LevelJob*)J, off, e.nj, e.nblk,
                       e.smem, sms, max_ctas, s);
    return;
  }
  if (t >= OP_MD3E_C && t < OP_MD3W_C) {
    const int u = t - OP_MD3E_C;  // (odd, decomp, kind)
    launch_md3_batch((u / 3) % 2 == 1, u >= 6, u % 3, (const MD3Job*)J, off, e.nj, e.nblk,
                     e.smem, sms, max_ctas, s);
    return;
  }
  if (t >= OP_MD3W_C && t < OP_LOR) {
    const int u = t - OP_MD3W_C;
    launch_md3w_batch(u >= 3, u % 3, (const MD3WJob*)J, off, e.nj, e.nblk, sms, max_ctas, s);
    return;
  }
  if (t >= OP_LOR && t < OP_COUNT) {
    launch_lorenzo_batch(t - OP_LOR, (const LorenzoJob*)J, off, e.nj, e.nblk, e.smem, s);
    return;
  }
  switch (t) {
    case OP_INIT: launch_init_ctl_batch((const InitJob*)J, e.nj, s); break;
    case OP_RANGE: launch_range_batch((const RangeJob*)J, off, e.nj, e.nblk, s); break;
    case OP_PARAMS: launch_params_batch((const ParamsJob*)J, e.nj, s); break;
    case OP_ANCHOR: launch_anchor_batch((const AnchorJob*)J, off, e.nj, e.nblk, s); break;
    case OP_UPS: launch_upsample_batch((const UpsampleJob*)J, off, e.nj, e.nblk, s); break;
    case OP_PASS_C: launch_pass_batch(false, (const PassJob*)J, off, e.nj, e.nblk, s); break;
    case OP_PASS_D: launch_pass_batch(true, (const PassJob*)J, off, e.nj, e.nblk, s); break;
    case OP_ZERO: launch_zero_batch((const ZeroJob*)J, off, e.nj, e.nblk, s); break;
    case OP_HIST: launch_hist_batch((const HistJob*)J, off, e.nj, e.nblk, s); break;
    case OP_SCAN: launch_scan_batch((const ScanJob*)J, e.nj, s); break;
    case OP_CODEBOOK: launch_codebook_batch((const CodebookJob*)J, e.nj, s); break;
    case OP_ENCLEN: launch_enc_len_batch((const EncLenJob*)J, off, e.nj, e.nblk, s); break;
    case OP_LAYOUT: launch_layout_batch((const LayoutJob*)J, e.nj, s); break;
    case OP_PACK: launch_pack_batch((const PackJob*)J, off, e.nj, e.nblk, s); break;
    case OP_OUTL: launch_outliers_batch((const OutlierJob*)J, off, e.nj, e.nblk, s); break;
    case OP_FINAL: launch_finalize_batch((const FinalizeJob*)J, off, e.nj, e.nblk, s); break;
    case OP_CWORDS: launch_chunk_words_batch((const ChunkWordsJob*)J, off, e.nj, e.nblk, s); break;
    case OP_DECTAB: launch_dec_tables_batch((const DecTablesJob*)J, e.nj, s); break;
    case OP_DECODE: launch_decode_batch((const DecodeJob*)J, off, e.nj, e.nblk, s); break;
    case OP_FILL: launch_fill_batch((const FillJob*)J, off, e.nj, e.nblk, s); break;
    case OP_RESULT: launch_result_batch((const ResultJob*)J, e.nj, s); break;
  }
}

// A tick's launches of different operation kinds are independent (they
// belong to different requests): they fan out over a main stream and up to
// kSide side streams, joined again at the end of the tick.
constexpr int kSide = 3;

struct TickStreams {
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kSide] = {};
  int create() {
    int rc = cuda_check(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (int i = 0; !rc && i < kSide; ++i) {
      rc = cuda_check(cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking));
      if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming));
    }
    return rc;
  }
  void destroy() {
    for (int i = 0; i < kSide; ++i) {
      if (side[i]) cudaStreamDestroy(side[i]);
      if (join[i]) cudaEventDestroy(join[i]);
      side[i] = nullptr;
      join[i] = nullptr;
    }
    if (fork) cudaEventDestroy(fork);
    fork = nullptr;
  }
};

void enqueue_tick(const std::vector<Entry>& es, const unsigned char* d_tab, int sms,
                  int max_ctas, cudaStream_t s, TickStreams& ts) {
  const int n = (int)es.size();
  const int nside = std::min(kSide, n - 1);
  if (nside <= 0 || !ts.fork) {
    for (const Entry& e : es) launch_entry(e, d_tab, sms, max_ctas, s);
    return;
  }
  cudaEventRecord(ts.fork, s);
  for (int i = 0; i < nside; ++i) cudaStreamWaitEvent(ts.side[i], ts.fork, 0);
  for (int i = 0; i < n; ++i) {
    const int k = i % (nside + 1);
    launch_entry(es[i], d_tab, sms, max_ctas, k == 0 ? s : ts.side[k - 1]);
  }
  for (int i = 0; i < nside; ++i) {
    cudaEventRecord(ts.join[i], ts.side[i]);
    cudaStreamWaitEvent(s, ts.join[i], 0);
  }
}

int upload(const Request& r) {
  for (const Upload& u : r.uploads)
    if (cudaMemcpy(u.dst, u.bytes.data(), u.bytes.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return cuda_check(cudaGetLastError());
  return HPEZ_OK;
}

}  // namespace

// =====================================================================
// batched form
// =====================================================================
struct hpez_batch {
  hpez_ctx* ctx = nullptr;
  int device = 0;  // the context's device, kept for destroy
  int n = 0;
  int decomp = 0;
  char* ws = nullptr;             // request workspaces + results
  unsigned char* d_tab = nullptr; // every tick's job tables
  unsigned long long* d_sizes = nullptr;
  int* d_status = nullptr;
  std::vector<std::vector<Entry>> ticks;
  std::vector<uint32_t> tick_keys;  // the op key of each tick
  uint64_t launches = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  TickStreams ts;
};

namespace {

int batch_create(hpez_ctx* ctx, int n, int decomp, const void* descs,
                 hpez_batch** out) {
  if (!ctx || !out || n < 1 || !descs) return HPEZ_ERR_INVALID_ARG;
  *out = nullptr;
  cudaSetDevice(ctx->device);
  std::vector<Request> reqs(n);
  auto plan = [&](int i, char* base, unsigned long long* d_size, int* d_status) {
    Request& r = reqs[i];
    r.ops.clear();
    r.uploads.clear();
    if (!decomp) {
      const hpez_field_desc& d = static_cast<const hpez_field_desc*>(descs)[i];
      return plan_compress(ctx, d.d_in, d.ndim, d.dims, d.eb_mode, d.eb, d.cfg,
                           d.d_out, d.out_cap, base, r, d_size, d_status);
    }
    const hpez_stream_desc& d = static_cast<const hpez_stream_desc*>(descs)[i];
    return plan_decompress(ctx, d.d_in, d.in_size, d.h_header, d.d_out,
                           d.out_cap_elems, base, r, d_status);
  };
  size_t total = 0;
  std::vector<size_t> at(n);
  for (int i = 0; i < n; ++i) {
    const int rc = plan(i, nullptr, nullptr, nullptr);
    if (rc) return rc;
    at[i] = total;
    total += al256(reqs[i].ws_bytes);
  }
  const size_t o_sizes = total;
  total += al256(sizeof(unsigned long long) * n);
  const size_t o_status = total;
  total += al256(sizeof(int) * n);
  hpez_batch* b = new hpez_batch();
  b->ctx = ctx;
  b->device = ctx->device;
  b->n = n;
  b->decomp = decomp;
  if (cudaMalloc(&b->ws, total) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return HPEZ_ERR_NO_MEMORY;
  }
  b->d_sizes = reinterpret_cast<unsigned long long*>(b->ws + o_sizes);
  b->d_status = reinterpret_cast<int*>(b->ws + o_status);
  cudaMemset(b->ws + o_sizes, 0, total - o_sizes);
  for (int i = 0; i < n; ++i) {
    int rc = plan(i, b->ws + at[i], b->d_sizes + i, b->d_status + i);
    if (!rc) rc = upload(reqs[i]);
    if (rc) {
      hpez_batch_destroy(b);
      return rc;
    }
  }
  // the tick sequence: one tick per op key, in key order (a request's keys
  // increase along its ops), so every field's level l shares the launches
  // of that level
  std::map<uint32_t, std::vector<const Op*>> by_key;
  for (int i = 0; i < n; ++i)
    for (const Op& o : reqs[i].ops) by_key[o.key].push_back(&o);
  std::vector<unsigned char> tab;
  for (auto& kv : by_key) {
    std::vector<Entry> es;
    build_tick(kv.second, tab, es);
    b->launches += es.size();
    b->ticks.push_back(std::move(es));
    b->tick_keys.push_back(kv.first);
  }
  if (b->ts.create()) {
    cudaGetLastError();
    hpez_batch_destroy(b);
    return HPEZ_ERR_CUDA;
  }
  if (cudaMalloc(&b->d_tab, tab.size() ? tab.size() : 256) != cudaSuccess) {
    cudaGetLastError();
    hpez_batch_destroy(b);
    return HPEZ_ERR_NO_MEMORY;
  }
  if (cudaMemcpy(b->d_tab, tab.data(), tab.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    const int rc = cuda_check(cudaGetLastError());
    hpez_batch_destroy(b);
    return rc;
  }
  *out = b;
  return HPEZ_OK;
}

void batch_enqueue(hpez_batch* b, cudaStream_t s) {
  for (const auto& es : b->ticks)
    enqueue_tick(es, b->d_tab, b->ctx->num_sms, b->ctx->batch_ctas, s, b->ts);
}

}  // namespace

extern "C" {

int hpez_batch_create_compress(hpez_ctx* ctx, int n, const hpez_field_desc* fields,
                               hpez_batch** out) {
  return batch_create(ctx, n, 0, fields, out);
}

int hpez_batch_create_decompress(hpez_ctx* ctx, int n,
                                 const hpez_stream_desc* streams,
                                 hpez_batch** out) {
  return batch_create(ctx, n, 1, streams, out);
}

int hpez_batch_run(hpez_batch* b, void* stream) {
  if (!b) return HPEZ_ERR_INVALID_ARG;
  cudaSetDevice(b->ctx->device);
  batch_enqueue(b, static_cast<cudaStream_t>(stream));
  b->ctx->launches += b->launches;
  return cuda_check(cudaGetLastError());
}

int hpez_batch_run_graph(hpez_batch* b, void* stream) {
  if (!b) return HPEZ_ERR_INVALID_ARG;
  cudaSetDevice(b->ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!b->exec) {
    // capture on a stream of our own (the legacy default stream cannot be
    // captured); the graph is then launched on the caller's stream
    cudaStream_t cs;
    int rc = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    if (rc) return rc;
    rc = cuda_check(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    if (rc) {
      cudaStreamDestroy(cs);
      return rc;
    }
    batch_enqueue(b, cs);
    rc = cuda_check(cudaStreamEndCapture(cs, &b->graph));
    cudaStreamDestroy(cs);
    if (rc) return rc;
    rc = cuda_check(cudaGraphInstantiate(&b->exec, b->graph, 0));
    if (rc) return rc;
  }
  b->ctx->launches += b->launches;
  return cuda_check(cudaGraphLaunch(b->exec, s));
}

int hpez_batch_results(hpez_batch* b, void* stream, uint64_t* h_sizes,
                       int32_t* h_status) {
  if (!b) return HPEZ_ERR_INVALID_ARG;
  cudaSetDevice(b->ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = 0;
  if (h_sizes)
    rc = cuda_check(cudaMemcpyAsync(h_sizes, b->d_sizes, sizeof(uint64_t) * b->n,
                                    cudaMemcpyDeviceToHost, s));
  if (!rc && h_status)
    rc = cuda_check(cudaMemcpyAsync(h_status, b->d_status, sizeof(int32_t) * b->n,
                                    cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  return rc;
}

int hpez_batch_launch_count(hpez_batch* b, uint64_t* launches, uint64_t* ticks) {
  if (!b) return HPEZ_ERR_INVALID_ARG;
  if (launches) *launches = b->launches;
  if (ticks) *ticks = b->ticks.size();
  return HPEZ_OK;
}

int hpez_batch_destroy(hpez_batch* b) {
  if (!b) return HPEZ_OK;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->ws) cudaFree(b->ws);
  if (b->d_tab) cudaFree(b->d_tab);
  b->ts.destroy();
  delete b;
  return HPEZ_OK;
}

}  // extern "C"

// =====================================================================
// offline search of level schedules
// =====================================================================
namespace {

// The candidate schedules of the search: every family with tile shapes or
// chunk counts from a fixed list (slot extents slowest first).
std::vector<hpez_level_sched> sched_candidates(int ndim, int ke1) {
  std::vector<hpez_level_sched> c;
  auto add = [&](int fam, int t0, int t1, int t2, int chunks) {
    hpez_level_sched v;
    v.family = fam;
    v.tile[0] = t0;
    v.tile[1] = t1;
    v.tile[2] = t2;
    v.chunks = chunks;
    v.time_us = 0.f;
    c.push_back(v);
  };
  if (ndim == 3) {
    for (int e1 : {2, 4, 8, 16, 32}) add(HPEZ_FAM_LEVEL3D, 0, e1, 0, 0);
    // warp strips: chunks of K even planes of the finest level
    add(HPEZ_FAM_MD3W, 0, 0, 0, 0);
    int last = -1;
    for (int K : {2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 16, 24}) {
      const int ch = (ke1 + K - 1) / K;
      if (ch >= 1 && ch != last) add(HPEZ_FAM_MD3W, 0, 0, 0, ch);
      last = ch;
    }
    for (int e1 : {2, 4, 8, 16, 32}) add(HPEZ_FAM_MD3, 0, e1, 0, 0);
    const int f3[][3] = {{1, 2, 512}, {1, 4, 256}, {1, 8, 128}, {2, 8, 128},
                         {2, 4, 256}, {1, 16, 64}, {2, 16, 64}, {4, 8, 64}};
    for (const auto& f : f3) add(HPEZ_FAM_FUSED, f[0], f[1], f[2], 0);
  } else {
    const int f2[][2] = {{2, 512}, {4, 256}, {8, 128}, {16, 64},
                         {8, 256}, {16, 128}, {32, 64}, {4, 512}};
    for (const auto& f : f2) add(HPEZ_FAM_FUSED, 1, f[0], f[1], 0);
  }
  add(HPEZ_FAM_PASS, 0, 0, 0, 0);
  return c;
}

int level_of_key(uint32_t key) {
  if (key < kKeyLevel || key >= kKeyPost) return 0;
  return (int)(kMaxLevels + 1) - (int)((key - kKeyLevel) >> 8);
}

// One run of the batch with an event before every tick and after the last;
// per level l (1..kMaxLevels) the milliseconds of its ticks, added to ms[l].
int timed_run(hpez_batch* b, cudaStream_t s, std::vector<double>& ms) {
  const size_t n = b->ticks.size();
  std::vector<cudaEvent_t> ev(n + 1, nullptr);
  int rc = HPEZ_OK;
  for (size_t i = 0; i <= n && !rc; ++i) rc = cuda_check(cudaEventCreate(&ev[i]));
  if (!rc) {
    for (size_t i = 0; i < n; ++i) {
      cudaEventRecord(ev[i], s);
      enqueue_tick(b->ticks[i], b->d_tab, b->ctx->num_sms, b->ctx->batch_ctas, s, b->ts);
    }
    cudaEventRecord(ev[n], s);
    rc = cuda_check(cudaStreamSynchronize(s));
  }
  ms.assign(kMaxLevels + 1, 0.0);
  for (size_t i = 0; i < n && !rc; ++i) {
    float t = 0.f;
    rc = cuda_check(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
    const int l = level_of_key(b->tick_keys[i]);
    if (l >= 1 && l <= kMaxLevels) ms[l] += t;
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  return rc;
}

// The median over `reps` timed runs (after one warm-up run) of each
// level's time, in microseconds.
int time_levels(hpez_batch* b, cudaStream_t s, int reps, std::vector<double>& us) {
  std::vector<double> ms;
  int rc = timed_run(b, s, ms);
  std::vector<std::vector<double>> all(kMaxLevels + 1);
  for (int r = 0; r < reps && !rc; ++r) {
    rc = timed_run(b, s, ms);
    for (int l = 1; l <= kMaxLevels; ++l) all[l].push_back(ms[l]);
  }
  us.assign(kMaxLevels + 1, 0.0);
  for (int l = 1; l <= kMaxLevels && !rc; ++l) {
    std::sort(all[l].begin(), all[l].end());
    us[l] = all[l].empty() ? 0.0 : 1000.0 * all[l][all[l].size() / 2];
  }
  return rc;
}

}  // namespace

extern "C" int hpez_tuning_search(hpez_ctx* ctx, hpez_tuning* t, const float* d_x, int ndim,
                                  const uint64_t* dims, int eb_mode, double eb,
                                  const hpez_config* cfg_in, int copies, int reps,
                                  void* stream) {
  if (!ctx || !t || !d_x || !dims || ndim < 1 || ndim > 3) return HPEZ_ERR_INVALID_ARG;
  if (copies < 0 || copies > 1024 || reps < 1 || reps > 100) return HPEZ_ERR_INVALID_ARG;
  hpez_config cfg;
  if (cfg_in)
    cfg = *cfg_in;
  else
    default_config(ndim, &cfg);
  Plan p;
  int rc = plan_geometry(p, ndim, dims, cfg.anchor_stride, cfg.frozen_dim);
  if (rc) return rc;
  if ((rc = check_config(p, cfg))) return rc;
  if (cfg.blockwise && !cfg.h_blockmap) return HPEZ_ERR_INVALID_ARG;
  if (cfg.predictor) return HPEZ_ERR_UNSUPPORTED;
  plan_chunks_blocks(p, cfg);
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (copies == 0) copies = (int)std::max<uint64_t>(1, std::min<uint64_t>(64, (1ull << 25) / p.N));
  uint64_t bound = 0;
  if ((rc = hpez_compress_bound(ndim, dims, &bound))) return rc;
  bound = (bound + 255) & ~255ull;
  const uint64_t out_f = ((uint64_t)p.N * 4 + 255) & ~255ull;
  char* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)copies * (bound + out_f)) != cudaSuccess) {
    cudaGetLastError();
    return HPEZ_ERR_NO_MEMORY;
  }
  const hpez_config sc = sweep_config(cfg, cfg.h_blockmap, p.nblocks);
  // every level key of this field in both directions (compress plans the
  // sweep config, decompress the header's config)
  std::vector<std::array<int32_t, 8>> keys[2];
  for (int dir = 0; dir < 2; ++dir)
    for (int l = 1; l <= p.L; ++l) keys[dir].push_back(sched_key(p, dir ? cfg : sc, l, dir != 0));
  const hpez_tuning saved = ctx->sched;
  // best[dir][l]: the fastest feasible candidate so far
  std::vector<hpez_level_sched> best[2];
  for (int dir = 0; dir < 2; ++dir) {
    best[dir].assign(p.L + 1, hpez_level_sched());
    for (auto& v : best[dir]) {
      v.family = 0;
      v.time_us = INFINITY;
    }
  }
  std::vector<hpez_field_desc> fd(copies);
  std::vector<hpez_stream_desc> sd(copies);
  std::vector<uint64_t> sizes(copies);
  std::vector<int32_t> status(copies);
  std::vector<uint8_t> hdr(kHeaderBytes);
  for (const hpez_level_sched& c : sched_candidates(ndim, (int)(p.grid[0].m[0] + 1) / 2)) {
    if (rc) break;
    ctx->sched.m.clear();
    for (int dir = 0; dir < 2; ++dir)
      for (const auto& k : keys[dir]) ctx->sched.m[k] = c;
    // the levels that run this candidate
    bool feas[2][kMaxLevels + 1] = {};
    bool any = false;
    for (int dir = 0; dir < 2; ++dir)
      for (int l = 1; l <= p.L; ++l) {
        LevelPick k;
        const void* in = dir ? reinterpret_cast<const void*>((uintptr_t)256) : d_x;
        const void* rs = reinterpret_cast<const void*>((uintptr_t)(buf + (size_t)copies * bound));
        feas[dir][l] = pick_family(ctx, p, dir ? cfg : sc, l, dir != 0, in, rs, c.family,
                                   c.tile, c.chunks, k);
        any = any || feas[dir][l];
      }
    if (!any) continue;
    for (int i = 0; i < copies; ++i) {
      hpez_field_desc& f = fd[i];
      std::memset(&f, 0, sizeof(f));
      f.d_in = d_x;
      f.ndim = ndim;
      f.eb_mode = eb_mode;
      for (int d = 0; d < ndim; ++d) f.dims[d] = dims[d];
      f.eb = eb;
      f.cfg = &cfg;
      f.d_out = buf + (size_t)i * bound;
      f.out_cap = bound;
    }
    hpez_batch* bc = nullptr;
    rc = batch_create(ctx, copies, 0, fd.data(), &bc);
    if (rc) break;
    std::vector<double> us;
    rc = time_levels(bc, s, reps, us);
    if (!rc) rc = hpez_batch_results(bc, s, sizes.data(), status.data());
    hpez_batch_destroy(bc);
    for (int i = 0; i < copies && !rc; ++i)
      if (status[i]) rc = status[i];
    if (rc) break;
    for (int l = 1; l <= p.L; ++l)
      if (feas[0][l] && us[l] < best[0][l].time_us) {
        best[0][l] = c;
        best[0][l].time_us = (float)us[l];
      }
    rc = cuda_check(cudaMemcpy(hdr.data(), buf, kHeaderBytes, cudaMemcpyDeviceToHost));
    if (rc) break;
    for (int i = 0; i < copies; ++i) {
      hpez_stream_desc& d = sd[i];
      d.d_in = buf + (size_t)i * bound;
      d.in_size = sizes[i];
      d.h_header = hdr.data();
      d.d_out = reinterpret_cast<float*>(buf + (size_t)copies * bound + (size_t)i * out_f);
      d.out_cap_elems = p.N;
    }
    hpez_batch* bd = nullptr;
    rc = batch_create(ctx, copies, 1, sd.data(), &bd);
    if (rc) break;
    rc = time_levels(bd, s, reps, us);
    if (!rc) rc = hpez_batch_results(bd, s, nullptr, status.data());
    hpez_batch_destroy(bd);
    for (int i = 0; i < copies && !rc; ++i)
      if (status[i]) rc = status[i];
    if (rc) break;
    for (int l = 1; l <= p.L; ++l)
      if (feas[1][l] && us[l] < best[1][l].time_us) {
        best[1][l] = c;
        best[1][l].time_us = (float)us[l];
      }
  }
  ctx->sched = saved;
  cudaFree(buf);
  if (rc) return rc;
  for (int dir = 0; dir < 2; ++dir)
    for (int l = 1; l <= p.L; ++l)
      if (best[dir][l].family) t->m[keys[dir][l - 1]] = best[dir][l];
  return HPEZ_OK;
}

// =====================================================================
// served form
// =====================================================================
namespace {

enum ReqState { RS_QUEUED, RS_ACTIVE, RS_RESULT, RS_COPYING, RS_DONE };

struct SrvReq {
  uint64_t id = 0;
  bool full_bound = false;  // compress output sized by hpez_compress_bound
  hpez_request rq;
  hpez_config cfg;
  bool has_cfg = false;
  std::vector<uint8_t> bmap;   // the config's block map, copied at submit
  std::vector<uint8_t> header; // decompress: the stream's header
  size_t need = 0;             // device bytes: input + output + workspace
  size_t pool_off = 0;
  int slot = -1;
  Request plan;
  size_t cursor = 0;
  int state = RS_QUEUED;
  cudaEvent_t ev = nullptr;     // result ready / output copied
  cudaEvent_t ev_in = nullptr;  // input on the device
  bool wait_in = false;
  int status = 0;
  uint64_t size = 0;
  double t_submit = 0;
};

double now_s() {
  return std::chrono::duration<double>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// first-fit allocator over [0, cap), 256-byte granules
struct Pool {
  std::map<size_t, size_t> free_;  // offset -> size
  size_t used = 0;
  void init(size_t cap) {
    free_.clear();
    free_[0] = cap;
    used = 0;
  }
  bool alloc(size_t n, size_t* off) {
    n = al256(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      *off = it->first;
      const size_t rest = it->second - n;
      const size_t at = it->first + n;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used += n;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = al256(n);
    used -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

constexpr int kRing = 8;

}  // namespace

struct hpez_server {
  hpez_ctx* ctx = nullptr;
  int device = 0;  // the context's device, kept for destroy
  cudaStream_t s = nullptr;      // kernels (the caller's stream)
  cudaStream_t s_in = nullptr;   // host -> device copies
  cudaStream_t s_out = nullptr;  // device -> host copies
  char* pool_mem = nullptr;
  size_t budget = 0;
  Pool pool;
  int max_slots = 0;
  std::vector<int> free_slots;
  unsigned long long* d_sizes = nullptr;  // per slot
  int* d_status = nullptr;
  unsigned long long* h_sizes = nullptr;  // pinned mirrors
  int* h_status = nullptr;
  uint64_t next_id = 1;
  std::deque<SrvReq*> queue;
  std::vector<SrvReq*> active;  // admitted, not yet retired
  std::vector<SrvReq*> done;
  // tick tables: pinned ring + one device buffer (stream-ordered)
  unsigned char* h_tab[kRing] = {};
  size_t h_tab_cap[kRing] = {};
  cudaEvent_t tab_ev[kRing] = {};
  bool tab_used[kRing] = {};
  int ring = 0;
  unsigned char* d_tab = nullptr;
  size_t d_tab_cap = 0;
  uint64_t ticks = 0, launches = 0;
  TickStreams ts;
};

namespace {

// bytes of device memory a request needs; plans it when base != nullptr
int srv_plan(hpez_server* S, SrvReq* q, char* base) {
  const hpez_request& r = q->rq;
  q->plan = Request();
  if (r.op == HPEZ_REQ_COMPRESS) {
    uint64_t N = 1;
    for (int d = 0; d < r.ndim; ++d) N *= r.dims[d];
    uint64_t bound = 0;
    int rc = hpez_compress_bound(r.ndim, r.dims, &bound);
    if (rc) return rc;
    // the stream rarely needs the bound (every point an outlier); start
    // with 4.5 bytes per point and retry with the bound if that overflows
    if (!q->full_bound) bound = std::min<uint64_t>(bound, N * 9 / 2 + (1u << 20));
    const size_t o_in = 0, o_out = al256(N * 4), o_ws = o_out + al256(bound);
    float* d_in = base ? reinterpret_cast<float*>(base + o_in) : reinterpret_cast<float*>(256);
    void* d_out = base ? base + o_out : reinterpret_cast<void*>(512);
    rc = plan_compress(S->ctx, d_in, r.ndim, r.dims, r.eb_mode, r.eb,
                       q->has_cfg ? &q->cfg : nullptr, d_out, bound,
                       base ? base + o_ws : nullptr, q->plan,
                       base ? S->d_sizes + q->slot : nullptr,
                       base ? S->d_status + q->slot : nullptr);
    if (rc) return rc;
    q->plan.in_bytes = N * 4;
    q->plan.out_cap = bound;
    q->need = o_ws + q->plan.ws_bytes;
    return HPEZ_OK;
  }
  StreamInfo si;
  int rc = parse_stream_header(q->header.data(), r.in_bytes, si);
  if (rc) return rc;
  const size_t o_in = 0, o_out = al256(r.in_bytes), o_ws = o_out + al256(si.N * 4);
  const void* d_in = base ? base + o_in : reinterpret_cast<void*>(256);
  float* d_out = base ? reinterpret_cast<float*>(base + o_out) : reinterpret_cast<float*>(512);
  rc = plan_decompress(S->ctx, d_in, r.in_bytes, q->header.data(), d_out, si.N,
                       base ? base + o_ws : nullptr, q->plan,
                       base ? S->d_status + q->slot : nullptr);
  if (rc) return rc;
  q->plan.in_bytes = r.in_bytes;
  q->plan.out_cap = si.N * 4;
  q->need = o_ws + q->plan.ws_bytes;
  return HPEZ_OK;
}

void srv_retire(hpez_server* S, SrvReq* q) {
  S->pool.release(q->pool_off, q->need);
  S->free_slots.push_back(q->slot);
  q->state = RS_DONE;
  S->done.push_back(q);
}

}  // namespace

extern "C" {

int hpez_server_create(hpez_ctx* ctx, uint64_t budget_bytes, int max_slots,
                       void* stream, hpez_server** out) {
  if (!ctx || !out || max_slots < 1 || budget_bytes < 4096) return HPEZ_ERR_INVALID_ARG;
  *out = nullptr;
  cudaSetDevice(ctx->device);
  hpez_server* S = new hpez_server();
  S->ctx = ctx;
  S->device = ctx->device;
  S->s = static_cast<cudaStream_t>(stream);
  S->budget = budget_bytes;
  S->max_slots = max_slots;
  bool ok = cudaMalloc(&S->pool_mem, budget_bytes) == cudaSuccess &&
            cudaMalloc(&S->d_sizes, sizeof(unsigned long long) * max_slots) == cudaSuccess &&
            cudaMalloc(&S->d_status, sizeof(int) * max_slots) == cudaSuccess &&
            cudaMallocHost(&S->h_sizes, sizeof(unsigned long long) * max_slots) == cudaSuccess &&
            cudaMallocHost(&S->h_status, sizeof(int) * max_slots) == cudaSuccess;
  for (int k = 0; ok && k < kRing; ++k)
    ok = cudaEventCreateWithFlags(&S->tab_ev[k], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&S->s_in, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&S->s_out, cudaStreamNonBlocking) == cudaSuccess &&
       S->ts.create() == HPEZ_OK;
  if (!ok) {
    cudaGetLastError();
    hpez_server_destroy(S);
    return HPEZ_ERR_NO_MEMORY;
  }
  S->pool.init(budget_bytes);
  for (int i = max_slots - 1; i >= 0; --i) S->free_slots.push_back(i);
  *out = S;
  return HPEZ_OK;
}

int hpez_server_submit(hpez_server* S, const hpez_request* req, uint64_t* id) {
  if (!S || !req || !req->h_in || !req->h_out) return HPEZ_ERR_INVALID_ARG;
  if (req->op != HPEZ_REQ_COMPRESS && req->op != HPEZ_REQ_DECOMPRESS)
    return HPEZ_ERR_INVALID_ARG;
  SrvReq* q = new SrvReq();
  q->rq = *req;
  if (req->op == HPEZ_REQ_COMPRESS) {
    if (req->ndim < 1 || req->ndim > 3) {
      delete q;
      return HPEZ_ERR_INVALID_ARG;
    }
    if (req->cfg) {
      q->cfg = *req->cfg;
      q->has_cfg = true;
      if (q->cfg.blockwise && q->cfg.h_blockmap) {
        const uint64_t nb = hpez_blockmap_size(req->ndim, req->dims, q->cfg.block_size);
        q->bmap.assign(q->cfg.h_blockmap, q->cfg.h_blockmap + nb);
        q->cfg.h_blockmap = q->bmap.data();
      }
    }
  } else {
    if (req->in_bytes < (uint64_t)kHeaderBytes) {
      delete q;
      return HPEZ_ERR_CORRUPT_STREAM;
    }
    const uint8_t* h = static_cast<const uint8_t*>(req->h_in);
    q->header.assign(h, h + kHeaderBytes);
  }
  const int rc = srv_plan(S, q, nullptr);  // validates and sizes
  if (rc) {
    delete q;
    return rc;
  }
  const uint64_t out_need = q->plan.decomp ? q->plan.out_cap : 0;
  const int bad = q->need > S->budget ? HPEZ_ERR_TOO_LARGE
                  : (out_need && req->out_cap < out_need) ? HPEZ_ERR_OUT_TOO_SMALL
                                                          : HPEZ_OK;
  if (bad) {
    delete q;
    return bad;
  }
  q->id = S->next_id++;
  q->t_submit = now_s();
  S->queue.push_back(q);
  if (id) *id = q->id;
  return HPEZ_OK;
}

int hpez_server_step(hpez_server* S) {
  if (!S) return HPEZ_ERR_INVALID_ARG;
  cudaSetDevice(S->ctx->device);
  cudaStream_t s = S->s;
  // 1. retire: results read, outputs copied back
  for (size_t i = 0; i < S->active.size();) {
    SrvReq* q = S->active[i];
    bool gone = false;
    if (q->state == RS_RESULT && cudaEventQuery(q->ev) == cudaSuccess) {
      q->status = S->h_status[q->slot];
      char* base = S->pool_mem + q->pool_off;
      if (!q->status) {
        if (!q->plan.decomp) {
          q->size = S->h_sizes[q->slot];
          if (q->size > q->rq.out_cap) q->status = HPEZ_ERR_OUT_TOO_SMALL;
        } else {
          q->size = q->plan.out_cap;
        }
      }
      if (q->status == HPEZ_ERR_OUT_TOO_SMALL && !q->plan.decomp && !q->full_bound &&
          q->size == 0) {
        // the short output overflowed: run again with the full bound
        cudaEventDestroy(q->ev);
        cudaEventDestroy(q->ev_in);
        q->ev = q->ev_in = nullptr;
        S->pool.release(q->pool_off, q->need);
        S->free_slots.push_back(q->slot);
        q->full_bound = true;
        q->status = 0;
        q->state = RS_QUEUED;
        srv_plan(S, q, nullptr);
        S->queue.push_front(q);
        S->active.erase(S->active.begin() + i);
        continue;
      }
      if (!q->status) {
        const size_t o_out = al256(q->plan.in_bytes);
        cudaMemcpyAsync(q->rq.h_out, base + o_out, q->size, cudaMemcpyDeviceToHost,
                        S->s_out);
        cudaEventRecord(q->ev, S->s_out);
        q->state = RS_COPYING;
      } else {
        gone = true;
      }
    } else if (q->state == RS_COPYING && cudaEventQuery(q->ev) == cudaSuccess) {
      gone = true;
    }
    if (gone) {
      cudaEventDestroy(q->ev);
      cudaEventDestroy(q->ev_in);
      q->ev = q->ev_in = nullptr;
      srv_retire(S, q);
      S->active.erase(S->active.begin() + i);
    } else {
      ++i;
    }
  }
  cudaGetLastError();
  // 2. admit, first come first served
  while (!S->queue.empty() && !S->free_slots.empty()) {
    SrvReq* q = S->queue.front();
    if (q->need > S->budget) {  // a retry that can never fit
      S->queue.pop_front();
      q->status = HPEZ_ERR_TOO_LARGE;
      q->state = RS_DONE;
      S->done.push_back(q);
      continue;
    }
    size_t off;
    if (!S->pool.alloc(q->need, &off)) break;
    S->queue.pop_front();
    q->pool_off = off;
    q->slot = S->free_slots.back();
    S->free_slots.pop_back();
    char* base = S->pool_mem + off;
    int rc = srv_plan(S, q, base);
    if (!rc)
      rc = cuda_check(cudaMemcpyAsync(base, q->rq.h_in, q->plan.in_bytes,
                                      cudaMemcpyHostToDevice, S->s_in));
    for (const Upload& u : q->plan.uploads)
      if (!rc)
        rc = cuda_check(cudaMemcpyAsync(u.dst, u.bytes.data(), u.bytes.size(),
                                        cudaMemcpyHostToDevice, S->s_in));
    if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming));
    if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&q->ev_in, cudaEventDisableTiming));
    if (!rc) rc = cuda_check(cudaEventRecord(q->ev_in, S->s_in));
    if (rc) {
      if (q->ev) cudaEventDestroy(q->ev);
      if (q->ev_in) cudaEventDestroy(q->ev_in);
      q->ev = q->ev_in = nullptr;
      q->status = rc;
      srv_retire(S, q);
      continue;
    }
    q->state = RS_ACTIVE;
    q->cursor = 0;
    q->wait_in = true;
    S->active.push_back(q);
  }
  // 3. one tick over every active request
  std::vector<const Op*> now;
  std::vector<SrvReq*> finishing;
  for (SrvReq* q : S->active) {
    if (q->state != RS_ACTIVE) continue;
    if (q->wait_in) {
      // a request joins the ticks once its input is on the device, so
      // the copies of later requests overlap the work of earlier ones
      if (cudaEventQuery(q->ev_in) != cudaSuccess) continue;
      q->wait_in = false;
    }
    now.push_back(&q->plan.ops[q->cursor++]);
    if (q->cursor == q->plan.ops.size()) finishing.push_back(q);
  }
  if (now.empty()) return HPEZ_OK;
  std::vector<unsigned char> tab;
  std::vector<Entry> es;
  build_tick(now, tab, es);
  const int k = S->ring;
  S->ring = (S->ring + 1) % kRing;
  if (S->tab_used[k]) cudaEventSynchronize(S->tab_ev[k]);
  if (S->h_tab_cap[k] < tab.size()) {
    if (S->h_tab[k]) cudaFreeHost(S->h_tab[k]);
    S->h_tab[k] = nullptr;
    const size_t cap = std::max(tab.size() * 2, (size_t)1 << 16);
    if (cudaMallocHost(&S->h_tab[k], cap) != cudaSuccess) {
      S->h_tab_cap[k] = 0;
      return HPEZ_ERR_NO_MEMORY;
    }
    S->h_tab_cap[k] = cap;
  }
  if (S->d_tab_cap < tab.size()) {
    cudaStreamSynchronize(s);
    if (S->d_tab) cudaFree(S->d_tab);
    S->d_tab = nullptr;
    const size_t cap = std::max(tab.size() * 2, (size_t)1 << 16);
    if (cudaMalloc(&S->d_tab, cap) != cudaSuccess) {
      S->d_tab_cap = 0;
      cudaGetLastError();
      return HPEZ_ERR_NO_MEMORY;
    }
    S->d_tab_cap = cap;
  }
  std::memcpy(S->h_tab[k], tab.data(), tab.size());
  cudaMemcpyAsync(S->d_tab, S->h_tab[k], tab.size(), cudaMemcpyHostToDevice, s);
  cudaEventRecord(S->tab_ev[k], s);
  S->tab_used[k] = true;
  enqueue_tick(es, S->d_tab, S->ctx->num_sms, S->ctx->batch_ctas, s, S->ts);
  S->launches += es.size();
  S->ctx->launches += es.size();
  ++S->ticks;
  if (!finishing.empty()) {
    cudaMemcpyAsync(S->h_sizes, S->d_sizes, sizeof(unsigned long long) * S->max_slots,
                    cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(S->h_status, S->d_status, sizeof(int) * S->max_slots,
                    cudaMemcpyDeviceToHost, s);
    for (SrvReq* q : finishing) {
      cudaEventRecord(q->ev, s);
      q->state = RS_RESULT;
    }
  }
  return cuda_check(cudaGetLastError());
}

int hpez_server_poll(hpez_server* S, int cap, uint64_t* ids, int32_t* status,
                     uint64_t* sizes, double* latency_s, int* n) {
  if (!S || !n || cap < 0) return HPEZ_ERR_INVALID_ARG;
  const double t = now_s();
  int k = 0;
  while (k < cap && !S->done.empty()) {
    SrvReq* q = S->done.front();
    S->done.erase(S->done.begin());
    if (ids) ids[k] = q->id;
    if (status) status[k] = q->status;
    if (sizes) sizes[k] = q->size;
    if (latency_s) latency_s[k] = t - q->t_submit;
    delete q;
    ++k;
  }
  *n = k;
  return HPEZ_OK;
}

int hpez_server_stats(hpez_server* S, int* active, int* queued,
                      uint64_t* used_bytes, uint64_t* ticks, uint64_t* launches) {
  if (!S) return HPEZ_ERR_INVALID_ARG;
  if (active) *active = (int)S->active.size();
  if (queued) *queued = (int)S->queue.size();
  if (used_bytes) *used_bytes = S->pool.used;
  if (ticks) *ticks = S->ticks;
  if (launches) *launches = S->launches;
  return HPEZ_OK;
}

int hpez_server_destroy(hpez_server* S) {
  if (!S) return HPEZ_OK;
  cudaSetDevice(S->device);
  cudaDeviceSynchronize();
  for (SrvReq* q : S->queue) delete q;
  for (SrvReq* q : S->active) {
    if (q->ev) cudaEventDestroy(q->ev);
    if (q->ev_in) cudaEventDestroy(q->ev_in);
    delete q;
  }
  if (S->s_in) cudaStreamDestroy(S->s_in);
  if (S->s_out) cudaStreamDestroy(S->s_out);
  S->ts.destroy();
  for (SrvReq* q : S->done) delete q;
  for (int k = 0; k < kRing; ++k) {
    if (S->h_tab[k]) cudaFreeHost(S->h_tab[k]);
    if (S->tab_ev[k]) cudaEventDestroy(S->tab_ev[k]);
  }
  if (S->d_tab) cudaFree(S->d_tab);
  if (S->pool_mem) cudaFree(S->pool_mem);
  if (S->d_sizes) cudaFree(S->d_sizes);
  if (S->d_status) cudaFree(S->d_status);
  if (S->h_sizes) cudaFreeHost(S->h_sizes);
  if (S->h_status) cudaFreeHost(S->h_status);
  delete S;
  return HPEZ_OK;
}

}  // extern "C"
