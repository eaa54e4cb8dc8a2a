// hpez_tune.cu -- hpez_tune (declared in include/hpez.h): the host side of
// the auto-tuner of Sec. 6.  It lays out the samples, builds the candidate
// thetas, launches the compression tests of k_tune.cu and takes the
// argmins over the integer scores the kernels return.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hpez.h"
#include "hpez_ctx.h"
#include "hpez_internal.cuh"
#include "hpez_launch.h"

using namespace hpez;
using namespace hpez::host;

namespace {

constexpr size_t kTuneSmemMax = 200 * 1024;
constexpr int kMaxVariants = 72;
const double kAlpha[5] = {1.0, 1.25, 1.5, 1.75, 2.0};
const double kBeta[4] = {2.0, 4.0, 8.0, 16.0};

// One candidate of the per-level tuning (Sec. 6.2); ord lists real dims.
struct Cand {
  int kind, md, same;
  uint8_t ord[3];
};

// Linear, not-a-knot, natural; for each the 1D-style orders of the
// interpolation dims (lexicographic) and then the multi-dimensional
// paradigm; for the cubic ones without and with same-level interpolation.
std::vector<Cand> candidates(const hpez_tune_params& tp, int ndim,
                             int frozen) {
  std::vector<int> dims;
  for (int d = 0; d < ndim; ++d)
    if (d != frozen) dims.push_back(d);
  const int k = (int)dims.size();
  std::vector<std::vector<int>> perms;
  std::vector<int> p = dims;
  do perms.push_back(p);
  while (std::next_permutation(p.begin(), p.end()));
  const int nvar = (int)perms.size() + (k >= 2 ? 1 : 0);
  std::vector<Cand> out;
  for (int kd = 0; kd < 3; ++kd) {
    if (kd == HPEZ_CUBIC_NAT && !tp.allow_natural) continue;
    const int nsl = (kd == HPEZ_LINEAR || !tp.allow_same_level) ? 1 : 2;
    for (int v = 0; v < nvar; ++v)
      for (int sl = 0; sl < nsl; ++sl) {
        Cand c;
        c.kind = kd;
        c.same = sl;
        c.md = v >= (int)perms.size();
        for (int q = 0; q < 3; ++q)
          c.ord[q] = (uint8_t)(q < k ? (c.md ? dims[q] : perms[v][q]) : 255);
        out.push_back(c);
      }
  }
  return out;
}

void set_level(hpez_config& c, int l, const Cand& k) {
  c.interp[l - 1] = (uint8_t)k.kind;
  c.paradigm[l - 1] = (uint8_t)(k.md ? HPEZ_PARADIGM_MD : HPEZ_PARADIGM_1D);
  c.same_level[l - 1] = (uint8_t)k.same;
  for (int q = 0; q < 3; ++q) c.order[l - 1][q] = k.ord[q];
}

// Device form of a theta: orders as slots, Eq. 14 weights per odd-slot
// mask; the level bounds are filled in on the device.
TuneCfg to_device(const Plan& p, const hpez_config& c) {
  TuneCfg t;
  std::memset(&t, 0, sizeof(t));
  for (int l = 0; l < kMaxLevels; ++l) {
    t.kind[l] = c.interp[l];
    t.md[l] = c.paradigm[l] == HPEZ_PARADIGM_MD;
    t.same[l] = c.same_level[l];
    for (int j = 0; j < 3; ++j)
      t.ord[l][j] = (uint8_t)(j < p.k ? c.order[l][j] + p.off : 0);
  }
  t.alpha = c.alpha;
  t.beta = c.beta;
  unsigned imask = 0;
  for (int s = 0; s < 3; ++s)
    if (p.interp[s]) imask |= 1u << s;
  for (unsigned S = 1; S < 8; ++S) {
    if ((S & imask) != S) continue;
    for (int s = 0; s < 3; ++s)
      if (S & (1u << s)) t.mdw[S][s] = md_weight(p, c, S, s);
  }
  return t;
}

// device buffers of one hpez_tune call
// histograms: the (alpha, beta) grid with and without freezing, then the
// two Lorenzo tests
constexpr int kMaxHists = 36;
constexpr int kLorenzoSlot = 34;

struct Bufs {
  Ctl* ctl;
  Ctl* ctl2;  // codebook status, one per histogram
  CodebookJob* cbjobs;
  unsigned long long* acc;
  TuneCfg* cfgs;
  TuneCfg* base;     // each variant's theta during the level rounds
  TuneCand* cands;   // the candidates of both variants
  uint8_t* choice;   // per variant and level: the chosen candidate
  unsigned long long* best;  // and its score
  unsigned long long* score;
  unsigned long long* nout;
  unsigned long long* cost;
  uint32_t* hists;
  unsigned long long* gkeys;  // codebook scratch of alphabets beyond shared memory
  unsigned long long* giw;
  uint8_t* bmap;
  unsigned long long* bscore;  // block-wise candidate scores
  float* state;                // sample blocks' reconstruction, per variant
};

struct Call {
  hpez_ctx* ctx;
  cudaStream_t s;
  const float* x;
  int ndim;
  const uint64_t* dims;
  const hpez_tune_params* tp;
  Bufs b;
};

int sync_check(Call& k) {
  const cudaError_t e = cudaStreamSynchronize(k.s);
  if (e != cudaSuccess) return cuda_check(e);
  return cuda_check(cudaGetLastError());
}

// Sample blocks of A+1 points every tau blocks per dim (Sec. 6.2), tau
// the smallest stride giving at most round(block_rate * N / A^ndim) (>= 1)
// blocks.  Returns the block count.
int sample_geometry(const Plan& p, const hpez_tune_params& tp, TuneGeom& g) {
  const int A = p.A;
  uint64_t nb[3], N = 1, vol = 1;
  for (int s = 0; s < 3; ++s) {
    g.n[s] = p.n[s];
    g.fst[s] = p.fst[s];
    g.interp[s] = p.interp[s];
    nb[s] = s < p.off ? 0 : (p.n[s] - 1) / (uint64_t)A;
  }
  for (int d = 0; d < p.ndim; ++d) {
    N *= p.n[d + p.off];
    vol *= (uint64_t)A;
  }
  g.k = p.k;
  g.off = p.off;
  g.A = A;
  g.L = p.L;
  const double tgt = std::floor(tp.block_rate * (double)N / (double)vol + 0.5);
  const uint64_t target = tgt < 1.0 ? 1 : (uint64_t)tgt;
  uint64_t tau = 1;
  for (;;) {
    uint64_t cnt = 1;
    for (int s = p.off; s < 3; ++s) {
      const uint64_t m = nb[s] ? nb[s] : 1;
      cnt *= (m + tau - 1) / tau;
    }
    if (cnt <= target) break;
    ++tau;
  }
  int total = 1;
  for (int s = 0; s < 3; ++s) {
    if (s < p.off) {
      g.ext[s] = 1;
      g.cnt[s] = 1;
      g.step[s] = 0;
    } else if (nb[s]) {
      g.ext[s] = (uint32_t)A + 1;
      g.cnt[s] = (uint32_t)((nb[s] + tau - 1) / tau);
      g.step[s] = (uint32_t)(tau * (uint64_t)A);
    } else {
      g.ext[s] = p.n[s];
      g.cnt[s] = 1;
      g.step[s] = 0;
    }
    total *= (int)g.cnt[s];
  }
  return total;
}

// anchors of one sample block (every interpolation coordinate a multiple
// of A)
uint64_t block_anchors(const TuneGeom& g) {
  uint64_t na = 1;
  for (int s = 0; s < 3; ++s)
    na *= g.interp[s] ? (g.ext[s] + (uint64_t)g.A - 1) / (uint64_t)g.A : g.ext[s];
  return na;
}

// Huffman bits of the histograms in `slots` into b.cost[0, n): one launch,
// a CTA per histogram
void hist_costs(Call& k, const std::vector<int>& slots) {
  uint64_t& nl = k.ctx->launches;
  const int n = (int)slots.size();
  CodebookJob jobs[kMaxHists];
  for (int v = 0; v < n; ++v) {
    const size_t h = (size_t)slots[v] * 65536, o = (size_t)v * 65536;
    // only the cost: no codes, tables, lengths or parents are written
    jobs[v] = CodebookJob{k.b.hists + h, nullptr, nullptr, nullptr, k.b.gkeys + o,
                          k.b.giw + o, nullptr, nullptr, k.b.ctl2 + v};
  }
  cudaMemsetAsync(k.b.ctl2, 0, sizeof(Ctl) * n, k.s);
  cudaMemcpyAsync(k.b.cbjobs, jobs, sizeof(CodebookJob) * n,
                  cudaMemcpyHostToDevice, k.s);
  launch_hcost_batch(k.b.cbjobs, n, k.b.cost, k.s);
  nl += 1;
}

// status of the histogram codebooks (0 when every one was built)
int costs_status(Call& k, int nvar) {
  std::vector<Ctl> st(nvar);
  cudaMemcpyAsync(st.data(), k.b.ctl2, sizeof(Ctl) * nvar, cudaMemcpyDeviceToHost,
                  k.s);
  int rc = sync_check(k);
  if (rc) return rc;
  for (int v = 0; v < nvar; ++v)
    if (st[v].status) return HPEZ_ERR_UNSUPPORTED;
  return HPEZ_OK;
}

// One global tuning (Sec. 6.2 + 6.4) for one choice of frozen dimension.
struct Variant {
  int frozen = -1;
  int slot = 0;        // report slot: 0 without, 1 with freezing
  hpez_config cfg;
  Plan p;
  TuneGeom g;
  int nblk = 0;
  std::vector<Cand> cands;
  uint64_t bits = 0;
};

int init_variant(Call& k, Variant& v, const double inv_var[3]) {
  const hpez_tune_params& tp = *k.tp;
  hpez_config& cfg = v.cfg;
  default_config(k.ndim, &cfg);
  if (tp.anchor_stride) cfg.anchor_stride = tp.anchor_stride;
  cfg.frozen_dim = v.frozen;
  for (int d = 0; d < 3; ++d) cfg.md_inv_var[d] = inv_var[d];
  for (int l = 0; l < HPEZ_MAX_LEVELS; ++l) {
    int q = 0;
    for (int d = 0; d < k.ndim; ++d)
      if (d != v.frozen) cfg.order[l][q++] = (uint8_t)d;
    for (; q < 3; ++q) cfg.order[l][q] = 255;
  }
  int rc = plan_geometry(v.p, k.ndim, k.dims, cfg.anchor_stride, v.frozen);
  if (rc) return rc;
  v.nblk = sample_geometry(v.p, tp, v.g);
  if (tune_test_smem(v.g) > kTuneSmemMax || tune_lorenzo_smem(v.g) > kTuneSmemMax)
    return HPEZ_ERR_UNSUPPORTED;
  // the Lorenzo wavefront keeps at most 4 (i0, i1) pairs per thread
  if ((uint64_t)v.g.ext[0] * v.g.ext[1] > 4096) return HPEZ_ERR_UNSUPPORTED;
  v.cands = candidates(tp, k.ndim, v.frozen);
  if ((int)v.cands.size() * 2 > kMaxVariants) return HPEZ_ERR_UNSUPPORTED;
  return HPEZ_OK;
}

// Sec. 6.2 + 6.4 for every variant at once: each level's candidate tests
// (and then the (alpha, beta) tests) of all variants go out together, with
// one synchronization per round.
int tune_globals(Call& k, std::vector<Variant>& vs, hpez_tune_report* rep,
                 const std::vector<int>& extra, cudaEvent_t extra_ready,
                 std::vector<unsigned long long>& extra_cost) {
  const hpez_tune_params& tp = *k.tp;
  uint64_t& nl = k.ctx->launches;
  PhaseProfiler& prof = k.ctx->prof;
  const int nv = (int)vs.size();
  std::vector<TuneCfg> host(kMaxVariants);
  int rc;
  if (rep) rep->n_sample_blocks = (uint32_t)vs[0].nblk;
  const int L = vs[0].p.L;
  if (tp.tune_levels) {
    // The levels' rounds run on the device end to end: each variant's
    // theta lives in b.base; a round expands it into the candidates of
    // level l, tests them, and selects the first best candidate into it
    // (the same choice as a host-side argmin); the choices come back once.
    const int n0 = (int)vs[0].cands.size(), n1 = nv > 1 ? (int)vs[1].cands.size() : 0;
    std::vector<TuneCand> tc;
    for (int i = 0; i < nv; ++i) {
      host[i] = to_device(vs[i].p, vs[i].cfg);
      for (const Cand& c : vs[i].cands) {
        TuneCand t;
        t.kind = (uint8_t)c.kind;
        t.md = (uint8_t)(c.md ? 1 : 0);
        t.same = (uint8_t)c.same;
        for (int j = 0; j < 3; ++j)
          t.ord[j] = (uint8_t)(j < vs[i].p.k ? c.ord[j] + vs[i].p.off : 0);
        tc.push_back(t);
      }
    }
    prof.begin(HPEZ_PH_TUNE_LEVELS, k.s);
    cudaMemcpyAsync(k.b.base, host.data(), sizeof(TuneCfg) * nv, cudaMemcpyHostToDevice,
                    k.s);
    cudaMemcpyAsync(k.b.cands, tc.data(), sizeof(TuneCand) * tc.size(),
                    cudaMemcpyHostToDevice, k.s);
    launch_tune_params(k.b.base, nv, kMaxLevels, k.b.ctl, k.s);
    nl += 1;
    prof.end(k.s);
    for (int l = L; l >= 1; --l) {
      prof.begin(HPEZ_PH_TUNE_LEVELS, k.s);
      launch_tune_expand(k.b.base, k.b.cands, n0, n1, l, k.b.cfgs, k.s);
      cudaMemsetAsync(k.b.score, 0, sizeof(unsigned long long) * (n0 + n1), k.s);
      // every variant's candidates in one launch (escapes unused here),
      // from the blocks' state after the levels above l
      launch_tune_test(k.x, vs[0].g, vs[nv - 1].g, n0, k.b.cfgs, n0 + n1, vs[0].nblk, l,
                       false, k.b.score, nullptr, nullptr, k.b.state, k.s);
      launch_tune_select(k.b.score, k.b.cands, n0, n1, nv, l, k.b.base, k.b.choice,
                         k.b.best, k.s);
      nl += 3;
      // the chosen level l of each variant, kept for the finer levels
      if (l > 1) {
        launch_tune_advance(k.x, vs[0].g, vs[nv - 1].g, nv, vs[0].nblk, k.b.base, l,
                            k.b.state, k.s);
        ++nl;
      }
      prof.end(k.s);
    }
    uint8_t choice[2 * kMaxLevels];
    unsigned long long best[2 * kMaxLevels];
    cudaMemcpyAsync(choice, k.b.choice, sizeof(choice), cudaMemcpyDeviceToHost, k.s);
    cudaMemcpyAsync(best, k.b.best, sizeof(best), cudaMemcpyDeviceToHost, k.s);
    if ((rc = sync_check(k))) return rc;
    for (int i = 0; i < nv; ++i)
      for (int l = L; l >= 1; --l) {
        const int c = choice[i * kMaxLevels + l - 1];
        set_level(vs[i].cfg, l, vs[i].cands[c]);
        if (rep) {
          rep->level_choice[vs[i].slot][l - 1] = (uint8_t)c;
          rep->level_score[vs[i].slot][l - 1] = best[i * kMaxLevels + l - 1];
        }
      }
  }

  // (alpha, beta): the grid, or the defaults alone
  std::vector<std::pair<double, double>> grid;
  if (tp.tune_eb) {
    grid.push_back({1.0, 1.0});
    for (int a = 1; a < 5; ++a)
      for (int b = 0; b < 4; ++b) grid.push_back({kAlpha[a], kBeta[b]});
  } else {
    grid.push_back({vs[0].cfg.alpha, vs[0].cfg.beta});
  }
  const int ng = (int)grid.size();
  // Pairs whose level factors min(alpha^(l-1), beta) (Eq. 15, the double
  // products the device forms) agree at every level the tests run give the
  // same level bounds, hence the same test: each distinct one runs once.
  const int Lt = std::max(vs[0].g.L, vs[nv - 1].g.L);
  std::vector<int> uniq_of(ng), reps;
  std::vector<std::vector<double>> facs;
  for (int v = 0; v < ng; ++v) {
    std::vector<double> f(Lt);
    for (int l = 1; l <= Lt; ++l) {
      double ap = 1.0;
      for (int i = 1; i < l; ++i) ap = ap * grid[v].first;
      f[l - 1] = ap < grid[v].second ? ap : grid[v].second;
    }
    int u = 0;
    while (u < (int)facs.size() && facs[u] != f) ++u;
    if (u == (int)facs.size()) {
      facs.push_back(f);
      reps.push_back(v);
    }
    uniq_of[v] = u;
  }
  const int nu = (int)reps.size();
  const int nh = nu * nv;
  for (int i = 0; i < nv; ++i)
    for (int u = 0; u < nu; ++u) {
      hpez_config c2 = vs[i].cfg;
      c2.alpha = grid[reps[u]].first;
      c2.beta = grid[reps[u]].second;
      host[i * nu + u] = to_device(vs[i].p, c2);
    }
  prof.begin(HPEZ_PH_TUNE_EB, k.s);
  cudaMemcpyAsync(k.b.cfgs, host.data(), sizeof(TuneCfg) * nh,
                  cudaMemcpyHostToDevice, k.s);
  launch_tune_params(k.b.cfgs, nh, kMaxLevels, k.b.ctl, k.s);
  cudaMemsetAsync(k.b.hists, 0, sizeof(uint32_t) * 65536 * nh, k.s);
  cudaMemsetAsync(k.b.nout, 0, sizeof(unsigned long long) * nh, k.s);
  cudaMemsetAsync(k.b.score, 0, sizeof(unsigned long long) * nh, k.s);
  launch_tune_test(k.x, vs[0].g, vs[nv - 1].g, nu, k.b.cfgs, nh, vs[0].nblk, 1,
                   true, k.b.score, k.b.hists, k.b.nout, nullptr, k.s);
  nl += 2;
  // the codebooks of these histograms and of the extra ones (the Lorenzo
  // tests, run on the side stream) in one launch
  std::vector<int> slots;
  for (int v = 0; v < nh; ++v) slots.push_back(v);
  if (!extra.empty()) {
    cudaStreamWaitEvent(k.s, extra_ready, 0);
    for (int v : extra) slots.push_back(v);
  }
  const int nc = (int)slots.size();
  hist_costs(k, slots);
  prof.end(k.s);
  std::vector<unsigned long long> cost(nc), nout(nh);
  cudaMemcpyAsync(cost.data(), k.b.cost, sizeof(unsigned long long) * nc,
                  cudaMemcpyDeviceToHost, k.s);
  cudaMemcpyAsync(nout.data(), k.b.nout, sizeof(unsigned long long) * nh,
                  cudaMemcpyDeviceToHost, k.s);
  if ((rc = costs_status(k, nc))) return rc;
  extra_cost.assign(cost.begin() + nh, cost.end());
  for (int i = 0; i < nv; ++i) {
    const uint64_t na = block_anchors(vs[i].g) * (uint64_t)vs[i].nblk;
    int best = 0;
    uint64_t best_bits = 0;
    for (int v = 0; v < ng; ++v) {
      const int h = i * nu + uniq_of[v];
      const uint64_t b = cost[h] + 32ull * nout[h] + 32ull * na;
      if (v == 0 || b < best_bits) {
        best_bits = b;
        best = v;
      }
    }
    vs[i].cfg.alpha = grid[best].first;
    vs[i].cfg.beta = grid[best].second;
    vs[i].bits = best_bits;
    if (rep) rep->bits[vs[i].slot] = best_bits;
  }
  return HPEZ_OK;
}

// the side stream and its two events (created on first use)
int ensure_aux(hpez_ctx* ctx) {
  int rc;
  if (!ctx->aux_stream &&
      (rc = cuda_check(cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking))))
    return rc;
  if (!ctx->aux_ev[0] &&
      ((rc = cuda_check(cudaEventCreateWithFlags(&ctx->aux_ev[0], cudaEventDisableTiming))) ||
       (rc = cuda_check(cudaEventCreateWithFlags(&ctx->aux_ev[1], cudaEventDisableTiming)))))
    return rc;
  return HPEZ_OK;
}

}  // namespace

extern "C" {

int hpez_default_tune_params(hpez_tune_params* t) {
  if (!t) return HPEZ_ERR_INVALID_ARG;
  std::memset(t, 0, sizeof(*t));
  t->sample_rate = 0.002;
  t->block_rate = 0.01;
  t->sub_frac = 0.04;
  t->lorenzo_coef = 1.0;
  t->block_size = 32;
  t->tune_levels = 1;
  t->tune_eb = 1;
  t->tune_freeze = 1;
  t->tune_lorenzo = 1;
  t->tune_blockwise = 1;
  t->allow_natural = 1;
  t->allow_same_level = 1;
  t->anchor_stride = 0;
  return HPEZ_OK;
}

uint64_t hpez_blockmap_size(int ndim, const uint64_t* dims, int bs) {
  if (!dims || bs < 1 || ndim < 1 || ndim > 3) return 0;
  uint64_t t = 1;
  for (int d = 0; d < ndim; ++d) t *= (dims[d] + (uint64_t)bs - 1) / (uint64_t)bs;
  return t;
}

int hpez_tune(hpez_ctx* ctx, const float* d_in, int ndim, const uint64_t* dims,
              int eb_mode, double eb, const hpez_tune_params* tp_in,
              hpez_config* h_cfg, uint8_t* h_blockmap, uint64_t blockmap_cap,
              hpez_tune_report* rep, void* stream) {
  if (!ctx || !d_in || !dims || !h_cfg || ndim < 1 || ndim > 3)
    return HPEZ_ERR_INVALID_ARG;
  hpez_tune_params tpd;
  if (!tp_in) {
    hpez_default_tune_params(&tpd);
    tp_in = &tpd;
  }
  const hpez_tune_params& tp = *tp_in;
  if (eb_mode != HPEZ_EB_ABS && eb_mode != HPEZ_EB_REL) return HPEZ_ERR_INVALID_ARG;
  if (!(eb > 0.0) || !std::isfinite(eb)) return HPEZ_ERR_INVALID_ARG;
  if (tp.block_size < 1 || !(tp.sample_rate > 0.0) || !(tp.block_rate > 0.0) ||
      !(tp.sub_frac > 0.0) || tp.sub_frac > 1.0)
    return HPEZ_ERR_INVALID_ARG;
  const uint64_t nbm = hpez_blockmap_size(ndim, dims, tp.block_size);
  if (tp.tune_blockwise && (!h_blockmap || blockmap_cap < nbm))
    return HPEZ_ERR_OUT_TOO_SMALL;
  if (rep) std::memset(rep, 0, sizeof(*rep));
  default_config(ndim, h_cfg);
  if (tp.anchor_stride) h_cfg->anchor_stride = tp.anchor_stride;
  Plan p0;
  int rc = plan_geometry(p0, ndim, dims, h_cfg->anchor_stride, -1);
  if (rc) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  Arena ar;
  const size_t o_ctl = ar.take<Ctl>(1);
  const size_t o_ctl2 = ar.take<Ctl>(kMaxHists);
  const size_t o_cbjobs = ar.take<CodebookJob>(kMaxHists);
  const size_t o_acc = ar.take<unsigned long long>(8);
  const size_t o_cfgs = ar.take<TuneCfg>(kMaxVariants);
  const size_t o_base = ar.take<TuneCfg>(2);
  const size_t o_cands = ar.take<TuneCand>(kMaxVariants);
  const size_t o_choice = ar.take<uint8_t>(2 * kMaxLevels);
  const size_t o_best = ar.take<unsigned long long>(2 * kMaxLevels);
  const size_t o_score = ar.take<unsigned long long>(kMaxVariants);
  const size_t o_nout = ar.take<unsigned long long>(kMaxVariants);
  const size_t o_cost = ar.take<unsigned long long>(kMaxVariants);
  const size_t o_hists = ar.take<uint32_t>((size_t)65536 * kMaxHists);
  const size_t o_gkeys = ar.take<unsigned long long>((size_t)65536 * kMaxHists);
  const size_t o_giw = ar.take<unsigned long long>((size_t)65536 * kMaxHists);
  const size_t o_bmap = ar.take<uint8_t>(nbm ? nbm : 1);
  const size_t o_bscore = ar.take<unsigned long long>(5 * (nbm ? nbm : 1));
  // the sample blocks' state, per frozen-dimension variant
  TuneGeom gs;
  const int nblk0 = sample_geometry(p0, tp, gs);
  const size_t o_state =
      ar.take<float>(2 * (size_t)nblk0 * (tune_test_smem(gs) / sizeof(float)));
  if ((rc = ensure_scratch(ctx, ar.off))) return rc;
  char* base = ctx->scratch;
  Call k;
  k.ctx = ctx;
  k.s = s;
  k.x = d_in;
  k.ndim = ndim;
  k.dims = dims;
  k.tp = &tp;
  k.b.ctl = reinterpret_cast<Ctl*>(base + o_ctl);
  k.b.ctl2 = reinterpret_cast<Ctl*>(base + o_ctl2);
  k.b.cbjobs = reinterpret_cast<CodebookJob*>(base + o_cbjobs);
  k.b.acc = reinterpret_cast<unsigned long long*>(base + o_acc);
  k.b.cfgs = reinterpret_cast<TuneCfg*>(base + o_cfgs);
  k.b.base = reinterpret_cast<TuneCfg*>(base + o_base);
  k.b.cands = reinterpret_cast<TuneCand*>(base + o_cands);
  k.b.choice = reinterpret_cast<uint8_t*>(base + o_choice);
  k.b.best = reinterpret_cast<unsigned long long*>(base + o_best);
  k.b.score = reinterpret_cast<unsigned long long*>(base + o_score);
  k.b.nout = reinterpret_cast<unsigned long long*>(base + o_nout);
  k.b.cost = reinterpret_cast<unsigned long long*>(base + o_cost);
  k.b.hists = reinterpret_cast<uint32_t*>(base + o_hists);
  k.b.gkeys = reinterpret_cast<unsigned long long*>(base + o_gkeys);
  k.b.giw = reinterpret_cast<unsigned long long*>(base + o_giw);
  k.b.bmap = reinterpret_cast<uint8_t*>(base + o_bmap);
  k.b.bscore = reinterpret_cast<unsigned long long*>(base + o_bscore);
  k.b.state = reinterpret_cast<float*>(base + o_state);
  uint64_t& nl = ctx->launches;
  PhaseProfiler& prof = ctx->prof;

  // the absolute bound, exactly as the compressor derives it
  launch_init_ctl(k.b.ctl, s);
  ++nl;
  if (eb_mode == HPEZ_EB_REL) {
    prof.begin(HPEZ_PH_RANGE, s);
    launch_range(d_in, p0.N, k.b.ctl, ctx->num_sms, s);
    prof.end(s);
    ++nl;
  }
  launch_params(k.b.ctl, eb_mode, eb, 1.0, 1.0, p0.L, d_in, s);
  ++nl;
  cudaMemcpyAsync(ctx->h_ctl, k.b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
  if ((rc = sync_check(k))) return rc;
  if (ctx->h_ctl->status) return map_status(ctx->h_ctl->status);
  ctx->range_x = nullptr;
  if (eb_mode == HPEZ_EB_REL && !ctx->h_ctl->nonfinite) {
    ctx->range_x = d_in;
    ctx->range_n = p0.N;
    ctx->range_kmin = ctx->h_ctl->vmin_key;
    ctx->range_kmax = ctx->h_ctl->vmax_key;
  }
  if (ctx->h_ctl->is_const) {
    prof.collect();
    return HPEZ_OK;  // constant field: nothing to tune
  }

  // Sec. 6.1 statistics on the lattice
  int t = 1;
  for (;;) {
    double pp = 1.0;
    for (int d = 0; d < ndim; ++d) pp *= (double)t;
    if (pp * tp.sample_rate >= 1.0) break;
    ++t;
  }
  bool ok = true;
  int real[3];
  for (int sl = 0; sl < 3; ++sl) {
    real[sl] = sl >= p0.off;
    if (real[sl] && p0.n[sl] < 7) ok = false;
  }
  unsigned long long acc[8] = {0};
  if (ok) {
    prof.begin(HPEZ_PH_TUNE_STATS, s);
    cudaMemsetAsync(k.b.acc, 0, sizeof(unsigned long long) * 8, s);
    launch_tune_stats(d_in, p0.n, p0.fst, real, t, k.b.ctl, k.b.acc,
                      ctx->num_sms, s);
    ++nl;
    prof.end(s);
    cudaMemcpyAsync(acc, k.b.acc, sizeof(acc), cudaMemcpyDeviceToHost, s);
    if ((rc = sync_check(k))) return rc;
  }
  const uint64_t cnt = acc[0];
  double inv_var[3] = {1.0, 1.0, 1.0};
  int nonsmooth = -1;
  if (cnt) {
    uint64_t mx = 0;
    for (int d = 0; d < ndim; ++d) {
      const uint64_t cub = acc[4 + d + p0.off];
      inv_var[d] = (double)cnt * 256.0 / (double)(cub ? cub : 1);
      if (nonsmooth < 0 || cub > mx) {
        mx = cub;
        nonsmooth = d;
      }
    }
  }
  if (rep) {
    rep->stats_count = cnt;
    for (int d = 0; d < 3; ++d) {
      rep->mse_lin[d] = d < ndim ? acc[1 + d + p0.off] : 0;
      rep->mse_cub[d] = d < ndim ? acc[4 + d + p0.off] : 0;
    }
    rep->nonsmooth_dim = nonsmooth;
    rep->froze = 0;
  }

  // Sec. 6.2 + 6.4 without freezing, and (Sec. 6.3) with the most
  // non-smooth dim frozen, side by side; the smaller estimate wins
  std::vector<Variant> vs(1);
  vs[0].frozen = -1;
  vs[0].slot = 0;
  if (tp.tune_freeze && cnt && ndim >= 2) {
    vs.emplace_back();
    vs[1].frozen = nonsmooth;
    vs[1].slot = 1;
  }
  for (Variant& v : vs)
    if ((rc = init_variant(k, v, inv_var))) return rc;
  // Sec. 6.5: order-1 and order-2 Lorenzo tests on the same sample blocks,
  // on a side stream, overlapping the candidate tests
  std::vector<int> lor_slots;
  if ((tp.tune_lorenzo || tp.tune_blockwise) && (rc = ensure_aux(ctx))) return rc;
  if (tp.tune_lorenzo) {
    cudaStream_t s2 = ctx->aux_stream;
    cudaEventRecord(ctx->aux_ev[0], s);
    cudaStreamWaitEvent(s2, ctx->aux_ev[0], 0);
    prof.begin(HPEZ_PH_TUNE_LORENZO, s2);
    cudaMemsetAsync(k.b.hists + (size_t)kLorenzoSlot * 65536, 0,
                    sizeof(uint32_t) * 65536 * 2, s2);
    cudaMemsetAsync(k.b.nout + kLorenzoSlot, 0, sizeof(unsigned long long) * 2, s2);
    launch_tune_lorenzo(d_in, vs[0].g, vs[0].nblk, k.b.ctl,
                        k.b.hists + (size_t)kLorenzoSlot * 65536,
                        k.b.nout + kLorenzoSlot, s2);
    prof.end(s2);
    cudaEventRecord(ctx->aux_ev[1], s2);
    ++nl;
    lor_slots = {kLorenzoSlot, kLorenzoSlot + 1};
  }
  std::vector<unsigned long long> lor_cost;
  if ((rc = tune_globals(k, vs, rep, lor_slots, ctx->aux_ev[1], lor_cost))) return rc;
  hpez_config out = vs[0].cfg;
  uint64_t bits_best = vs[0].bits;
  if (vs.size() > 1 && vs[1].bits < vs[0].bits) {
    out = vs[1].cfg;
    bits_best = vs[1].bits;
    if (rep) rep->froze = 1;
  }

  // Lorenzo bits from the costs and escapes computed above
  if (tp.tune_lorenzo) {
    unsigned long long nout[2];
    cudaMemcpyAsync(nout, k.b.nout + kLorenzoSlot, sizeof(nout),
                    cudaMemcpyDeviceToHost, s);
    if ((rc = sync_check(k))) return rc;
    const uint64_t lb0 = lor_cost[0] + 32ull * nout[0];
    const uint64_t lb1 = lor_cost[1] + 32ull * nout[1];
    const uint64_t m = lb0 <= lb1 ? lb0 : lb1;
    const bool better = (double)m * tp.lorenzo_coef < (double)bits_best;
    if (rep) {
      rep->lorenzo_bits[0] = lb0;
      rep->lorenzo_bits[1] = lb1;
      rep->lorenzo_better = better;
    }
    // Sec. 6.5: the Lorenzo predictor of the order with the smaller
    // estimate (order 1 on a tie) replaces interpolation when it wins;
    // block-wise interpolator tuning then has nothing to choose
    if (better) {
      out.predictor = lb0 <= lb1 ? 1 : 2;
      prof.collect();
      *h_cfg = out;
      return HPEZ_OK;
    }
  }

  // Sec. 6.6: block-wise interpolator map
  if (tp.tune_blockwise) {
    Plan p;
    if ((rc = plan_geometry(p, ndim, dims, out.anchor_stride, out.frozen_dim)))
      return rc;
    const int bsz = tp.block_size;
    const double q0 = 32.0 * std::pow(tp.sub_frac, 1.0 / (double)ndim);
    int Q = (int)std::floor((double)bsz / 32.0 * q0 + 0.5);
    if (Q < 5) Q = 5;
    size_t vol = 1;
    for (int d = 0; d < ndim; ++d) vol *= (size_t)std::min(Q, bsz);
    if (vol * sizeof(float) > kTuneSmemMax) return HPEZ_ERR_UNSUPPORTED;
    TuneGeom g;
    sample_geometry(p, tp, g);
    uint32_t nb[3];
    for (int sl = 0; sl < 3; ++sl)
      nb[sl] = sl < p.off ? 1u : (p.n[sl] + (uint32_t)bsz - 1) / (uint32_t)bsz;
    TuneCfg host = to_device(p, out);
    prof.begin(HPEZ_PH_TUNE_BLOCKS, s);
    cudaMemcpyAsync(k.b.cfgs, &host, sizeof(TuneCfg), cudaMemcpyHostToDevice, s);
    launch_tune_params(k.b.cfgs, 1, kMaxLevels, k.b.ctl, s);
    const unsigned allow = (tp.allow_natural ? 1u : 0u) | (tp.allow_same_level ? 2u : 0u);
    nl += 1 + launch_tune_blockwise(d_in, g, bsz, Q,
                                    out.frozen_dim < 0 ? -1 : out.frozen_dim + p.off, nb,
                                    (uint32_t)nbm, k.b.cfgs, allow, k.b.bscore, k.b.bmap, s,
                                    ctx->aux_stream, ctx->aux_ev[0], ctx->aux_ev[1]);
    prof.end(s);
    cudaMemcpyAsync(h_blockmap, k.b.bmap, nbm, cudaMemcpyDeviceToHost, s);
    if ((rc = sync_check(k))) return rc;
    out.blockwise = 1;
    out.block_size = bsz;
    out.h_blockmap = h_blockmap;
  }
  prof.collect();
  *h_cfg = out;
  return HPEZ_OK;
}

int hpez_compress_auto(hpez_ctx* ctx, const float* d_in, int ndim,
                       const uint64_t* dims, int eb_mode, double eb,
                       const hpez_tune_params* tp, void* d_out, uint64_t out_cap,
                       uint64_t* h_out_size, hpez_tune_report* h_report,
                       void* stream) {
  if (!ctx || !dims || ndim < 1 || ndim > 3) return HPEZ_ERR_INVALID_ARG;
  const int bs = tp ? tp->block_size : 32;
  const uint64_t nbm = hpez_blockmap_size(ndim, dims, bs);
  std::vector<uint8_t>& bm = ctx->h_bmap;
  if (bm.size() < nbm) bm.resize(nbm);
  hpez_config cfg;
  int rc = hpez_tune(ctx, d_in, ndim, dims, eb_mode, eb, tp, &cfg,
                     bm.empty() ? nullptr : bm.data(), bm.size(), h_report, stream);
  if (rc) return rc;
  ctx->range_hint_on = true;  // the tuner's pass over d_in found the range
  rc = hpez_compress(ctx, d_in, ndim, dims, eb_mode, eb, &cfg, d_out, out_cap,
                     h_out_size, stream);
  ctx->range_hint_on = false;
  return rc;
}

int hpez_compress_auto_host(hpez_ctx* ctx, const float* h_in, int ndim,
                            const uint64_t* dims, int eb_mode, double eb,
                            const hpez_tune_params* tp, void* h_out,
                            uint64_t out_cap, uint64_t* h_out_size, void* stream) {
  if (!ctx || !h_in || !h_out || !h_out_size || !dims || ndim < 1 || ndim > 3)
    return HPEZ_ERR_INVALID_ARG;
  uint64_t N = 1;
  for (int d = 0; d < ndim; ++d) N *= dims[d];
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = ensure_io(&ctx->io_in, &ctx->io_in_cap, N * sizeof(float));
  if (!rc) rc = ensure_io(&ctx->io_out, &ctx->io_out_cap, out_cap);
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(ctx->io_in, h_in, N * sizeof(float),
                                    cudaMemcpyHostToDevice, s));
  if (!rc)
    rc = hpez_compress_auto(ctx, static_cast<const float*>(ctx->io_in), ndim, dims,
                            eb_mode, eb, tp, ctx->io_out, out_cap, h_out_size,
                            nullptr, stream);
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(h_out, ctx->io_out, *h_out_size,
                                    cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  return rc;
}

}  // extern "C"
