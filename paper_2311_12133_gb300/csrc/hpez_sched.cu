// hpez_sched.cu -- the level-schedule table of the batched and served
// forms: keys, entries, the text file, and the context's copy.  Host code
// only; the offline search that fills the table is in hpez_engine.cu.
//
// A schedule says how the GPU runs one level (kernel family, tile shape,
// chunks of planes), never what it computes: every stream and field is the
// same under any table.
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "hpez_ctx.h"

using namespace hpez;
using namespace hpez::host;

namespace {

// half-octave class of an extent: floor(2 log2 n) = floor(log2 n^2)
int half_octave(uint32_t n) {
  const unsigned long long sq = (unsigned long long)n * n;
  int c = 0;
  while (c < 63 && (sq >> (c + 1)) != 0) ++c;
  return c;
}

std::array<int32_t, 8> to_array(const hpez_level_key& k) {
  return {k.ndim, k.cls[0], k.cls[1], k.cls[2], k.stride, k.interp, k.paradigm, k.decomp};
}

hpez_level_key from_array(const std::array<int32_t, 8>& a) {
  hpez_level_key k;
  k.ndim = a[0];
  k.cls[0] = a[1];
  k.cls[1] = a[2];
  k.cls[2] = a[3];
  k.stride = a[4];
  k.interp = a[5];
  k.paradigm = a[6];
  k.decomp = a[7];
  return k;
}

bool key_ok(const hpez_level_key& k) {
  if (k.ndim < 1 || k.ndim > 3) return false;
  for (int s = 0; s < 3; ++s)
    if (k.cls[s] < 0 || k.cls[s] > 64) return false;
  if (k.stride < 1 || k.stride > (1 << 20) || (k.stride & (k.stride - 1))) return false;
  if (k.interp < 0 || k.interp > 3) return false;
  if (k.paradigm < 0 || k.paradigm > 1) return false;
  return k.decomp == 0 || k.decomp == 1;
}

bool sched_ok(const hpez_level_sched& v) {
  if (v.family < HPEZ_FAM_LEVEL3D || v.family > HPEZ_FAM_PASS) return false;
  for (int s = 0; s < 3; ++s)
    if (v.tile[s] < 0 || v.tile[s] > 4096) return false;
  if (v.chunks < 0 || v.chunks > 65536) return false;
  return std::isfinite(v.time_us);
}

}  // namespace

namespace hpez {
namespace host {

std::array<int32_t, 8> sched_key(const Plan& p, const hpez_config& sc, int l, bool decomp) {
  const bool per_point = sc.blockwise || sc.same_level[l - 1];
  return {p.ndim,
          half_octave(p.n[0]),
          half_octave(p.n[1]),
          half_octave(p.n[2]),
          1 << (l - 1),
          per_point ? 3 : (int32_t)sc.interp[l - 1],
          (int32_t)sc.paradigm[l - 1],
          decomp ? 1 : 0};
}

}  // namespace host
}  // namespace hpez

extern "C" {

int hpez_tuning_create(hpez_tuning** out) {
  if (!out) return HPEZ_ERR_INVALID_ARG;
  *out = new hpez_tuning();
  return HPEZ_OK;
}

int hpez_tuning_destroy(hpez_tuning* t) {
  delete t;
  return HPEZ_OK;
}

int hpez_tuning_set(hpez_tuning* t, const hpez_level_key* key, const hpez_level_sched* sched) {
  if (!t || !key || !sched || !key_ok(*key) || !sched_ok(*sched)) return HPEZ_ERR_INVALID_ARG;
  t->m[to_array(*key)] = *sched;
  return HPEZ_OK;
}

int hpez_tuning_get(const hpez_tuning* t, const hpez_level_key* key, hpez_level_sched* sched,
                    int* found) {
  if (!t || !key || !sched || !found) return HPEZ_ERR_INVALID_ARG;
  const auto it = t->m.find(to_array(*key));
  *found = it != t->m.end() ? 1 : 0;
  if (*found) *sched = it->second;
  return HPEZ_OK;
}

int hpez_tuning_count(const hpez_tuning* t, uint64_t* n) {
  if (!t || !n) return HPEZ_ERR_INVALID_ARG;
  *n = t->m.size();
  return HPEZ_OK;
}

int hpez_tuning_save(const hpez_tuning* t, const char* path) {
  if (!t || !path) return HPEZ_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "w");
  if (!f) return HPEZ_ERR_INVALID_ARG;
  std::fprintf(f,
               "# level schedules: ndim cls0 cls1 cls2 stride interp paradigm decomp"
               " family tile0 tile1 tile2 chunks time_us\n");
  for (const auto& kv : t->m) {
    const auto& a = kv.first;
    const hpez_level_sched& v = kv.second;
    std::fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %d %.3f\n", a[0], a[1], a[2], a[3],
                 a[4], a[5], a[6], a[7], v.family, v.tile[0], v.tile[1], v.tile[2], v.chunks,
                 (double)v.time_us);
  }
  const bool ok = std::fflush(f) == 0;
  std::fclose(f);
  return ok ? HPEZ_OK : HPEZ_ERR_INVALID_ARG;
}

int hpez_tuning_load(hpez_tuning* t, const char* path) {
  if (!t || !path) return HPEZ_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) return HPEZ_ERR_INVALID_ARG;
  hpez_tuning add;
  char line[512];
  bool ok = true;
  while (ok && std::fgets(line, sizeof line, f)) {
    const size_t n = std::strlen(line);
    if (n + 1 == sizeof line && line[n - 1] != '\n') {
      ok = false;  // an overlong line
      break;
    }
    const char* c = line;
    while (*c == ' ' || *c == '\t') ++c;
    if (*c == '#' || *c == '\n' || *c == '\r' || *c == 0) continue;
    long v[13];
    char* e = const_cast<char*>(c);
    for (int i = 0; i < 13 && ok; ++i) {
      errno = 0;
      char* q;
      v[i] = std::strtol(e, &q, 10);
      if (q == e || errno || v[i] < -1000000 || v[i] > 1000000) ok = false;
      e = q;
    }
    if (!ok) break;
    errno = 0;
    char* q;
    const double tu = std::strtod(e, &q);
    if (q == e || errno) {
      ok = false;
      break;
    }
    while (*q == ' ' || *q == '\t' || *q == '\r' || *q == '\n') ++q;
    if (*q) {
      ok = false;
      break;
    }
    hpez_level_key k;
    k.ndim = (int32_t)v[0];
    for (int s = 0; s < 3; ++s) k.cls[s] = (int32_t)v[1 + s];
    k.stride = (int32_t)v[4];
    k.interp = (int32_t)v[5];
    k.paradigm = (int32_t)v[6];
    k.decomp = (int32_t)v[7];
    hpez_level_sched sc;
    sc.family = (int32_t)v[8];
    for (int s = 0; s < 3; ++s) sc.tile[s] = (int32_t)v[9 + s];
    sc.chunks = (int32_t)v[12];
    sc.time_us = (float)tu;
    if (!key_ok(k) || !sched_ok(sc)) {
      ok = false;
      break;
    }
    add.m[to_array(k)] = sc;
  }
  if (std::ferror(f)) ok = false;
  std::fclose(f);
  if (!ok) return HPEZ_ERR_INVALID_ARG;
  for (const auto& kv : add.m) t->m[kv.first] = kv.second;
  return HPEZ_OK;
}

int hpez_level_key_of(int ndim, const uint64_t* dims, const hpez_config* cfg_in, int level,
                      int decomp, hpez_level_key* out) {
  if (!dims || !out || ndim < 1 || ndim > 3) return HPEZ_ERR_INVALID_ARG;
  hpez_config cfg;
  if (cfg_in)
    cfg = *cfg_in;
  else
    default_config(ndim, &cfg);
  Plan p;
  int rc = plan_geometry(p, ndim, dims, cfg.anchor_stride, cfg.frozen_dim);
  if (rc) return rc;
  if ((rc = check_config(p, cfg))) return rc;
  if (level < 1 || level > p.L) return HPEZ_ERR_INVALID_ARG;
  if (cfg.blockwise && !cfg.h_blockmap) return HPEZ_ERR_INVALID_ARG;
  plan_chunks_blocks(p, cfg);
  // compress runs the sweep config (a uniform block map becomes its
  // interpolator); decompress plans from the stream's header config
  const hpez_config sc = decomp ? cfg : sweep_config(cfg, cfg.h_blockmap, p.nblocks);
  *out = from_array(sched_key(p, sc, level, decomp != 0));
  return HPEZ_OK;
}

int hpez_use_tuning(hpez_ctx* ctx, const hpez_tuning* t) {
  if (!ctx) return HPEZ_ERR_INVALID_ARG;
  if (t)
    ctx->sched.m = t->m;
  else
    ctx->sched.m.clear();
  return HPEZ_OK;
}

}  // extern "C"
