// hpez_ctx.h -- host-side state shared by the C-ABI translation units:
// the context, its phase profiler, the field geometry plan and the scratch
// arena, and the plan/config helpers that compress, decompress and the
// tuner all use.
#pragma once

#include <array>
#include <cstdint>
#include <map>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "hpez.h"
#include "hpez_internal.cuh"

// Opt-in phase timer: CUDA events recorded on the call's stream around
// each phase, read after the call's final synchronization.
struct PhaseProfiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
  double total_ms[HPEZ_PROFILE_PHASES] = {};
  uint64_t count[HPEZ_PROFILE_PHASES] = {};
  cudaEvent_t take() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  void begin(int ph, cudaStream_t s) {
    if (!on) return;
    cudaEvent_t e = take();
    cudaEventRecord(e, s);
    marks.push_back({ph, {e, nullptr}});
  }
  void end(cudaStream_t s) {
    if (!on || marks.empty()) return;
    cudaEvent_t e = take();
    cudaEventRecord(e, s);
    marks.back().second.second = e;
  }
  // after the stream has been synchronized
  void collect() {
    for (auto& m : marks) {
      float ms = 0.f;
      if (m.second.second &&
          cudaEventElapsedTime(&ms, m.second.first, m.second.second) == cudaSuccess) {
        total_ms[m.first] += ms;
        count[m.first] += 1;
      }
    }
    marks.clear();
    used = 0;
    cudaGetLastError();
  }
  void reset() {
    marks.clear();
    used = 0;
    for (int i = 0; i < HPEZ_PROFILE_PHASES; ++i) {
      total_ms[i] = 0;
      count[i] = 0;
    }
  }
  ~PhaseProfiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// A table of level schedules of the batched and served forms, keyed by
// (ndim, cls0, cls1, cls2, stride, interp, paradigm, decomp).
struct hpez_tuning {
  std::map<std::array<int32_t, 8>, hpez_level_sched> m;
};

struct hpez_ctx {
  PhaseProfiler prof;
  hpez_tuning sched;           // hpez_use_tuning's copy (empty: fixed rules)
  uint64_t launches = 0;
  int fused_levels = 1;        // HPEZ_OPT_FUSED_LEVELS
  int level3d = 1;             // HPEZ_OPT_LEVEL3D
  int stream_levels = 1;       // HPEZ_OPT_STREAM_LEVELS
  int warp_levels = 1;         // HPEZ_OPT_WARP_LEVELS
  int drop_copy = 0;           // HPEZ_OPT_DROP_COPY
  int stream_chunks = 0;       // HPEZ_OPT_STREAM_CHUNKS (0 = heuristic)
  int lorenzo_ctas = 0;        // HPEZ_OPT_LORENZO_CTAS (0 = resident CTAs)
  int batch_ctas = 0;          // HPEZ_OPT_BATCH_CTAS (0 = resident CTAs)
  // the value range of the last tuned input (order-preserving keys), which
  // the compress call of hpez_compress_auto reuses instead of a second pass
  bool range_hint_on = false;
  const void* range_x = nullptr;
  uint64_t range_n = 0;
  unsigned range_kmin = 0, range_kmax = 0;
  bool x_aligned16 = true;     // per call: input pointer 16-byte aligned
  bool codes_aligned16 = true;
  bool out_aligned16 = true;   // per call: decompress output 16-byte aligned
  int tile_e[3] = {0, 0, 0};   // HPEZ_OPT_TILE_E0..2 (0 = heuristic)
  size_t fused_smem_cap = 96 * 1024;
  int device = 0;
  int num_sms = 152;
  char* scratch = nullptr;
  size_t scratch_cap = 0;
  hpez::Ctl* h_ctl = nullptr;        // pinned
  uint8_t* h_hdr = nullptr;    // pinned, 512 bytes
  void* io_in = nullptr;       // device staging for the *_host calls
  size_t io_in_cap = 0;
  void* io_out = nullptr;
  size_t io_out_cap = 0;
  void* typed_buf = nullptr;   // binary32 staging of the typed and PSNR-target calls
  size_t typed_cap = 0;
  void* typed_red = nullptr;   // their reduction words (256 bytes)
  void* lz_buf = nullptr;      // scratch of the lossless stage
  size_t lz_cap = 0;
  void* lz_stream = nullptr;   // a stream with the lossless stage undone
  size_t lz_stream_cap = 0;
  std::vector<uint8_t> h_bmap;  // block map of the last auto-tuned compress
  cudaStream_t aux_stream = nullptr;  // the tuner's side stream
  cudaEvent_t aux_ev[2] = {nullptr, nullptr};
};

namespace hpez {
namespace host {

// ---------------------------------------------------------------------
// header layout (byte offsets)
// ---------------------------------------------------------------------
enum : int {
  H_MAGIC = 0, H_VERSION = 4, H_FLAGS = 8, H_NDIM = 12, H_DIMS = 16,
  H_EBMODE = 40, H_ANCHOR = 44, H_EBVALUE = 48, H_E = 56, H_CONST = 60,
  H_FROZEN = 64, H_CHUNK = 68, H_ALPHA = 72, H_BETA = 80, H_MDIV = 88,
  H_INTERP = 112, H_PARADIGM = 128, H_SAME = 144, H_ORDER = 160,
  H_PREDICTOR = 208, H_BLOCKWISE = 212, H_NANCHORS = 216, H_NOUTLIERS = 224,
  H_NUSED = 232, H_BLOCKSIZE = 236, H_NCHUNKS = 240, H_TOTALWORDS = 248,
  H_OFF_ANCHORS = 256, H_OFF_CHUNKW = 264, H_OFF_TABLE = 272,
  H_OFF_OUTLIERS = 280, H_OFF_BITS = 288, H_OFF_BLOCKMAP = 296,
  H_TOTAL = 304, H_NBLOCKS = 312
};
constexpr uint32_t kMagic = 0x5A455048u;  // "HPEZ"
constexpr uint32_t kVersion = 1u;

// geometry plan
struct Plan {
  int ndim = 0, off = 0;
  uint32_t n[3] = {1, 1, 1};
  uint32_t fst[3] = {0, 0, 1};
  uint32_t N = 1;
  bool interp[3] = {false, false, false};
  int k = 0, A = 0, L = 0;
  LevelGeom grid[kMaxLevels + 1];  // grid[g]: stride 2^g (g = L: anchors)
  uint32_t gsize[kMaxLevels + 1];
  uint32_t C = 4096, nch = 0;
  uint32_t nb[3] = {1, 1, 1};
  uint32_t nblocks = 0;
};

// scratch arena: 256-byte aligned sub-allocations of one device buffer
struct Arena {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    const size_t o = (off + 255) & ~(size_t)255;
    off = o + count * sizeof(T);
    return o;
  }
};

// one launch of the per-pass path
struct Launch {
  PassBox pb;
  int group;  // launches of the same group are independent
};

int plan_geometry(Plan& p, int ndim, const uint64_t* dims, int A, int frozen);
void plan_chunks_blocks(Plan& p, const hpez_config& c);
std::vector<Launch> level_schedule(const Plan& p, const hpez_config& c, int l);
bool plan_fused(const hpez_ctx* ctx, const Plan& p, const hpez_config& c, int l,
                bool decomp, FusedLevel& F);
bool plan_level3d(const hpez_ctx* ctx, const Plan& p, const hpez_config& c,
                  int l, bool decomp, Level3D& F);
uint64_t n_anchors(const Plan& p);
bool plan_md(const hpez_ctx* ctx, const Plan& p, const hpez_config& c, int l,
             bool decomp, LevelMD& F);
// the schedule-table key of level l of a planned field (sc: the config
// the sweep runs)
std::array<int32_t, 8> sched_key(const Plan& p, const hpez_config& sc, int l, bool decomp);
// a 3D multi-dimensional level as even-plane and odd-plane launches of
// E1-row tiles (HPEZ_OPT_TILE_E1 > 0 sets the rows)
bool plan_md3(const hpez_ctx* ctx, const Plan& p, const hpez_config& c, int l,
              bool decomp, LevelMD& F, int& E1);
// the predictor a sweep runs: a block map with one interpolator for every
// block becomes that interpolator at every level
hpez_config sweep_config(const hpez_config& c, const uint8_t* h_bmap,
                         uint32_t nblocks);
void header_templates(const Plan& p, const hpez_config& c, int eb_mode,
                      double eb, uint64_t off_anchors, uint64_t off_bmap,
                      uint64_t off_chw, uint8_t* h, uint8_t* hc);
uint64_t a16(uint64_t v);

// a validated stream header
struct StreamInfo {
  int nd;
  uint64_t dims[3];
  uint64_t N;
  hpez_config cfg;
  bool is_const;
  float const_value;
  Plan p;
  float e;
  uint64_t na, nout, nch, twords;
  uint32_t nused;
  uint64_t oa, ocw, ot, oo, ob, obm;
};
int parse_stream_header(const uint8_t* h, uint64_t in_size, StreamInfo& si);
uint32_t rd32(const uint8_t* b, int o);
uint64_t rd64(const uint8_t* b, int o);
double rdf64(const uint8_t* b, int o);
float rdf32(const uint8_t* b, int o);
int check_config(const Plan& p, const hpez_config& c);
// Eq. 14 weight of slot `slot` within the slot mask S
float md_weight(const Plan& p, const hpez_config& c, unsigned S, int slot);
int ensure_scratch(hpez_ctx* ctx, size_t bytes);
// device staging buffer of the host-memory entry points, grown on demand
int ensure_io(void** buf, size_t* cap, size_t bytes);
int map_status(int st);
// the header of a stream that went through the lossless stage (and its raw
// size); hpez_decompress undoes the stage first
bool lossless_flagged(const uint8_t* hdr, uint64_t* raw);
int cuda_check(cudaError_t e);
void default_config(int ndim, hpez_config* c);

}  // namespace host
}  // namespace hpez
