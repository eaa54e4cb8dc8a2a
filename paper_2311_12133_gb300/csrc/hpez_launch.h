// hpez_launch.h -- host-side launchers of the HPEZ kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hpez_internal.cuh"

namespace hpez {

// Grid of a persistent batched launch: the CTAs of `kernel` resident on
// num_sms SMs at once (at most max_ctas when > 0), never more than the
// launch's nblk virtual blocks.
template <class K>
unsigned persistent_grid(K kernel, int threads, size_t smem, uint32_t nblk, int num_sms,
                         int max_ctas) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  if (per_sm < 1) per_sm = 1;
  uint64_t g = (uint64_t)per_sm * (uint64_t)(num_sms > 0 ? num_sms : 1);
  if (max_ctas > 0 && (uint64_t)max_ctas < g) g = (uint64_t)max_ctas;
  if (g > nblk) g = nblk;
  return (unsigned)(g ? g : 1);
}

// k_sweep.cu
void launch_init_ctl(Ctl* ctl, cudaStream_t s);
void launch_fill(float* out, uint32_t N, float v, int num_sms,
                 cudaStream_t s);
void launch_range(const float* x, uint32_t N, Ctl* ctl, int num_sms,
                  cudaStream_t s);
void launch_set_range(Ctl* ctl, unsigned kmin, unsigned kmax, cudaStream_t s);
void launch_params(Ctl* ctl, int eb_mode, double eb, double alpha,
                   double beta, int L, const float* x, cudaStream_t s);
void launch_anchor_gather(const float* x, const LevelGeom& ga, uint32_t total,
                          float* RA, uint16_t* CA, const Ctl* ctl,
                          cudaStream_t s);
void launch_upsample(const LevelGeom& gc, uint32_t total_c,
                     const LevelGeom& gs, const float* Rc, const uint16_t* Cc,
                     float* Rs, uint16_t* Cs, const Ctl* ctl, cudaStream_t s);
void launch_pass(bool decomp, const LevelGeom& g, const PassBox& pb,
                 const SweepBufs& B, int num_sms, cudaStream_t s);

// k_level.cu
size_t fused_smem_bytes(const FusedLevel& P, bool decomp);
void launch_level(bool decomp, const FusedLevel& P, const SweepBufs& B,
                  const float* Rc, const uint16_t* Cc, float* Rs, uint16_t* Cs,
                  cudaStream_t s);

// k_level3d.cu
size_t level3d_smem_bytes(const Level3D& P, bool decomp);
void launch_level3d(bool decomp, const Level3D& P, const SweepBufs& B,
                    const float* Rc, const uint16_t* Cc, float* Rs, uint16_t* Cs,
                    cudaStream_t s);

// k_level_md.cu
void launch_level_md(bool decomp, int kind, const LevelMD& P, const SweepBufs& B,
                     const float* Rc, const uint16_t* Cc, float* Rs, uint16_t* Cs,
                     int num_sms, cudaStream_t s);

// k_level_md3.cu
size_t md3_smem_bytes(const LevelMD& P, int E1);
void launch_level_md3(bool decomp, int kind, const LevelMD& P, int E1,
                      const SweepBufs& B, const float* Rc, const uint16_t* Cc,
                      float* Rs, uint16_t* Cs, cudaStream_t s);
bool md3s_supported(const LevelMD& P, bool decomp, const void* in, const float* Rc,
                    const uint16_t* Cc);
int launch_level_md3s(bool decomp, int kind, const LevelMD& P, const SweepBufs& B,
                      const float* Rc, const uint16_t* Cc, float* Rs, uint16_t* Cs,
                      Ctl* ctl, int num_sms, int drop_copy, int chunks, cudaStream_t s);

// k_level_md3w.cu
bool md3w_supported(const LevelMD& P, bool decomp, const void* in, const float* Rc,
                    const uint16_t* Cc, const float* Rs, const uint16_t* Cs);
int launch_level_md3w(bool decomp, int kind, const LevelMD& P, const SweepBufs& B,
                      const float* Rc, const uint16_t* Cc, float* Rs, uint16_t* Cs,
                      const Ctl* ctl, int num_sms, int chunks, cudaStream_t s);

// k_spline.cu
void launch_spline_pass(bool decomp, const LevelGeom& g, const PassBox& pb, const SweepBufs& B,
                        float* dscr, int num_sms, cudaStream_t s);

// k_lorenzo.cu
bool lorenzo_supported(const uint32_t n[3], const uint32_t fst[3], int off, int A);
int launch_lorenzo(bool decomp, int order, const uint32_t n[3], const uint32_t fst[3],
                   int off, int A, bool vec, const float* x, uint16_t* codes, float* out,
                   const Ctl* ctl, int num_sms, int drop_copy, int max_ctas,
                   cudaStream_t s);

// batched Lorenzo pass: the job's geometry (G.g for its CTA count), op
// variant, CTA count and shared memory; false for geometries the kernel does
// not take
constexpr int kLorVariants = 2 * 2 * 3 * 2 * 2 * 6;
bool lorenzo_batch_job(bool decomp, int order, const uint32_t n[3], const uint32_t fst[3],
                       int off, int A, bool vec, int num_sms, int max_ctas, LorGeom* G,
                       int* variant, uint32_t* ctas, size_t* smem);
void launch_lorenzo_batch(int variant, const LorenzoJob* J, const uint32_t* off, int nj,
                          uint32_t nblk, size_t smem, cudaStream_t s);
// k_huffman.cu
void launch_hist(const uint16_t* codes, uint32_t N, uint32_t C, uint32_t nch,
                 uint32_t* hist, uint32_t* zc, const Ctl* ctl, int num_sms,
                 cudaStream_t s);
void launch_codebook(const uint32_t* hist, unsigned long long* enc,
                     uint16_t* tsyms, uint8_t* tlens, unsigned long long* gkeys,
                     unsigned long long* giw, uint32_t* gpar,
                     uint8_t* lens_by_sym, Ctl* ctl, cudaStream_t s);
void launch_enc_len(const uint16_t* codes, uint32_t N, uint32_t C,
                    uint32_t nch, const unsigned long long* enc,
                    uint16_t* lanebits, uint32_t* chw, const Ctl* ctl,
                    int num_sms, cudaStream_t s);
void launch_pack(const uint16_t* codes, uint32_t N, uint32_t C, uint32_t nch,
                 const unsigned long long* enc, const uint16_t* lanebits,
                 const uint32_t* chw, const unsigned long long* woff,
                 uint8_t* out, const Ctl* ctl, int num_sms, cudaStream_t s);
void launch_chunk_words(const uint8_t* lanebits_bytes, uint32_t nch,
                        uint32_t* chw, int num_sms, cudaStream_t s);
// lane bit counts, chunk offsets (decoupled look-back) and packing in one
// kernel; flags: nch + 1 words of scratch; the stream layout's offsets
// must be set, its capacity check happens here
void launch_encode(const uint16_t* codes, uint32_t N, uint32_t C, uint32_t nch,
                   const unsigned long long* enc, uint16_t* lanebits,
                   unsigned long long* flags, uint8_t* out, Ctl* ctl,
                   unsigned long long cap, int num_sms, cudaStream_t s);
void launch_outliers(bool gather, const uint16_t* codes, uint32_t N,
                     uint32_t C, uint32_t nch, const uint32_t* zc,
                     const unsigned long long* zoff, const float* src,
                     float* dst, uint8_t* stream, unsigned long long max_out,
                     Ctl* ctl, int num_sms, cudaStream_t s);
void launch_dec_tables(const uint8_t* stream, uint32_t n_used,
                       uint64_t off_table, uint32_t* lut, uint32_t* cnt,
                       unsigned long long* first, uint32_t* offs,
                       uint16_t* sorted, unsigned long long* gkeys, Ctl* ctl,
                       cudaStream_t s);
void launch_decode(const uint8_t* stream, uint64_t off_bits,
                   uint64_t total_words, const uint8_t* lanebits_bytes,
                   const unsigned long long* woff, uint32_t N, uint32_t C,
                   uint32_t nch, uint32_t n_used, uint16_t single_sym,
                   const uint32_t* lut, const uint32_t* cnt,
                   const unsigned long long* first, const uint32_t* offs,
                   const uint16_t* sorted, uint16_t* codes, uint32_t* zc,
                   Ctl* ctl, int num_sms, cudaStream_t s,
                   const uint8_t* single_src = nullptr);

// k_stream.cu
void launch_scan(const uint32_t* in, unsigned long long* out, uint32_t n,
                 unsigned long long* total, const Ctl* ctl, cudaStream_t s);
void launch_layout(Ctl* ctl, unsigned long long off_table,
                   unsigned long long cap, cudaStream_t s);
void launch_finalize(const uint8_t* hdr, const uint8_t* hdr_const,
                     uint8_t* out, const float* RA, uint32_t na,
                     unsigned long long off_anchors, const uint8_t* bmap,
                     uint32_t nblocks, unsigned long long off_bmap,
                     const uint16_t* lanebits, uint32_t nch,
                     unsigned long long off_chw, const uint16_t* tsyms,
                     const uint8_t* tlens, const Ctl* ctl, int num_sms,
                     cudaStream_t s);

// batched forms (one launch for many fields; job j owns the launch's blocks
// [off[j], off[j+1]); single-CTA stages run one block per job)
void launch_init_ctl_batch(const InitJob* J, int nj, cudaStream_t s);
void launch_range_batch(const RangeJob* J, const uint32_t* off, int nj,
                        uint32_t nblk, cudaStream_t s);
void launch_params_batch(const ParamsJob* J, int nj, cudaStream_t s);
void launch_anchor_batch(const AnchorJob* J, const uint32_t* off, int nj,
                         uint32_t nblk, cudaStream_t s);
void launch_fill_batch(const FillJob* J, const uint32_t* off, int nj,
                       uint32_t nblk, cudaStream_t s);
// persistent level launches (at most max_ctas CTAs when > 0)
void launch_level3d_batch(bool decomp, int kind, const Level3DJob* J,
                          const uint32_t* off, int nj, uint32_t nblk,
                          size_t smem, int num_sms, int max_ctas, cudaStream_t s);
void launch_level_batch(bool decomp, int kind, const LevelJob* J,
                        const uint32_t* off, int nj, uint32_t nblk, size_t smem,
                        int num_sms, int max_ctas, cudaStream_t s);
void launch_md3_batch(bool decomp, bool odd, int kind, const MD3Job* J, const uint32_t* off,
                      int nj, uint32_t nblk, size_t smem, int num_sms, int max_ctas,
                      cudaStream_t s);
void md3w_geometry(bool decomp, int kind, const LevelMD& P, int num_sms, int chunks, int* n1,
                   int* n2, int* K, uint32_t* ctas);
void launch_md3w_batch(bool decomp, int kind, const MD3WJob* J, const uint32_t* off, int nj,
                       uint32_t nblk, int num_sms, int max_ctas, cudaStream_t s);
int level_kind(const SweepBufs& B);
uint32_t hist_blocks(uint32_t nch, int num_sms);
uint32_t enc_blocks(uint32_t nch, int num_sms);
uint32_t decode_blocks(uint32_t nch, int num_sms);
uint32_t chunk_words_blocks(uint32_t nch, int num_sms);
uint32_t finalize_blocks(uint32_t na, uint32_t nch, int num_sms);
void launch_hist_batch(const HistJob* J, const uint32_t* off, int nj,
                       uint32_t nblk, cudaStream_t s);
void launch_codebook_batch(const CodebookJob* J, int nj, cudaStream_t s);
void launch_hcost_batch(const CodebookJob* J, int nj, unsigned long long* cost,
                        cudaStream_t s);
void launch_enc_len_batch(const EncLenJob* J, const uint32_t* off, int nj,
                          uint32_t nblk, cudaStream_t s);
void launch_pack_batch(const PackJob* J, const uint32_t* off, int nj,
                       uint32_t nblk, cudaStream_t s);
void launch_chunk_words_batch(const ChunkWordsJob* J, const uint32_t* off,
                              int nj, uint32_t nblk, cudaStream_t s);
void launch_outliers_batch(const OutlierJob* J, const uint32_t* off, int nj,
                           uint32_t nblk, cudaStream_t s);
void launch_dec_tables_batch(const DecTablesJob* J, int nj, cudaStream_t s);
void launch_decode_batch(const DecodeJob* J, const uint32_t* off, int nj,
                         uint32_t nblk, cudaStream_t s);
void launch_scan_batch(const ScanJob* J, int nj, cudaStream_t s);
void launch_layout_batch(const LayoutJob* J, int nj, cudaStream_t s);
void launch_finalize_batch(const FinalizeJob* J, const uint32_t* off, int nj,
                           uint32_t nblk, cudaStream_t s);
void launch_result_batch(const ResultJob* J, int nj, cudaStream_t s);
// one request's outcome (the job by value)
void launch_result_one(const ResultJob& J, cudaStream_t s);
void launch_upsample_batch(const UpsampleJob* J, const uint32_t* off, int nj,
                           uint32_t nblk, cudaStream_t s);
void launch_pass_batch(bool decomp, const PassJob* J, const uint32_t* off,
                       int nj, uint32_t nblk, cudaStream_t s);
void launch_zero_batch(const ZeroJob* J, const uint32_t* off, int nj,
                       uint32_t nblk, cudaStream_t s);
uint32_t grid_blocks(uint64_t n, unsigned cap);
uint32_t pass_blocks(uint32_t total, int num_sms);

// k_tune.cu
void launch_tune_stats(const float* x, const uint32_t n[3],
                       const uint32_t fst[3], const int real[3], int t,
                       const Ctl* ctl, unsigned long long* acc, int num_sms,
                       cudaStream_t s);
void launch_tune_params(TuneCfg* cfgs, int nvar, int L, const Ctl* ctl,
                        cudaStream_t s);
// cfgs[t] (t < n0 + n1) = base[variant of t] with level l's fields from
// cands[t] (variant 0: t < n0)
void launch_tune_expand(const TuneCfg* base, const TuneCand* cands, int n0, int n1, int l,
                        TuneCfg* cfgs, cudaStream_t s);
// per variant (nv <= 2): the first candidate with the smallest score; its
// fields go into base[v] at level l, its index and score to
// choice/best[v * 16 + l - 1]
void launch_tune_select(const unsigned long long* score, const TuneCand* cands, int n0,
                        int n1, int nv, int l, TuneCfg* base, uint8_t* choice,
                        unsigned long long* best, cudaStream_t s);
size_t tune_test_smem(const TuneGeom& g);
size_t tune_lorenzo_smem(const TuneGeom& g);
// (sample block, variant) CTAs; variants < ny0 use geometry g0, the rest g1.
// state: each block's reconstruction after the levels above l_stop (run
// level l_stop only), or null (run levels L..l_stop from the anchors)
void launch_tune_test(const float* x, const TuneGeom& g0, const TuneGeom& g1,
                      int ny0, const TuneCfg* cfgs, int nvar, int nblk,
                      int l_stop, bool hist, unsigned long long* score,
                      uint32_t* hists, unsigned long long* nout, float* state,
                      cudaStream_t s);
// runs level l with the chosen config of each of nv variants and keeps the
// result in state
void launch_tune_advance(const float* x, const TuneGeom& g0, const TuneGeom& g1,
                         int nv, int nblk, const TuneCfg* cfgs, int l, float* state,
                         cudaStream_t s);
void launch_tune_lorenzo(const float* x, const TuneGeom& g, int nblk,
                         const Ctl* ctl, uint32_t* hists,
                         unsigned long long* nout, cudaStream_t s);
int launch_tune_blockwise(const float* x, const TuneGeom& g, int bs, int Q,
                           int frozen_slot, const uint32_t nb[3],
                           uint32_t nblocks, const TuneCfg* base,
                           unsigned allow, unsigned long long* scores,
                           uint8_t* bmap, cudaStream_t s, cudaStream_t s2,
                           cudaEvent_t fork, cudaEvent_t join);

}  // namespace hpez
