// k_lossless.cu -- the lossless stage after Huffman (Sec. 4, Step 5), read
// as run suppression of repeated 32-bit words of the stream body, and its
// C-ABI entry points (hpez_lossless_encode / hpez_lossless_decode, declared
// in include/hpez.h).
//
// Format: the 512-byte header (flag bit 2, the raw size at byte 328), four
// u64 counts (words, kept words, kept block masks, 0), one mask per group
// of 32 blocks marking the blocks whose mask is not 0, those block masks,
// and the kept words.  A block mask marks the words of its 32 that differ
// from the word before them (the word before the first is 0).
//
// GPU layout: a warp owns a group of 32 blocks (1024 words) and walks its
// blocks, one coalesced 128-byte row of words per step; a lane keeps the
// mask of the block with its index, so the group mask is one ballot.  Two
// exclusive scans over the groups place the kept masks and words.
#include <cstring>

#include "hpez.h"
#include "hpez_ctx.h"
#include "hpez_internal.cuh"
#include "hpez_launch.h"

using namespace hpez;
using namespace hpez::host;

namespace {

constexpr int kLzHdr = 512, kLzCounts = 32;
constexpr int kLzRawSize = 328;
constexpr unsigned kFlagLossless = 2u;
constexpr int kLzWarps = 8;
constexpr int kScanThreads = 1024;

// body word i (the last one zero-padded)
__device__ __forceinline__ uint32_t lz_word(const uint8_t* __restrict__ body, uint64_t nbytes,
                                            uint64_t i) {
  if (4 * i + 4 <= nbytes) return __ldg(reinterpret_cast<const uint32_t*>(body) + i);
  uint32_t v = 0;
  for (int k = 0; k < 4; ++k) {
    const uint64_t o = 4 * i + (uint64_t)k;
    if (o < nbytes) v |= (uint32_t)body[o] << (8 * k);
  }
  return v;
}

// per group: its group mask (written to the output), the block masks (a
// scratch array), the counts of kept masks and words
__global__ void __launch_bounds__(32 * kLzWarps)
    k_lz_count(const uint8_t* __restrict__ body, uint64_t nbytes, uint64_t nw, uint64_t nb,
               uint64_t ng, uint32_t* __restrict__ m2out, uint32_t* __restrict__ m1,
               uint32_t* __restrict__ cmask, uint32_t* __restrict__ clit) {
  const int lane = threadIdx.x & 31;
  const uint64_t g = (uint64_t)blockIdx.x * kLzWarps + (threadIdx.x >> 5);
  if (g >= ng) return;
  uint32_t mine = 0, lits = 0;
  for (int t = 0; t < 32; ++t) {
    const uint64_t b = 32 * g + (uint64_t)t;
    if (b >= nb) break;  // warp-uniform
    const uint64_t i = 32 * b + (uint64_t)lane;
    const uint32_t w = i < nw ? lz_word(body, nbytes, i) : 0u;
    uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, w, 1);
    if (lane == 0) prev = i == 0 ? 0u : lz_word(body, nbytes, i - 1);
    const uint32_t mask = __ballot_sync(0xFFFFFFFFu, i < nw && w != prev);
    if (lane == t) mine = mask;
    lits += (uint32_t)__popc(mask);
  }
  const uint64_t b = 32 * g + (uint64_t)lane;
  if (b < nb) m1[b] = mine;
  const uint32_t gm = __ballot_sync(0xFFFFFFFFu, b < nb && mine != 0);
  if (lane == 0) {
    m2out[g] = gm;
    cmask[g] = (uint32_t)__popc(gm);
    clit[g] = lits;
  }
}

// exclusive scan of n counts (one CTA), the total in out[n]
__global__ void __launch_bounds__(kScanThreads)
    k_lz_scan(const uint32_t* __restrict__ in, unsigned long long* __restrict__ out, uint64_t n) {
  __shared__ unsigned long long part[kScanThreads];
  const uint64_t per = (n + kScanThreads - 1) / kScanThreads;
  const uint64_t a = (uint64_t)threadIdx.x * per, e = a + per < n ? a + per : n;
  unsigned long long s = 0;
  for (uint64_t i = a; i < e; ++i) s += in[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {  // inclusive scan of the parts
    const unsigned long long v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0ull;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = threadIdx.x ? part[threadIdx.x - 1] : 0ull;
  for (uint64_t i = a; i < e; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (threadIdx.x == kScanThreads - 1) out[n] = part[kScanThreads - 1];
}

// the kept block masks and words of each group at their offsets
__global__ void __launch_bounds__(32 * kLzWarps)
    k_lz_write(const uint8_t* __restrict__ body, uint64_t nbytes, uint64_t nw, uint64_t nb,
               uint64_t ng, const uint32_t* __restrict__ m1, const uint32_t* __restrict__ m2,
               const unsigned long long* __restrict__ moff,
               const unsigned long long* __restrict__ loff, uint32_t* __restrict__ zmask,
               uint32_t* __restrict__ zlit) {
  const int lane = threadIdx.x & 31;
  const uint64_t g = (uint64_t)blockIdx.x * kLzWarps + (threadIdx.x >> 5);
  if (g >= ng) return;
  const uint64_t b0 = 32 * g + (uint64_t)lane;
  const uint32_t mine = b0 < nb ? m1[b0] : 0u;
  const uint32_t gm = m2[g];
  const uint32_t lt = (1u << lane) - 1u;
  if (mine) zmask[moff[g] + (unsigned)__popc(gm & lt)] = mine;
  unsigned long long at = loff[g];
  for (int t = 0; t < 32; ++t) {
    const uint64_t b = 32 * g + (uint64_t)t;
    if (b >= nb) break;
    const uint32_t mask = __shfl_sync(0xFFFFFFFFu, mine, t);
    if (!mask) continue;
    const uint64_t i = 32 * b + (uint64_t)lane;
    if ((mask >> lane) & 1u) zlit[at + (unsigned)__popc(mask & lt)] = lz_word(body, nbytes, i);
    at += (unsigned)__popc(mask);
  }
}

}  // namespace

namespace {

// decode, first pass: kept block masks per group
__global__ void k_lzd_cmask(const uint32_t* __restrict__ m2, uint64_t ng,
                            uint32_t* __restrict__ cmask) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < ng) cmask[g] = (uint32_t)__popc(m2[g]);
}

// decode, second pass: kept words per group; bad: a kept block mask of 0
// (and bits for blocks or words beyond the body)
__global__ void __launch_bounds__(32 * kLzWarps)
    k_lzd_clit(const uint32_t* __restrict__ m2, const uint32_t* __restrict__ zmask,
               const unsigned long long* __restrict__ moff, uint64_t ng, uint64_t nb,
               uint64_t nw, uint32_t* __restrict__ clit, unsigned* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const uint64_t g = (uint64_t)blockIdx.x * kLzWarps + (threadIdx.x >> 5);
  if (g >= ng) return;
  const uint32_t gm = m2[g];
  const int cnt = __popc(gm);
  const uint32_t m = lane < cnt ? zmask[moff[g] + (unsigned)lane] : 1u;
  if (__any_sync(0xFFFFFFFFu, m == 0u) && lane == 0) atomicExch(bad, 1u);
  if (g == ng - 1 && lane == 0) {
    const unsigned p = (unsigned)(nb - 1 - 32 * g);  // the last block's place in the group
    if (p < 31 && (gm >> (p + 1))) atomicExch(bad, 1u);
    const unsigned nlast = (unsigned)(nw - 32 * (nb - 1));  // words of the last block
    if (((gm >> p) & 1u) && nlast < 32) {
      const uint32_t ml = zmask[moff[g] + (unsigned)__popc(gm & ((1u << p) - 1u))];
      if (ml >> nlast) atomicExch(bad, 1u);
    }
  }
  unsigned c = (unsigned)__popc(lane < cnt ? m : 0u);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  if (lane == 0) clit[g] = c;
}

// decode: every word of the group's blocks; a word not kept repeats the
// word before it (the last kept word before the group, or 0)
__global__ void __launch_bounds__(32 * kLzWarps)
    k_lzd_write(const uint32_t* __restrict__ m2, const uint32_t* __restrict__ zmask,
                const uint32_t* __restrict__ zlit, const unsigned long long* __restrict__ moff,
                const unsigned long long* __restrict__ loff, uint64_t nw, uint64_t nb,
                uint64_t ng, uint64_t nbytes, uint8_t* __restrict__ body) {
  const int lane = threadIdx.x & 31;
  const uint64_t g = (uint64_t)blockIdx.x * kLzWarps + (threadIdx.x >> 5);
  if (g >= ng) return;
  const uint32_t gm = m2[g];
  const uint32_t lt = (1u << lane) - 1u, le = (2u << lane) - 1u;
  const uint32_t mine = ((gm >> lane) & 1u) ? zmask[moff[g] + (unsigned)__popc(gm & lt)] : 0u;
  unsigned long long at = loff[g];
  uint32_t carry = at > 0 ? zlit[at - 1] : 0u;
  for (int t = 0; t < 32; ++t) {
    const uint64_t b = 32 * g + (uint64_t)t;
    if (b >= nb) break;
    const uint32_t mask = __shfl_sync(0xFFFFFFFFu, mine, t);
    const unsigned k = (unsigned)__popc(mask & le);
    const uint32_t v = k ? zlit[at + k - 1] : carry;
    const uint64_t i = 32 * b + (uint64_t)lane;
    if (4 * i + 4 <= nbytes) {
      reinterpret_cast<uint32_t*>(body)[i] = v;
    } else if (i < nw) {
      for (int q = 0; q < 4; ++q)
        if (4 * i + (uint64_t)q < nbytes) body[4 * i + (uint64_t)q] = (uint8_t)(v >> (8 * q));
    }
    carry = __shfl_sync(0xFFFFFFFFu, v, 31);
    at += (unsigned)__popc(mask);
  }
}

uint64_t rd64h(const uint8_t* b, int o) {
  uint64_t v;
  std::memcpy(&v, b + o, 8);
  return v;
}
void wr64h(uint8_t* b, int o, uint64_t v) { std::memcpy(b + o, &v, 8); }
uint32_t rd32h(const uint8_t* b, int o) {
  uint32_t v;
  std::memcpy(&v, b + o, 4);
  return v;
}
void wr32h(uint8_t* b, int o, uint32_t v) { std::memcpy(b + o, &v, 4); }

// scratch of one call: ng counts twice, ng + 1 offsets twice, nb block
// masks, ng group masks, a flag
struct LzScratch {
  uint32_t *cmask, *clit, *m1, *m2;
  unsigned long long *moff, *loff;
  unsigned* bad;
};

int lz_scratch(hpez_ctx* ctx, uint64_t nb, uint64_t ng, LzScratch& S) {
  Arena ar;
  const size_t o_cm = ar.take<uint32_t>(ng), o_cl = ar.take<uint32_t>(ng);
  const size_t o_m1 = ar.take<uint32_t>(nb ? nb : 1), o_m2 = ar.take<uint32_t>(ng);
  const size_t o_mo = ar.take<unsigned long long>(ng + 1);
  const size_t o_lo = ar.take<unsigned long long>(ng + 1);
  const size_t o_bad = ar.take<unsigned>(1);
  const int rc = ensure_io(&ctx->lz_buf, &ctx->lz_cap, ar.off);
  if (rc) return rc;
  char* p = static_cast<char*>(ctx->lz_buf);
  S.cmask = reinterpret_cast<uint32_t*>(p + o_cm);
  S.clit = reinterpret_cast<uint32_t*>(p + o_cl);
  S.m1 = reinterpret_cast<uint32_t*>(p + o_m1);
  S.m2 = reinterpret_cast<uint32_t*>(p + o_m2);
  S.moff = reinterpret_cast<unsigned long long*>(p + o_mo);
  S.loff = reinterpret_cast<unsigned long long*>(p + o_lo);
  S.bad = reinterpret_cast<unsigned*>(p + o_bad);
  return HPEZ_OK;
}

unsigned lz_grid(uint64_t ng) { return (unsigned)((ng + kLzWarps - 1) / kLzWarps); }

}  // namespace

int hpez_lossless_encode(hpez_ctx* ctx, const void* d_in, uint64_t in_size, void* d_out,
                         uint64_t out_cap, uint64_t* h_out_size, void* stream) {
  if (!ctx || !d_in || !d_out || !h_out_size || in_size < (uint64_t)kLzHdr)
    return HPEZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_in) & 15u) || (reinterpret_cast<uintptr_t>(d_out) & 15u))
    return HPEZ_ERR_INVALID_ARG;
  const uint8_t* in = static_cast<const uint8_t*>(d_in);
  uint8_t* out = static_cast<uint8_t*>(d_out);
  if (out < in + in_size && in < out + out_cap) return HPEZ_ERR_INVALID_ARG;  // no overlap
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t hdr[kLzHdr + kLzCounts];
  int rc = cuda_check(cudaMemcpyAsync(hdr, in, kLzHdr, cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc) return rc;
  if (rd32h(hdr, H_FLAGS) & kFlagLossless) return HPEZ_ERR_INVALID_ARG;
  const uint64_t nbytes = in_size - kLzHdr, nw = (nbytes + 3) / 4, nb = (nw + 31) / 32,
                 ng = (nb + 31) / 32;
  uint64_t zsize = in_size;
  if (ng > 0) {
    LzScratch S;
    if ((rc = lz_scratch(ctx, nb, ng, S))) return rc;
    const uint8_t* body = in + kLzHdr;
    k_lz_count<<<lz_grid(ng), 32 * kLzWarps, 0, s>>>(body, nbytes, nw, nb, ng, S.m2, S.m1,
                                                     S.cmask, S.clit);
    k_lz_scan<<<1, kScanThreads, 0, s>>>(S.cmask, S.moff, ng);
    k_lz_scan<<<1, kScanThreads, 0, s>>>(S.clit, S.loff, ng);
    ctx->launches += 3;
    unsigned long long tot[2];
    rc = cuda_check(cudaMemcpyAsync(&tot[0], S.moff + ng, 8, cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_check(cudaMemcpyAsync(&tot[1], S.loff + ng, 8, cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
    if (rc) return rc;
    const uint64_t nmask = tot[0], nlit = tot[1];
    zsize = kLzHdr + kLzCounts + 4 * (ng + nmask + nlit);
    if (zsize < in_size) {
      if (zsize > out_cap) return HPEZ_ERR_OUT_TOO_SMALL;
      wr32h(hdr, H_FLAGS, rd32h(hdr, H_FLAGS) | kFlagLossless);
      wr64h(hdr, kLzRawSize, in_size);
      wr64h(hdr, kLzHdr, nw);
      wr64h(hdr, kLzHdr + 8, nlit);
      wr64h(hdr, kLzHdr + 16, nmask);
      wr64h(hdr, kLzHdr + 24, 0);
      uint32_t* zm2 = reinterpret_cast<uint32_t*>(out + kLzHdr + kLzCounts);
      rc = cuda_check(cudaMemcpyAsync(out, hdr, kLzHdr + kLzCounts, cudaMemcpyHostToDevice, s));
      if (!rc) rc = cuda_check(cudaMemcpyAsync(zm2, S.m2, 4 * ng, cudaMemcpyDeviceToDevice, s));
      if (rc) return rc;
      k_lz_write<<<lz_grid(ng), 32 * kLzWarps, 0, s>>>(body, nbytes, nw, nb, ng, S.m1, S.m2,
                                                       S.moff, S.loff, zm2 + ng,
                                                       zm2 + ng + nmask);
      ++ctx->launches;
      rc = cuda_check(cudaGetLastError());
      if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
      if (rc) return rc;
      *h_out_size = zsize;
      return HPEZ_OK;
    }
  }
  // no gain: the stream as it is
  if (in_size > out_cap) return HPEZ_ERR_OUT_TOO_SMALL;
  rc = cuda_check(cudaMemcpyAsync(out, in, in_size, cudaMemcpyDeviceToDevice, s));
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc) return rc;
  *h_out_size = in_size;
  return HPEZ_OK;
}

int hpez_lossless_decode(hpez_ctx* ctx, const void* d_in, uint64_t in_size, void* d_out,
                         uint64_t out_cap, uint64_t* h_out_size, void* stream) {
  if (!ctx || !d_in || !d_out || !h_out_size) return HPEZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_in) & 15u) || (reinterpret_cast<uintptr_t>(d_out) & 15u))
    return HPEZ_ERR_INVALID_ARG;
  if (in_size < (uint64_t)(kLzHdr + kLzCounts)) return HPEZ_ERR_CORRUPT_STREAM;
  const uint8_t* in = static_cast<const uint8_t*>(d_in);
  uint8_t* out = static_cast<uint8_t*>(d_out);
  if (out < in + in_size && in < out + out_cap) return HPEZ_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t hdr[kLzHdr + kLzCounts];
  int rc = cuda_check(cudaMemcpyAsync(hdr, in, kLzHdr + kLzCounts, cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc) return rc;
  if (!(rd32h(hdr, H_FLAGS) & kFlagLossless)) return HPEZ_ERR_INVALID_ARG;
  const uint64_t raw = rd64h(hdr, kLzRawSize);
  if (raw < (uint64_t)kLzHdr) return HPEZ_ERR_CORRUPT_STREAM;
  if (raw > out_cap) return HPEZ_ERR_OUT_TOO_SMALL;
  const uint64_t nbytes = raw - kLzHdr, nw = rd64h(hdr, kLzHdr), nlit = rd64h(hdr, kLzHdr + 8),
                 nmask = rd64h(hdr, kLzHdr + 16);
  if (nw != (nbytes + 3) / 4 || rd64h(hdr, kLzHdr + 24) != 0) return HPEZ_ERR_CORRUPT_STREAM;
  const uint64_t nb = (nw + 31) / 32, ng = (nb + 31) / 32;
  if (nmask > nb || nlit > nw || in_size != kLzHdr + kLzCounts + 4 * (ng + nmask + nlit))
    return HPEZ_ERR_CORRUPT_STREAM;
  // the header as it was before the stage
  wr32h(hdr, H_FLAGS, rd32h(hdr, H_FLAGS) & ~kFlagLossless);
  wr64h(hdr, kLzRawSize, 0);
  rc = cuda_check(cudaMemcpyAsync(out, hdr, kLzHdr, cudaMemcpyHostToDevice, s));
  if (rc) return rc;
  if (ng > 0) {
    LzScratch S;
    if ((rc = lz_scratch(ctx, nb, ng, S))) return rc;
    const uint32_t* zm2 = reinterpret_cast<const uint32_t*>(in + kLzHdr + kLzCounts);
    const uint32_t* zmask = zm2 + ng;
    const uint32_t* zlit = zmask + nmask;
    cudaMemsetAsync(S.bad, 0, sizeof(unsigned), s);
    k_lzd_cmask<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(zm2, ng, S.cmask);
    k_lz_scan<<<1, kScanThreads, 0, s>>>(S.cmask, S.moff, ng);
    ctx->launches += 2;
    unsigned long long tm = 0;
    rc = cuda_check(cudaMemcpyAsync(&tm, S.moff + ng, 8, cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
    if (rc) return rc;
    if (tm != nmask) return HPEZ_ERR_CORRUPT_STREAM;
    k_lzd_clit<<<lz_grid(ng), 32 * kLzWarps, 0, s>>>(zm2, zmask, S.moff, ng, nb, nw, S.clit,
                                                     S.bad);
    k_lz_scan<<<1, kScanThreads, 0, s>>>(S.clit, S.loff, ng);
    ctx->launches += 2;
    unsigned long long tl = 0;
    unsigned bad = 0;
    rc = cuda_check(cudaMemcpyAsync(&tl, S.loff + ng, 8, cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_check(cudaMemcpyAsync(&bad, S.bad, 4, cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
    if (rc) return rc;
    if (tl != nlit || bad) return HPEZ_ERR_CORRUPT_STREAM;
    k_lzd_write<<<lz_grid(ng), 32 * kLzWarps, 0, s>>>(zm2, zmask, zlit, S.moff, S.loff, nw, nb,
                                                      ng, nbytes, out + kLzHdr);
    ++ctx->launches;
    rc = cuda_check(cudaGetLastError());
  }
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc) return rc;
  *h_out_size = raw;
  return HPEZ_OK;
}

namespace hpez {
namespace host {

bool lossless_flagged(const uint8_t* hdr, uint64_t* raw) {
  if (!(rd32h(hdr, H_FLAGS) & kFlagLossless)) return false;
  *raw = rd64h(hdr, kLzRawSize);
  return true;
}

}  // namespace host
}  // namespace hpez
