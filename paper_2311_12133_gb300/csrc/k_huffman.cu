// k_huffman.cu -- code histogram, canonical Huffman codebook, chunked
// encode and decode of the quantization codes (Sec. 4 Step 4).
//
// Stream convention (shared with the decoder): the row-major code array is
// cut into chunks of C symbols; a chunk is coded as 32 lanes, lane l holding
// the chunk's symbols l, l+32, l+64, ...; the lanes' bits follow one another
// MSB-first in 32-bit words, each chunk starting on a fresh word, and every
// lane's bit count is stored (u16), so one warp encodes or decodes a chunk
// with coalesced symbol access and no atomics inside a lane's words.  Codebook: two-queue Huffman merge
// over leaves sorted by (frequency, symbol), ties taking the leaf; lengths
// are leaf depths; canonical codes ordered by (length, symbol).
#include "hpez_internal.cuh"
#include "hpez_launch.h"

namespace hpez {

constexpr int kHistWin = 2048;              // bins per warp-private window
constexpr int kHistLo = kRadius - kHistWin / 2;
constexpr int kHistWarps = 8;
// the codes of the first chunks (this many bytes) are read with the normal
// cache policy and the rest as streaming loads, so that the start of the
// code array is still in L2 when the encoder (which takes the chunks in
// order) reads it
constexpr uint64_t kHistKeepBytes = 64ull << 20;

// ---------------------------------------------------------------------
// histogram of the 65536 code symbols + per-chunk count of code 0.  Each
// warp owns a private window of bins in shared memory (contention only
// between lanes of one warp) and counts the zero-error code in a register;
// a code outside the window (rare: large errors and outliers, code 0
// among them) goes to a global atomic on a path taken only when one of a
// lane's 8 codes needs it, so the common code costs a window test and one
// shared atomic.
// ---------------------------------------------------------------------
__device__ __forceinline__ void hist_body(const uint16_t* __restrict__ codes,
                                          uint32_t N, uint32_t C, uint32_t nch,
                                          uint32_t* __restrict__ hist,
                                          uint32_t* __restrict__ zc,
                                          const Ctl* __restrict__ ctl,
                                          unsigned bid, unsigned nblk) {
  if (ctl->status || ctl->is_const) return;
  extern __shared__ uint32_t shw[];  // [kHistWarps][kHistWin]
  for (int i = threadIdx.x; i < kHistWarps * kHistWin; i += blockDim.x) shw[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  uint32_t* sh = shw + (threadIdx.x >> 5) * kHistWin;
  const uint32_t warp = (bid * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (nblk * blockDim.x) >> 5;
  uint32_t c0 = 0;  // the zero-error code
  // one code into the window or the centre register; false: outside
  auto add_win = [&](unsigned v) -> bool {
    const unsigned o = v - (unsigned)kHistLo;
    c0 += (v == (unsigned)kRadius);
    if (o < (unsigned)kHistWin) {
      if (v != (unsigned)kRadius) atomicAdd(&sh[o], 1u);
      return true;
    }
    return false;
  };
  auto add_far = [&](unsigned v, uint32_t& zeros) {
    if (v - (unsigned)kHistLo >= (unsigned)kHistWin) {
      atomicAdd(&hist[v], 1u);
      zeros += (v == 0u);
    }
  };
  for (uint32_t c = warp; c < nch; c += nwarps) {
    const uint32_t beg = c * C;
    const uint32_t end = min(beg + C, N);
    uint32_t zeros = 0;
    if (end - beg == C && (C & 7u) == 0u) {
      const uint4* p = reinterpret_cast<const uint4*>(codes + beg);
      const uint32_t nq = C / 8;
      const bool keep = (uint64_t)beg * sizeof(uint16_t) < kHistKeepBytes;
      for (uint32_t i = lane; i < nq; i += 128) {
        uint4 v[4];
#pragma unroll
        for (int h = 0; h < 4; ++h)
          if (i + 32u * h < nq) v[h] = keep ? __ldg(p + i + 32u * h) : __ldcs(p + i + 32u * h);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          if (i + 32u * h >= nq) break;
          const unsigned w[4] = {v[h].x, v[h].y, v[h].z, v[h].w};
          bool in = true;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            in &= add_win(w[k] & 0xFFFFu);
            in &= add_win(w[k] >> 16);
          }
          if (!in) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              add_far(w[k] & 0xFFFFu, zeros);
              add_far(w[k] >> 16, zeros);
            }
          }
        }
      }
    } else {
      for (uint32_t i = beg + lane; i < end; i += 32) {
        const unsigned v = codes[i];
        if (!add_win(v)) add_far(v, zeros);
      }
    }
    for (int o = 16; o > 0; o >>= 1) zeros += __shfl_xor_sync(0xffffffffu, zeros, o);
    if (lane == 0) zc[c] = zeros;
  }
  for (int o = 16; o > 0; o >>= 1) c0 += __shfl_xor_sync(0xffffffffu, c0, o);
  __syncwarp();
  if (lane == 0) sh[kRadius - kHistLo] += c0;
  __syncthreads();
  for (int i = threadIdx.x; i < kHistWin; i += blockDim.x) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < kHistWarps; ++w) t += shw[w * kHistWin + i];
    if (t) atomicAdd(&hist[kHistLo + i], t);
  }
}

__global__ void __launch_bounds__(256)
    k_hist(const uint16_t* __restrict__ codes, uint32_t N, uint32_t C,
           uint32_t nch, uint32_t* __restrict__ hist, uint32_t* __restrict__ zc,
           const Ctl* __restrict__ ctl) {
  hist_body(codes, N, C, nch, hist, zc, ctl, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------
// single-CTA helpers
// ---------------------------------------------------------------------
// exclusive scan of one value per thread over the block (blockDim <= 1024)
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    uint32_t s = lane < nw ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) warp_sums[lane] = s;
  }
  __syncthreads();
  const uint32_t before = (w ? warp_sums[w - 1] : 0) + x - v;
  if (total) *total = warp_sums[((blockDim.x + 31) >> 5) - 1];
  __syncthreads();
  return before;
}

// ascending bitonic sort of P (power of two) u64 keys, whole block
__device__ void bitonic_sort(unsigned long long* a, uint32_t P) {
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long x = a[i], y = a[ixj];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

__host__ __device__ inline uint32_t next_pow2(uint32_t v) {
  uint32_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

constexpr uint32_t kSmemLeaves = 8192;  // codebook fits shared memory
constexpr uint32_t kRankSort = 2048;    // alphabets sorted by rank counting
constexpr size_t kCodebookSmem =
    (size_t)kSmemLeaves * 8 + (size_t)kSmemLeaves * 8 + (size_t)kSmemLeaves * 8;

// ---------------------------------------------------------------------
// The two-queue Huffman merge, run by one warp.  keys[0..n) are the leaves
// sorted by (frequency, symbol) as (frequency << 16) | symbol; iw receives
// the internal weights in creation order, par (if not null) every node's
// parent (leaves 0..n-1 in sorted order, internal nodes n, n+1, ...).
// Returns the sum of the internal weights, the code's total bits.
//
// The sequential merge picks the two lightest waiting nodes n - 1 times, a
// leaf before an internal node of the same weight and internal nodes in
// creation order; the internal weights never decrease.  A round here reads
// the first 32 waiting leaves and the first 32 waiting internal nodes and
// ranks them in that pick order (a leaf's rank counts the lighter internal
// nodes, an internal node's the leaves no heavier than it).  Every new node
// of the round weighs at least w0, the sum of its first two picks, and
// comes after every waiting node of weight <= w0; so the ranked picks up to
// the last one of weight <= w0 are exactly the sequential ones, and the
// round commits them in pairs.  A run of equal small frequencies goes 16
// pairs per round.
// ---------------------------------------------------------------------
__device__ unsigned long long warp_huffman_merge(const unsigned long long* keys,
                                                 uint32_t n, unsigned long long* iw,
                                                 uint32_t* par) {
  __shared__ unsigned long long pv[32];
  __shared__ uint32_t pid[32];
  constexpr unsigned kFull = 0xffffffffu;
  constexpr unsigned long long kInf = ~0ull;
  const uint32_t lane = threadIdx.x & 31;
  uint32_t a = 0, b = 0, m = 0;  // leaf head, internal head, internal count
  unsigned long long cost = 0;
  while ((n - a) + (m - b) >= 2) {
    const unsigned long long lv = a + lane < n ? (keys[a + lane] >> 16) : kInf;
    const unsigned long long iv = b + lane < m ? iw[b + lane] : kInf;
    // cl = internal nodes lighter than lv, ci = leaves not heavier than iv
    // (both lists ascend across the lanes)
    uint32_t cl = 0, ci = 0;
#pragma unroll
    for (uint32_t st = 16; st >= 1; st >>= 1) {
      const unsigned long long pi = __shfl_sync(kFull, iv, (int)(cl + st - 1));
      const unsigned long long pl = __shfl_sync(kFull, lv, (int)(ci + st - 1));
      if (pi < lv) cl += st;
      if (pl <= iv) ci += st;
    }
    if (__shfl_sync(kFull, iv, (int)cl) < lv) ++cl;
    if (__shfl_sync(kFull, lv, (int)ci) <= iv) ++ci;
    const uint32_t rl = lane + cl, ri = lane + ci;
    const unsigned long long l0 = __shfl_sync(kFull, lv, 0), l1 = __shfl_sync(kFull, lv, 1);
    const unsigned long long i0 = __shfl_sync(kFull, iv, 0), i1 = __shfl_sync(kFull, iv, 1);
    unsigned long long s0, s1;
    if (l0 <= i0) {
      s0 = l0;
      s1 = l1 <= i0 ? l1 : i0;
    } else {
      s0 = i0;
      s1 = l0 <= i1 ? l0 : i1;
    }
    const unsigned long long w0 = s0 + s1;
    const uint32_t q = min(32u, (uint32_t)(__popc(__ballot_sync(kFull, lv <= w0)) +
                                           __popc(__ballot_sync(kFull, iv <= w0))));
    const uint32_t take = q & ~1u;
    const bool ul = lv <= w0 && rl < take, ui = iv <= w0 && ri < take;
    if (ul) {
      pv[rl] = lv;
      pid[rl] = a + lane;
    }
    if (ui) {
      pv[ri] = iv;
      pid[ri] = n + b + lane;
    }
    __syncwarp();
    const uint32_t c = take >> 1;
    if (lane < c) {
      const unsigned long long w = pv[2 * lane] + pv[2 * lane + 1];
      iw[m + lane] = w;
      cost += w;
      if (par) {
        par[pid[2 * lane]] = n + m + lane;
        par[pid[2 * lane + 1]] = n + m + lane;
      }
    }
    a += __popc(__ballot_sync(kFull, ul));
    b += __popc(__ballot_sync(kFull, ui));
    m += c;
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) cost += __shfl_xor_sync(kFull, cost, o);
  return cost;
}

// ---------------------------------------------------------------------
// codebook: one CTA of 1024 threads
//   hist[65536] -> enc[sym] = (len << 56) | code, table (syms asc, lens),
//   ctl->n_used, ctl->max_len
// scratch (global): gkeys u64[65536], giw u64[65536], gpar u32[131072],
//                   lens_by_sym u8[65536]
// kCostOnly: only the code's total bits (sum of frequency x length, the
// same for every optimal code) to *cost; enc, tables and lengths untouched.
// ---------------------------------------------------------------------
template <bool kCostOnly>
__device__ __forceinline__ void codebook_body(
    const uint32_t* __restrict__ hist, unsigned long long* enc, uint16_t* tsyms,
    uint8_t* tlens, unsigned long long* gkeys, unsigned long long* giw,
    uint32_t* gpar, uint8_t* lens_by_sym, Ctl* ctl,
    unsigned long long* cost = nullptr) {
  if (ctl->status || ctl->is_const) return;
  extern __shared__ unsigned long long smem[];
  __shared__ uint32_t s_n;
  __shared__ uint32_t bl_count[64];
  __shared__ unsigned long long first_code[64];
  __shared__ uint32_t start_pos[64];
  __shared__ uint32_t s_maxlen;

  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  // 1. compaction of used symbols, ascending: warp w owns bins
  //    [2048 w, 2048 (w+1)), read 32 at a time (coalesced); the ballot masks
  //    give every used bin its position
  __shared__ uint32_t masks[32][64];
  __shared__ uint32_t wtot[32];
  const uint32_t* hw = hist + wid * 2048 + lane;
  {
    // 16 loads in flight per thread, then their ballots
    uint32_t c = 0;
#pragma unroll
    for (int g = 0; g < 64; g += 16) {
      uint32_t f[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) f[u] = hw[(g + u) * 32];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const uint32_t m = __ballot_sync(0xffffffffu, f[u] != 0);
        if (lane == 0) masks[wid][g + u] = m;
        c += __popc(m);
      }
    }
    if (lane == 0) wtot[wid] = c;
  }
  if (tid == 0) s_maxlen = 0;
  for (int i = tid; i < 64; i += blockDim.x) bl_count[i] = 0;
  __syncthreads();
  if (tid == 0) {
    uint32_t run = 0;
    for (int w = 0; w < 32; ++w) {
      const uint32_t t = wtot[w];
      wtot[w] = run;
      run += t;
    }
    s_n = run;
  }
  __syncthreads();
  const uint32_t n = s_n;
  const bool in_smem = n <= kSmemLeaves;
  const uint32_t P = next_pow2(n);
  unsigned long long* keys = in_smem ? smem : gkeys;
  unsigned long long* iw = in_smem ? smem + kSmemLeaves : giw;
  uint32_t* par = in_smem ? reinterpret_cast<uint32_t*>(smem + 2 * kSmemLeaves)
                          : gpar;
  {
    uint32_t pos = wtot[wid];
#pragma unroll
    for (int g = 0; g < 64; g += 16) {
      uint32_t f[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) f[u] = hw[(g + u) * 32];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const uint32_t m = masks[wid][g + u];
        const uint32_t b = wid * 2048 + (g + u) * 32 + lane;
        if (m & (1u << lane)) {
          const uint32_t k = pos + __popc(m & ((1u << lane) - 1u));
          keys[k] = ((unsigned long long)f[u] << 16) | b;
          if (!kCostOnly) tsyms[k] = (uint16_t)b;
        }
        pos += __popc(m);
      }
    }
  }
  for (uint32_t i = n + tid; i < P; i += blockDim.x) keys[i] = ~0ull;
  __syncthreads();
  if (kCostOnly && n <= 1) {  // a lone symbol gets the empty code
    if (tid == 0) *cost = 0;
    return;
  }
  if (n == 1) {
    if (tid == 0) {
      const uint32_t sym = (uint32_t)(keys[0] & 0xFFFFu);
      enc[sym] = 0ull;  // the empty code
      tlens[0] = 0;
      ctl->n_used = 1;
      ctl->max_len = 0;
    }
    return;
  }
  // 2. leaves by (frequency, symbol): small alphabets by rank counting
  //    (keys are distinct), large ones by a bitonic sort
  const bool small = n <= kRankSort;
  if (small) {
    unsigned long long* tmp = smem + 3 * kSmemLeaves / 2;  // scratch half of par
    for (uint32_t i = tid; i < n; i += blockDim.x) tmp[i] = keys[i];
    __syncthreads();
    for (uint32_t i = tid; i < n; i += blockDim.x) {
      const unsigned long long k = tmp[i];
      uint32_t r = 0;
      for (uint32_t j = 0; j < n; ++j) r += tmp[j] < k;
      keys[r] = k;
    }
    __syncthreads();
  } else {
    bitonic_sort(keys, P);
  }
  // 3. two-queue merge
  if (wid == 0) {
    const unsigned long long c = warp_huffman_merge(keys, n, iw, kCostOnly ? nullptr : par);
    if (kCostOnly && lane == 0) *cost = c;
  }
  if (kCostOnly) return;
  __syncthreads();
  // 4. leaf depths by walking to the root (one walk per leaf)
  const uint32_t root = 2 * n - 2;
  uint32_t my_max = 0;
  for (uint32_t i = tid; i < n; i += blockDim.x) {
    uint32_t d = 0, v = i;
    while (v != root && d < 64) {  // depth <= 63 for any valid tree
      v = par[v];
      ++d;
    }
    const uint32_t sym = (uint32_t)(keys[i] & 0xFFFFu);
    lens_by_sym[sym] = (uint8_t)d;
    my_max = max(my_max, d);
    atomicAdd(&bl_count[d < 63 ? d : 63], 1u);
  }
  atomicMax(&s_maxlen, my_max);
  __syncthreads();
  const uint32_t maxlen = s_maxlen;
  if (maxlen > 56) {
    if (tid == 0) ctl->status = ST_INVALID;
    return;
  }
  // 5. canonical order (length, symbol)
  if (small) {
    // rank of a symbol among the symbols of its length = number of smaller
    // symbols of that length; symbols are ascending in tsyms
    uint8_t* lsym = reinterpret_cast<uint8_t*>(smem + 3 * kSmemLeaves / 2);
    for (uint32_t k = tid; k < n; k += blockDim.x) lsym[k] = lens_by_sym[tsyms[k]];
    __syncthreads();
    if (tid == 0) {
      unsigned long long code = 0;
      bl_count[0] = 0;
      for (uint32_t bits = 1; bits <= maxlen; ++bits) {
        code = (code + bl_count[bits - 1]) << 1;
        first_code[bits] = code;
      }
      ctl->n_used = n;
      ctl->max_len = maxlen;
    }
    __syncthreads();
    for (uint32_t k = tid; k < n; k += blockDim.x) {
      const uint8_t L = lsym[k];
      uint32_t r = 0;
      for (uint32_t j = 0; j < k; ++j) r += lsym[j] == L;
      const uint32_t sym = tsyms[k];
      enc[sym] = ((unsigned long long)L << 56) | (first_code[L] + r);
      tlens[k] = L;
    }
    return;
  }
  for (uint32_t i = tid; i < n; i += blockDim.x) {
    const uint32_t sym = (uint32_t)(keys[i] & 0xFFFFu);
    keys[i] = ((unsigned long long)lens_by_sym[sym] << 16) | sym;
  }
  __syncthreads();
  bitonic_sort(keys, P);
  if (tid == 0) {
    unsigned long long code = 0;
    uint32_t p = 0;
    bl_count[0] = 0;
    for (uint32_t bits = 1; bits <= maxlen; ++bits) {
      code = (code + bl_count[bits - 1]) << 1;
      first_code[bits] = code;
      start_pos[bits] = p;
      p += bl_count[bits];
    }
    ctl->n_used = n;
    ctl->max_len = maxlen;
  }
  __syncthreads();
  for (uint32_t i = tid; i < n; i += blockDim.x) {
    const uint32_t len = (uint32_t)(keys[i] >> 16);
    const uint32_t sym = (uint32_t)(keys[i] & 0xFFFFu);
    const unsigned long long code = first_code[len] + (i - start_pos[len]);
    enc[sym] = ((unsigned long long)len << 56) | code;
  }
  for (uint32_t k = tid; k < n; k += blockDim.x) tlens[k] = lens_by_sym[tsyms[k]];
}

__global__ void __launch_bounds__(1024)
    k_codebook(const uint32_t* __restrict__ hist, unsigned long long* enc,
               uint16_t* tsyms, uint8_t* tlens, unsigned long long* gkeys,
               unsigned long long* giw, uint32_t* gpar, uint8_t* lens_by_sym,
               Ctl* ctl) {
  codebook_body<false>(hist, enc, tsyms, tlens, gkeys, giw, gpar, lens_by_sym, ctl);
}

// ---------------------------------------------------------------------
// encode: lane bit counts and chunk word counts
// ---------------------------------------------------------------------
__device__ __forceinline__ void enc_len_body(
    const uint16_t* __restrict__ codes, uint32_t N, uint32_t C, uint32_t nch,
    const unsigned long long* __restrict__ enc, uint16_t* __restrict__ lanebits,
    uint32_t* __restrict__ chw, const Ctl* __restrict__ ctl, unsigned bid,
    unsigned nblk) {
  if (ctl->status || ctl->is_const) return;
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (bid * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (nblk * blockDim.x) >> 5;
  for (uint32_t c = warp; c < nch; c += nwarps) {
    const uint32_t beg = c * C, nc = min(C, N - beg);
    uint32_t bits = 0;
    // batches of 8: all code loads, then all table lookups, in flight
    uint32_t j = lane;
    for (; j + 7 * 32 < nc; j += 8 * 32) {
      unsigned cd[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) cd[k] = codes[beg + j + 32 * k];
      unsigned long long e[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) e[k] = __ldg(enc + cd[k]);
#pragma unroll
      for (int k = 0; k < 8; ++k) bits += (uint32_t)(e[k] >> 56);
    }
    for (; j < nc; j += 32) bits += (uint32_t)(enc[codes[beg + j]] >> 56);
    lanebits[(size_t)c * 32 + lane] = (uint16_t)bits;
    uint32_t tot = bits;
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) chw[c] = (tot + 31) >> 5;
  }
}

__global__ void __launch_bounds__(256)
    k_enc_len(const uint16_t* __restrict__ codes, uint32_t N, uint32_t C,
              uint32_t nch, const unsigned long long* __restrict__ enc,
              uint16_t* __restrict__ lanebits, uint32_t* __restrict__ chw,
              const Ctl* __restrict__ ctl) {
  enc_len_body(codes, N, C, nch, enc, lanebits, chw, ctl, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------
// encode: packing, one warp per chunk, lane l writes its own bit range
// ---------------------------------------------------------------------
struct BitWriter {
  uint32_t* words;   // chunk base
  uint32_t wi;       // current word index
  unsigned long long acc;
  int nacc;
  bool shared_first;
  __device__ void emit(uint32_t w) {
    if (shared_first) {
      atomicOr(words + wi, w);
      shared_first = false;
    } else {
      words[wi] = w;
    }
    ++wi;
  }
  __device__ void put(uint32_t v, int n) {  // n <= 32, nacc < 32
    if (n == 0) return;
    acc |= (unsigned long long)v << (64 - nacc - n);
    nacc += n;
    if (nacc >= 32) {
      emit((uint32_t)(acc >> 32));
      acc <<= 32;
      nacc -= 32;
    }
  }
  __device__ void put_code(unsigned long long e) {
    const int len = (int)(e >> 56);
    const unsigned long long code = e & ((1ull << 56) - 1);
    if (len > 32) {
      put((uint32_t)(code >> 32), len - 32);
      put((uint32_t)code, 32);
    } else {
      put((uint32_t)code, len);
    }
  }
  __device__ void flush() {
    if (nacc > 0) atomicOr(words + wi, (uint32_t)(acc >> 32));
  }
};

// one chunk's packing by its warp: the chunk's nw words at `words`, lane
// `lane` holding mybits bits of the chunk's codes beg + lane + 32 k
__device__ __forceinline__ void pack_chunk(const uint16_t* __restrict__ codes, uint32_t beg,
                                           uint32_t nc, const unsigned long long* __restrict__ enc,
                                           uint32_t mybits, uint32_t* words, uint32_t nw,
                                           int lane) {
    for (uint32_t i = lane; i < nw; i += 32) words[i] = 0u;
    __syncwarp();
    uint32_t off = mybits;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, off, o);
      if (lane >= o) off += y;
    }
    off -= mybits;
    BitWriter bw;
    bw.words = words;
    bw.wi = off >> 5;
    bw.nacc = (int)(off & 31);
    bw.acc = 0;
    bw.shared_first = bw.nacc != 0;
    uint32_t j = lane;
    // the codes of the next batch are loaded while this one is packed
    unsigned nx[8];
    if (j + 7 * 32 < nc) {
#pragma unroll
      for (int k = 0; k < 8; ++k) nx[k] = codes[beg + j + 32 * k];
    }
    for (; j + 7 * 32 < nc; j += 8 * 32) {
      unsigned cd[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) cd[k] = nx[k];
      if (j + 15 * 32 < nc) {
#pragma unroll
        for (int k = 0; k < 8; ++k) nx[k] = codes[beg + j + 256 + 32 * k];
      }
      unsigned long long e[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) e[k] = __ldg(enc + cd[k]);
      // two consecutive codes of the lane whose lengths add up to at most
      // 32 bits go out as one word fragment (the same bits, fewer steps)
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        const int l0 = (int)(e[k] >> 56), l1 = (int)(e[k + 1] >> 56);
        if (l0 + l1 <= 32) {
          const unsigned long long v =
              ((e[k] & ((1ull << 56) - 1)) << l1) | (e[k + 1] & ((1ull << 56) - 1));
          bw.put((uint32_t)v, l0 + l1);
        } else {
          bw.put_code(e[k]);
          bw.put_code(e[k + 1]);
        }
      }
    }
    for (; j < nc; j += 32) bw.put_code(enc[codes[beg + j]]);
    bw.flush();
    __syncwarp();
}

__device__ __forceinline__ void pack_body(
    const uint16_t* __restrict__ codes, uint32_t N, uint32_t C, uint32_t nch,
    const unsigned long long* __restrict__ enc,
    const uint16_t* __restrict__ lanebits, const uint32_t* __restrict__ chw,
    const unsigned long long* __restrict__ woff, uint8_t* out,
    const Ctl* __restrict__ ctl, unsigned bid, unsigned nblk) {
  if (ctl->status || ctl->is_const) return;
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (bid * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (nblk * blockDim.x) >> 5;
  uint32_t* bits = reinterpret_cast<uint32_t*>(out + ctl->off_bits);
  for (uint32_t c = warp; c < nch; c += nwarps) {
    const uint32_t beg = c * C, nc = min(C, N - beg);
    pack_chunk(codes, beg, nc, enc, lanebits[(size_t)c * 32 + lane], bits + woff[c], chw[c],
               lane);
  }
}

// ---------------------------------------------------------------------
// encode in one pass (single field): a CTA of kEncWarps warps takes the
// chunks in order from a counter.  Per chunk it stages the chunk's codes in
// shared memory by asynchronous 16-byte copies (the codes leave DRAM once;
// both passes read them there), counts its lanes' bits, publishes the
// chunk's word count, finds the chunk's word offset by a decoupled
// look-back over the flags of the chunks before it (a flag holds a count:
// status 1 = this chunk's words, 2 = the words of every chunk up to it),
// publishes that inclusive count and packs the chunk.  Warp w counts and
// packs part w of every lane's codes (lane l: codes l + 32 k, k in the
// part's range): a part starts at its lane's bit offset plus the bits of
// the lane's earlier parts and shares at most its first and last word with
// the neighbouring parts (atomicOr, as between lanes).  Warp 0 publishes
// and looks back.  Chunks are taken in order, so every chunk a look-back
// waits for is held by a running CTA.  The waits are bounded: on expiry
// the call fails with a timeout.
// ---------------------------------------------------------------------
constexpr unsigned long long kEncWaitPolls = 1ull << 22;

__device__ __forceinline__ unsigned long long load_flag(const unsigned long long* f) {
  return *reinterpret_cast<const volatile unsigned long long*>(f);
}

constexpr int kEncWarps = 8;

// 16 bytes global -> shared without registers (both 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// part [k0, k1) of lane `lane`'s codes in a staged chunk of nc codes, from
// bit `off` of the chunk's words
__device__ __forceinline__ void pack_part(const uint16_t* sc, uint32_t nc, int lane,
                                          uint32_t k0, uint32_t k1,
                                          const unsigned long long* __restrict__ enc,
                                          uint32_t* words, uint32_t off) {
  BitWriter bw;
  bw.words = words;
  bw.wi = off >> 5;
  bw.nacc = (int)(off & 31);
  bw.acc = 0;
  bw.shared_first = bw.nacc != 0;
  if (k1 > k0 && lane + 32 * (k1 - 1) >= nc) --k1;  // the lane's last code may be missing
  uint32_t k = k0;
  for (; k + 8 <= k1; k += 8) {
    unsigned long long e[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) e[u] = __ldg(enc + sc[lane + 32 * (k + u)]);
    // two codes whose lengths add up to at most 32 bits go out as one
    // word fragment (the same bits, fewer steps)
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      const int l0 = (int)(e[u] >> 56), l1 = (int)(e[u + 1] >> 56);
      if (l0 + l1 <= 32) {
        const unsigned long long v =
            ((e[u] & ((1ull << 56) - 1)) << l1) | (e[u + 1] & ((1ull << 56) - 1));
        bw.put((uint32_t)v, l0 + l1);
      } else {
        bw.put_code(e[u]);
        bw.put_code(e[u + 1]);
      }
    }
  }
  for (; k < k1; ++k) bw.put_code(__ldg(enc + sc[lane + 32 * k]));
  bw.flush();
}

__global__ void __launch_bounds__(kEncWarps * 32)
    k_encode_staged(const uint16_t* __restrict__ codes, uint32_t N, uint32_t C, uint32_t nch,
                    const unsigned long long* __restrict__ enc, uint16_t* __restrict__ lanebits,
                    unsigned long long* flags, uint32_t* counter, uint8_t* out, Ctl* ctl,
                    unsigned long long cap) {
  extern __shared__ uint4 sc4[];  // the chunk's codes
  const uint16_t* sc = reinterpret_cast<const uint16_t*>(sc4);
  __shared__ uint32_t cnt[kEncWarps][32];  // bits per (part, lane)
  __shared__ uint32_t laneoff[32];         // lane bit offsets in the chunk
  __shared__ uint32_t s_c, s_nw;
  __shared__ unsigned long long s_prefix;
  __shared__ int s_state;  // 0 pack, 1 past the capacity, 2 timed out
  // one reading of the status for the whole CTA (other CTAs of this launch
  // may set it while this one starts; its warps meet at barriers)
  if (threadIdx.x == 0) s_state = (ctl->status || ctl->is_const) ? 2 : 0;
  __syncthreads();
  if (s_state == 2) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned long long off_bits = ctl->off_bits;
  uint32_t* bits = reinterpret_cast<uint32_t*>(out + off_bits);
  for (;;) {
    if (threadIdx.x == 0) s_c = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t c = s_c;
    if (c >= nch) return;
    const uint32_t beg = c * C, nc = min(C, N - beg);
    // stage: asynchronous 16-byte copies straight into shared memory, all
    // of the chunk in flight at once
    {
      const uint32_t n8 = nc / 8;
      const uint4* src = reinterpret_cast<const uint4*>(codes + beg);
      for (uint32_t i = threadIdx.x; i < n8; i += blockDim.x) cp_async16(sc4 + i, src + i);
      cp_async_wait_all();
      uint16_t* sct = reinterpret_cast<uint16_t*>(sc4);
      for (uint32_t i = 8 * n8 + threadIdx.x; i < nc; i += blockDim.x) sct[i] = codes[beg + i];
    }
    __syncthreads();
    // part w of the lane's codes: k in [k0, k1)
    const uint32_t kmax = (nc + 31) / 32;
    const uint32_t k0 = (uint32_t)((uint64_t)kmax * w / kEncWarps);
    const uint32_t k1 = (uint32_t)((uint64_t)kmax * (w + 1) / kEncWarps);
    {
      uint32_t pb = 0;
      uint32_t k = k0;
      for (; k + 8 <= k1 && lane + 32 * (k + 7) < nc; k += 8) {
        unsigned long long e[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) e[u] = __ldg(enc + sc[lane + 32 * (k + u)]);
#pragma unroll
        for (int u = 0; u < 8; ++u) pb += (uint32_t)(e[u] >> 56);
      }
      for (; k < k1; ++k)
        if (lane + 32 * k < nc) pb += (uint32_t)(__ldg(enc + sc[lane + 32 * k]) >> 56);
      cnt[w][lane] = pb;
    }
    __syncthreads();
    if (w == 0) {
      uint32_t mybits = 0;
#pragma unroll
      for (int q = 0; q < kEncWarps; ++q) mybits += cnt[q][lane];
      lanebits[(size_t)c * 32 + lane] = (uint16_t)mybits;
      uint32_t incl = mybits;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      laneoff[lane] = incl - mybits;
      const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      const unsigned long long nw = (tot + 31) >> 5;
      if (lane == 0) atomicExch(flags + c, (nw << 2) | 1ull);
      unsigned long long prefix = 0;
      bool timed_out = false;
      for (long long j = (long long)c - 1; j >= 0;) {
        const long long jj = j - lane;
        unsigned long long f = jj >= 0 ? load_flag(flags + jj) : 2ull;
        unsigned long long polls = 0;
        while (__any_sync(0xffffffffu, (f & 3ull) == 0ull)) {
          if (++polls > kEncWaitPolls) {
            timed_out = true;
            break;
          }
          __nanosleep(64);
          if ((f & 3ull) == 0ull) f = load_flag(flags + jj);
        }
        if (timed_out) break;
        const unsigned inc = __ballot_sync(0xffffffffu, (f & 3ull) == 2ull);
        const int upto = inc ? __ffs(inc) - 1 : 31;
        unsigned long long v = lane <= upto ? (f >> 2) : 0ull;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        prefix += v;
        if (inc) break;
        j -= 32;
      }
      if (lane == 0) {
        if (timed_out) {
          atomicCAS(&ctl->status, 0, ST_TIMEOUT);
          s_state = 2;
        } else {
          atomicExch(flags + c, ((prefix + nw) << 2) | 2ull);
          if (c + 1 == nch) {
            ctl->total_words = prefix + nw;
            ctl->total_size = off_bits + 4ull * (prefix + nw);
            if (ctl->total_size > cap) atomicCAS(&ctl->status, 0, ST_OUT_TOO_SMALL);
          }
          // nothing written past the output's capacity
          s_state = off_bits + 4ull * (prefix + nw) > cap ? 1 : 0;
          s_prefix = prefix;
          s_nw = (uint32_t)nw;
        }
      }
    }
    __syncthreads();
    if (s_state == 2) return;
    if (s_state == 1) continue;
    uint32_t* words = bits + s_prefix;
    for (uint32_t i = threadIdx.x; i < s_nw; i += blockDim.x) words[i] = 0u;
    __syncthreads();
    uint32_t off = laneoff[lane];
    for (int q = 0; q < w; ++q) off += cnt[q][lane];
    pack_part(sc, nc, lane, k0, k1, enc, words, off);
  }
}

__global__ void __launch_bounds__(256)
    k_pack(const uint16_t* __restrict__ codes, uint32_t N, uint32_t C,
           uint32_t nch, const unsigned long long* __restrict__ enc,
           const uint16_t* __restrict__ lanebits,
           const uint32_t* __restrict__ chw,
           const unsigned long long* __restrict__ woff, uint8_t* out,
           const Ctl* __restrict__ ctl) {
  pack_body(codes, N, C, nch, enc, lanebits, chw, woff, out, ctl, blockIdx.x,
            gridDim.x);
}

// chunk word counts from the stored lane bit counts (decompress)
__device__ __forceinline__ void chunk_words_body(
    const uint8_t* __restrict__ lanebits_bytes, uint32_t nch,
    uint32_t* __restrict__ chw, unsigned bid, unsigned nblk) {
  for (uint32_t c = bid * blockDim.x + threadIdx.x; c < nch;
       c += nblk * blockDim.x) {
    const uint8_t* p = lanebits_bytes + (size_t)c * 64;
    uint32_t s = 0;
    for (int l = 0; l < 32; ++l) s += (uint32_t)p[2 * l] | ((uint32_t)p[2 * l + 1] << 8);
    chw[c] = (s + 31) >> 5;
  }
}

__global__ void k_chunk_words(const uint8_t* __restrict__ lanebits_bytes,
                              uint32_t nch, uint32_t* __restrict__ chw) {
  chunk_words_body(lanebits_bytes, nch, chw, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------
// outlier gather (compress) / scatter (decompress), row-major order.
// One CTA per chunk; CTAs of chunks without an outlier leave at once.
// Each thread counts the escapes (code 0) in a contiguous run of the
// chunk, a block scan turns the counts into ranks, and the thread moves
// its outliers in order.
// ---------------------------------------------------------------------
__device__ __forceinline__ void outliers_body(
    bool gather, const uint16_t* __restrict__ codes, uint32_t N, uint32_t C,
    uint32_t nch, const uint32_t* __restrict__ zc,
    const unsigned long long* __restrict__ zoff, const float* src, float* dst,
    uint8_t* stream, unsigned long long max_out, Ctl* ctl, unsigned bid) {
  if (ctl->status || ctl->is_const) return;
  const uint32_t c = bid;
  if (c >= nch || zc[c] == 0) return;
  float* outl = reinterpret_cast<float*>(stream + ctl->off_outliers);
  const uint32_t beg = c * C, end = min(beg + C, N);
  const uint32_t per = (C + blockDim.x - 1) / blockDim.x;
  const uint32_t tb = min(beg + threadIdx.x * per, end), te = min(tb + per, end);
  uint32_t mine = 0;
  const bool vec = (per % 8 == 0) && (te - tb == per);
  if (vec) {
    const uint4* p = reinterpret_cast<const uint4*>(codes + tb);
    for (uint32_t k = 0; k < per / 8; ++k) {
      const uint4 v = p[k];
      const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) mine += ((w[q] & 0xFFFFu) == 0) + ((w[q] >> 16) == 0);
    }
  } else {
    for (uint32_t i = tb; i < te; ++i) mine += codes[i] == 0;
  }
  uint32_t total;
  uint32_t rank = block_exclusive_scan(mine, &total);
  if (mine == 0) return;
  unsigned long long k = zoff[c] + rank;
  for (uint32_t i = tb; i < te; ++i) {
    if (codes[i] != 0) continue;
    if (k >= max_out) {  // more escapes than stored outliers: corrupt
      atomicExch(&ctl->status, ST_CORRUPT);
      return;
    }
    if (gather)
      outl[k] = src[i];
    else
      dst[i] = outl[k];
    ++k;
  }
}

__global__ void __launch_bounds__(256)
    k_outliers(bool gather, const uint16_t* __restrict__ codes, uint32_t N,
               uint32_t C, uint32_t nch, const uint32_t* __restrict__ zc,
               const unsigned long long* __restrict__ zoff, const float* src,
               float* dst, uint8_t* stream, unsigned long long max_out,
               Ctl* ctl) {
  outliers_body(gather, codes, N, C, nch, zc, zoff, src, dst, stream, max_out,
                ctl, blockIdx.x);
}

// ---------------------------------------------------------------------
// decode tables from the stream's (symbol, length) table
//   dec: [0,4096) LUT (len << 16 | sym, 0 = longer than 12 bits)
//        then count[64], first[64] (u64), offs[64], sorted syms
// ---------------------------------------------------------------------
constexpr int kLutBits = 12;

__device__ __forceinline__ void dec_tables_body(
    const uint8_t* __restrict__ stream, uint32_t n_used, uint64_t off_table,
    uint32_t* lut, uint32_t* cnt, unsigned long long* first, uint32_t* offs,
    uint16_t* sorted, unsigned long long* gkeys, Ctl* ctl) {
  extern __shared__ unsigned long long smem[];
  __shared__ uint32_t s_bad;
  __shared__ uint32_t s_cnt[64];
  const int tid = threadIdx.x;
  const uint8_t* tab = stream + off_table;
  if (tid == 0) s_bad = 0;
  for (int i = tid; i < 64; i += blockDim.x) s_cnt[i] = 0;
  for (int i = tid; i < (1 << kLutBits); i += blockDim.x) lut[i] = 0;
  __syncthreads();
  const uint32_t P = next_pow2(n_used);
  unsigned long long* keys = n_used <= kSmemLeaves ? smem : gkeys;
  for (uint32_t k = tid; k < P; k += blockDim.x) {
    if (k < n_used) {
      const uint32_t sym = (uint32_t)tab[2 * k] | ((uint32_t)tab[2 * k + 1] << 8);
      const uint32_t len = tab[2 * (size_t)n_used + k];
      if (k > 0) {
        const uint32_t prev =
            (uint32_t)tab[2 * k - 2] | ((uint32_t)tab[2 * k - 1] << 8);
        if (sym <= prev) s_bad = 1;
      }
      if (len > 56 || (n_used > 1 && len == 0) || (n_used == 1 && len != 0))
        s_bad = 1;
      keys[k] = ((unsigned long long)len << 16) | sym;
      atomicAdd(&s_cnt[len & 63], 1u);
    } else {
      keys[k] = ~0ull;
    }
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) ctl->status = ST_CORRUPT;
    return;
  }
  bitonic_sort(keys, P);
  if (tid == 0) {
    unsigned long long code = 0;
    uint32_t p = 0;
    unsigned long long kraft = 0;
    for (int b = 0; b < 64; ++b) {
      cnt[b] = s_cnt[b];
      first[b] = 0;
      offs[b] = 0;
    }
    for (int b = 1; b < 64; ++b) {
      code = (code + (b - 1 >= 1 ? s_cnt[b - 1] : 0)) << 1;
      first[b] = code;
      offs[b] = p;
      p += s_cnt[b];
      if (b <= 56) kraft += (unsigned long long)s_cnt[b] << (56 - b);
    }
    if (n_used > 1 && kraft != (1ull << 56)) ctl->status = ST_CORRUPT;
  }
  __syncthreads();
  for (uint32_t i = tid; i < n_used; i += blockDim.x) {
    const uint32_t len = (uint32_t)(keys[i] >> 16);
    const uint32_t sym = (uint32_t)(keys[i] & 0xFFFFu);
    sorted[i] = (uint16_t)sym;
    if (len >= 1 && len <= kLutBits) {
      // code = first[len] + rank within its length
      uint32_t lo_pos = 0;
      unsigned long long fc = 0;
      {
        unsigned long long c2 = 0;
        uint32_t p2 = 0;
        for (uint32_t b = 1; b <= len; ++b) {
          c2 = (c2 + (b - 1 >= 1 ? s_cnt[b - 1] : 0)) << 1;
          if (b == len) {
            fc = c2;
            lo_pos = p2;
          }
          p2 += s_cnt[b];
        }
      }
      const unsigned long long code = fc + (i - lo_pos);
      const uint32_t a = (uint32_t)(code << (kLutBits - len));
      const uint32_t e = (uint32_t)((code + 1) << (kLutBits - len));
      for (uint32_t j = a; j < e && j < (1u << kLutBits); ++j)
        lut[j] = (len << 16) | sym;
    }
  }
}

__global__ void __launch_bounds__(1024)
    k_dec_tables(const uint8_t* __restrict__ stream, uint32_t n_used,
                 uint64_t off_table, uint32_t* lut, uint32_t* cnt,
                 unsigned long long* first, uint32_t* offs, uint16_t* sorted,
                 unsigned long long* gkeys, Ctl* ctl) {
  dec_tables_body(stream, n_used, off_table, lut, cnt, first, offs, sorted,
                  gkeys, ctl);
}

// ---------------------------------------------------------------------
// decode: one warp per chunk, lane l decodes its own bit range
// ---------------------------------------------------------------------
__device__ __forceinline__ void decode_body(
    const uint8_t* __restrict__ stream, uint64_t off_bits, uint64_t total_words,
    const uint8_t* __restrict__ lanebits_bytes,
    const unsigned long long* __restrict__ woff, uint32_t N, uint32_t C,
    uint32_t nch, uint32_t n_used, uint16_t single_sym,
    const uint32_t* __restrict__ g_lut, const uint32_t* __restrict__ g_cnt,
    const unsigned long long* __restrict__ g_first,
    const uint32_t* __restrict__ g_offs, const uint16_t* __restrict__ sorted,
    uint16_t* __restrict__ codes, uint32_t* __restrict__ zc, Ctl* ctl,
    unsigned bid, unsigned nblk) {
  __shared__ uint32_t lut[1 << kLutBits];
  __shared__ uint32_t cnt[64], offs[64];
  __shared__ unsigned long long first[64];
  for (int i = threadIdx.x; i < (1 << kLutBits); i += blockDim.x) lut[i] = g_lut[i];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    cnt[i] = g_cnt[i];
    offs[i] = g_offs[i];
    first[i] = g_first[i];
  }
  __syncthreads();
  if (ctl->status) return;
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (bid * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (nblk * blockDim.x) >> 5;
  const uint32_t* allw = reinterpret_cast<const uint32_t*>(stream + off_bits);
  for (uint32_t c = warp; c < nch; c += nwarps) {
    const uint32_t beg = c * C, nc = min(C, N - beg);
    const uint8_t* lb = lanebits_bytes + (size_t)c * 64;
    const uint32_t mybits = (uint32_t)lb[2 * lane] | ((uint32_t)lb[2 * lane + 1] << 8);
    uint32_t start = mybits, tot;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, start, o);
      if (lane >= o) start += y;
    }
    tot = __shfl_sync(0xffffffffu, start, 31);
    start -= mybits;
    const uint32_t nw = (tot + 31) >> 5;
    const unsigned long long w0 = woff[c];
    uint32_t zeros = 0;
    bool bad = w0 + nw > total_words;
    if (n_used == 1) {
      bad |= mybits != 0;
      if (!bad)
        for (uint32_t j = lane; j < nc; j += 32) codes[beg + j] = single_sym;
      zeros = single_sym == 0 ? (nc + 31 - lane) / 32 : 0;
    } else if (!bad) {
      const uint32_t* words = allw + w0;
      uint32_t wi = start >> 5;
      unsigned long long buf = 0;
      int nbuf = 0;
      {
        const uint32_t w = wi < nw ? __ldg(words + wi) : 0u;
        const int sh = (int)(start & 31);
        buf = ((unsigned long long)w << 32) << sh;
        nbuf = 32 - sh;
        ++wi;
      }
      // the lane's next two words are loaded ahead, so a refill takes a
      // word that has arrived while earlier symbols were decoded (word wi
      // and wi + 1 of the lane, 0 past the chunk's words)
      uint32_t nx0 = wi < nw ? __ldg(words + wi) : 0u;
      uint32_t nx1 = wi + 1 < nw ? __ldg(words + wi + 1) : 0u;
      uint32_t left = mybits;  // bits of this lane not consumed yet
      for (uint32_t j = lane; j < nc; j += 32) {
        while (nbuf <= 32) {
          buf |= (unsigned long long)nx0 << (32 - nbuf);
          nbuf += 32;
          ++wi;
          nx0 = nx1;
          nx1 = wi + 1 < nw ? __ldg(words + wi + 1) : 0u;
        }
        const uint32_t e = lut[(uint32_t)(buf >> (64 - kLutBits))];
        uint32_t sym = 0, len = 0;
        if (e != 0) {
          len = e >> 16;
          sym = e & 0xFFFFu;
        } else {
          for (uint32_t L = kLutBits + 1; L < 57; ++L) {
            const unsigned long long v = buf >> (64 - L);
            if (cnt[L] && v >= first[L] && v - first[L] < cnt[L]) {
              sym = sorted[offs[L] + (uint32_t)(v - first[L])];
              len = L;
              break;
            }
          }
        }
        if (len == 0 || len > left) {
          bad = true;
          break;
        }
        left -= len;
        buf <<= len;
        nbuf -= (int)len;
        zeros += sym == 0;
        codes[beg + j] = (uint16_t)sym;
      }
      bad |= left != 0;
    }
    if (bad) atomicExch(&ctl->status, ST_CORRUPT);
    for (int o = 16; o > 0; o >>= 1) zeros += __shfl_xor_sync(0xffffffffu, zeros, o);
    if (lane == 0) zc[c] = zeros;
  }
}

__global__ void __launch_bounds__(256)
    k_decode(const uint8_t* __restrict__ stream, uint64_t off_bits,
             uint64_t total_words, const uint8_t* __restrict__ lanebits_bytes,
             const unsigned long long* __restrict__ woff, uint32_t N,
             uint32_t C, uint32_t nch, uint32_t n_used, uint16_t single_sym,
             const uint32_t* __restrict__ g_lut,
             const uint32_t* __restrict__ g_cnt,
             const unsigned long long* __restrict__ g_first,
             const uint32_t* __restrict__ g_offs,
             const uint16_t* __restrict__ sorted, uint16_t* __restrict__ codes,
             uint32_t* __restrict__ zc, Ctl* ctl, const uint8_t* __restrict__ single_src) {
  // single_src: the lone symbol of a one-symbol table read from the stream
  // here (no host read), else single_sym as given
  const uint16_t sym =
      single_src ? (uint16_t)(single_src[0] | (single_src[1] << 8)) : single_sym;
  decode_body(stream, off_bits, total_words, lanebits_bytes, woff, N, C, nch,
              n_used, sym, g_lut, g_cnt, g_first, g_offs, sorted, codes,
              zc, ctl, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------
// batched forms
// ---------------------------------------------------------------------
__global__ void __launch_bounds__(256)
    k_hist_batch(const HistJob* __restrict__ J, const uint32_t* __restrict__ off,
                 int nj) {
  const int j = batch_job(off, nj);
  const HistJob& q = J[j];
  hist_body(q.codes, q.N, q.C, q.nch, q.hist, q.zc, q.ctl, blockIdx.x - off[j],
            off[j + 1] - off[j]);
}

__global__ void __launch_bounds__(1024) k_codebook_batch(const CodebookJob* __restrict__ J) {
  const CodebookJob& q = J[blockIdx.x];
  codebook_body<false>(q.hist, q.enc, q.tsyms, q.tlens, q.gkeys, q.giw, q.gpar,
                       q.lens_by_sym, q.ctl);
}

// total bits of an optimal code of each job's histogram (the tuner's
// estimate), one CTA per job
__global__ void __launch_bounds__(1024)
    k_hcost_batch(const CodebookJob* __restrict__ J, unsigned long long* cost) {
  const CodebookJob& q = J[blockIdx.x];
  codebook_body<true>(q.hist, q.enc, q.tsyms, q.tlens, q.gkeys, q.giw, q.gpar,
                      q.lens_by_sym, q.ctl, cost + blockIdx.x);
}

__global__ void __launch_bounds__(256)
    k_enc_len_batch(const EncLenJob* __restrict__ J,
                    const uint32_t* __restrict__ off, int nj) {
  const int j = batch_job(off, nj);
  const EncLenJob& q = J[j];
  enc_len_body(q.codes, q.N, q.C, q.nch, q.enc, q.lanebits, q.chw, q.ctl,
               blockIdx.x - off[j], off[j + 1] - off[j]);
}

__global__ void __launch_bounds__(256)
    k_pack_batch(const PackJob* __restrict__ J, const uint32_t* __restrict__ off,
                 int nj) {
  const int j = batch_job(off, nj);
  const PackJob& q = J[j];
  pack_body(q.codes, q.N, q.C, q.nch, q.enc, q.lanebits, q.chw, q.woff, q.out,
            q.ctl, blockIdx.x - off[j], off[j + 1] - off[j]);
}

__global__ void k_chunk_words_batch(const ChunkWordsJob* __restrict__ J,
                                    const uint32_t* __restrict__ off, int nj) {
  const int j = batch_job(off, nj);
  chunk_words_body(J[j].lanebits_bytes, J[j].nch, J[j].chw, blockIdx.x - off[j],
                   off[j + 1] - off[j]);
}

__global__ void __launch_bounds__(256)
    k_outliers_batch(const OutlierJob* __restrict__ J,
                     const uint32_t* __restrict__ off, int nj) {
  const int j = batch_job(off, nj);
  const OutlierJob& q = J[j];
  outliers_body(q.gather != 0, q.codes, q.N, q.C, q.nch, q.zc, q.zoff, q.src,
                q.dst, q.stream, q.max_out, q.ctl, blockIdx.x - off[j]);
}

__global__ void __launch_bounds__(1024)
    k_dec_tables_batch(const DecTablesJob* __restrict__ J) {
  const DecTablesJob& q = J[blockIdx.x];
  dec_tables_body(q.stream, q.n_used, q.off_table, q.lut, q.cnt, q.first,
                  q.offs, q.sorted, q.gkeys, q.ctl);
}

__global__ void __launch_bounds__(256)
    k_decode_batch(const DecodeJob* __restrict__ J,
                   const uint32_t* __restrict__ off, int nj) {
  const int j = batch_job(off, nj);
  const DecodeJob& q = J[j];
  const uint16_t single =
      q.single_src ? (uint16_t)(q.single_src[0] | (q.single_src[1] << 8)) : 0;
  decode_body(q.stream, q.off_bits, q.total_words, q.lanebits_bytes, q.woff, q.N,
              q.C, q.nch, q.n_used, single, q.lut, q.cnt, q.first, q.offs,
              q.sorted, q.codes, q.zc, q.ctl, blockIdx.x - off[j],
              off[j + 1] - off[j]);
}

// ---------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------
static inline unsigned warps_grid(uint32_t nch, int num_sms) {
  uint64_t g = ((uint64_t)nch + 7) / 8;
  const uint64_t cap = (uint64_t)num_sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

void launch_hist(const uint16_t* codes, uint32_t N, uint32_t C, uint32_t nch,
                 uint32_t* hist, uint32_t* zc, const Ctl* ctl, int num_sms,
                 cudaStream_t s) {
  static bool attr = false;
  const int smem = kHistWarps * kHistWin * (int)sizeof(uint32_t);
  if (!attr) {
    cudaFuncSetAttribute(k_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  k_hist<<<warps_grid(nch, num_sms), 256, smem, s>>>(codes, N, C, nch, hist, zc,
                                                     ctl);
}

void launch_codebook(const uint32_t* hist, unsigned long long* enc,
                     uint16_t* tsyms, uint8_t* tlens, unsigned long long* gkeys,
                     unsigned long long* giw, uint32_t* gpar,
                     uint8_t* lens_by_sym, Ctl* ctl, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kCodebookSmem);
    cudaFuncSetAttribute(k_dec_tables,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kSmemLeaves * 8));
    attr = true;
  }
  k_codebook<<<1, 1024, kCodebookSmem, s>>>(hist, enc, tsyms, tlens, gkeys, giw,
                                            gpar, lens_by_sym, ctl);
}

void launch_enc_len(const uint16_t* codes, uint32_t N, uint32_t C,
                    uint32_t nch, const unsigned long long* enc,
                    uint16_t* lanebits, uint32_t* chw, const Ctl* ctl,
                    int num_sms, cudaStream_t s) {
  k_enc_len<<<warps_grid(nch, num_sms), 256, 0, s>>>(codes, N, C, nch, enc,
                                                     lanebits, chw, ctl);
}

void launch_pack(const uint16_t* codes, uint32_t N, uint32_t C, uint32_t nch,
                 const unsigned long long* enc, const uint16_t* lanebits,
                 const uint32_t* chw, const unsigned long long* woff,
                 uint8_t* out, const Ctl* ctl, int num_sms, cudaStream_t s) {
  k_pack<<<warps_grid(nch, num_sms), 256, 0, s>>>(codes, N, C, nch, enc,
                                                  lanebits, chw, woff, out, ctl);
}

void launch_encode(const uint16_t* codes, uint32_t N, uint32_t C, uint32_t nch,
                   const unsigned long long* enc, uint16_t* lanebits,
                   unsigned long long* flags, uint8_t* out, Ctl* ctl,
                   unsigned long long cap, int num_sms, cudaStream_t s) {
  // flags[0, nch) and the chunk counter (the word after them) start at 0
  cudaMemsetAsync(flags, 0, sizeof(unsigned long long) * ((size_t)nch + 1), s);
  uint32_t* counter = reinterpret_cast<uint32_t*>(flags + nch);
  // a CTA per chunk with the codes in shared memory, as many CTAs as fit.
  // C is a power of two in [256, 32768] (checked with the config: at most
  // 64 KB of codes to stage) and the code array starts on a 256-byte
  // boundary, so every chunk starts on a 16-byte one
  const int smem = (int)(C * sizeof(uint16_t));
  static int attr_smem = 0;
  if (smem > 48 * 1024 && smem > attr_smem) {
    cudaFuncSetAttribute(k_encode_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr_smem = smem;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_encode_staged, kEncWarps * 32, smem);
  if (per_sm < 1) per_sm = 1;
  uint64_t g = (uint64_t)per_sm * num_sms;
  if (g > nch) g = nch;
  if (g < 1) g = 1;
  k_encode_staged<<<(unsigned)g, kEncWarps * 32, smem, s>>>(codes, N, C, nch, enc, lanebits,
                                                            flags, counter, out, ctl, cap);
}

void launch_chunk_words(const uint8_t* lanebits_bytes, uint32_t nch,
                        uint32_t* chw, int num_sms, cudaStream_t s) {
  unsigned g = (nch + 255) / 256;
  if (g < 1) g = 1;
  if (g > (unsigned)num_sms * 8) g = num_sms * 8;
  k_chunk_words<<<g, 256, 0, s>>>(lanebits_bytes, nch, chw);
}

void launch_outliers(bool gather, const uint16_t* codes, uint32_t N,
                     uint32_t C, uint32_t nch, const uint32_t* zc,
                     const unsigned long long* zoff, const float* src,
                     float* dst, uint8_t* stream, unsigned long long max_out,
                     Ctl* ctl, int num_sms, cudaStream_t s) {
  k_outliers<<<nch, 256, 0, s>>>(gather, codes, N, C, nch, zc, zoff, src, dst,
                                 stream, max_out, ctl);
}

void launch_dec_tables(const uint8_t* stream, uint32_t n_used,
                       uint64_t off_table, uint32_t* lut, uint32_t* cnt,
                       unsigned long long* first, uint32_t* offs,
                       uint16_t* sorted, unsigned long long* gkeys, Ctl* ctl,
                       cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dec_tables,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kSmemLeaves * 8));
    attr = true;
  }
  k_dec_tables<<<1, 1024, kSmemLeaves * 8, s>>>(stream, n_used, off_table, lut,
                                                cnt, first, offs, sorted, gkeys,
                                                ctl);
}

void launch_decode(const uint8_t* stream, uint64_t off_bits,
                   uint64_t total_words, const uint8_t* lanebits_bytes,
                   const unsigned long long* woff, uint32_t N, uint32_t C,
                   uint32_t nch, uint32_t n_used, uint16_t single_sym,
                   const uint32_t* lut, const uint32_t* cnt,
                   const unsigned long long* first, const uint32_t* offs,
                   const uint16_t* sorted, uint16_t* codes, uint32_t* zc,
                   Ctl* ctl, int num_sms, cudaStream_t s, const uint8_t* single_src) {
  k_decode<<<warps_grid(nch, num_sms * 2), 256, 0, s>>>(
      stream, off_bits, total_words, lanebits_bytes, woff, N, C, nch, n_used,
      single_sym, lut, cnt, first, offs, sorted, codes, zc, ctl, single_src);
}

// ---------------------------------------------------------------------
// batched launchers (block counts per job: the *_blocks helpers)
// ---------------------------------------------------------------------
uint32_t hist_blocks(uint32_t nch, int num_sms) { return warps_grid(nch, num_sms); }
uint32_t enc_blocks(uint32_t nch, int num_sms) { return warps_grid(nch, num_sms); }
uint32_t decode_blocks(uint32_t nch, int num_sms) {
  return warps_grid(nch, num_sms * 2);
}
uint32_t chunk_words_blocks(uint32_t nch, int num_sms) {
  unsigned g = (nch + 255) / 256;
  if (g < 1) g = 1;
  if (g > (unsigned)num_sms * 8) g = num_sms * 8;
  return g;
}

void launch_hist_batch(const HistJob* J, const uint32_t* off, int nj,
                       uint32_t nblk, cudaStream_t s) {
  static bool attr = false;
  const int smem = kHistWarps * kHistWin * (int)sizeof(uint32_t);
  if (!attr) {
    cudaFuncSetAttribute(k_hist_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    attr = true;
  }
  if (nblk) k_hist_batch<<<nblk, 256, smem, s>>>(J, off, nj);
}

void launch_codebook_batch(const CodebookJob* J, int nj, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_codebook_batch,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kCodebookSmem);
    attr = true;
  }
  if (nj > 0) k_codebook_batch<<<nj, 1024, kCodebookSmem, s>>>(J);
}

void launch_hcost_batch(const CodebookJob* J, int nj, unsigned long long* cost,
                        cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_hcost_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kCodebookSmem);
    attr = true;
  }
  if (nj > 0) k_hcost_batch<<<nj, 1024, kCodebookSmem, s>>>(J, cost);
}

void launch_enc_len_batch(const EncLenJob* J, const uint32_t* off, int nj,
                          uint32_t nblk, cudaStream_t s) {
  if (nblk) k_enc_len_batch<<<nblk, 256, 0, s>>>(J, off, nj);
}

void launch_pack_batch(const PackJob* J, const uint32_t* off, int nj,
                       uint32_t nblk, cudaStream_t s) {
  if (nblk) k_pack_batch<<<nblk, 256, 0, s>>>(J, off, nj);
}

void launch_chunk_words_batch(const ChunkWordsJob* J, const uint32_t* off,
                              int nj, uint32_t nblk, cudaStream_t s) {
  if (nblk) k_chunk_words_batch<<<nblk, 256, 0, s>>>(J, off, nj);
}

void launch_outliers_batch(const OutlierJob* J, const uint32_t* off, int nj,
                           uint32_t nblk, cudaStream_t s) {
  if (nblk) k_outliers_batch<<<nblk, 256, 0, s>>>(J, off, nj);
}

void launch_dec_tables_batch(const DecTablesJob* J, int nj, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dec_tables_batch,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kSmemLeaves * 8));
    attr = true;
  }
  if (nj > 0) k_dec_tables_batch<<<nj, 1024, kSmemLeaves * 8, s>>>(J);
}

void launch_decode_batch(const DecodeJob* J, const uint32_t* off, int nj,
                         uint32_t nblk, cudaStream_t s) {
  if (nblk) k_decode_batch<<<nblk, 256, 0, s>>>(J, off, nj);
}

}  // namespace hpez
