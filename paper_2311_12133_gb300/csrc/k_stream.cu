// k_stream.cu -- prefix scans and assembly of the compressed container.
//
// Container (little-endian): a 512-byte header, then 16-byte aligned
// sections: anchors (f32, compact anchor grid in row-major order), block
// map (u8 per block, optional),
// lane bit counts (u16, 32 per chunk), code table (u16 symbols ascending,
// then u8 lengths), outliers (f32, row-major order of their points),
// bitstream (u32 words).  Padding bytes are zero.
#include "hpez_internal.cuh"
#include "hpez_launch.h"

namespace hpez {

// exclusive scan of n u32 values into u64, single CTA of 1024 threads;
// *total receives the sum
__device__ __forceinline__ void scan_body(const uint32_t* __restrict__ in,
                                          unsigned long long* __restrict__ out,
                                          uint32_t n, unsigned long long* total,
                                          const Ctl* __restrict__ ctl) {
  if (ctl->status || ctl->is_const) return;
  __shared__ unsigned long long warp_sums[32];
  __shared__ unsigned long long carry;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += blockDim.x * 8u) {
    // each thread owns 8 consecutive values of this tile
    unsigned long long v[8], s = 0;
    const uint32_t i0 = base + tid * 8u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v[k] = (i0 + k < n) ? in[i0 + k] : 0u;
      s += v[k];
    }
    unsigned long long x = s;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned long long t = warp_sums[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_sums[lane] = t;
    }
    __syncthreads();
    unsigned long long run = carry + (w ? warp_sums[w - 1] : 0) + x - s;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (i0 + k < n) out[i0 + k] = run;
      run += v[k];
    }
    __syncthreads();
    if (tid == 0) carry += warp_sums[31];
    __syncthreads();
  }
  if (tid == 0) *total = carry;
}

__global__ void __launch_bounds__(1024)
    k_scan(const uint32_t* __restrict__ in, unsigned long long* __restrict__ out,
           uint32_t n, unsigned long long* total, const Ctl* __restrict__ ctl) {
  scan_body(in, out, n, total, ctl);
}

__host__ __device__ inline unsigned long long align16(unsigned long long v) {
  return (v + 15ull) & ~15ull;
}

// dynamic section offsets + capacity check
__device__ __forceinline__ void layout_body(Ctl* ctl,
                                            unsigned long long off_table,
                                            unsigned long long cap) {
  if (threadIdx.x != 0 || ctl->status) return;
  if (ctl->is_const) {
    ctl->total_size = kHeaderBytes;
    if (cap < (unsigned long long)kHeaderBytes) ctl->status = ST_OUT_TOO_SMALL;
    return;
  }
  ctl->off_table = off_table;
  ctl->off_outliers = align16(off_table + 3ull * ctl->n_used);
  ctl->off_bits = align16(ctl->off_outliers + 4ull * ctl->n_out);
  ctl->total_size = ctl->off_bits + 4ull * ctl->total_words;
  if (ctl->total_size > cap) ctl->status = ST_OUT_TOO_SMALL;
}

__global__ void k_layout(Ctl* ctl, unsigned long long off_table,
                         unsigned long long cap) {
  layout_body(ctl, off_table, cap);
}

struct HeaderImage {
  uint8_t b[kHeaderBytes];
};

__device__ inline void put_u32(uint8_t* p, uint32_t v) {
  p[0] = (uint8_t)v;
  p[1] = (uint8_t)(v >> 8);
  p[2] = (uint8_t)(v >> 16);
  p[3] = (uint8_t)(v >> 24);
}
__device__ inline void put_u64(uint8_t* p, unsigned long long v) {
  for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i));
}

// header byte offsets patched on the device
constexpr int kHE = 56, kHConst = 60, kHNOut = 224, kHNUsed = 232,
              kHTotalWords = 248, kHOffTable = 272, kHOffOutliers = 280,
              kHOffBits = 288, kHTotal = 304;

// Writes the header and the static-size sections; pads every section end
// with zeros up to the next 16-byte boundary.
__device__ __forceinline__ void finalize_body(
    const uint8_t* hdr, const uint8_t* hdr_const, uint8_t* __restrict__ out,
    const float* __restrict__ RA, uint32_t na, unsigned long long off_anchors,
    const uint8_t* __restrict__ bmap, uint32_t nblocks,
    unsigned long long off_bmap, const uint16_t* __restrict__ lanebits,
    uint32_t nch, unsigned long long off_chw, const uint16_t* __restrict__ tsyms,
    const uint8_t* __restrict__ tlens, const Ctl* __restrict__ ctl,
    unsigned bid, unsigned nblk) {
  if (ctl->status) return;
  const uint32_t tid = bid * blockDim.x + threadIdx.x;
  const uint32_t nthr = nblk * blockDim.x;
  if (ctl->is_const) {
    for (uint32_t i = tid; i < (uint32_t)kHeaderBytes; i += nthr) {
      uint8_t v = hdr_const[i];
      if (i >= kHConst && i < kHConst + 4)
        v = (uint8_t)(__float_as_uint(ctl->const_value) >> (8 * (i - kHConst)));
      out[i] = v;
    }
    return;
  }
  if (tid == 0) {
    uint8_t h[kHeaderBytes];
    for (int i = 0; i < kHeaderBytes; ++i) h[i] = hdr[i];
    put_u32(h + kHE, __float_as_uint(ctl->e));
    put_u64(h + kHNOut, ctl->n_out);
    put_u32(h + kHNUsed, ctl->n_used);
    put_u64(h + kHTotalWords, ctl->total_words);
    put_u64(h + kHOffTable, ctl->off_table);
    put_u64(h + kHOffOutliers, ctl->off_outliers);
    put_u64(h + kHOffBits, ctl->off_bits);
    put_u64(h + kHTotal, ctl->total_size);
    for (int i = 0; i < kHeaderBytes; i += 4)
      *reinterpret_cast<uint32_t*>(out + i) =
          (uint32_t)h[i] | ((uint32_t)h[i + 1] << 8) |
          ((uint32_t)h[i + 2] << 16) | ((uint32_t)h[i + 3] << 24);
  }
  // anchors
  float* fa = reinterpret_cast<float*>(out + off_anchors);
  for (uint32_t i = tid; i < na; i += nthr) fa[i] = RA[i];
  // block map
  for (uint32_t i = tid; i < nblocks; i += nthr) out[off_bmap + i] = bmap[i];
  // lane bit counts (32 per chunk)
  uint32_t* fc = reinterpret_cast<uint32_t*>(out + off_chw);
  const uint32_t* lb32 = reinterpret_cast<const uint32_t*>(lanebits);
  for (uint32_t i = tid; i < 16u * nch; i += nthr) fc[i] = lb32[i];
  // code table: symbols then lengths
  const uint32_t nu = ctl->n_used;
  const unsigned long long ot = ctl->off_table;
  for (uint32_t k = tid; k < nu; k += nthr) {
    const uint16_t sy = tsyms[k];
    out[ot + 2ull * k] = (uint8_t)sy;
    out[ot + 2ull * k + 1] = (uint8_t)(sy >> 8);
    out[ot + 2ull * nu + k] = tlens[k];
  }
  // zero padding at the end of each section
  const unsigned long long ends[5] = {off_anchors + 4ull * na,
                                      off_bmap + nblocks, off_chw + 64ull * nch,
                                      ot + 3ull * nu,
                                      ctl->off_outliers + 4ull * ctl->n_out};
  if (tid < 5) {
    for (unsigned long long p = ends[tid]; p < align16(ends[tid]); ++p) out[p] = 0;
  }
}

__global__ void k_finalize(HeaderImage hdr, HeaderImage hdr_const,
                           uint8_t* __restrict__ out,
                           const float* __restrict__ RA, uint32_t na,
                           unsigned long long off_anchors,
                           const uint8_t* __restrict__ bmap, uint32_t nblocks,
                           unsigned long long off_bmap,
                           const uint16_t* __restrict__ lanebits,
                           uint32_t nch, unsigned long long off_chw,
                           const uint16_t* __restrict__ tsyms,
                           const uint8_t* __restrict__ tlens,
                           const Ctl* __restrict__ ctl) {
  finalize_body(hdr.b, hdr_const.b, out, RA, na, off_anchors, bmap, nblocks,
                off_bmap, lanebits, nch, off_chw, tsyms, tlens, ctl, blockIdx.x,
                gridDim.x);
}

// ---------------------------------------------------------------------
// batched forms
// ---------------------------------------------------------------------
// Per request: the device status (its values equal the C-ABI error codes)
// and, for compress, the stream size; decompress also checks that the
// decoded word and outlier counts match the header.
__device__ __forceinline__ void result_body(const ResultJob& q) {
  int st = q.ctl->status;
  unsigned long long size = 0;
  if (!q.decomp) {
    size = st ? 0ull : q.ctl->total_size;
  } else if (!st && q.tot && (q.tot[0] != q.twords || q.tot[1] != q.nout)) {
    st = ST_CORRUPT;
  }
  if (q.size_out) *q.size_out = size;
  if (q.status_out) *q.status_out = st;
}

__global__ void k_result_batch(const ResultJob* __restrict__ J, int nj) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nj) return;
  result_body(J[j]);
}

__global__ void k_result_one(ResultJob q) { result_body(q); }

__global__ void __launch_bounds__(1024) k_scan_batch(const ScanJob* __restrict__ J) {
  const ScanJob& q = J[blockIdx.x];
  scan_body(q.in, q.out, q.n, q.total, q.ctl);
}

__global__ void k_layout_batch(const LayoutJob* __restrict__ J) {
  layout_body(J[blockIdx.x].ctl, J[blockIdx.x].off_table, J[blockIdx.x].cap);
}

__global__ void k_finalize_batch(const FinalizeJob* __restrict__ J,
                                 const uint32_t* __restrict__ off, int nj) {
  const int j = batch_job(off, nj);
  const FinalizeJob& q = J[j];
  finalize_body(q.hdr, q.hdr_const, q.out, q.RA, q.na, q.off_anchors, q.bmap,
                q.nblocks, q.off_bmap, q.lanebits, q.nch, q.off_chw, q.tsyms,
                q.tlens, q.ctl, blockIdx.x - off[j], off[j + 1] - off[j]);
}

// ---------------------------------------------------------------------
void launch_scan(const uint32_t* in, unsigned long long* out, uint32_t n,
                 unsigned long long* total, const Ctl* ctl, cudaStream_t s) {
  k_scan<<<1, 1024, 0, s>>>(in, out, n, total, ctl);
}

void launch_layout(Ctl* ctl, unsigned long long off_table,
                   unsigned long long cap, cudaStream_t s) {
  k_layout<<<1, 32, 0, s>>>(ctl, off_table, cap);
}

void launch_finalize(const uint8_t* hdr, const uint8_t* hdr_const,
                     uint8_t* out, const float* RA, uint32_t na,
                     unsigned long long off_anchors, const uint8_t* bmap,
                     uint32_t nblocks, unsigned long long off_bmap,
                     const uint16_t* lanebits, uint32_t nch,
                     unsigned long long off_chw, const uint16_t* tsyms,
                     const uint8_t* tlens, const Ctl* ctl, int num_sms,
                     cudaStream_t s) {
  HeaderImage h, hc;
  for (int i = 0; i < kHeaderBytes; ++i) {
    h.b[i] = hdr[i];
    hc.b[i] = hdr_const[i];
  }
  uint64_t work = na;
  if (16ull * nch > work) work = 16ull * nch;
  unsigned grid = (unsigned)((work + 255) / 256);
  if (grid < 1) grid = 1;
  if (grid > (unsigned)num_sms * 4) grid = num_sms * 4;
  k_finalize<<<grid, 256, 0, s>>>(h, hc, out, RA, na, off_anchors, bmap,
                                  nblocks, off_bmap, lanebits, nch, off_chw, tsyms,
                                  tlens, ctl);
}

void launch_result_batch(const ResultJob* J, int nj, cudaStream_t s) {
  if (nj > 0) k_result_batch<<<(nj + 127) / 128, 128, 0, s>>>(J, nj);
}

void launch_result_one(const ResultJob& J, cudaStream_t s) { k_result_one<<<1, 1, 0, s>>>(J); }

void launch_scan_batch(const ScanJob* J, int nj, cudaStream_t s) {
  if (nj > 0) k_scan_batch<<<nj, 1024, 0, s>>>(J);
}

void launch_layout_batch(const LayoutJob* J, int nj, cudaStream_t s) {
  if (nj > 0) k_layout_batch<<<nj, 32, 0, s>>>(J);
}

void launch_finalize_batch(const FinalizeJob* J, const uint32_t* off, int nj,
                           uint32_t nblk, cudaStream_t s) {
  if (nblk) k_finalize_batch<<<nblk, 256, 0, s>>>(J, off, nj);
}

// blocks the single-field finalize would use
uint32_t finalize_blocks(uint32_t na, uint32_t nch, int num_sms) {
  uint64_t work = na;
  if (16ull * nch > work) work = 16ull * nch;
  unsigned grid = (unsigned)((work + 255) / 256);
  if (grid < 1) grid = 1;
  if (grid > (unsigned)num_sms * 4) grid = num_sms * 4;
  return grid;
}

}  // namespace hpez
