// hpez_typed.cu -- the quality-metric target (Sec. 3.1, Eq. 1 with M =
// PSNR) and integer inputs, declared in include/hpez.h.
//
// Both sit on top of the compressor: hpez_psnr is a device reduction of the
// squared errors in a fixed-point unit (an exact integer sum, so its value
// does not depend on the reduction order), hpez_compress_psnr searches the
// absolute bound on the host with auto-tuned round trips on the device, and
// the typed calls widen integer fields to binary32 on the device, compress
// them at the float bound just below floor(e) + 1/2, and round back to the
// nearest integer on decompression.
#include <cmath>
#include <cstring>

#include "hpez.h"
#include "hpez_ctx.h"
#include "hpez_internal.cuh"
#include "hpez_launch.h"

using namespace hpez;
using namespace hpez::host;

namespace {

constexpr int kHdrDtype = 320;  // header byte of the input type
constexpr int kRedThreads = 256;

// reduction words: [0] sum of q^2, [1] bad flag, [2] min key, [3] max key
struct Red {
  unsigned long long sse;
  unsigned int bad;
  unsigned int kmin, kmax;
  int imin, imax;
  unsigned int pad;
};

__device__ __forceinline__ void red_minmax_key(Red* r, unsigned kmin, unsigned kmax) {
  for (int o = 16; o > 0; o >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(0xFFFFFFFFu, kmin, o));
    kmax = max(kmax, __shfl_xor_sync(0xFFFFFFFFu, kmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&r->kmin, kmin);
    atomicMax(&r->kmax, kmax);
  }
}

// Sum of q_i^2, q_i = rint((x_i - y_i) / unit) in double, with the value
// range of x (order-preserving keys); bad: 1 a non-finite x, 2 |q| > 2^16.
__global__ void __launch_bounds__(kRedThreads)
    k_sse_fixed(const float* __restrict__ x, const float* __restrict__ y, uint64_t n,
                double unit, Red* r) {
  unsigned long long acc = 0;
  unsigned kmin = 0xFFFFFFFFu, kmax = 0u;
  bool bad = false, nonfin = false;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const float xv = x[i];
    if (!isfinite(xv)) nonfin = true;
    const double q = rint(((double)xv - (double)y[i]) / unit);
    if (!(fabs(q) <= 65536.0)) {
      bad = true;
    } else {
      const long long iq = (long long)q;
      acc += (unsigned long long)(iq * iq);
    }
    const unsigned k = f2key(xv);
    kmin = min(kmin, k);
    kmax = max(kmax, k);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&r->sse, acc);
  const bool wb = __any_sync(0xFFFFFFFFu, bad), wn = __any_sync(0xFFFFFFFFu, nonfin);
  if ((threadIdx.x & 31) == 0 && (wb || wn)) atomicOr(&r->bad, (wn ? 1u : 0u) | (wb ? 2u : 0u));
  red_minmax_key(r, kmin, kmax);
}

// integer -> binary32 (exact for |v| <= 2^24) with the integer range; bad:
// an int32 beyond 2^24
template <class T>
__global__ void __launch_bounds__(kRedThreads)
    k_widen(const T* __restrict__ in, float* __restrict__ out, uint64_t n, Red* r) {
  int vmin = 0x7FFFFFFF, vmax = (int)0x80000000;
  bool bad = false;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const int v = (int)in[i];
    if (v > (1 << 24) || v < -(1 << 24)) bad = true;
    out[i] = (float)v;
    vmin = min(vmin, v);
    vmax = max(vmax, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    vmin = min(vmin, __shfl_xor_sync(0xFFFFFFFFu, vmin, o));
    vmax = max(vmax, __shfl_xor_sync(0xFFFFFFFFu, vmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&r->imin, vmin);
    atomicMax(&r->imax, vmax);
  }
  if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicExch(&r->bad, 1u);
}

// binary32 -> integer: nearest (ties to even), clamped to the type's range
template <class T>
__global__ void __launch_bounds__(kRedThreads)
    k_narrow(const float* __restrict__ in, T* __restrict__ out, uint64_t n, float lo, float hi) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const float v = fminf(fmaxf(rintf(in[i]), lo), hi);
    out[i] = (T)v;
  }
}

__global__ void k_red_init(Red* r) {
  r->sse = 0;
  r->bad = 0;
  r->kmin = 0xFFFFFFFFu;
  r->kmax = 0u;
  r->imin = 0x7FFFFFFF;
  r->imax = (int)0x80000000;
}

unsigned grid_for(const hpez_ctx* ctx, uint64_t n) {
  const uint64_t want = (n + kRedThreads - 1) / kRedThreads;
  const uint64_t cap = (uint64_t)ctx->num_sms * 8;
  return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

int ensure_typed(hpez_ctx* ctx, uint64_t n) {
  if (!ctx->typed_red && cudaMalloc(&ctx->typed_red, 256) != cudaSuccess) {
    cudaGetLastError();
    ctx->typed_red = nullptr;
    return HPEZ_ERR_NO_MEMORY;
  }
  return ensure_io(&ctx->typed_buf, &ctx->typed_cap, (size_t)n * sizeof(float));
}

float key_value(unsigned k) {
  const unsigned u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// PSNR from the fixed-point sum, in the oracle's formula and order
double psnr_of(unsigned long long sse, double unit, uint64_t n, double vmin, double vmax) {
  if (sse == 0) return INFINITY;
  const double mse = (double)sse * unit * unit / (double)n;
  return 20.0 * std::log10(vmax - vmin) - 10.0 * std::log10(mse);
}

int dtype_ok(int dtype) {
  return dtype == HPEZ_DTYPE_F32 || dtype == HPEZ_DTYPE_I16 || dtype == HPEZ_DTYPE_U16 ||
         dtype == HPEZ_DTYPE_I32;
}

uint64_t count(int ndim, const uint64_t* dims) {
  uint64_t n = 1;
  for (int d = 0; d < ndim; ++d) n *= dims[d];
  return n;
}

}  // namespace

int hpez_psnr(hpez_ctx* ctx, const float* d_x, const float* d_y, uint64_t n, double unit,
              double* h_psnr, uint64_t* h_sse, void* stream) {
  if (!ctx || !d_x || !d_y || n == 0 || !(unit > 0.0) || !std::isfinite(unit))
    return HPEZ_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = ensure_typed(ctx, 1);
  if (rc) return rc;
  Red* r = static_cast<Red*>(ctx->typed_red);
  k_red_init<<<1, 1, 0, s>>>(r);
  k_sse_fixed<<<grid_for(ctx, n), kRedThreads, 0, s>>>(d_x, d_y, n, unit, r);
  ctx->launches += 2;
  Red h;
  rc = cuda_check(cudaMemcpyAsync(&h, r, sizeof(Red), cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc) return rc;
  if (h.bad & 1u) return HPEZ_ERR_NONFINITE_INPUT;
  if (h.bad) return HPEZ_ERR_INVALID_ARG;
  if (h_sse) *h_sse = h.sse;
  if (h_psnr)
    *h_psnr = psnr_of(h.sse, unit, n, (double)key_value(h.kmin), (double)key_value(h.kmax));
  return HPEZ_OK;
}

namespace {

// one probe of the bound search: tune + compress at absolute bound e into
// d_out, decompress into the context's staging, PSNR in the unit of the
// stored bound
int probe_psnr(hpez_ctx* ctx, const float* d_in, int ndim, const uint64_t* dims, uint64_t n,
               double e, const hpez_tune_params* tp, void* d_out, uint64_t cap,
               uint64_t* size, double* psnr, cudaStream_t s) {
  int rc = hpez_compress_auto(ctx, d_in, ndim, dims, HPEZ_EB_ABS, e, tp, d_out, cap, size,
                              nullptr, s);
  if (rc) return rc;
  float* y = static_cast<float*>(ctx->typed_buf);
  rc = hpez_decompress(ctx, d_out, *size, y, n, s);
  if (rc) return rc;
  float ef;
  rc = cuda_check(cudaMemcpyAsync(&ef, static_cast<const uint8_t*>(d_out) + H_E, 4,
                                  cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc) return rc;
  return hpez_psnr(ctx, d_in, y, n, (double)ef / 65536.0, psnr, nullptr, s);
}

}  // namespace

int hpez_compress_psnr(hpez_ctx* ctx, const float* d_in, int ndim, const uint64_t* dims,
                       double target_db, const hpez_tune_params* tp, void* d_out,
                       uint64_t out_cap, uint64_t* h_out_size, double* h_eb, double* h_psnr,
                       void* stream) {
  if (!ctx || !d_in || !d_out || !h_out_size || !dims || ndim < 1 || ndim > 3 ||
      !std::isfinite(target_db))
    return HPEZ_ERR_INVALID_ARG;
  const uint64_t n = count(ndim, dims);
  if (n == 0) return HPEZ_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = ensure_typed(ctx, n);
  if (rc) return rc;
  // the value range (and finiteness) of the input
  Red* r = static_cast<Red*>(ctx->typed_red);
  k_red_init<<<1, 1, 0, s>>>(r);
  k_sse_fixed<<<grid_for(ctx, n), kRedThreads, 0, s>>>(d_in, d_in, n, 1.0, r);
  ctx->launches += 2;
  Red h;
  rc = cuda_check(cudaMemcpyAsync(&h, r, sizeof(Red), cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc) return rc;
  if (h.bad) return HPEZ_ERR_NONFINITE_INPUT;
  const double range = (double)key_value(h.kmax) - (double)key_value(h.kmin);
  // the search (same steps as its definition in the header): from the bound
  // at which uniform errors give the target, double or halve up to 6 times
  // to bracket it, then 8 geometric bisection steps keeping PSNR(lo) >= m0
  double e = range > 0.0 ? range * std::sqrt(3.0) * std::pow(10.0, -target_db / 20.0) : 1.0;
  if (!(e > 0.0) || !std::isfinite(e)) return HPEZ_ERR_INVALID_ARG;
  uint64_t size = 0;
  double ps = 0.0, lo = 0.0, hi = 0.0;
  bool found = false;
  if ((rc = probe_psnr(ctx, d_in, ndim, dims, n, e, tp, d_out, out_cap, &size, &ps, s)))
    return rc;
  if (ps >= target_db) {
    lo = e;
    hi = 2.0 * e;
    found = true;
    int g;
    for (g = 0; g < 6; ++g) {
      if ((rc = probe_psnr(ctx, d_in, ndim, dims, n, hi, tp, d_out, out_cap, &size, &ps, s)))
        return rc;
      if (ps < target_db) break;
      lo = hi;
      hi = 2.0 * hi;
    }
    if (g == 6) hi = 0.0;  // the target holds at every bound tried
  } else {
    hi = e;
    lo = 0.5 * e;
    int g;
    for (g = 0; g < 6; ++g) {
      if ((rc = probe_psnr(ctx, d_in, ndim, dims, n, lo, tp, d_out, out_cap, &size, &ps, s)))
        return rc;
      if (ps >= target_db) break;
      hi = lo;
      lo = 0.5 * lo;
    }
    found = g < 6;
    if (!found) hi = 0.0;
  }
  if (hi > 0.0) {
    for (int it = 0; it < 8; ++it) {
      const double mid = std::sqrt(lo * hi);
      if ((rc = probe_psnr(ctx, d_in, ndim, dims, n, mid, tp, d_out, out_cap, &size, &ps, s)))
        return rc;
      if (ps >= target_db)
        lo = mid;
      else
        hi = mid;
    }
  }
  if (!found) lo = 2.0 * lo;  // the smallest bound tried
  if ((rc = probe_psnr(ctx, d_in, ndim, dims, n, lo, tp, d_out, out_cap, &size, &ps, s)))
    return rc;
  *h_out_size = size;
  if (h_eb) *h_eb = lo;
  if (h_psnr) *h_psnr = ps;
  return HPEZ_OK;
}

int hpez_compress_typed(hpez_ctx* ctx, const void* d_in, int dtype, int ndim,
                        const uint64_t* dims, int eb_mode, double eb, const hpez_config* cfg,
                        int tune, const hpez_tune_params* tp, void* d_out, uint64_t out_cap,
                        uint64_t* h_out_size, void* stream) {
  if (!ctx || !d_in || !d_out || !h_out_size || !dims || ndim < 1 || ndim > 3 ||
      !dtype_ok(dtype))
    return HPEZ_ERR_INVALID_ARG;
  if (eb_mode != HPEZ_EB_ABS && eb_mode != HPEZ_EB_REL) return HPEZ_ERR_INVALID_ARG;
  const uint64_t n = count(ndim, dims);
  if (n == 0) return HPEZ_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float* x = static_cast<const float*>(d_in);
  int mode = eb_mode;
  double e = eb;
  int rc;
  if (dtype != HPEZ_DTYPE_F32) {
    if ((rc = ensure_typed(ctx, n))) return rc;
    Red* r = static_cast<Red*>(ctx->typed_red);
    float* xf = static_cast<float*>(ctx->typed_buf);
    k_red_init<<<1, 1, 0, s>>>(r);
    const unsigned grid = grid_for(ctx, n);
    if (dtype == HPEZ_DTYPE_I16)
      k_widen<int16_t><<<grid, kRedThreads, 0, s>>>(static_cast<const int16_t*>(d_in), xf, n, r);
    else if (dtype == HPEZ_DTYPE_U16)
      k_widen<uint16_t><<<grid, kRedThreads, 0, s>>>(static_cast<const uint16_t*>(d_in), xf, n,
                                                     r);
    else
      k_widen<int32_t><<<grid, kRedThreads, 0, s>>>(static_cast<const int32_t*>(d_in), xf, n, r);
    ctx->launches += 2;
    Red h;
    rc = cuda_check(cudaMemcpyAsync(&h, r, sizeof(Red), cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
    if (rc) return rc;
    if (h.bad) return HPEZ_ERR_INVALID_ARG;
    // the integer bound, and the float bound that keeps the rounded
    // reconstruction within it
    const double ei = eb_mode == HPEZ_EB_REL ? eb * ((double)h.imax - (double)h.imin) : eb;
    if (!(ei >= 0.0) || !std::isfinite(ei) || ei > 4194304.0) return HPEZ_ERR_INVALID_ARG;
    e = (double)std::nextafter((float)(std::floor(ei) + 0.5), 0.0f);
    mode = HPEZ_EB_ABS;
    x = xf;
  }
  if (tune)
    rc = hpez_compress_auto(ctx, x, ndim, dims, mode, e, tp, d_out, out_cap, h_out_size,
                            nullptr, stream);
  else
    rc = hpez_compress(ctx, x, ndim, dims, mode, e, cfg, d_out, out_cap, h_out_size, stream);
  if (rc) return rc;
  if (dtype != HPEZ_DTYPE_F32) {
    const uint32_t dt = (uint32_t)dtype;
    rc = cuda_check(cudaMemcpyAsync(static_cast<uint8_t*>(d_out) + kHdrDtype, &dt, 4,
                                    cudaMemcpyHostToDevice, s));
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  }
  return rc;
}

int hpez_decompress_typed(hpez_ctx* ctx, const void* d_in, uint64_t in_size, void* d_out,
                          int dtype, uint64_t out_cap_elems, void* stream) {
  if (!ctx || !d_in || !d_out || !dtype_ok(dtype)) return HPEZ_ERR_INVALID_ARG;
  if (in_size < (uint64_t)kHeaderBytes) return HPEZ_ERR_CORRUPT_STREAM;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t hdr[kHeaderBytes];
  int rc = cuda_check(cudaMemcpyAsync(hdr, d_in, kHeaderBytes, cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc) return rc;
  if ((int)rd32(hdr, kHdrDtype) != dtype) return HPEZ_ERR_INVALID_ARG;
  int nd;
  uint64_t dims[3];
  if ((rc = hpez_inspect(hdr, kHeaderBytes, &nd, dims, nullptr))) return rc;
  const uint64_t n = count(nd, dims);
  if (n > out_cap_elems) return HPEZ_ERR_OUT_TOO_SMALL;
  if (dtype == HPEZ_DTYPE_F32)
    return hpez_decompress(ctx, d_in, in_size, static_cast<float*>(d_out), out_cap_elems, stream);
  if ((rc = ensure_typed(ctx, n))) return rc;
  float* y = static_cast<float*>(ctx->typed_buf);
  if ((rc = hpez_decompress(ctx, d_in, in_size, y, n, stream))) return rc;
  const unsigned grid = grid_for(ctx, n);
  if (dtype == HPEZ_DTYPE_I16)
    k_narrow<int16_t><<<grid, kRedThreads, 0, s>>>(y, static_cast<int16_t*>(d_out), n, -32768.0f,
                                                  32767.0f);
  else if (dtype == HPEZ_DTYPE_U16)
    k_narrow<uint16_t><<<grid, kRedThreads, 0, s>>>(y, static_cast<uint16_t*>(d_out), n, 0.0f,
                                                   65535.0f);
  else
    k_narrow<int32_t><<<grid, kRedThreads, 0, s>>>(y, static_cast<int32_t*>(d_out), n,
                                                  -2147483520.0f, 2147483520.0f);
  ctx->launches += 1;
  rc = cuda_check(cudaGetLastError());
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s));
  return rc;
}
