// Beam splitters (Results, "Towards large-scale discovery", and Methods, "The large-scale search
// space": beam splitters with a continuous ratio in [0, 1] connect the paths of the optical
// table; the optimiser can switch a path off by driving a ratio to 0 or 1).
// Reading: lossless and non-polarising, R the reflected intensity fraction, t = sqrt(1 - R),
// r = sqrt(R), the reflected amplitude carrying the factor i:
//   out_t = t a + i r b,  out_r = i r a + t b          (the same on every component),
// adjoint g_a = t g_t - i r g_r, g_b = -i r g_t + t g_r, and
//   dL/dR = Re sum conj(g_t) (dt a + i dr b) + conj(g_r) (i dr a + dt b),
//   dt = -1 / (2 t), dr = 1 / (2 r).
// Element-wise and bandwidth-bound: each pixel is read and written once per call.
#include <cmath>

#include "xl_runtime.h"

namespace xl {
namespace {

constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_bs_fwd(const cplx<T>* __restrict__ a, const cplx<T>* __restrict__ b,
                                                     cplx<T>* __restrict__ out_t, cplx<T>* __restrict__ out_r,
                                                     int64_t n, const double* __restrict__ R) {
  typedef cplx<T> C;
  const int e = blockIdx.y;
  const double Rd = R[e];
  const T t = (T)sqrt(1.0 - Rd), r = (T)sqrt(Rd);
  const int64_t base = (int64_t)e * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const C av = a ? a[base + i] : mk((T)0, (T)0);
    const C bv = b ? b[base + i] : mk((T)0, (T)0);
    // i r x = (-r x.y, r x.x)
    if (out_t) out_t[base + i] = mk(t * av.x - r * bv.y, t * av.y + r * bv.x);
    if (out_r) out_r[base + i] = mk(t * bv.x - r * av.y, t * bv.y + r * av.x);
  }
}

__device__ __forceinline__ double warp_block_sum(double v, double* sbuf) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sbuf[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) s += sbuf[i];
  return s;
}

// dR partials: part[e][blockIdx.x] (reduced afterwards in fixed order).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bs_bwd(const cplx<T>* __restrict__ g_t, const cplx<T>* __restrict__ g_r,
                                                     const cplx<T>* __restrict__ a, const cplx<T>* __restrict__ b,
                                                     cplx<T>* __restrict__ g_a, cplx<T>* __restrict__ g_b,
                                                     double* __restrict__ part, int64_t n,
                                                     const double* __restrict__ R) {
  typedef cplx<T> C;
  __shared__ double sbuf[kThreads / 32];
  const int e = blockIdx.y;
  const double Rd = R[e];
  const double td = sqrt(1.0 - Rd), rd = sqrt(Rd);
  const T t = (T)td, r = (T)rd;
  const T dt = (T)(-0.5 / td), dr = (T)(0.5 / rd);
  const int64_t base = (int64_t)e * n;
  // per-thread sums in T (a few tens of terms), the block and batch sums in double
  T acc = (T)0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const C gt = g_t ? g_t[base + i] : mk((T)0, (T)0);
    const C gr = g_r ? g_r[base + i] : mk((T)0, (T)0);
    // -i r x = (r x.y, -r x.x)
    if (g_a) g_a[base + i] = mk(t * gt.x + r * gr.y, t * gt.y - r * gr.x);
    if (g_b) g_b[base + i] = mk(t * gr.x + r * gt.y, t * gr.y - r * gt.x);
    if (part) {
      const C av = a ? a[base + i] : mk((T)0, (T)0);
      const C bv = b ? b[base + i] : mk((T)0, (T)0);
      const C dot = mk(dt * av.x - dr * bv.y, dt * av.y + dr * bv.x);   // dt a + i dr b
      const C dor = mk(dt * bv.x - dr * av.y, dt * bv.y + dr * av.x);   // i dr a + dt b
      acc += (gt.x * dot.x + gt.y * dot.y) + (gr.x * dor.x + gr.y * dor.y);
    }
  }
  if (part) {
    const double s = warp_block_sum((double)acc, sbuf);
    if (threadIdx.x == 0) part[(int64_t)e * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_bs_reduce(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  __shared__ double sbuf[kThreads / 32];
  const int e = blockIdx.x;
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) s += part[(int64_t)e * nblk + k];
  s = warp_block_sum(s, sbuf);
  if (threadIdx.x == 0) out[e] = s;
}

int blocks_for(int64_t n) {
  const int64_t per = (int64_t)kThreads * 4;  // about four elements per thread
  int64_t nb = (n + per - 1) / per;
  if (nb < 1) nb = 1;
  if (nb > 1024) nb = 1024;
  return (int)nb;
}

xl_status check(int32_t batch, int64_t n, const double* R, int32_t dtype) {
  if (batch < 0 || n < 0) return fail(XL_ERR_ARG, "batch and elems must be >= 0");
  if (batch > 65535) return fail(XL_ERR_UNSUPPORTED, "batch > 65535");
  if (dtype != XL_C64 && dtype != XL_C128) return fail(XL_ERR_ARG, "dtype must be XL_C64 or XL_C128");
  if (batch > 0 && n > 0 && !R) return fail(XL_ERR_ARG, "R is NULL");
  return XL_OK;
}

template <typename T>
xl_status fwd(const void* a, const void* b, void* ot, void* orr, int32_t batch, int64_t n,
              const double* R, cudaStream_t s) {
  typedef cplx<T> C;
  LaunchScope ls("beam_splitter", s);
  k_bs_fwd<T><<<dim3(blocks_for(n), batch), kThreads, 0, s>>>((const C*)a, (const C*)b, (C*)ot, (C*)orr, n, R);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

template <typename T>
xl_status bwd(const void* gt, const void* gr, const void* a, const void* b, void* ga, void* gb,
              double* gR, int32_t batch, int64_t n, const double* R, cudaStream_t s) {
  typedef cplx<T> C;
  const int nblk = blocks_for(n);
  double* part = nullptr;
  if (gR) {
    void* ws = nullptr;
    XL_TRY(workspace(s, (size_t)batch * nblk * sizeof(double), &ws, 2));
    part = (double*)ws;
  }
  {
    LaunchScope ls("beam_splitter_bwd", s);
    k_bs_bwd<T><<<dim3(nblk, batch), kThreads, 0, s>>>((const C*)gt, (const C*)gr, (const C*)a, (const C*)b,
                                                        (C*)ga, (C*)gb, part, n, R);
    XL_CUDA_TRY(cudaGetLastError());
  }
  if (gR) {
    LaunchScope ls("beam_splitter_reduce", s);
    k_bs_reduce<<<batch, kThreads, 0, s>>>(part, nblk, gR);
    XL_CUDA_TRY(cudaGetLastError());
  }
  return XL_OK;
}

}  // namespace
}  // namespace xl

using namespace xl;

extern "C" {

xl_status xl_beam_splitter(const void* a, const void* b, void* out_t, void* out_r, int32_t batch,
                           int64_t elems, const double* R, int32_t dtype, void* stream) {
  XL_TRY(check(batch, elems, R, dtype));
  if (batch == 0 || elems == 0 || (!out_t && !out_r)) return XL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == XL_C128) return fwd<double>(a, b, out_t, out_r, batch, elems, R, s);
  return fwd<float>(a, b, out_t, out_r, batch, elems, R, s);
}

xl_status xl_beam_splitter_backward(const void* g_t, const void* g_r, const void* a, const void* b,
                                    void* g_a, void* g_b, double* g_R, int32_t batch, int64_t elems,
                                    const double* R, int32_t dtype, void* stream) {
  XL_TRY(check(batch, elems, R, dtype));
  if (batch == 0) return XL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (elems == 0) {
    if (g_R) XL_CUDA_TRY(cudaMemsetAsync(g_R, 0, (size_t)batch * sizeof(double), s));
    return XL_OK;
  }
  if (!g_a && !g_b && !g_R) return XL_OK;
  if (dtype == XL_C128) return bwd<double>(g_t, g_r, a, b, g_a, g_b, g_R, batch, elems, R, s);
  return bwd<float>(g_t, g_r, a, b, g_a, g_b, g_R, batch, elems, R, s);
}

}  // extern "C"
