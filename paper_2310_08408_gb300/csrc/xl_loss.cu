// Camera intensity and losses with their adjoints (Methods, "Loss function"; the camera
// intensities of the Results: |Ex|^2 + |Ey|^2, |Ez|^2 or the total).
//
//   I = sum over the components selected by comp_mask of |E_c|^2
//   XL_SECOND_MOMENT (reading; the paper's own spot metric is (pi/4) FWHMx FWHMy):
//       P = sum I, xbar = sum I x / P, L = sum I ((x - xbar)^2 + (y - ybar)^2) / P
//   XL_DENSITY (Methods, "Loss function"): threshold eps i_max with a strict ">",
//       L = Area / I_eps (pixel count and intensity sum above the threshold)
// Two sweeps per loss: the first forms (P, sum I x, sum I y) or i_max, the second the centred
// second moment or the thresholded count / sum, so no moment is formed by cancellation. Each
// sweep reduces per block (thread sums in the field's precision, block tree in double) and a
// one-block-per-batch finaliser combines the partials in a fixed order (deterministic).
// Gradient (g = 2 dL/dI E on the selected components):
//   second moment  dL/dI = [(x - xbar)^2 + (y - ybar)^2 - L] / P
//   density        dL/dI = -Area / I_eps^2 above the threshold, 0 elsewhere (no gradient through
//                  i_max or Area, as with a where-based selection).
//   XL_MSE (Results, "Data-driven rediscovery"): L = mean (I - I_target)^2, one sweep.
// Optionally I is the STED effective intensity of an excitation and a depletion field (Methods,
// "Stimulated emission depletion model"), fused into both sweeps and the gradient.
// A non-finite loss sets a device status bit that xl_device_status() reports as
// XL_ERR_NONFINITE.
#include <cmath>

#include "xl_runtime.h"

namespace xl {

__device__ unsigned int g_status_bits = 0;  // bit 0: non-finite loss

constexpr int kLossThreads = 256;

struct LossDims {
  int nx, ny, comps;
  unsigned mask;
  int64_t plane;
  double x0, dx, y0, dy, eps;
  int mode;
  const void* dep;     // depletion field (STED effective intensity) or nullptr
  double beta;         // STED quenching efficiency
  const void* target;  // MSE target intensity [batch][ny][nx] (real) or nullptr
};

// NC: the field's component count (1..3), a compile-time constant so that the component loop
// unrolls and the loads of consecutive pixels can be in flight together.
template <typename T, int NC>
__device__ __forceinline__ T intensity_of(const cplx<T>* f, const LossDims& d, int64_t i) {
  T s = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (d.mask & (1u << c)) {
      cplx<T> e = f[c * d.plane + i];
      s += e.x * e.x + e.y * e.y;
    }
  return s;
}

// STED effective intensity (Methods, "Stimulated emission depletion model"):
// I_eff = I_ex [1 - beta (1 - exp(-I_dep / I_ex))], 0 where I_ex = 0.
template <typename T> __device__ __forceinline__ T sted_eff(T ie, T idp, T beta) {
  return ie > (T)0 ? ie * ((T)1 - beta * ((T)1 - exp(-idp / ie))) : (T)0;
}

// Camera intensity of batch element b at pixel i: |E|^2 over the selected components, or the
// STED effective intensity of the excitation (f) and depletion (d.dep) fields.
template <typename T, int NC>
__device__ __forceinline__ T intensity(const cplx<T>* f, const LossDims& d, int64_t i, int b) {
  const T ie = intensity_of<T, NC>(f, d, i);
  if (!d.dep) return ie;
  const cplx<T>* g = (const cplx<T>*)d.dep + (int64_t)b * NC * d.plane;
  return sted_eff<T>(ie, intensity_of<T, NC>(g, d, i), (T)d.beta);
}

__device__ __forceinline__ double bsum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}
// Block sums of N values in one pass (each summed in bsum's order); valid in thread 0.
// red: 32 * N doubles.
template <int N>
__device__ __forceinline__ void bsum_n(double (&v)[N], double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int j = 0; j < N; ++j) red[j * 32 + (threadIdx.x >> 5)] = v[j];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[j * 32 + w];
      v[j] = s;
    }
}
__device__ __forceinline__ double bmax(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = fmax(s, red[w]);
  return s;
}

// Pixels a thread visits per step of a row: a compile-time count with no branch between them,
// so that their loads are all in flight together.
constexpr int kLossPix = 8;

// Pixels of a block: the rows [r0, r1) of gridDim.x equal row ranges, each row swept by the
// block's threads in coalesced steps of kLossPix * blockDim.x pixels; fn(i, x, y, live) gets the
// pixel index and its coordinates, formed in T from per-launch bases (no per-pixel integer
// division or double arithmetic). Lanes past the row's end (live false) get the row's last
// pixel, an in-range index, and must add nothing and store nothing.
template <typename T, typename F>
__device__ __forceinline__ void for_pixels(const LossDims& d, F&& fn) {
  const int rpb = (d.ny + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rpb, r1 = min(d.ny, r0 + rpb);
  const T X0 = (T)d.x0, DX = (T)d.dx, Y0 = (T)d.y0, DY = (T)d.dy;
  for (int r = r0; r < r1; ++r) {
    const T y = Y0 + (T)r * DY;
    const int64_t base = (int64_t)r * d.nx;
    for (int c0 = 0; c0 < d.nx; c0 += kLossPix * (int)blockDim.x) {
#pragma unroll
      for (int k = 0; k < kLossPix; ++k) {
        const int xi = c0 + k * (int)blockDim.x + (int)threadIdx.x;
        const bool live = xi < d.nx;
        const int xc = live ? xi : d.nx - 1;
        fn(base + xc, X0 + (T)xc * DX, y, live);
      }
    }
  }
}

// Sweep 1. partial: [batch][blocks][3]. grid (loss_blocks, batch). INTEN: also store the
// intensity (a separate instance, so that the sweep without it has no store between its loads).
template <typename T, int NC, int MODE, bool INTEN>
__global__ void __launch_bounds__(kLossThreads, NC == 1 && sizeof(T) == 4 && MODE == XL_SECOND_MOMENT ? 8 : 1) k_loss_sweep1(const cplx<T>* __restrict__ field, LossDims d,
                                                              double* __restrict__ partial,
                                                              T* __restrict__ inten) {
  __shared__ double red[32 * 3];
  const int b = blockIdx.y;
  const cplx<T>* f = field + (int64_t)b * NC * d.plane;
  T s0 = 0, s1 = 0, s2 = 0;
  for_pixels<T>(d, [&](int64_t i, T x, T y, bool live) {
    const T Iv = intensity<T, NC>(f, d, i, b);
    if (INTEN && live) inten[(int64_t)b * d.plane + i] = Iv;
    const T I = live ? Iv : (T)0;
    if (MODE == XL_SECOND_MOMENT) {
      s0 += I;
      s1 += I * x;
      s2 += I * y;
    } else if (MODE == XL_MSE) {
      const T e = live ? I - ((const T*)d.target)[(int64_t)b * d.plane + i] : (T)0;
      s0 += e * e;
    } else {
      s0 = fmax(s0, I);
    }
  });
  double* p = partial + ((int64_t)b * gridDim.x + blockIdx.x) * 3;
  if (MODE == XL_SECOND_MOMENT || MODE == XL_MSE) {
    double v[3] = {(double)s0, (double)s1, (double)s2};
    bsum_n<3>(v, red);
    if (threadIdx.x == 0) {
      p[0] = v[0];
      p[1] = v[1];
      p[2] = v[2];
    }
  } else {
    double m = bmax((double)s0, red);
    if (threadIdx.x == 0) p[0] = m;
  }
}

// Sweep 2 (needs st[b][.] from finalise 1). partial: [batch][blocks][3].
template <typename T, int NC, int MODE>
__global__ void __launch_bounds__(kLossThreads) k_loss_sweep2(const cplx<T>* __restrict__ field, LossDims d,
                                                              const double* __restrict__ st,
                                                              double* __restrict__ partial) {
  __shared__ double red[32 * 2];
  const int b = blockIdx.y;
  const cplx<T>* f = field + (int64_t)b * NC * d.plane;
  const double* sb = st + (int64_t)b * 8;
  T s0 = 0, s1 = 0;
  if (MODE == XL_MSE) {
    // single sweep: nothing to add
  } else if (MODE == XL_SECOND_MOMENT) {
    const T xb = (T)sb[1], yb = (T)sb[2];
    for_pixels<T>(d, [&](int64_t i, T x, T y, bool live) {
      const T I = live ? intensity<T, NC>(f, d, i, b) : (T)0;
      const T ex = x - xb, ey = y - yb;
      s0 += I * (ex * ex + ey * ey);
    });
  } else {
    const T thr = (T)sb[3];
    for_pixels<T>(d, [&](int64_t i, T, T, bool live) {
      const T I = intensity<T, NC>(f, d, i, b);
      if (live && I > thr) {
        s0 += (T)1;
        s1 += I;
      }
    });
  }
  double v[2] = {(double)s0, (double)s1};
  bsum_n<2>(v, red);
  if (threadIdx.x == 0) {
    double* p = partial + ((int64_t)b * gridDim.x + blockIdx.x) * 3;
    p[0] = v[0];
    p[1] = v[1];
  }
}

// Finalisers: one block per batch element, fixed-order sums of the partials.
// st[b]: [0] P, [1] xbar, [2] ybar, [3] threshold, [4] i_max, [5] L, [6] Area, [7] I_eps
__global__ void k_loss_fin1(const double* __restrict__ partial, int nblk, LossDims d, double* __restrict__ st) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  const double* p = partial + (int64_t)b * nblk * 3;
  double* s = st + (int64_t)b * 8;
  if (d.mode == XL_SECOND_MOMENT || d.mode == XL_MSE) {
    double a = 0, x = 0, y = 0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) {
      a += p[3 * k];
      x += p[3 * k + 1];
      y += p[3 * k + 2];
    }
    a = bsum(a, red);
    x = bsum(x, red);
    y = bsum(y, red);
    if (threadIdx.x == 0) {
      s[0] = a;
      s[1] = d.mode == XL_MSE ? 0.0 : x / a;
      s[2] = d.mode == XL_MSE ? 0.0 : y / a;
    }
  } else {
    double m = 0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) m = fmax(m, p[3 * k]);
    m = bmax(m, red);
    if (threadIdx.x == 0) {
      s[4] = m;
      s[3] = d.eps * m;
    }
  }
}

__global__ void k_loss_fin2(const double* __restrict__ partial, int nblk, LossDims d, double* __restrict__ st,
                            double* __restrict__ loss) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  const double* p = partial + (int64_t)b * nblk * 3;
  double* s = st + (int64_t)b * 8;
  double a = 0, c = 0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) {
    a += p[3 * k];
    c += p[3 * k + 1];
  }
  a = bsum(a, red);
  c = bsum(c, red);
  if (threadIdx.x == 0) {
    double L;
    if (d.mode == XL_SECOND_MOMENT) {
      L = a / s[0];
    } else if (d.mode == XL_MSE) {
      L = s[0] / (double)d.plane;
    } else {
      s[6] = a;
      s[7] = c;
      L = a / c;
    }
    s[5] = L;
    if (loss) loss[b] = L;
    if (!isfinite(L)) atomicOr(&g_status_bits, 1u);
  }
}

// g_field = 2 g_loss dL/dI E on the selected components (0 elsewhere); with a depletion field
// the chain rule through I_eff gives g_field = 2 g dL/dI_eff dI_eff/dI_ex E_ex and
// g_dep = 2 g dL/dI_eff dI_eff/dI_dep E_dep, with dI_eff/dI_ex = 1 - beta + beta e^{-r} (1 + r),
// dI_eff/dI_dep = -beta e^{-r}, r = I_dep / I_ex (limits (1 - beta, 0) at I_ex = 0).
// grid (blocks, batch).
template <typename T, int NC, int MODE>
__global__ void __launch_bounds__(kLossThreads) k_loss_grad(const cplx<T>* __restrict__ field, LossDims d,
                                                            const double* __restrict__ st,
                                                            const double* __restrict__ g_loss,
                                                            cplx<T>* __restrict__ gf,
                                                            cplx<T>* __restrict__ gdep) {
  const int b = blockIdx.y;
  const cplx<T>* f = field + (int64_t)b * NC * d.plane;
  const cplx<T>* fd = d.dep ? (const cplx<T>*)d.dep + (int64_t)b * NC * d.plane : nullptr;
  cplx<T>* g = gf + (int64_t)b * NC * d.plane;
  cplx<T>* gd = gdep ? gdep + (int64_t)b * NC * d.plane : nullptr;
  const double* sb = st + (int64_t)b * 8;
  const double gl = g_loss ? g_loss[b] : 1.0;
  // the two quotients in double once for the block (FP64 runs at a small fraction of the FP32
  // rate; a division in every thread kept its pipe busy)
  __shared__ T q_s[2];
  if (threadIdx.x == 0) {
    q_s[0] = (T)(1.0 / sb[0]);
    q_s[1] = (T)(-sb[6] / (sb[7] * sb[7]));
  }
  __syncthreads();
  const T xb = (T)sb[1], yb = (T)sb[2], L = (T)sb[5], iP = q_s[0];
  const T thr = (T)sb[3], dens = q_s[1];
  const T beta = (T)d.beta;
  for_pixels<T>(d, [&](int64_t i, T x, T y, bool live) {
    T dI;
    if (MODE == XL_SECOND_MOMENT) {
      const T ex = x - xb, ey = y - yb;
      dI = (ex * ex + ey * ey - L) * iP;
    } else if (MODE == XL_MSE) {
      dI = (T)2 * (intensity<T, NC>(f, d, i, b) - ((const T*)d.target)[(int64_t)b * d.plane + i]) /
           (T)d.plane;
    } else {
      dI = intensity<T, NC>(f, d, i, b) > thr ? dens : (T)0;
    }
    T wex = (T)(2.0 * gl) * dI, wdp = (T)0;
    if (fd) {
      const T ie = intensity_of<T, NC>(f, d, i), idp = intensity_of<T, NC>(fd, d, i);
      if (ie > (T)0) {
        const T r = idp / ie, e = exp(-r);
        wdp = wex * (-beta * e);
        wex = wex * ((T)1 - beta + beta * e * ((T)1 + r));
      } else {
        wex = wex * ((T)1 - beta);
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const bool on = (d.mask & (1u << c)) != 0;
      const cplx<T> gv = on ? cscale(f[c * d.plane + i], wex) : mk((T)0, (T)0);
      if (live) g[c * d.plane + i] = gv;
      if (gd) {
        const cplx<T> gdv = on ? cscale(fd[c * d.plane + i], wdp) : mk((T)0, (T)0);
        if (live) gd[c * d.plane + i] = gdv;
      }
    }
  });
}

// softmin over detectors: out[b] = -log(sum_d exp(-beta l[b][d])) / beta (minimum subtracted),
// w[b][d] = d out[b] / d l[b][d] = exp(-beta (l - min)) / sum.
__global__ void k_softmin(const double* __restrict__ l, int batch, int n, double beta,
                          double* __restrict__ out, double* __restrict__ w) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const double* lb = l + (int64_t)b * n;
  double mn = lb[0];
  for (int d = 1; d < n; ++d) mn = fmin(mn, lb[d]);
  double s = 0;
  for (int d = 0; d < n; ++d) s += exp(-beta * (lb[d] - mn));
  out[b] = mn - log(s) / beta;
  if (w)
    for (int d = 0; d < n; ++d) w[(int64_t)b * n + d] = exp(-beta * (lb[d] - mn)) / s;
}

namespace {

xl_status loss_check(const void* field, int32_t batch, int32_t comps, uint32_t mask,
                     const xl_grid* g, int32_t mode, double eps, int32_t dtype, LossDims* d,
                     const void* dep = nullptr, double beta = 0.0, const void* target = nullptr) {
  if (!g) return fail(XL_ERR_ARG, "grid is NULL");
  if (batch < 0) return fail(XL_ERR_ARG, "batch < 0");
  if (comps < 1 || comps > 3) return fail(XL_ERR_ARG, "comps must be 1..3");
  if ((mask & ((1u << comps) - 1)) == 0) return fail(XL_ERR_ARG, "comp_mask selects no component");
  if (mode != XL_SECOND_MOMENT && mode != XL_DENSITY && mode != XL_MSE)
    return fail(XL_ERR_ARG, "unknown loss mode");
  if (mode == XL_MSE && !target) return fail(XL_ERR_ARG, "XL_MSE needs a target intensity");
  if (dep && !(beta >= 0 && beta <= 1)) return fail(XL_ERR_ARG, "STED beta must be in [0, 1]");
  if (mode == XL_DENSITY && !(eps >= 0 && eps <= 1)) return fail(XL_ERR_ARG, "eps must be in [0, 1]");
  if (g->nx < 1 || g->ny < 1) return fail(XL_ERR_ARG, "empty grid");
  if (dtype != XL_C64 && dtype != XL_C128) return fail(XL_ERR_ARG, "bad dtype");
  if (batch > 0 && !field) return fail(XL_ERR_ARG, "field is NULL");
  d->nx = g->nx;
  d->ny = g->ny;
  d->comps = comps;
  d->mask = mask & ((1u << comps) - 1);
  d->plane = (int64_t)g->nx * g->ny;
  d->x0 = g->x0;
  d->dx = g->dx;
  d->y0 = g->y0;
  d->dy = g->dy;
  d->eps = eps;
  d->mode = mode;
  d->dep = dep;
  d->beta = beta;
  d->target = target;
  return XL_OK;
}

int loss_blocks(const LossDims& d) {
  int64_t need = (d.plane + kLossThreads * 4 - 1) / (kLossThreads * 4);
  // per batch element at most two blocks per SM of the device, and at most one per row
  need = std::min<int64_t>(need, d.ny);
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, 2 * (int64_t)sm_count()));
}

// Both sweeps and finalisers (st / loss in the workspace or caller memory) and, with `grad`, the
// field gradient dL/dE (g_loss nullable = 1) from the statistics they leave in st.
template <typename T, int NC, int MODE>
xl_status loss_run(const void* field, int32_t batch, const LossDims& d, double* st, double* loss,
                   void* inten, double* partial, bool grad, const double* g_loss, void* g_field,
                   void* g_dep, cudaStream_t s) {
  typedef cplx<T> C;
  const int nb = loss_blocks(d);
  dim3 grid(nb, batch);
  {
    LaunchScope ls("loss_sweep1", s);
    if (inten)
      k_loss_sweep1<T, NC, MODE, true><<<grid, kLossThreads, 0, s>>>((const C*)field, d, partial, (T*)inten);
    else
      k_loss_sweep1<T, NC, MODE, false><<<grid, kLossThreads, 0, s>>>((const C*)field, d, partial, nullptr);
    XL_CUDA_TRY(cudaGetLastError());
  }
  {
    LaunchScope ls("loss_fin1", s);
    k_loss_fin1<<<batch, 256, 0, s>>>(partial, nb, d, st);
    XL_CUDA_TRY(cudaGetLastError());
  }
  if (MODE != XL_MSE) {
    LaunchScope ls("loss_sweep2", s);
    k_loss_sweep2<T, NC, MODE><<<grid, kLossThreads, 0, s>>>((const C*)field, d, st, partial);
    XL_CUDA_TRY(cudaGetLastError());
  }
  {
    LaunchScope ls("loss_fin2", s);
    k_loss_fin2<<<batch, 256, 0, s>>>(partial, nb, d, st, loss);
    XL_CUDA_TRY(cudaGetLastError());
  }
  if (grad) {
    LaunchScope ls("loss_grad", s);
    k_loss_grad<T, NC, MODE><<<grid, kLossThreads, 0, s>>>((const C*)field, d, st, g_loss, (C*)g_field,
                                                           (C*)g_dep);
    XL_CUDA_TRY(cudaGetLastError());
  }
  return XL_OK;
}

template <typename T>
xl_status loss_dispatch(const void* field, int32_t batch, const LossDims& d, double* st, double* loss,
                        void* inten, double* partial, bool grad, const double* g_loss, void* g_field,
                        void* g_dep, cudaStream_t s) {
#define XL_LOSS_CASE(NC, MODE)                                                                \
  if (d.comps == NC && d.mode == MODE)                                                        \
    return loss_run<T, NC, MODE>(field, batch, d, st, loss, inten, partial, grad, g_loss, g_field, \
                                 g_dep, s);
  XL_LOSS_CASE(1, XL_SECOND_MOMENT) XL_LOSS_CASE(2, XL_SECOND_MOMENT) XL_LOSS_CASE(3, XL_SECOND_MOMENT)
  XL_LOSS_CASE(1, XL_DENSITY) XL_LOSS_CASE(2, XL_DENSITY) XL_LOSS_CASE(3, XL_DENSITY)
  XL_LOSS_CASE(1, XL_MSE) XL_LOSS_CASE(2, XL_MSE) XL_LOSS_CASE(3, XL_MSE)
#undef XL_LOSS_CASE
  return fail(XL_ERR_ARG, "loss: unsupported component count or mode");
}

// Workspace statistics [batch][8] and block partials of one call.
xl_status loss_workspace(int32_t batch, const LossDims& d, cudaStream_t s, double** st, double** partial) {
  const int nb = loss_blocks(d);
  void* ws = nullptr;
  const size_t st_bytes = (size_t)batch * 8 * sizeof(double);
  const size_t pb = (size_t)batch * nb * 3 * sizeof(double);
  XL_TRY(workspace(s, st_bytes + pb + 256, &ws, 3));
  *st = (double*)ws;
  *partial = (double*)((char*)ws + ((st_bytes + 255) & ~(size_t)255));
  return XL_OK;
}

}  // namespace
}  // namespace xl

using namespace xl;

extern "C" {

xl_status xl_intensity_loss_ex(const void* field, const void* field_dep, const void* target,
                               int32_t batch, int32_t comps, uint32_t comp_mask,
                               const xl_grid* grid, int32_t mode, double eps, double beta,
                               double* loss, void* intensity, int32_t dtype, void* stream) {
  LossDims d;
  XL_TRY(loss_check(field, batch, comps, comp_mask, grid, mode, eps, dtype, &d, field_dep, beta,
                    target));
  if (batch == 0) return XL_OK;
  if (!loss) return fail(XL_ERR_ARG, "loss is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  double *st = nullptr, *partial = nullptr;
  XL_TRY(loss_workspace(batch, d, s, &st, &partial));
  return dtype == XL_C128
             ? loss_dispatch<double>(field, batch, d, st, loss, intensity, partial, false, nullptr, nullptr, nullptr, s)
             : loss_dispatch<float>(field, batch, d, st, loss, intensity, partial, false, nullptr, nullptr, nullptr, s);
}

xl_status xl_intensity_loss(const void* field, int32_t batch, int32_t comps, uint32_t comp_mask,
                            const xl_grid* grid, int32_t mode, double eps, double* loss,
                            void* intensity, int32_t dtype, void* stream) {
  if (mode == XL_MSE) return fail(XL_ERR_ARG, "XL_MSE needs xl_intensity_loss_ex (a target)");
  return xl_intensity_loss_ex(field, nullptr, nullptr, batch, comps, comp_mask, grid, mode, eps,
                              0.0, loss, intensity, dtype, stream);
}

namespace {
xl_status loss_grad_call(const void* field, const void* field_dep, const void* target, int32_t batch,
                         int32_t comps, uint32_t comp_mask, const xl_grid* grid, int32_t mode,
                         double eps, double beta, double* loss, const double* g_loss, void* g_field,
                         void* g_field_dep, int32_t dtype, void* stream) {
  LossDims d;
  XL_TRY(loss_check(field, batch, comps, comp_mask, grid, mode, eps, dtype, &d, field_dep, beta,
                    target));
  if (batch == 0) return XL_OK;
  if (!g_field) return fail(XL_ERR_ARG, "g_field is NULL");
  if (g_field == field) return fail(XL_ERR_ARG, "g_field may not alias field");
  if (field_dep && !g_field_dep) return fail(XL_ERR_ARG, "g_field_dep is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  double *st = nullptr, *partial = nullptr;
  XL_TRY(loss_workspace(batch, d, s, &st, &partial));
  void* gdep = field_dep ? g_field_dep : nullptr;
  return dtype == XL_C128
             ? loss_dispatch<double>(field, batch, d, st, loss, nullptr, partial, true, g_loss, g_field, gdep, s)
             : loss_dispatch<float>(field, batch, d, st, loss, nullptr, partial, true, g_loss, g_field, gdep, s);
}
}  // namespace

xl_status xl_intensity_loss_ex_backward(const void* field, const void* field_dep,
                                        const void* target, int32_t batch, int32_t comps,
                                        uint32_t comp_mask, const xl_grid* grid, int32_t mode,
                                        double eps, double beta, const double* g_loss,
                                        void* g_field, void* g_field_dep, int32_t dtype,
                                        void* stream) {
  return loss_grad_call(field, field_dep, target, batch, comps, comp_mask, grid, mode, eps, beta,
                        nullptr, g_loss, g_field, g_field_dep, dtype, stream);
}

xl_status xl_intensity_loss_and_grad(const void* field, const void* field_dep, const void* target,
                                     int32_t batch, int32_t comps, uint32_t comp_mask,
                                     const xl_grid* grid, int32_t mode, double eps, double beta,
                                     double* loss, void* g_field, void* g_field_dep, int32_t dtype,
                                     void* stream) {
  if (!loss) return fail(XL_ERR_ARG, "loss is NULL");
  return loss_grad_call(field, field_dep, target, batch, comps, comp_mask, grid, mode, eps, beta,
                        loss, nullptr, g_field, g_field_dep, dtype, stream);
}

xl_status xl_intensity_loss_backward(const void* field, int32_t batch, int32_t comps,
                                     uint32_t comp_mask, const xl_grid* grid, int32_t mode,
                                     double eps, const double* g_loss, void* g_field,
                                     int32_t dtype, void* stream) {
  if (mode == XL_MSE) return fail(XL_ERR_ARG, "XL_MSE needs xl_intensity_loss_ex_backward");
  return xl_intensity_loss_ex_backward(field, nullptr, nullptr, batch, comps, comp_mask, grid,
                                       mode, eps, 0.0, g_loss, g_field, nullptr, dtype, stream);
}

xl_status xl_softmin(const double* losses, int32_t batch, int32_t n_det, double beta, double* out,
                     double* weights, void* stream) {
  if (batch < 0 || n_det < 1) return fail(XL_ERR_ARG, "softmin: bad sizes");
  if (!(beta > 0) || !std::isfinite(beta)) return fail(XL_ERR_ARG, "softmin: beta must be > 0");
  if (batch == 0) return XL_OK;
  if (!losses || !out) return fail(XL_ERR_ARG, "softmin: NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  LaunchScope ls("softmin", s);
  k_softmin<<<(batch + 127) / 128, 128, 0, s>>>(losses, batch, n_det, beta, out, weights);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

xl_status xl_device_status(void* stream) {
  XL_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned int bits = 0, zero = 0;
  XL_CUDA_TRY(cudaMemcpyFromSymbol(&bits, g_status_bits, sizeof(bits)));
  XL_CUDA_TRY(cudaMemcpyToSymbol(g_status_bits, &zero, sizeof(zero)));
  if (bits & 1u) return fail(XL_ERR_NONFINITE, "a loss reduction produced a non-finite value");
  unsigned int w = 0;
  XL_TRY(status_word_take((cudaStream_t)stream, &w));
  if (w & 2u) return fail(XL_ERR_TIMEOUT, "a kernel gave up waiting for a bulk copy");
  return XL_OK;
}

}  // extern "C"
