// Adam optimiser step (the optimiser of the paper's discovery and benchmark runs: Results and
// Methods, Adam with step sizes 0.1, 0.01 and 0.03; Kingma & Ba). Bias-corrected, step t >= 1:
//   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
//   p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
// AdamW (the decoupled weight decay the paper's data-driven and topology runs use: Methods,
// weight decay 1e-4) also subtracts lr * wd * p (p before the step).
// The step number can live on the device so that a captured CUDA graph replays correct bias
// corrections; xl_step_advance increments it in-stream.
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "xl_runtime.h"

namespace xl {

struct AdamArgs {
  int64_t n;
  double lr, b1, b2, eps, wd;
  const int32_t* t_dev;
  int32_t t_host;
  int vec;  // the arrays are 16-byte aligned: the bulk runs on 16-byte vectors
};

template <typename R>
__global__ void __launch_bounds__(256) k_adam(R* __restrict__ p, R* __restrict__ m, R* __restrict__ v,
                                              const R* __restrict__ g, AdamArgs a) {
  __shared__ R c[4];
  if (threadIdx.x == 0) {
    const double t = (double)(a.t_dev ? *a.t_dev : a.t_host);
    const double c1 = 1.0 - pow(a.b1, t), c2 = 1.0 - pow(a.b2, t);
    c[0] = (R)(a.lr / c1);  // lr / (1 - b1^t)
    c[1] = (R)(1.0 / c2);   // 1 / (1 - b2^t)
    c[2] = (R)a.eps;
    c[3] = (R)(a.lr * a.wd);  // decoupled weight decay (AdamW)
  }
  __syncthreads();
  const R b1 = (R)a.b1, b2 = (R)a.b2, s = c[0], iv = c[1], eps = c[2], dec = c[3];
  auto upd = [&](R& pi, R& mi, R& vi, R gi) {
    mi = b1 * mi + ((R)1 - b1) * gi;
    vi = b2 * vi + ((R)1 - b2) * gi * gi;
    pi = pi - s * mi / (sqrt(vi * iv) + eps) - dec * pi;
  };
  // 16-byte vectors of 16 / sizeof(R) parameters (all four arrays are 16-byte aligned: the host
  // checks), so that each thread keeps four 16-byte loads in flight; the scalar tail follows
  typedef typename std::conditional<sizeof(R) == 4, float4, double2>::type V;
  constexpr int K = 16 / sizeof(R);
  const int64_t nv = a.vec ? a.n / K : 0;
  V* pv = reinterpret_cast<V*>(p);
  V* mv = reinterpret_cast<V*>(m);
  V* vv = reinterpret_cast<V*>(v);
  const V* gv = reinterpret_cast<const V*>(g);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
       i += (int64_t)gridDim.x * blockDim.x) {
    V P = pv[i], Mm = mv[i], Vv = vv[i];
    const V G = gv[i];
    R* pp = reinterpret_cast<R*>(&P);
    R* mm = reinterpret_cast<R*>(&Mm);
    R* ww = reinterpret_cast<R*>(&Vv);
    const R* gg = reinterpret_cast<const R*>(&G);
#pragma unroll
    for (int k = 0; k < K; ++k) upd(pp[k], mm[k], ww[k], gg[k]);
    pv[i] = P;
    mv[i] = Mm;
    vv[i] = Vv;
  }
  for (int64_t i = nv * K + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    R pi = p[i], mi = m[i], vi = v[i];
    upd(pi, mi, vi, g[i]);
    m[i] = mi;
    v[i] = vi;
    p[i] = pi;
  }
}

__global__ void k_step_advance(int32_t* t) { *t += 1; }

}  // namespace xl

using namespace xl;

extern "C" {

xl_status xl_adamw_step(void* params, void* m, void* v, const void* grad, int64_t n,
                        int32_t real_dtype, double lr, double beta1, double beta2, double eps,
                        double weight_decay, const int32_t* t_dev, int32_t t_host, void* stream) {
  if (n < 0) return fail(XL_ERR_ARG, "n < 0");
  if (real_dtype != 0 && real_dtype != 1) return fail(XL_ERR_ARG, "real_dtype must be 0 (float) or 1 (double)");
  if (!(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return fail(XL_ERR_ARG, "need 0 <= beta < 1 and eps > 0");
  if (!t_dev && t_host < 1) return fail(XL_ERR_ARG, "step number must be >= 1");
  if (n == 0) return XL_OK;
  if (!params || !m || !v || !grad) return fail(XL_ERR_ARG, "NULL pointer");
  if (!(weight_decay >= 0) || !std::isfinite(weight_decay)) return fail(XL_ERR_ARG, "weight decay must be >= 0");
  auto a16 = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
  AdamArgs a{n, lr, beta1, beta2, eps, weight_decay, t_dev, t_host,
             a16(params) && a16(m) && a16(v) && a16(grad) ? 1 : 0};
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8 * (int64_t)sm_count());
  LaunchScope ls("adam", s);
  if (real_dtype == 1)
    k_adam<double><<<blocks, 256, 0, s>>>((double*)params, (double*)m, (double*)v, (const double*)grad, a);
  else
    k_adam<float><<<blocks, 256, 0, s>>>((float*)params, (float*)m, (float*)v, (const float*)grad, a);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

xl_status xl_adam_step(void* params, void* m, void* v, const void* grad, int64_t n,
                       int32_t real_dtype, double lr, double beta1, double beta2, double eps,
                       const int32_t* t_dev, int32_t t_host, void* stream) {
  return xl_adamw_step(params, m, v, grad, n, real_dtype, lr, beta1, beta2, eps, 0.0, t_dev, t_host,
                       stream);
}

xl_status xl_step_advance(int32_t* t_dev, void* stream) {
  if (!t_dev) return fail(XL_ERR_ARG, "NULL step counter");
  cudaStream_t s = (cudaStream_t)stream;
  LaunchScope ls("step_advance", s);
  k_step_advance<<<1, 1, 0, s>>>(t_dev);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

}  // extern "C"
