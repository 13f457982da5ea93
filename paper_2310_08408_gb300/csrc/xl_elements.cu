// Fused optical-element chains and their adjoints (Methods, "Features and performance": spatial
// light modulators (SLM), the super-SLM imprinting independent phases on the horizontal and
// vertical components, planar lenses, polarisers and variable retarders / wave plates).
//
// Readings (the paper names the elements only):
//   SLM        every component times exp(i phi)
//   super-SLM  Ex times exp(i phi_x), Ey times exp(i phi_y)
//   lens       every component times exp(-i k (x^2 + y^2) / (2 f))
//   polariser  J = R(-a) diag(1, 0) R(a)
//   wave plate J = R(-t) diag(1, exp(i eta)) R(t),  R(t) = [[cos t, sin t], [-sin t, cos t]]
//   to-vector  (Ex, Ey) = (u, 0)
// Three-component fields (Ex, Ey, Ez): phase masks and lenses act on all three components, Jones
// elements on (Ex, Ey) only.
// One thread handles one pixel of one batch element and applies the whole chain in registers
// (the chain is read from kernel parameters), so a chain costs one read and one write of the
// field. The lens phase is separable, exp(-ik x^2/2f) exp(-ik y^2/2f): both factors are
// tabulated per call in double precision (reduced modulo 2 pi, rounded once), so the per-pixel
// work is one complex multiply.
// Backward: the forward states are recomputed per pixel, then g <- J^H g element by element in
// reverse; dL/dphi = Im(g_out conj(u_out)) per pixel (summed over the batch when the mask is
// shared), and the scalar gradients dL/d{f, alpha, eta, theta} = Re sum conj(g_out) dJ u_in are
// reduced per block in double precision and then in fixed order per batch element.
#include <cmath>
#include <cstring>
#include <vector>

#include "xl_runtime.h"

namespace xl {

constexpr int kMaxElem = 8;

struct ElemSet {
  int n;
  int kind[kMaxElem];
  int lens_slot[kMaxElem];      // lens table index (-1 if not a lens)
  const void* phx[kMaxElem];
  const void* phy[kMaxElem];
  int64_t phstride[kMaxElem];
  double hp[kMaxElem][4];       // host parameters {f, alpha, eta, theta}
};

struct ElemDims {
  int nx, ny, comps_in, comps_out;
  int nx_shift;                 // log2(nx) when nx is a power of two, else -1
  int64_t plane;
  double x0, dx, y0, dy, k;
  const double* params_dev;     // [batch][n][4] or nullptr (host parameters)
};

template <typename T> struct Jones2 {
  cplx<T> a, b, c, d;
};

template <typename T>
__device__ __forceinline__ Jones2<T> mul2(const Jones2<T>& x, const Jones2<T>& y) {
  return {cadd(cmul(x.a, y.a), cmul(x.b, y.c)), cadd(cmul(x.a, y.b), cmul(x.b, y.d)),
          cadd(cmul(x.c, y.a), cmul(x.d, y.c)), cadd(cmul(x.c, y.b), cmul(x.d, y.d))};
}
template <typename T> __device__ __forceinline__ Jones2<T> rot2(T c, T s) {
  return {mk(c, (T)0), mk(s, (T)0), mk(-s, (T)0), mk(c, (T)0)};
}

// J, and its derivatives where relevant, for polariser (alpha) and wave plate (eta, theta).
template <typename T>
__device__ __forceinline__ void polarizer(double a, Jones2<T>* J, Jones2<T>* dJ) {
  T c, s;
  xsincos((T)a, &s, &c);
  *J = {mk(c * c, (T)0), mk(c * s, (T)0), mk(c * s, (T)0), mk(s * s, (T)0)};
  if (dJ) *dJ = {mk(-2 * c * s, (T)0), mk(c * c - s * s, (T)0), mk(c * c - s * s, (T)0), mk(2 * c * s, (T)0)};
}

template <typename T>
__device__ __forceinline__ void waveplate(double eta, double th, Jones2<T>* J, Jones2<T>* dJe,
                                          Jones2<T>* dJt) {
  T c, s, ec, es;
  xsincos((T)th, &s, &c);
  xsincos((T)eta, &es, &ec);
  const cplx<T> e = mk(ec, es);
  const cplx<T> one = mk((T)1, (T)0), zero = mk((T)0, (T)0);
  Jones2<T> D = {one, zero, zero, e};
  Jones2<T> Rm = rot2<T>(c, -s), Rp = rot2<T>(c, s);  // R(-t), R(t)
  *J = mul2(Rm, mul2(D, Rp));
  if (dJe) {
    Jones2<T> dD = {zero, zero, zero, mk(-e.y, e.x)};
    *dJe = mul2(Rm, mul2(dD, Rp));
  }
  if (dJt) {
    // d/dt R(t) = [[-s, c], [-c, -s]];  d/dt R(-t) = [[-s, -c], [c, -s]]
    Jones2<T> dRp = {mk(-s, (T)0), mk(c, (T)0), mk(-c, (T)0), mk(-s, (T)0)};
    Jones2<T> dRm = {mk(-s, (T)0), mk(-c, (T)0), mk(c, (T)0), mk(-s, (T)0)};
    Jones2<T> A = mul2(dRm, mul2(D, Rp)), B = mul2(Rm, mul2(D, dRp));
    *dJt = {cadd(A.a, B.a), cadd(A.b, B.b), cadd(A.c, B.c), cadd(A.d, B.d)};
  }
}

template <typename T>
__device__ __forceinline__ void japply(const Jones2<T>& J, cplx<T>& u0, cplx<T>& u1) {
  cplx<T> a = cadd(cmul(J.a, u0), cmul(J.b, u1));
  cplx<T> b = cadd(cmul(J.c, u0), cmul(J.d, u1));
  u0 = a;
  u1 = b;
}
// g <- J^H g
template <typename T>
__device__ __forceinline__ void japply_h(const Jones2<T>& J, cplx<T>& g0, cplx<T>& g1) {
  cplx<T> a = cadd(cmul(cconj(J.a), g0), cmul(cconj(J.c), g1));
  cplx<T> b = cadd(cmul(cconj(J.b), g0), cmul(cconj(J.d), g1));
  g0 = a;
  g1 = b;
}
// Re(conj(g) . (J u))
template <typename T>
__device__ __forceinline__ T jre(const Jones2<T>& J, cplx<T> g0, cplx<T> g1, cplx<T> u0, cplx<T> u1) {
  cplx<T> a = cadd(cmul(J.a, u0), cmul(J.b, u1));
  cplx<T> b = cadd(cmul(J.c, u0), cmul(J.d, u1));
  return cdot_re(g0, a) + cdot_re(g1, b);
}

__device__ __forceinline__ double eparam(const ElemSet& E, const ElemDims& d, int b, int e, int j) {
  return d.params_dev ? d.params_dev[((int64_t)b * E.n + e) * 4 + j] : E.hp[e][j];
}

template <typename T>
__device__ __forceinline__ T phase_at(const void* p, int64_t stride, int b, int64_t i) {
  // masks are never written by the element kernels: the read-only path lets the loads of later
  // pixels be issued ahead of this pixel's stores
  return __ldg((const T*)p + (int64_t)b * stride + i);
}

// Lens tables: for lens slot s and batch element b, Lx[m] then Ly[n] (complex T).
__device__ __forceinline__ double red2pi_e(double x) { return x - kTwoPi * rint(x * (1.0 / kTwoPi)); }

template <typename T>
__global__ void k_lens_tables(cplx<T>* __restrict__ tab, ElemSet E, ElemDims d, int batch, int nlens) {
  const int64_t per = (int64_t)d.nx + d.ny;
  const int64_t total = per * nlens * batch;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = i % per;
    const int s = (int)((i / per) % nlens);
    const int b = (int)(i / (per * nlens));
    int e = 0;
    for (int q = 0; q < E.n; ++q)
      if (E.lens_slot[q] == s) e = q;
    const double f = eparam(E, d, b, e, 0);
    const double c = j < d.nx ? d.x0 + j * d.dx : d.y0 + (j - d.nx) * d.dy;
    const double ph = -red2pi_e(d.k * c * c / (2.0 * f));
    T sn, cs;
    xsincos((T)ph, &sn, &cs);
    tab[i] = mk(cs, sn);
  }
}

template <typename T>
__device__ __forceinline__ cplx<T> lens_factor(const cplx<T>* tab, int s, int b, int nlens,
                                               const ElemDims& d, int m, int n) {
  const cplx<T>* t = tab + ((int64_t)b * nlens + s) * ((int64_t)d.nx + d.ny);
  return cmul(t[m], t[d.nx + n]);
}

// Column m and row n of pixel i (a shift and a mask for power-of-two rows, no integer division).
__device__ __forceinline__ void pix_mn(const ElemDims& d, int64_t i, int& m, int& n) {
  if (d.nx_shift >= 0) {
    m = (int)(i & (d.nx - 1));
    n = (int)(i >> d.nx_shift);
  } else {  // plane < 2^31: 32-bit division
    m = (int)i % d.nx;
    n = (int)i / d.nx;
  }
}

// Jones matrices of the polarisers and wave plates of batch element b (and their parameter
// derivatives), one entry per element: they depend on the element's parameters only, so a block
// whose pixels share b forms them once in shared memory instead of once per pixel.
template <typename T> struct JonesTab {
  Jones2<T> J[kMaxElem], dA[kMaxElem], dB[kMaxElem];  // dA: d/dalpha or d/deta; dB: d/dtheta
  T lens_c[kMaxElem];  // lenses: k / (2 f^2), so that d out / d f = i lens_c (x^2 + y^2) out
};
// Threads 0..E.n-1 fill entry e = threadIdx.x for batch element b; callers synchronise after.
template <typename T>
__device__ __forceinline__ void jones_fill(JonesTab<T>& jt, const ElemSet& E, const ElemDims& d, int b,
                                           bool derivs) {
  const int e = threadIdx.x;
  if (e >= E.n) return;
  if (E.kind[e] == XL_LENS) {
    const double f = eparam(E, d, b, e, 0);
    jt.lens_c[e] = (T)(d.k / (2.0 * f * f));
  } else if (E.kind[e] == XL_POLARIZER) {
    polarizer<T>(eparam(E, d, b, e, 1), &jt.J[e], derivs ? &jt.dA[e] : nullptr);
  } else if (E.kind[e] == XL_WAVEPLATE) {
    waveplate<T>(eparam(E, d, b, e, 2), eparam(E, d, b, e, 3), &jt.J[e], derivs ? &jt.dA[e] : nullptr,
                 derivs ? &jt.dB[e] : nullptr);
  }
}

// Applies element e to (c0, c1). Returns the state after it. jt: the element's Jones matrices.
// ph (nullable): receives the mask phasors exp(i phi) of an SLM (ph[0]) or super-SLM (ph[0],
// ph[1]), so that an adjoint can reuse them. Pixel i sits at column m = i % nx, row n = i / nx
// (formed only for lenses).
template <typename T>
__device__ __forceinline__ void elem_fwd(const ElemSet& E, const ElemDims& d, const cplx<T>* lens,
                                         int nlens, int e, int b, int64_t i, cplx<T>& c0,
                                         cplx<T>& c1, cplx<T>& c2, const JonesTab<T>& jt,
                                         cplx<T>* ph = nullptr) {
  switch (E.kind[e]) {
    case XL_SLM: {
      T s, c;
      xsincos(phase_at<T>(E.phx[e], E.phstride[e], b, i), &s, &c);
      c0 = cmul(c0, mk(c, s));
      c1 = cmul(c1, mk(c, s));
      c2 = cmul(c2, mk(c, s));
      if (ph) ph[0] = mk(c, s);
      break;
    }
    case XL_SSLM: {
      T s, c;
      xsincos(phase_at<T>(E.phx[e], E.phstride[e], b, i), &s, &c);
      c0 = cmul(c0, mk(c, s));
      if (ph) ph[0] = mk(c, s);
      xsincos(phase_at<T>(E.phy[e], E.phstride[e], b, i), &s, &c);
      c1 = cmul(c1, mk(c, s));
      if (ph) ph[1] = mk(c, s);
      break;
    }
    case XL_LENS: {
      int m, n;
      pix_mn(d, i, m, n);
      cplx<T> L = lens_factor<T>(lens, E.lens_slot[e], d.params_dev ? b : 0, nlens, d, m, n);
      c0 = cmul(c0, L);
      c1 = cmul(c1, L);
      c2 = cmul(c2, L);
      break;
    }
    case XL_POLARIZER:
    case XL_WAVEPLATE:
      japply(jt.J[e], c0, c1);
      break;
    case XL_TO_VECTOR:
      c1 = mk((T)0, (T)0);
      break;
  }
}

// Pixels a thread of the forward takes (kPixFwd pixels blockDim.x apart: coalesced, and the
// block's Jones table is formed once for 256 * kPixFwd pixels).
constexpr int kPixFwd = 4;

// grid: (ceil(plane / (256 kPixFwd)), batch)
template <typename T>
__global__ void __launch_bounds__(256) k_elem_fwd(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out,
                                                  ElemSet E, ElemDims d, const cplx<T>* __restrict__ lens,
                                                  int nlens) {
  const int b = blockIdx.y;
  __shared__ JonesTab<T> jt;
  jones_fill<T>(jt, E, d, b, false);
  __syncthreads();
  const cplx<T>* src = in + (int64_t)b * d.comps_in * d.plane;
  cplx<T>* dst = out + (int64_t)b * d.comps_out * d.plane;
#pragma unroll
  for (int k = 0; k < kPixFwd; ++k) {
    const int64_t i = ((int64_t)blockIdx.x * kPixFwd + k) * blockDim.x + threadIdx.x;
    if (i >= d.plane) break;
    cplx<T> c0 = src[i];
    cplx<T> c1 = d.comps_in >= 2 ? src[d.plane + i] : mk((T)0, (T)0);
    cplx<T> c2 = d.comps_in == 3 ? src[2 * d.plane + i] : mk((T)0, (T)0);
    for (int e = 0; e < E.n; ++e) elem_fwd<T>(E, d, lens, nlens, e, b, i, c0, c1, c2, jt);
    dst[i] = c0;
    if (d.comps_out >= 2) dst[d.plane + i] = c1;
    if (d.comps_out == 3) dst[2 * d.plane + i] = c2;
  }
}

struct ElemGrad {
  void* gphx[kMaxElem];
  void* gphy[kMaxElem];
  double* partial;  // [batch][n * 4][nblocks] block partials of the scalar gradients (or nullptr)
  int accumulate_shared;  // masks with stride 0 are shared: sum over the batch inside the thread
};

// Whether element kind `kind` has scalar parameter j (0 f, 1 alpha, 2 eta, 3 theta).
__host__ __device__ __forceinline__ bool has_scalar(int kind, int j) {
  return (kind == XL_LENS && j == 0) || (kind == XL_POLARIZER && j == 1) ||
         (kind == XL_WAVEPLATE && (j == 2 || j == 3));
}

// Pixels a thread of the per-element backward takes (the block reductions of the scalar
// gradients then cover 256 * kPixBwd pixels each).
constexpr int kPixBwd = 8;

// Backward. grid: (ceil(plane / (256 pix)), batch), or (ceil(plane / 256), 1) with pix = 1 when
// masks are shared (stride 0): the batch loop then runs inside the thread so that dL/dphi sums
// over the batch without atomics.
// NE: the number of elements (E.n), a compile-time bound so that the per-pixel states take
// registers for NE elements only. ST: some element's mask or scalar gradient is asked for, so the
// forward states are recomputed from the input; without (ST false) only the cotangent is read and
// each element's adjoint applied to it, last element first.
template <typename T, int NE, bool ST = true>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (NE <= 1 ? 4 : 2) : 1) k_elem_bwd(const cplx<T>* __restrict__ gout, const cplx<T>* __restrict__ in,
                                                  cplx<T>* __restrict__ gin, ElemSet E, ElemDims d,
                                                  const cplx<T>* __restrict__ lens, int nlens,
                                                  ElemGrad G, int batch, int pix) {
  __shared__ double red[32];
  const int b_lo = G.accumulate_shared ? 0 : blockIdx.y;
  const int b_hi = G.accumulate_shared ? batch : blockIdx.y + 1;
  T gphx_acc[NE > 0 ? NE : 1], gphy_acc[NE > 0 ? NE : 1];
#pragma unroll
  for (int e = 0; e < NE; ++e) gphx_acc[e] = gphy_acc[e] = (T)0;
  __shared__ JonesTab<T> jt;
  for (int b = b_lo; b < b_hi; ++b) {
    jones_fill<T>(jt, E, d, b, true);
    __syncthreads();
    // this thread's sums of the scalar gradients over its pixels (in T: FP64 runs at a small
    // fraction of the FP32 rate; the block sums below are in double)
    T sg[NE > 0 ? NE : 1][4];
#pragma unroll
    for (int e = 0; e < NE; ++e) sg[e][0] = sg[e][1] = sg[e][2] = sg[e][3] = (T)0;
    // the pixel count is kPixBwd or 1; the constant bound lets the loads of consecutive pixels
    // be issued together
    constexpr int kUnroll = NE <= 1 ? 4 : 2;  // pixels whose states are live together
#pragma unroll kUnroll
    for (int k = 0; k < (pix == kPixBwd ? kPixBwd : 1); ++k) {
      const int64_t i = ((int64_t)blockIdx.x * pix + k) * blockDim.x + threadIdx.x;
      const bool live = i < d.plane;
      const int64_t ii = live ? i : d.plane - 1;
      if constexpr (!ST) {
        const cplx<T>* gs = gout + (int64_t)b * d.comps_out * d.plane;
        cplx<T> h0 = gs[ii];
        cplx<T> h1 = d.comps_out >= 2 ? gs[d.plane + ii] : mk((T)0, (T)0);
        cplx<T> h2 = d.comps_out == 3 ? gs[2 * d.plane + ii] : mk((T)0, (T)0);
#pragma unroll
        for (int e = NE - 1; e >= 0; --e) {
          switch (E.kind[e]) {
            case XL_SLM: {
              T sn, cs;
              xsincos(phase_at<T>(E.phx[e], E.phstride[e], b, ii), &sn, &cs);
              h0 = cmulc(h0, mk(cs, sn));
              h1 = cmulc(h1, mk(cs, sn));
              h2 = cmulc(h2, mk(cs, sn));
              break;
            }
            case XL_SSLM: {
              T sn, cs;
              xsincos(phase_at<T>(E.phx[e], E.phstride[e], b, ii), &sn, &cs);
              h0 = cmulc(h0, mk(cs, sn));
              xsincos(phase_at<T>(E.phy[e], E.phstride[e], b, ii), &sn, &cs);
              h1 = cmulc(h1, mk(cs, sn));
              break;
            }
            case XL_LENS: {
              int m, n;
              pix_mn(d, ii, m, n);
              const cplx<T> L = lens_factor<T>(lens, E.lens_slot[e], d.params_dev ? b : 0, nlens, d, m, n);
              h0 = cmulc(h0, L);
              h1 = cmulc(h1, L);
              h2 = cmulc(h2, L);
              break;
            }
            case XL_POLARIZER:
            case XL_WAVEPLATE:
              japply_h(jt.J[e], h0, h1);
              break;
            case XL_TO_VECTOR:
              h1 = mk((T)0, (T)0);
              break;
          }
        }
        if (live && gin) {
          cplx<T>* dst = gin + (int64_t)b * d.comps_in * d.plane;
          dst[i] = h0;
          if (d.comps_in >= 2) dst[d.plane + i] = h1;
          if (d.comps_in == 3) dst[2 * d.plane + i] = h2;
        }
        continue;
      }
      cplx<T> s0[NE + 1], s1[NE + 1], s2[NE + 1];
      cplx<T> ph[NE > 0 ? NE : 1][2];  // mask phasors of the SLMs, reused by their adjoints
      const cplx<T>* src = in + (int64_t)b * d.comps_in * d.plane;
      s0[0] = src[ii];
      s1[0] = d.comps_in >= 2 ? src[d.plane + ii] : mk((T)0, (T)0);
      s2[0] = d.comps_in == 3 ? src[2 * d.plane + ii] : mk((T)0, (T)0);
#pragma unroll
      for (int e = 0; e < NE; ++e) {
        s0[e + 1] = s0[e];
        s1[e + 1] = s1[e];
        s2[e + 1] = s2[e];
        elem_fwd<T>(E, d, lens, nlens, e, b, ii, s0[e + 1], s1[e + 1], s2[e + 1], jt, ph[e]);
      }
      const cplx<T>* gsrc = gout + (int64_t)b * d.comps_out * d.plane;
      cplx<T> g0 = gsrc[ii];
      cplx<T> g1 = d.comps_out >= 2 ? gsrc[d.plane + ii] : mk((T)0, (T)0);
      cplx<T> g2 = d.comps_out == 3 ? gsrc[2 * d.plane + ii] : mk((T)0, (T)0);
      const T wlive = live ? (T)1 : (T)0;  // dead lanes add nothing to the scalar gradients
#pragma unroll
      for (int e = NE - 1; e >= 0; --e) {
        const cplx<T> u0 = s0[e], u1 = s1[e], o0 = s0[e + 1], o1 = s1[e + 1], o2 = s2[e + 1];
        switch (E.kind[e]) {
          case XL_SLM: {
            gphx_acc[e] += cmulc(g0, o0).y + cmulc(g1, o1).y + cmulc(g2, o2).y;
            g0 = cmulc(g0, ph[e][0]);
            g1 = cmulc(g1, ph[e][0]);
            g2 = cmulc(g2, ph[e][0]);
            break;
          }
          case XL_SSLM: {
            gphx_acc[e] += cmulc(g0, o0).y;
            gphy_acc[e] += cmulc(g1, o1).y;
            g0 = cmulc(g0, ph[e][0]);
            g1 = cmulc(g1, ph[e][1]);
            break;
          }
          case XL_LENS: {
            int m, n;
            pix_mn(d, ii, m, n);
            const T xm = (T)d.x0 + (T)m * (T)d.dx, yn = (T)d.y0 + (T)n * (T)d.dy;
            const T coef = jt.lens_c[e] * (xm * xm + yn * yn);  // d out / d f = i coef out
            sg[e][0] += wlive * (cdot_re(g0, mk(-o0.y * coef, o0.x * coef)) +
                                 cdot_re(g1, mk(-o1.y * coef, o1.x * coef)) +
                                 cdot_re(g2, mk(-o2.y * coef, o2.x * coef)));
            cplx<T> L = lens_factor<T>(lens, E.lens_slot[e], d.params_dev ? b : 0, nlens, d, m, n);
            g0 = cmulc(g0, L);
            g1 = cmulc(g1, L);
            g2 = cmulc(g2, L);
            break;
          }
          case XL_POLARIZER: {
            sg[e][1] += wlive * jre(jt.dA[e], g0, g1, u0, u1);
            japply_h(jt.J[e], g0, g1);
            break;
          }
          case XL_WAVEPLATE: {
            sg[e][2] += wlive * jre(jt.dA[e], g0, g1, u0, u1);
            sg[e][3] += wlive * jre(jt.dB[e], g0, g1, u0, u1);
            japply_h(jt.J[e], g0, g1);
            break;
          }
          case XL_TO_VECTOR:
            g1 = mk((T)0, (T)0);
            break;
        }
      }
      if (live && gin) {
        cplx<T>* dst = gin + (int64_t)b * d.comps_in * d.plane;
        dst[i] = g0;
        if (d.comps_in >= 2) dst[d.plane + i] = g1;
        if (d.comps_in == 3) dst[2 * d.plane + i] = g2;
      }
      if (!G.accumulate_shared) {
#pragma unroll
        for (int e = 0; e < NE; ++e) {
          if (live && G.gphx[e]) ((T*)G.gphx[e])[(int64_t)b * E.phstride[e] + i] = gphx_acc[e];
          if (live && G.gphy[e]) ((T*)G.gphy[e])[(int64_t)b * E.phstride[e] + i] = gphy_acc[e];
          gphx_acc[e] = gphy_acc[e] = (T)0;
        }
      }
    }
    if (G.partial) {
      // block reduction of the scalar gradients this batch element has, fixed order; the rows
      // of parameters an element does not have get zero
      for (int e = 0; e < NE; ++e)
        for (int j = 0; j < 4; ++j) {
          double* dst = &G.partial[(((int64_t)b * E.n + e) * 4 + j) * gridDim.x + blockIdx.x];
          if (!has_scalar(E.kind[e], j)) {  // uniform over the block
            if (threadIdx.x == 0) *dst = 0.0;
            continue;
          }
          double v = (double)sg[e][j];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
          __syncthreads();
          if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
          __syncthreads();
          if (threadIdx.x == 0) {
            double s = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
            *dst = s;
          }
        }
    }
    __syncthreads();  // every thread is done with this element's Jones matrices
  }
  if (G.accumulate_shared) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < d.plane) {
#pragma unroll
      for (int e = 0; e < NE; ++e) {
        if (G.gphx[e]) ((T*)G.gphx[e])[i] = gphx_acc[e];
        if (G.gphy[e]) ((T*)G.gphy[e])[i] = gphy_acc[e];
      }
    }
  }
}

// Adjoint of a chain that is a single phase mask (an SLM, or a super-SLM with its x and y
// masks) with masks per batch element and no scalar parameters: per pixel it reads only the
// input, the cotangent and the masks (no Jones table, no per-element dispatch), with the
// arithmetic of k_elem_bwd. kPixMask pixels a thread, a compile-time count: the loads of all of
// them are issued before the first store (lanes past the plane read its last pixel and store
// nothing). grid: (ceil(plane / (256 kPixMask)), batch).
constexpr int kPixMask = 4;

template <typename T, int NC, bool SUPER>
__global__ void __launch_bounds__(256) k_mask_bwd(const cplx<T>* __restrict__ gout, const cplx<T>* __restrict__ in,
                                                  cplx<T>* __restrict__ gin, const T* __restrict__ phx,
                                                  const T* __restrict__ phy, int64_t stride,
                                                  T* __restrict__ gpx, T* __restrict__ gpy, int64_t plane) {
  const int b = blockIdx.y;
  const cplx<T>* u = in + (int64_t)b * NC * plane;
  const cplx<T>* g = gout + (int64_t)b * NC * plane;
  const T* px = phx + (int64_t)b * stride;
  const T* py = SUPER ? phy + (int64_t)b * stride : nullptr;
  cplx<T> rg[kPixMask][NC];
  T rx[kPixMask], ry[kPixMask];
#pragma unroll
  for (int k = 0; k < kPixMask; ++k) {
    const int64_t i = ((int64_t)blockIdx.x * kPixMask + k) * blockDim.x + threadIdx.x;
    const int64_t ii = i < plane ? i : plane - 1;
    T s, c;
    xsincos(__ldg(px + ii), &s, &c);
    const cplx<T> e0 = mk(c, s);
    cplx<T> e1 = e0;
    if constexpr (SUPER) {
      xsincos(__ldg(py + ii), &s, &c);
      e1 = mk(c, s);
    }
    cplx<T> uc[NC], gc[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      uc[q] = u[q * plane + ii];
      gc[q] = g[q * plane + ii];
    }
    if constexpr (SUPER) {
      // the x mask on Ex, the y mask on Ey, Ez unchanged
      rx[k] = cmulc(gc[0], cmul(uc[0], e0)).y;
      ry[k] = cmulc(gc[1], cmul(uc[1], e1)).y;
      rg[k][0] = cmulc(gc[0], e0);
      rg[k][1] = cmulc(gc[1], e1);
      if constexpr (NC == 3) rg[k][2] = gc[2];
    } else {
      T acc = cmulc(gc[0], cmul(uc[0], e0)).y;
#pragma unroll
      for (int q = 1; q < NC; ++q) acc = acc + cmulc(gc[q], cmul(uc[q], e0)).y;
      rx[k] = acc;
      ry[k] = (T)0;
#pragma unroll
      for (int q = 0; q < NC; ++q) rg[k][q] = cmulc(gc[q], e0);
    }
  }
#pragma unroll
  for (int k = 0; k < kPixMask; ++k) {
    const int64_t i = ((int64_t)blockIdx.x * kPixMask + k) * blockDim.x + threadIdx.x;
    if (i >= plane) break;
    if (gin) {
#pragma unroll
      for (int q = 0; q < NC; ++q) gin[((int64_t)b * NC + q) * plane + i] = rg[k][q];
    }
    if (gpx) gpx[(int64_t)b * stride + i] = rx[k];
    if (SUPER && gpy) gpy[(int64_t)b * stride + i] = ry[k];
  }
}

// g_params[r] = sum_k partial[r][k], r < rows (fixed order).
__global__ void k_elem_reduce(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
  __shared__ double red[32];
  const int r = blockIdx.x;
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) s += partial[(int64_t)r * nblk + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[r] = t;
  }
}

namespace {

xl_status prepare(const xl_element* el, int32_t n_el, int32_t comps_in, const xl_grid* g,
                  double wavelength, const double* params, int32_t flags, ElemSet* E, ElemDims* d,
                  int* nlens) {
  if (!g || !el || n_el < 0 || n_el > kMaxElem)
    return fail(XL_ERR_ARG, "elements: NULL grid/list or more than 8 elements");
  if (g->nx < 1 || g->ny < 1) return fail(XL_ERR_ARG, "elements: empty grid");
  if (!(wavelength > 0)) return fail(XL_ERR_ARG, "elements: wavelength must be positive");
  if (comps_in < 1 || comps_in > 3) return fail(XL_ERR_ARG, "elements: comps_in must be 1, 2 or 3");
  if (flags & ~XL_Z_DEVICE) return fail(XL_ERR_ARG, "elements: unknown flag bits");
  if ((flags & XL_Z_DEVICE) && !params) return fail(XL_ERR_ARG, "elements: device parameters are NULL");
  std::memset(E, 0, sizeof(*E));
  E->n = n_el;
  int c = comps_in;
  *nlens = 0;
  for (int e = 0; e < n_el; ++e) {
    const xl_element& x = el[e];
    E->kind[e] = x.kind;
    E->phx[e] = x.phi_x;
    E->phy[e] = x.phi_y;
    E->phstride[e] = x.phi_stride;
    E->hp[e][0] = x.f;
    E->hp[e][1] = x.alpha;
    E->hp[e][2] = x.eta;
    E->hp[e][3] = x.theta;
    E->lens_slot[e] = -1;
    switch (x.kind) {
      case XL_SLM:
        if (!x.phi_x) return fail(XL_ERR_ARG, "SLM needs phi_x");
        break;
      case XL_SSLM:
        if (c < 2) return fail(XL_ERR_ARG, "super-SLM needs a vector field");
        if (!x.phi_x || !x.phi_y) return fail(XL_ERR_ARG, "super-SLM needs phi_x and phi_y");
        break;
      case XL_LENS:
        if (!(flags & XL_Z_DEVICE) && !(x.f != 0) ) return fail(XL_ERR_ARG, "lens focal length must be non-zero");
        E->lens_slot[e] = (*nlens)++;
        break;
      case XL_POLARIZER:
      case XL_WAVEPLATE:
        if (c < 2) return fail(XL_ERR_ARG, "polariser / wave plate need a vector field");
        break;
      case XL_TO_VECTOR:
        if (c != 1) return fail(XL_ERR_ARG, "to-vector needs a 1-component field");
        c = 2;
        break;
      default:
        return fail(XL_ERR_ARG, "unknown element kind");
    }
    if (x.phi_stride < 0) return fail(XL_ERR_ARG, "phi_stride must be >= 0");
  }
  d->nx = g->nx;
  d->nx_shift = is_pow2(g->nx) ? ilog2(g->nx) : -1;
  d->ny = g->ny;
  d->comps_in = comps_in;
  d->comps_out = c;
  d->plane = (int64_t)g->nx * g->ny;
  d->x0 = g->x0;
  d->dx = g->dx;
  d->y0 = g->y0;
  d->dy = g->dy;
  d->k = kTwoPi / wavelength;
  d->params_dev = (flags & XL_Z_DEVICE) ? params : nullptr;
  return XL_OK;
}

template <typename T>
xl_status lens_tables(const ElemSet& E, const ElemDims& d, int batch, int nlens, void* buf,
                      cudaStream_t s) {
  const int64_t total = ((int64_t)d.nx + d.ny) * nlens * batch;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  LaunchScope ls("lens_tables", s);
  k_lens_tables<T><<<blocks, 256, 0, s>>>((cplx<T>*)buf, E, d, batch, nlens);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

template <typename T>
xl_status run_fwd(const void* in, void* out, int32_t batch, const ElemSet& E, const ElemDims& d,
                  int nlens, cudaStream_t s) {
  void* lens = nullptr;
  // parameters shared by the batch (host values) need one lens table per lens
  const int lb = d.params_dev ? batch : 1;
  if (nlens) {
    XL_TRY(workspace(s, ((size_t)d.nx + d.ny) * nlens * lb * sizeof(cplx<T>), &lens, 2));
    XL_TRY(lens_tables<T>(E, d, lb, nlens, lens, s));
  }
  dim3 grid((unsigned)((d.plane + 256 * kPixFwd - 1) / (256 * kPixFwd)), batch);
  LaunchScope ls("elements_fwd", s);
  k_elem_fwd<T><<<grid, 256, 0, s>>>((const cplx<T>*)in, (cplx<T>*)out, E, d, (const cplx<T>*)lens, nlens);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

template <typename T>
xl_status run_bwd(const void* gout, const void* in, void* gin, int32_t batch, const ElemSet& E,
                  const ElemDims& d, int nlens, void* const* gpx, void* const* gpy, double* gparams,
                  cudaStream_t s) {
  ElemGrad G;
  std::memset(&G, 0, sizeof(G));
  bool any_shared = false, any_batched = false;
  for (int e = 0; e < E.n; ++e) {
    G.gphx[e] = gpx ? gpx[e] : nullptr;
    G.gphy[e] = gpy ? gpy[e] : nullptr;
    if (G.gphx[e] || G.gphy[e]) (E.phstride[e] == 0 ? any_shared : any_batched) = true;
  }
  if (any_shared && any_batched && batch > 1)
    return fail(XL_ERR_UNSUPPORTED, "elements backward: mixing shared and per-batch masks");
  G.accumulate_shared = any_shared && batch > 1;
  const bool one_mask = E.n == 1 && !gparams && !G.accumulate_shared && d.comps_in == d.comps_out &&
                        (E.kind[0] == XL_SLM || (E.kind[0] == XL_SSLM && d.comps_in >= 2));
  if (one_mask) {
    dim3 grid((unsigned)((d.plane + 256 * kPixMask - 1) / (256 * kPixMask)), batch);
    LaunchScope ls("elements_bwd_mask", s);
    const bool sup = E.kind[0] == XL_SSLM;
#define XL_MBWD(NC, SUP)                                                                            \
  k_mask_bwd<T, NC, SUP><<<grid, 256, 0, s>>>((const cplx<T>*)gout, (const cplx<T>*)in, (cplx<T>*)gin, \
                                              (const T*)E.phx[0], (const T*)E.phy[0], E.phstride[0],  \
                                              (T*)G.gphx[0], (T*)G.gphy[0], d.plane)
    if (!sup && d.comps_in == 1) XL_MBWD(1, false);
    else if (!sup && d.comps_in == 2) XL_MBWD(2, false);
    else if (!sup) XL_MBWD(3, false);
    else if (d.comps_in == 2) XL_MBWD(2, true);
    else XL_MBWD(3, true);
#undef XL_MBWD
    XL_CUDA_TRY(cudaGetLastError());
    return XL_OK;
  }
  const int pix = G.accumulate_shared ? 1 : kPixBwd;
  const int nblk = (int)((d.plane + 256 * pix - 1) / (256 * pix));
  const int lb = d.params_dev ? batch : 1;
  const size_t cs = sizeof(cplx<T>);
  auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
  const size_t lens_bytes = nlens ? ((size_t)d.nx + d.ny) * nlens * lb * cs : 0;
  const size_t part_bytes = gparams ? (size_t)batch * E.n * 4 * nblk * sizeof(double) : 0;
  void* ws = nullptr;
  XL_TRY(workspace(s, al(lens_bytes) + al(part_bytes) + 256, &ws, 2));
  void* lens = ws;
  G.partial = gparams ? (double*)((char*)ws + al(lens_bytes)) : nullptr;
  if (nlens) XL_TRY(lens_tables<T>(E, d, lb, nlens, lens, s));
  dim3 grid(nblk, G.accumulate_shared ? 1 : batch);
  {
    LaunchScope ls("elements_bwd", s);
    // the forward states are recomputed only when a mask or scalar gradient is asked for
    const bool st = gparams != nullptr || any_shared || any_batched;
#define XL_EBWD(NE)                                                                                   \
  case NE:                                                                                            \
    if (st)                                                                                           \
      k_elem_bwd<T, NE, true><<<grid, 256, 0, s>>>((const cplx<T>*)gout, (const cplx<T>*)in,          \
                                                   (cplx<T>*)gin, E, d, (const cplx<T>*)lens, nlens, \
                                                   G, batch, pix);                                   \
    else                                                                                              \
      k_elem_bwd<T, NE, false><<<grid, 256, 0, s>>>((const cplx<T>*)gout, (const cplx<T>*)in,         \
                                                    (cplx<T>*)gin, E, d, (const cplx<T>*)lens, nlens, \
                                                    G, batch, pix);                                  \
    break;
    switch (E.n) {
      XL_EBWD(0) XL_EBWD(1) XL_EBWD(2) XL_EBWD(3) XL_EBWD(4) XL_EBWD(5) XL_EBWD(6) XL_EBWD(7) XL_EBWD(8)
      default: return fail(XL_ERR_ARG, "elements backward: element count");
    }
#undef XL_EBWD
    XL_CUDA_TRY(cudaGetLastError());
  }
  if (gparams && E.n > 0) {
    LaunchScope ls("elements_reduce", s);
    k_elem_reduce<<<batch * E.n * 4, 256, 0, s>>>(G.partial, nblk, gparams);
    XL_CUDA_TRY(cudaGetLastError());
  }
  return XL_OK;
}

}  // namespace
}  // namespace xl

using namespace xl;

extern "C" {

xl_status xl_apply_elements(const void* in, void* out, int32_t batch, int32_t comps_in,
                            const xl_grid* grid, double wavelength, const xl_element* elements,
                            int32_t n_elem, const double* params, int32_t flags, int32_t dtype,
                            void* stream) {
  ElemSet E;
  ElemDims d;
  int nlens = 0;
  XL_TRY(prepare(elements, n_elem, comps_in, grid, wavelength, params, flags, &E, &d, &nlens));
  if (batch < 0) return fail(XL_ERR_ARG, "batch < 0");
  if (dtype != XL_C64 && dtype != XL_C128) return fail(XL_ERR_ARG, "bad dtype");
  if (batch == 0) return XL_OK;
  if (!in || !out) return fail(XL_ERR_ARG, "field pointer is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == XL_C128 ? run_fwd<double>(in, out, batch, E, d, nlens, s)
                          : run_fwd<float>(in, out, batch, E, d, nlens, s);
}

xl_status xl_apply_elements_backward(const void* g_out, const void* in, void* g_in, int32_t batch,
                                     int32_t comps_in, const xl_grid* grid, double wavelength,
                                     const xl_element* elements, int32_t n_elem,
                                     const double* params, int32_t flags, void* const* g_phi_x,
                                     void* const* g_phi_y, double* g_params, int32_t dtype,
                                     void* stream) {
  ElemSet E;
  ElemDims d;
  int nlens = 0;
  XL_TRY(prepare(elements, n_elem, comps_in, grid, wavelength, params, flags, &E, &d, &nlens));
  if (batch < 0) return fail(XL_ERR_ARG, "batch < 0");
  if (dtype != XL_C64 && dtype != XL_C128) return fail(XL_ERR_ARG, "bad dtype");
  if (batch == 0) return XL_OK;
  if (!g_out || !in) return fail(XL_ERR_ARG, "field pointer is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == XL_C128
             ? run_bwd<double>(g_out, in, g_in, batch, E, d, nlens, g_phi_x, g_phi_y, g_params, s)
             : run_bwd<float>(g_out, in, g_in, batch, E, d, nlens, g_phi_x, g_phi_y, g_params, s);
}

}  // extern "C"
