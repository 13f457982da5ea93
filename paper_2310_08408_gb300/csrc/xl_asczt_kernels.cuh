// Angular-spectrum CZT (the exact-RS reading of the CZT propagator of Hu et al., Methods,
// "Features and performance"): the spectrum of the field, times the free-space transfer function
// exp(i z kz), summed onto an arbitrary window by the two Bluestein passes of xl_czt_kernels.cuh
// (with the tables of k_asczt_tables).
//
// Spectrum passes (row length L = the field's nx or ny, no padding):
//   A: rows u[y][.] times (-1)^(x+y), forward transform, stored transposed into T[kx][y];
//   B: rows T[kx][.], forward transform, times Hc[kx][ky], stored transposed into S[ky][kx].
// The factor (-1)^(x+y) centres the spectrum: bin m holds the signed frequency index m - L/2,
// which is the index order the window passes need. Adjoints run the same steps backwards with
// transposed loads, conj(Hc), the inverse-direction transform and row stores; with a distance
// gradient the adjoint of B also transforms the forward input's T rows (pass A of u) and sums
// Re(conj(G) dHc S), dHc = i kz Hc, the derivative of the transfer function.
#pragma once

#include "xl_czt_kernels.cuh"

namespace xl {

// Per-element offsets of the transfer tables of one launch (up to kCztRun elements).
struct AsShift {
  int per_elem;
  int64_t s[kCztRun];
  __host__ __device__ __forceinline__ int64_t at(int b) const {
    return per_elem ? s[b < kCztRun ? b : kCztRun - 1] : 0;
  }
};
inline AsShift as_shared() {
  AsShift h;
  h.per_elem = 0;
  for (int i = 0; i < kCztRun; ++i) h.s[i] = 0;
  return h;
}

// Teams (rows) per block: as in the transposing RS passes, whole 32-byte sectors per column when
// possible; the adjoint with a distance gradient keeps a second row per team, so it holds half as
// many teams. Register budget: 1024 threads an SM for complex64, 512 for complex128.
template <int L, int CS, bool DZ> __host__ __device__ constexpr int as_rows() {
  constexpr int r = CS == 8 ? (L >= 8192 ? 2 : ((4096 / L) > 4 ? 4096 / L : 4))
                            : (L >= 8192 ? 1 : ((4096 / L) > 2 ? 4096 / L : 2));
  return DZ ? (r / 2 > 1 ? r / 2 : 1) : r;
}
template <int L, int CS, bool DZ> __host__ __device__ constexpr int as_min_blocks() {
  return ((CS == 8 ? 1024 : 512) / (as_rows<L, CS, DZ>() * (L / 16))) > 1
             ? (CS == 8 ? 1024 : 512) / (as_rows<L, CS, DZ>() * (L / 16))
             : 1;
}

// Transfer function of the centred spectrum: Hc[kx][ky] = exp(i z kz), dHc = i kz Hc, with
// f = (kx - nx/2) / (nx dx), g = (ky - ny/2) / (ny dy), kz = sqrt(k^2 - (2 pi f)^2 - (2 pi g)^2),
// kz = i sqrt(...) beyond the light cone (decay). Double-precision phase, reduced, rounded once.
struct AsTransferArgs {
  int nx, ny;
  double dx, dy, k;
  const double* zdev;  // device distance (or nullptr: zval)
  double zval;
};

template <typename T>
__global__ void k_as_transfer(cplx<T>* __restrict__ Hc, cplx<T>* __restrict__ dHc, AsTransferArgs a) {
  typedef cplx<T> C;
  const double z = a.zdev ? *a.zdev : a.zval;
  const int64_t n = (int64_t)a.nx * a.ny;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i / a.ny), ky = (int)(i % a.ny);
    const double f = (double)(kx - a.nx / 2) / ((double)a.nx * a.dx);
    const double g = (double)(ky - a.ny / 2) / ((double)a.ny * a.dy);
    const double s = a.k * a.k - kTwoPi * kTwoPi * (f * f + g * g);
    C h, dh;
    if (s >= 0.0) {
      const double kz = sqrt(s);
      double sn, cs;
      sincos(red2pi(z * kz), &sn, &cs);
      h = mk((T)cs, (T)sn);
      dh = mk((T)(-kz * sn), (T)(kz * cs));
    } else {
      const double kap = sqrt(-s), m = exp(-z * kap);
      h = mk((T)m, (T)0);
      dh = mk((T)(-kap * m), (T)0);
    }
    Hc[i] = h;
    if (dHc) dHc[i] = dh;
  }
}

enum { AS_STAGE_A = 0, AS_STAGE_B = 1 };

// Forward spectrum pass. in: [batch][nrows][L] rows; out: [batch][L][nrows] (transposed).
// STAGE_A multiplies the input by (-1)^(column + row); STAGE_B multiplies the transform by
// Hc[row][.] of batch element b at hs.at(b) elements from Hc (each element's distance has its
// own tables; all elements share Hc when per_elem is 0).
// grid: (ceil(nrows / ROWS), batch).
template <typename T, int L, int STAGE>
__global__ void __launch_bounds__(as_rows<L, sizeof(cplx<T>), false>() * (L / 16),
                                  as_min_blocks<L, sizeof(cplx<T>), false>())
k_as_fwd(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int nrows,
         const cplx<T>* __restrict__ Hc, AsShift hs, const cplx<T>* __restrict__ tw) {
  typedef cplx<T> C;
  constexpr int ROWS = as_rows<L, sizeof(C), false>();
  static_assert(team_barriers_fit<L>(ROWS * (L / 16)), "too many teams for the named barriers");
  constexpr int TT = L / 16;
  constexpr int P = tpitch(L, sizeof(C), ROWS);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int b = blockIdx.y;
  const int r0 = blockIdx.x * ROWS;
  const int row = min(r0 + team, nrows - 1);  // teams past the edge compute a valid row, store nothing
  const int64_t plane = (int64_t)nrows * L;
  const C* src = in + b * plane + (int64_t)row * L;
  C v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = src[t + q * TT];
  if constexpr (STAGE == AS_STAGE_A) {
    // (-1)^(column + row); L / 16 is even, so the column parity is that of t
    if ((t + row) & 1) {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = mk(-v[q].x, -v[q].y);
    }
  }
  C* rowp = sm + team * P;
  team_fft<L, -1>(v, rowp, t, tw);
  if constexpr (STAGE == AS_STAGE_B) {
    const C* h = Hc + hs.at(b) + (int64_t)row * L;
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = cmul(v[q], __ldg(h + t + q * TT));
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) rowp[spad(t + q * TT)] = v[q];
  __syncthreads();
  store_rows_transposed<L, ROWS, P>(sm, L, out + b * plane, nrows, r0, nrows);
}

// Adjoint spectrum pass. in: [batch][L][nrows] (the transposed layout); out: [batch][nrows][L].
// STAGE_B: times conj(Hc[row][.]) before the inverse-direction transform; with DZ, also
//   dz_part[b][block] = sum over the block's rows of Re(conj(G) dHc S), S the forward transform
//   of the rows TU[row][.] (pass A of the forward input).
// STAGE_A: times (-1)^(column + row) after the transform.
template <typename T, int L, int STAGE, bool DZ>
__global__ void __launch_bounds__(as_rows<L, sizeof(cplx<T>), DZ>() * (L / 16),
                                  as_min_blocks<L, sizeof(cplx<T>), DZ>())
k_as_adj(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int nrows,
         const cplx<T>* __restrict__ Hc, const cplx<T>* __restrict__ dHc, AsShift hs,
         const cplx<T>* __restrict__ TU, double* __restrict__ dz_part, const cplx<T>* __restrict__ tw) {
  typedef cplx<T> C;
  constexpr int ROWS = as_rows<L, sizeof(C), DZ>();
  static_assert(team_barriers_fit<L>(ROWS * (L / 16)), "too many teams for the named barriers");
  constexpr int TT = L / 16;
  constexpr int P = tpitch(L, sizeof(C), ROWS);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  __shared__ double red[32];
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int b = blockIdx.y;
  const int r0 = blockIdx.x * ROWS;
  const int row = min(r0 + team, nrows - 1);
  const bool live = r0 + team < nrows;
  const int64_t plane = (int64_t)nrows * L;
  C* rowp = sm + team * P;
  C v[16];
  // with DZ: U's spectrum times dHc, parked in the team's second row (thread-private entries)
  C* ur = sm + (ROWS + team) * P;
  if constexpr (DZ) {
    const C* us = TU + b * plane + (int64_t)row * L;
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = us[t + q * TT];
    team_fft<L, -1>(v, rowp, t, tw);
    const C* dh = dHc + hs.at(b) + (int64_t)row * L;
#pragma unroll
    for (int q = 0; q < 16; ++q) ur[spad(t + q * TT)] = cmul(v[q], __ldg(dh + t + q * TT));
  }
  __syncthreads();
  load_rows_transposed<L, ROWS, P>(sm, L, L, in + b * plane, nrows, r0, nrows);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = rowp[spad(t + q * TT)];
  __syncthreads();
  if constexpr (STAGE == AS_STAGE_B) {
    if constexpr (DZ) {
      T acc = (T)0;
#pragma unroll
      for (int q = 0; q < 16; ++q) acc += cdot_re(v[q], ur[spad(t + q * TT)]);
      double s = (double)(live ? acc : (T)0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) tot += red[i];
        dz_part[(int64_t)b * gridDim.x + blockIdx.x] = tot;
      }
    }
    const C* h = Hc + hs.at(b) + (int64_t)row * L;
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = cmulc(v[q], __ldg(h + t + q * TT));
  }
  team_fft<L, +1>(v, rowp, t, tw);
  if constexpr (STAGE == AS_STAGE_A) {
    if ((t + row) & 1) {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = mk(-v[q].x, -v[q].y);
    }
  }
  if (live) {
    C* dst = out + b * plane + (int64_t)row * L;
#pragma unroll
    for (int q = 0; q < 16; ++q) dst[t + q * TT] = v[q];
  }
}

// g_z[b] = sum_i part[b][i] (fixed order).
static __global__ void k_as_reduce(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[(int64_t)b * n + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) tot += red[i];
    out[b] = tot;
  }
}

}  // namespace xl
