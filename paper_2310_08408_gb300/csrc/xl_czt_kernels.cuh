// CZT / VCZT propagation kernels (Methods, "Features and performance": the chirped z-transform
// evaluates the propagation on an arbitrarily placed and sampled output window; Bluestein method).
//
// Reading: the CZT propagator is the Fresnel form of the RS integral on the output window
//   U1(X_p, Y_q) = exp(ikz)/(i lambda z) dx dy sum_{m,n} U0[n][m] A_x(p, m) A_y(q, n),
//   A(p, m) = exp(i k (X_p - x_m)^2 / (2 z)).
// With X_p = X0 + p d, x_m = x0 + m D and alpha = k d D / z, Bluestein's identity
// p m = (p^2 + m^2 - (p - m)^2) / 2 factors A(p, m) = post(p) pre(m) b(p - m):
//   pre(m)  = exp(i [k x_m^2/(2z) - (k/z) X0 m D - alpha m^2/2]),
//   post(p) = exp(i [k X_p^2/(2z) - (k/z) (X0 x0 + p d x0) - alpha p^2/2]),
//   b(j)    = exp(i alpha j^2 / 2).
// Each axis is then a linear convolution with b, evaluated as a cyclic one of length
// L = 2^ceil(log2(N + M - 1)) (zero-padded input, b placed at j mod L for -(N-1) <= j <= M-1).
// The two axes run as two passes (x, then y); the intermediate is stored transposed so both
// passes read rows. All chirp phases are computed in double precision and reduced modulo 2 pi
// before rounding (xl_czt.cu, k_czt_tables); bhat = DFT_L(b) / L carries the 1/L of the inverse
// transform, and the y-axis post-chirp carries exp(ikz)/(i lambda z) dx dy.
//
// Vectorial CZT: Ex' = C Ex, Ey' = C Ey, and Ez' from the kernel -(offset / z) A, which by
// linearity equals -(1/z) [X_p Ex' + Y_q Ey' - C(x Ex + y Ey)]; the third transform is of
// S = x Ex + y Ey and the combination is formed in registers by the y pass.
// Adjoint: each axis is the conjugate-chirp convolution of length L in the other direction
// (pre-multiply conj(post), kernel b* placed for -(M-1) <= j <= N-1, post-multiply conj(pre)).
// Because b is even in j, that kernel is b placed for the forward range, mirrored and
// conjugated, and its DFT is conj(bhat): one table per axis serves both directions.
// Vectorial adjoint: g_Ex = C^H(Gx - (X/z) Gz) + (x/z) C^H(Gz), g_Ey likewise with y.
#pragma once

#include <cuda.h>

#include "xl_fft.cuh"

namespace xl {

// One axis of chirp tables (device, complex T). Layout of the table buffer per axis:
// pre[N] | post[M] | bhat[L].
template <typename C> struct Axis {
  const C* pre;
  const C* post;
  const C* bhat;
};

// Batch elements of one launch with their own distance (and so their own chirp tables).
constexpr int kCztRun = 32;

// The axis tables of every batch element of a launch: element b's tables start shift[b] elements
// after the first element's (all zero, and b unbounded, when per_elem is 0).
template <typename C> struct AxisRun : Axis<C> {
  int per_elem;
  int64_t shift[kCztRun];
  __device__ __forceinline__ Axis<C> at(int b) const {
    const int64_t s = per_elem ? shift[b < kCztRun ? b : kCztRun - 1] : 0;
    return Axis<C>{this->pre + s, this->post + s, this->bhat + s};
  }
};
template <typename C> inline AxisRun<C> axis_run(const Axis<C>& a) {
  AxisRun<C> r;
  r.pre = a.pre;
  r.post = a.post;
  r.bhat = a.bhat;
  r.per_elem = 0;
  for (int i = 0; i < kCztRun; ++i) r.shift[i] = 0;
  return r;
}

struct CztDims {
  int nx, ny, mx, my;
  double x0, dx, y0, dy;      // input grid
  double xo0, dxo, yo0, dyo;  // output window
  const double* zdev;         // device z of the launch's single element (or nullptr)
  double z[kCztRun];          // host distance of each batch element of the launch
  int adjoint;                // 1 for the adjoint passes: the chirp spectrum is conj(bhat)
  int in_planes;              // planes per batch element of the input-grid field (fwd x input,
                              // adjoint x output): 1, 2, or 3 (a vector field whose Ez is unused)
};

// Launch shape of the row passes. A block holds ROWS teams of L/16 threads; the scalar passes
// use all of shared memory for the teams' transform rows. The vectorial passes carry one
// 16-element complex array per thread across transforms (the Ez accumulator of the forward y
// pass, Gz in the adjoint y pass, C_x^H(Z) in the adjoint x pass): they run a quarter as many teams
// per block and keep that array in a second, thread-private shared-memory row per team when it
// fits (in registers otherwise), so that the transforms do not spill. Their loops over the 2-3
// planes are unrolled on purpose: as runtime loops, the compiler hoisted loop-invariant work of
// the transforms out of them and spilled 400-600 bytes a thread.
// Scalar passes also build the autotuner's variants V (rows per block: 1 = half the default,
// 2 = twice the default where a block stays within 1024 threads and an SM's shared memory).
template <int L, int CS, bool VEC = false, int V = 0> __host__ __device__ constexpr int czt_rows() {
  constexpr int r = CS == 8 ? (L >= 4096 ? 2 : ((4096 / L) > 4 ? 4096 / L : 4))
                            : (L >= 8192 ? 1 : ((4096 / L) > 2 ? 4096 / L : 2));
  constexpr bool dbl = 2 * r * (L / 16) <= 1024 && (size_t)2 * r * tpitch(L, CS, 2 * r) * CS <= (size_t)227 * 1024 &&
                       team_barriers_fit<L>(2 * r * (L / 16));
  return VEC ? (r / 4 > 1 ? r / 4 : 1) : (V == 1 ? (r / 2 > 1 ? r / 2 : 1) : (V == 2 && dbl ? 2 * r : r));
}
template <int L, int CS, bool VEC, int V = 0> __host__ __device__ constexpr bool czt_stash_smem() {
  return VEC && (size_t)2 * czt_rows<L, CS, VEC, V>() * tpitch(L, CS, czt_rows<L, CS, VEC, V>()) * CS <= (size_t)227 * 1024;
}
template <int L, int CS, bool VEC, int V = 0> __host__ __device__ constexpr size_t czt_smem_bytes() {
  return (size_t)czt_rows<L, CS, VEC, V>() * (czt_stash_smem<L, CS, VEC, V>() ? 2 : 1) * tpitch(L, CS, czt_rows<L, CS, VEC, V>()) * CS;
}
template <int L, int CS, bool VEC, int V = 0> __host__ __device__ constexpr int czt_threads() {
  return czt_rows<L, CS, VEC, V>() * (L / 16);
}
// Resident blocks per SM the register budget aims at: up to 1024 threads, as shared memory allows
// (1 KB of each block's shared memory is reserved by the runtime).
template <int L, int CS, bool VEC, int V = 0> __host__ __device__ constexpr int czt_min_blocks() {
  constexpr int by_threads = 1024 / czt_threads<L, CS, VEC, V>() > 1 ? 1024 / czt_threads<L, CS, VEC, V>() : 1;
  constexpr int by_smem = (int)(((size_t)228 * 1024) / (czt_smem_bytes<L, CS, VEC, V>() + 1024));
  return by_smem < 1 ? 1 : (by_smem < by_threads ? by_smem : by_threads);
}

// Convolution of the register row with the chirp kernel: FFT, multiply by bhat (conj(bhat) for
// the adjoint), inverse FFT. The direction is a runtime value on purpose: the two multiply
// loops become separate basic blocks, which keeps the compiler from interleaving the inverse
// transform's loads and address arithmetic into the forward transform (with both transforms in
// one block, two back-to-back transforms of length 4096 spilled about 500 bytes a thread at the
// 64-register budget that two 512-thread blocks per SM allow).
template <int L, typename C>
__device__ __forceinline__ void chirp_conv(C (&v)[16], C* row, int t, const C* __restrict__ tw,
                                           const C* __restrict__ bhat, bool cj) {
  constexpr int TT = L / 16;
  team_fft<L, -1>(v, row, t, tw);
  if (cj) {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = cmulc(v[q], __ldg(bhat + t + q * TT));
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = cmul(v[q], __ldg(bhat + t + q * TT));
  }
  team_fft<L, +1>(v, row, t, tw);
}

// Writes the team's register row to its shared-memory row (pitch tpitch), then the block
// stores the first n_out entries of its ROWS rows transposed: dst[j * ld + c0 + r]. Ends with a
// barrier: callers that transform again reuse the same rows.
template <int L, int ROWS, typename C>
__device__ __forceinline__ void store_transposed(const C (&v)[16], C* sm, int team, int t, int n_out,
                                                 C* __restrict__ dst, int64_t ld, int c0, int n_cols) {
  constexpr int TT = L / 16;
  constexpr int P = tpitch(L, sizeof(C), ROWS);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q)
    if (q * TT < n_out) sm[team * P + spad(t + q * TT)] = v[q];  // block-uniform test
  __syncthreads();
  store_rows_transposed<L, ROWS, P>(sm, n_out, dst, ld, c0, n_cols);
  __syncthreads();
}

// Loads ROWS columns transposed: the team's row r gets src[j * ld + c0 + r] for j < n_in, into
// registers. Entries at j >= n_in are not defined (left over in shared memory): every caller
// masks them right after the load.
template <int L, int ROWS, typename C>
__device__ __forceinline__ void load_transposed(C (&v)[16], C* sm, int team, int t, int n_in,
                                                const C* __restrict__ src, int64_t ld, int c0,
                                                int n_cols) {
  constexpr int TT = L / 16;
  constexpr int P = tpitch(L, sizeof(C), ROWS);
  __syncthreads();
  load_rows_transposed<L, ROWS, P>(sm, n_in, n_in, src, ld, c0, n_cols);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q)
    v[q] = sm[team * P + spad(t + q * TT)];
  __syncthreads();
}

__device__ __forceinline__ double czt_z(const CztDims& d, int b) {
  return d.zdev ? *d.zdev : d.z[b < kCztRun ? b : kCztRun - 1];
}

#define XL_CZT_BOUNDS(T, L, VEC, V) \
  __launch_bounds__(czt_threads<L, sizeof(cplx<T>), VEC, V>(), czt_min_blocks<L, sizeof(cplx<T>), VEC, V>())

// Coordinates of the samples a thread holds, s0 + (t + q L/16) D, as base + q step in T (one
// double-precision operation per row instead of one per sample: FP64 runs at a small fraction
// of the FP32 rate).
template <typename T> struct Coord {
  T base, step;
  __device__ __forceinline__ Coord(double s0, double D, int t, int TT)
      : base((T)(s0 + t * D)), step((T)(TT * D)) {}
  __device__ __forceinline__ T at(int q) const { return base + (T)q * step; }
};

// Forward x pass. Planes of element b: input cin (1 or 2), T planes cT (1 or 3). For VEC the
// third T plane is the transform of S = x Ex + y Ey.
// grid: (ceil(ny / ROWS), nbatch). T plane layout: [mx][ny] (row p holds all n).
template <typename T, int L, bool VEC, int V = 0>
__global__ void XL_CZT_BOUNDS(T, L, VEC, V)
k_czt_fwd_x(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ Tb, CztDims d, AxisRun<cplx<T>> ax_run,
            const cplx<T>* __restrict__ tw) {
  typedef cplx<T> C;
  constexpr int ROWS = czt_rows<L, sizeof(C), VEC, V>();
  static_assert(team_barriers_fit<L>(ROWS * (L / 16)), "too many teams for the named barriers");
  constexpr int TT = L / 16;
  constexpr int SR = tpitch(L, sizeof(C), ROWS);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int b = blockIdx.y;
  const Axis<C> ax = ax_run.at(b);
  const int n0 = blockIdx.x * ROWS;
  const int n = min(n0 + team, d.ny - 1);  // teams past the edge compute a valid row, store nothing
  const int cT = VEC ? 3 : 1;
  const int64_t plane = (int64_t)d.nx * d.ny, tplane = (int64_t)d.mx * d.ny;
  C* row = sm + team * SR;
  const Coord<T> xm(d.x0, d.dx, t, TT);
  const T yn = (T)(d.y0 + n * d.dy);
#pragma unroll
  for (int c = 0; c < cT; ++c) {
    C v[16];
    const C* s0 = in + ((int64_t)b * d.in_planes) * plane + (int64_t)n * d.nx;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int m = t + q * TT;
      C a = mk((T)0, (T)0);
      if (q * TT < d.nx && m < d.nx) {
        if (c < 2) a = s0[c * plane + m];
        else a = cadd(cscale(s0[m], xm.at(q)), cscale(s0[plane + m], yn));
        a = cmul(a, __ldg(ax.pre + m));
      }
      v[q] = a;
    }
    chirp_conv<L>(v, row, t, tw, ax.bhat, d.adjoint);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int p = t + q * TT;
      if (q * TT < d.mx && p < d.mx) v[q] = cmul(v[q], __ldg(ax.post + p));
    }
    store_transposed<L, ROWS>(v, sm, team, t, d.mx, Tb + ((int64_t)b * cT + c) * tplane, d.ny, n0,
                              d.ny);
  }
}

// Forward y pass: rows p of the T planes -> window planes [my][mx] (stored transposed).
// For VEC the y pass forms Ez' = -(1/z)(X_p Ex' + Y_q Ey' - S'), accumulating X_p Ex' + Y_q Ey'
// in the thread's stash.
// grid: (ceil(mx / ROWS), nbatch).
template <typename T, int L, bool VEC, int V = 0>
__global__ void XL_CZT_BOUNDS(T, L, VEC, V)
k_czt_fwd_y(const cplx<T>* __restrict__ Tb, cplx<T>* __restrict__ out, CztDims d, AxisRun<cplx<T>> ay_run,
            const cplx<T>* __restrict__ tw) {
  typedef cplx<T> C;
  constexpr int ROWS = czt_rows<L, sizeof(C), VEC, V>();
  static_assert(team_barriers_fit<L>(ROWS * (L / 16)), "too many teams for the named barriers");
  constexpr int TT = L / 16;
  constexpr int SR = tpitch(L, sizeof(C), ROWS);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int b = blockIdx.y;
  const Axis<C> ay = ay_run.at(b);
  const int p0 = blockIdx.x * ROWS;
  const int p = min(p0 + team, d.mx - 1);
  const int cT = VEC ? 3 : 1;
  const int64_t tplane = (int64_t)d.mx * d.ny, oplane = (int64_t)d.mx * d.my;
  C* row = sm + team * SR;
  Stash<C, TT, czt_stash_smem<L, sizeof(C), VEC, V>()> acc;
  acc.init(sm + (ROWS + team) * SR, t);
  T Xp = (T)0, iz = (T)0;
  if constexpr (VEC) {
    Xp = (T)(d.xo0 + p * d.dxo);
    iz = (T)(-1.0 / czt_z(d, b));
  }
  const Coord<T> yq(d.yo0, d.dyo, t, TT);
#pragma unroll
  for (int c = 0; c < cT; ++c) {
    C v[16];
    const C* s = Tb + ((int64_t)b * cT + c) * tplane + (int64_t)p * d.ny;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int n = t + q * TT;
      v[q] = q * TT < d.ny && n < d.ny ? cmul(s[n], __ldg(ay.pre + n)) : mk((T)0, (T)0);
    }
    chirp_conv<L>(v, row, t, tw, ay.bhat, d.adjoint);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int qq = t + q * TT;
      if (q * TT < d.my && qq < d.my) v[q] = cmul(v[q], __ldg(ay.post + qq));
    }
    if constexpr (VEC) {
      if (c == 0) {
#pragma unroll
        for (int q = 0; q < 16; ++q) acc.set(q, cscale(v[q], Xp));
      } else if (c == 1) {
#pragma unroll
        for (int q = 0; q < 16; ++q) acc.set(q, cadd(acc.get(q), cscale(v[q], yq.at(q))));
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = cscale(csub(acc.get(q), v[q]), iz);
      }
    }
    store_transposed<L, ROWS>(v, sm, team, t, d.my, out + ((int64_t)b * cT + c) * oplane, d.mx, p0,
                              d.mx);
  }
}

// Scalar forward of complex64 with a row-major intermediate Tr[ny][mx] (the x pass stores each
// row's window values as they stand; the y pass gathers its columns with tiled bulk tensor
// copies). Teams per block of the x pass: one 256-thread team at L = 4096.
template <int L> __host__ __device__ constexpr int czt_rm_rows() { return (4096 / L) > 1 ? 4096 / L : 1; }

template <int L>
__global__ void __launch_bounds__(czt_rm_rows<L>() * (L / 16),
                                  (1024 / (czt_rm_rows<L>() * (L / 16))) > 0 ? 1024 / (czt_rm_rows<L>() * (L / 16)) : 1)
k_czt_fwd_x_rm(const float2* __restrict__ in, float2* __restrict__ Tr, CztDims d,
               AxisRun<float2> ax_run, const float2* __restrict__ tw) {
  constexpr int ROWS = czt_rm_rows<L>();
  constexpr int TT = L / 16;
  static_assert(team_barriers_fit<L>(ROWS * TT), "too many teams for the named barriers");
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int b = blockIdx.y;
  const Axis<float2> ax = ax_run.at(b);
  const int n_raw = blockIdx.x * ROWS + team;
  const bool live = n_raw < d.ny;
  const int n = live ? n_raw : d.ny - 1;
  const int64_t plane = (int64_t)d.nx * d.ny;
  const float2* s0 = in + ((int64_t)b * d.in_planes) * plane + (int64_t)n * d.nx;
  float2 v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int m = t + q * TT;
    v[q] = q * TT < d.nx && m < d.nx ? cmul(s0[m], __ldg(ax.pre + m)) : make_float2(0.f, 0.f);
  }
  chirp_conv<L>(v, sm + team * srow(L), t, tw, ax.bhat, d.adjoint);
  if (live) {
    float2* dst = Tr + ((int64_t)b * d.ny + n) * d.mx;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int p = t + q * TT;
      if (q * TT < d.mx && p < d.mx) dst[p] = cmul(v[q], __ldg(ax.post + p));
    }
  }
}

// The y pass of that forward: ROWS teams take window columns p0..p0+ROWS-1; one thread issues
// ceil(ny / box) tiled bulk tensor copies of W x box elements (W = max(ROWS, 2) consecutive p,
// box <= 256 rows of n) from Tr, completing on one shared-memory barrier (bounded wait: bit 1 of
// `status` and the block ends); each team reads its column from the tile, which then gives its
// memory back to the transform rows; the window values are stored transposed as before.
template <int L, int ROWS>
__global__ void __launch_bounds__(ROWS * (L / 16), (1024 / (ROWS * (L / 16))) > 0 ? 1024 / (ROWS * (L / 16)) : 1)
k_czt_fwd_y_rm(const __grid_constant__ CUtensorMap tin, float2* __restrict__ out, CztDims d,
               AxisRun<float2> ay_run, const float2* __restrict__ tw, unsigned* __restrict__ status) {
  constexpr int TT = L / 16;
  constexpr int W = ROWS >= 2 ? ROWS : 2;
  constexpr int P = tpitch(L, sizeof(float2), ROWS);
  static_assert(ROWS >= 2 && W * L <= ROWS * P, "the gathered columns fit the transform rows");
  static_assert(team_barriers_fit<L>(ROWS * TT), "too many teams for the named barriers");
  extern __shared__ __align__(128) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw + ((128u - (smem_addr(smraw) & 127u)) & 127u));
  __shared__ __align__(8) unsigned long long bar;
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int b = blockIdx.y;
  const Axis<float2> ay = ay_run.at(b);
  const int p0 = blockIdx.x * ROWS;
  const int pw0 = p0 & ~(W - 1);
  const int p = min(p0 + team, d.mx - 1);
  const int boxr = d.ny < 256 ? d.ny : 256;
  const int ncopy = (d.ny + boxr - 1) / boxr;
  const unsigned ba = smem_addr(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(ba) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(ba),
                 "r"((unsigned)(ncopy * boxr * W * sizeof(float2)))
                 : "memory");
#pragma unroll 1
    for (int c = 0; c < ncopy; ++c)
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
              "r"(smem_addr(sm + c * boxr * W)),
          "l"(reinterpret_cast<uint64_t>(&tin)), "r"(pw0), "r"(b * d.ny + c * boxr), "r"(ba)
          : "memory");
  }
  unsigned done = 0;
  for (unsigned it = 0; !done && it < kWaitLimit; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(ba)
        : "memory");
  if (__syncthreads_or(!done)) {
    if (threadIdx.x == 0) atomicOr(status, 2u);
    return;
  }
  float2 v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int n = t + q * TT;
    v[q] = q * TT < d.ny && n < d.ny ? cmul(sm[n * W + (p - pw0)], __ldg(ay.pre + n)) : make_float2(0.f, 0.f);
  }
  __syncthreads();  // every team has its column before the transforms reuse the tile's memory
  chirp_conv<L>(v, sm + team * P, t, tw, ay.bhat, d.adjoint);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int qq = t + q * TT;
    if (q * TT < d.my && qq < d.my) v[q] = cmul(v[q], __ldg(ay.post + qq));
  }
  store_transposed<L, ROWS>(v, sm, team, t, d.my, out + (int64_t)b * d.mx * d.my, d.mx, p0, d.mx);
}

// Adjoint y pass: columns p of the window gradient planes [my][mx] -> T planes [mx][ny] (rows).
// VEC: T planes A = C_y^H(Gx - (X_p/z) Gz), B = C_y^H(Gy - (Y_q/z) Gz), Z = C_y^H(Gz); Gz is
// loaded once into the thread's stash.
// grid: (ceil(mx / ROWS), nbatch).
template <typename T, int L, bool VEC, int V = 0>
__global__ void XL_CZT_BOUNDS(T, L, VEC, V)
k_czt_adj_y(const cplx<T>* __restrict__ G, cplx<T>* __restrict__ Tb, CztDims d, AxisRun<cplx<T>> ay_run,
            const cplx<T>* __restrict__ tw) {
  typedef cplx<T> C;
  constexpr int ROWS = czt_rows<L, sizeof(C), VEC, V>();
  static_assert(team_barriers_fit<L>(ROWS * (L / 16)), "too many teams for the named barriers");
  constexpr bool SMST = czt_stash_smem<L, sizeof(C), VEC, V>();
  constexpr int TT = L / 16;
  constexpr int SR = tpitch(L, sizeof(C), ROWS);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int b = blockIdx.y;
  const Axis<C> ay = ay_run.at(b);
  const int p0 = blockIdx.x * ROWS;
  const int p = min(p0 + team, d.mx - 1);
  const bool live = p0 + team < d.mx;
  const int cT = VEC ? 3 : 1;
  const int64_t tplane = (int64_t)d.mx * d.ny, oplane = (int64_t)d.mx * d.my;
  C* row = sm + team * SR;
  Stash<C, TT, SMST> gz;
  gz.init(sm + (ROWS + team) * SR, t);
  T Xp = (T)0, iz = (T)0;
  if constexpr (VEC) {
    Xp = (T)(d.xo0 + p * d.dxo);
    iz = (T)(1.0 / czt_z(d, b));
    const C* gzsrc = G + ((int64_t)b * 3 + 2) * oplane;
    if constexpr (SMST) {
      load_rows_transposed<L, ROWS, SR>(sm + ROWS * SR, d.my, d.my, gzsrc, d.mx, p0, d.mx);
      __syncthreads();
    } else {
      load_transposed<L, ROWS>(gz.r, sm, team, t, d.my, gzsrc, d.mx, p0, d.mx);
    }
  }
  const Coord<T> yq(d.yo0, d.dyo, t, TT);
#pragma unroll
  for (int c = 0; c < cT; ++c) {
    C v[16];
    if (c < 2) {
      load_transposed<L, ROWS>(v, sm, team, t, d.my, G + ((int64_t)b * cT + c) * oplane, d.mx, p0, d.mx);
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = gz.get(q);
    }
    if constexpr (VEC) {
      if (c < 2) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const T w = c == 0 ? Xp : yq.at(q);
          v[q] = csub(v[q], cscale(gz.get(q), w * iz));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int qq = t + q * TT;
      v[q] = q * TT < d.my && qq < d.my ? cmulc(v[q], __ldg(ay.post + qq)) : mk((T)0, (T)0);
    }
    chirp_conv<L>(v, row, t, tw, ay.bhat, d.adjoint);
    if (live) {
      C* dst = Tb + ((int64_t)b * cT + c) * tplane + (int64_t)p * d.ny;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int n = t + q * TT;
        if (q * TT < d.ny && n < d.ny) dst[n] = cmulc(v[q], __ldg(ay.pre + n));
      }
    }
  }
}

// Adjoint x pass: columns n of the T planes -> input-grid gradient rows [ny][nx].
// VEC: g_Ex = C_x^H(A) + (x/z) C_x^H(Z), g_Ey = C_x^H(B) + (y/z) C_x^H(Z); (1/z) C_x^H(Z) is
// transformed first and kept in the thread's stash.
// grid: (ceil(ny / ROWS), nbatch).
template <typename T, int L, bool VEC, int V = 0>
__global__ void XL_CZT_BOUNDS(T, L, VEC, V)
k_czt_adj_x(const cplx<T>* __restrict__ Tb, cplx<T>* __restrict__ gin, CztDims d, AxisRun<cplx<T>> ax_run,
            const cplx<T>* __restrict__ tw) {
  typedef cplx<T> C;
  constexpr int ROWS = czt_rows<L, sizeof(C), VEC, V>();
  static_assert(team_barriers_fit<L>(ROWS * (L / 16)), "too many teams for the named barriers");
  constexpr int TT = L / 16;
  constexpr int SR = tpitch(L, sizeof(C), ROWS);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int b = blockIdx.y;
  const Axis<C> ax = ax_run.at(b);
  const int n0 = blockIdx.x * ROWS;
  const int n = min(n0 + team, d.ny - 1);
  const bool live = n0 + team < d.ny;
  const int cT = VEC ? 3 : 1, cout = VEC ? 2 : 1;
  const int64_t tplane = (int64_t)d.mx * d.ny, plane = (int64_t)d.nx * d.ny;
  C* row = sm + team * SR;
  Stash<C, TT, czt_stash_smem<L, sizeof(C), VEC, V>()> zz;
  zz.init(sm + (ROWS + team) * SR, t);
  const Coord<T> xm(d.x0, d.dx, t, TT);
  const T yn = (T)(d.y0 + n * d.dy);
  if constexpr (VEC) {
    const T iz = (T)(1.0 / czt_z(d, b));
    C v[16];
    load_transposed<L, ROWS>(v, sm, team, t, d.mx, Tb + ((int64_t)b * 3 + 2) * tplane, d.ny, n0, d.ny);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int pp = t + q * TT;
      v[q] = q * TT < d.mx && pp < d.mx ? cmulc(v[q], __ldg(ax.post + pp)) : mk((T)0, (T)0);
    }
    chirp_conv<L>(v, row, t, tw, ax.bhat, d.adjoint);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int m = t + q * TT;
      zz.set(q, q * TT < d.nx && m < d.nx ? cscale(cmulc(v[q], __ldg(ax.pre + m)), iz) : mk((T)0, (T)0));
    }
  }
#pragma unroll
  for (int c = 0; c < cout; ++c) {
    C v[16];
    load_transposed<L, ROWS>(v, sm, team, t, d.mx, Tb + ((int64_t)b * cT + c) * tplane, d.ny, n0, d.ny);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int pp = t + q * TT;
      v[q] = q * TT < d.mx && pp < d.mx ? cmulc(v[q], __ldg(ax.post + pp)) : mk((T)0, (T)0);
    }
    chirp_conv<L>(v, row, t, tw, ax.bhat, d.adjoint);
    if (live) {
      C* dst = gin + ((int64_t)b * d.in_planes + c) * plane + (int64_t)n * d.nx;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int m = t + q * TT;
        if (q * TT < d.nx && m < d.nx) {
          C r = cmulc(v[q], __ldg(ax.pre + m));
          if constexpr (VEC) r = cadd(r, cscale(zz.get(q), c == 0 ? xm.at(q) : yn));
          dst[m] = r;
        }
      }
    }
  }
}

// Chirp tables for both axes. Entries: x axis then y axis, each pre[N] | post[M] | b[L] (b is
// transformed afterwards by k_czt_bhat). Double-precision phases, reduced modulo 2 pi, rounded
// once.
struct CztTabArgs {
  int nx, ny, mx, my, Lx, Ly;
  double x0, dx, y0, dy, xo0, dxo, yo0, dyo, k, lambda;
  const double* zdev;
  double zval;
  int64_t off_y;  // element offset of the y-axis block
};

__device__ __forceinline__ double red2pi(double x) { return x - kTwoPi * rint(x * (1.0 / kTwoPi)); }

template <typename T>
__global__ void k_czt_tables(cplx<T>* __restrict__ tab, CztTabArgs a) {
  typedef cplx<T> C;
  const double z = a.zdev ? *a.zdev : a.zval;
  const int64_t tx = (int64_t)a.nx + a.mx + a.Lx;
  const int64_t ty = (int64_t)a.ny + a.my + a.Ly;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tx + ty;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool isy = i >= tx;
    const int64_t j = isy ? i - tx : i;
    const int N = isy ? a.ny : a.nx, M = isy ? a.my : a.mx, L = isy ? a.Ly : a.Lx;
    const double s0 = isy ? a.y0 : a.x0, D = isy ? a.dy : a.dx;
    const double S0 = isy ? a.yo0 : a.xo0, dd = isy ? a.dyo : a.dxo;
    const double alpha = a.k * dd * D / z;
    double ph;
    bool zero = false;
    double amp_re = 1.0, amp_im = 0.0;  // extra complex factor (y post-chirp prefactor)
    if (j < N) {  // pre(m)
      const double m = (double)j, xm = s0 + m * D;
      ph = red2pi(a.k * xm * xm / (2.0 * z)) - red2pi(a.k / z * S0 * m * D) - red2pi(0.5 * alpha * m * m);
    } else if (j < N + M) {  // post(p)
      const double p = (double)(j - N), Xp = S0 + p * dd;
      ph = red2pi(a.k * Xp * Xp / (2.0 * z)) - red2pi(a.k / z * (S0 * s0 + p * dd * s0)) -
           red2pi(0.5 * alpha * p * p);
      if (isy) {
        // exp(ikz) / (i lambda z) dx dy = exp(i (kz - pi/2)) dx dy / (lambda z)
        ph += red2pi(a.k * z) - 0.5 * kPi;
        amp_re = a.dx * a.dy / (a.lambda * z);
      }
    } else {  // b placed mod L for -(N-1) <= jj <= M-1
      const int64_t idx = j - N - M;
      const int64_t jj = idx <= M - 1 ? idx : idx - L;
      zero = jj < -(N - 1);
      ph = red2pi(0.5 * alpha * (double)jj * (double)jj);
    }
    C v;
    if (zero) {
      v = mk((T)0, (T)0);
    } else {
      ph = red2pi(ph);
      T sn, cs;
      xsincos((T)ph, &sn, &cs);
      v = mk((T)(cs * amp_re), (T)(sn * amp_re));
      (void)amp_im;
    }
    tab[(isy ? a.off_y : 0) + j] = v;
  }
}

// Chirp tables of the angular-spectrum reading (the window sums of the inverse transform of a
// centred spectrum; same layout as k_czt_tables). Per axis, bin m (signed index m' = m - N/2,
// frequency f = m' / (N D)), window (S0, dd), grid origin s0, beta = 2 pi dd / (N D):
//   pre(m)  = exp(i [2 pi f (S0 - s0) + beta m'^2 / 2]),
//   post(p) = exp(i beta p^2 / 2) / N,
//   b(j)    = exp(-i beta (j + N/2)^2 / 2) for -(N-1) <= j <= M-1, placed mod L,
// so that post(p) sum_m a[m] pre(m) b(p - m) = (1/N) sum_m a[m] exp(2 pi i f (X_p - s0)): the
// 1/N of the inverse transform and the phase of the grid origin are in the tables. No distance.
template <typename T>
__global__ void k_asczt_tables(cplx<T>* __restrict__ tab, CztTabArgs a) {
  typedef cplx<T> C;
  const int64_t tx = (int64_t)a.nx + a.mx + a.Lx;
  const int64_t ty = (int64_t)a.ny + a.my + a.Ly;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tx + ty;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool isy = i >= tx;
    const int64_t j = isy ? i - tx : i;
    const int N = isy ? a.ny : a.nx, M = isy ? a.my : a.mx, L = isy ? a.Ly : a.Lx;
    const double s0 = isy ? a.y0 : a.x0, D = isy ? a.dy : a.dx;
    const double S0 = isy ? a.yo0 : a.xo0, dd = isy ? a.dyo : a.dxo;
    const double beta = kTwoPi * dd / ((double)N * D);
    double ph, amp = 1.0;
    bool zero = false;
    if (j < N) {  // pre(m)
      const double mp = (double)(j - N / 2);
      ph = red2pi(kTwoPi * (mp / ((double)N * D)) * (S0 - s0)) + red2pi(0.5 * beta * mp * mp);
    } else if (j < N + M) {  // post(p)
      const double p = (double)(j - N);
      ph = red2pi(0.5 * beta * p * p);
      amp = 1.0 / (double)N;
    } else {  // b placed mod L for -(N-1) <= jj <= M-1
      const int64_t idx = j - N - M;
      const int64_t jj = idx <= M - 1 ? idx : idx - L;
      zero = jj < -(N - 1);
      const double o = (double)(jj + N / 2);
      ph = -red2pi(0.5 * beta * o * o);
    }
    C v;
    if (zero) {
      v = mk((T)0, (T)0);
    } else {
      ph = red2pi(ph);
      T sn, cs;
      xsincos((T)ph, &sn, &cs);
      v = mk((T)(cs * amp), (T)(sn * amp));
    }
    tab[(isy ? a.off_y : 0) + j] = v;
  }
}

// In-place DFT of rows of length L (one team per row), scaled by 1/L: the chirp kernels.
template <typename T, int L>
__global__ void __launch_bounds__(L / 16) k_czt_bhat(cplx<T>* __restrict__ rows, int64_t stride,
                                                    const cplx<T>* __restrict__ tw) {
  typedef cplx<T> C;
  constexpr int TT = L / 16;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int t = threadIdx.x;
  C* r = rows + blockIdx.x * stride;
  C v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = r[t + q * TT];
  team_fft<L, -1>(v, sm, t, tw);
  const T s = (T)(1.0 / L);
#pragma unroll
  for (int q = 0; q < 16; ++q) r[t + q * TT] = cscale(v[q], s);
}

}  // namespace xl
