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
// Each axis is then a linear convolution with b. The grid side (N samples) is cut into S
// segments of Ns = ceil(N / S) samples; segment s convolves with b shifted by s Ns,
//   b_s(j) = b(j - s Ns),  -(Ns - 1) <= j <= M - 1,
// evaluated as a cyclic convolution of length L = 2^ceil(log2(Ns + M - 1)), and the segments'
// spectra are summed before one inverse transform: out = IDFT(sum_s DFT(a_s) DFT(b_s) / L).
// S = 1 is the plain Bluestein method; the host picks S (and with it L) to minimise the
// (S + 1) L log2 L transform work (2048 -> 512: five transforms of 1024 instead of two of 4096).
// The two axes run as two passes (x, then y); the intermediate is stored transposed so both
// passes read rows. All chirp phases are computed in double precision and reduced modulo 2 pi
// before rounding (k_czt_tables); bhat_s = DFT_L(b_s) / L carries the 1/L of the inverse
// transform, and the y-axis post-chirp carries exp(ikz)/(i lambda z) dx dy.
//
// Vectorial CZT: Ex' = C Ex, Ey' = C Ey, and Ez' from the kernel -(offset / z) A, which by
// linearity equals -(1/z) [X_p Ex' + Y_q Ey' - C(x Ex + y Ey)]; the third transform is of
// S = x Ex + y Ey and the combination is formed in registers by the y pass.
// Adjoint: the adjoint of a cyclic convolution with spectrum bhat is the one with conj(bhat),
// so each axis transforms its window-side input once and, per segment of the grid side,
// multiplies by conj(bhat_s) and transforms back (pre-multiply conj(post), post-multiply
// conj(pre)). Vectorial adjoint: g_Ex = C^H(Gx - (X/z) Gz) + (x/z) C^H(Gz), g_Ey likewise.
//
// Distance gradient (derived here from the kernel above; the paper trains distances through
// its propagators). dA/dz = -(i k / (2 z^2)) d^2 A with d = X_p - x_m, and the prefactor gives
// (ik - 1/z), so for a cotangent G on the window
//   dL/dz = Re[(ik - 1/z) <G, U1> - (ik / (2 z^2)) (Dx + Dy)],
//   Dx = sum conj(G_qp) P A_y(q, n) d_x(p, m)^2 A_x(p, m) U0[n][m], Dy likewise with d_y.
// With p' = p - pc, m' = m - mc (pc = M/2, mc = N/2) and a = X_pc - x_mc,
//   d^2 = F(p) + G(m) + d D (j - jc)^2,  j = p - m, jc = pc - mc,
//   F(p) = a^2 + 2 a d p' + (d^2 - d D) p'^2,  G(m) = (D^2 - d D) m'^2 - 2 a D m',
// so each axis's Dx splits into (i) the window-side weight F on the product of the adjoint's
// intermediate with the forward's, (ii) the grid-side weight G on the product of the adjoint's
// output with the forward's input, and (iii) the kernel (j - jc)^2 b(j), whose term is
// sum_f conj(DFT(conj(post) W)_f) * sum_s DFT(a_s)_f DFT(b2_s)_f / L by Parseval: the adjoint's
// own first transform against a sum the forward forms from its own segment transforms (b2 =
// (j - jc)^2 b_s). The forward therefore saves its intermediate, those sums and its window field,
// and the adjoint needs no extra transform.
#pragma once

#include <cuda.h>

#include "xl_fft.cuh"

namespace xl {

// One axis of chirp tables (device, complex T). Layout of the table buffer per axis:
// pre[N] | post[M] | bhat[S][L] | b2hat[S][L] (b2hat: distance-gradient kernels; absent in the
// angular-spectrum tables).
template <typename C> struct Axis {
  const C* pre;
  const C* post;
  const C* bhat;
  const C* b2hat;
};

// Batch elements of one launch with their own distance (and so their own chirp tables).
constexpr int kCztRun = 32;

// The axis tables of every batch element of a launch: element b's tables start shift[b] elements
// after the first element's (all zero, and b unbounded, when per_elem is 0). nseg segments of seg
// samples cut the grid side of the axis.
template <typename C> struct AxisRun : Axis<C> {
  int per_elem;
  int nseg, seg;
  int64_t shift[kCztRun];
  __device__ __forceinline__ Axis<C> at(int b) const {
    const int64_t s = per_elem ? shift[b < kCztRun ? b : kCztRun - 1] : 0;
    return Axis<C>{this->pre + s, this->post + s, this->bhat + s,
                   this->b2hat ? this->b2hat + s : nullptr};
  }
};
template <typename C> inline AxisRun<C> axis_run(const Axis<C>& a, int nseg, int seg) {
  AxisRun<C> r;
  r.pre = a.pre;
  r.post = a.post;
  r.bhat = a.bhat;
  r.b2hat = a.b2hat;
  r.per_elem = 0;
  r.nseg = nseg;
  r.seg = seg;
  for (int i = 0; i < kCztRun; ++i) r.shift[i] = 0;
  return r;
}

// Distance-gradient geometry of one axis: F(p) = a2 + f1 p' + f2 p'^2 (window side, p' = p - pc),
// G(m) = g2 m'^2 + g1 m' (grid side, m' = m - mc), and the kernel weight dD = d D.
struct DzAxis {
  float a2, f1, f2, g1, g2, dD;
  int pc, mc;
};

struct CztDims {
  int nx, ny, mx, my;
  double x0, dx, y0, dy;      // input grid
  double xo0, dxo, yo0, dyo;  // output window
  const double* zdev;         // device z of the launch's single element (or nullptr)
  double z[kCztRun];          // host distance of each batch element of the launch
  int adjoint;                // 1 for the adjoint passes: the chirp spectra are conjugated
  int in_planes;              // planes per batch element of the input-grid field (fwd x input,
                              // adjoint x output): 1, 2, or 3 (a vector field whose Ez is unused)
  int64_t tb_elem;            // elements between batch elements in the intermediate T
  int accumulate;             // adjoint x pass: add to the output (and the finaliser to g_z)
  DzAxis dzx, dzy;            // distance-gradient geometry (kernels with DZ)
};

// What a forward with DZ saves per batch element (cT planes of each): the intermediate V
// [cT][mx][ny] (that is T itself: tb_elem = elem), the x sums A2x [cT][ny][Lx], the y sums
// A2y [cT][mx][Ly] and the per-plane window fields Up [cT][my][mx] (Ex', Ey', C(S) for VCZT).
template <typename C> struct CztSaved {
  C* base;
  int64_t elem, off_a2x, off_a2y, off_up;
  __device__ __forceinline__ C* a2x(int b, int c, int ny, int Lx) const {
    return base + b * elem + off_a2x + (int64_t)c * ny * Lx;
  }
  __device__ __forceinline__ C* a2y(int b, int c, int mx, int Ly) const {
    return base + b * elem + off_a2y + (int64_t)c * mx * Ly;
  }
  __device__ __forceinline__ C* up(int b, int c, int mx, int my) const {
    return base + b * elem + off_up + (int64_t)c * mx * my;
  }
};

// Launch shape of the row passes. A block holds ROWS teams of L/16 threads; the scalar passes
// use all of shared memory for the teams' transform rows. The vectorial passes carry one
// 16-element complex array per thread across transforms (the Ez accumulator of the forward y
// pass, Gz in the adjoint y pass): they run a quarter as many teams per block and keep that
// array in a thread-private shared-memory row per team when it fits (in registers otherwise),
// so that the transforms do not spill. Their loops over the 2-3 planes are unrolled on purpose:
// as runtime loops, the compiler hoisted loop-invariant work of the transforms out of them and
// spilled 400-600 bytes a thread.
// Scalar passes also build the autotuner's variants V (rows per block: 1 = half the default,
// 2 = twice the default where a block stays within 1024 threads and an SM's shared memory).
// Variants 3 and 4 keep the default rows and use radix plans 1 and 2 (xl_fft.cuh).
template <int V> __host__ __device__ constexpr int czt_plan_of() { return V >= 3 ? V - 2 : 0; }
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
// Shared-memory rows per team: the transform row, the vectorial stash (when in shared memory),
// the running sum over segments (when there is more than one), the distance-gradient sum of the
// forward passes (DZ).
template <int L, int CS, bool VEC, int V = 0>
__host__ __device__ constexpr int czt_smem_rows(bool multi_seg, bool dz_fwd) {
  return 1 + (czt_stash_smem<L, CS, VEC, V>() ? 1 : 0) + (multi_seg ? 1 : 0) + (dz_fwd ? 1 : 0);
}
template <int L, int CS, bool VEC, int V = 0>
__host__ __device__ constexpr size_t czt_smem_bytes(bool multi_seg = false, bool dz_fwd = false) {
  return (size_t)czt_rows<L, CS, VEC, V>() * czt_smem_rows<L, CS, VEC, V>(multi_seg, dz_fwd) *
         tpitch(L, CS, czt_rows<L, CS, VEC, V>()) * CS;
}
template <int L, int CS, bool VEC, int V = 0> __host__ __device__ constexpr int czt_threads() {
  return czt_rows<L, CS, VEC, V>() * (L / 16);
}
// Resident blocks per SM the register budget aims at: up to 1024 threads, as shared memory allows
// with the segment stash (and the DZ sum row of the forward passes) in place (1 KB of each
// block's shared memory is reserved by the runtime).
template <int L, int CS, bool VEC, int V = 0, bool DZ = false> __host__ __device__ constexpr int czt_min_blocks() {
  constexpr int by_threads = 1024 / czt_threads<L, CS, VEC, V>() > 1 ? 1024 / czt_threads<L, CS, VEC, V>() : 1;
  constexpr int by_smem = (int)(((size_t)228 * 1024) / (czt_smem_bytes<L, CS, VEC, V>(true, DZ) + 1024));
  return by_smem < 1 ? 1 : (by_smem < by_threads ? by_smem : by_threads);
}

// Convolution of the register row with the chirp kernel of one segment: FFT, multiply by bhat
// (conj(bhat) for the adjoint), inverse FFT. The direction is a runtime value on purpose: the
// two multiply loops become separate basic blocks, which keeps the compiler from interleaving
// the inverse transform's loads and address arithmetic into the forward transform (with both
// transforms in one block, two back-to-back transforms of length 4096 spilled about 500 bytes a
// thread at the 64-register budget that two 512-thread blocks per SM allow).
template <int L, int PLAN = 0, typename C>
__device__ __forceinline__ void chirp_conv(C (&v)[16], C* row, int t, const C* __restrict__ tw,
                                           const C* __restrict__ bhat, bool cj) {
  constexpr int TT = L / 16;
  team_fft<L, -1, PLAN>(v, row, t, tw);
  if (cj) {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = cmulc(v[q], __ldg(bhat + t + q * TT));
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = cmul(v[q], __ldg(bhat + t + q * TT));
  }
  team_fft<L, +1, PLAN>(v, row, t, tw);
}

// Segmented convolution in the forward direction (grid side in, window side out):
// v = IDFT(sum_s bhat_s DFT(a_s)), where load(s, v) fills v with segment s of the pre-chirped
// input (zero beyond the segment). With more than one segment the running sum lives in the
// thread's stash row `acc`. DZ: also a2 = sum_s b2hat_s DFT(a_s) in stash row `a2`; FUSE: both
// running sums in one loop over the samples (fewer live registers in the scalar passes; the
// vectorial ones, with more state, allocate better with two loops).
template <int L, bool DZ, int PLAN = 0, bool FUSE = true, typename C, typename Load, typename St>
__device__ __forceinline__ void seg_conv_fwd(C (&v)[16], C* row, int t, const C* __restrict__ tw,
                                             const Axis<C>& ax, int nseg, bool cj, Load&& load,
                                             St& acc, St& a2) {
  constexpr int TT = L / 16;
  load(0, v);
  team_fft<L, -1, PLAN>(v, row, t, tw);
  if constexpr (DZ) {
#pragma unroll
    for (int q = 0; q < 16; ++q) a2.set(q, cmul(v[q], __ldg(ax.b2hat + t + q * TT)));
  }
  if (cj) {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = cmulc(v[q], __ldg(ax.bhat + t + q * TT));
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = cmul(v[q], __ldg(ax.bhat + t + q * TT));
  }
  if (nseg > 1) {
#pragma unroll
    for (int q = 0; q < 16; ++q) acc.set(q, v[q]);
#pragma unroll 1
    for (int s = 1; s < nseg; ++s) {
      load(s, v);
      team_fft<L, -1, PLAN>(v, row, t, tw);
      const C* bs = ax.bhat + (int64_t)s * L;
      if constexpr (DZ) {
        const C* b2 = ax.b2hat + (int64_t)s * L;
        if constexpr (FUSE) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const C bq = __ldg(bs + t + q * TT);
            a2.set(q, cadd(a2.get(q), cmul(v[q], __ldg(b2 + t + q * TT))));
            acc.set(q, cadd(acc.get(q), cj ? cmulc(v[q], bq) : cmul(v[q], bq)));
          }
          continue;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) a2.set(q, cadd(a2.get(q), cmul(v[q], __ldg(b2 + t + q * TT))));
      }
      if (cj) {
#pragma unroll
        for (int q = 0; q < 16; ++q) acc.set(q, cadd(acc.get(q), cmulc(v[q], __ldg(bs + t + q * TT))));
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) acc.set(q, cadd(acc.get(q), cmul(v[q], __ldg(bs + t + q * TT))));
      }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = acc.get(q);
  }
  team_fft<L, +1, PLAN>(v, row, t, tw);
}

// Segmented convolution in the adjoint direction (window side in, grid side out): F = DFT(v),
// then per segment s, v = IDFT(F conj(bhat_s)) handed to store(s, v). spec(F) sees the
// transform first (the distance gradient's Parseval term). With more than one segment F is kept
// in the thread's stash row.
template <int L, int PLAN = 0, typename C, typename Spec, typename Store, typename St>
__device__ __forceinline__ void seg_conv_adj(C (&v)[16], C* row, int t, const C* __restrict__ tw,
                                             const Axis<C>& ax, int nseg, bool cj, Spec&& spec,
                                             Store&& store, St& F) {
  constexpr int TT = L / 16;
  team_fft<L, -1, PLAN>(v, row, t, tw);
  spec(v);
  if (nseg > 1) {
#pragma unroll
    for (int q = 0; q < 16; ++q) F.set(q, v[q]);
  }
#pragma unroll 1
  for (int s = 0; s < nseg; ++s) {
    if (s > 0) {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = F.get(q);
    }
    const C* bs = ax.bhat + (int64_t)s * L;
    if (cj) {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = cmulc(v[q], __ldg(bs + t + q * TT));
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = cmul(v[q], __ldg(bs + t + q * TT));
    }
    team_fft<L, +1, PLAN>(v, row, t, tw);
    store(s, v);
  }
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

// 1 / z (times sgn) of batch element b in T, the double division done once for the block (FP64
// runs at a small fraction of the FP32 rate). Every thread of the block calls it.
template <typename T>
__device__ __forceinline__ T czt_inv_z(const CztDims& d, int b, double sgn) {
  __shared__ T iz_s;
  if (threadIdx.x == 0) iz_s = (T)(sgn / czt_z(d, b));
  __syncthreads();
  return iz_s;
}

#define XL_CZT_BOUNDS(T, L, VEC, V, DZ) \
  __launch_bounds__(czt_threads<L, sizeof(cplx<T>), VEC, V>(), czt_min_blocks<L, sizeof(cplx<T>), VEC, V, DZ>())

// Coordinates of the samples a thread holds, s0 + (t + q L/16) D, as base + q step in T (one
// double-precision operation per row instead of one per sample: FP64 runs at a small fraction
// of the FP32 rate).
template <typename T> struct Coord {
  T base, step;
  __device__ __forceinline__ Coord(double s0, double D, int t, int TT)
      : base((T)(s0 + t * D)), step((T)(TT * D)) {}
  __device__ __forceinline__ T at(int q) const { return base + (T)q * step; }
};

// Shared-memory row of slot k (0: transform rows; 1..: stashes) of team `team`.
template <typename C>
__device__ __forceinline__ C* czt_slot(C* sm, int k, int rows, int P, int team) {
  return sm + ((int64_t)k * rows + team) * P;
}

// Sum of K doubles over the block (every thread passes its values; thread 0 gets the sums).
template <int K>
__device__ __forceinline__ void czt_block_sum(double (&v)[K], double* sbuf /* [32][K] */) {
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sbuf[w * K + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int i = 0; i < nw; ++i) s += sbuf[i * K + k];
      v[k] = s;
    }
}

// F(p) and G(m) of the distance gradient (see the file comment).
__device__ __forceinline__ float dz_F(const DzAxis& a, int p) {
  const float pp = (float)(p - a.pc);
  return a.a2 + pp * (a.f1 + pp * a.f2);
}
__device__ __forceinline__ float dz_G(const DzAxis& a, int m) {
  const float mm = (float)(m - a.mc);
  return mm * (a.g1 + mm * a.g2);
}
template <typename C> __device__ __forceinline__ C cfma_conj(C acc, C a, C b, float w) {
  // acc + w conj(a) b
  return mk(acc.x + w * (a.x * b.x + a.y * b.y), acc.y + w * (a.x * b.y - a.y * b.x));
}

// Forward x pass. Planes of element b: input cin (1 or 2), T planes cT (1 or 3). For VEC the
// third T plane is the transform of S = x Ex + y Ey. Segment s of a row covers x samples
// [s seg, s seg + seg).
// grid: (ceil(ny / ROWS), nbatch). T plane layout: [mx][ny] (row p holds all n).
// DZ: also stores each row's sum a2 = sum_s b2hat_s DFT(a_s) (L entries) into sv.a2x.
template <typename T, int L, bool VEC, int V = 0, bool DZ = false>
__global__ void XL_CZT_BOUNDS(T, L, VEC, V, DZ)
k_czt_fwd_x(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ Tb, CztDims d, AxisRun<cplx<T>> ax_run,
            const cplx<T>* __restrict__ tw, CztSaved<cplx<T>> sv) {
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
  const int nseg = ax_run.nseg, seg = ax_run.seg;
  const int n0 = blockIdx.x * ROWS;
  const bool live = n0 + team < d.ny;
  const int n = min(n0 + team, d.ny - 1);  // teams past the edge compute a valid row, store nothing
  const int cT = VEC ? 3 : 1;
  const int64_t plane = (int64_t)d.nx * d.ny, tplane = (int64_t)d.mx * d.ny;
  C* row = sm + team * SR;
  const int k_acc = 1 + (czt_stash_smem<L, sizeof(C), VEC, V>() ? 1 : 0);
  Stash<C, TT, true> acc, a2;
  acc.init(czt_slot(sm, k_acc, ROWS, SR, team), t);
  a2.init(czt_slot(sm, k_acc + (nseg > 1 ? 1 : 0), ROWS, SR, team), t);
  const T yn = (T)(d.y0 + n * d.dy);
  const C* s0 = in + ((int64_t)b * d.in_planes) * plane + (int64_t)n * d.nx;
  if (t == 0 && live)  // the input row, asked of L2 before the segments read it
    for (int c = 0; c < d.in_planes; ++c) prefetch_l2(s0 + c * plane, (size_t)d.nx * sizeof(C));
#pragma unroll
  for (int c = 0; c < cT; ++c) {
    C v[16];
    auto load = [&](int s, C (&u)[16]) {
      const int m0 = s * seg, ns = min(seg, d.nx - m0);
      const Coord<T> xm(d.x0 + m0 * d.dx, d.dx, t, TT);
      // the input samples first, then the chirp (one loop over both keeps twice the loads in
      // flight, and the extra registers spill in the scalar passes)
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int j = t + q * TT;
        C a = mk((T)0, (T)0);
        if (q * TT < ns && j < ns) {
          const int m = m0 + j;
          if (c < 2) a = s0[c * plane + m];
          else a = cadd(cscale(s0[m], xm.at(q)), cscale(s0[plane + m], yn));
          if constexpr (VEC) a = cmul(a, __ldg(ax.pre + m));
        }
        u[q] = a;
      }
      if constexpr (!VEC) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = t + q * TT;
          if (q * TT < ns && j < ns) u[q] = cmul(u[q], __ldg(ax.pre + m0 + j));
        }
      }
    };
    seg_conv_fwd<L, DZ, czt_plan_of<V>(), !VEC>(v, row, t, tw, ax, nseg, d.adjoint, load, acc, a2);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int p = t + q * TT;
      if (q * TT < d.mx && p < d.mx) v[q] = cmul(v[q], __ldg(ax.post + p));
    }
    if constexpr (DZ) {
      if (live) {
        C* a2d = sv.a2x(b, c, d.ny, L) + (int64_t)n * L;
#pragma unroll
        for (int q = 0; q < 16; ++q) a2d[t + q * TT] = a2.get(q);
      }
    }
    store_transposed<L, ROWS>(v, sm, team, t, d.mx, Tb + (int64_t)b * d.tb_elem + c * tplane, d.ny,
                              n0, d.ny);
  }
}

// Forward y pass: rows p of the T planes -> window planes [my][mx] (stored transposed).
// For VEC the y pass forms Ez' = -(1/z)(X_p Ex' + Y_q Ey' - S'), accumulating X_p Ex' + Y_q Ey'
// in the thread's stash. DZ: also stores each column's sum a2 (sv.a2y) and the per-plane window
// values before Ez is formed (sv.up).
// grid: (ceil(mx / ROWS), nbatch).
template <typename T, int L, bool VEC, int V = 0, bool DZ = false>
__global__ void XL_CZT_BOUNDS(T, L, VEC, V, DZ)
k_czt_fwd_y(const cplx<T>* __restrict__ Tb, cplx<T>* __restrict__ out, CztDims d, AxisRun<cplx<T>> ay_run,
            const cplx<T>* __restrict__ tw, CztSaved<cplx<T>> sv) {
  typedef cplx<T> C;
  constexpr int ROWS = czt_rows<L, sizeof(C), VEC, V>();
  static_assert(team_barriers_fit<L>(ROWS * (L / 16)), "too many teams for the named barriers");
  constexpr int TT = L / 16;
  constexpr int SR = tpitch(L, sizeof(C), ROWS);
  constexpr bool SMST = czt_stash_smem<L, sizeof(C), VEC, V>();
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int b = blockIdx.y;
  const Axis<C> ay = ay_run.at(b);
  const int nseg = ay_run.nseg, seg = ay_run.seg;
  const int p0 = blockIdx.x * ROWS;
  const bool live = p0 + team < d.mx;
  const int p = min(p0 + team, d.mx - 1);
  const int cT = VEC ? 3 : 1;
  const int64_t tplane = (int64_t)d.mx * d.ny, oplane = (int64_t)d.mx * d.my;
  C* row = sm + team * SR;
  Stash<C, TT, SMST> ez;
  ez.init(czt_slot(sm, 1, ROWS, SR, team), t);
  const int k_acc = 1 + (SMST ? 1 : 0);
  Stash<C, TT, true> acc, a2;
  acc.init(czt_slot(sm, k_acc, ROWS, SR, team), t);
  a2.init(czt_slot(sm, k_acc + (nseg > 1 ? 1 : 0), ROWS, SR, team), t);
  T Xp = (T)0, iz = (T)0;
  if constexpr (VEC) {
    Xp = (T)(d.xo0 + p * d.dxo);
    iz = czt_inv_z<T>(d, b, -1.0);
  }
  const Coord<T> yq(d.yo0, d.dyo, t, TT);
#pragma unroll
  for (int c = 0; c < cT; ++c) {
    C v[16];
    const C* src = Tb + (int64_t)b * d.tb_elem + c * tplane + (int64_t)p * d.ny;
    auto load = [&](int s, C (&u)[16]) {
      const int m0 = s * seg, ns = min(seg, d.ny - m0);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int j = t + q * TT;
        u[q] = q * TT < ns && j < ns ? cmul(src[m0 + j], __ldg(ay.pre + m0 + j)) : mk((T)0, (T)0);
      }
    };
    seg_conv_fwd<L, DZ, czt_plan_of<V>(), !VEC>(v, row, t, tw, ay, nseg, d.adjoint, load, acc, a2);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int qq = t + q * TT;
      if (q * TT < d.my && qq < d.my) v[q] = cmul(v[q], __ldg(ay.post + qq));
    }
    if constexpr (DZ) {
      if (live) {
        C* a2d = sv.a2y(b, c, d.mx, L) + (int64_t)p * L;
#pragma unroll
        for (int q = 0; q < 16; ++q) a2d[t + q * TT] = a2.get(q);
      }
      store_transposed<L, ROWS>(v, sm, team, t, d.my, sv.up(b, c, d.mx, d.my), d.mx, p0, d.mx);
    }
    if constexpr (VEC) {
      if (c == 0) {
#pragma unroll
        for (int q = 0; q < 16; ++q) ez.set(q, cscale(v[q], Xp));
      } else if (c == 1) {
#pragma unroll
        for (int q = 0; q < 16; ++q) ez.set(q, cadd(ez.get(q), cscale(v[q], yq.at(q))));
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = cscale(csub(ez.get(q), v[q]), iz);
      }
    }
    store_transposed<L, ROWS>(v, sm, team, t, d.my, out + ((int64_t)b * cT + c) * oplane, d.mx, p0,
                              d.mx);
  }
}

// Adjoint y pass: columns p of the window gradient planes [my][mx] -> T planes [mx][ny] (rows).
// VEC: T planes A = C_y^H(Gx - (X_p/z) Gz), B = C_y^H(Gy - (Y_q/z) Gz), Z = C_y^H(Gz); Gz is
// loaded once into the thread's stash.
// DZ: block partial sums [b][block][6] of E1 = <G, U1>, Dy and E0 (VCZT: <Gz, X Ex' + Y Ey' - S'>)
// from the saved forward (see the file comment); plane 2 of VCZT carries the cotangent Gz / z.
// The window-side term (i) of Dx is summed here too, into the Dy slot: it weights the same
// product of this pass's output row with the forward's T row, and the finaliser adds Dx and Dy.
// grid: (ceil(mx / ROWS), nbatch).
template <typename T, int L, bool VEC, int V = 0, bool DZ = false>
__global__ void XL_CZT_BOUNDS(T, L, VEC, V, false)
k_czt_adj_y(const cplx<T>* __restrict__ G, cplx<T>* __restrict__ Tb, CztDims d, AxisRun<cplx<T>> ay_run,
            const cplx<T>* __restrict__ tw, CztSaved<cplx<T>> sv, double* __restrict__ dzp) {
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
  const int nseg = ay_run.nseg, seg = ay_run.seg;
  const int p0 = blockIdx.x * ROWS;
  const int p = min(p0 + team, d.mx - 1);
  const bool live = p0 + team < d.mx;
  const int cT = VEC ? 3 : 1;
  const int64_t tplane = (int64_t)d.mx * d.ny, oplane = (int64_t)d.mx * d.my;
  C* row = sm + team * SR;
  Stash<C, TT, SMST> gz;
  gz.init(czt_slot(sm, 1, ROWS, SR, team), t);
  Stash<C, TT, true> F;
  F.init(czt_slot(sm, 1 + (SMST ? 1 : 0), ROWS, SR, team), t);
  T Xp = (T)0, iz = (T)0;
  if constexpr (VEC) {
    Xp = (T)(d.xo0 + p * d.dxo);
    iz = czt_inv_z<T>(d, b, 1.0);
    const C* gzsrc = G + ((int64_t)b * 3 + 2) * oplane;
    if constexpr (SMST) {
      load_rows_transposed<L, ROWS, SR>(czt_slot(sm, 1, ROWS, SR, 0), d.my, d.my, gzsrc, d.mx, p0, d.mx);
      __syncthreads();
    } else {
      load_transposed<L, ROWS>(gz.r, sm, team, t, d.my, gzsrc, d.mx, p0, d.mx);
    }
  }
  const Coord<T> yq(d.yo0, d.dyo, t, TT);
  C e1 = mk((T)0, (T)0), dy = mk((T)0, (T)0), e0 = mk((T)0, (T)0);
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
    // weight of this plane's terms in the distance gradient (VCZT plane 2: cotangent Gz / z)
    const T wc = (VEC && c == 2) ? iz : (T)1;
    if constexpr (DZ) {
      C u1[16];
      load_transposed<L, ROWS>(u1, sm, team, t, d.my, sv.up(b, c, d.mx, d.my), d.mx, p0, d.mx);
      if (live) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int qq = t + q * TT;
          if (q * TT < d.my && qq < d.my) {
            e1 = cfma_conj(e1, v[q], u1[q], (float)wc);
            dy = cfma_conj(dy, v[q], u1[q], (float)wc * dz_F(d.dzy, qq));
            if constexpr (VEC) {
              const T w = c == 0 ? Xp : (c == 1 ? yq.at(q) : (T)-1);
              e0 = cfma_conj(e0, gz.get(q), u1[q], (float)w);
            }
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int qq = t + q * TT;
      v[q] = q * TT < d.my && qq < d.my ? cmulc(v[q], __ldg(ay.post + qq)) : mk((T)0, (T)0);
    }
    C* dst = Tb + (int64_t)b * d.tb_elem + c * tplane + (int64_t)p * d.ny;
    // the forward's T row p (DZ) and the x-axis term F_x(p) of this row: the sums over the T
    // plane of both axes' separable weights are taken here, where T row p meets its cotangent
    const C* vsv = DZ ? sv.base + (int64_t)b * sv.elem + c * tplane + (int64_t)p * d.ny : nullptr;
    const float fx = DZ ? dz_F(d.dzx, p) : 0.f;
    auto spec = [&](const C (&f)[16]) {
      if constexpr (DZ) {
        if (live) {
          const C* a2 = sv.a2y(b, c, d.mx, L) + (int64_t)p * L;
          C s3 = mk((T)0, (T)0);
#pragma unroll
          for (int q = 0; q < 16; ++q) s3 = cfma_conj(s3, f[q], a2[t + q * TT], 1.f);
          dy = cadd(dy, cscale(s3, (T)d.dzy.dD * wc));
        }
      }
    };
    auto store = [&](int s, const C (&u)[16]) {
      const int m0 = s * seg, ns = min(seg, d.ny - m0);
      if (live) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = t + q * TT;
          if (q * TT < ns && j < ns) {
            const C w = cmulc(u[q], __ldg(ay.pre + m0 + j));
            dst[m0 + j] = w;
            if constexpr (DZ) dy = cfma_conj(dy, w, vsv[m0 + j], (float)wc * (dz_G(d.dzy, m0 + j) + fx));
          }
        }
      }
    };
    seg_conv_adj<L, czt_plan_of<V>()>(v, row, t, tw, ay, nseg, d.adjoint, spec, store, F);
  }
  if constexpr (DZ) {
    __shared__ double rbuf[32 * 6];
    double r[6] = {(double)e1.x, (double)e1.y, (double)dy.x, (double)dy.y, (double)e0.x, (double)e0.y};
    czt_block_sum<6>(r, rbuf);
    if (threadIdx.x == 0) {
      double* o = dzp + ((int64_t)b * gridDim.x + blockIdx.x) * 6;
#pragma unroll
      for (int k = 0; k < 6; ++k) o[k] = r[k];
    }
  }
}

// Adjoint x pass: columns n of the T planes -> input-grid gradient rows [ny][nx].
// Scalar: g = C_x^H(W). VEC: the Z plane first, writing (x/z) C_x^H(Z) and (y/z) C_x^H(Z) into
// the two output planes, then g_Ex += C_x^H(A), g_Ey += C_x^H(B) (each thread adds to the
// elements it wrote). With d.accumulate the results are added to what the output holds.
// DZ: block partial sums [b][block][2] of the grid-side term (ii) of Dx, from the forward input
// u_in and the output, and of its kernel term (iii), from the sums a2 the forward saved (see the
// file comment; the adjoint y pass takes term (i)).
// grid: (ceil(ny / ROWS), nbatch).
template <typename T, int L, bool VEC, int V = 0, bool DZ = false>
__global__ void XL_CZT_BOUNDS(T, L, VEC, V, false)
k_czt_adj_x(const cplx<T>* __restrict__ Tb, cplx<T>* __restrict__ gin, CztDims d, AxisRun<cplx<T>> ax_run,
            const cplx<T>* __restrict__ tw, CztSaved<cplx<T>> sv, double* __restrict__ dzp,
            const cplx<T>* __restrict__ u_in) {
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
  const int nseg = ax_run.nseg, seg = ax_run.seg;
  const int n0 = blockIdx.x * ROWS;
  const int n = min(n0 + team, d.ny - 1);
  const bool live = n0 + team < d.ny;
  const int cT = VEC ? 3 : 1;
  const int64_t tplane = (int64_t)d.mx * d.ny, plane = (int64_t)d.nx * d.ny;
  C* row = sm + team * SR;
  Stash<C, TT, true> F;
  F.init(czt_slot(sm, 1 + (czt_stash_smem<L, sizeof(C), VEC, V>() ? 1 : 0), ROWS, SR, team), t);
  const T yn = (T)(d.y0 + n * d.dy);
  T iz = (T)1;
  if constexpr (VEC) iz = czt_inv_z<T>(d, b, 1.0);
  C dx = mk((T)0, (T)0);

#pragma unroll
  for (int ci = 0; ci < cT; ++ci) {
    const int c = VEC ? (ci + 2) % 3 : 0;  // VEC: Z (2) first, then A (0) and B (1)
    const T wc = (VEC && c == 2) ? iz : (T)1;
    C v[16];
    load_transposed<L, ROWS>(v, sm, team, t, d.mx, Tb + (int64_t)b * d.tb_elem + c * tplane, d.ny, n0, d.ny);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int pp = t + q * TT;
      v[q] = q * TT < d.mx && pp < d.mx ? cmulc(v[q], __ldg(ax.post + pp)) : mk((T)0, (T)0);
    }
    C* d0 = gin + ((int64_t)b * d.in_planes) * plane + (int64_t)n * d.nx;
    const C* u0 = DZ ? u_in + ((int64_t)b * d.in_planes) * plane + (int64_t)n * d.nx : nullptr;
    auto spec = [&](const C (&f)[16]) {
      if constexpr (DZ) {
        if (live) {
          const C* a2 = sv.a2x(b, c, d.ny, L) + (int64_t)n * L;
          C s3 = mk((T)0, (T)0);
#pragma unroll
          for (int q = 0; q < 16; ++q) s3 = cfma_conj(s3, f[q], a2[t + q * TT], 1.f);
          dx = cadd(dx, cscale(s3, (T)d.dzx.dD * wc));
        }
      }
    };
    auto store = [&](int s, const C (&u)[16]) {
      const int m0 = s * seg, ns = min(seg, d.nx - m0);
      const Coord<T> xm(d.x0 + m0 * d.dx, d.dx, t, TT);
      if (live) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = t + q * TT;
          if (q * TT < ns && j < ns) {
            const int m = m0 + j;
            const C g = cmulc(u[q], __ldg(ax.pre + m));
            if constexpr (VEC) {
              if (c == 2) {
                const C gs = cscale(g, iz);
                const C gx = cscale(gs, xm.at(q)), gy = cscale(gs, yn);
                d0[m] = d.accumulate ? cadd(d0[m], gx) : gx;
                d0[plane + m] = d.accumulate ? cadd(d0[plane + m], gy) : gy;
              } else {
                d0[c * plane + m] = cadd(d0[c * plane + m], g);
              }
            } else {
              d0[m] = d.accumulate ? cadd(d0[m], g) : g;
            }
            if constexpr (DZ) {
              C uu;
              if (c < 2) uu = u0[c * plane + m];
              else uu = cadd(cscale(u0[m], xm.at(q)), cscale(u0[plane + m], yn));
              dx = cfma_conj(dx, g, uu, (float)wc * dz_G(d.dzx, m));
            }
          }
        }
      }
    };
    seg_conv_adj<L, czt_plan_of<V>()>(v, row, t, tw, ax, nseg, d.adjoint, spec, store, F);
  }
  if constexpr (DZ) {
    __shared__ double rbuf[32 * 2];
    double r[2] = {(double)dx.x, (double)dx.y};
    czt_block_sum<2>(r, rbuf);
    if (threadIdx.x == 0) {
      double* o = dzp + ((int64_t)b * gridDim.x + blockIdx.x) * 2;
      o[0] = r[0];
      o[1] = r[1];
    }
  }
}

// dL/dz of every batch element from the partial sums of the two adjoint passes, in fixed order
// (one block per element): dz = Re[(ik - 1/z) E1 - (ik / (2 z^2)) (Dx + Dy)] + Re(E0) / z^2;
// phase_invariant leaves out the ik E1 term (zero for losses blind to a constant phase).
static __global__ void k_czt_dz_finalize(const double* __restrict__ py, int nby, const double* __restrict__ px,
                                  int nbx, const double* zdev, CztDims d, double k, int phase_invariant,
                                  double* __restrict__ g_z) {
  __shared__ double rbuf[32 * 8];
  const int b = blockIdx.x;
  double r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < nby; i += blockDim.x)
#pragma unroll
    for (int j = 0; j < 6; ++j) r[j] += py[((int64_t)b * nby + i) * 6 + j];
  for (int i = threadIdx.x; i < nbx; i += blockDim.x) {
    r[6] += px[((int64_t)b * nbx + i) * 2];
    r[7] += px[((int64_t)b * nbx + i) * 2 + 1];
  }
  czt_block_sum<8>(r, rbuf);
  if (threadIdx.x == 0) {
    const double z = zdev ? zdev[b] : d.z[b < kCztRun ? b : kCztRun - 1];
    const double e1r = r[0], e1i = r[1], dim = r[3] + r[7], e0r = r[4];
    double v = -e1r / z + k / (2.0 * z * z) * dim + e0r / (z * z);
    if (!phase_invariant) v -= k * e1i;
    g_z[b] = d.accumulate ? g_z[b] + v : v;
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

// Chirp tables for both axes. Entries: x axis then y axis, each pre[N] | post[M] | b rows
// [S][L] | b2 rows [S][L] (b2 only with dz; the rows are transformed afterwards by k_czt_bhat).
// Double-precision phases, reduced modulo 2 pi, rounded once.
struct CztTabArgs {
  int nx, ny, mx, my, Lx, Ly;
  int Sx, Sy, segx, segy;  // segments of each axis's grid side and their length
  int dz;                  // also the distance-gradient kernels b2
  int jcx, jcy;            // centre offsets jc = M/2 - N/2 of b2 = (j - jc)^2 b
  double x0, dx, y0, dy, xo0, dxo, yo0, dyo, k, lambda;
  const double* zdev;
  double zval;
  int64_t off_y;  // element offset of the y-axis block
};

// Complex entries of one axis block of the tables.
__host__ __device__ inline int64_t czt_axis_elems(int N, int M, int L, int S, int dz) {
  return (int64_t)N + M + (int64_t)(dz ? 2 : 1) * S * L;
}

__device__ __forceinline__ double red2pi(double x) { return x - kTwoPi * rint(x * (1.0 / kTwoPi)); }

// Row entry idx of the kernel rows of one axis: row r = idx / L holds segment s = r % S (b2 for
// r >= S), entry i = idx % L the offset jj = i (i <= M - 1) or i - L, valid for
// -(ns - 1) <= jj <= M - 1 with ns the segment's length; the true offset is jt = jj - s seg.
struct SegEntry {
  bool zero, b2;
  int64_t jt;
};
__device__ __forceinline__ SegEntry seg_entry(int64_t idx, int N, int M, int L, int S, int seg) {
  const int64_t r = idx / L, i = idx % L;
  const int s = (int)(r % S);
  const int ns = min(seg, N - s * seg);
  const int64_t jj = i <= M - 1 ? i : i - L;
  return SegEntry{jj < -(int64_t)(ns - 1), r >= S, jj - (int64_t)s * seg};
}

template <typename T>
__global__ void k_czt_tables(cplx<T>* __restrict__ tab, CztTabArgs a) {
  typedef cplx<T> C;
  const double z = a.zdev ? *a.zdev : a.zval;
  const int64_t tx = czt_axis_elems(a.nx, a.mx, a.Lx, a.Sx, a.dz);
  const int64_t ty = czt_axis_elems(a.ny, a.my, a.Ly, a.Sy, a.dz);
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
    double amp = 1.0;  // real factor (y post-chirp prefactor, b2 weight)
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
        amp = a.dx * a.dy / (a.lambda * z);
      }
    } else {  // b_s (and b2_s) rows
      const SegEntry e = seg_entry(j - N - M, N, M, L, isy ? a.Sy : a.Sx, isy ? a.segy : a.segx);
      zero = e.zero;
      ph = red2pi(0.5 * alpha * (double)e.jt * (double)e.jt);
      if (e.b2) {
        const double w = (double)(e.jt - (isy ? a.jcy : a.jcx));
        amp = w * w;
      }
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

// Chirp tables of the angular-spectrum reading (the window sums of the inverse transform of a
// centred spectrum; same layout as k_czt_tables, without b2 rows). Per axis, bin m (signed index
// m' = m - N/2, frequency f = m' / (N D)), window (S0, dd), grid origin s0, beta = 2 pi dd / (N D):
//   pre(m)  = exp(i [2 pi f (S0 - s0) + beta m'^2 / 2]),
//   post(p) = exp(i beta p^2 / 2) / N,
//   b(j)    = exp(-i beta (j + N/2)^2 / 2) for -(N-1) <= j <= M-1 (segment s: b(j - s seg)),
// so that post(p) sum_m a[m] pre(m) b(p - m) = (1/N) sum_m a[m] exp(2 pi i f (X_p - s0)): the
// 1/N of the inverse transform and the phase of the grid origin are in the tables. No distance.
template <typename T>
__global__ void k_asczt_tables(cplx<T>* __restrict__ tab, CztTabArgs a) {
  typedef cplx<T> C;
  const int64_t tx = czt_axis_elems(a.nx, a.mx, a.Lx, a.Sx, 0);
  const int64_t ty = czt_axis_elems(a.ny, a.my, a.Ly, a.Sy, 0);
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
    } else {  // b_s rows
      const SegEntry e = seg_entry(j - N - M, N, M, L, isy ? a.Sy : a.Sx, isy ? a.segy : a.segx);
      zero = e.zero;
      const double o = (double)(e.jt + N / 2);
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

// In-place DFT of rows of length L (one team per row, one block per row), scaled by 1/L: the
// chirp kernels.
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
