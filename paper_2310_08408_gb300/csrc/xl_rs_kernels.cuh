// RS / VRS propagation kernels: a three-pass zero-padded 2D FFT convolution and the
// transfer-spectrum generator (Methods, "Features and performance": FFT-based numerical
// integration of the Rayleigh-Sommerfeld integral, scalar and vectorial).
//
// Layout. A field plane is [ny][nx]. The padded transform size is LX = 2 nx by LY = 2 ny. The
// intermediate after the row pass is stored transposed as T[kx][y] (LX rows of ny values): only
// the ny non-zero input rows exist, so the padded grid is never materialised (half the bytes of a
// [LY][LX] array), and at 2048^2 complex64 one plane of T (67 MB) stays resident in the 126 MB L2
// between the passes.
//   pass 1  row FFT along x of every input row (zero-padding fused into the load), store T.
//   pass 2  per kx: FFT along y (zero-padded), multiply by the spectrum, inverse FFT along y,
//           keep the first ny outputs, store in place. Spectral reductions (dz) are fused here.
//   pass 3  per y: inverse FFT along x, keep the first nx outputs (crop fused into the store).
//
// Spectra. The sampled kernels are even or odd in each offset (h even/even, h_x odd in a, h_y odd
// in b), so their DFTs have the same parity and only the quadrant kx in [0, nx], ky in [0, ny]
// is stored: Hq[kind][kx][ky], ((nx+1) x (ny+1) per kind), scaled by 1 / (LX LY) so that pass 2
// needs no separate normalisation. The generator evaluates the kernel with the phase k r
// computed in double precision as k z + k rho^2 / (r + z) (no cancellation), each term reduced
// modulo 2 pi, before a single-precision sincos; it then runs the same two-pass FFT.
#pragma once

#include <cuda.h>

#include "xl_fft.cuh"

namespace xl {

// kernel kinds (bit i of a kind mask selects spectrum i)
enum { KH = 0, KHX = 1, KHY = 2, KDH = 3, KDHX = 4, KDHY = 5, NKIND = 6 };
__host__ __device__ constexpr bool kind_odd_x(int k) { return k == KHX || k == KDHX; }
__host__ __device__ constexpr bool kind_odd_y(int k) { return k == KHY || k == KDHY; }

// Rows per block: the transposing passes (1 and 3) write/read whole 32-byte sectors per kx when
// a block holds at least 32 / sizeof(complex) rows; pass 2 aims at 256 threads per block.
// Pass 1 (and the generator's first pass): 4 rows at L = 4096 (whole sectors per kx, measured
// fastest); pass 3: 2 rows at L >= 4096 (two or more resident blocks per SM, measured fastest).
template <int L, int CS> __host__ __device__ constexpr int rows_transp() {
  return CS == 8 ? (L >= 8192 ? 2 : ((4096 / L) > 4 ? 4096 / L : 4))
                 : (L >= 8192 ? 1 : ((4096 / L) > 2 ? 4096 / L : 2));
}
template <int L, int CS> __host__ __device__ constexpr int rows_p3() {
  return CS == 8 ? (L >= 4096 ? 2 : ((4096 / L) > 4 ? 4096 / L : 4))
                 : (L >= 8192 ? 1 : ((4096 / L) > 2 ? 4096 / L : 2));
}
// Minimum resident blocks the transposing kernels ask the register allocator for: 1024 threads
// an SM for complex64 (64 registers a thread), 512 for complex128 (128 registers: an element
// takes four).
template <int THREADS, int CS> __host__ __device__ constexpr int min_blocks_rows() {
  return ((CS == 8 ? 1024 : 512) / THREADS) > 1 ? (CS == 8 ? 1024 : 512) / THREADS : 1;
}
template <int L> __host__ __device__ constexpr int rows_cols() { return (4096 / L) > 1 ? 4096 / L : 1; }

// Rows per block of autotuner variant V of a transposing pass whose default is R rows: 0 the
// default, 1 half as many, 2 twice as many when the block stays within 1024 threads, the shared
// memory of an SM and the named team barriers (otherwise the default).
template <int R, int L, int CS, int V> __host__ __device__ constexpr int rows_variant() {
  return V == 1 ? (R / 2 > 1 ? R / 2 : 1)
                : (V == 2 && 2 * R * (L / 16) <= 1024 && (size_t)2 * R * tpitch(L, CS, 2 * R) * CS <= (size_t)227 * 1024 &&
                           team_barriers_fit<L>(2 * R * (L / 16))
                       ? 2 * R
                       : R);
}
template <int L, int CS, int V> __host__ __device__ constexpr int rows_p1v() {
  return rows_variant<rows_transp<L, CS>(), L, CS, V>();
}
template <int L, int CS, int V> __host__ __device__ constexpr int rows_p3v() {
  return rows_variant<rows_p3<L, CS>(), L, CS, V>();
}

// ---------------------------------------------------------------------------------------------
// Spectrum access: value of spectrum `kind` at full-grid frequency (kx, ky), kx < LX, ky < LY.
template <typename C>
__device__ __forceinline__ C spec_at(const C* __restrict__ Hk, int kx, int ky, int nx, int ny,
                                     bool oddx, bool oddy) {
  const int LX = 2 * nx, LY = 2 * ny;
  const bool fx = kx > nx, fy = ky > ny;
  const int ax = fx ? LX - kx : kx, ay = fy ? LY - ky : ky;
  C h = __ldg(Hk + (int64_t)ax * (ny + 1) + ay);
  if ((oddx && fx) != (oddy && fy)) h = mk(-h.x, -h.y);
  return h;
}

// ---------------------------------------------------------------------------------------------
// Pass 1: row FFT (forward) of planes [ny][nx] into T[kx][y].
// Plane p of the input maps to plane (p / cin) * cT + (p % cin) of the T buffer.
template <typename T, int LX, int V = 0>
__global__ void __launch_bounds__(rows_p1v<LX, sizeof(cplx<T>), V>() * (LX / 16),
                                  min_blocks_rows<rows_p1v<LX, sizeof(cplx<T>), V>() * (LX / 16), sizeof(cplx<T>)>())
k_rs_pass1(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ Tb, int nx, int ny, int cin,
           int cT, const cplx<T>* __restrict__ tw) {
  typedef cplx<T> C;
  constexpr int ROWS = rows_p1v<LX, sizeof(C), V>();
  static_assert(team_barriers_fit<LX>(ROWS * (LX / 16)), "too many teams for the named barriers");
  constexpr int TT = LX / 16;
  constexpr int P = tpitch(LX, sizeof(C), ROWS);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int p = blockIdx.y;
  const int y0 = blockIdx.x * ROWS;
  const int y = y0 + team;
  const C* src = in + (int64_t)p * nx * ny + (int64_t)y * nx;
  C* dst = Tb + ((int64_t)(p / cin) * cT + (p % cin)) * (int64_t)LX * ny;
  C v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = (q < 8 && y < ny) ? src[t + q * TT] : mk((T)0, (T)0);
  C* row = sm + team * P;
  team_fft<LX, -1, 0, PRUNE_IN>(v, row, t, tw);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) row[spad(t + q * TT)] = v[q];
  __syncthreads();
  store_rows_transposed<LX, ROWS, P>(sm, LX, dst, ny, y0, ny);
}

// Pass 1 into the row-major intermediate Tr[plane][y][kx] (complex64; read by pass 2 through
// bulk tensor copies): one row per team, the transform's registers stored straight to the row.
template <int LX>
__global__ void __launch_bounds__(rows_cols<LX>() * (LX / 16),
                                  (1024 / (rows_cols<LX>() * (LX / 16))) > 0 ? 1024 / (rows_cols<LX>() * (LX / 16)) : 1)
k_rs_pass1_rm(const float2* __restrict__ in, float2* __restrict__ Tr, int nx, int ny, int cin,
              int cT, const float2* __restrict__ tw) {
  constexpr int ROWS = rows_cols<LX>();
  constexpr int TT = LX / 16;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int p = blockIdx.y;
  const int y_raw = blockIdx.x * ROWS + team;
  const bool live = y_raw < ny;
  const int y = live ? y_raw : ny - 1;  // dead teams transform a valid row and store nothing
  const float2* src = in + (int64_t)p * nx * ny + (int64_t)y * nx;
  float2 v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = q < 8 ? src[t + q * TT] : make_float2(0.f, 0.f);
  team_fft<LX, -1, 0, PRUNE_IN>(v, sm + team * srow(LX), t, tw);
  if (live) {
    float2* d = Tr + ((int64_t)(p / cin) * cT + (p % cin)) * (int64_t)LX * ny + (int64_t)y * LX;
#pragma unroll
    for (int q = 0; q < 16; ++q) d[t + q * TT] = v[q];
  }
}

// Block-wide sum of a double (one value per thread) -> thread 0; sbuf holds 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sbuf) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sbuf[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) s += sbuf[i];
  return s;
}

// Optional fixed-order reduction of the pass-2 distance partials, done by the blocks of
// column 0 of pass 3 (which runs right after pass 2 on the same stream):
// out[b] = sum_i part[b * n + i] for the batch element b of the block's plane.
struct DzReduce {
  const double* part;
  int n;
  double* out;
};

// Pass 3: inverse row FFT from T[kx][y] into planes [ny][nx] (crop to x < nx).
// Plane p of the output maps to plane (p / cout) * cT + (p % cout) of T.
template <typename T, int LX, int V = 0>
__global__ void __launch_bounds__(rows_p3v<LX, sizeof(cplx<T>), V>() * (LX / 16),
                                  min_blocks_rows<rows_p3v<LX, sizeof(cplx<T>), V>() * (LX / 16), sizeof(cplx<T>)>())
k_rs_pass3(const cplx<T>* __restrict__ Tb, cplx<T>* __restrict__ out, int nx, int ny, int cout,
           int cT, const cplx<T>* __restrict__ tw, DzReduce red) {
  typedef cplx<T> C;
  constexpr int ROWS = rows_p3v<LX, sizeof(C), V>();
  static_assert(team_barriers_fit<LX>(ROWS * (LX / 16)), "too many teams for the named barriers");
  constexpr int TT = LX / 16;
  constexpr int P = tpitch(LX, sizeof(C), ROWS);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int p = blockIdx.y;
  const int y0 = blockIdx.x * ROWS;
  if (red.part != nullptr && blockIdx.x == 0 && p % cout == 0) {
    __shared__ double rbuf[32];
    const int b = p / cout;
    double acc = 0.0;
    for (int i = threadIdx.x; i < red.n; i += blockDim.x) acc += red.part[(int64_t)b * red.n + i];
    acc = block_sum(acc, rbuf);
    if (threadIdx.x == 0) red.out[b] = acc;
  }
  const C* src = Tb + ((int64_t)(p / cout) * cT + (p % cout)) * (int64_t)LX * ny;
  load_rows_transposed<LX, ROWS, P, C, true>(sm, LX, LX, src, ny, y0, ny);
  __syncthreads();
  C* row = sm + team * P;
  C v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = row[spad(t + q * TT)];
  __syncthreads();
  team_fft<LX, +1, 0, PRUNE_OUT>(v, row, t, tw);
  const int y = y0 + team;
  if (y < ny) {
    C* d = out + (int64_t)p * nx * ny + (int64_t)y * nx;
#pragma unroll
    for (int q = 0; q < 8; ++q) d[t + q * TT] = v[q];
  }
}

// Pass 3 for complex64 with the gather done by the tensor-memory accelerator: one thread issues
// LX / 256 tiled bulk copies of a box of 2 y by 256 kx each (4 KB; the tensor map sees T as rows
// of ny 8-byte elements, one row per kx of every plane), completing on one shared-memory barrier.
// The tile lands kx-major ([kx][2 y]), is read into registers and the same shared memory then
// serves as the two transform rows. Two rows per block, as the asynchronous-copy gather.
// A wait that does not complete within a bound sets bit 1 of `status` and ends the block.
constexpr int kP3TmaRows = 2;

template <int LX>
__global__ void __launch_bounds__(kP3TmaRows * (LX / 16), min_blocks_rows<kP3TmaRows * (LX / 16), 8>())
k_rs_pass3_tma(const __grid_constant__ CUtensorMap tmap, float2* __restrict__ out, int nx, int ny,
               int cout, int cT, const float2* __restrict__ tw, DzReduce red,
               unsigned* __restrict__ status) {
  typedef float2 C;
  constexpr int ROWS = kP3TmaRows;
  constexpr int TT = LX / 16;
  constexpr int NCOPY = LX / 256;
  static_assert(ROWS * LX <= ROWS * srow(LX), "the gathered tile fits the transform rows");
  extern __shared__ __align__(128) unsigned char smraw[];
  // bulk tensor copies land on 128-byte boundaries: the launch adds 128 bytes for the shift
  C* sm = reinterpret_cast<C*>(smraw + ((128u - (smem_addr(smraw) & 127u)) & 127u));
  __shared__ __align__(8) unsigned long long bar;
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int p = blockIdx.y;
  const int y0 = blockIdx.x * ROWS;
  if (red.part != nullptr && blockIdx.x == 0 && p % cout == 0) {
    __shared__ double rbuf[32];
    const int b = p / cout;
    double acc = 0.0;
    for (int i = threadIdx.x; i < red.n; i += blockDim.x) acc += red.part[(int64_t)b * red.n + i];
    acc = block_sum(acc, rbuf);
    if (threadIdx.x == 0) red.out[b] = acc;
  }
  const unsigned ba = smem_addr(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(ba) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(ba),
                 "r"((unsigned)(NCOPY * 256 * ROWS * sizeof(C)))
                 : "memory");
    const int row0 = ((p / cout) * cT + (p % cout)) * LX;  // first kx row of the T plane
#pragma unroll 1
    for (int c = 0; c < NCOPY; ++c)
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
              "r"(smem_addr(sm + c * 256 * ROWS)),
          "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(y0), "r"(row0 + c * 256), "r"(ba)
          : "memory");
  }
  unsigned done = 0;
  for (unsigned it = 0; !done && it < kWaitLimit; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(ba)
        : "memory");
  if (__syncthreads_or(!done)) {  // the whole block gives up together
    if (threadIdx.x == 0) atomicOr(status, 2u);
    return;
  }
  C v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = sm[(t + q * TT) * ROWS + team];
  __syncthreads();  // every thread has its inputs before the transforms reuse the tile's memory
  team_fft<LX, +1, 0, PRUNE_OUT>(v, sm + team * srow(LX), t, tw);
  const int y = y0 + team;
  if (y < ny) {
    C* d = out + (int64_t)p * nx * ny + (int64_t)y * nx;
#pragma unroll
    for (int q = 0; q < 8; ++q) d[t + q * TT] = v[q];
  }
}

// ---------------------------------------------------------------------------------------------
// Pass 2 modes.
enum {
  P2_RS = 0,        // T0 <- IFFT(FFT(T0) * S0)                      (S0 = H or conj H)
  P2_VRS = 1,       // T0,T1,T2 <- from T0,T1: x*Hz, y*Hz, x*Hx + y*Hy
  P2_RS_BWD = 2,    // T0 <- IFFT(FFT(T0) conj Hz); dz partial from T0, U0 (optional)
  P2_VRS_BWD = 3,   // T0,T1 <- from T0,T1,T2 (gx, gy, gz) with conj spectra; dz from U0,U1
  P2_RS_BWD_S = 4,  // P2_RS_BWD with U's column spectra read from saved spectra (no transform)
  P2_VRS_BWD_S = 5, // P2_VRS_BWD likewise
};

// Batch elements of one pass-2 launch with their own distance (and so their own spectra).
constexpr int kP2Run = 32;

struct P2Args {
  int nx, ny;
  int64_t t_plane;      // elements of one T plane (LX * ny)
  int64_t hq_kind;      // elements of one spectrum quadrant ((nx+1)(ny+1))
  int cT;               // T planes per batch element
  int cU;               // U planes per batch element (dz)
  int want_field;       // write the field result (backward: g_in requested)
  int want_dz;          // accumulate the dz partials
  int conj;             // P2_RS: use conj(H) (adjoint without dz)
  int slot[NKIND];      // spectrum kind -> slot in the Hq buffer (-1: absent)
  void* spec_out;       // forward modes: also store the input planes' column spectra (before
                        // the transfer spectrum) here, [b][cS][LX][LY] (nullable)
  const void* spec_in;  // *_BWD_S modes: U's column spectra saved by a forward, same layout
  int cS;               // planes per batch element of spec_out / spec_in
  int per_elem;         // 1: element b's spectra start hshift[b] elements after Hq (its own
                        // distance); 0: every element uses Hq
  int64_t hshift[kP2Run];
  unsigned* status;     // device status word (bulk-copy gather of row-major input)
};

// Spectrum `Hk` along one kx row at ky = t + q TT (TT = LY / 16, ny = 8 TT): the quadrant row
// ax = mirror(kx) is fixed per row; ky mirrors for q > 8 (and for q == 8 when t > 0).
template <typename C>
__device__ __forceinline__ C spec_row(const C* __restrict__ hrow, int q, int t, int TT, bool flipx,
                                      bool oddx, bool oddy) {
  bool fy;
  int ay;
  if (q < 8) {  // q is a compile-time constant after unrolling
    fy = false;
    ay = t + q * TT;
  } else if (q == 8) {
    fy = t > 0;
    ay = fy ? 8 * TT - t : 8 * TT;
  } else {
    fy = true;
    ay = (16 - q) * TT - t;
  }
  C h = __ldg(hrow + ay);
  if ((oddx && flipx) != (oddy && fy)) h = mk(-h.x, -h.y);
  return h;
}

// Block-scope memory fence placed after a transform: memory operations are not moved across
// it, so the compiler cannot pull the next transform's loads and stores (and the registers they
// hold) into this one. In the vectorial forward pass, five transforms in one block otherwise
// spilled 424 bytes a thread at 128 registers.
__device__ __forceinline__ void transform_fence() { __threadfence_block(); }

// Compiler-only memory fence: keeps the spectrum loads of the multiply loops in groups of four
// (without it all 16-32 loads are hoisted ahead of the arithmetic and the registers spill).
#define XL_GROUP_FENCE(q) \
  if (((q) & 3) == 3) asm volatile("" ::: "memory")

template <typename C>
__device__ __forceinline__ void load_col(C (&v)[16], const C* __restrict__ src, int t, int TT) {
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = q < 8 ? src[t + q * TT] : mk((decltype(v[0].x))0, (decltype(v[0].x))0);
}
template <typename C>
__device__ __forceinline__ void store_col(const C (&v)[16], C* __restrict__ dst, int t, int TT) {
#pragma unroll
  for (int q = 0; q < 8; ++q) dst[t + q * TT] = v[q];
}
template <typename C>
__device__ __forceinline__ void store_full(const C (&v)[16], C* __restrict__ dst, int t, int TT) {
#pragma unroll
  for (int q = 0; q < 16; ++q) dst[t + q * TT] = v[q];
}

// Column gather of pass 2 from the row-major layout Tr[plane][y][kx] that pass 1 writes for the
// scalar forward and saved-spectrum adjoint (complex64): one thread issues ny / box tiled bulk
// tensor copies of W x box elements (W = max(ROWS, 2) consecutive kx, box <= 256 rows of y)
// completing on one shared-memory barrier; each team reads its kx from the tile, which then
// gives its memory back to the transform rows. Returns false (every thread of the block) when the
// bounded wait gave up; bit 1 of `status` is set.
// Column group of a pass-2 block. With PAIR, groups run in the order 0, n-1, 1, n-2, 2, ...: the
// columns kx and LX - kx read the same spectrum rows (the quadrant's mirror), so the second read
// finds them in L2. It pays in the modes that read several spectra (measured: the saved-spectrum
// adjoint 1.47 -> 1.44 ms a step; the forward, one spectrum, 1.29 -> 1.31 ms: launch order there).
template <bool PAIR> __device__ __forceinline__ int p2_group() {
  if constexpr (!PAIR) return (int)blockIdx.x;
  const int ng = (int)gridDim.x, i = (int)blockIdx.x;
  return (i & 1) ? ng - (i + 1) / 2 : i / 2;
}

template <int LY, int ROWS>
__device__ __forceinline__ bool gather_col_rm(float2 (&v)[16], float2* tile, const CUtensorMap& map,
                                              unsigned long long* bar, int kx, int gx, int row0,
                                              int ny, int t, unsigned* status) {
  constexpr int TT = LY / 16;
  constexpr int W = ROWS >= 2 ? ROWS : 2;
  const int kx0 = (gx * ROWS) & ~(W - 1);  // first column of the block's group gx
  const int boxr = ny < 256 ? ny : 256;
  const int ncopy = ny / boxr;
  const unsigned ba = smem_addr(bar);
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
              "r"(smem_addr(tile + c * boxr * W)),
          "l"(reinterpret_cast<uint64_t>(&map)), "r"(kx0), "r"(row0 + c * boxr), "r"(ba)
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
    return false;
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = q < 8 ? tile[(t + q * TT) * W + (kx - kx0)] : make_float2(0.f, 0.f);
  __syncthreads();  // every team has its column before the transforms reuse the tile's memory
  return true;
}

// Blocks per SM the register budget of each pass-2 mode aims at (256-thread blocks).
template <int MODE> __host__ __device__ constexpr int p2_min_blocks() {
  return MODE == P2_RS || MODE == P2_RS_BWD_S ? 4 : (MODE == P2_RS_BWD ? 3 : 2);
}
// Shared-memory rows per team of each mode. VRS modes keep the Ez or Gz spectrum in a second
// row; the adjoints with a distance gradient park U's column spectrum (times the dz spectrum for
// the scalar adjoint) in one more row when it fits in an SM's shared memory (in registers
// otherwise), so that one 16-element array is live per transform.
template <typename T, int LY, int MODE> __host__ __device__ constexpr bool p2_ustash_smem() {
  return (MODE == P2_RS_BWD || MODE == P2_VRS_BWD) &&
         (size_t)(MODE == P2_RS_BWD ? 2 : 3) * rows_cols<LY>() * srow(LY) * sizeof(cplx<T>) <=
             (size_t)227 * 1024;
}
template <typename T, int LY, int MODE> __host__ __device__ constexpr int p2_rows_per_team() {
  return (MODE == P2_VRS || MODE == P2_VRS_BWD || MODE == P2_VRS_BWD_S ? 2 : 1) +
         (p2_ustash_smem<T, LY, MODE>() ? 1 : 0);
}

// grid: (ceil(LX / ROWS), nbatch). Hq: spectra [slots][nx+1][ny+1].
// dz_part: [nbatch][gridDim.x] partial sums, reduced later in fixed order.
// Resident blocks of a pass-2 launch the register budget aims at (halved for complex128).
template <typename T, int LY, int MODE> __host__ __device__ constexpr int p2_launch_min_blocks() {
  return (p2_min_blocks<MODE>() * 256 / (int)(sizeof(T) / 4)) / (rows_cols<LY>() * (LY / 16)) > 0
             ? (p2_min_blocks<MODE>() * 256 / (int)(sizeof(T) / 4)) / (rows_cols<LY>() * (LY / 16))
             : 1;
}

// RM: the input columns (T0 of the scalar forward and saved-spectrum adjoint, complex64) come
// from the row-major intermediate through the tensor map `tin` (gather_col_rm); the results go
// to the column-major Tb as usual.
template <typename T, int LY, int MODE, bool RM = false>
__global__ void __launch_bounds__(rows_cols<LY>() * (LY / 16), p2_launch_min_blocks<T, LY, MODE>())
k_rs_pass2(cplx<T>* __restrict__ Tb, const cplx<T>* __restrict__ Ub, const cplx<T>* __restrict__ Hq,
           double* __restrict__ dz_part, P2Args a, const cplx<T>* __restrict__ tw,
           const __grid_constant__ CUtensorMap tin) {
  typedef cplx<T> C;
  constexpr int ROWS = rows_cols<LY>();
  static_assert(team_barriers_fit<LY>(ROWS * (LY / 16)), "too many teams for the named barriers");
  constexpr int TT = LY / 16;
  constexpr int SR = srow(LY);
  extern __shared__ __align__(128) unsigned char smraw[];
  // with RM the tile of the bulk copies starts on a 128-byte boundary (the launch adds 128 bytes)
  C* sm = reinterpret_cast<C*>(RM ? smraw + ((128u - (smem_addr(smraw) & 127u)) & 127u) : smraw);
  __shared__ __align__(8) unsigned long long rm_bar;
  __shared__ double red[32];
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int LX = 2 * a.nx;
  constexpr bool PAIR = MODE != P2_RS;
  const int gx = p2_group<PAIR>();
  const int kx_raw = gx * ROWS + team;
  const bool live = kx_raw < LX;
  const int kx = live ? kx_raw : LX - 1;  // dead teams run the same code on a valid row, no stores
  const int b = blockIdx.y;
  C* row = sm + team * SR;
  C* T0 = Tb + (int64_t)b * a.cT * a.t_plane + (int64_t)kx * a.ny;
  const bool flipx = kx > a.nx;
  const int64_t hrow_off = (int64_t)(flipx ? LX - kx : kx) * (a.ny + 1);
  const cplx<T>* Hqb = Hq + (a.per_elem ? a.hshift[b < kP2Run ? b : kP2Run - 1] : 0);
  auto H = [&](int kind) { return Hqb + a.slot[kind] * a.hq_kind + hrow_off; };
  C v[16];
  double dz = 0.0;

  // saved column spectra: [b][cS][LX][LY], column kx of plane c
  const int64_t spec_plane = (int64_t)LX * LY;
  auto spec_out = [&](int c) {
    return reinterpret_cast<C*>(a.spec_out) + ((int64_t)b * a.cS + c) * spec_plane + (int64_t)kx * LY;
  };
  auto spec_in = [&](int c) {
    return reinterpret_cast<const C*>(a.spec_in) + ((int64_t)b * a.cS + c) * spec_plane + (int64_t)kx * LY;
  };
  // One thread of the team asks L2 for the spectrum rows and saved spectra this column reads
  // after its first transform, so that those loads do not wait on DRAM.
  if (t == 0) {
    const size_t row_bytes = (size_t)(a.ny + 1) * sizeof(C), col_bytes = (size_t)LY * sizeof(C);
    auto pf = [&](int kind) { prefetch_l2(H(kind), row_bytes); };
    if constexpr (MODE == P2_RS) {
      pf(KH);
    } else if constexpr (MODE == P2_VRS) {
      pf(KH); pf(KHX); pf(KHY);
    } else if constexpr (MODE == P2_RS_BWD_S) {
      if (a.want_dz) { prefetch_l2(spec_in(0), col_bytes); pf(KDH); }
      if (a.want_field) pf(KH);
    } else if constexpr (MODE == P2_VRS_BWD_S) {
      if (a.want_dz) {
        prefetch_l2(spec_in(0), col_bytes); prefetch_l2(spec_in(1), col_bytes);
        pf(KDH); pf(KDHX); pf(KDHY);
      }
      if (a.want_field) { pf(KH); pf(KHX); pf(KHY); }
    }
  }
  if constexpr (MODE == P2_RS) {
    if constexpr (RM) {
      if (!gather_col_rm<LY, ROWS>(v, sm, tin, &rm_bar, kx, gx, b * a.cT * a.ny, a.ny, t, a.status)) return;
    } else {
      load_col(v, T0, t, TT);
    }
    team_fft<LY, -1, 0, PRUNE_IN>(v, row, t, tw);
    if (a.spec_out && live) store_full(v, spec_out(0), t, TT);
    const C* h = H(KH);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const C hv = spec_row(h, q, t, TT, flipx, false, false);
      v[q] = a.conj ? cmulc(v[q], hv) : cmul(v[q], hv);
    }
    team_fft<LY, +1, 0, PRUNE_OUT>(v, row, t, tw);
    if (live) store_col(v, T0, t, TT);
  } else if constexpr (MODE == P2_VRS) {
    // Ez accumulates in a second shared-memory row of the team (each thread touches only its
    // own elements t + q TT, so no synchronisation is needed for it).
    C* T1 = T0 + a.t_plane;
    C* T2 = T1 + a.t_plane;
    C* zr = sm + ROWS * SR + team * SR;
    const C *hz = H(KH), *hx = H(KHX), *hy = H(KHY);
    load_col(v, T0, t, TT);
    team_fft<LY, -1, 0, PRUNE_IN>(v, row, t, tw);
    if (a.spec_out && live) store_full(v, spec_out(0), t, TT);
    transform_fence();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      zr[spad(t + q * TT)] = cmul(v[q], spec_row(hx, q, t, TT, flipx, true, false));
      v[q] = cmul(v[q], spec_row(hz, q, t, TT, flipx, false, false));
      XL_GROUP_FENCE(q);
    }
    team_fft<LY, +1, 0, PRUNE_OUT>(v, row, t, tw);
    transform_fence();
    if (live) store_col(v, T0, t, TT);
    load_col(v, T1, t, TT);
    team_fft<LY, -1, 0, PRUNE_IN>(v, row, t, tw);
    if (a.spec_out && live) store_full(v, spec_out(1), t, TT);
    transform_fence();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int iz = spad(t + q * TT);
      zr[iz] = cadd(zr[iz], cmul(v[q], spec_row(hy, q, t, TT, flipx, false, true)));
      v[q] = cmul(v[q], spec_row(hz, q, t, TT, flipx, false, false));
      XL_GROUP_FENCE(q);
    }
    team_fft<LY, +1, 0, PRUNE_OUT>(v, row, t, tw);
    transform_fence();
    if (live) store_col(v, T1, t, TT);
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = zr[spad(t + q * TT)];
    team_fft<LY, +1, 0, PRUNE_OUT>(v, row, t, tw);
    transform_fence();
    if (live) store_col(v, T2, t, TT);
  } else if constexpr (MODE == P2_RS_BWD) {
    // With dz, U's column spectrum times the dz spectrum is formed first and parked (thread-
    // private entries). The 16 products of a thread are summed in T, the rest of the sum in
    // double (FP64 runs at a small fraction of the FP32 rate).
    Stash<C, TT, p2_ustash_smem<T, LY, MODE>()> ur;
    ur.init(sm + ROWS * SR + team * SR, t);
    if (a.want_dz) {
      const C* U0 = Ub + (int64_t)b * a.cU * a.t_plane + (int64_t)kx * a.ny;
      load_col(v, U0, t, TT);
      team_fft<LY, -1, 0, PRUNE_IN>(v, row, t, tw);
      const C* hd = H(KDH);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        ur.set(q, cmul(v[q], spec_row(hd, q, t, TT, flipx, false, false)));
        XL_GROUP_FENCE(q);
      }
    }
    load_col(v, T0, t, TT);
    team_fft<LY, -1, 0, PRUNE_IN>(v, row, t, tw);
    if (a.want_dz) {
      T acc = (T)0;
#pragma unroll
      for (int q = 0; q < 16; ++q) acc += cdot_re(v[q], ur.get(q));
      dz = (double)acc;
    }
    if (a.want_field) {
      const C* h = H(KH);
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = cmulc(v[q], spec_row(h, q, t, TT, flipx, false, false));
      team_fft<LY, +1, 0, PRUNE_OUT>(v, row, t, tw);
      if (live) store_col(v, T0, t, TT);
    }
  } else if constexpr (MODE == P2_VRS_BWD) {
    // the spectrum of gz lives in a second shared-memory row of the team, U_c's column spectrum
    // (with dz) in a third when it fits (thread-private entries). The plane loop is unrolled: as a
    // runtime loop its invariant transform work was hoisted out of it and spilled.
    C* T1 = T0 + a.t_plane;
    C* T2 = T1 + a.t_plane;
    C* zr = sm + ROWS * SR + team * SR;
    Stash<C, TT, p2_ustash_smem<T, LY, MODE>()> ur;
    ur.init(sm + 2 * ROWS * SR + team * SR, t);
    load_col(v, T2, t, TT);
    team_fft<LY, -1, 0, PRUNE_IN>(v, row, t, tw);
#pragma unroll
    for (int q = 0; q < 16; ++q) zr[spad(t + q * TT)] = v[q];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      C* Tc = c == 0 ? T0 : T1;
      const bool ox = c == 0, oy = c == 1;
      if (a.want_dz) {
        const C* Uc = Ub + ((int64_t)b * a.cU + c) * a.t_plane + (int64_t)kx * a.ny;
        load_col(v, Uc, t, TT);
        team_fft<LY, -1, 0, PRUNE_IN>(v, row, t, tw);
#pragma unroll
        for (int q = 0; q < 16; ++q) ur.set(q, v[q]);
      }
      load_col(v, Tc, t, TT);
      team_fft<LY, -1, 0, PRUNE_IN>(v, row, t, tw);
      if (a.want_dz) {
        const C *hd = H(KDH), *ho = H(c == 0 ? KDHX : KDHY);
        T acc = (T)0;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const C u = ur.get(q);
          acc += cdot_re(v[q], cmul(u, spec_row(hd, q, t, TT, flipx, false, false))) +
                 cdot_re(zr[spad(t + q * TT)], cmul(u, spec_row(ho, q, t, TT, flipx, ox, oy)));
          XL_GROUP_FENCE(q);
        }
        dz += (double)acc;
      }
      if (a.want_field) {
        const C *hz = H(KH), *ho = H(c == 0 ? KHX : KHY);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          v[q] = cadd(cmulc(v[q], spec_row(hz, q, t, TT, flipx, false, false)),
                      cmulc(zr[spad(t + q * TT)], spec_row(ho, q, t, TT, flipx, ox, oy)));
          XL_GROUP_FENCE(q);
        }
        team_fft<LY, +1, 0, PRUNE_OUT>(v, row, t, tw);
        if (live) store_col(v, Tc, t, TT);
      }
    }
  } else if constexpr (MODE == P2_RS_BWD_S) {
    // U's column spectrum comes from the forward's saved spectra: one transform fewer and no
    // parked row (the products are formed as the saved values stream in)
    if constexpr (RM) {
      if (!gather_col_rm<LY, ROWS>(v, sm, tin, &rm_bar, kx, gx, b * a.cT * a.ny, a.ny, t, a.status)) return;
    } else {
      load_col(v, T0, t, TT);
    }
    team_fft<LY, -1, 0, PRUNE_IN>(v, row, t, tw);
    if (a.want_dz) {
      const C* su = spec_in(0);
      const C* hd = H(KDH);
      T acc = (T)0;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        acc += cdot_re(v[q], cmul(su[t + q * TT], spec_row(hd, q, t, TT, flipx, false, false)));
        XL_GROUP_FENCE(q);
      }
      dz = (double)acc;
    }
    if (a.want_field) {
      const C* h = H(KH);
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = cmulc(v[q], spec_row(h, q, t, TT, flipx, false, false));
      team_fft<LY, +1, 0, PRUNE_OUT>(v, row, t, tw);
      if (live) store_col(v, T0, t, TT);
    }
  } else if constexpr (MODE == P2_VRS_BWD_S) {
    // as P2_VRS_BWD with U_c's column spectra read from the saved spectra
    C* T1 = T0 + a.t_plane;
    C* T2 = T1 + a.t_plane;
    C* zr = sm + ROWS * SR + team * SR;
    load_col(v, T2, t, TT);
    team_fft<LY, -1, 0, PRUNE_IN>(v, row, t, tw);
#pragma unroll
    for (int q = 0; q < 16; ++q) zr[spad(t + q * TT)] = v[q];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      C* Tc = c == 0 ? T0 : T1;
      const bool ox = c == 0, oy = c == 1;
      load_col(v, Tc, t, TT);
      team_fft<LY, -1, 0, PRUNE_IN>(v, row, t, tw);
      if (a.want_dz) {
        const C* su = spec_in(c);
        const C *hd = H(KDH), *ho = H(c == 0 ? KDHX : KDHY);
        T acc = (T)0;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const C u = su[t + q * TT];
          acc += cdot_re(v[q], cmul(u, spec_row(hd, q, t, TT, flipx, false, false))) +
                 cdot_re(zr[spad(t + q * TT)], cmul(u, spec_row(ho, q, t, TT, flipx, ox, oy)));
          XL_GROUP_FENCE(q);
        }
        dz += (double)acc;
      }
      if (a.want_field) {
        const C *hz = H(KH), *ho = H(c == 0 ? KHX : KHY);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          v[q] = cadd(cmulc(v[q], spec_row(hz, q, t, TT, flipx, false, false)),
                      cmulc(zr[spad(t + q * TT)], spec_row(ho, q, t, TT, flipx, ox, oy)));
          XL_GROUP_FENCE(q);
        }
        team_fft<LY, +1, 0, PRUNE_OUT>(v, row, t, tw);
        transform_fence();
        if (live) store_col(v, Tc, t, TT);
      }
    }
  }
  if constexpr (MODE == P2_RS_BWD || MODE == P2_VRS_BWD || MODE == P2_RS_BWD_S ||
                MODE == P2_VRS_BWD_S) {
    if (a.want_dz) {
      double s = block_sum(live ? dz : 0.0, red);
      if (threadIdx.x == 0) dz_part[(int64_t)b * gridDim.x + p2_group<PAIR>()] = s;
    }
  }
}

// Fixed-order final reduction of the dz partials: g_z[b] = sum_i part[b][i].
static __global__ void k_reduce_rows(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[(int64_t)b * n + i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[b] = s;
}

// ---------------------------------------------------------------------------------------------
// Spectrum generation.
struct GenArgs {
  int nx, ny;
  double dx, dy, k;
  double zval;            // host distance (used when zdev == nullptr)
  const double* zdev;     // device distance
  unsigned kinds;         // bit mask of the spectra to produce
  int64_t s_plane;        // elements of one S plane ((nx+1) * ny)
  int64_t hq_kind;        // elements of one quadrant
  double scale;           // 1 / (LX LY)
  int slot[NKIND];        // kind -> slot of the S / Hq buffers (-1: not produced)
  int dz_rest;            // distance-derivative kinds carry dh/dz - i k h (phase-invariant losses)
  int64_t s_elem, h_elem; // device distances: element blockIdx.y reads zdev[blockIdx.y] and
                          // writes its S and Hq at these element strides
};

// ---------------------------------------------------------------------------------------------
// Double-float arithmetic (an unevaluated sum hi + lo of two floats, about 44 significant bits;
// Dekker 1971 / Knuth's two-sum, with the fused multiply-add giving exact products). It carries
// the phase k r of the single-precision spectrum generator: r up to ~1.5 mm and k ~ 10 / um give
// phases of ~1e4 rad that must be known to ~1e-6 rad before the final sincos, which single
// precision cannot do and double precision does at a small fraction of the FP32 rate on GB300.
struct df {
  float hi, lo;
};
__device__ __forceinline__ df df_two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df df_norm(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df df_of(double d) {
  const float hi = (float)d;
  return {hi, (float)(d - (double)hi)};
}
__device__ __forceinline__ df df_add(df x, df y) {
  df s = df_two_sum(x.hi, y.hi);
  return df_norm(s.hi, s.lo + x.lo + y.lo);
}
__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df df_mul(df x, df y) {
  df p = df_two_prod(x.hi, y.hi);
  return df_norm(p.hi, p.lo + (x.hi * y.lo + x.lo * y.hi));
}
__device__ __forceinline__ df df_mul_f(df x, float y) {
  df p = df_two_prod(x.hi, y);
  return df_norm(p.hi, fmaf(x.lo, y, p.lo));
}
__device__ __forceinline__ df df_div(df x, df y) {
  const float q1 = x.hi / y.hi;
  df r = df_add(x, df_neg(df_mul_f(y, q1)));
  const float q2 = r.hi / y.hi;
  r = df_add(r, df_neg(df_mul_f(y, q2)));
  const float q3 = r.hi / y.hi;
  df q = df_norm(q1, q2);
  return df_add(q, {q3, 0.f});
}
__device__ __forceinline__ df df_sqrt(df x) {
  const float y = sqrtf(x.hi);
  const df e = df_add(x, df_neg(df_two_prod(y, y)));
  return df_norm(y, e.hi / (2.f * y));
}

// Per-thread constants of the kernel samples for one distance.
template <typename T> struct RsPhase;
template <> struct RsPhase<float> {
  df dx2, dy2, z, z2, k, twopi;
  float kz_red, zf, izf, kf, c0, dxf, dyf;
  RsPhase() = default;
  __device__ RsPhase(const GenArgs& g, double zz) {
    dxf = (float)g.dx;
    dyf = (float)g.dy;
    dx2 = df_of(g.dx * g.dx);
    dy2 = df_of(g.dy * g.dy);
    z = df_of(zz);
    z2 = df_of(zz * zz);
    k = df_of(g.k);
    twopi = df_of(kTwoPi);
    kz_red = (float)(g.k * zz - kTwoPi * rint(g.k * zz / kTwoPi));
    zf = (float)zz;
    izf = (float)(1.0 / zz);
    kf = (float)g.k;
    c0 = (float)(g.dx * g.dy / kTwoPi);
  }
};
template <> struct RsPhase<double> {
  double kz_red, z;
  RsPhase() = default;
  __device__ RsPhase(const GenArgs& g, double zz) {
    kz_red = g.k * zz - kTwoPi * rint(g.k * zz / kTwoPi);
    z = zz;
  }
};

// dh/dz and the odd kinds from h, r and the unit phasor (shared by both precisions).
// ir = 1 / r and iz = 1 / z come in precomputed (a sample then needs no division but the one of
// the phase-invariant dz kinds).
template <typename T>
__device__ __forceinline__ cplx<T> rs_kinds(int kind, cplx<T> e, T r, T ir, T X, T Y, T z, T iz, T k,
                                            T c0, bool rest) {
  typedef cplx<T> C;
  const T ir2 = ir * ir, ir3 = ir2 * ir;
  // h = c0 z (1/r - i k) e / r^2
  const C h = cmul(e, mk(c0 * z * ir3, -c0 * z * k * ir2));
  if (kind == KH) return h;
  if (kind == KHX) return cscale(h, -X * iz);
  if (kind == KHY) return cscale(h, -Y * iz);
  // dh/dz = c0 e [(1/r^3 - i k / r^2) + z^2 (k^2/r^3 + 3 i k / r^4 - 3 / r^5)]
  const T z2 = z * z;
  const T re = ir3 + z2 * (k * k * ir3 - (T)3 * ir3 * ir2);
  const T im = -k * ir2 + z2 * (T)3 * k * ir2 * ir2;
  C dh;
  if (!rest) {
    dh = cmul(e, mk(c0 * re, c0 * im));
  } else {
    // dh/dz - i k h without cancellation (r - z = rho^2 / (r + z)):
    //   c0 e [ 1/r^3 - 3 z^2/r^5 - k^2 z rho^2 / ((r + z) r^3)  +  i k (3 z^2/r^4 - 1/r^2 - z/r^3) ]
    const T rho2 = X * X + Y * Y;
    const T rr = ir3 - (T)3 * z2 * ir3 * ir2 - k * k * z * rho2 * ir3 / (r + z);
    const T ri = k * ((T)3 * z2 * ir2 * ir2 - ir2 - z * ir3);
    dh = cmul(e, mk(c0 * rr, c0 * ri));
  }
  if (kind == KDH) return dh;
  // d/dz[-(X/z) h] = -(X/z)(dh - h/z)
  const C dmh = csub(dh, cscale(h, iz));
  return cscale(dmh, kind == KDHX ? -X * iz : -Y * iz);
}

// The parts of a kernel sample at pixel offset (a, b) that every kind shares: the unit phasor
// exp(i k r) and r; rs_kinds then forms any kind from them. Single precision: r and the phase
// k (r - z) = k rho^2 / (r + z) in double-float (exact a^2, b^2 times dx^2, dy^2), reduced modulo
// 2 pi before adding k z mod 2 pi and one sincosf (the costly part). Double precision: the same
// formula in double.
__device__ __forceinline__ void rs_phasor(int a, int b, const GenArgs& g, double, const RsPhase<float>& P,
                                          float2* e, float* r) {
  const float A = (float)(a * a), B = (float)(b * b);  // exact (|a|, |b| < 4096)
  const df rho2 = df_add(df_mul_f(P.dx2, A), df_mul_f(P.dy2, B));
  const df rr = df_sqrt(df_add(rho2, P.z2));
  const df ph = df_div(df_mul(P.k, rho2), df_add(rr, P.z));
  const float n = rintf(ph.hi * 0.15915494309189535f);
  const df red = df_add(ph, df_neg(df_mul_f(P.twopi, n)));
  float sn, cs;
  sincosf(red.hi + red.lo + P.kz_red, &sn, &cs);
  *e = make_float2(cs, sn);
  *r = rr.hi;
}
__device__ __forceinline__ void rs_phasor(int a, int b, const GenArgs& g, double z, const RsPhase<double>& P,
                                          double2* e, double* r) {
  const double X = a * g.dx, Y = b * g.dy;
  const double rho2 = X * X + Y * Y;
  *r = sqrt(rho2 + z * z);
  double ph = g.k * rho2 / (*r + z);
  ph -= kTwoPi * rint(ph * (1.0 / kTwoPi));
  double sn, cs;
  sincos(ph + P.kz_red, &sn, &cs);
  *e = make_double2(cs, sn);
}
// Kind `kind` at offset (a, b) from its phasor e; r from the offsets (plain precision is enough:
// r only scales amplitudes).
__device__ __forceinline__ float2 rs_from_phasor(int kind, float2 e, int a, int b, const GenArgs& g,
                                                 const RsPhase<float>& P, float r) {
  const float X = (float)a * P.dxf, Y = (float)b * P.dyf;
  float ir;
  if (r < 0.f) {  // r from the offsets: one reciprocal square root
    const float r2 = fmaf(X, X, fmaf(Y, Y, P.zf * P.zf));
    ir = rsqrtf(r2);
    r = r2 * ir;
  } else {
    ir = 1.f / r;
  }
  return rs_kinds<float>(kind, e, r, ir, X, Y, P.zf, P.izf, P.kf, P.c0, g.dz_rest != 0);
}
__device__ __forceinline__ double2 rs_from_phasor(int kind, double2 e, int a, int b, const GenArgs& g,
                                                  const RsPhase<double>& P, double r) {
  const double X = a * g.dx, Y = b * g.dy;
  const double z = P.z;
  if (r < 0.0) r = sqrt(X * X + Y * Y + z * z);
  return rs_kinds<double>(kind, e, r, 1.0 / r, X, Y, z, 1.0 / z, g.k, g.dx * g.dy / kTwoPi,
                          g.dz_rest != 0);
}

// Generator pass A: for each b in [0, ny) and each kind, FFT along a of the kernel row placed
// mod LX; keep kx in [0, nx]; store transposed S[kind][kx][b]. CACHE: the phasors of the row are
// evaluated once per |a| < nx into shared memory after the transform rows, and every kind starts
// from them (the phase is the costly part of a sample).
template <typename T, int LX, bool CACHE = true>
__global__ void __launch_bounds__(rows_transp<LX, sizeof(cplx<T>)>() * (LX / 16),
                                  min_blocks_rows<rows_transp<LX, sizeof(cplx<T>)>() * (LX / 16), sizeof(cplx<T>)>())
k_gen_pass_a(cplx<T>* __restrict__ S, GenArgs g, const cplx<T>* __restrict__ tw) {
  typedef cplx<T> C;
  constexpr int ROWS = rows_transp<LX, sizeof(C)>();
  static_assert(team_barriers_fit<LX>(ROWS * (LX / 16)), "too many teams for the named barriers");
  constexpr int TT = LX / 16;
  constexpr int P = tpitch(LX, sizeof(C), ROWS);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int b0 = blockIdx.x * ROWS;
  const int b = b0 + team;
  const double z = g.zdev ? g.zdev[blockIdx.y] : g.zval;
  S += (int64_t)blockIdx.y * g.s_elem;
  // the distance's constants, formed once for the block (they take double divisions, and FP64
  // runs at a small fraction of the FP32 rate)
  __shared__ RsPhase<T> ph_s;
  if (threadIdx.x == 0) ph_s = RsPhase<T>(g, z);
  __syncthreads();
  const RsPhase<T>& ph = ph_s;  // read from shared memory where used (no registers held)
  C* row = sm + team * P;
  C* phc = sm + ROWS * P + team * (LX / 2);  // phasors of |a| < nx (CACHE)
  if constexpr (CACHE) {
    // the row's phasors, once per |a| (the kernel is even in a): thread t takes a = t + q TT
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      const int a = t + q * TT;
      C e;
      T r;
      rs_phasor(a, b < g.ny ? b : 0, g, z, ph, &e, &r);
      phc[a] = e;
    }
    team_sync<LX>();
  }
  for (int kind = 0; kind < NKIND; ++kind) {
    if (!(g.kinds & (1u << kind))) continue;  // uniform over the block
    C v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int i = t + q * TT;
      const int a = i < g.nx ? i : i - LX;
      if (i == g.nx || b >= g.ny) {
        v[q] = mk((T)0, (T)0);
      } else if constexpr (CACHE) {
        v[q] = rs_from_phasor(kind, phc[a >= 0 ? a : -a], a, b, g, ph, (T)-1);
      } else {
        C e;
        T r;
        rs_phasor(a, b, g, z, ph, &e, &r);
        v[q] = rs_from_phasor(kind, e, a, b, g, ph, r);
      }
    }
    team_fft<LX, -1>(v, row, t, tw);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) row[spad(t + q * TT)] = v[q];
    __syncthreads();
    store_rows_transposed<LX, ROWS, P>(sm, g.nx + 1, S + (int64_t)g.slot[kind] * g.s_plane, g.ny, b0, g.ny);
    __syncthreads();
  }
}

// Generator pass B: for each kx in [0, nx] and kind, FFT along b of the even/odd extension of
// S[kind][kx][.]; keep ky in [0, ny]; store Hq[kind][kx][ky] * scale.
template <typename T, int LY>
__global__ void __launch_bounds__(rows_cols<LY>() * (LY / 16))
k_gen_pass_b(const cplx<T>* __restrict__ S, cplx<T>* __restrict__ Hq, GenArgs g,
             const cplx<T>* __restrict__ tw) {
  typedef cplx<T> C;
  constexpr int ROWS = rows_cols<LY>();
  static_assert(team_barriers_fit<LY>(ROWS * (LY / 16)), "too many teams for the named barriers");
  constexpr int TT = LY / 16;
  constexpr int SR = srow(LY);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int team = threadIdx.x / TT, t = threadIdx.x % TT;
  const int kx_raw = blockIdx.x * ROWS + team;
  const bool live = kx_raw <= g.nx;
  const int kx = live ? kx_raw : g.nx;
  S += (int64_t)blockIdx.y * g.s_elem;
  Hq += (int64_t)blockIdx.y * g.h_elem;
  C* row = sm + team * SR;
  if (t == 0)  // every kind's column, asked of L2 before the first transform
    for (int kind = 0; kind < NKIND; ++kind)
      if (g.kinds & (1u << kind))
        prefetch_l2(S + (int64_t)g.slot[kind] * g.s_plane + (int64_t)kx * g.ny, (size_t)g.ny * sizeof(C));
  for (int kind = 0; kind < NKIND; ++kind) {
    if (!(g.kinds & (1u << kind))) continue;
    const C* src = S + (int64_t)g.slot[kind] * g.s_plane + (int64_t)kx * g.ny;
    const bool odd = kind_odd_y(kind);
    C v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int j = t + q * TT;
      if (j < g.ny) {
        v[q] = src[j];
      } else if (j == g.ny) {
        v[q] = mk((T)0, (T)0);
      } else {
        C s = src[LY - j];
        v[q] = odd ? mk(-s.x, -s.y) : s;
      }
    }
    team_fft<LY, -1>(v, row, t, tw);
    if (live) {
      C* dst = Hq + (int64_t)g.slot[kind] * g.hq_kind + (int64_t)kx * (g.ny + 1);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int ky = t + q * TT;
        if (ky <= g.ny) dst[ky] = cscale(v[q], (T)g.scale);
      }
    }
  }
}

}  // namespace xl
