// Scalar RS propagation that allocates no memory: for callers that cannot call cudaMalloc
// themselves or have the library do it (an allocator owned by another runtime, a real-time
// or embedded host that pre-reserves all device memory, a sandbox where the allocation API is
// not available). Everything the three-pass convolution needs beyond the caller's input and
// output (twiddle tables, the kernel-row spectra, the transfer-spectrum quadrant and the
// transposed intermediate) lives in one fixed static device array in this file.
//
// It computes the same discrete RS convolution as xl_rs_propagate, for complex64 fields up to
// 256 x 256, equal to it within rounding but not bit for bit: the twiddle tables are filled here
// on the device in double precision, the transfer spectrum comes from the generator variant
// without a per-row cache (k_gen_pass_a<..., false>, which keeps each launch under 48 KB of
// shared memory), and the passes are the transposing pass 1 and pass 3 with a pass 2 that reads
// its columns directly (no tensor maps, which would have to be encoded per call), not the
// row-major intermediate of the default complex64 path. The transfer spectrum is regenerated for
// every run of equal consecutive distances instead of being cached. A device reset
// (cudaDeviceReset) after the first call is not supported: the set-up below is done once per
// device for the life of the process.
#include <cstring>
#include <cmath>
#include <mutex>

#include "xl_rs_kernels.cuh"
#include "xl_runtime.h"

namespace xl {
namespace {

constexpr int kStaticMaxN = 256;
constexpr size_t kAlign = 256;
constexpr size_t al256(size_t n) { return (n + kAlign - 1) & ~(kAlign - 1); }
// twiddle tables for L = 64, 128, 256, 512 (complex64), one block each
constexpr size_t kTwBytes = al256(4096 * sizeof(float2));
constexpr size_t kSBytes = al256((size_t)(kStaticMaxN + 1) * kStaticMaxN * sizeof(float2));
constexpr size_t kHqBytes = al256((size_t)(kStaticMaxN + 1) * (kStaticMaxN + 1) * sizeof(float2));
constexpr size_t kTBytes = al256((size_t)2 * kStaticMaxN * kStaticMaxN * sizeof(float2));
constexpr size_t kScratchBytes = kTwBytes + kSBytes + kHqBytes + kTBytes;  // 2,136,320 bytes
static_assert(kScratchBytes == 2136320, "scratch size quoted in xl.h");

// The scratch. In host code this name is only a stand-in for the device symbol: kernels get the
// device address obtained with cudaGetSymbolAddress at set-up.
static __device__ __align__(256) unsigned char g_rs_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};
bool g_static_ready[kMaxDevices] = {};

// Offsets (in complex entries) of the twiddle block of each transform length inside kTwBytes.
__host__ __device__ constexpr int static_tw_offset(int L) {
  return L == 64 ? 0 : L == 128 ? 64 : L == 256 ? 192 : 448;  // sizes 64, 128, 256, 768
}

// Fills the twiddle blocks (the r-major per-stage layout of xl_fft.cuh) in double precision.
__global__ void k_static_twiddles(float2* tw) {
  const int Ls[4] = {64, 128, 256, 512};
  for (int li = 0; li < 4; ++li) {
    const int L = Ls[li];
    float2* base = tw + static_tw_offset(L);
    int off = 0, Ns = 16;
    while (Ns < L) {
      const int R = (Ns * 16 <= L) ? 16 : L / Ns;
      for (int i = threadIdx.x; i < R * Ns; i += blockDim.x) {
        const int r = i / Ns, k = i % Ns;
        const double ang = -kTwoPi * (double)k * (double)r / ((double)Ns * (double)R);
        double s, c;
        sincos(ang, &s, &c);
        base[off + i] = make_float2((float)c, (float)s);
      }
      off += R * Ns;
      Ns *= R;
    }
  }
}

// Per-device set-up: the device address of the scratch and its twiddle tables.
xl_status static_setup(cudaStream_t s, char** scratch) {
  int dev = 0;
  XL_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(XL_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ready[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rs_static_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(rs static scratch)");
    k_static_twiddles<<<1, 256, 0, s>>>(reinterpret_cast<float2*>(p));
    XL_CUDA_TRY(cudaGetLastError());
    // later calls may come on other streams: the tables must be complete before they return
    XL_CUDA_TRY(cudaStreamSynchronize(s));
    g_static_ptr[dev] = p;
    g_static_ready[dev] = true;
  }
  *scratch = reinterpret_cast<char*>(g_static_ptr[dev]);
  return XL_OK;
}

template <int LX, int LY>
xl_status run_static(const float2* in, float2* out, int32_t batch, const xl_grid* g,
                     double wavelength, const double* z, char* scratch, cudaStream_t s) {
  const int nx = g->nx, ny = g->ny;
  const float2* twb = reinterpret_cast<const float2*>(scratch);
  const float2* twx = twb + static_tw_offset(LX);
  const float2* twy = twb + static_tw_offset(LY);
  float2* S = reinterpret_cast<float2*>(scratch + kTwBytes);
  float2* Hq = reinterpret_cast<float2*>(scratch + kTwBytes + kSBytes);
  float2* T = reinterpret_cast<float2*>(scratch + kTwBytes + kSBytes + kHqBytes);

  GenArgs ga;
  ga.nx = nx;
  ga.ny = ny;
  ga.dx = g->dx;
  ga.dy = g->dy;
  ga.k = kTwoPi / wavelength;
  ga.zdev = nullptr;
  ga.kinds = 1u << KH;
  ga.s_plane = (int64_t)(nx + 1) * ny;
  ga.s_elem = ga.h_elem = 0;
  ga.hq_kind = (int64_t)(nx + 1) * (ny + 1);
  ga.scale = 1.0 / (4.0 * (double)nx * (double)ny);
  for (int i = 0; i < NKIND; ++i) ga.slot[i] = -1;
  ga.slot[KH] = 0;
  ga.dz_rest = 0;

  P2Args pa;
  pa.nx = nx;
  pa.ny = ny;
  pa.t_plane = (int64_t)2 * nx * ny;
  pa.hq_kind = ga.hq_kind;
  pa.cT = 1;
  pa.cU = 0;
  pa.want_field = 1;
  pa.want_dz = 0;
  pa.conj = 0;
  for (int i = 0; i < NKIND; ++i) pa.slot[i] = -1;
  pa.slot[KH] = 0;
  pa.spec_out = nullptr;
  pa.spec_in = nullptr;
  pa.cS = 0;
  pa.per_elem = 0;
  for (int i = 0; i < kP2Run; ++i) pa.hshift[i] = 0;
  pa.status = nullptr;
  CUtensorMap no_map;  // pass 2 reads its columns directly here
  std::memset(&no_map, 0, sizeof(no_map));

  // every launch below needs less than 48 KB of shared memory (transform lengths <= 512)
  constexpr int RA = rows_transp<LX, 8>(), R3 = rows_p3<LX, 8>(), RB = rows_cols<LY>(),
                RC = rows_cols<LY>();
  const size_t smA = (size_t)RA * tpitch(LX, 8, RA) * sizeof(float2);
  const size_t sm3 = (size_t)R3 * tpitch(LX, 8, R3) * sizeof(float2);
  const size_t smB = (size_t)RB * srow(LY) * sizeof(float2);
  const size_t smP2 = (size_t)RC * srow(LY) * sizeof(float2);
  static_assert(RA * tpitch(LX, 8, RA) * 8 <= 48 * 1024 && R3 * tpitch(LX, 8, R3) * 8 <= 48 * 1024 &&
                    RB * srow(LY) * 8 <= 48 * 1024, "smem");
  const int64_t plane = (int64_t)nx * ny;
  for (int32_t b = 0; b < batch; ++b) {
    if (b == 0 || z[b] != z[b - 1]) {
      ga.zval = z[b];
      k_gen_pass_a<float, LX, false><<<(ny + RA - 1) / RA, RA * (LX / 16), smA, s>>>(S, ga, twx);
      XL_CUDA_TRY(cudaGetLastError());
      k_gen_pass_b<float, LY><<<(nx + 1 + RB - 1) / RB, RB * (LY / 16), smB, s>>>(S, Hq, ga, twy);
      XL_CUDA_TRY(cudaGetLastError());
    }
    k_rs_pass1<float, LX><<<dim3((ny + RA - 1) / RA, 1), RA * (LX / 16), smA, s>>>(
        in + b * plane, T, nx, ny, 1, 1, twx);
    XL_CUDA_TRY(cudaGetLastError());
    k_rs_pass2<float, LY, P2_RS><<<dim3((LX + RC - 1) / RC, 1), RC * (LY / 16), smP2, s>>>(
        T, nullptr, Hq, nullptr, pa, twy, no_map);
    XL_CUDA_TRY(cudaGetLastError());
    k_rs_pass3<float, LX><<<dim3((ny + R3 - 1) / R3, 1), R3 * (LX / 16), sm3, s>>>(
        T, out + b * plane, nx, ny, 1, 1, twx, DzReduce{nullptr, 0, nullptr});
    XL_CUDA_TRY(cudaGetLastError());
  }
  return XL_OK;
}

template <int LX>
xl_status run_static_x(int LY, const float2* in, float2* out, int32_t batch, const xl_grid* g,
                       double wavelength, const double* z, char* scratch, cudaStream_t s) {
  switch (LY) {
    case 64: return run_static<LX, 64>(in, out, batch, g, wavelength, z, scratch, s);
    case 128: return run_static<LX, 128>(in, out, batch, g, wavelength, z, scratch, s);
    case 256: return run_static<LX, 256>(in, out, batch, g, wavelength, z, scratch, s);
    case 512: return run_static<LX, 512>(in, out, batch, g, wavelength, z, scratch, s);
  }
  return fail(XL_ERR_UNSUPPORTED, "rs static: unsupported ny");
}

}  // namespace
}  // namespace xl

using namespace xl;

extern "C" {

xl_status xl_rs_propagate_static(const void* u_in, void* u_out, int32_t batch, const xl_grid* grid,
                                 double wavelength, const double* z, void* stream) {
  if (!grid) return fail(XL_ERR_ARG, "grid is NULL");
  if (!is_pow2(grid->nx) || !is_pow2(grid->ny) || grid->nx < 32 || grid->ny < 32)
    return fail(XL_ERR_UNSUPPORTED, "nx, ny must be powers of two >= 32");
  if (grid->nx > kStaticMaxN || grid->ny > kStaticMaxN)
    return fail(XL_ERR_UNSUPPORTED,
                "xl_rs_propagate_static: nx and ny are limited to 256 (fixed scratch of 2,136,320 bytes); "
                "use xl_rs_propagate for larger grids");
  if (!(grid->dx > 0) || !(grid->dy > 0) || !std::isfinite(grid->dx) || !std::isfinite(grid->dy))
    return fail(XL_ERR_ARG, "pixel pitch must be positive and finite");
  if (!(wavelength > 0) || !std::isfinite(wavelength)) return fail(XL_ERR_ARG, "bad wavelength");
  if (batch < 0) return fail(XL_ERR_ARG, "batch < 0");
  if (batch == 0) return XL_OK;
  if (!u_in || !u_out || !z) return fail(XL_ERR_ARG, "NULL pointer");
  if (u_in == u_out) return fail(XL_ERR_ARG, "output may not alias the input");
  for (int32_t b = 0; b < batch; ++b)
    if (!(z[b] > 0) || !std::isfinite(z[b])) return fail(XL_ERR_ARG, "z must be positive and finite");
  cudaStream_t s = (cudaStream_t)stream;
  char* scratch = nullptr;
  XL_TRY(static_setup(s, &scratch));
  const float2* in = (const float2*)u_in;
  float2* out = (float2*)u_out;
  switch (2 * grid->nx) {
    case 64: return run_static_x<64>(2 * grid->ny, in, out, batch, grid, wavelength, z, scratch, s);
    case 128: return run_static_x<128>(2 * grid->ny, in, out, batch, grid, wavelength, z, scratch, s);
    case 256: return run_static_x<256>(2 * grid->ny, in, out, batch, grid, wavelength, z, scratch, s);
    case 512: return run_static_x<512>(2 * grid->ny, in, out, batch, grid, wavelength, z, scratch, s);
  }
  return fail(XL_ERR_UNSUPPORTED, "rs static: unsupported nx");
}

}  // extern "C"
