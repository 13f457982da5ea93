// Shared device/host helpers of the xl CUDA library: complex arithmetic on float2/double2,
// status handling, and per-type constants.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/xl.h"

namespace xl {

// ------------------------------------------------------------------ complex types
template <typename T> struct CT;
template <> struct CT<float> { typedef float2 type; };
template <> struct CT<double> { typedef double2 type; };

template <typename T> using cplx = typename CT<T>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }

// complex64 sums on the paired single-precision instructions of sm_100 and later (add / sub
// .rn.f32x2: both components in one instruction, each rounded as the scalar operation rounds, so
// the results are the scalar ones bit for bit). The transforms are issue-bound and consist mostly
// of complex additions, so halving their instruction count frees issue slots.
#if defined(__CUDA_ARCH__)
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 f2_from(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(r);
}
#endif
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) {
  return mk(a.x * s, a.y * s);
}
// conj(a) * b, real part
template <typename C> __host__ __device__ __forceinline__ auto cdot_re(C a, C b) -> decltype(a.x) {
  return a.x * b.x + a.y * b.y;
}

// accurate sincos per precision (never the fast intrinsics: phases feed 2e-5 field parity)
__device__ __forceinline__ void xsincos(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void xsincos(double a, double* s, double* c) { sincos(a, s, c); }

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double kTwoPi = 6.28318530717958647692528676655900577;

// ------------------------------------------------------------------ status
// Thread-local message of the last failing call (read by xl_last_error()).
void set_error(const std::string& msg);
xl_status fail(xl_status code, const std::string& msg);
xl_status cuda_status(cudaError_t e, const char* where);

#define XL_CUDA_TRY(expr)                                           \
  do {                                                              \
    cudaError_t _e = (expr);                                        \
    if (_e != cudaSuccess) return ::xl::cuda_status(_e, #expr);     \
  } while (0)

#define XL_TRY(expr)                     \
  do {                                   \
    xl_status _s = (expr);               \
    if (_s != XL_OK) return _s;          \
  } while (0)

inline bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }
inline int ilog2(int64_t n) {
  int l = 0;
  while ((int64_t(1) << l) < n) ++l;
  return l;
}

}  // namespace xl
