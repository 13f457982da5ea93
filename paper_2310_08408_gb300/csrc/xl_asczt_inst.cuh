// Definitions of the angular-spectrum CZT launchers for one precision; included with XL_REAL
// defined.
#include <algorithm>
#include <string>

#include "xl_asczt_launch.h"

namespace xl {
namespace {

template <typename T, int L, int STAGE>
xl_status fwd_L(const void* in, void* out, int nrows, const void* Hc, const AsShift& hs, int nb,
                cudaStream_t s) {
  typedef cplx<T> C;
  constexpr int ROWS = as_rows<L, sizeof(C), false>();
  const size_t sm = (size_t)ROWS * tpitch(L, sizeof(C), ROWS) * sizeof(C);
  const void* tw;
  XL_TRY(twiddles(L, sizeof(T) == 8 ? XL_C128 : XL_C64, &tw));
  XL_TRY(smem_attr((const void*)k_as_fwd<T, L, STAGE>, sm));
  LaunchScope ls(std::string(STAGE == AS_STAGE_A ? "asczt_spec_a<" : "asczt_spec_b<") +
                     std::to_string(L) + ">", s);
  k_as_fwd<T, L, STAGE><<<dim3((nrows + ROWS - 1) / ROWS, nb), ROWS * (L / 16), sm, s>>>(
      (const C*)in, (C*)out, nrows, (const C*)Hc, hs, (const C*)tw);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

template <typename T, int L, int STAGE, bool DZ>
xl_status adj_L(const void* in, void* out, int nrows, const void* Hc, const void* dHc,
                const AsShift& hs, const void* TU, double* dz_part, int nb, cudaStream_t s) {
  typedef cplx<T> C;
  constexpr int ROWS = as_rows<L, sizeof(C), DZ>();
  const size_t sm = (size_t)ROWS * (DZ ? 2 : 1) * tpitch(L, sizeof(C), ROWS) * sizeof(C);
  const void* tw;
  XL_TRY(twiddles(L, sizeof(T) == 8 ? XL_C128 : XL_C64, &tw));
  XL_TRY(smem_attr((const void*)k_as_adj<T, L, STAGE, DZ>, sm));
  LaunchScope ls(std::string(STAGE == AS_STAGE_A ? "asczt_spec_a_adj<" : (DZ ? "asczt_spec_b_adj_dz<" : "asczt_spec_b_adj<")) +
                     std::to_string(L) + ">", s);
  k_as_adj<T, L, STAGE, DZ><<<dim3((nrows + ROWS - 1) / ROWS, nb), ROWS * (L / 16), sm, s>>>(
      (const C*)in, (C*)out, nrows, (const C*)Hc, (const C*)dHc, hs, (const C*)TU, dz_part,
      (const C*)tw);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

}  // namespace

#define XL_AS_SWITCH(L, CASE)                                                      \
  switch (L) {                                                                     \
    case 64: return CASE(64);                                                      \
    case 128: return CASE(128);                                                    \
    case 256: return CASE(256);                                                    \
    case 512: return CASE(512);                                                    \
    case 1024: return CASE(1024);                                                  \
    case 2048: return CASE(2048);                                                  \
    case 4096: return CASE(4096);                                                  \
  }

template <>
xl_status as_fwd_pass<XL_REAL>(int stage, int L, const void* in, void* out, int nrows,
                               const void* Hc, const AsShift& hs, int nb, cudaStream_t s) {
#define FA(LL) fwd_L<XL_REAL, LL, AS_STAGE_A>(in, out, nrows, Hc, hs, nb, s)
#define FB(LL) fwd_L<XL_REAL, LL, AS_STAGE_B>(in, out, nrows, Hc, hs, nb, s)
  if (stage == AS_STAGE_A) {
    XL_AS_SWITCH(L, FA)
  } else {
    XL_AS_SWITCH(L, FB)
  }
#undef FA
#undef FB
  return fail(XL_ERR_UNSUPPORTED, "asczt: unsupported row length");
}

template <>
xl_status as_adj_pass<XL_REAL>(int stage, int L, const void* in, void* out, int nrows,
                               const void* Hc, const void* dHc, const AsShift& hs, const void* TU,
                               double* dz_part, int nb, cudaStream_t s) {
#define AA(LL) adj_L<XL_REAL, LL, AS_STAGE_A, false>(in, out, nrows, Hc, dHc, hs, TU, dz_part, nb, s)
#define AB(LL) adj_L<XL_REAL, LL, AS_STAGE_B, false>(in, out, nrows, Hc, dHc, hs, TU, dz_part, nb, s)
#define AD(LL) adj_L<XL_REAL, LL, AS_STAGE_B, true>(in, out, nrows, Hc, dHc, hs, TU, dz_part, nb, s)
  if (stage == AS_STAGE_A) {
    XL_AS_SWITCH(L, AA)
  } else if (!dz_part) {
    XL_AS_SWITCH(L, AB)
  } else {
    XL_AS_SWITCH(L, AD)
  }
#undef AA
#undef AB
#undef AD
  return fail(XL_ERR_UNSUPPORTED, "asczt: unsupported row length");
}

template <>
int as_dz_blocks<XL_REAL>(int L, int nrows) {
  int rows = 1;
#define RW(LL) (rows = as_rows<LL, sizeof(cplx<XL_REAL>), true>(), 0)
  switch (L) {
    case 64: RW(64); break;
    case 128: RW(128); break;
    case 256: RW(256); break;
    case 512: RW(512); break;
    case 1024: RW(1024); break;
    case 2048: RW(2048); break;
    case 4096: RW(4096); break;
  }
#undef RW
  return (nrows + rows - 1) / rows;
}

template <>
xl_status as_transfer<XL_REAL>(void* Hc, void* dHc, const AsTransferArgs& a, cudaStream_t s) {
  typedef cplx<XL_REAL> C;
  const int64_t n = (int64_t)a.nx * a.ny;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  LaunchScope ls("asczt_transfer", s);
  k_as_transfer<XL_REAL><<<blocks, 256, 0, s>>>((C*)Hc, (C*)dHc, a);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

#undef XL_AS_SWITCH

}  // namespace xl
