// Definitions of the RS launchers for one precision; included by xl_rs_c64.cu / xl_rs_c128.cu
// with XL_REAL defined.
#include "xl_rs_launch.h"

namespace xl {

namespace {

template <typename T, int LX, int V>
xl_status pass1_LV(const void* in, void* Tb, int nx, int ny, int cin, int cT, int np, cudaStream_t s) {
  constexpr int ROWS = rows_p1v<LX, sizeof(cplx<T>), V>();
  const size_t sm = (size_t)ROWS * tpitch(LX, sizeof(cplx<T>), ROWS) * sizeof(cplx<T>);
  const void* tw;
  XL_TRY(twiddles(LX, sizeof(T) == 8 ? XL_C128 : XL_C64, &tw));
  XL_TRY(smem_attr((const void*)k_rs_pass1<T, LX, V>, sm));
  dim3 grid((ny + ROWS - 1) / ROWS, np);
  LaunchScope ls("rs_pass1<" + std::to_string(LX) + ">", s);
  k_rs_pass1<T, LX, V><<<grid, ROWS * (LX / 16), sm, s>>>(
      (const cplx<T>*)in, (cplx<T>*)Tb, nx, ny, cin, cT, (const cplx<T>*)tw);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

// the autotuner's variant of this length (only long rows have more than the default)
template <typename T, int LX>
xl_status pass1_L(const void* in, void* Tb, int nx, int ny, int cin, int cT, int np, cudaStream_t s) {
  if constexpr (LX >= kTuneMinL) {
    switch (tuned_variant(TUNE_RS_PASS1, LX, sizeof(T) == 8 ? XL_C128 : XL_C64)) {
      case 1: return pass1_LV<T, LX, 1>(in, Tb, nx, ny, cin, cT, np, s);
      case 2: return pass1_LV<T, LX, 2>(in, Tb, nx, ny, cin, cT, np, s);
    }
  }
  return pass1_LV<T, LX, 0>(in, Tb, nx, ny, cin, cT, np, s);
}

template <typename T, int LX, int V>
xl_status pass3_LV(const void* Tb, void* out, int nx, int ny, int cout, int cT, int np, cudaStream_t s,
                   DzReduce red) {
  constexpr int ROWS = rows_p3v<LX, sizeof(cplx<T>), V>();
  const size_t sm = (size_t)ROWS * tpitch(LX, sizeof(cplx<T>), ROWS) * sizeof(cplx<T>);
  const void* tw;
  XL_TRY(twiddles(LX, sizeof(T) == 8 ? XL_C128 : XL_C64, &tw));
  XL_TRY(smem_attr((const void*)k_rs_pass3<T, LX, V>, sm));
  dim3 grid((ny + ROWS - 1) / ROWS, np);
  LaunchScope ls("rs_pass3<" + std::to_string(LX) + ">", s);
  k_rs_pass3<T, LX, V><<<grid, ROWS * (LX / 16), sm, s>>>(
      (const cplx<T>*)Tb, (cplx<T>*)out, nx, ny, cout, cT, (const cplx<T>*)tw, red);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

// Pass 3 with the bulk-tensor gather (complex64, the default two rows per block).
template <int LX>
xl_status pass3_tma(const void* Tb, void* out, int nx, int ny, int cout, int cT, int np, cudaStream_t s,
                    DzReduce red) {
  constexpr int ROWS = kP3TmaRows;
  const size_t sm = (size_t)ROWS * srow(LX) * sizeof(float2) + 128;  // + alignment slack
  const void* tw;
  XL_TRY(twiddles(LX, XL_C64, &tw));
  XL_TRY(smem_attr((const void*)k_rs_pass3_tma<LX>, sm));
  const int last = ((np - 1) / cout) * cT + (np - 1) % cout;  // highest T plane read
  alignas(64) unsigned char map[128];
  XL_TRY(tensor_map_2d_u64(Tb, (uint64_t)ny, (uint64_t)(last + 1) * LX, (uint64_t)ny * sizeof(float2),
                           ROWS, 256, map));
  unsigned int* status = nullptr;
  XL_TRY(status_word(&status));
  dim3 grid((ny + ROWS - 1) / ROWS, np);
  LaunchScope ls("rs_pass3<" + std::to_string(LX) + ">", s);
  k_rs_pass3_tma<LX><<<grid, ROWS * (LX / 16), sm, s>>>(*reinterpret_cast<const CUtensorMap*>(map),
                                                        (float2*)out, nx, ny, cout, cT,
                                                        (const float2*)tw, red, status);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

inline bool pass3_tma_enabled() {
  const char* e = getenv("XL_P3_TMA");
  return !(e && e[0] == '0');
}

template <typename T, int LX>
xl_status pass3_L(const void* Tb, void* out, int nx, int ny, int cout, int cT, int np, cudaStream_t s,
                  DzReduce red) {
  if constexpr (sizeof(T) == 4 && LX >= 256) {
    if ((LX < kTuneMinL || tuned_variant(TUNE_RS_PASS3, LX, XL_C64) == 0) && ny % 2 == 0 &&
        pass3_tma_enabled())
      return pass3_tma<LX>(Tb, out, nx, ny, cout, cT, np, s, red);
  }
  if constexpr (LX >= kTuneMinL) {
    switch (tuned_variant(TUNE_RS_PASS3, LX, sizeof(T) == 8 ? XL_C128 : XL_C64)) {
      case 1: return pass3_LV<T, LX, 1>(Tb, out, nx, ny, cout, cT, np, s, red);
      case 2: return pass3_LV<T, LX, 2>(Tb, out, nx, ny, cout, cT, np, s, red);
    }
  }
  return pass3_LV<T, LX, 0>(Tb, out, nx, ny, cout, cT, np, s, red);
}

template <typename T, int LY, int MODE>
xl_status pass2_LM(void* Tb, const void* Ub, const void* Hq, double* dz, const P2Args& a, int nb,
                   cudaStream_t s, const void* Tr) {
  constexpr int ROWS = rows_cols<LY>();
  size_t sm = (size_t)p2_rows_per_team<T, LY, MODE>() * ROWS * srow(LY) * sizeof(cplx<T>);
  if (sm > (size_t)227 * 1024)
    return fail(XL_ERR_UNSUPPORTED,
                "vectorial RS: a column of this length needs more shared memory than an SM has "
                "(complex128 with nx = 4096)");
  const void* tw;
  XL_TRY(twiddles(LY, sizeof(T) == 8 ? XL_C128 : XL_C64, &tw));
  const int LX = 2 * a.nx;
  dim3 grid((LX + ROWS - 1) / ROWS, nb);
  LaunchScope ls("rs_pass2_m" + std::to_string(MODE) + (a.spec_out ? "_save<" : "<") + std::to_string(LY) + ">", s);
  alignas(64) unsigned char map[128] = {};
  if constexpr (sizeof(T) == 4 && (MODE == P2_RS || MODE == P2_RS_BWD_S)) {
    if (Tr) {  // input columns gathered from the row-major intermediate by bulk tensor copies
      constexpr int W = ROWS >= 2 ? ROWS : 2;
      const int ny = a.ny, boxr = ny < 256 ? ny : 256;
      XL_TRY(tensor_map_2d_u64(Tr, (uint64_t)LX, (uint64_t)nb * a.cT * ny, (uint64_t)LX * sizeof(float2),
                               W, boxr, map));
      P2Args ar = a;
      XL_TRY(status_word(&ar.status));
      sm += 128;  // alignment slack of the tile
      XL_TRY(smem_attr((const void*)k_rs_pass2<T, LY, MODE, true>, sm));
      k_rs_pass2<T, LY, MODE, true><<<grid, ROWS * (LY / 16), sm, s>>>(
          (cplx<T>*)Tb, (const cplx<T>*)Ub, (const cplx<T>*)Hq, dz, ar, (const cplx<T>*)tw,
          *reinterpret_cast<const CUtensorMap*>(map));
      XL_CUDA_TRY(cudaGetLastError());
      return XL_OK;
    }
  }
  if (Tr) return fail(XL_ERR_ARG, "rs_pass2: row-major input for this mode / precision");
  XL_TRY(smem_attr((const void*)k_rs_pass2<T, LY, MODE>, sm));
  k_rs_pass2<T, LY, MODE><<<grid, ROWS * (LY / 16), sm, s>>>(
      (cplx<T>*)Tb, (const cplx<T>*)Ub, (const cplx<T>*)Hq, dz, a, (const cplx<T>*)tw,
      *reinterpret_cast<const CUtensorMap*>(map));
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

template <typename T, int LY>
xl_status pass2_L(int mode, void* Tb, const void* Ub, const void* Hq, double* dz, const P2Args& a,
                  int nb, cudaStream_t s, const void* Tr) {
  switch (mode) {
    case P2_RS: return pass2_LM<T, LY, P2_RS>(Tb, Ub, Hq, dz, a, nb, s, Tr);
    case P2_VRS: return pass2_LM<T, LY, P2_VRS>(Tb, Ub, Hq, dz, a, nb, s, Tr);
    case P2_RS_BWD: return pass2_LM<T, LY, P2_RS_BWD>(Tb, Ub, Hq, dz, a, nb, s, Tr);
    case P2_VRS_BWD: return pass2_LM<T, LY, P2_VRS_BWD>(Tb, Ub, Hq, dz, a, nb, s, Tr);
    case P2_RS_BWD_S: return pass2_LM<T, LY, P2_RS_BWD_S>(Tb, Ub, Hq, dz, a, nb, s, Tr);
    case P2_VRS_BWD_S: return pass2_LM<T, LY, P2_VRS_BWD_S>(Tb, Ub, Hq, dz, a, nb, s, Tr);
  }
  return fail(XL_ERR_ARG, "rs_pass2: bad mode");
}

// Pass 1 into the row-major intermediate (complex64).
template <int LX>
xl_status pass1_rm_L(const void* in, void* Tr, int nx, int ny, int cin, int cT, int np, cudaStream_t s) {
  constexpr int ROWS = rows_cols<LX>();
  const size_t sm = (size_t)ROWS * srow(LX) * sizeof(float2);
  const void* tw;
  XL_TRY(twiddles(LX, XL_C64, &tw));
  XL_TRY(smem_attr((const void*)k_rs_pass1_rm<LX>, sm));
  dim3 grid((ny + ROWS - 1) / ROWS, np);
  LaunchScope ls("rs_pass1<" + std::to_string(LX) + ">", s);
  k_rs_pass1_rm<LX><<<grid, ROWS * (LX / 16), sm, s>>>((const float2*)in, (float2*)Tr, nx, ny, cin,
                                                      cT, (const float2*)tw);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

template <typename T, int LX, int LY>
xl_status gen_LL(void* S, void* Hq, const GenArgs& g, int nb, cudaStream_t s) {
  constexpr int RA = rows_transp<LX, sizeof(cplx<T>)>();
  constexpr int RB = rows_cols<LY>();
  const size_t sa = (size_t)RA * (tpitch(LX, sizeof(cplx<T>), RA) + LX / 2) * sizeof(cplx<T>);
  const size_t sb = (size_t)RB * srow(LY) * sizeof(cplx<T>);
  const void *twx, *twy;
  XL_TRY(twiddles(LX, sizeof(T) == 8 ? XL_C128 : XL_C64, &twx));
  XL_TRY(twiddles(LY, sizeof(T) == 8 ? XL_C128 : XL_C64, &twy));
  XL_TRY(smem_attr((const void*)k_gen_pass_a<T, LX>, sa));
  XL_TRY(smem_attr((const void*)k_gen_pass_b<T, LY>, sb));
  {
  LaunchScope ls("rs_gen_a<" + std::to_string(LX) + ">", s);
  k_gen_pass_a<T, LX><<<dim3((g.ny + RA - 1) / RA, nb), RA * (LX / 16), sa, s>>>(
      (cplx<T>*)S, g, (const cplx<T>*)twx);
  }
  XL_CUDA_TRY(cudaGetLastError());
  LaunchScope lsb("rs_gen_b<" + std::to_string(LY) + ">", s);
  k_gen_pass_b<T, LY><<<dim3((g.nx + 1 + RB - 1) / RB, nb), RB * (LY / 16), sb, s>>>(
      (const cplx<T>*)S, (cplx<T>*)Hq, g, (const cplx<T>*)twy);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

template <typename T, int LX>
xl_status gen_L(void* S, void* Hq, const GenArgs& g, int nb, cudaStream_t s) {
  switch (2 * g.ny) {
    case 64: return gen_LL<T, LX, 64>(S, Hq, g, nb, s);
    case 128: return gen_LL<T, LX, 128>(S, Hq, g, nb, s);
    case 256: return gen_LL<T, LX, 256>(S, Hq, g, nb, s);
    case 512: return gen_LL<T, LX, 512>(S, Hq, g, nb, s);
    case 1024: return gen_LL<T, LX, 1024>(S, Hq, g, nb, s);
    case 2048: return gen_LL<T, LX, 2048>(S, Hq, g, nb, s);
    case 4096: return gen_LL<T, LX, 4096>(S, Hq, g, nb, s);
    case 8192: return gen_LL<T, LX, 8192>(S, Hq, g, nb, s);
  }
  return fail(XL_ERR_UNSUPPORTED, "rs_generate: unsupported ny");
}

}  // namespace

#define XL_SWITCH_L(L, CALL)                               \
  switch (L) {                                             \
    case 64: return CALL(64);                              \
    case 128: return CALL(128);                            \
    case 256: return CALL(256);                            \
    case 512: return CALL(512);                            \
    case 1024: return CALL(1024);                          \
    case 2048: return CALL(2048);                          \
    case 4096: return CALL(4096);                          \
    case 8192: return CALL(8192);                          \
  }

template <>
xl_status rs_pass1_rm<XL_REAL>(const void* in, void* Tr, int nx, int ny, int cin, int cT, int np,
                               cudaStream_t s) {
  if constexpr (sizeof(XL_REAL) == 4) {
    switch (2 * nx) {
      case 256: return pass1_rm_L<256>(in, Tr, nx, ny, cin, cT, np, s);
      case 512: return pass1_rm_L<512>(in, Tr, nx, ny, cin, cT, np, s);
      case 1024: return pass1_rm_L<1024>(in, Tr, nx, ny, cin, cT, np, s);
      case 2048: return pass1_rm_L<2048>(in, Tr, nx, ny, cin, cT, np, s);
      case 4096: return pass1_rm_L<4096>(in, Tr, nx, ny, cin, cT, np, s);
      case 8192: return pass1_rm_L<8192>(in, Tr, nx, ny, cin, cT, np, s);
    }
  }
  return fail(XL_ERR_UNSUPPORTED, "rs_pass1_rm: complex64 rows of 256..8192");
}

template <>
xl_status rs_pass1<XL_REAL>(const void* in, void* Tb, int nx, int ny, int cin, int cT, int np,
                            cudaStream_t s) {
#define C1(L) pass1_L<XL_REAL, L>(in, Tb, nx, ny, cin, cT, np, s)
  XL_SWITCH_L(2 * nx, C1)
#undef C1
  return fail(XL_ERR_UNSUPPORTED, "rs_pass1: unsupported nx");
}

template <>
xl_status rs_pass3<XL_REAL>(const void* Tb, void* out, int nx, int ny, int cout, int cT, int np,
                            cudaStream_t s, DzReduce red) {
#define C3(L) pass3_L<XL_REAL, L>(Tb, out, nx, ny, cout, cT, np, s, red)
  XL_SWITCH_L(2 * nx, C3)
#undef C3
  return fail(XL_ERR_UNSUPPORTED, "rs_pass3: unsupported nx");
}

template <>
xl_status rs_pass2<XL_REAL>(int mode, void* Tb, const void* Ub, const void* Hq, double* dz,
                            const P2Args& a, int nb, cudaStream_t s, const void* Tr) {
#define C2(L) pass2_L<XL_REAL, L>(mode, Tb, Ub, Hq, dz, a, nb, s, Tr)
  XL_SWITCH_L(2 * a.ny, C2)
#undef C2
  return fail(XL_ERR_UNSUPPORTED, "rs_pass2: unsupported ny");
}

template <>
int rs_pass2_blocks<XL_REAL>(int nx, int ny) {
  const int LY = 2 * ny, TT = LY / 16;
  const int rows = (256 / TT) > 1 ? 256 / TT : 1;
  return (2 * nx + rows - 1) / rows;
}

template <>
xl_status rs_generate<XL_REAL>(void* S, void* Hq, const GenArgs& g, int nb, cudaStream_t s) {
#define CG(L) gen_L<XL_REAL, L>(S, Hq, g, nb, s)
  XL_SWITCH_L(2 * g.nx, CG)
#undef CG
  return fail(XL_ERR_UNSUPPORTED, "rs_generate: unsupported nx");
}

}  // namespace xl
