// Definitions of the CZT launchers for one precision; included with XL_REAL defined.
// The window-pass kernels of each transform length are instantiated in part files
// (XL_CZT_LENGTHS defined: xl_czt_c64_*.cu / xl_czt_c128_*.cu) so that they compile in
// parallel; the dispatching file (XL_CZT_LENGTHS undefined) holds the switch, the chirp-table
// launchers and extern declarations of those instantiations.
#include "xl_czt_launch.h"

namespace xl {

template <typename T, int L, bool VEC, int V, bool DZ>
xl_status pass_LVV(int which, const void* src, void* dst, const CztDims& d, const AxisRun<cplx<T>>& ax,
                   int nb, cudaStream_t s, const CztDzArgs<cplx<T>>* dz, int* blocks) {
  typedef cplx<T> C;
  constexpr int ROWS = czt_rows<L, sizeof(C), VEC, V>();
  const bool fwd = which == CZT_FWD_X || which == CZT_FWD_Y;
  const size_t sm = czt_smem_bytes<L, sizeof(C), VEC, V>(ax.nseg > 1, DZ && fwd);
  if (sm > (size_t)227 * 1024) return fail(XL_ERR_UNSUPPORTED, "czt: segment plan exceeds shared memory");
  const void* tw;
  XL_TRY(twiddles(L, sizeof(T) == 8 ? XL_C128 : XL_C64, czt_plan_of<V>(), &tw));
  const C* twc = (const C*)tw;
  const dim3 blk(ROWS * (L / 16));
  const CztSaved<C> sv = dz ? dz->sv : CztSaved<C>{nullptr, 0, 0, 0, 0};
  double* dzp = dz ? dz->dzp : nullptr;
  const std::string tag = std::string(VEC ? "_vec<" : "<") + std::to_string(L) + ">" + (DZ ? "_dz" : "") +
                          (czt_plan_of<V>() ? "_p" + std::to_string(czt_plan_of<V>()) : "");
  int gx = 0;
  switch (which) {
    case CZT_FWD_X:
      gx = (d.ny + ROWS - 1) / ROWS;
      XL_TRY(smem_attr((const void*)k_czt_fwd_x<T, L, VEC, V, DZ>, sm));
      {
        LaunchScope ls("czt_fwd_x" + tag, s);
        k_czt_fwd_x<T, L, VEC, V, DZ><<<dim3(gx, nb), blk, sm, s>>>((const C*)src, (C*)dst, d, ax, twc, sv);
      }
      break;
    case CZT_FWD_Y:
      gx = (d.mx + ROWS - 1) / ROWS;
      XL_TRY(smem_attr((const void*)k_czt_fwd_y<T, L, VEC, V, DZ>, sm));
      {
        LaunchScope ls("czt_fwd_y" + tag, s);
        k_czt_fwd_y<T, L, VEC, V, DZ><<<dim3(gx, nb), blk, sm, s>>>((const C*)src, (C*)dst, d, ax, twc, sv);
      }
      break;
    case CZT_ADJ_Y:
      gx = (d.mx + ROWS - 1) / ROWS;
      XL_TRY(smem_attr((const void*)k_czt_adj_y<T, L, VEC, V, DZ>, sm));
      {
        LaunchScope ls("czt_adj_y" + tag, s);
        k_czt_adj_y<T, L, VEC, V, DZ><<<dim3(gx, nb), blk, sm, s>>>((const C*)src, (C*)dst, d, ax, twc, sv,
                                                                    dzp);
      }
      break;
    case CZT_ADJ_X:
      gx = (d.ny + ROWS - 1) / ROWS;
      XL_TRY(smem_attr((const void*)k_czt_adj_x<T, L, VEC, V, DZ>, sm));
      {
        LaunchScope ls("czt_adj_x" + tag, s);
        k_czt_adj_x<T, L, VEC, V, DZ><<<dim3(gx, nb), blk, sm, s>>>((const C*)src, (C*)dst, d, ax, twc, sv,
                                                                    dzp, dz ? dz->u_in : nullptr);
      }
      break;
    default:
      return fail(XL_ERR_ARG, "czt_pass: bad pass");
  }
  XL_CUDA_TRY(cudaGetLastError());
  if (blocks) *blocks = gx;
  return XL_OK;
}

// The autotuner's variant for this pass and length (scalar passes of long rows only; the
// distance-gradient forms use the default shape).
template <typename T, int L, bool VEC>
xl_status pass_LV(int which, const void* src, void* dst, const CztDims& d, const AxisRun<cplx<T>>& ax,
                  int nb, cudaStream_t s, const CztDzArgs<cplx<T>>* dz, int* blocks) {
  constexpr int CS = sizeof(cplx<T>);
  const int fam = which == CZT_FWD_X ? TUNE_CZT_FWD_X : which == CZT_FWD_Y ? TUNE_CZT_FWD_Y
                : which == CZT_ADJ_X ? TUNE_CZT_ADJ_X : TUNE_CZT_ADJ_Y;
  const int var = (!VEC && L >= 512) ? tuned_variant(fam, L, sizeof(T) == 8 ? XL_C128 : XL_C64) : 0;
  // radix-plan variants (complex64 scalar passes of the lengths with an odd stage); the
  // distance-gradient forms follow the plan, not the rows variants
  constexpr bool PLANS = CS == 8 && !VEC && (L == 512 || L == 1024 || L == 2048);
  if (dz && dz->on) {
    if constexpr (PLANS) {
      if (var == 3) return pass_LVV<T, L, VEC, 3, true>(which, src, dst, d, ax, nb, s, dz, blocks);
      if (var == 4) return pass_LVV<T, L, VEC, 4, true>(which, src, dst, d, ax, nb, s, dz, blocks);
    }
    return pass_LVV<T, L, VEC, 0, true>(which, src, dst, d, ax, nb, s, dz, blocks);
  }
  if constexpr (PLANS) {
    if (var == 3) return pass_LVV<T, L, VEC, 3, false>(which, src, dst, d, ax, nb, s, nullptr, blocks);
    if (var == 4) return pass_LVV<T, L, VEC, 4, false>(which, src, dst, d, ax, nb, s, nullptr, blocks);
  }
  if constexpr (!VEC && L >= kTuneMinL) {
    const bool multi = ax.nseg > 1;
    switch (var) {
      case 1:
        if (czt_smem_bytes<L, CS, VEC, 1>(multi) <= (size_t)227 * 1024)
          return pass_LVV<T, L, VEC, 1, false>(which, src, dst, d, ax, nb, s, nullptr, blocks);
        break;
      case 2:
        if (czt_smem_bytes<L, CS, VEC, 2>(multi) <= (size_t)227 * 1024)
          return pass_LVV<T, L, VEC, 2, false>(which, src, dst, d, ax, nb, s, nullptr, blocks);
        break;
    }
  }
  return pass_LVV<T, L, VEC, 0, false>(which, src, dst, d, ax, nb, s, nullptr, blocks);
}

#define XL_CZT_PASS_SIG(LL, VV)                                                                    \
  xl_status pass_LV<XL_REAL, LL, VV>(int, const void*, void*, const CztDims&, const AxisRun<cplx<XL_REAL>>&, \
                                     int, cudaStream_t, const CztDzArgs<cplx<XL_REAL>>*, int*)
#define XL_CZT_INSTANTIATE(LL) \
  template XL_CZT_PASS_SIG(LL, false); \
  template XL_CZT_PASS_SIG(LL, true);
#define XL_CZT_EXTERN(LL) \
  extern template XL_CZT_PASS_SIG(LL, false); \
  extern template XL_CZT_PASS_SIG(LL, true);

#ifdef XL_CZT_LENGTHS
XL_CZT_LENGTHS(XL_CZT_INSTANTIATE)
}  // namespace xl
#else
XL_CZT_EXTERN(64) XL_CZT_EXTERN(128) XL_CZT_EXTERN(256) XL_CZT_EXTERN(512)
XL_CZT_EXTERN(1024) XL_CZT_EXTERN(2048) XL_CZT_EXTERN(4096) XL_CZT_EXTERN(8192)

namespace {

template <typename T, int L>
xl_status bhat_L(cplx<T>* rows, int64_t stride, int nrows, cudaStream_t s) {
  const size_t sm = (size_t)srow(L) * sizeof(cplx<T>);
  const void* tw;
  XL_TRY(twiddles(L, sizeof(T) == 8 ? XL_C128 : XL_C64, &tw));
  XL_TRY(smem_attr((const void*)k_czt_bhat<T, L>, sm));
  LaunchScope ls("czt_bhat<" + std::to_string(L) + ">", s);
  k_czt_bhat<T, L><<<nrows, L / 16, sm, s>>>(rows, stride, (const cplx<T>*)tw);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

template <typename T>
xl_status bhat(int L, cplx<T>* rows, int64_t stride, int nrows, cudaStream_t s) {
  switch (L) {
    case 64: return bhat_L<T, 64>(rows, stride, nrows, s);
    case 128: return bhat_L<T, 128>(rows, stride, nrows, s);
    case 256: return bhat_L<T, 256>(rows, stride, nrows, s);
    case 512: return bhat_L<T, 512>(rows, stride, nrows, s);
    case 1024: return bhat_L<T, 1024>(rows, stride, nrows, s);
    case 2048: return bhat_L<T, 2048>(rows, stride, nrows, s);
    case 4096: return bhat_L<T, 4096>(rows, stride, nrows, s);
    case 8192: return bhat_L<T, 8192>(rows, stride, nrows, s);
  }
  return fail(XL_ERR_UNSUPPORTED, "czt: unsupported transform length");
}

// Scalar complex64 forward with the row-major intermediate: x pass and y pass of one length each.
template <int L>
xl_status rm_x_L(const void* src, void* Tr, const CztDims& d, const AxisRun<float2>& ax, int nb,
                 cudaStream_t s) {
  constexpr int ROWS = czt_rm_rows<L>();
  const size_t sm = (size_t)ROWS * srow(L) * sizeof(float2);
  const void* tw;
  XL_TRY(twiddles(L, XL_C64, &tw));
  XL_TRY(smem_attr((const void*)k_czt_fwd_x_rm<L>, sm));
  LaunchScope ls("czt_fwd_x<" + std::to_string(L) + ">", s);
  k_czt_fwd_x_rm<L><<<dim3((d.ny + ROWS - 1) / ROWS, nb), ROWS * (L / 16), sm, s>>>(
      (const float2*)src, (float2*)Tr, d, ax, (const float2*)tw);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

template <int L>
xl_status rm_y_L(const void* Tr, void* dst, const CztDims& d, const AxisRun<float2>& ay, int nb,
                 cudaStream_t s) {
  constexpr int ROWS = czt_rows<L, 8, false, 0>();
  constexpr int W = ROWS >= 2 ? ROWS : 2;
  const size_t sm = (size_t)ROWS * tpitch(L, 8, ROWS) * sizeof(float2) + 128;  // + alignment slack
  const void* tw;
  XL_TRY(twiddles(L, XL_C64, &tw));
  XL_TRY(smem_attr((const void*)k_czt_fwd_y_rm<L, ROWS>, sm));
  alignas(64) unsigned char map[128];
  XL_TRY(tensor_map_2d_u64(Tr, (uint64_t)d.mx, (uint64_t)nb * d.ny, (uint64_t)d.mx * sizeof(float2), W,
                           d.ny < 256 ? d.ny : 256, map));
  unsigned int* status = nullptr;
  XL_TRY(status_word(&status));
  LaunchScope ls("czt_fwd_y<" + std::to_string(L) + ">", s);
  k_czt_fwd_y_rm<L, ROWS><<<dim3((d.mx + ROWS - 1) / ROWS, nb), ROWS * (L / 16), sm, s>>>(
      *reinterpret_cast<const CUtensorMap*>(map), (float2*)dst, d, ay, (const float2*)tw, status);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

template <typename T>
xl_status fwd_rm(int Lx, int Ly, const void* src, void* Tr, void* dst, const CztDims& d,
                 const AxisRun<cplx<T>>& ax, const AxisRun<cplx<T>>& ay, int nb, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    xl_status st = XL_ERR_UNSUPPORTED;
#define RX(LL) case LL: st = rm_x_L<LL>(src, Tr, d, ax, nb, s); break;
#define RY(LL) case LL: st = rm_y_L<LL>(Tr, dst, d, ay, nb, s); break;
    switch (Lx) { RX(256) RX(512) RX(1024) RX(2048) RX(4096) RX(8192) }
    if (st != XL_OK) return st == XL_ERR_UNSUPPORTED ? fail(st, "czt rm: unsupported length") : st;
    st = XL_ERR_UNSUPPORTED;
    switch (Ly) { RY(256) RY(512) RY(1024) RY(2048) RY(4096) RY(8192) }
#undef RX
#undef RY
    if (st != XL_OK) return st == XL_ERR_UNSUPPORTED ? fail(st, "czt rm: unsupported length") : st;
    return XL_OK;
  } else {
    return fail(XL_ERR_UNSUPPORTED, "czt rm: complex64 only");
  }
}

}  // namespace

template <>
xl_status czt_fwd_rm<XL_REAL>(int Lx, int Ly, const void* src, void* Tr, void* dst, const CztDims& d,
                              const AxisRun<cplx<XL_REAL>>& ax, const AxisRun<cplx<XL_REAL>>& ay,
                              int nb, cudaStream_t s) {
  return fwd_rm<XL_REAL>(Lx, Ly, src, Tr, dst, d, ax, ay, nb, s);
}

template <>
xl_status czt_pass<XL_REAL>(int which, bool vec, int L, const void* src, void* dst,
                            const CztDims& d, const AxisRun<cplx<XL_REAL>>& ax, int nb, cudaStream_t s,
                            const CztDzArgs<cplx<XL_REAL>>* dz, int* blocks) {
#define CP(LL)                                                                           \
  case LL:                                                                               \
    return vec ? pass_LV<XL_REAL, LL, true>(which, src, dst, d, ax, nb, s, dz, blocks)  \
               : pass_LV<XL_REAL, LL, false>(which, src, dst, d, ax, nb, s, dz, blocks);
  switch (L) {
    CP(64) CP(128) CP(256) CP(512) CP(1024) CP(2048) CP(4096) CP(8192)
  }
#undef CP
  return fail(XL_ERR_UNSUPPORTED, "czt: unsupported transform length");
}

template <>
xl_status czt_tables<XL_REAL>(void* tab, const CztTabArgs& a, cudaStream_t s) {
  typedef cplx<XL_REAL> C;
  const int64_t total = czt_axis_elems(a.nx, a.mx, a.Lx, a.Sx, a.dz) + czt_axis_elems(a.ny, a.my, a.Ly, a.Sy, a.dz);
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 1024);
  {
  LaunchScope ls("czt_tables", s);
  k_czt_tables<XL_REAL><<<blocks, 256, 0, s>>>((C*)tab, a);
  }
  XL_CUDA_TRY(cudaGetLastError());
  C* t = (C*)tab;
  const int rx = (a.dz ? 2 : 1) * a.Sx, ry = (a.dz ? 2 : 1) * a.Sy;
  XL_TRY(bhat<XL_REAL>(a.Lx, t + a.nx + a.mx, a.Lx, rx, s));
  XL_TRY(bhat<XL_REAL>(a.Ly, t + a.off_y + a.ny + a.my, a.Ly, ry, s));
  return XL_OK;
}

template <>
xl_status asczt_tables<XL_REAL>(void* tab, const CztTabArgs& a, cudaStream_t s) {
  typedef cplx<XL_REAL> C;
  const int64_t total = czt_axis_elems(a.nx, a.mx, a.Lx, a.Sx, 0) + czt_axis_elems(a.ny, a.my, a.Ly, a.Sy, 0);
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 1024);
  {
    LaunchScope ls("asczt_tables", s);
    k_asczt_tables<XL_REAL><<<blocks, 256, 0, s>>>((C*)tab, a);
  }
  XL_CUDA_TRY(cudaGetLastError());
  C* t = (C*)tab;
  XL_TRY(bhat<XL_REAL>(a.Lx, t + a.nx + a.mx, a.Lx, a.Sx, s));
  XL_TRY(bhat<XL_REAL>(a.Ly, t + a.off_y + a.ny + a.my, a.Ly, a.Sy, s));
  return XL_OK;
}

}  // namespace xl
#endif  // XL_CZT_LENGTHS
