// C ABI of CZT / VCZT propagation onto an output window and its adjoint (host orchestration of
// xl_czt_kernels.cuh). Methods, "Features and performance": the chirped z-transform propagates
// onto an arbitrarily selected and sampled region of interest.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>

#include "xl_czt_launch.h"

namespace xl {
namespace {

int czt_len(int n, int m) {
  int L = 64;
  while (L < n + m - 1) L <<= 1;
  return L;
}

xl_status check_czt(const xl_grid* g, const xl_window* w, double wavelength, int32_t batch,
                    const double* z, int32_t flags, int32_t dtype) {
  if (!g || !w) return fail(XL_ERR_ARG, "grid or window is NULL");
  if (g->nx < 1 || g->ny < 1 || w->mx < 1 || w->my < 1)
    return fail(XL_ERR_ARG, "grid and window sizes must be positive");
  if (g->nx + w->mx - 1 > 8192 || g->ny + w->my - 1 > 8192)
    return fail(XL_ERR_UNSUPPORTED, "N + M - 1 must not exceed 8192 per axis");
  if (!(g->dx > 0) || !(g->dy > 0) || !(w->dxo > 0) || !(w->dyo > 0))
    return fail(XL_ERR_ARG, "pitches must be positive");
  if (!std::isfinite(g->x0) || !std::isfinite(g->y0) || !std::isfinite(w->xo0) || !std::isfinite(w->yo0))
    return fail(XL_ERR_ARG, "origins must be finite");
  if (!(wavelength > 0) || !std::isfinite(wavelength)) return fail(XL_ERR_ARG, "bad wavelength");
  if (batch < 0) return fail(XL_ERR_ARG, "batch < 0");
  if (dtype != XL_C64 && dtype != XL_C128) return fail(XL_ERR_ARG, "bad dtype");
  if (flags & ~XL_Z_DEVICE) return fail(XL_ERR_ARG, "unknown flag bits");
  if (batch > 0 && !z) return fail(XL_ERR_ARG, "z is NULL");
  if (batch > 0 && !(flags & XL_Z_DEVICE))
    for (int32_t b = 0; b < batch; ++b)
      if (!(z[b] > 0) || !std::isfinite(z[b])) return fail(XL_ERR_ARG, "z must be positive and finite");
  return XL_OK;
}

CztTabArgs tab_args(const xl_grid* g, const xl_window* w, double wavelength) {
  CztTabArgs a;
  a.nx = g->nx; a.ny = g->ny; a.mx = w->mx; a.my = w->my;
  a.Lx = czt_len(g->nx, w->mx);
  a.Ly = czt_len(g->ny, w->my);
  a.x0 = g->x0; a.dx = g->dx; a.y0 = g->y0; a.dy = g->dy;
  a.xo0 = w->xo0; a.dxo = w->dxo; a.yo0 = w->yo0; a.dyo = w->dyo;
  a.k = kTwoPi / wavelength;
  a.lambda = wavelength;
  a.zdev = nullptr;
  a.zval = 0;
  a.off_y = (int64_t)a.nx + a.mx + a.Lx;
  return a;
}

int64_t tab_elems(const CztTabArgs& a) { return a.off_y + a.ny + a.my + a.Ly; }

template <typename T>
xl_status get_tables(const xl_grid* g, const xl_window* w, double wavelength, const double* z,
                     int32_t flags, int32_t dtype, void* dev_tab, cudaStream_t s, const void** out) {
  CztTabArgs a = tab_args(g, w, wavelength);
  if (flags & XL_Z_DEVICE) {
    a.zdev = z;
    XL_TRY(czt_tables<T>(dev_tab, a, s));
    *out = dev_tab;
    return XL_OK;
  }
  a.zval = *z;
  std::string key = "czt";
  key_put(key, *g);
  key_put(key, *w);
  key_put(key, wavelength);
  key_put(key, *z);
  key_put(key, dtype);
  void* p = nullptr;
  XL_TRY(cached_table(key, (size_t)tab_elems(a) * sizeof(cplx<T>), s,
                      [&](void* buf) { return czt_tables<T>(buf, a, s); }, &p));
  *out = p;
  return XL_OK;
}

template <typename T>
void axes(const void* tab, const CztTabArgs& a, Axis<cplx<T>>* ax, Axis<cplx<T>>* ay) {
  const cplx<T>* t = (const cplx<T>*)tab;
  ax->pre = t;
  ax->post = t + a.nx;
  ax->bhat = t + a.nx + a.mx;
  const cplx<T>* u = t + a.off_y;
  ay->pre = u;
  ay->post = u + a.ny;
  ay->bhat = u + a.ny + a.my;
}

template <typename T>
xl_status run(bool adjoint, const void* in, void* out, int32_t batch, bool vec, int in_planes,
              const xl_grid* g, const xl_window* w, double wavelength, const double* z,
              int32_t flags, int32_t dtype, cudaStream_t s) {
  const CztTabArgs ta = tab_args(g, w, wavelength);
  const bool zdev = (flags & XL_Z_DEVICE) != 0;
  const int cT = vec ? 3 : 1;
  const size_t cs = sizeof(cplx<T>);
  const int64_t tplane = (int64_t)w->mx * g->ny;
  const int64_t in_plane = (int64_t)g->nx * g->ny, win_plane = (int64_t)w->mx * w->my;
  // Batch elements per launch: up to kCztRun, whatever their distances (each element reads the
  // chirp tables of its own distance), within 2 GB of T planes; the chunk's tables stay within
  // half of the table cache, so that filling one never evicts another of the same launch.
  const size_t tab_bytes1 = (size_t)tab_elems(ta) * cs;
  int64_t chunk = std::max<int64_t>(1, ((int64_t)2048 << 20) / (cT * tplane * (int64_t)cs));
  chunk = std::min<int64_t>(chunk, std::max<int64_t>(1, (int64_t)(table_cache_cap() / 2 / tab_bytes1)));
  chunk = std::min<int64_t>(chunk, kCztRun);
  if (zdev) chunk = 1;
  chunk = std::min<int64_t>(chunk, batch);
  auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
  const size_t t_bytes = (size_t)chunk * cT * tplane * cs;
  const size_t tab_bytes = zdev ? tab_bytes1 : 0;
  void* ws = nullptr;
  XL_TRY(workspace(s, al(t_bytes) + al(tab_bytes), &ws));
  void* Tb = ws;
  void* dev_tab = (char*)ws + al(t_bytes);
  CztDims d;
  std::memset(&d, 0, sizeof(d));
  d.nx = g->nx; d.ny = g->ny; d.mx = w->mx; d.my = w->my;
  d.x0 = g->x0; d.dx = g->dx; d.y0 = g->y0; d.dy = g->dy;
  d.xo0 = w->xo0; d.dxo = w->dxo; d.yo0 = w->yo0; d.dyo = w->dyo;
  const int cin = in_planes, cwin = vec ? 3 : 1;
  // scalar complex64 forward: row-major intermediate (XL_CZT_RM=0 keeps the transposed one)
  const char* rm_env = getenv("XL_CZT_RM");
  const bool rm = !adjoint && !vec && sizeof(T) == 4 && ta.Lx >= 256 && ta.Ly >= 256 &&
                  ta.Lx <= 8192 && ta.Ly <= 8192 && w->mx % 2 == 0 && !(rm_env && rm_env[0] == '0');
  d.in_planes = in_planes;
  d.adjoint = adjoint ? 1 : 0;
  for (int32_t b0 = 0; b0 < batch;) {
    const int nb = (int)std::min<int64_t>(chunk, batch - b0);
    AxisRun<cplx<T>> ax, ay;
    const void* tab0 = nullptr;  // element 0's tables: the base of the shifts
    const void* tab = nullptr;
    for (int e = 0; e < nb; ++e) {  // (nb is 1 with device distances)
      if (e == 0 || z[b0 + e] != z[b0 + e - 1])
        XL_TRY(get_tables<T>(g, w, wavelength, z + b0 + e, flags, dtype, dev_tab, s, &tab));
      if (e == 0) {
        Axis<cplx<T>> x1, y1;
        axes<T>(tab, ta, &x1, &y1);
        ax = axis_run(x1);
        ay = axis_run(y1);
        ax.per_elem = ay.per_elem = 1;
        tab0 = tab;
      }
      ax.shift[e] = ay.shift[e] = (const cplx<T>*)tab - (const cplx<T>*)tab0;
      d.z[e] = zdev ? 0.0 : z[b0 + e];
    }
    d.zdev = zdev ? z + b0 : nullptr;
    if (!adjoint) {
      const char* src = (const char*)in + (size_t)b0 * cin * in_plane * cs;
      char* dst = (char*)out + (size_t)b0 * cwin * win_plane * cs;
      if (rm) {  // the x pass stores row-major, the y pass gathers columns by bulk tensor copies
        XL_TRY(czt_fwd_rm<T>(ta.Lx, ta.Ly, src, Tb, dst, d, ax, ay, nb, s));
      } else {
        XL_TRY(czt_pass<T>(CZT_FWD_X, vec, ta.Lx, src, Tb, d, ax, nb, s));
        XL_TRY(czt_pass<T>(CZT_FWD_Y, vec, ta.Ly, Tb, dst, d, ay, nb, s));
      }
    } else {
      const char* src = (const char*)in + (size_t)b0 * cwin * win_plane * cs;
      char* dst = (char*)out + (size_t)b0 * cin * in_plane * cs;
      XL_TRY(czt_pass<T>(CZT_ADJ_Y, vec, ta.Ly, src, Tb, d, ay, nb, s));
      XL_TRY(czt_pass<T>(CZT_ADJ_X, vec, ta.Lx, Tb, dst, d, ax, nb, s));
      if (in_planes == 3) {
        // the unused Ez plane of a 3-component input receives a zero gradient
        XL_CUDA_TRY(cudaMemset2DAsync(dst + 2 * in_plane * cs, 3 * in_plane * cs, 0, in_plane * cs, nb, s));
      }
    }
    b0 += nb;
  }
  return XL_OK;
}

xl_status dispatch(bool adjoint, const void* in, void* out, int32_t batch, int32_t vec,
                   const xl_grid* g, const xl_window* w, double wavelength, const double* z,
                   int32_t flags, int32_t dtype, void* stream) {
  XL_TRY(check_czt(g, w, wavelength, batch, z, flags, dtype));
  if (batch == 0) return XL_OK;
  if (!in || !out) return fail(XL_ERR_ARG, "field pointer is NULL");
  if (in == out) return fail(XL_ERR_ARG, "output may not alias the input");
  if (vec < 0 || vec > 2) return fail(XL_ERR_ARG, "vectorial must be 0, 1 or 2");
  cudaStream_t s = (cudaStream_t)stream;
  const int in_planes = vec == 0 ? 1 : (vec == 1 ? 2 : 3);
  if (dtype == XL_C128) return run<double>(adjoint, in, out, batch, vec != 0, in_planes, g, w, wavelength, z, flags, dtype, s);
  return run<float>(adjoint, in, out, batch, vec != 0, in_planes, g, w, wavelength, z, flags, dtype, s);
}

}  // namespace
}  // namespace xl

using namespace xl;

extern "C" {

xl_status xl_czt_propagate(const void* u_in, void* u_out, int32_t batch, int32_t vectorial,
                           const xl_grid* grid, const xl_window* window, double wavelength,
                           const double* z, int32_t flags, int32_t dtype, void* stream) {
  return dispatch(false, u_in, u_out, batch, vectorial, grid, window, wavelength, z, flags, dtype,
                  stream);
}

xl_status xl_czt_propagate_backward(const void* g_out, void* g_in, int32_t batch,
                                    int32_t vectorial, const xl_grid* grid,
                                    const xl_window* window, double wavelength, const double* z,
                                    int32_t flags, int32_t dtype, void* stream) {
  return dispatch(true, g_out, g_in, batch, vectorial, grid, window, wavelength, z, flags, dtype,
                  stream);
}

}  // extern "C"
