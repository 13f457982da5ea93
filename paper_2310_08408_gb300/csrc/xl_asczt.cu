// C ABI of the angular-spectrum CZT and its adjoint (host orchestration of
// xl_asczt_kernels.cuh and the window passes of xl_czt_kernels.cuh). The exact-RS reading of the
// CZT propagator (Methods, "Features and performance"; CZT of Hu et al.): the spectrum of the
// sampled field times exp(i z kz), evaluated on an arbitrary window.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "xl_asczt_launch.h"
#include "xl_czt_launch.h"

namespace xl {
namespace {

xl_status check(const xl_grid* g, const xl_window* w, double wavelength, int32_t batch,
                const double* z, int32_t flags, int32_t dtype) {
  if (!g || !w) return fail(XL_ERR_ARG, "grid or window is NULL");
  if (!is_pow2(g->nx) || !is_pow2(g->ny) || g->nx < 64 || g->ny < 64 || g->nx > 4096 || g->ny > 4096)
    return fail(XL_ERR_UNSUPPORTED, "nx, ny must be powers of two in [64, 4096]");
  if (w->mx < 1 || w->my < 1) return fail(XL_ERR_ARG, "window sizes must be positive");
  if (g->nx + w->mx - 1 > 8192 || g->ny + w->my - 1 > 8192)
    return fail(XL_ERR_UNSUPPORTED, "N + M - 1 must not exceed 8192 per axis");
  if (!(g->dx > 0) || !(g->dy > 0) || !(w->dxo > 0) || !(w->dyo > 0) || !std::isfinite(g->dx) ||
      !std::isfinite(g->dy) || !std::isfinite(w->dxo) || !std::isfinite(w->dyo))
    return fail(XL_ERR_ARG, "pitches must be positive and finite");
  if (!std::isfinite(g->x0) || !std::isfinite(g->y0) || !std::isfinite(w->xo0) || !std::isfinite(w->yo0))
    return fail(XL_ERR_ARG, "origins must be finite");
  if (!(wavelength > 0) || !std::isfinite(wavelength)) return fail(XL_ERR_ARG, "bad wavelength");
  if (batch < 0) return fail(XL_ERR_ARG, "batch < 0");
  if (batch > 65535) return fail(XL_ERR_UNSUPPORTED, "batch > 65535");
  if (dtype != XL_C64 && dtype != XL_C128) return fail(XL_ERR_ARG, "bad dtype");
  if (flags & ~XL_Z_DEVICE) return fail(XL_ERR_ARG, "unknown flag bits");
  if (batch > 0 && !z) return fail(XL_ERR_ARG, "z is NULL");
  if (batch > 0 && !(flags & XL_Z_DEVICE))
    for (int32_t b = 0; b < batch; ++b)
      if (!(z[b] >= 0) || !std::isfinite(z[b])) return fail(XL_ERR_ARG, "z must be finite and >= 0");
  return XL_OK;
}

// Window-pass tables with the segment plan of each axis (no distance: no b2 rows).
CztTabArgs tab_args(const xl_grid* g, const xl_window* w, double wavelength, int dtype) {
  const int cs = dtype == XL_C128 ? 16 : 8;
  const CztAxisPlan px = czt_axis_plan(g->nx, w->mx, cs, false, false);
  const CztAxisPlan py = czt_axis_plan(g->ny, w->my, cs, false, false);
  CztTabArgs a;
  a.nx = g->nx; a.ny = g->ny; a.mx = w->mx; a.my = w->my;
  a.Lx = px.L; a.Ly = py.L;
  a.Sx = px.S; a.Sy = py.S;
  a.segx = px.seg; a.segy = py.seg;
  a.dz = 0;
  a.jcx = a.jcy = 0;
  a.x0 = g->x0; a.dx = g->dx; a.y0 = g->y0; a.dy = g->dy;
  a.xo0 = w->xo0; a.dxo = w->dxo; a.yo0 = w->yo0; a.dyo = w->dyo;
  a.k = kTwoPi / wavelength;
  a.lambda = wavelength;
  a.zdev = nullptr;
  a.zval = 0;
  a.off_y = czt_axis_elems(a.nx, a.mx, a.Lx, a.Sx, 0);
  return a;
}

template <typename T>
xl_status run(bool adjoint, const void* in, const void* u_in, void* out, double* g_z,
              int32_t batch, const xl_grid* g, const xl_window* w, double wavelength,
              const double* z, int32_t flags, int32_t dtype, cudaStream_t s) {
  typedef cplx<T> C;
  const size_t cs = sizeof(C);
  const int nx = g->nx, ny = g->ny, mx = w->mx, my = w->my;
  const int64_t plane = (int64_t)nx * ny, wplane = (int64_t)mx * my, tplane = (int64_t)mx * ny;
  const bool zdev = (flags & XL_Z_DEVICE) != 0;
  const bool want_field = !adjoint || out != nullptr;
  const bool want_dz = adjoint && g_z != nullptr;
  const CztTabArgs ta = tab_args(g, w, wavelength, dtype);
  if (ta.Lx == 0 || ta.Ly == 0) return fail(XL_ERR_UNSUPPORTED, "asczt: no transform plan fits");
  // window tables: no distance in them, cached per (grid, window, dtype)
  const int64_t tab_n = ta.off_y + czt_axis_elems(ta.ny, ta.my, ta.Ly, ta.Sy, 0);
  std::string key = "asczt2";
  key_put(key, *g);
  key_put(key, *w);
  key_put(key, dtype);
  void* tab = nullptr;
  XL_TRY(cached_table(key, (size_t)tab_n * cs, s,
                      [&](void* buf) { return asczt_tables<T>(buf, ta, s); }, &tab));
  AxisRun<C> ax, ay;  // one table for every element (no distance in the window sums)
  {
    const C* t = (const C*)tab;
    const C* u = t + ta.off_y;
    ax = axis_run(Axis<C>{t, t + nx, t + nx + mx, nullptr}, ta.Sx, ta.segx);
    ay = axis_run(Axis<C>{u, u + ny, u + ny + my, nullptr}, ta.Sy, ta.segy);
  }
  // Batch elements per launch: up to kCztRun whatever their distances (each element reads the
  // transfer tables of its own distance), within 2 GB of spectrum planes; the chunk's transfer
  // tables stay within half of the table cache, so that filling one never evicts another of the
  // same launch.
  const size_t h_bytes1 = (size_t)2 * plane * cs;
  int64_t chunk = std::max<int64_t>(1, ((int64_t)2048 << 20) / ((2 * plane + tplane + plane) * (int64_t)cs));
  chunk = std::min<int64_t>(chunk, std::max<int64_t>(1, (int64_t)(table_cache_cap() / 2 / h_bytes1)));
  chunk = std::min<int64_t>(chunk, kCztRun);
  if (zdev) chunk = 1;
  chunk = std::min<int64_t>(chunk, batch);
  const int nblk = want_dz ? as_dz_blocks<T>(ny, nx) : 0;
  auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
  const size_t b_plane = (size_t)chunk * plane * cs, b_t2 = (size_t)chunk * tplane * cs;
  const size_t b_tu = want_dz ? b_plane : 0, b_dz = (size_t)chunk * nblk * sizeof(double);
  const size_t b_h = zdev ? (size_t)2 * plane * cs : 0;
  void* ws = nullptr;
  XL_TRY(workspace(s, al(b_plane) * 2 + al(b_t2) + al(b_tu) + al(b_dz) + al(b_h), &ws));
  char* p = (char*)ws;
  void* Tb = p;
  void* Sb = p + al(b_plane);
  void* T2 = p + 2 * al(b_plane);
  void* TU = p + 2 * al(b_plane) + al(b_t2);
  double* dzp = (double*)(p + 2 * al(b_plane) + al(b_t2) + al(b_tu));
  void* Hdev = p + 2 * al(b_plane) + al(b_t2) + al(b_tu) + al(b_dz);

  CztDims d;
  std::memset(&d, 0, sizeof(d));
  d.nx = nx; d.ny = ny; d.mx = mx; d.my = my;
  d.x0 = g->x0; d.dx = g->dx; d.y0 = g->y0; d.dy = g->dy;
  d.xo0 = w->xo0; d.dxo = w->dxo; d.yo0 = w->yo0; d.dyo = w->dyo;
  d.zdev = nullptr;
  for (int i = 0; i < kCztRun; ++i) d.z[i] = 0.0;
  d.in_planes = 1;
  d.adjoint = adjoint ? 1 : 0;
  d.tb_elem = tplane;

  AsTransferArgs tr;
  tr.nx = nx; tr.ny = ny; tr.dx = g->dx; tr.dy = g->dy; tr.k = kTwoPi / wavelength;
  for (int32_t b0 = 0; b0 < batch;) {
    const int nb = (int)std::min<int64_t>(chunk, batch - b0);
    // transfer tables Hc | dHc of each element's distance
    const void* H = nullptr;
    AsShift hs = as_shared();
    if (zdev) {
      tr.zdev = z + b0;
      tr.zval = 0.0;
      XL_TRY(as_transfer<T>(Hdev, (char*)Hdev + plane * cs, tr, s));
      H = Hdev;
    } else {
      const void* he = nullptr;
      for (int e = 0; e < nb; ++e) {
        if (e == 0 || z[b0 + e] != z[b0 + e - 1]) {
          tr.zdev = nullptr;
          tr.zval = z[b0 + e];
          std::string hk = "asczt_h";
          key_put(hk, nx);
          key_put(hk, ny);
          key_put(hk, g->dx);
          key_put(hk, g->dy);
          key_put(hk, wavelength);
          key_put(hk, z[b0 + e]);
          key_put(hk, dtype);
          void* hp = nullptr;
          XL_TRY(cached_table(hk, h_bytes1, s, [&](void* buf) {
            return as_transfer<T>(buf, (char*)buf + plane * cs, tr, s);
          }, &hp));
          he = hp;
        }
        if (e == 0) H = he;
        hs.s[e] = (const C*)he - (const C*)H;
      }
      hs.per_elem = nb > 1 ? 1 : 0;
    }
    const void* dH = (const char*)H + plane * cs;
    if (!adjoint) {
      const char* src = (const char*)in + (size_t)b0 * plane * cs;
      char* dst = (char*)out + (size_t)b0 * wplane * cs;
      XL_TRY(as_fwd_pass<T>(AS_STAGE_A, nx, src, Tb, ny, nullptr, as_shared(), nb, s));
      XL_TRY(as_fwd_pass<T>(AS_STAGE_B, ny, Tb, Sb, nx, H, hs, nb, s));
      XL_TRY(czt_pass<T>(CZT_FWD_X, false, ta.Lx, Sb, T2, d, ax, nb, s));
      XL_TRY(czt_pass<T>(CZT_FWD_Y, false, ta.Ly, T2, dst, d, ay, nb, s));
    } else {
      const char* src = (const char*)in + (size_t)b0 * wplane * cs;
      XL_TRY(czt_pass<T>(CZT_ADJ_Y, false, ta.Ly, src, T2, d, ay, nb, s));
      XL_TRY(czt_pass<T>(CZT_ADJ_X, false, ta.Lx, T2, Sb, d, ax, nb, s));
      if (want_dz)
        XL_TRY(as_fwd_pass<T>(AS_STAGE_A, nx, (const char*)u_in + (size_t)b0 * plane * cs, TU, ny,
                              nullptr, as_shared(), nb, s));
      XL_TRY(as_adj_pass<T>(AS_STAGE_B, ny, Sb, Tb, nx, H, dH, hs, want_dz ? TU : nullptr,
                            want_dz ? dzp : nullptr, nb, s));
      if (want_field)
        XL_TRY(as_adj_pass<T>(AS_STAGE_A, nx, Tb, (char*)out + (size_t)b0 * plane * cs, ny, nullptr,
                              nullptr, as_shared(), nullptr, nullptr, nb, s));
      if (want_dz) {
        LaunchScope ls("asczt_reduce", s);
        k_as_reduce<<<nb, 256, 0, s>>>(dzp, nblk, g_z + b0);
        XL_CUDA_TRY(cudaGetLastError());
      }
    }
    b0 += nb;
  }
  return XL_OK;
}

xl_status dispatch(bool adjoint, const void* in, const void* u_in, void* out, double* g_z,
                   int32_t batch, const xl_grid* g, const xl_window* w, double wavelength,
                   const double* z, int32_t flags, int32_t dtype, void* stream) {
  XL_TRY(check(g, w, wavelength, batch, z, flags, dtype));
  if (batch == 0) return XL_OK;
  if (!in) return fail(XL_ERR_ARG, "input field is NULL");
  if (!adjoint && !out) return fail(XL_ERR_ARG, "output field is NULL");
  if (adjoint && g_z && !u_in) return fail(XL_ERR_ARG, "g_z requested but the forward input is NULL");
  if (adjoint && !out && !g_z) return XL_OK;
  if (in == out) return fail(XL_ERR_ARG, "output may not alias the input");
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == XL_C128)
    return run<double>(adjoint, in, u_in, out, g_z, batch, g, w, wavelength, z, flags, dtype, s);
  return run<float>(adjoint, in, u_in, out, g_z, batch, g, w, wavelength, z, flags, dtype, s);
}

}  // namespace
}  // namespace xl

using namespace xl;

extern "C" {

xl_status xl_asczt_propagate(const void* u_in, void* u_out, int32_t batch, const xl_grid* grid,
                             const xl_window* window, double wavelength, const double* z,
                             int32_t flags, int32_t dtype, void* stream) {
  return dispatch(false, u_in, nullptr, u_out, nullptr, batch, grid, window, wavelength, z, flags,
                  dtype, stream);
}

xl_status xl_asczt_propagate_backward(const void* g_out, const void* u_in, void* g_in,
                                      double* g_z, int32_t batch, const xl_grid* grid,
                                      const xl_window* window, double wavelength, const double* z,
                                      int32_t flags, int32_t dtype, void* stream) {
  return dispatch(true, g_out, u_in, g_in, g_z, batch, grid, window, wavelength, z, flags, dtype,
                  stream);
}

}  // extern "C"
