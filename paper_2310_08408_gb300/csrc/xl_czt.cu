// C ABI of CZT / VCZT propagation onto an output window, its adjoint and its distance gradient
// (host orchestration of xl_czt_kernels.cuh). Methods, "Features and performance": the chirped
// z-transform propagates onto an arbitrarily selected and sampled region of interest.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>

#include "xl_czt_launch.h"

namespace xl {

namespace {

template <int L> size_t smem_need_L(int cs, bool vec, bool multi, bool dz) {
  if (cs == 8) return vec ? czt_smem_bytes<L, 8, true, 0>(multi, dz) : czt_smem_bytes<L, 8, false, 0>(multi, dz);
  return vec ? czt_smem_bytes<L, 16, true, 0>(multi, dz) : czt_smem_bytes<L, 16, false, 0>(multi, dz);
}

size_t czt_smem_need(int L, int cs, bool vec, bool multi, bool dz) {
  switch (L) {
    case 64: return smem_need_L<64>(cs, vec, multi, dz);
    case 128: return smem_need_L<128>(cs, vec, multi, dz);
    case 256: return smem_need_L<256>(cs, vec, multi, dz);
    case 512: return smem_need_L<512>(cs, vec, multi, dz);
    case 1024: return smem_need_L<1024>(cs, vec, multi, dz);
    case 2048: return smem_need_L<2048>(cs, vec, multi, dz);
    case 4096: return smem_need_L<4096>(cs, vec, multi, dz);
    case 8192: return smem_need_L<8192>(cs, vec, multi, dz);
  }
  return ~(size_t)0;
}

}  // namespace

CztAxisPlan czt_axis_plan(int N, int M, int csize, bool vec, bool dz) {
  CztAxisPlan best{0, 1, N};
  double best_cost = 1e300;
  for (int S = 1; S <= 64 && S <= N; S *= 2) {
    const int seg = (N + S - 1) / S;
    if ((int64_t)(S - 1) * seg >= N) continue;  // a segment would be empty
    int L = 64;
    while (L < seg + M - 1) L <<= 1;
    if (L > 8192) continue;
    if (czt_smem_need(L, csize, vec, S > 1, dz) > (size_t)227 * 1024) continue;
    // S forward transforms and one inverse (or one forward and S inverse), plus the per-segment
    // loads and spectrum products
    const double cost = (S + 1.0) * L * std::log2((double)L) + 4.0 * S * L;
    if (cost < best_cost * (1.0 - 1e-9)) {
      best = CztAxisPlan{L, S, seg};
      best_cost = cost;
    }
  }
  return best;
}

xl_status czt_dz_finalize(const double* py, int nby, const double* px, int nbx, const double* zdev,
                          const CztDims& d, double k, bool phase_invariant, double* g_z, int nb,
                          cudaStream_t s) {
  LaunchScope ls("czt_dz_finalize", s);
  k_czt_dz_finalize<<<nb, 256, 0, s>>>(py, nby, px, nbx, zdev, d, k, phase_invariant ? 1 : 0, g_z);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

namespace {

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
  if (flags & ~(XL_Z_DEVICE | XL_PHASE_INVARIANT | XL_ACCUMULATE)) return fail(XL_ERR_ARG, "unknown flag bits");
  if (batch > 0 && !z) return fail(XL_ERR_ARG, "z is NULL");
  if (batch > 0 && !(flags & XL_Z_DEVICE))
    for (int32_t b = 0; b < batch; ++b)
      if (!(z[b] > 0) || !std::isfinite(z[b])) return fail(XL_ERR_ARG, "z must be positive and finite");
  return XL_OK;
}

struct Plans {
  CztAxisPlan x, y;
};

Plans plans(const xl_grid* g, const xl_window* w, int dtype, bool vec, bool dz) {
  const int cs = dtype == XL_C128 ? 16 : 8;
  return Plans{czt_axis_plan(g->nx, w->mx, cs, vec, dz), czt_axis_plan(g->ny, w->my, cs, vec, dz)};
}

// The tables always hold the distance-gradient rows b2 (a few transforms of length L).
CztTabArgs tab_args(const xl_grid* g, const xl_window* w, double wavelength, const Plans& pl) {
  CztTabArgs a;
  a.nx = g->nx; a.ny = g->ny; a.mx = w->mx; a.my = w->my;
  a.Lx = pl.x.L; a.Ly = pl.y.L;
  a.Sx = pl.x.S; a.Sy = pl.y.S;
  a.segx = pl.x.seg; a.segy = pl.y.seg;
  a.dz = 1;
  a.jcx = w->mx / 2 - g->nx / 2;
  a.jcy = w->my / 2 - g->ny / 2;
  a.x0 = g->x0; a.dx = g->dx; a.y0 = g->y0; a.dy = g->dy;
  a.xo0 = w->xo0; a.dxo = w->dxo; a.yo0 = w->yo0; a.dyo = w->dyo;
  a.k = kTwoPi / wavelength;
  a.lambda = wavelength;
  a.zdev = nullptr;
  a.zval = 0;
  a.off_y = czt_axis_elems(a.nx, a.mx, a.Lx, a.Sx, a.dz);
  return a;
}

int64_t tab_elems(const CztTabArgs& a) { return a.off_y + czt_axis_elems(a.ny, a.my, a.Ly, a.Sy, a.dz); }

template <typename T>
xl_status get_tables(const xl_grid* g, const xl_window* w, double wavelength, const Plans& pl,
                     const double* z, int32_t flags, int32_t dtype, void* dev_tab, cudaStream_t s,
                     const void** out) {
  CztTabArgs a = tab_args(g, w, wavelength, pl);
  if (flags & XL_Z_DEVICE) {
    a.zdev = z;
    XL_TRY(czt_tables<T>(dev_tab, a, s));
    *out = dev_tab;
    return XL_OK;
  }
  a.zval = *z;
  std::string key = "czt2";
  key_put(key, *g);
  key_put(key, *w);
  key_put(key, wavelength);
  key_put(key, *z);
  key_put(key, dtype);
  key_put(key, pl);
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
  ax->b2hat = ax->bhat + (int64_t)a.Sx * a.Lx;
  const cplx<T>* u = t + a.off_y;
  ay->pre = u;
  ay->post = u + a.ny;
  ay->bhat = u + a.ny + a.my;
  ay->b2hat = ay->bhat + (int64_t)a.Sy * a.Ly;
}

// Complex elements a forward with saved sums keeps per batch element (see CztSaved).
struct SaveLayout {
  int64_t elem, off_a2x, off_a2y, off_up;
};
SaveLayout save_layout(const xl_grid* g, const xl_window* w, const Plans& pl, int cT) {
  SaveLayout L;
  const int64_t tplane = (int64_t)w->mx * g->ny;
  L.off_a2x = cT * tplane;
  L.off_a2y = L.off_a2x + (int64_t)cT * g->ny * pl.x.L;
  L.off_up = L.off_a2y + (int64_t)cT * w->mx * pl.y.L;
  L.elem = L.off_up + (int64_t)cT * w->mx * w->my;
  return L;
}

DzAxis dz_axis(int N, int M, double s0, double D, double S0, double dd) {
  const int pc = M / 2, mc = N / 2;
  const double a = (S0 + pc * dd) - (s0 + mc * D);
  DzAxis r;
  r.a2 = (float)(a * a);
  r.f1 = (float)(2.0 * a * dd);
  r.f2 = (float)(dd * dd - dd * D);
  r.g1 = (float)(-2.0 * a * D);
  r.g2 = (float)(D * D - dd * D);
  r.dD = (float)(dd * D);
  r.pc = pc;
  r.mc = mc;
  return r;
}

enum Mode { FWD = 0, FWD_SAVE = 1, ADJ = 2 };

// One call. FWD: in -> out. FWD_SAVE: in -> out, and the saved sums into `saved`.
// ADJ: in (window cotangent) -> out (grid gradient, nullable when only g_z is wanted); with g_z,
// the distance gradient from `saved` (or, when NULL, from a forward with saved sums run here into
// workspace on u_in).
template <typename T>
xl_status run(Mode mode, const void* in, void* out, const void* u_in, void* saved, double* g_z,
              int32_t batch, bool vec, int in_planes, const xl_grid* g, const xl_window* w,
              double wavelength, const double* z, int32_t flags, int32_t dtype, cudaStream_t s) {
  typedef cplx<T> C;
  const bool adjoint = mode == ADJ;
  const bool want_dz = adjoint && g_z != nullptr;
  const bool dzmode = want_dz || mode == FWD_SAVE;
  const Plans pl = plans(g, w, dtype, vec, dzmode);
  if (pl.x.L == 0 || pl.y.L == 0) return fail(XL_ERR_UNSUPPORTED, "czt: no transform plan fits");
  const CztTabArgs ta = tab_args(g, w, wavelength, pl);
  const bool zdev = (flags & XL_Z_DEVICE) != 0;
  const int cT = vec ? 3 : 1;
  const size_t cs = sizeof(C);
  const int64_t tplane = (int64_t)w->mx * g->ny;
  const int64_t in_plane = (int64_t)g->nx * g->ny, win_plane = (int64_t)w->mx * w->my;
  const SaveLayout sl = save_layout(g, w, pl, cT);
  const bool recompute = want_dz && saved == nullptr;  // saved sums formed here
  const bool scratch_gin = adjoint && out == nullptr;
  const int cwin = vec ? 3 : 1;
  // Batch elements per launch: up to kCztRun, whatever their distances (each element reads the
  // chirp tables of its own distance), within 2 GB of workspace; the chunk's tables stay within
  // half of the table cache, so that filling one never evicts another of the same launch.
  const size_t tab_bytes1 = (size_t)tab_elems(ta) * cs;
  int64_t per_elem = cT * tplane;
  if (recompute) per_elem += sl.elem + cwin * win_plane;
  if (scratch_gin) per_elem += in_planes * in_plane;
  int64_t chunk = std::max<int64_t>(1, ((int64_t)2048 << 20) / (per_elem * (int64_t)cs));
  chunk = std::min<int64_t>(chunk, std::max<int64_t>(1, (int64_t)(table_cache_cap() / 2 / tab_bytes1)));
  chunk = std::min<int64_t>(chunk, kCztRun);
  if (zdev) chunk = 1;
  chunk = std::min<int64_t>(chunk, batch);
  auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
  const size_t b_t = (size_t)chunk * cT * tplane * cs;
  const size_t b_tab = zdev ? tab_bytes1 : 0;
  const size_t b_py = want_dz ? (size_t)chunk * w->mx * 6 * sizeof(double) : 0;
  const size_t b_px = want_dz ? (size_t)chunk * g->ny * 2 * sizeof(double) : 0;
  const size_t b_sv = recompute ? (size_t)chunk * sl.elem * cs : 0;
  const size_t b_win = recompute ? (size_t)chunk * cwin * win_plane * cs : 0;
  const size_t b_gin = scratch_gin ? (size_t)chunk * in_planes * in_plane * cs : 0;
  void* ws = nullptr;
  XL_TRY(workspace(s, al(b_t) + al(b_tab) + al(b_py) + al(b_px) + al(b_sv) + al(b_win) + al(b_gin), &ws));
  char* wp = (char*)ws;
  void* Tb = wp;                 wp += al(b_t);
  void* dev_tab = wp;            wp += al(b_tab);
  double* py = (double*)wp;      wp += al(b_py);
  double* px = (double*)wp;      wp += al(b_px);
  C* sv_ws = (C*)wp;             wp += al(b_sv);
  C* win_ws = (C*)wp;            wp += al(b_win);
  C* gin_ws = (C*)wp;
  CztDims d;
  std::memset(&d, 0, sizeof(d));
  d.nx = g->nx; d.ny = g->ny; d.mx = w->mx; d.my = w->my;
  d.x0 = g->x0; d.dx = g->dx; d.y0 = g->y0; d.dy = g->dy;
  d.xo0 = w->xo0; d.dxo = w->dxo; d.yo0 = w->yo0; d.dyo = w->dyo;
  d.dzx = dz_axis(g->nx, w->mx, g->x0, g->dx, w->xo0, w->dxo);
  d.dzy = dz_axis(g->ny, w->my, g->y0, g->dy, w->yo0, w->dyo);
  // scalar complex64 forward with one segment per axis: row-major intermediate (XL_CZT_RM=0
  // keeps the transposed one)
  const char* rm_env = getenv("XL_CZT_RM");
  const bool rm = mode == FWD && !vec && sizeof(T) == 4 && pl.x.S == 1 && pl.y.S == 1 && ta.Lx >= 256 &&
                  ta.Ly >= 256 && w->mx % 2 == 0 && !(rm_env && rm_env[0] == '0');
  d.in_planes = in_planes;
  d.accumulate = adjoint && (flags & XL_ACCUMULATE) ? 1 : 0;
  const double k = kTwoPi / wavelength;
  for (int32_t b0 = 0; b0 < batch;) {
    const int nb = (int)std::min<int64_t>(chunk, batch - b0);
    AxisRun<C> ax, ay;
    const void* tab0 = nullptr;  // element 0's tables: the base of the shifts
    const void* tab = nullptr;
    for (int e = 0; e < nb; ++e) {  // (nb is 1 with device distances)
      if (e == 0 || z[b0 + e] != z[b0 + e - 1])
        XL_TRY(get_tables<T>(g, w, wavelength, pl, z + b0 + e, flags, dtype, dev_tab, s, &tab));
      if (e == 0) {
        Axis<C> x1, y1;
        axes<T>(tab, ta, &x1, &y1);
        ax = axis_run(x1, pl.x.S, pl.x.seg);
        ay = axis_run(y1, pl.y.S, pl.y.seg);
        ax.per_elem = ay.per_elem = 1;
        tab0 = tab;
      }
      ax.shift[e] = ay.shift[e] = (const C*)tab - (const C*)tab0;
      d.z[e] = zdev ? 0.0 : z[b0 + e];
    }
    d.zdev = zdev ? z + b0 : nullptr;
    // the saved sums of this chunk (caller's buffer, or formed here)
    C* svb = saved ? (C*)saved + (size_t)b0 * sl.elem : sv_ws;
    CztDzArgs<C> dza;
    dza.sv = CztSaved<C>{svb, sl.elem, sl.off_a2x, sl.off_a2y, sl.off_up};
    dza.dzp = nullptr;
    dza.u_in = nullptr;
    dza.on = true;
    auto forward = [&](const void* src, void* dst, bool save) -> xl_status {
      d.adjoint = 0;
      if (save) {
        d.tb_elem = sl.elem;  // the intermediate is the saved T
        XL_TRY(czt_pass<T>(CZT_FWD_X, vec, ta.Lx, src, svb, d, ax, nb, s, &dza));
        XL_TRY(czt_pass<T>(CZT_FWD_Y, vec, ta.Ly, svb, dst, d, ay, nb, s, &dza));
      } else if (rm) {  // the x pass stores row-major, the y pass gathers columns by bulk copies
        d.tb_elem = cT * tplane;
        XL_TRY(czt_fwd_rm<T>(ta.Lx, ta.Ly, src, Tb, dst, d, ax, ay, nb, s));
      } else {
        d.tb_elem = cT * tplane;
        XL_TRY(czt_pass<T>(CZT_FWD_X, vec, ta.Lx, src, Tb, d, ax, nb, s));
        XL_TRY(czt_pass<T>(CZT_FWD_Y, vec, ta.Ly, Tb, dst, d, ay, nb, s));
      }
      return XL_OK;
    };
    if (!adjoint) {
      const char* src = (const char*)in + (size_t)b0 * in_planes * in_plane * cs;
      char* dst = (char*)out + (size_t)b0 * cwin * win_plane * cs;
      XL_TRY(forward(src, dst, mode == FWD_SAVE));
    } else {
      const char* src = (const char*)in + (size_t)b0 * cwin * win_plane * cs;
      char* dst = scratch_gin ? (char*)gin_ws : (char*)out + (size_t)b0 * in_planes * in_plane * cs;
      const C* uin = want_dz ? (const C*)u_in + (size_t)b0 * in_planes * in_plane : nullptr;
      if (recompute) XL_TRY(forward(uin, win_ws, true));
      d.adjoint = 1;
      d.tb_elem = cT * tplane;
      int nby = 0, nbx = 0;
      if (want_dz) {
        dza.dzp = py;
        XL_TRY(czt_pass<T>(CZT_ADJ_Y, vec, ta.Ly, src, Tb, d, ay, nb, s, &dza, &nby));
        dza.dzp = px;
        dza.u_in = uin;
        XL_TRY(czt_pass<T>(CZT_ADJ_X, vec, ta.Lx, Tb, dst, d, ax, nb, s, &dza, &nbx));
        XL_TRY(czt_dz_finalize(py, nby, px, nbx, d.zdev, d, k, (flags & XL_PHASE_INVARIANT) != 0,
                               g_z + b0, nb, s));
      } else {
        XL_TRY(czt_pass<T>(CZT_ADJ_Y, vec, ta.Ly, src, Tb, d, ay, nb, s));
        XL_TRY(czt_pass<T>(CZT_ADJ_X, vec, ta.Lx, Tb, dst, d, ax, nb, s));
      }
      if (in_planes == 3 && !scratch_gin && !d.accumulate) {
        // the unused Ez plane of a 3-component input receives a zero gradient
        XL_CUDA_TRY(cudaMemset2DAsync(dst + 2 * in_plane * cs, 3 * in_plane * cs, 0, in_plane * cs, nb, s));
      }
    }
    b0 += nb;
  }
  return XL_OK;
}

int in_planes_of(int32_t vec) { return vec == 0 ? 1 : (vec == 1 ? 2 : 3); }

xl_status dispatch(Mode mode, const void* in, void* out, const void* u_in, void* saved, double* g_z,
                   int32_t batch, int32_t vec, const xl_grid* g, const xl_window* w,
                   double wavelength, const double* z, int32_t flags, int32_t dtype, void* stream) {
  XL_TRY(check_czt(g, w, wavelength, batch, z, flags, dtype));
  if (vec < 0 || vec > 2) return fail(XL_ERR_ARG, "vectorial must be 0, 1 or 2");
  if (batch == 0) return XL_OK;
  if (!in) return fail(XL_ERR_ARG, "input field is NULL");
  if (mode != ADJ && !out) return fail(XL_ERR_ARG, "output field is NULL");
  if (mode == FWD_SAVE && !saved) return fail(XL_ERR_ARG, "save buffer is NULL");
  if (mode == ADJ && g_z && !u_in) return fail(XL_ERR_ARG, "g_z requested but the forward input is NULL");
  if (mode == ADJ && !out && !g_z) return XL_OK;
  if (in == out || (saved && (saved == in || saved == out)))
    return fail(XL_ERR_ARG, "output and save buffers may not alias the input or each other");
  cudaStream_t s = (cudaStream_t)stream;
  const int in_planes = in_planes_of(vec);
  if (dtype == XL_C128)
    return run<double>(mode, in, out, u_in, saved, g_z, batch, vec != 0, in_planes, g, w, wavelength, z,
                       flags, dtype, s);
  return run<float>(mode, in, out, u_in, saved, g_z, batch, vec != 0, in_planes, g, w, wavelength, z,
                    flags, dtype, s);
}

}  // namespace
}  // namespace xl

using namespace xl;

extern "C" {

xl_status xl_czt_propagate(const void* u_in, void* u_out, int32_t batch, int32_t vectorial,
                           const xl_grid* grid, const xl_window* window, double wavelength,
                           const double* z, int32_t flags, int32_t dtype, void* stream) {
  if (flags & (XL_PHASE_INVARIANT | XL_ACCUMULATE))
    return fail(XL_ERR_ARG, "XL_PHASE_INVARIANT and XL_ACCUMULATE apply to backward calls");
  return dispatch(FWD, u_in, u_out, nullptr, nullptr, nullptr, batch, vectorial, grid, window,
                  wavelength, z, flags, dtype, stream);
}

int64_t xl_czt_save_elems(const xl_grid* grid, const xl_window* window, int32_t vectorial,
                          int32_t dtype) {
  if (!grid || !window || grid->nx < 1 || grid->ny < 1 || window->mx < 1 || window->my < 1 ||
      vectorial < 0 || vectorial > 2 || (dtype != XL_C64 && dtype != XL_C128))
    return -1;
  if (grid->nx + window->mx - 1 > 8192 || grid->ny + window->my - 1 > 8192) return -1;
  const Plans pl = plans(grid, window, dtype, vectorial != 0, true);
  if (pl.x.L == 0 || pl.y.L == 0) return -1;
  return save_layout(grid, window, pl, vectorial ? 3 : 1).elem;
}

xl_status xl_czt_propagate_save(const void* u_in, void* u_out, void* saved, int32_t batch,
                                int32_t vectorial, const xl_grid* grid, const xl_window* window,
                                double wavelength, const double* z, int32_t flags, int32_t dtype,
                                void* stream) {
  if (flags & (XL_PHASE_INVARIANT | XL_ACCUMULATE))
    return fail(XL_ERR_ARG, "XL_PHASE_INVARIANT and XL_ACCUMULATE apply to backward calls");
  return dispatch(FWD_SAVE, u_in, u_out, nullptr, saved, nullptr, batch, vectorial, grid, window,
                  wavelength, z, flags, dtype, stream);
}

xl_status xl_czt_propagate_backward(const void* g_out, const void* u_in, void* g_in, double* g_z,
                                    int32_t batch, int32_t vectorial, const xl_grid* grid,
                                    const xl_window* window, double wavelength, const double* z,
                                    int32_t flags, int32_t dtype, void* stream) {
  return dispatch(ADJ, g_out, g_in, u_in, nullptr, g_z, batch, vectorial, grid, window, wavelength,
                  z, flags, dtype, stream);
}

xl_status xl_czt_propagate_backward_saved(const void* g_out, const void* u_in, const void* saved,
                                          void* g_in, double* g_z, int32_t batch, int32_t vectorial,
                                          const xl_grid* grid, const xl_window* window,
                                          double wavelength, const double* z, int32_t flags,
                                          int32_t dtype, void* stream) {
  if (g_z && !saved) return fail(XL_ERR_ARG, "g_z requested but the saved sums are NULL");
  return dispatch(ADJ, g_out, g_in, u_in, const_cast<void*>(saved), g_z, batch, vectorial, grid,
                  window, wavelength, z, flags, dtype, stream);
}

}  // extern "C"
