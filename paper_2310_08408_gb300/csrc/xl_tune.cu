// Autotuner of the row passes: for a grid (and output window) it times the launch variants of RS
// passes 1 and 3 and of the four CZT window passes on synthetic data on the current device
// (launches over several planes, as batched calls make them), keeps the fastest per (kernel
// family, row length, dtype) for the launchers, and saves / loads the choices as text. Variants
// 0-2 differ in how many rows a block holds (threads per block, register budget, shared memory)
// and compute bit-identical results; variants 3 and 4 of the complex64 CZT passes at lengths
// 512, 1024 and 2048 change the FFT radix plan (where the radix-2/4/8 stage sits), which changes
// the rounding order only (results equal within rounding).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "xl_czt_launch.h"
#include "xl_rs_launch.h"

namespace xl {
namespace {

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  xl_status alloc(size_t bytes, cudaStream_t s) {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return cuda_status(e, "autotune cudaMalloc");
    e = cudaMemsetAsync(p, 0, bytes, s);
    if (e != cudaSuccess) return cuda_status(e, "autotune cudaMemsetAsync");
    return XL_OK;
  }
};

// Times `run` (one launch of the family's kernel) for each variant and records the fastest.
template <typename F>
xl_status tune_one(int family, int L, int dtype, int reps, cudaStream_t s, F run,
                   int nvar = kTuneVariants) {
  cudaEvent_t e0, e1;
  XL_CUDA_TRY(cudaEventCreate(&e0));
  XL_CUDA_TRY(cudaEventCreate(&e1));
  int best = 0;
  double best_us = 1e300;
  xl_status st = XL_OK;
  for (int v = 0; v < nvar && st == XL_OK; ++v) {
    set_tuned_variant(family, L, dtype, v, 0.0);
    st = run();  // warm-up (also sets the kernel's shared-memory limit)
    if (st != XL_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == XL_OK; ++r) st = run();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = cuda_status(cudaGetLastError(), "autotune sync");
    if (st != XL_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double us = 1000.0 * ms / reps;
    if (us < best_us) {
      best_us = us;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  set_tuned_variant(family, L, dtype, st == XL_OK ? best : 0, st == XL_OK ? best_us : 0.0);
  return st;
}

// Planes one timed launch processes: enough that its data exceeds L2 (256 MB of the larger
// per-plane buffer), as in the batched calls, which run the row passes over whole chunks of the
// batch (at most 16 planes).
int tune_planes(size_t plane_bytes) {
  const size_t want = (size_t)256 << 20;
  const size_t n = (want + plane_bytes - 1) / (plane_bytes ? plane_bytes : 1);
  return (int)std::min<size_t>(std::max<size_t>(n, 1), 16);
}

template <typename T>
xl_status tune_grid(const xl_grid* g, const xl_window* w, int dtype, int reps, cudaStream_t s) {
  typedef cplx<T> C;
  const int nx = g->nx, ny = g->ny;
  const size_t cs = sizeof(C);
  const int LX = 2 * nx;
  if (LX >= kTuneMinL && LX <= 8192) {
    const int np = tune_planes((size_t)LX * ny * cs);
    DevBuf in, Tb;
    XL_TRY(in.alloc((size_t)np * nx * ny * cs, s));
    XL_TRY(Tb.alloc((size_t)np * LX * ny * cs, s));
    XL_TRY(tune_one(TUNE_RS_PASS1, LX, dtype, reps, s,
                    [&] { return rs_pass1<T>(in.p, Tb.p, nx, ny, 1, 1, np, s); }));
    XL_TRY(tune_one(TUNE_RS_PASS3, LX, dtype, reps, s,
                    [&] { return rs_pass3<T>(Tb.p, in.p, nx, ny, 1, 1, np, s); }));
  }
  if (w) {
    const int mx = w->mx, my = w->my;
    const CztAxisPlan px = czt_axis_plan(nx, mx, (int)cs, false, false);
    const CztAxisPlan py = czt_axis_plan(ny, my, (int)cs, false, false);
    if (px.L == 0 || py.L == 0) return fail(XL_ERR_UNSUPPORTED, "autotune: no CZT plan fits");
    const int Lx = px.L, Ly = py.L;
    const int64_t tab_n = std::max<int64_t>(std::max(std::max(nx, ny), std::max(mx, my)),
                                            std::max((int64_t)px.S * Lx, (int64_t)py.S * Ly));
    const int np = std::min(tune_planes((size_t)std::max(nx, mx) * ny * cs), kCztRun);
    DevBuf in, Tb, out, tab;
    XL_TRY(in.alloc((size_t)np * nx * ny * cs, s));
    XL_TRY(Tb.alloc((size_t)np * mx * ny * cs, s));
    XL_TRY(out.alloc((size_t)np * mx * my * cs, s));
    XL_TRY(tab.alloc((size_t)tab_n * cs, s));  // zero chirps: the timing does not depend on values
    Axis<C> ax1;
    ax1.pre = ax1.post = ax1.bhat = (const C*)tab.p;
    ax1.b2hat = nullptr;
    const AxisRun<C> ax = axis_run(ax1, px.S, px.seg);
    const AxisRun<C> ay = axis_run(ax1, py.S, py.seg);
    CztDims d;
    std::memset(&d, 0, sizeof(d));
    d.nx = nx; d.ny = ny; d.mx = mx; d.my = my;
    d.dx = g->dx; d.dy = g->dy; d.dxo = w->dxo; d.dyo = w->dyo;
    d.z[0] = 1.0;
    d.in_planes = 1;
    d.tb_elem = (int64_t)mx * ny;
    // rows variants from kTuneMinL up; radix plans at the complex64 lengths that have them
    auto nv = [&](int L) {
      return (sizeof(T) == 4 && czt_plan_lengths(L)) ? kTuneVariantsPlans : (L >= kTuneMinL ? kTuneVariants : 1);
    };
    if (nv(Lx) > 1) {
      XL_TRY(tune_one(TUNE_CZT_FWD_X, Lx, dtype, reps, s,
                      [&] { return czt_pass<T>(CZT_FWD_X, false, Lx, in.p, Tb.p, d, ax, np, s); }, nv(Lx)));
      d.adjoint = 1;
      XL_TRY(tune_one(TUNE_CZT_ADJ_X, Lx, dtype, reps, s,
                      [&] { return czt_pass<T>(CZT_ADJ_X, false, Lx, Tb.p, in.p, d, ax, np, s); }, nv(Lx)));
      d.adjoint = 0;
    }
    if (nv(Ly) > 1) {
      XL_TRY(tune_one(TUNE_CZT_FWD_Y, Ly, dtype, reps, s,
                      [&] { return czt_pass<T>(CZT_FWD_Y, false, Ly, Tb.p, out.p, d, ay, np, s); }, nv(Ly)));
      d.adjoint = 1;
      XL_TRY(tune_one(TUNE_CZT_ADJ_Y, Ly, dtype, reps, s,
                      [&] { return czt_pass<T>(CZT_ADJ_Y, false, Ly, out.p, Tb.p, d, ay, np, s); }, nv(Ly)));
      d.adjoint = 0;
    }
  }
  return XL_OK;
}

int family_index(const char* name) {
  for (int f = 0; f < TUNE_NFAMILY; ++f)
    if (std::strcmp(name, tune_family_name(f)) == 0) return f;
  return -1;
}

}  // namespace
}  // namespace xl

using namespace xl;

extern "C" {

xl_status xl_autotune(const xl_grid* grid, const xl_window* window, int32_t dtype, int32_t reps,
                      void* stream) {
  if (!grid) return fail(XL_ERR_ARG, "grid is NULL");
  if (!is_pow2(grid->nx) || !is_pow2(grid->ny) || grid->nx < 32 || grid->ny < 32 || grid->nx > 4096 ||
      grid->ny > 4096)
    return fail(XL_ERR_UNSUPPORTED, "nx, ny must be powers of two in [32, 4096]");
  if (window && (window->mx < 1 || window->my < 1)) return fail(XL_ERR_ARG, "window sizes must be positive");
  if (dtype != XL_C64 && dtype != XL_C128) return fail(XL_ERR_ARG, "bad dtype");
  if (reps < 1 || reps > 1000) return fail(XL_ERR_ARG, "reps must be in [1, 1000]");
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == XL_C128) return tune_grid<double>(grid, window, dtype, reps, s);
  return tune_grid<float>(grid, window, dtype, reps, s);
}

int32_t xl_tune_get(int32_t family, int32_t L, int32_t dtype) {
  if (family < 0 || family >= TUNE_NFAMILY) return -1;
  return tuned_variant(family, L, dtype);
}

xl_status xl_tune_set(int32_t family, int32_t L, int32_t dtype, int32_t variant) {
  if (family < 0 || family >= TUNE_NFAMILY) return fail(XL_ERR_ARG, "unknown tuning family");
  if (!is_pow2(L) || L < 64 || L > 8192) return fail(XL_ERR_ARG, "L must be a power of two in [64, 8192]");
  if (dtype != XL_C64 && dtype != XL_C128) return fail(XL_ERR_ARG, "bad dtype");
  const int nmax = family >= TUNE_CZT_FWD_X ? kTuneVariantsPlans : kTuneVariants;
  if (variant < 0 || variant >= nmax)
    return fail(XL_ERR_ARG, nmax == kTuneVariants ? "variant must be 0, 1 or 2" : "variant must be 0 to 4");
  set_tuned_variant(family, L, dtype, variant, 0.0);
  return XL_OK;
}

xl_status xl_tune_clear(void) {
  tune_clear();
  return XL_OK;
}

xl_status xl_tune_save(const char* path) {
  if (!path) return fail(XL_ERR_ARG, "path is NULL");
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(XL_ERR_ARG, std::string("cannot write ") + path);
  const std::string text = tune_table_text();
  std::fputs("# xl autotune v1: family L dtype variant microseconds\n", f);
  std::fputs(text.c_str(), f);
  const bool ok = std::fclose(f) == 0;
  return ok ? XL_OK : fail(XL_ERR_ARG, std::string("write failed: ") + path);
}

xl_status xl_tune_load(const char* path) {
  if (!path) return fail(XL_ERR_ARG, "path is NULL");
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(XL_ERR_ARG, std::string("cannot read ") + path);
  char line[256];
  int lineno = 0;
  xl_status st = XL_OK;
  std::vector<std::tuple<int, int, int, int, double>> rows;
  while (std::fgets(line, sizeof(line), f)) {
    ++lineno;
    if (line[0] == '#' || line[0] == '\n') continue;
    char fam[64], dt[16];
    int L = 0, v = 0;
    double us = 0.0;
    if (std::sscanf(line, "%63s %d %15s %d %lf", fam, &L, dt, &v, &us) != 5) {
      st = fail(XL_ERR_ARG, "autotune file: bad line " + std::to_string(lineno));
      break;
    }
    const int fi = family_index(fam);
    const int dtype = std::strcmp(dt, "c64") == 0 ? XL_C64 : (std::strcmp(dt, "c128") == 0 ? XL_C128 : -1);
    const int nmax = fi >= TUNE_CZT_FWD_X ? kTuneVariantsPlans : kTuneVariants;
    if (fi < 0 || dtype < 0 || v < 0 || v >= nmax || !is_pow2(L) || L < 64 || L > 8192) {
      st = fail(XL_ERR_ARG, "autotune file: bad entry on line " + std::to_string(lineno));
      break;
    }
    rows.emplace_back(fi, L, dtype, v, us);
  }
  std::fclose(f);
  if (st != XL_OK) return st;  // nothing applied from a malformed file
  for (const auto& r : rows)
    set_tuned_variant(std::get<0>(r), std::get<1>(r), std::get<2>(r), std::get<3>(r), std::get<4>(r));
  return XL_OK;
}

}  // extern "C"
