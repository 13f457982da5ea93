// C ABI of scalar and vectorial RS propagation and their adjoints (host orchestration of the
// kernels in xl_rs_kernels.cuh). Methods, "Features and performance": FFT-based numerical
// integration of the Rayleigh-Sommerfeld integral, scalar (RS) and vectorial (VRS).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>

#include "xl_rs_launch.h"

namespace xl {

namespace {

struct Spectra {
  unsigned kinds = 0;
  int slot[NKIND];
  int count = 0;
  explicit Spectra(unsigned k) : kinds(k) {
    for (int i = 0; i < NKIND; ++i) slot[i] = (k & (1u << i)) ? count++ : -1;
  }
};

xl_status check_grid(const xl_grid* g, double wavelength) {
  if (!g) return fail(XL_ERR_ARG, "grid is NULL");
  if (!is_pow2(g->nx) || !is_pow2(g->ny) || g->nx < 32 || g->ny < 32 || g->nx > 4096 ||
      g->ny > 4096)
    return fail(XL_ERR_UNSUPPORTED, "nx, ny must be powers of two in [32, 4096]");
  if (!(g->dx > 0) || !(g->dy > 0) || !std::isfinite(g->dx) || !std::isfinite(g->dy))
    return fail(XL_ERR_ARG, "pixel pitch must be positive and finite");
  if (!(wavelength > 0) || !std::isfinite(wavelength))
    return fail(XL_ERR_ARG, "wavelength must be positive and finite");
  return XL_OK;
}

xl_status check_common(int32_t batch, const double* z, int32_t flags, int32_t dtype) {
  if (batch < 0) return fail(XL_ERR_ARG, "batch < 0");
  if (dtype != XL_C64 && dtype != XL_C128) return fail(XL_ERR_ARG, "dtype must be XL_C64 or XL_C128");
  if (flags & ~(XL_Z_DEVICE | XL_PHASE_INVARIANT)) return fail(XL_ERR_ARG, "unknown flag bits");
  if (batch > 0 && !z) return fail(XL_ERR_ARG, "z is NULL");
  if (batch > 0 && !(flags & XL_Z_DEVICE))
    for (int32_t b = 0; b < batch; ++b)
      if (!(z[b] > 0) || !std::isfinite(z[b]))
        return fail(XL_ERR_ARG, "z must be positive and finite");
  return XL_OK;
}

GenArgs gen_args(const xl_grid* g, double wavelength, const Spectra& sp) {
  GenArgs a;
  a.nx = g->nx;
  a.ny = g->ny;
  a.dx = g->dx;
  a.dy = g->dy;
  a.k = kTwoPi / wavelength;
  a.zval = 0;
  a.zdev = nullptr;
  a.kinds = sp.kinds;
  a.s_plane = (int64_t)(g->nx + 1) * g->ny;
  a.hq_kind = (int64_t)(g->nx + 1) * (g->ny + 1);
  a.scale = 1.0 / (4.0 * (double)g->nx * (double)g->ny);
  for (int i = 0; i < NKIND; ++i) a.slot[i] = sp.slot[i];
  a.dz_rest = 0;
  a.s_elem = a.h_elem = 0;
  return a;
}

template <typename T>
xl_status generate(void* S, void* Hq, const GenArgs& a, int nb, cudaStream_t s) {
  return rs_generate<T>(S, Hq, a, nb, s);
}

// Spectra for one distance: cached (host z), or generated into `dev_hq` (device z) for the nb
// consecutive distances z[0..nb-1], element e's spectra at e * count * (nx+1)(ny+1).
xl_status get_spectra(const xl_grid* g, double wavelength, const Spectra& sp, int32_t dtype,
                      const double* z, int32_t flags, void* dev_s, void* dev_hq, cudaStream_t s,
                      const void** out, int nb = 1) {
  GenArgs a = gen_args(g, wavelength, sp);
  a.dz_rest = (flags & XL_PHASE_INVARIANT) ? 1 : 0;
  const size_t cs = dtype_csize(dtype);
  const size_t hq_bytes = (size_t)sp.count * a.hq_kind * cs;
  auto run = [&](void* S, void* Hq, int n) -> xl_status {
    return dtype == XL_C128 ? generate<double>(S, Hq, a, n, s) : generate<float>(S, Hq, a, n, s);
  };
  if (flags & XL_Z_DEVICE) {
    a.zdev = z;
    a.s_elem = (int64_t)sp.count * a.s_plane;
    a.h_elem = (int64_t)sp.count * a.hq_kind;
    XL_TRY(run(dev_s, dev_hq, nb));
    *out = dev_hq;
    return XL_OK;
  }
  a.zval = *z;
  std::string key = "rs";
  key_put(key, sp.kinds);
  key_put(key, a.dz_rest);
  key_put(key, g->nx);
  key_put(key, g->ny);
  key_put(key, g->dx);
  key_put(key, g->dy);
  key_put(key, wavelength);
  key_put(key, *z);
  key_put(key, dtype);
  void* p = nullptr;
  XL_TRY(cached_table(key, hq_bytes, s, [&](void* Hq) -> xl_status {
    void* S = nullptr;
    XL_TRY(workspace(s, (size_t)sp.count * a.s_plane * cs, &S, 1));
    return run(S, Hq, 1);
  }, &p));
  *out = p;
  return XL_OK;
}

P2Args p2_args(const xl_grid* g, const Spectra& sp, int cT, int cU) {
  P2Args a;
  a.nx = g->nx;
  a.ny = g->ny;
  a.t_plane = (int64_t)2 * g->nx * g->ny;
  a.hq_kind = (int64_t)(g->nx + 1) * (g->ny + 1);
  a.cT = cT;
  a.cU = cU;
  a.want_field = 1;
  a.want_dz = 0;
  a.conj = 0;
  for (int i = 0; i < NKIND; ++i) a.slot[i] = sp.slot[i];
  a.spec_out = nullptr;
  a.spec_in = nullptr;
  a.cS = 0;
  a.per_elem = 0;
  for (int i = 0; i < kP2Run; ++i) a.hshift[i] = 0;
  a.status = nullptr;
  return a;
}

template <typename T>
xl_status launch_reduce(const double* part, int n, double* out, int nb, cudaStream_t s) {
  LaunchScope ls("reduce_rows", s);
  k_reduce_rows<<<nb, 256, 0, s>>>(part, n, out);
  XL_CUDA_TRY(cudaGetLastError());
  return XL_OK;
}

// How many batch elements the row passes (1 and 3) process per launch: as many as fit a byte
// budget for their T planes (XL_RS_CHUNK_MB, default 2048 MB); pass 2 takes the chunk in groups
// of up to kP2Run elements, each reading the spectra of its own distance. Measured on 16 fields of
// 2048^2 (T planes of 67 MB each): one chunk of all 16 runs the row passes 25% faster than chunks
// of one field kept resident in L2, because the row passes then fill every SM for many waves;
// pass 2 is unaffected by reading T from DRAM.
int chunk_size(int64_t t_bytes_per_elem, int32_t remaining) {
  int64_t budget = (int64_t)2048 << 20;
  if (const char* e = getenv("XL_RS_CHUNK_MB")) {
    const long long mb = atoll(e);
    if (mb > 0) budget = (int64_t)mb << 20;
  }
  int64_t c = budget / (t_bytes_per_elem > 0 ? t_bytes_per_elem : 1);
  if (c < 1) c = 1;
  return (int)(c < remaining ? c : remaining);
}

enum Op { OP_RS_FWD, OP_RS_BWD, OP_VRS_FWD, OP_VRS_BWD };

// save_out (forward): receives the 2D spectra of the zero-padded input planes (the column
// transforms pass 2 computes anyway), [batch][cin][2nx][2ny];
// save_in (adjoint): those spectra in place of u_in for the distance gradient.
template <typename T>
xl_status run_op(Op op, const void* in, const void* u_in, void* out, double* g_z, int32_t batch,
                 const xl_grid* g, double wavelength, const double* z, int32_t flags, int32_t dtype,
                 cudaStream_t s, void* save_out = nullptr, const void* save_in = nullptr) {
  const bool vec = (op == OP_VRS_FWD || op == OP_VRS_BWD);
  const bool bwd = (op == OP_RS_BWD || op == OP_VRS_BWD);
  const bool want_field = !bwd || out != nullptr;
  const bool want_dz = bwd && g_z != nullptr;
  unsigned kinds = 0;
  if (!vec) {
    if (want_field) kinds |= 1u << KH;
    if (want_dz) kinds |= 1u << KDH;
  } else {
    if (want_field || !bwd) kinds |= (1u << KH) | (1u << KHX) | (1u << KHY);
    if (want_dz) kinds |= (1u << KH) | (1u << KHX) | (1u << KHY) | (1u << KDH) | (1u << KDHX) |
                          (1u << KDHY);
  }
  if (!kinds) return XL_OK;  // nothing requested
  Spectra sp(kinds);
  const int nx = g->nx, ny = g->ny;
  const size_t cs = sizeof(cplx<T>);
  const int64_t t_plane = (int64_t)2 * nx * ny;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t spec_plane = (int64_t)4 * nx * ny;  // one 2nx x 2ny spectrum
  // planes per element: input to pass 1, T planes, U planes (dz), output of pass 3
  const int cin = op == OP_RS_FWD || op == OP_RS_BWD ? 1 : (op == OP_VRS_FWD ? 2 : 3);
  const int cT = vec ? 3 : 1;
  const int cU = want_dz ? (vec ? 2 : 1) : 0;
  const int cout = op == OP_VRS_FWD ? 3 : (op == OP_VRS_BWD ? 2 : 1);
  const int p2blocks = rs_pass2_blocks<T>(nx, ny);
  const bool zdev = (flags & XL_Z_DEVICE) != 0;
  const int cUw = save_in ? 0 : cU;  // U planes computed into the workspace
  const size_t hq_bytes1 = (size_t)sp.count * (nx + 1) * (ny + 1) * cs;
  const size_t s_bytes1 = (size_t)sp.count * (nx + 1) * ny * cs;
  // device distances: every element of a chunk gets its spectra generated into the workspace
  // Row-major intermediate (complex64 scalar forward and saved-spectrum adjoint, rows of 256 and
  // more): pass 1 stores each row's transform as it stands, pass 2 gathers its columns with bulk
  // tensor copies (XL_RS_RM=0 keeps the transposing pass 1).
  int mode = op == OP_RS_FWD ? P2_RS : op == OP_VRS_FWD ? P2_VRS : op == OP_RS_BWD ? P2_RS_BWD
                                                                                  : P2_VRS_BWD;
  if (want_dz && save_in) mode = op == OP_RS_BWD ? P2_RS_BWD_S : P2_VRS_BWD_S;
  const char* rm_env = getenv("XL_RS_RM");
  const bool rm = sizeof(T) == 4 && (mode == P2_RS || mode == P2_RS_BWD_S) && 2 * nx >= 256 &&
                  !(rm_env && rm_env[0] == '0');
  const int64_t elem_ws = (int64_t)(cT * (rm ? 2 : 1) + cUw) * t_plane * cs +
                          (zdev ? (int64_t)(s_bytes1 + hq_bytes1) : 0);
  const int chunk_max = zdev ? std::min(chunk_size(elem_ws, batch), kP2Run) : chunk_size(elem_ws, batch);
  // pass-2 group: up to kP2Run elements whose spectra together stay within half of the table
  // cache, so that fetching one never evicts another of the same launch (device distances: the
  // chunk, whose spectra live in the workspace)
  const int group_max = zdev ? chunk_max
                             : (int)std::max<int64_t>(1, std::min<int64_t>(kP2Run,
                                   (int64_t)(table_cache_cap() / 2 / hq_bytes1)));
  // workspace: T (chunk * cT planes) | U (chunk * cU planes) | dz partials | [S | Hq] (device z)
  const size_t t_bytes = (size_t)chunk_max * cT * t_plane * cs;
  const size_t u_bytes = (size_t)chunk_max * cUw * t_plane * cs;
  const size_t dz_bytes = want_dz ? (size_t)chunk_max * p2blocks * sizeof(double) : 0;
  const size_t s_bytes = zdev ? (size_t)chunk_max * s_bytes1 : 0;
  const size_t hq_bytes = zdev ? (size_t)chunk_max * hq_bytes1 : 0;
  auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
  void* ws = nullptr;
  const size_t r_bytes = rm ? t_bytes : 0;
  XL_TRY(workspace(s, al(t_bytes) + al(u_bytes) + al(dz_bytes) + al(s_bytes) + al(hq_bytes) + al(r_bytes),
                   &ws));
  char* w = (char*)ws;
  void* Tb = w;
  void* Ub = w + al(t_bytes);
  double* dzp = (double*)(w + al(t_bytes) + al(u_bytes));
  void* dev_s = w + al(t_bytes) + al(u_bytes) + al(dz_bytes);
  void* dev_hq = (char*)dev_s + al(s_bytes);
  void* Tr = rm ? (char*)dev_hq + al(hq_bytes) : nullptr;

  const char* src = (const char*)in;
  const char* usrc = (const char*)u_in;
  char* dst = (char*)out;
  for (int32_t b0 = 0; b0 < batch;) {
    // a chunk of elements: row passes over all of it, pass 2 per run of equal distances
    const int nc = chunk_max < batch - b0 ? chunk_max : batch - b0;
    if (rm)
      XL_TRY(rs_pass1_rm<T>(src + (size_t)b0 * cin * plane * cs, Tr, nx, ny, cin, cT, nc * cin, s));
    else
      XL_TRY(rs_pass1<T>(src + (size_t)b0 * cin * plane * cs, Tb, nx, ny, cin, cT, nc * cin, s));
    if (want_dz && !save_in)
      XL_TRY(rs_pass1<T>(usrc + (size_t)b0 * cU * plane * cs, Ub, nx, ny, cU, cU, nc * cU, s));
    // pass 2 over groups of up to kP2Run elements, each element with the spectra of its own
    // distance (device distances: the whole chunk, its spectra generated by one launch pair)
    for (int32_t r0 = b0; r0 < b0 + nc;) {
      const int nb = (int)std::min<int64_t>(group_max, b0 + nc - r0);
      const int64_t e0 = r0 - b0;  // first element of the group within the chunk
      P2Args a = p2_args(g, sp, cT, cU);
      const void* Hq0 = nullptr;
      const void* Hq = nullptr;
      if (zdev) {  // one generation for the group, element e's spectra at e * count * quadrant
        XL_TRY(get_spectra(g, wavelength, sp, dtype, z + r0, flags, dev_s, dev_hq, s, &Hq0, nb));
        for (int e = 0; e < nb; ++e) a.hshift[e] = (int64_t)e * sp.count * (nx + 1) * (ny + 1);
      } else {
        for (int e = 0; e < nb; ++e) {
          if (e == 0 || z[r0 + e] != z[r0 + e - 1])
            XL_TRY(get_spectra(g, wavelength, sp, dtype, z + r0 + e, flags, dev_s, dev_hq, s, &Hq));
          if (e == 0) Hq0 = Hq;
          a.hshift[e] = (const cplx<T>*)Hq - (const cplx<T>*)Hq0;
        }
      }
      a.per_elem = nb > 1 ? 1 : 0;
      if (save_out) {  // pass 2 also stores the column spectra of the inputs
        a.spec_out = (char*)save_out + (size_t)r0 * cin * spec_plane * cs;
        a.cS = cin;
      }
      if (want_dz && save_in) {
        a.spec_in = (const char*)save_in + (size_t)r0 * cU * spec_plane * cs;
        a.cS = cU;
      }
      a.want_field = want_field;
      a.want_dz = want_dz;
      XL_TRY(rs_pass2<T>(mode, (char*)Tb + e0 * cT * t_plane * cs,
                         (const char*)Ub + e0 * cUw * t_plane * cs, Hq0, dzp + e0 * p2blocks, a, nb,
                         s, rm ? (const char*)Tr + e0 * cT * t_plane * cs : nullptr));
      // the distance partials are summed by pass 3 when it runs, else by their own launch
      if (want_dz && !want_field)
        XL_TRY(launch_reduce<T>(dzp + e0 * p2blocks, p2blocks, g_z + r0, nb, s));
      r0 += nb;
    }
    if (want_field)
      XL_TRY(rs_pass3<T>(Tb, dst + (size_t)b0 * cout * plane * cs, nx, ny, cout, cT, nc * cout, s,
                         want_dz ? DzReduce{dzp, p2blocks, g_z + b0} : DzReduce{nullptr, 0, nullptr}));
    b0 += nc;
  }
  return XL_OK;
}

// u_in (adjoint) is the forward input, or with `saved` set the forward's saved row transforms.
xl_status dispatch(Op op, const void* in, const void* u_in, void* out, double* g_z, int32_t batch,
                   const xl_grid* g, double wavelength, const double* z, int32_t flags,
                   int32_t dtype, void* stream, void* save_out = nullptr, bool saved = false) {
  XL_TRY(check_grid(g, wavelength));
  XL_TRY(check_common(batch, z, flags, dtype));
  if (batch == 0) return XL_OK;
  const bool bwd = (op == OP_RS_BWD || op == OP_VRS_BWD);
  if (!in) return fail(XL_ERR_ARG, "input field is NULL");
  if (!bwd && !out) return fail(XL_ERR_ARG, "output field is NULL");
  if (bwd && g_z && !u_in)
    return fail(XL_ERR_ARG, saved ? "g_z requested but the saved row transforms are NULL"
                                   : "g_z requested but the forward input is NULL");
  if (!bwd && in == out) return fail(XL_ERR_ARG, "output may not alias the input");
  if (!bwd && (flags & XL_PHASE_INVARIANT)) return fail(XL_ERR_ARG, "XL_PHASE_INVARIANT applies to backward passes");
  if (save_out && (save_out == in || save_out == out))
    return fail(XL_ERR_ARG, "the save buffer may not alias the fields");
  cudaStream_t s = (cudaStream_t)stream;
  const void* uf = saved ? nullptr : u_in;
  const void* us = saved ? u_in : nullptr;
  if (dtype == XL_C128)
    return run_op<double>(op, in, uf, out, g_z, batch, g, wavelength, z, flags, dtype, s, save_out, us);
  return run_op<float>(op, in, uf, out, g_z, batch, g, wavelength, z, flags, dtype, s, save_out, us);
}

}  // namespace
}  // namespace xl

using namespace xl;

extern "C" {

xl_status xl_rs_propagate(const void* u_in, void* u_out, int32_t batch, const xl_grid* grid,
                          double wavelength, const double* z, int32_t flags, int32_t dtype,
                          void* stream) {
  return dispatch(OP_RS_FWD, u_in, nullptr, u_out, nullptr, batch, grid, wavelength, z, flags,
                  dtype, stream);
}

xl_status xl_rs_propagate_backward(const void* g_out, const void* u_in, void* g_in, double* g_z,
                                   int32_t batch, const xl_grid* grid, double wavelength,
                                   const double* z, int32_t flags, int32_t dtype, void* stream) {
  return dispatch(OP_RS_BWD, g_out, u_in, g_in, g_z, batch, grid, wavelength, z, flags, dtype,
                  stream);
}

xl_status xl_vrs_propagate(const void* exy_in, void* exyz_out, int32_t batch, const xl_grid* grid,
                           double wavelength, const double* z, int32_t flags, int32_t dtype,
                           void* stream) {
  return dispatch(OP_VRS_FWD, exy_in, nullptr, exyz_out, nullptr, batch, grid, wavelength, z,
                  flags, dtype, stream);
}

xl_status xl_vrs_propagate_backward(const void* g_exyz, const void* exy_in, void* g_exy,
                                    double* g_z, int32_t batch, const xl_grid* grid,
                                    double wavelength, const double* z, int32_t flags,
                                    int32_t dtype, void* stream) {
  return dispatch(OP_VRS_BWD, g_exyz, exy_in, g_exy, g_z, batch, grid, wavelength, z, flags, dtype,
                  stream);
}

xl_status xl_rs_propagate_save(const void* u_in, void* u_out, void* saved, int32_t batch,
                               const xl_grid* grid, double wavelength, const double* z,
                               int32_t flags, int32_t dtype, void* stream) {
  if (!saved) return fail(XL_ERR_ARG, "saved is NULL");
  return dispatch(OP_RS_FWD, u_in, nullptr, u_out, nullptr, batch, grid, wavelength, z, flags,
                  dtype, stream, saved);
}

xl_status xl_rs_propagate_backward_saved(const void* g_out, const void* saved, void* g_in,
                                         double* g_z, int32_t batch, const xl_grid* grid,
                                         double wavelength, const double* z, int32_t flags,
                                         int32_t dtype, void* stream) {
  return dispatch(OP_RS_BWD, g_out, saved, g_in, g_z, batch, grid, wavelength, z, flags, dtype,
                  stream, nullptr, true);
}

xl_status xl_vrs_propagate_save(const void* exy_in, void* exyz_out, void* saved, int32_t batch,
                                const xl_grid* grid, double wavelength, const double* z,
                                int32_t flags, int32_t dtype, void* stream) {
  if (!saved) return fail(XL_ERR_ARG, "saved is NULL");
  return dispatch(OP_VRS_FWD, exy_in, nullptr, exyz_out, nullptr, batch, grid, wavelength, z,
                  flags, dtype, stream, saved);
}

xl_status xl_vrs_propagate_backward_saved(const void* g_exyz, const void* saved, void* g_exy,
                                          double* g_z, int32_t batch, const xl_grid* grid,
                                          double wavelength, const double* z, int32_t flags,
                                          int32_t dtype, void* stream) {
  return dispatch(OP_VRS_BWD, g_exyz, saved, g_exy, g_z, batch, grid, wavelength, z, flags,
                  dtype, stream, nullptr, true);
}

}  // extern "C"
