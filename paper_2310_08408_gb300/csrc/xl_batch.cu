// Batched optimisation of many optical-table setups (the paper's batching of independent setups
// or samples with vmap, Methods "Data-driven rediscovery" and "Features and performance";
// the tables of Results "Towards large-scale discovery").
//
// Each setup is the differentiable table
//   x-polarised Gaussian -> SLM1 (phi1) -> RS z1 -> SLM2 (phi2) -> to-vector -> half-wave plate
//   (theta) -> VRS z2 -> lens f -> VCZT f onto the camera -> second-moment spot size (total I)
// with its own masks, theta, z1, z2 and grid size N (pitch = extent / N, so every setup sees the
// same physical window). Setups are grouped by N; every stage of a group runs as one batched
// library call with device-resident parameters (distances and angles are read by the kernels at
// run time). One step = forward, backward (adjoints of every stage) and Adam for all setups. The
// whole step can be captured once into a CUDA graph and replayed: after one eager warm-up step
// every workspace has its final size, so the captured calls allocate nothing.
//
// Memory per setup: the fields at the optical planes the adjoints read (source, after SLM1,
// after RS, after the wave plate, after VRS, the camera), two 3-component gradient buffers used in
// turn by the backward stages (the field after the lens shares one of them: nothing reads it
// after the forward), masks, their gradients and Adam moments. cfg.checkpoint selects what the
// RS and VRS adjoints read for their distance gradients: 0 keeps the 2D spectra of their zero-
// padded inputs (4 and 8 field planes a setup; no input transform in the adjoints), 1 keeps only
// the plane fields and the adjoints transform their inputs again (about half the memory, one
// more column transform in each adjoint's pass 2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <vector>

#include "xl_runtime.h"

namespace xl {

struct Group {
  int n = 0, count = 0;
  double pitch = 0;
  std::vector<int> setups;  // indices into the batch
  xl_grid grid{};
  // device buffers (complex T unless noted)
  void *src = nullptr, *a0 = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *a4 = nullptr,
       *a5 = nullptr;
  void *g5 = nullptr;                 // camera gradient
  void *gx = nullptr, *gy = nullptr;  // 3-component gradient buffers (a4 lives in gx)
  void *s1 = nullptr, *s2 = nullptr;  // spectra the RS / VRS forwards keep (checkpoint 0)
  void *phi1 = nullptr, *phi2 = nullptr, *gphi1 = nullptr, *gphi2 = nullptr;  // real T [count][n][n]
  void *m1 = nullptr, *v1 = nullptr, *m2 = nullptr, *v2 = nullptr;            // Adam moments (real T)
  double *p1 = nullptr, *p2 = nullptr, *pl = nullptr;  // element params [count][n_el][4]
  double *z1 = nullptr, *z2 = nullptr;                 // [count]
  std::vector<double> zf;                              // host: VCZT distance f per setup
  double *gp2 = nullptr, *gz1 = nullptr, *gz2 = nullptr;
  double *sm = nullptr, *sv = nullptr;                 // scalar Adam moments [count][3]
  double *loss = nullptr;                              // [count]
};

}  // namespace xl

struct xl_batch {
  xl_table_config cfg{};
  int n_setups = 0;
  int64_t bytes = 0;        // device memory the batch holds
  int32_t* step = nullptr;  // device step counter
  std::vector<xl::Group> groups;
  std::vector<void*> allocs;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t own = nullptr;      // non-blocking stream of the graph path (capture needs one)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool warmed = false;
};

namespace xl {

namespace {

xl_status dalloc(xl_batch* b, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return cuda_status(e, "batch cudaMalloc");
  b->allocs.push_back(*p);
  b->bytes += (int64_t)bytes;
  return XL_OK;
}

// SplitMix64 (Steele, Lea & Flood 2014): state = seed + (i + 1) * 0x9E3779B97F4A7C15; the double
// (z >> 11) * 2^-53 is uniform in [0, 1).
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// Initial state of a group: Gaussian source (peak 1), masks uniform in [0, 2 pi) drawn with
// SplitMix64 from seed_mask + setup index (mask 1) and + 0x10000 (mask 2), one draw per pixel
// in row-major order.
template <typename T>
__global__ void k_batch_init(cplx<T>* src, T* phi1, T* phi2, int n, double x0, double pitch,
                             double w0, const int* setup_ids, uint64_t seed, int count) {
  const int64_t plane = (int64_t)n * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < plane * count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(i / plane);
    const int64_t j = i % plane;
    const double x = x0 + (j % n) * pitch, y = x0 + (j / n) * pitch;
    src[i] = mk((T)exp(-(x * x + y * y) / (w0 * w0)), (T)0);
    const uint64_t s = seed + (uint64_t)setup_ids[g];
    phi1[i] = (T)(kTwoPi * splitmix_uniform(s, (uint64_t)j));
    phi2[i] = (T)(kTwoPi * splitmix_uniform(s + 0x10000ull, (uint64_t)j));
  }
}

// Adam on the per-setup scalars (theta in the wave-plate slot of p2, z1, z2), moments [count][3].
__global__ void k_batch_scalar_adam(double* p2, double* z1, double* z2, const double* gp2,
                                    const double* gz1, const double* gz2, double* m, double* v,
                                    const int32_t* step, int count, double lr_theta, double lr_z) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  const double t = (double)*step;
  const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  double* pp[3] = {p2 + (int64_t)g * 12 + 2 * 4 + 3, z1 + g, z2 + g};
  const double gg[3] = {gp2[(int64_t)g * 12 + 2 * 4 + 3], gz1[g], gz2[g]};
  const double lr[3] = {lr_theta, lr_z, lr_z};
  for (int k = 0; k < 3; ++k) {
    double& mm = m[g * 3 + k];
    double& vv = v[g * 3 + k];
    mm = b1 * mm + (1 - b1) * gg[k];
    vv = b2 * vv + (1 - b2) * gg[k] * gg[k];
    *pp[k] -= lr[k] * (mm / c1) / (sqrt(vv / c2) + eps);
  }
}

struct Buf {
  void** p;
  size_t bytes;
};

// The device buffers of a group (cnt setups of side n), in allocation order. spectra: keep the
// RS / VRS input spectra (checkpoint 0).
template <typename T>
std::vector<Buf> group_buffers(const xl_table_config& c, Group& G, bool spectra) {
  const size_t cs = sizeof(cplx<T>), rs = sizeof(T);
  const size_t plane = (size_t)G.n * G.n, cnt = (size_t)G.count;
  const size_t cam = (size_t)c.cam_m * c.cam_m;
  return {
      {&G.src, cnt * plane * cs},     {&G.a0, cnt * plane * cs},     {&G.a1, cnt * plane * cs},
      {&G.a2, cnt * 2 * plane * cs},  {&G.a3, cnt * 3 * plane * cs},
      {&G.a5, cnt * 3 * cam * cs},    {&G.g5, cnt * 3 * cam * cs},
      {&G.gx, cnt * 3 * plane * cs},  {&G.gy, cnt * 3 * plane * cs},
      {&G.s1, spectra ? cnt * 4 * plane * cs : 0}, {&G.s2, spectra ? cnt * 8 * plane * cs : 0},
      {&G.phi1, cnt * plane * rs},    {&G.phi2, cnt * plane * rs},
      {&G.gphi1, cnt * plane * rs},   {&G.gphi2, cnt * plane * rs},  {&G.m1, cnt * plane * rs},
      {&G.v1, cnt * plane * rs},      {&G.m2, cnt * plane * rs},     {&G.v2, cnt * plane * rs},
      {(void**)&G.p1, cnt * 4 * 8},   {(void**)&G.p2, cnt * 12 * 8}, {(void**)&G.pl, cnt * 4 * 8},
      {(void**)&G.z1, cnt * 8},       {(void**)&G.z2, cnt * 8},
      {(void**)&G.gp2, cnt * 12 * 8}, {(void**)&G.gz1, cnt * 8},     {(void**)&G.gz2, cnt * 8},
      {(void**)&G.sm, cnt * 3 * 8},   {(void**)&G.sv, cnt * 3 * 8},  {(void**)&G.loss, cnt * 8},
  };
}

// Bytes xl_batch_create allocates for the setups' grid sizes in checkpoint mode `mode` (0 or 1):
// every group's buffers, its setup-index table and the step counter.
int64_t plan_bytes(const xl_table_config& c, int n_setups, const int32_t* grid_n, int mode) {
  std::map<int, int> counts;
  for (int i = 0; i < n_setups; ++i) counts[grid_n[i]]++;
  int64_t total = sizeof(int32_t);
  for (auto& kv : counts) {
    Group G;
    G.n = kv.first;
    G.count = kv.second;
    const auto bufs = c.dtype == XL_C128 ? group_buffers<double>(c, G, mode == 0)
                                         : group_buffers<float>(c, G, mode == 0);
    for (const Buf& bf : bufs) total += (int64_t)bf.bytes;
    total += (int64_t)G.count * sizeof(int);
  }
  return total;
}

// cfg.checkpoint as the batch runs it: XL_CHECKPOINT_AUTO keeps the spectra (0) when they fit
// in cfg.memory_budget (or when there is no budget), else the plane fields only (1).
int resolve_checkpoint(const xl_table_config& c, int n_setups, const int32_t* grid_n) {
  if (c.checkpoint != XL_CHECKPOINT_AUTO) return c.checkpoint;
  if (c.memory_budget <= 0 || plan_bytes(c, n_setups, grid_n, 0) <= c.memory_budget) return 0;
  return 1;
}

template <typename T>
xl_status group_alloc(xl_batch* b, Group& G, const double* init, uint64_t seed, cudaStream_t s) {
  const size_t rs = sizeof(T);
  const int64_t plane = (int64_t)G.n * G.n, cnt = G.count;
  const auto bufs = group_buffers<T>(b->cfg, G, b->cfg.checkpoint == 0);
  for (auto& bf : bufs)
    if (bf.bytes) XL_TRY(dalloc(b, bf.p, bf.bytes));
  G.a4 = G.gx;  // the field after the lens: read by the VCZT forward only
  for (void* p : {G.m1, G.v1, G.m2, G.v2}) XL_CUDA_TRY(cudaMemsetAsync(p, 0, cnt * plane * rs, s));
  XL_CUDA_TRY(cudaMemsetAsync(G.sm, 0, cnt * 3 * 8, s));
  XL_CUDA_TRY(cudaMemsetAsync(G.sv, 0, cnt * 3 * 8, s));
  // element parameters: p1 (SLM1) zero; p2 = SLM2, to-vector, wave plate {0, 0, pi, theta};
  // pl = lens {f}; distances from `init`
  std::vector<double> p1(cnt * 4, 0.0), p2(cnt * 12, 0.0), pl(cnt * 4, 0.0), z1(cnt), z2(cnt);
  G.zf.assign(cnt, b->cfg.f);
  for (int g = 0; g < cnt; ++g) {
    const int id = G.setups[g];
    p2[g * 12 + 8 + 2] = kPi;
    p2[g * 12 + 8 + 3] = init[id * 3 + 0];
    z1[g] = init[id * 3 + 1];
    z2[g] = init[id * 3 + 2];
    pl[g * 4 + 0] = b->cfg.f;
  }
  XL_CUDA_TRY(cudaMemcpyAsync(G.p1, p1.data(), p1.size() * 8, cudaMemcpyHostToDevice, s));
  XL_CUDA_TRY(cudaMemcpyAsync(G.p2, p2.data(), p2.size() * 8, cudaMemcpyHostToDevice, s));
  XL_CUDA_TRY(cudaMemcpyAsync(G.pl, pl.data(), pl.size() * 8, cudaMemcpyHostToDevice, s));
  XL_CUDA_TRY(cudaMemcpyAsync(G.z1, z1.data(), cnt * 8, cudaMemcpyHostToDevice, s));
  XL_CUDA_TRY(cudaMemcpyAsync(G.z2, z2.data(), cnt * 8, cudaMemcpyHostToDevice, s));
  int* ids = nullptr;
  XL_TRY(dalloc(b, (void**)&ids, cnt * sizeof(int)));
  XL_CUDA_TRY(cudaMemcpyAsync(ids, G.setups.data(), cnt * sizeof(int), cudaMemcpyHostToDevice, s));
  {
    LaunchScope ls("batch_init", s);
    k_batch_init<T><<<1024, 256, 0, s>>>((cplx<T>*)G.src, (T*)G.phi1, (T*)G.phi2, G.n, G.grid.x0,
                                         G.pitch, b->cfg.w0, ids, seed, cnt);
    XL_CUDA_TRY(cudaGetLastError());
  }
  XL_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors above go out of scope
  return XL_OK;
}

xl_element el(int kind, const void* phx = nullptr, int64_t stride = 0) {
  xl_element e;
  std::memset(&e, 0, sizeof(e));
  e.kind = kind;
  e.phi_x = phx;
  e.phi_stride = stride;
  return e;
}

// One forward + backward + Adam step of one group.
xl_status group_step(xl_batch* b, Group& G, cudaStream_t s) {
  const xl_table_config& c = b->cfg;
  const int32_t dt = c.dtype;
  const int cnt = G.count;
  const int64_t plane = (int64_t)G.n * G.n;
  const double lam = c.wavelength;
  const xl_grid* g = &G.grid;
  xl_window win;
  win.mx = win.my = c.cam_m;
  win.dxo = win.dyo = c.cam_width / c.cam_m;
  win.xo0 = win.yo0 = -c.cam_width / 2;
  xl_grid wg{c.cam_m, c.cam_m, win.dxo, win.dyo, win.xo0, win.yo0};
  xl_element e_slm1[1] = {el(XL_SLM, G.phi1, plane)};
  xl_element e_mid[3] = {el(XL_SLM, G.phi2, plane), el(XL_TO_VECTOR), el(XL_WAVEPLATE)};
  xl_element e_lens[1] = {el(XL_LENS)};
  // forward
  const bool spectra = c.checkpoint == 0;
  const int32_t zf = XL_Z_DEVICE, zfb = XL_Z_DEVICE | XL_PHASE_INVARIANT;
  XL_TRY(xl_apply_elements(G.src, G.a0, cnt, 1, g, lam, e_slm1, 1, G.p1, zf, dt, s));
  if (spectra) XL_TRY(xl_rs_propagate_save(G.a0, G.a1, G.s1, cnt, g, lam, G.z1, zf, dt, s));
  else XL_TRY(xl_rs_propagate(G.a0, G.a1, cnt, g, lam, G.z1, zf, dt, s));
  XL_TRY(xl_apply_elements(G.a1, G.a2, cnt, 1, g, lam, e_mid, 3, G.p2, zf, dt, s));
  if (spectra) XL_TRY(xl_vrs_propagate_save(G.a2, G.a3, G.s2, cnt, g, lam, G.z2, zf, dt, s));
  else XL_TRY(xl_vrs_propagate(G.a2, G.a3, cnt, g, lam, G.z2, zf, dt, s));
  XL_TRY(xl_apply_elements(G.a3, G.a4, cnt, 3, g, lam, e_lens, 1, G.pl, zf, dt, s));
  // the VCZT distance is the fixed focal length: host distances, cached chirp tables
  XL_TRY(xl_czt_propagate(G.a4, G.a5, cnt, 2, g, &win, lam, G.zf.data(), 0, dt, s));
  // the loss and, starting the backward, its gradient; the gradients then alternate between gx
  // and gy (a4, in gx, is not read any more)
  XL_TRY(xl_intensity_loss_and_grad(G.a5, nullptr, nullptr, cnt, 3, 7u, &wg, XL_SECOND_MOMENT, 0.0, 0.0,
                                    G.loss, G.g5, nullptr, dt, s));
  XL_TRY(xl_czt_propagate_backward(G.g5, nullptr, G.gx, nullptr, cnt, 2, g, &win, lam, G.zf.data(), 0,
                                   dt, s));
  XL_TRY(xl_apply_elements_backward(G.gx, G.a3, G.gy, cnt, 3, g, lam, e_lens, 1, G.pl, zf,
                                    nullptr, nullptr, nullptr, dt, s));
  // the camera loss is invariant under a constant phase on every plane: drop the e^{ikz} term
  if (spectra)
    XL_TRY(xl_vrs_propagate_backward_saved(G.gy, G.s2, G.gx, G.gz2, cnt, g, lam, G.z2, zfb, dt, s));
  else
    XL_TRY(xl_vrs_propagate_backward(G.gy, G.a2, G.gx, G.gz2, cnt, g, lam, G.z2, zfb, dt, s));
  void* gpx_mid[3] = {G.gphi2, nullptr, nullptr};
  XL_TRY(xl_apply_elements_backward(G.gx, G.a1, G.gy, cnt, 1, g, lam, e_mid, 3, G.p2, zf,
                                    gpx_mid, nullptr, G.gp2, dt, s));
  if (spectra)
    XL_TRY(xl_rs_propagate_backward_saved(G.gy, G.s1, G.gx, G.gz1, cnt, g, lam, G.z1, zfb, dt, s));
  else
    XL_TRY(xl_rs_propagate_backward(G.gy, G.a0, G.gx, G.gz1, cnt, g, lam, G.z1, zfb, dt, s));
  void* gpx1[1] = {G.gphi1};
  XL_TRY(xl_apply_elements_backward(G.gx, G.src, nullptr, cnt, 1, g, lam, e_slm1, 1, G.p1,
                                    zf, gpx1, nullptr, nullptr, dt, s));
  // Adam on the masks and the scalars
  const int rd = dt == XL_C128 ? 1 : 0;
  XL_TRY(xl_adam_step(G.phi1, G.m1, G.v1, G.gphi1, cnt * plane, rd, c.lr, 0.9, 0.999, 1e-8, b->step, 0, s));
  XL_TRY(xl_adam_step(G.phi2, G.m2, G.v2, G.gphi2, cnt * plane, rd, c.lr, 0.9, 0.999, 1e-8, b->step, 0, s));
  {
    LaunchScope ls("batch_scalar_adam", s);
    k_batch_scalar_adam<<<(cnt + 127) / 128, 128, 0, s>>>(G.p2, G.z1, G.z2, G.gp2, G.gz1, G.gz2,
                                                          G.sm, G.sv, b->step, cnt, c.lr, c.lr_z);
    XL_CUDA_TRY(cudaGetLastError());
  }
  return XL_OK;
}

xl_status batch_step_eager(xl_batch* b, cudaStream_t s) {
  XL_TRY(xl_step_advance(b->step, s));
  for (Group& G : b->groups) XL_TRY(group_step(b, G, s));
  return XL_OK;
}

}  // namespace
}  // namespace xl

using namespace xl;

extern "C" {

xl_status xl_batch_create(const xl_table_config* cfg, int32_t n_setups, const int32_t* grid_n,
                          const double* init, uint64_t seed, xl_batch** out, void* stream) {
  if (!cfg || !grid_n || !init || !out) return fail(XL_ERR_ARG, "batch: NULL argument");
  if (n_setups < 1) return fail(XL_ERR_ARG, "batch: n_setups must be >= 1");
  if (cfg->dtype != XL_C64 && cfg->dtype != XL_C128) return fail(XL_ERR_ARG, "batch: bad dtype");
  if (cfg->checkpoint < 0 || cfg->checkpoint > XL_CHECKPOINT_AUTO)
    return fail(XL_ERR_ARG, "batch: checkpoint must be 0, 1 or XL_CHECKPOINT_AUTO");
  if (cfg->memory_budget < 0) return fail(XL_ERR_ARG, "batch: memory_budget must be >= 0");
  if (!(cfg->extent > 0) || !(cfg->wavelength > 0) || !(cfg->w0 > 0) || !(cfg->f > 0) ||
      cfg->cam_m < 1 || !(cfg->cam_width > 0))
    return fail(XL_ERR_ARG, "batch: bad table configuration");
  for (int i = 0; i < n_setups; ++i) {
    if (!is_pow2(grid_n[i]) || grid_n[i] < 32 || grid_n[i] > 4096)
      return fail(XL_ERR_UNSUPPORTED, "batch: grid sizes must be powers of two in [32, 4096]");
    if (!(init[3 * i + 1] > 0) || !(init[3 * i + 2] > 0)) return fail(XL_ERR_ARG, "batch: z must be > 0");
  }
  const int mode = resolve_checkpoint(*cfg, n_setups, grid_n);
  const int64_t need = plan_bytes(*cfg, n_setups, grid_n, mode);
  if (cfg->memory_budget > 0 && need > cfg->memory_budget)
    return fail(XL_ERR_NOMEM, "batch: the setups need more device memory than memory_budget");
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<xl_batch> b(new xl_batch);
  b->cfg = *cfg;
  b->cfg.checkpoint = mode;
  b->n_setups = n_setups;
  std::map<int, std::vector<int>> by_n;
  for (int i = 0; i < n_setups; ++i) by_n[grid_n[i]].push_back(i);
  for (auto& kv : by_n) {
    Group G;
    G.n = kv.first;
    G.count = (int)kv.second.size();
    G.setups = kv.second;
    G.pitch = cfg->extent / G.n;
    G.grid = xl_grid{G.n, G.n, G.pitch, G.pitch, -(G.n / 2) * G.pitch, -(G.n / 2) * G.pitch};
    b->groups.push_back(G);
  }
  xl_status st = XL_OK;
  if (dalloc(b.get(), (void**)&b->step, sizeof(int32_t)) != XL_OK) st = XL_ERR_NOMEM;
  if (st == XL_OK) {
    int32_t zero = 0;
    if (cudaMemcpyAsync(b->step, &zero, 4, cudaMemcpyHostToDevice, s) != cudaSuccess) st = XL_ERR_CUDA;
  }
  for (Group& G : b->groups) {
    if (st != XL_OK) break;
    st = cfg->dtype == XL_C128 ? group_alloc<double>(b.get(), G, init, seed, s)
                               : group_alloc<float>(b.get(), G, init, seed, s);
  }
  if (st != XL_OK) {
    for (void* p : b->allocs) cudaFree(p);
    return st;
  }
  *out = b.release();
  return XL_OK;
}

xl_status xl_batch_step(xl_batch* b, int32_t use_graph, void* stream) {
  if (!b) return fail(XL_ERR_ARG, "batch is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) return batch_step_eager(b, s);
  // The graph path runs on the batch's own non-blocking stream (a capture cannot use the legacy
  // default stream), ordered after and before the caller's stream by events. Its first call is
  // eager on that stream (it sizes the per-stream workspaces); the second captures the step.
  if (!b->own) {
    XL_CUDA_TRY(cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking));
    XL_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    XL_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
  }
  XL_CUDA_TRY(cudaEventRecord(b->ev_in, s));
  XL_CUDA_TRY(cudaStreamWaitEvent(b->own, b->ev_in, 0));
  if (!b->warmed) {
    XL_TRY(batch_step_eager(b, b->own));
    b->warmed = true;
  } else {
    if (!b->exec) {
      XL_CUDA_TRY(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal));
      xl_status st = batch_step_eager(b, b->own);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(b->own, &graph);
      if (st != XL_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return cuda_status(e, "batch graph capture");
      XL_CUDA_TRY(cudaGraphInstantiate(&b->exec, graph, 0));
      b->graph = graph;
    }
    XL_CUDA_TRY(cudaGraphLaunch(b->exec, b->own));
  }
  XL_CUDA_TRY(cudaEventRecord(b->ev_out, b->own));
  XL_CUDA_TRY(cudaStreamWaitEvent(s, b->ev_out, 0));
  return XL_OK;
}

xl_status xl_batch_read(xl_batch* b, int32_t what, int32_t setup, void* host_out, void* stream) {
  if (!b || !host_out) return fail(XL_ERR_ARG, "batch read: NULL argument");
  if (setup < 0 || setup >= b->n_setups) return fail(XL_ERR_ARG, "batch read: bad setup index");
  cudaStream_t s = (cudaStream_t)stream;
  for (Group& G : b->groups)
    for (int g = 0; g < G.count; ++g) {
      if (G.setups[g] != setup) continue;
      const size_t rs = b->cfg.dtype == XL_C128 ? 8 : 4;
      const int64_t plane = (int64_t)G.n * G.n;
      switch (what) {
        case XL_BATCH_LOSS:
          XL_CUDA_TRY(cudaMemcpyAsync(host_out, G.loss + g, 8, cudaMemcpyDeviceToHost, s));
          break;
        case XL_BATCH_SCALARS: {
          double* o = (double*)host_out;
          XL_CUDA_TRY(cudaMemcpyAsync(o, G.p2 + g * 12 + 11, 8, cudaMemcpyDeviceToHost, s));
          XL_CUDA_TRY(cudaMemcpyAsync(o + 1, G.z1 + g, 8, cudaMemcpyDeviceToHost, s));
          XL_CUDA_TRY(cudaMemcpyAsync(o + 2, G.z2 + g, 8, cudaMemcpyDeviceToHost, s));
          break;
        }
        case XL_BATCH_GRAD_SCALARS: {
          double* o = (double*)host_out;
          XL_CUDA_TRY(cudaMemcpyAsync(o, G.gp2 + g * 12 + 11, 8, cudaMemcpyDeviceToHost, s));
          XL_CUDA_TRY(cudaMemcpyAsync(o + 1, G.gz1 + g, 8, cudaMemcpyDeviceToHost, s));
          XL_CUDA_TRY(cudaMemcpyAsync(o + 2, G.gz2 + g, 8, cudaMemcpyDeviceToHost, s));
          break;
        }
        case XL_BATCH_PHI1:
        case XL_BATCH_PHI2:
        case XL_BATCH_GRAD_PHI1:
        case XL_BATCH_GRAD_PHI2: {
          void* src = what == XL_BATCH_PHI1 ? G.phi1 : what == XL_BATCH_PHI2 ? G.phi2
                    : what == XL_BATCH_GRAD_PHI1 ? G.gphi1 : G.gphi2;
          XL_CUDA_TRY(cudaMemcpyAsync(host_out, (char*)src + g * plane * rs, plane * rs,
                                      cudaMemcpyDeviceToHost, s));
          break;
        }
        default:
          return fail(XL_ERR_ARG, "batch read: unknown quantity");
      }
      XL_CUDA_TRY(cudaStreamSynchronize(s));
      return XL_OK;
    }
  return fail(XL_ERR_ARG, "batch read: setup not found");
}

int64_t xl_batch_memory(xl_batch* b) { return b ? b->bytes : -1; }

int64_t xl_batch_plan_memory(const xl_table_config* cfg, int32_t n_setups, const int32_t* grid_n,
                             int32_t* mode_out) {
  if (!cfg || !grid_n || n_setups < 1) return -1;
  if (cfg->dtype != XL_C64 && cfg->dtype != XL_C128) return -1;
  if (cfg->checkpoint < 0 || cfg->checkpoint > XL_CHECKPOINT_AUTO || cfg->memory_budget < 0) return -1;
  if (cfg->cam_m < 1) return -1;
  for (int i = 0; i < n_setups; ++i)
    if (!is_pow2(grid_n[i]) || grid_n[i] < 32 || grid_n[i] > 4096) return -1;
  const int mode = resolve_checkpoint(*cfg, n_setups, grid_n);
  if (mode_out) *mode_out = mode;
  return plan_bytes(*cfg, n_setups, grid_n, mode);
}

int32_t xl_batch_grid(xl_batch* b, int32_t setup) {
  if (!b) return -1;
  for (Group& G : b->groups)
    for (int g = 0; g < G.count; ++g)
      if (G.setups[g] == setup) return G.n;
  return -1;
}

xl_status xl_batch_destroy(xl_batch* b) {
  if (!b) return XL_OK;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->own) cudaStreamDestroy(b->own);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (void* p : b->allocs) cudaFree(p);
  delete b;
  return XL_OK;
}

}  // extern "C"
