// Host runtime: error strings, twiddle tables, workspaces, table cache.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <list>
#include <map>
#include <tuple>
#include <mutex>
#include <unordered_map>
#include <vector>
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "xl_runtime.h"

namespace xl {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

xl_status fail(xl_status code, const std::string& msg) {
  set_error(msg);
  return code;
}

xl_status cuda_status(cudaError_t e, const char* where) {
  cudaGetLastError();  // clear a sticky launch error so the next call starts clean
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  set_error(m);
  return e == cudaErrorMemoryAllocation ? XL_ERR_NOMEM : XL_ERR_CUDA;
}

size_t dtype_csize(int dtype) { return dtype == XL_C128 ? 16 : 8; }

namespace {

struct Entry {
  void* ptr = nullptr;
  size_t bytes = 0;
  cudaEvent_t ready = nullptr;
  cudaStream_t owner = nullptr;
  std::list<std::string>::iterator lru_it;
};

struct DeviceState {
  std::map<std::pair<int, int>, void*> tw;                        // (L, dtype) -> table
  std::map<std::pair<cudaStream_t, int>, std::pair<void*, size_t>> ws;  // workspaces
  std::unordered_map<std::string, Entry> cache;
  std::list<std::string> lru;  // front = most recent
  size_t cache_bytes = 0;
};

std::mutex g_mu;
std::map<int, DeviceState> g_dev;
std::map<const void*, size_t> g_smem_set;

size_t cache_cap() {
  static size_t cap = [] {
    const char* e = std::getenv("XL_CACHE_BYTES");
    return e ? (size_t)std::strtoull(e, nullptr, 10) : (size_t)8 << 30;
  }();
  return cap;
}

DeviceState& cur(int* dev_out = nullptr) {
  int d = 0;
  cudaGetDevice(&d);
  if (dev_out) *dev_out = d;
  return g_dev[d];
}

}  // namespace

size_t table_cache_cap() { return cache_cap(); }

// ---------------------------------------------------------------------------------------------
// Autotuner choices: (family, L, dtype) -> (variant, measured microseconds). Process-wide (the
// variants are properties of the kernels, and the library serves one GPU model per process).
namespace {
struct TuneEntry {
  int variant;
  double us;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TuneEntry> g_tune;
const char* const kTuneNames[TUNE_NFAMILY] = {"rs_pass1", "rs_pass3", "czt_fwd_x",
                                              "czt_fwd_y", "czt_adj_x", "czt_adj_y"};
}  // namespace

const char* tune_family_name(int family) {
  return family >= 0 && family < TUNE_NFAMILY ? kTuneNames[family] : "?";
}

int tuned_variant(int family, int L, int dtype) {
  if (L < kTuneMinL && !(family >= TUNE_CZT_FWD_X && czt_plan_lengths(L))) return 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(family, L, dtype));
  return it == g_tune.end() ? 0 : it->second.variant;
}

void set_tuned_variant(int family, int L, int dtype, int variant, double us) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[std::make_tuple(family, L, dtype)] = TuneEntry{variant, us};
}

std::string tune_table_text() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::string out;
  char line[160];
  for (const auto& kv : g_tune) {
    std::snprintf(line, sizeof(line), "%s %d %s %d %.3f\n", tune_family_name(std::get<0>(kv.first)),
                  std::get<1>(kv.first), std::get<2>(kv.first) == XL_C128 ? "c128" : "c64",
                  kv.second.variant, kv.second.us);
    out += line;
  }
  return out;
}

void tune_clear() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

int sm_count() {
  static int counts[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (counts[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
    counts[dev] = n;
  }
  return counts[dev];
}

xl_status smem_attr(const void* func, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_smem_set.find(func);
  if (it != g_smem_set.end() && it->second >= bytes) return XL_OK;
  XL_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  g_smem_set[func] = bytes;
  return XL_OK;
}

xl_status tensor_map_2d_u64(const void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                            uint32_t box_inner, uint32_t box_outer, void* map_out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      XL_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q));
      if (q != cudaDriverEntryPointSuccess || !fn)
        return fail(XL_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
      encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
  }
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode((CUtensorMap*)map_out, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                            const_cast<void*>(base), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(XL_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return XL_OK;
}

xl_status status_word(unsigned int** out) {
  static std::map<int, unsigned int*> words;
  int dev = 0;
  XL_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = words.find(dev);
  if (it == words.end()) {
    unsigned int* w = nullptr;
    XL_CUDA_TRY(cudaMalloc(&w, sizeof(unsigned int)));
    XL_CUDA_TRY(cudaMemset(w, 0, sizeof(unsigned int)));
    XL_CUDA_TRY(cudaDeviceSynchronize());
    it = words.emplace(dev, w).first;
  }
  *out = it->second;
  return XL_OK;
}

xl_status status_word_take(cudaStream_t s, unsigned int* bits) {
  unsigned int* w = nullptr;
  XL_TRY(status_word(&w));
  XL_CUDA_TRY(cudaMemcpyAsync(bits, w, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  XL_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(unsigned int), s));
  XL_CUDA_TRY(cudaStreamSynchronize(s));
  return XL_OK;
}

xl_status twiddles(int L, int dtype, const void** out) { return twiddles(L, dtype, 0, out); }

xl_status twiddles(int L, int dtype, int plan, const void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceState& st = cur();
  auto key = std::make_pair(L, dtype + 16 * plan);
  auto it = st.tw.find(key);
  if (it != st.tw.end()) {
    *out = it->second;
    return XL_OK;
  }
  // per-stage blocks: stage s >= 1 has R x Ns entries exp(-2 pi i k r / (Ns R)), r-major (the
  // layout read by apply_twiddles in xl_fft.cuh); the stages' radices follow the plan (all 16
  // but one of 2^(log2 L mod 4), which sits last, first or second)
  const int lg = ilog2(L), rem = lg % 4, nst = lg / 4 + (rem ? 1 : 0);
  const int pos = rem == 0 ? -1 : (plan == 1 ? 0 : (plan == 2 && nst > 2 ? 1 : nst - 1));
  std::vector<double> w;
  int Ns = pos == 0 ? (1 << rem) : 16;
  for (int s = 1; s < nst; ++s) {
    const int R = s == pos ? (1 << rem) : 16;
    for (int r = 0; r < R; ++r)
      for (int k = 0; k < Ns; ++k) {
        const double ang = -kTwoPi * (double)k * (double)r / ((double)Ns * (double)R);
        w.push_back(std::cos(ang));
        w.push_back(std::sin(ang));
      }
    Ns *= R;
  }
  if (w.empty()) w.assign(2, 0.0);
  void* d = nullptr;
  const size_t n = w.size() / 2;
  size_t bytes = n * dtype_csize(dtype);
  XL_CUDA_TRY(cudaMalloc(&d, bytes));
  if (dtype == XL_C128) {
    XL_CUDA_TRY(cudaMemcpy(d, w.data(), bytes, cudaMemcpyHostToDevice));
  } else {
    std::vector<float> f(w.size());
    for (size_t i = 0; i < f.size(); ++i) f[i] = (float)w[i];
    XL_CUDA_TRY(cudaMemcpy(d, f.data(), bytes, cudaMemcpyHostToDevice));
  }
  st.tw[key] = d;
  *out = d;
  return XL_OK;
}

xl_status workspace(cudaStream_t stream, size_t bytes, void** out, int slot) {
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceState& st = cur();
  auto& e = st.ws[std::make_pair(stream, slot)];
  if (e.second < bytes) {
    if (e.first) {
      XL_CUDA_TRY(cudaStreamSynchronize(stream));
      XL_CUDA_TRY(cudaFree(e.first));
      e.first = nullptr;
      e.second = 0;
    }
    size_t n = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    cudaError_t err = cudaMalloc(&p, n);
    if (err != cudaSuccess) return cuda_status(err, "workspace cudaMalloc");
    e.first = p;
    e.second = n;
  }
  *out = e.first;
  return XL_OK;
}

xl_status cached_table(const std::string& key, size_t bytes, cudaStream_t stream,
                       const std::function<xl_status(void*)>& gen, void** out) {
  std::unique_lock<std::mutex> lk(g_mu);
  int dev = 0;
  DeviceState& st = cur(&dev);
  auto it = st.cache.find(key);
  if (it != st.cache.end()) {
    Entry& e = it->second;
    st.lru.erase(e.lru_it);
    st.lru.push_front(key);
    e.lru_it = st.lru.begin();
    *out = e.ptr;  // complete: the generating call synchronised its stream
    return XL_OK;
  }
  // evict least-recently-used entries until the new one fits under the cap
  while (!st.lru.empty() && st.cache_bytes + bytes > cache_cap()) {
    std::string victim = st.lru.back();
    st.lru.pop_back();
    Entry& v = st.cache[victim];
    XL_CUDA_TRY(cudaEventSynchronize(v.ready));
    XL_CUDA_TRY(cudaFree(v.ptr));
    XL_CUDA_TRY(cudaEventDestroy(v.ready));
    st.cache_bytes -= v.bytes;
    st.cache.erase(victim);
  }
  Entry e;
  e.bytes = bytes;
  e.owner = stream;
  cudaError_t err = cudaMalloc(&e.ptr, bytes);
  if (err != cudaSuccess) return cuda_status(err, "spectrum cache cudaMalloc");
  XL_CUDA_TRY(cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming));
  lk.unlock();
  xl_status s = gen(e.ptr);
  lk.lock();
  if (s != XL_OK) {
    cudaFree(e.ptr);
    cudaEventDestroy(e.ready);
    return s;
  }
  // Wait for the generation on the host (misses happen once per table), so that every stream,
  // and every later graph capture, may use the entry without an event dependency.
  XL_CUDA_TRY(cudaEventRecord(e.ready, stream));
  XL_CUDA_TRY(cudaEventSynchronize(e.ready));
  st.lru.push_front(key);
  e.lru_it = st.lru.begin();
  st.cache_bytes += bytes;
  st.cache[key] = e;
  *out = e.ptr;
  return XL_OK;
}

namespace {
struct ProfRec {
  std::string name;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_ev_pool;
int64_t g_launches = 0;

cudaEvent_t ev_get() {
  if (!g_ev_pool.empty()) {
    cudaEvent_t e = g_ev_pool.back();
    g_ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

LaunchScope::LaunchScope(const std::string& name, cudaStream_t s) : s_(s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ++g_launches;
  if (!g_prof_on) return;
  ProfRec r{name, ev_get(), ev_get()};
  cudaEventRecord(r.a, s);
  slot_ = (int)g_prof.size();
  g_prof.push_back(r);
}

LaunchScope::~LaunchScope() {
  if (slot_ < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEventRecord(g_prof[slot_].b, s_);
}

}  // namespace xl

using namespace xl;

extern "C" {

const char* xl_version(void) { return "xl 0.1 (sm_103a)"; }

const char* xl_last_error(void) { return g_last_error.c_str(); }

xl_status xl_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  int dev0 = 0;
  cudaGetDevice(&dev0);
  for (auto& kv : g_dev) {
    XL_CUDA_TRY(cudaSetDevice(kv.first));
    XL_CUDA_TRY(cudaDeviceSynchronize());
    DeviceState& st = kv.second;
    for (auto& c : st.cache) {
      cudaFree(c.second.ptr);
      cudaEventDestroy(c.second.ready);
    }
    st.cache.clear();
    st.lru.clear();
    st.cache_bytes = 0;
    for (auto& w : st.ws) cudaFree(w.second.first);
    st.ws.clear();
  }
  XL_CUDA_TRY(cudaSetDevice(dev0));
  return XL_OK;
}

int64_t xl_launch_count(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_launches;
}

xl_status xl_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return XL_OK;
}

int32_t xl_profile_report(char* buf, int32_t len) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::map<std::string, std::pair<int64_t, double>> agg;
  for (auto& r : g_prof) {
    float ms = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& e = agg[r.name];
    e.first += 1;
    e.second += ms;
    g_ev_pool.push_back(r.a);
    g_ev_pool.push_back(r.b);
  }
  g_prof.clear();
  std::string out;
  char line[256];
  for (auto& kv : agg) {
    snprintf(line, sizeof(line), "%s %lld %.6f\n", kv.first.c_str(), (long long)kv.second.first,
             kv.second.second);
    out += line;
  }
  if (buf && len > 0) {
    int32_t n = (int32_t)std::min<size_t>(out.size(), (size_t)len - 1);
    std::memcpy(buf, out.data(), n);
    buf[n] = 0;
  }
  return (int32_t)out.size() + 1;
}

int64_t xl_cache_bytes(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  int64_t n = 0;
  for (auto& kv : g_dev) {
    n += (int64_t)kv.second.cache_bytes;
    for (auto& w : kv.second.ws) n += (int64_t)w.second.second;
  }
  return n;
}

}  // extern "C"
