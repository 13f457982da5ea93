// Host-side runtime of the xl library: twiddle tables, per-stream workspaces and the cache of
// transfer spectra / chirp tables. All state is per device and guarded by one mutex.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>

#include "xl_common.cuh"

namespace xl {

// Twiddle tables of a length-L transform in the precision of dtype (float2 or double2): for each
// stage s >= 1 (sub-transform size Ns, radix R) the R x Ns values exp(-2 pi i k r / (Ns R)),
// computed in double precision on the host. Created on first use (synchronous upload).
xl_status twiddles(int L, int dtype, const void** out);
// The same for radix plan `plan` of xl_fft.cuh (0 is the table above).
xl_status twiddles(int L, int dtype, int plan, const void** out);

// Workspace of at least `bytes` for `stream` on the current device. Growing it synchronises the
// device (cudaFree); the pointer stays valid until the next call that grows it or xl_cache_clear.
xl_status workspace(cudaStream_t stream, size_t bytes, void** out, int slot = 0);

// Cache of generated tables. The key is an opaque byte string built by the caller. On a miss
// the buffer is allocated (evicting least-recently-used entries above the byte cap), `gen` is
// enqueued on `stream` to fill it and the host waits for it, so a hit needs no synchronisation.
xl_status cached_table(const std::string& key, size_t bytes, cudaStream_t stream,
                       const std::function<xl_status(void*)>& gen, void** out);

// Byte cap of that cache (XL_CACHE_BYTES, default 8 GiB). A caller that holds several entries
// for one launch keeps their total within half of it, so that filling one never evicts another.
size_t table_cache_cap();

// Key helper: appends the raw bytes of a value.
template <typename V> inline void key_put(std::string& k, const V& v) {
  k.append(reinterpret_cast<const char*>(&v), sizeof(V));
}

// Sets the dynamic shared memory limit of a kernel once (per process).
xl_status smem_attr(const void* func, size_t bytes);

// Tensor map of a row-major 2D array of 8-byte elements (inner extent `inner`, `outer` rows of
// `row_bytes` each) for tiled bulk copies of box_inner x box_outer elements; out-of-range
// elements read as zero. The base must be 16-byte aligned and row_bytes a multiple of 16.
xl_status tensor_map_2d_u64(const void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                            uint32_t box_inner, uint32_t box_outer, void* map_out /* 128 bytes */);

// Device word of error bits that kernels set (bit 1: a wait on a bulk copy gave up); read and
// cleared by xl_device_status().
xl_status status_word(unsigned int** out);
xl_status status_word_take(cudaStream_t s, unsigned int* bits);

size_t dtype_csize(int dtype);  // bytes of one complex element

// Streaming multiprocessors of the current device (queried once per device; 152 on a GB300).
int sm_count();

// Launch variants chosen by the autotuner (xl_autotune): for each tunable kernel family, row
// length L and dtype, the variant index (0 = the built-in default). Families: the transposing
// row passes, whose variants differ in rows per block (threads per block, register budget and
// shared memory): 1 = half the default rows, 2 = twice the default rows (where that fits).
enum TuneFamily {
  TUNE_RS_PASS1 = 0,
  TUNE_RS_PASS3 = 1,
  TUNE_CZT_FWD_X = 2,
  TUNE_CZT_FWD_Y = 3,
  TUNE_CZT_ADJ_X = 4,
  TUNE_CZT_ADJ_Y = 5,
  TUNE_NFAMILY = 6
};
constexpr int kTuneVariants = 3;
constexpr int kTuneMinL = 1024;  // shorter rows build only the default variant
// The CZT window passes of complex64 scalar fields at the lengths with a radix-2/4/8 stage
// (512, 1024, 2048) have two more variants: the default rows with radix plan 1 (3) and plan 2 (4)
// (the odd stage first or second instead of last).
constexpr int kTuneVariantsPlans = 5;
inline bool czt_plan_lengths(int L) { return L == 512 || L == 1024 || L == 2048; }
const char* tune_family_name(int family);
int tuned_variant(int family, int L, int dtype);
void set_tuned_variant(int family, int L, int dtype, int variant, double us);
// The recorded choices as text lines "family L dtype variant microseconds".
std::string tune_table_text();
void tune_clear();

// Brackets one kernel launch: counts it and, while profiling is enabled, records CUDA events on
// its stream before and after it (name = kernel family, e.g. "rs_pass2<4096>").
class LaunchScope {
 public:
  LaunchScope(const std::string& name, cudaStream_t s);
  ~LaunchScope();

 private:
  int slot_ = -1;
  cudaStream_t s_;
};

}  // namespace xl
