// Allocation-free entry point: sparstencil_run_noalloc.
//
// Some callers cannot call cudaMalloc: latency-critical services that forbid device
// allocation once they are running (cudaMalloc can synchronise the device and take
// milliseconds), and processes whose device memory belongs to a framework's caching
// allocator with a fixed budget (a raw cudaMalloc bypasses its accounting).  For them this
// file keeps the two padded ping-pong grids and the planner's device tables in file-scope
// static device arrays of a fixed size, so a run allocates nothing.  Each GPU that loads
// the library holds these arrays until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "sparstencil.h"

namespace spst {
// Records a failure for sparstencil_last_error (implemented in capi.cpp).
sparstencil_status report_error(sparstencil_status s, const char* msg);
// Runs a plan with caller-provided device buffers (implemented in capi.cpp).
sparstencil_status run_plan_with_buffers(sparstencil_plan_t plan, const float* in, float* out, int64_t timesteps,
                                         cudaStream_t stream, float* scratch, size_t scratch_floats,
                                         uint32_t* tables, size_t table_words, unsigned* maxabs_word);
}  // namespace spst

namespace {

// Largest padded grid (rows x padded columns, in floats) the static scratch holds: two such
// grids, 2 x 16 MiB.  Example: a 2040 x 2040 grid with ghost width 4 pads to 2048 x 2048.
constexpr size_t kNoAllocGridFloats = (size_t)4 << 20;
// Device tables (lookup table, A'' pieces, metadata) for the full and the remainder sweep.
constexpr size_t kNoAllocTableWords = (size_t)128 << 10;

static __device__ __align__(256) float g_noalloc_scratch[2 * kNoAllocGridFloats];
static __device__ __align__(256) uint32_t g_noalloc_tables[kNoAllocTableWords];
// max |input| of the current run (FP16 operands' data scale)
static __device__ unsigned g_noalloc_maxabs;

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
float* g_scratch_ptr[kMaxDevices] = {nullptr};
uint32_t* g_tables_ptr[kMaxDevices] = {nullptr};
unsigned* g_maxabs_ptr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" sparstencil_status sparstencil_run_noalloc(sparstencil_plan_t plan, const float* in, float* out,
                                                      int64_t timesteps, cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return spst::report_error(SPST_ERR_CUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return spst::report_error(SPST_ERR_UNSUPPORTED, "device index out of range");
  float* scratch = nullptr;
  uint32_t* tables = nullptr;
  unsigned* maxabs = nullptr;
  {
    // One-time set-up per device, with that device current: the host-side names of the
    // arrays are not device addresses, so resolve them with cudaGetSymbolAddress.
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      void* s = nullptr;
      void* t = nullptr;
      if (cudaGetSymbolAddress(&s, g_noalloc_scratch) != cudaSuccess)
        return spst::report_error(SPST_ERR_CUDA, "cudaGetSymbolAddress(static scratch) failed");
      if (cudaGetSymbolAddress(&t, g_noalloc_tables) != cudaSuccess)
        return spst::report_error(SPST_ERR_CUDA, "cudaGetSymbolAddress(static tables) failed");
      void* m = nullptr;
      if (cudaGetSymbolAddress(&m, g_noalloc_maxabs) != cudaSuccess)
        return spst::report_error(SPST_ERR_CUDA, "cudaGetSymbolAddress(static data-scale word) failed");
      g_scratch_ptr[dev] = (float*)s;
      g_tables_ptr[dev] = (uint32_t*)t;
      g_maxabs_ptr[dev] = (unsigned*)m;
    }
    scratch = g_scratch_ptr[dev];
    tables = g_tables_ptr[dev];
    maxabs = g_maxabs_ptr[dev];
  }
  return spst::run_plan_with_buffers(plan, in, out, timesteps, stream, scratch, 2 * kNoAllocGridFloats, tables,
                                     kNoAllocTableWords, maxabs);
}
