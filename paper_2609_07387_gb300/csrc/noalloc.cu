// ucns_time_step_static: the CFL time-step reduction with its per-block
// partial minima in a fixed, file-scope device array instead of memory the
// library allocates, for callers that must not allocate device memory on
// their call path.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ucns_internal.hpp"

namespace ucns {
// defined in api.cu: k_dt_partial (one partial minimum per 256-cell block into
// `partials`) followed by k_dt_final (dt_out[0] = CFL * min of the partials)
int launch_dt_into(const ucns_mesh* m, const double* U, double* partials, int nblocks, double* dt_out,
                   cudaStream_t s);
}  // namespace ucns

namespace {

using ucns::kDtBlockCells;                         // cells per partial minimum (the kernel's block size)
constexpr int kStaticDtPartials = 32768;           // 256 KiB of doubles
constexpr int64_t kStaticDtMaxCells = (int64_t)kStaticDtPartials * kDtBlockCells;  // 8,388,608

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_dt_scratch[kStaticDtPartials];

constexpr int kMaxDevices = 128;
std::mutex g_setup_mu;
// device address of g_dt_scratch per device ordinal, resolved once for the
// life of the process: it belongs to the device's primary context, so a
// context reset (cudaDeviceReset) invalidates it, and this entry point must
// not be used after one
void* g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" int ucns_time_step_static(const ucns_mesh* m, const double* U, double* dt, void* stream) {
  using ucns::fail;
  if (!m) return fail(UCNS_ERR_INVALID_ARG, "mesh handle is NULL");
  if (!m->precomputed) return fail(UCNS_ERR_STATE, "ucns_precompute has not been called");
  if (!U || !dt) return fail(UCNS_ERR_INVALID_ARG, "U or dt is NULL");
  if (m->N > kStaticDtMaxCells)
    return fail(UCNS_ERR_INVALID_ARG, "ucns_time_step_static: " + std::to_string(m->N) +
                                          " cells exceed its static scratch maximum of " +
                                          std::to_string(kStaticDtMaxCells) + " cells");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(UCNS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(UCNS_ERR_CUDA, "device ordinal out of range");
  void* scratch = nullptr;
  {
    // first call on this device (with it current): resolve the array's device
    // address; host code cannot use the symbol itself as a device pointer
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_dt_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        return fail(UCNS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    scratch = g_scratch_addr[dev];
  }
  const int nblocks = (int)((m->N + kDtBlockCells - 1) / kDtBlockCells);
  return ucns::launch_dt_into(m, U, (double*)scratch, nblocks, dt, (cudaStream_t)stream);
}
