// cans_poisson_solve_noalloc: the Poisson solve for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a plugin hosted by a framework that owns the whole device
// memory pool and forbids side allocations, code under a hard device-memory budget fixed at start-up,
// or a time-critical loop where an allocation (which can wait for the device to go idle) is not
// acceptable.  Such a caller still owns f and p, but it cannot hand the mixed-precision solve the
// workspace that cans_poisson_workspace_size() asks for.  This entry point supplies that workspace
// from a fixed array that lives in the library itself.
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds it, at the
// size below, until the process exits.  Under CUDA's lazy module loading (the default) the memory is
// committed when the first call on a device loads this part of the library, so a caller whose pool
// will take the device's memory makes that first call before the pool does (and before any stream
// capture).  In host code the array's name is only a host-side stand-in, so the device address is
// looked up with cudaGetSymbolAddress, with that device current, on the first call made on it, and
// kept; later calls check the kept address with cudaPointerGetAttributes (a host-side query) and look
// it up again if the device was reset in between.  Every call shares the one array: calls that
// overlap on the GPU (two streams, two threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "cans.h"

namespace {

// Maximum scratch: 48 MiB, enough for the mixed solve of up to 4,194,304 points (12 bytes per point).
constexpr size_t kScratchBytes = size_t(48) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_lock;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (looked up on first use, and again when the kept
// address no longer belongs to this device's live context, e.g. after cudaDeviceReset); nullptr on
// failure.
void* scratch_address() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> guard(g_lock);
  if (g_scratch_ptr[dev] != nullptr) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, g_scratch_ptr[dev]) != cudaSuccess || attr.type != cudaMemoryTypeDevice ||
        attr.device != dev) {
      cudaGetLastError();  // the failed query leaves no sticky error behind
      g_scratch_ptr[dev] = nullptr;
    }
  }
  if (g_scratch_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess) return nullptr;
    g_scratch_ptr[dev] = ptr;
  }
  return g_scratch_ptr[dev];
}

}  // namespace

extern "C" {

size_t cans_noalloc_scratch_bytes(void) { return kScratchBytes; }

int cans_poisson_solve_noalloc(cans_plan_t plan, const double* f, double* p, void* cuda_stream, double* info) {
  if (!plan || !f || !p) return CANS_ERR_ARG;
  size_t need = 0;
  int st = cans_poisson_workspace_size(plan, &need);
  if (st != CANS_OK) return st;
  if (need > kScratchBytes) return CANS_ERR_WORKSPACE;  // the problem is larger than the fixed scratch
  void* ws = nullptr;
  if (need > 0) {
    ws = scratch_address();
    if (ws == nullptr) return CANS_ERR_CUDA;
  }
  // The solve writes every workspace word before reading it, so nothing needs clearing between calls.
  return cans_poisson_solve(plan, f, p, ws, cuda_stream, info);
}

}  // extern "C"
