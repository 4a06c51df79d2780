// Quartic coefficients of a line search without any device allocation.
//
// Some callers cannot allocate device memory when they need this step: a
// host runtime that has handed the whole device to its own memory pool, a
// code path that must not synchronise the device (cudaMalloc/cudaFree can),
// or an embedding where the library must not grow the footprint after start
// up. For them the scratch of the trace reduction (the per-block partial sums
// and the one-solve control block) lives in one file-scope device array,
// sized for n up to kNoAllocMaxN, that every GPU which loads this library
// keeps until the process exits.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the device address is looked up once per
// device with cudaGetSymbolAddress, on the first call made while that device
// is current, and handed to the kernels. That first call should therefore
// come before any stream capture. The address stays cached for the life of the
// process: after a cudaDeviceReset the device's modules are reloaded and the
// cached address no longer names the array, so this entry point must not be
// called again on a device that has been reset. Every call shares the one array: calls that
// overlap on the GPU (several streams, or several host threads) race and must
// be serialised by the caller. The control block is rewritten at the start of
// every call; the partial sums are fully overwritten by the trace kernel.
#include "../../include/omm_kernels.h"
#include "omm_internal.cuh"

#include <cstring>
#include <mutex>
#include <string>

using namespace omm;

namespace {

constexpr int kNoAllocMaxN = 2048;
constexpr long kMaxTiles = (long)((kNoAllocMaxN + 31) / 32) * ((kNoAllocMaxN + 31) / 32);
constexpr long kScalarSlots = ((long)sizeof(Scalars) + 255) / 256 * 256 / 8;  // keep partials 256-B aligned
constexpr long kScratchDoubles = kScalarSlots + kMaxTiles * kNumTraces;

// about 361 KB per device
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" omm_status omm_kernel_quartic_coefficients_noalloc(int n, const double* SWHW, const double* Proj,
                                                              double E, double* alpha, void* stream) {
  if (n <= 0 || !SWHW || !Proj || !alpha) {
    set_last_error("omm_kernel_quartic_coefficients_noalloc: invalid argument");
    return OMM_ERR_ARG;
  }
  if (n > kNoAllocMaxN) {
    set_last_error("omm_kernel_quartic_coefficients_noalloc: n = " + std::to_string(n) +
                   " exceeds the static scratch limit n <= " + std::to_string(kNoAllocMaxN));
    return OMM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  try {
    double* base = nullptr;
    OMM_CUDA_TRY(scratch_address(&base));
    Scalars* sc = reinterpret_cast<Scalars*>(base);
    double* part = base + kScalarSlots;
    Scalars h;
    std::memset(&h, 0, sizeof(h));
    h.E = E;
    h.max_iter = 1;
    OMM_CUDA_TRY(cudaMemcpyAsync(sc, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    launch_traces(st, n, SWHW, Proj, part, sc);
    launch_control_linesearch(st, sc, part, traces_partials(n));
    OMM_CUDA_TRY(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, st));
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
    for (int q = 0; q < 5; ++q) alpha[q] = h.alpha[q];
  } catch (const CudaError& e) {
    set_last_error(std::string("omm_kernel_quartic_coefficients_noalloc: ") + e.what + ": " +
                   cudaGetErrorString(e.err));
    return OMM_ERR_CUDA;
  }
  return OMM_OK;
}
