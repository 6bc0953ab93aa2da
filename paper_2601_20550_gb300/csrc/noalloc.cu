// Allocation-free RK4 propagation (heom_propagate_noalloc).
//
// Some callers cannot allocate device memory at the point where they propagate:
// code that runs while a framework's caching allocator owns the device memory
// pool, real-time loops in which a cudaMalloc (which may synchronise the device)
// is not acceptable, and plug-ins that are handed device buffers but no
// allocation rights.  This entry point serves them: the two RK4 scratch buffers
// live in a file-scope __device__ array of fixed size that every GPU loading the
// library holds until the process exits.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "heom2dvs.h"
#include "kernels.cuh"

namespace heom {
bool hier_on_device(const heom_hier *h);
const DevModel<double> &hier_dm64(const heom_hier *h);
void hier_set_error(const char *msg);
void count_launch(uint64_t n);
}  // namespace heom

using namespace heom;

namespace {

// Two scratch states of HEOM_NOALLOC_MAX_BYTES each (complex128 elements).
constexpr int64_t kScratchElems = HEOM_NOALLOC_MAX_BYTES / 16;
__device__ __align__(256) double2 g_noalloc_scratch[2 * kScratchElems];

constexpr int kMaxDevices = 64;
double2 *g_scratch_addr[kMaxDevices] = {nullptr};
int g_sm_count[kMaxDevices] = {0};
std::mutex g_scratch_mutex;

// Device address of the scratch array and the SM count of the current device
// (resolved once per device with that device current; the host-side symbol is
// not a device address).
cudaError_t scratch_address(double2 **out, int *sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_sm_count[dev] = n > 0 ? n : 1;
    g_scratch_addr[dev] = static_cast<double2 *>(p);
  }
  *out = g_scratch_addr[dev];
  *sms = g_sm_count[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" heom_status heom_propagate_noalloc(heom_hier *h, void *state, int branches, double dt_fs,
                                              int64_t n_steps, void *stream) {
  if (!h || !state || branches < 1 || n_steps < 0 || !(dt_fs > 0) || !std::isfinite(dt_fs)) {
    hier_set_error("heom_propagate_noalloc: bad arguments");
    return HEOM_EINVAL;
  }
  // complex128 elements: a misaligned pointer would fault in the kernel
  if ((uintptr_t)state & 15u) {
    hier_set_error("state buffers must be aligned to their complex element size");
    return HEOM_EINVAL;
  }
  if (!hier_on_device(h)) {
    hier_set_error("heom_propagate_noalloc: the hierarchy has no device tables yet; make one device call "
                   "(for example heom_state_create) first");
    return HEOM_EINVAL;
  }
  const DevModel<double> &dm = hier_dm64(h);
  const int64_t total = (int64_t)branches * dm.n_ado * dm.d * dm.d;
  if (total > kScratchElems) {
    const std::string msg = "heom_propagate_noalloc: state of " + std::to_string((long long)(total * 16)) +
                            " bytes exceeds the fixed scratch limit of " +
                            std::to_string((long long)(kScratchElems * 16)) + " bytes";
    hier_set_error(msg.c_str());
    return HEOM_EINVAL;
  }
  double2 *scratch = nullptr;
  int sms = 1;
  cudaError_t e = scratch_address(&scratch, &sms);
  if (e != cudaSuccess) {
    hier_set_error(cudaGetErrorString(e));
    return HEOM_ECUDA;
  }
  // clear an error left by an earlier, unrelated call so that only this call's
  // launches are reported below
  (void)cudaGetLastError();
  double2 *y = static_cast<double2 *>(state), *wa = scratch, *wb = scratch + kScratchElems;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t blocks = (total + 255) / 256;
  const int64_t cap = (int64_t)sms * 64;
  const int grid = (int)(blocks < cap ? blocks : cap);
  for (int64_t s = 0; s < n_steps; ++s) {
    stage_kernel<double><<<grid, 256, 0, st>>>(y, y, wa, dt_fs / 4, dm, total);
    stage_kernel<double><<<grid, 256, 0, st>>>(wa, y, wb, dt_fs / 3, dm, total);
    stage_kernel<double><<<grid, 256, 0, st>>>(wb, y, wa, dt_fs / 2, dm, total);
    stage_kernel<double><<<grid, 256, 0, st>>>(wa, y, y, dt_fs, dm, total);
    count_launch(4);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    hier_set_error(cudaGetErrorString(e));
    return HEOM_ECUDA;
  }
  return HEOM_OK;
}
