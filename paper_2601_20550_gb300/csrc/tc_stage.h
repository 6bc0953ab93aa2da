// Tensor-core (tcgen05) RK4 stage for the mixed-precision path (HEOM_BF16X3).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.cuh"
#include "model.h"

namespace heom {

struct TcOperators {
  bool ready = false;
  int d = 0, dpad = 0;
  DevModel<float> dm{};
};

// Prepare the tensor-core operator tiles of M (device allocations are appended to allocs).
void tc_build(TcOperators &tc, const Model &M, const DevModel<float> &dm, std::vector<void *> &allocs);
bool tc_supported(const TcOperators &tc);
// n RK4 steps (Horner form) on complex64 branches y with scratch wa, wb.
void tc_rk4_steps(const TcOperators &tc, float2 *y, float2 *wa, float2 *wb, int branches, double dt,
                  int64_t nsteps, cudaStream_t st);

}  // namespace heom
