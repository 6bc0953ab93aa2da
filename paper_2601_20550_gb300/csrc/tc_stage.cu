// Tensor-core (tcgen05) RK4 stage for the mixed-precision path.
#include "tc_stage.h"

#include <stdexcept>

namespace heom {

void tc_build(TcOperators &tc, const Model &M, const DevModel<float> &dm, std::vector<void *> &allocs) {
  (void)allocs;
  tc.d = M.d;
  tc.dm = dm;
  tc.ready = false;
  throw std::invalid_argument("HEOM_BF16X3 is not available for this basis size yet");
}

bool tc_supported(const TcOperators &tc) { return tc.ready; }

void tc_rk4_steps(const TcOperators &, float2 *, float2 *, float2 *, int, double, int64_t, cudaStream_t) {
  throw std::invalid_argument("tensor-core stage not built");
}

}  // namespace heom
