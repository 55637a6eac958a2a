// Kernels and level loop for 4-byte keys (uint32, int32, float32) with no payload.
#include "driver.cuh"

namespace binar {
int run_call_k4_v0(const Call &c) { return run_call_vb<4, 0>(c); }
}  // namespace binar
