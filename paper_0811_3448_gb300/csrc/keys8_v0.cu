// Kernels and level loop for 8-byte keys (uint64, int64, float64) with no payload.
#include "driver.cuh"

namespace binar {
int run_call_k8_v0(const Call &c) { return run_call_vb<8, 0>(c); }
}  // namespace binar
