// Kernels and level loop for 8-byte keys (uint64, int64, float64).
#include "driver.cuh"

namespace binar {
int run_call_k8(const Call &c) { return run_call<8>(c); }
}  // namespace binar
