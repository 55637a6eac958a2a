// Kernels and level loop for 4-byte keys (uint32, int32, float32).
#include "driver.cuh"

namespace binar {
int run_call_k4(const Call &c) { return run_call<4>(c); }
}  // namespace binar
