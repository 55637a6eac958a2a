// Kernels and level loop for 4-byte keys (uint32, int32, float32) with 8-byte payloads.
#include "driver.cuh"

namespace binar {
int run_call_k4_v8(const Call &c) { return run_call_vb<4, 8>(c); }
}  // namespace binar
