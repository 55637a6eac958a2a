// Kernels and level loop for 8-byte keys (uint64, int64, float64) with 8-byte payloads.
#include "driver.cuh"

namespace binar {
int run_call_k8_v8(const Call &c) { return run_call_vb<8, 8>(c); }
}  // namespace binar
