// Kernels and level loop for 8-byte keys (uint64, int64, float64) with 4-byte payloads.
#include "driver.cuh"

namespace binar {
int run_call_k8_v4(const Call &c) { return run_call_vb<8, 4>(c); }
}  // namespace binar
