// Kernels and level loop for 16-byte keys (byte strings, 128-bit integers) with no payload.
#include "driver.cuh"

namespace binar {
int run_call_k16_v0(const Call &c) { return run_call_vb<16, 0>(c); }
}  // namespace binar
