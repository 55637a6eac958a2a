// Kernels and level loop for 16-byte keys (byte strings, 128-bit integers) with 8-byte payloads.
#include "driver.cuh"

namespace binar {
int run_call_k16_v8(const Call &c) { return run_call_vb<16, 8>(c); }
}  // namespace binar
