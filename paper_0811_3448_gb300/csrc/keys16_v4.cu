// Kernels and level loop for 16-byte keys (byte strings, 128-bit integers) with 4-byte payloads.
#include "driver.cuh"

namespace binar {
int run_call_k16_v4(const Call &c) { return run_call_vb<16, 4>(c); }
}  // namespace binar
