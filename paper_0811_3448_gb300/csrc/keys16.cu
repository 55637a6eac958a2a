// Kernels and level loop for 16-byte keys (byte strings, 128-bit integers).
#include "driver.cuh"

namespace binar {
int run_call_k16(const Call &c) { return run_call<16>(c); }
}  // namespace binar
