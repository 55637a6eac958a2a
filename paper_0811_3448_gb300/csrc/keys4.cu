// Dispatch by payload width for 4-byte keys (uint32, int32, float32).  The kernels and level loop
// of each payload width compile in their own translation unit
// (keys4_v0.cu, keys4_v4.cu, keys4_v8.cu) so that they build in parallel.
#include "layout.cuh"

namespace binar {
int run_call_k4_v0(const Call &c);
int run_call_k4_v4(const Call &c);
int run_call_k4_v8(const Call &c);

int run_call_k4(const Call &c) {
    switch (c.vb) {
    case 0: return run_call_k4_v0(c);
    case 4: return run_call_k4_v4(c);
    case 8: return run_call_k4_v8(c);
    default: return BINAR_ERR_UNSUPPORTED;
    }
}
}  // namespace binar
