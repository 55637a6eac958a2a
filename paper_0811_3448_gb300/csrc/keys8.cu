// Dispatch by payload width for 8-byte keys (uint64, int64, float64).  The kernels and level loop
// of each payload width compile in their own translation unit
// (keys8_v0.cu, keys8_v4.cu, keys8_v8.cu) so that they build in parallel.
#include "layout.cuh"

namespace binar {
int run_call_k8_v0(const Call &c);
int run_call_k8_v4(const Call &c);
int run_call_k8_v8(const Call &c);

int run_call_k8(const Call &c) {
    switch (c.vb) {
    case 0: return run_call_k8_v0(c);
    case 4: return run_call_k8_v4(c);
    case 8: return run_call_k8_v8(c);
    default: return BINAR_ERR_UNSUPPORTED;
    }
}
}  // namespace binar
