// gen.cu -- binar_generate: synthetic keys on the device (SplitMix64), so that
// serving requests and large tests need no host-to-device copies of inputs.
#include "../../include/binar.h"

#include <cstdint>
#include <cuda_runtime.h>

namespace {

// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) used as a counter-based generator:
// value(seed, i) = mix(seed + (i + 1) * golden).
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <int EB>
__global__ void k_generate(void *out, long long n, unsigned long long seed,
                           unsigned long long start) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t v = splitmix64(seed, start + (uint64_t)i);
        if (EB == 4) reinterpret_cast<uint32_t *>(out)[i] = (uint32_t)v;
        else if (EB == 8) reinterpret_cast<uint64_t *>(out)[i] = v;
        else {
            const uint64_t w = splitmix64(seed ^ 0xD1B54A32D192ED03ull, start + (uint64_t)i);
            reinterpret_cast<uint4 *>(out)[i] =
                make_uint4((uint32_t)v, (uint32_t)(v >> 32), (uint32_t)w, (uint32_t)(w >> 32));
        }
    }
}

}  // namespace

extern "C" int binar_generate(void *d_out, int64_t n, int elem_bytes, uint64_t seed, void *stream) {
    if (n < 0 || (n > 0 && !d_out)) return BINAR_ERR_INVALID_ARG;
    if (elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16) return BINAR_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_out) & (uintptr_t)(elem_bytes - 1)) != 0)
        return BINAR_ERR_INVALID_ARG;
    if (n == 0) return BINAR_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    switch (elem_bytes) {
    case 4: k_generate<4><<<(int)blocks, 256, 0, s>>>(d_out, n, seed, 0); break;
    case 8: k_generate<8><<<(int)blocks, 256, 0, s>>>(d_out, n, seed, 0); break;
    default: k_generate<16><<<(int)blocks, 256, 0, s>>>(d_out, n, seed, 0); break;
    }
    return cudaGetLastError() == cudaSuccess ? BINAR_OK : BINAR_ERR_CUDA;
}
