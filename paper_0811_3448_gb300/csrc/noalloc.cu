// noalloc.cu -- binar_partition_pass_noalloc: the partition pass with its
// scratch memory in a fixed array inside the library, for callers that must
// not be asked for (or cause) any device allocation.
//
// Who cannot allocate: code that hands the library only the buffers it
// already owns -- for example a pipeline whose device memory is carved up
// front from one pool with a hard budget, or a real-time loop that must not
// pay for (or synchronise on) cudaMalloc -- and callers that cannot size and
// keep a workspace of their own.  This entry point takes only the inputs and
// outputs; its scratch lives in kScratchBytes of device memory declared here.
#include <atomic>
#include <cstring>
#include <mutex>

#include "layout.cuh"

namespace binar {
int run_call_k4(const Call &c);
int run_call_k8(const Call &c);
int run_call_k16(const Call &c);
}  // namespace binar

using namespace binar;

namespace {

// 4 MiB per GPU that loads the library, held until the process exits.  It
// covers the look-back cells, tile map, histograms and counters of one pass
// over up to 29,173,759 keys of 4 bytes alone, 25,006,079 of 4 bytes with a
// payload, 16,670,719 of 8 bytes or 8,335,359 of 16 bytes (one 1 KB cell row
// per tile of 7168 / 6144 / 4096 / 2048 keys).
constexpr size_t kScratchBytes = 4u << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevs = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevs];

// Device address of the scratch array on the current device.  The name of a
// __device__ array in host code is a host-side stand-in, not a device address,
// so the address is looked up once per device (with that device current).
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevs) return BINAR_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return BINAR_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return BINAR_OK;
}

// The pass needs the counters, one bucket slot, histograms, the tile map and
// the look-back cells -- not the ping-pong buffers or the finisher lists.
Layout pass_layout(long long n, int kb, int vb) {
    Layout L{};
    const long long T = tile_for(kb, vb);
    const long long m = 3;
    const long long t = n / T + 2;
    L.mcap = (uint32_t)m;
    L.tcap = (uint32_t)t;
    L.jcap = 1;
    L.ccap = 1;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.ctr = take(sizeof(Counters));
    L.altk = take(0);
    L.altv = take(0);
    for (int s = 0; s < 2; s++) {
        L.list[s] = take((size_t)m * sizeof(Bucket));
        L.hist[s] = take((size_t)m * kRadix * sizeof(uint32_t));
        L.andor[s] = take((size_t)m * 2 * sizeof(uint4));
        L.order[s] = take((size_t)m * sizeof(uint32_t));
    }
    L.tilemap = take((size_t)t * sizeof(uint32_t));
    L.cells = take((size_t)t * kRadix * sizeof(uint32_t));
    L.jobs = take(sizeof(Job));
    L.jobidx = take(sizeof(uint32_t));
    L.jobs2 = take(sizeof(Job));
    L.copies = take(sizeof(CopyJob));
    L.total = o;
    return L;
}

// Test hook (binar_partition_pass_noalloc_debug): a level-0 tile that never
// publishes (-1 = none) and the look-back limit (0 = 1 s) of the calls that
// follow.
std::atomic<int> g_skip_publish_tile{-1};
std::atomic<long long> g_timeout_ns{0};

bool aligned_to(const void *p, int bytes) {
    return (reinterpret_cast<uintptr_t>(p) & (uintptr_t)(bytes - 1)) == 0;
}

}  // namespace

extern "C" int binar_partition_pass_noalloc(const void *d_keys_in, const void *d_vals_in,
                                            void *d_keys_out, void *d_vals_out, int64_t n,
                                            int key_bytes, binar_key_map map, int val_bytes,
                                            int pos, int bits, int64_t *d_offsets, void *stream) {
    if (key_bytes != 4 && key_bytes != 8 && key_bytes != 16) return BINAR_ERR_INVALID_ARG;
    if (val_bytes != 0 && val_bytes != 4 && val_bytes != 8) return BINAR_ERR_INVALID_ARG;
    if (map < BINAR_MAP_UNSIGNED || map > BINAR_MAP_BYTES_BE) return BINAR_ERR_INVALID_ARG;
    if (map == BINAR_MAP_FLOAT && key_bytes == 16) return BINAR_ERR_UNSUPPORTED;
    if (bits < 0 || bits > kBits) return BINAR_ERR_UNSUPPORTED;
    if (n < 0 || pos < 0 || pos >= 8 * key_bytes) return BINAR_ERR_INVALID_ARG;
    if (n > 0 && (!d_keys_in || !d_keys_out || !aligned_to(d_keys_in, key_bytes) ||
                  !aligned_to(d_keys_out, key_bytes)))
        return BINAR_ERR_INVALID_ARG;
    if (val_bytes && n > 0 &&
        (!d_vals_in || !d_vals_out || !aligned_to(d_vals_in, val_bytes) ||
         !aligned_to(d_vals_out, val_bytes)))
        return BINAR_ERR_INVALID_ARG;
    const Layout lay = pass_layout(n, key_bytes, val_bytes);
    if (lay.total > kScratchBytes) return BINAR_ERR_WORKSPACE_TOO_SMALL;   // n above the limit
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        if (d_offsets &&
            cudaMemsetAsync(d_offsets, 0, sizeof(int64_t) * ((1 << (bits ? bits : kBits)) + 1),
                            s) != cudaSuccess)
            return BINAR_ERR_CUDA;
        return BINAR_OK;
    }
    Call c;
    std::memset(&c, 0, sizeof(c));
    c.cutoff = finish_cap_for(key_bytes, val_bytes);
    c.bits = bits ? bits : kBits;
    c.tile_variant = 0;
    const long long limit = g_timeout_ns.load();
    c.timeout_ns = limit > 0 ? limit : 1000000000LL;
    c.skip_publish_tile = g_skip_publish_tile.load();
    c.pass_mode = true;
    c.layout = &lay;
    c.keys_in = d_keys_in;
    c.vals_in = val_bytes ? d_vals_in : nullptr;
    c.keys_out = d_keys_out;
    c.vals_out = val_bytes ? d_vals_out : nullptr;
    c.pass_offsets = reinterpret_cast<long long *>(d_offsets);
    c.pass_pos = pos;
    c.n = n;
    c.map = map;
    c.vb = val_bytes;
    c.ws = scratch;
    c.stream = s;
    switch (key_bytes) {
    case 4: return run_call_k4(c);
    case 8: return run_call_k8(c);
    default: return run_call_k16(c);
    }
}

// The first word of the scratch array is the status word of the pass (the
// Counters header sits at offset 0 of the layout): read it after the
// caller's stream has drained, then clear it.  Copies to and from a host
// variable; nothing is allocated.
extern "C" int binar_partition_pass_noalloc_status(void *stream, int *out_status) {
    if (!out_status) return BINAR_ERR_INVALID_ARG;
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, scratch, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return BINAR_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BINAR_ERR_CUDA;
    const uint32_t zero = 0;
    if (cudaMemcpyAsync(scratch, &zero, sizeof(zero), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return BINAR_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BINAR_ERR_CUDA;
    *out_status = (int)v;
    return BINAR_OK;
}

extern "C" int binar_partition_pass_noalloc_debug(int skip_publish_tile, int64_t lookback_timeout_ns) {
    if (skip_publish_tile < 0 || lookback_timeout_ns < 0) return BINAR_ERR_INVALID_ARG;
    g_skip_publish_tile.store(skip_publish_tile - 1);
    g_timeout_ns.store(lookback_timeout_ns);
    return BINAR_OK;
}
