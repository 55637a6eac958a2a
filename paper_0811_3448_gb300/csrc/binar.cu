// binar.cu -- the C ABI of libbinar (include/binar.h): argument checks,
// configuration, workspace sizing, device status and per-kernel profiling.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "layout.cuh"

namespace binar {
int run_call_k4(const Call &c);
int run_call_k8(const Call &c);
int run_call_k16(const Call &c);
int sort_wide(void *keys, void *vals, long long n, int kb, int map, int vb, void *ws,
              const Call &tuning, cudaStream_t st);
size_t wide_workspace_bytes(long long n, int kb, int vb);
size_t strings_workspace_bytes(long long n);
int sort_strings(const void *bytes, const long long *offsets, long long n, long long max_len,
                 uint32_t *order, void *ws, const Call &tuning, cudaStream_t st);

// ---------------------------------------------------------------------------
// Device properties and occupancy, cached per device.
// ---------------------------------------------------------------------------
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
int g_sms[kMaxDevices];

struct OccEntry {
    const void *fn;
    int dev;
    size_t smem;
    int occ;
};
std::vector<OccEntry> g_occ;

bool g_prof_on = false;
struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
};
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_events;   // all events ever created (reused)
size_t g_events_used = 0;
}  // namespace

int device_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_sms[dev] == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
        g_sms[dev] = sms;
    }
    return g_sms[dev];
}

int kernel_ctas_per_sm(const void *fn, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto &e : g_occ)
        if (e.fn == fn && e.dev == dev && e.smem == smem) return e.occ;
    // the opt-in covers static plus dynamic shared memory above 48 KB (a
    // kernel with static arrays can pass the mark with a smaller dynamic part)
    if (smem > 0) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, smem) != cudaSuccess)
        occ = 1;
    cudaGetLastError();
    g_occ.push_back({fn, dev, smem, occ});
    return occ;
}

bool profiling_on() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_prof_on;
}

cudaEvent_t profile_event() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_events_used == g_events.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        g_events.push_back(e);
    }
    return g_events[g_events_used++];
}

void profile_record(const std::string &name, cudaEvent_t a, cudaEvent_t b) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_prof.push_back({name, a, b});
}

}  // namespace binar

using namespace binar;

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
// keys and payloads need their natural alignment (the kernels move whole elements)
bool aligned_to(const void *p, int bytes) {
    return (reinterpret_cast<uintptr_t>(p) & (uintptr_t)(bytes - 1)) == 0;
}

constexpr int kMaxWideKeyBytes = 256;

bool wide(int key_bytes) { return key_bytes > 16; }

// allow_wide: the call accepts keys of 17 .. kMaxWideKeyBytes bytes (the
// unsegmented sorts); the others take 4, 8 or 16.
int check_types(int key_bytes, int map, int val_bytes, bool allow_wide = false) {
    if (key_bytes != 4 && key_bytes != 8 && key_bytes != 16) {
        if (!wide(key_bytes) || key_bytes > kMaxWideKeyBytes) return BINAR_ERR_INVALID_ARG;
        if (!allow_wide) return BINAR_ERR_UNSUPPORTED;
    }
    if (val_bytes != 0 && val_bytes != 4 && val_bytes != 8) return BINAR_ERR_INVALID_ARG;
    if (map < BINAR_MAP_UNSIGNED || map > BINAR_MAP_BYTES_BE) return BINAR_ERR_INVALID_ARG;
    if (map == BINAR_MAP_FLOAT && key_bytes >= 16) return BINAR_ERR_UNSUPPORTED;
    return BINAR_OK;
}

// Resolves a (nullable) config for the key size into the call.
// min_bits: the smallest bits per pass the call accepts (a sort bounds its
// level count by kMinSortBits; a single pass takes any width down to 1).
int resolve_config(const binar_config *cfg, int key_bytes, int val_bytes, Call &c,
                   int min_bits = kMinSortBits, long long n = 0) {
    const int cap = finish_cap_for(key_bytes, val_bytes);
    c.cutoff = default_cutoff(key_bytes, val_bytes, n);
    c.ctas_per_sm = 0;
    c.timeout_ns = 1000000000LL;
    c.skip_publish_tile = -1;
    c.bits = kBits;
    c.tile_variant = 0;
    if (!cfg) return BINAR_OK;
    if (cfg->tile_keys != 0) {
        if (cfg->tile_keys == tile_for(key_bytes, val_bytes, 0)) c.tile_variant = 0;
        else if (cfg->tile_keys == tile_for(key_bytes, val_bytes, 1)) c.tile_variant = 1;
        else return BINAR_ERR_UNSUPPORTED;
    }
    if (cfg->bits_per_pass != 0) {
        if (cfg->bits_per_pass < min_bits || cfg->bits_per_pass > kBits) return BINAR_ERR_UNSUPPORTED;
        c.bits = cfg->bits_per_pass;
    }
    if (cfg->small_cutoff != 0) {
        if (cfg->small_cutoff < kMinCutoff || cfg->small_cutoff > cap) return BINAR_ERR_INVALID_ARG;
        c.cutoff = cfg->small_cutoff;
    }
    if (cfg->ctas_per_sm < 0 || cfg->lookback_timeout_ns < 0) return BINAR_ERR_INVALID_ARG;
    c.ctas_per_sm = cfg->ctas_per_sm;
    if (cfg->lookback_timeout_ns > 0) c.timeout_ns = cfg->lookback_timeout_ns;
    if (cfg->debug_skip_publish_tile > 0) c.skip_publish_tile = cfg->debug_skip_publish_tile - 1;
    return BINAR_OK;
}

int dispatch(const Call &c, int key_bytes) {
    switch (key_bytes) {
    case 4: return run_call_k4(c);
    case 8: return run_call_k8(c);
    case 16: return run_call_k16(c);
    default: return BINAR_ERR_INVALID_ARG;
    }
}

Call blank_call() {
    Call c;
    std::memset(&c, 0, sizeof(c));
    return c;
}

}  // namespace

extern "C" {

int binar_workspace_bytes(int64_t n, int64_t num_segments, int key_bytes, int val_bytes,
                          size_t *out) {
    if (!out || n < 0 || num_segments < 0) return BINAR_ERR_INVALID_ARG;
    if (key_bytes != 4 && key_bytes != 8 && key_bytes != 16 &&
        !(wide(key_bytes) && key_bytes <= kMaxWideKeyBytes))
        return BINAR_ERR_INVALID_ARG;
    if (val_bytes != 0 && val_bytes != 4 && val_bytes != 8) return BINAR_ERR_INVALID_ARG;
    if (wide(key_bytes)) {
        *out = wide_workspace_bytes(n, key_bytes, val_bytes);
        return BINAR_OK;
    }
    *out = make_layout(n, num_segments > 0 ? num_segments : 1, key_bytes, val_bytes).total;
    return BINAR_OK;
}

static int sort_common(void *d_keys, void *d_vals, const int64_t *d_offsets, int64_t num_segments,
                       int64_t n, int key_bytes, binar_key_map map, int val_bytes, void *d_ws,
                       size_t ws_bytes, const binar_config *cfg, void *stream) {
    int rc = check_types(key_bytes, map, val_bytes, d_offsets == nullptr);
    if (rc) return rc;
    if (n < 0) return BINAR_ERR_INVALID_ARG;
    if (!d_offsets && n > BINAR_MAX_BUCKET_KEYS) return BINAR_ERR_UNSUPPORTED;
    if (d_offsets && num_segments < 0) return BINAR_ERR_INVALID_ARG;
    if (n > 0 && (!d_keys || (!wide(key_bytes) && !aligned_to(d_keys, key_bytes))))
        return BINAR_ERR_INVALID_ARG;
    if (val_bytes && n > 0 && (!d_vals || !aligned_to(d_vals, val_bytes))) return BINAR_ERR_INVALID_ARG;
    if (!val_bytes && d_vals) return BINAR_ERR_INVALID_ARG;
    if (!d_ws || !aligned16(d_ws)) return BINAR_ERR_INVALID_ARG;
    const long long segs = d_offsets ? (num_segments > 0 ? num_segments : 1) : 1;
    if (wide(key_bytes)) {
        // keys past 16 bytes: window levels over the 16-byte sort (whose tile,
        // bits and cutoff the config sets)
        if (ws_bytes < wide_workspace_bytes(n, key_bytes, val_bytes))
            return BINAR_ERR_WORKSPACE_TOO_SMALL;
        Call t = blank_call();
        if ((rc = resolve_config(cfg, 16, 4, t, kMinSortBits, n))) return rc;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (n == 0)
            return cudaMemsetAsync(d_ws, 0, sizeof(uint32_t), s) == cudaSuccess ? BINAR_OK
                                                                             : BINAR_ERR_CUDA;
        return sort_wide(d_keys, val_bytes ? d_vals : nullptr, n, key_bytes, map, val_bytes, d_ws,
                         t, s);
    }
    if (ws_bytes < make_layout(n, segs, key_bytes, val_bytes).total)
        return BINAR_ERR_WORKSPACE_TOO_SMALL;
    Call c = blank_call();
    if ((rc = resolve_config(cfg, key_bytes, val_bytes, c, kMinSortBits, n))) return rc;
    if (n == 0 || (d_offsets && num_segments == 0)) {
        // nothing to sort; the status word still reports this call
        if (cudaMemsetAsync(d_ws, 0, sizeof(uint32_t), static_cast<cudaStream_t>(stream)) !=
            cudaSuccess)
            return BINAR_ERR_CUDA;
        return BINAR_OK;
    }
    c.keys = d_keys;
    c.vals = val_bytes ? d_vals : nullptr;
    c.offsets = reinterpret_cast<const long long *>(d_offsets);
    c.num_segments = num_segments;
    c.n = n;
    c.map = map;
    c.vb = val_bytes;
    c.ws = d_ws;
    c.stream = static_cast<cudaStream_t>(stream);
    return dispatch(c, key_bytes);
}

int binar_sort_keys(void *d_keys, int64_t n, int key_bytes, binar_key_map map, void *d_ws,
                    size_t ws_bytes, const binar_config *cfg, void *stream) {
    return sort_common(d_keys, nullptr, nullptr, 1, n, key_bytes, map, 0, d_ws, ws_bytes, cfg,
                       stream);
}

int binar_sort_pairs(void *d_keys, void *d_vals, int64_t n, int key_bytes, binar_key_map map,
                     int val_bytes, void *d_ws, size_t ws_bytes, const binar_config *cfg,
                     void *stream) {
    if (val_bytes == 0) return BINAR_ERR_INVALID_ARG;
    return sort_common(d_keys, d_vals, nullptr, 1, n, key_bytes, map, val_bytes, d_ws, ws_bytes,
                       cfg, stream);
}

int binar_sort_segmented(void *d_keys, void *d_vals, const int64_t *d_offsets,
                         int64_t num_segments, int64_t n, int key_bytes, binar_key_map map,
                         int val_bytes, void *d_ws, size_t ws_bytes, const binar_config *cfg,
                         void *stream) {
    if (!d_offsets) return BINAR_ERR_INVALID_ARG;
    return sort_common(d_keys, d_vals, d_offsets, num_segments, n, key_bytes, map, val_bytes,
                       d_ws, ws_bytes, cfg, stream);
}

int binar_partition_pass(const void *d_keys_in, const void *d_vals_in, void *d_keys_out,
                         void *d_vals_out, int64_t n, int key_bytes, binar_key_map map,
                         int val_bytes, int pos, int bits, int64_t *d_offsets, void *d_ws,
                         size_t ws_bytes, const binar_config *cfg, void *stream) {
    int rc = check_types(key_bytes, map, val_bytes);
    if (rc) return rc;
    if (bits < 0 || bits > kBits) return BINAR_ERR_UNSUPPORTED;
    if (n < 0 || n > BINAR_MAX_BUCKET_KEYS) return BINAR_ERR_INVALID_ARG;
    if (pos < 0 || pos >= 8 * key_bytes) return BINAR_ERR_INVALID_ARG;
    if (n > 0 && (!d_keys_in || !d_keys_out || !aligned_to(d_keys_in, key_bytes) ||
                  !aligned_to(d_keys_out, key_bytes)))
        return BINAR_ERR_INVALID_ARG;
    if (val_bytes && n > 0 &&
        (!d_vals_in || !d_vals_out || !aligned_to(d_vals_in, val_bytes) ||
         !aligned_to(d_vals_out, val_bytes)))
        return BINAR_ERR_INVALID_ARG;
    if (!d_ws || !aligned16(d_ws)) return BINAR_ERR_INVALID_ARG;
    if (ws_bytes < make_layout(n, 1, key_bytes, val_bytes).total)
        return BINAR_ERR_WORKSPACE_TOO_SMALL;
    Call c = blank_call();
    if ((rc = resolve_config(cfg, key_bytes, val_bytes, c, 1))) return rc;
    if (bits != 0) c.bits = bits;
    c.tile_variant = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        if (d_offsets &&
            cudaMemsetAsync(d_offsets, 0, sizeof(int64_t) * ((1 << c.bits) + 1), s) != cudaSuccess)
            return BINAR_ERR_CUDA;
        if (cudaMemsetAsync(d_ws, 0, sizeof(uint32_t), s) != cudaSuccess) return BINAR_ERR_CUDA;
        return BINAR_OK;
    }
    c.pass_mode = true;
    c.keys_in = d_keys_in;
    c.vals_in = val_bytes ? d_vals_in : nullptr;
    c.keys_out = d_keys_out;
    c.vals_out = val_bytes ? d_vals_out : nullptr;
    c.pass_offsets = reinterpret_cast<long long *>(d_offsets);
    c.pass_pos = pos;
    c.n = n;
    c.map = map;
    c.vb = val_bytes;
    c.ws = d_ws;
    c.stream = s;
    return dispatch(c, key_bytes);
}

// Cutoff of an in-place call (the config's, else the finisher's capacity);
// tile and bits per pass are fixed in that mode.
static int inplace_cutoff(const binar_config *cfg, int key_bytes, int val_bytes, long long n,
                          int *cutoff) {
    *cutoff = default_cutoff(key_bytes, val_bytes, n);
    if (!cfg) return BINAR_OK;
    if (cfg->tile_keys != 0 || (cfg->bits_per_pass != 0 && cfg->bits_per_pass != 1))
        return BINAR_ERR_UNSUPPORTED;
    if (cfg->small_cutoff != 0) {
        if (cfg->small_cutoff < kMinCutoff || cfg->small_cutoff > finish_cap_for(key_bytes, val_bytes))
            return BINAR_ERR_INVALID_ARG;
        *cutoff = cfg->small_cutoff;
    }
    if (cfg->ctas_per_sm < 0 || cfg->lookback_timeout_ns < 0) return BINAR_ERR_INVALID_ARG;
    return BINAR_OK;
}

int binar_inplace_workspace_bytes(int64_t n, int key_bytes, int val_bytes, const binar_config *cfg,
                                  size_t *out) {
    if (!out || n < 0 || n > BINAR_MAX_BUCKET_KEYS) return BINAR_ERR_INVALID_ARG;
    int rc = check_types(key_bytes, BINAR_MAP_UNSIGNED, val_bytes);
    if (rc) return rc;
    int cutoff = 0;
    if ((rc = inplace_cutoff(cfg, key_bytes, val_bytes, n, &cutoff))) return rc;
    *out = make_inplace_layout(n, key_bytes, cutoff).end;
    return BINAR_OK;
}

int binar_sort_inplace(void *d_keys, void *d_vals, int64_t n, int key_bytes, binar_key_map map,
                       int val_bytes, void *d_ws, size_t ws_bytes, const binar_config *cfg,
                       void *stream) {
    int rc = check_types(key_bytes, map, val_bytes);
    if (rc) return rc;
    if (n < 0 || n > BINAR_MAX_BUCKET_KEYS) return BINAR_ERR_INVALID_ARG;
    if (n > 0 && (!d_keys || !aligned_to(d_keys, key_bytes))) return BINAR_ERR_INVALID_ARG;
    if (val_bytes && n > 0 && (!d_vals || !aligned_to(d_vals, val_bytes))) return BINAR_ERR_INVALID_ARG;
    if (!val_bytes && d_vals) return BINAR_ERR_INVALID_ARG;
    if (!d_ws || !aligned16(d_ws)) return BINAR_ERR_INVALID_ARG;
    int cutoff = 0;
    if ((rc = inplace_cutoff(cfg, key_bytes, val_bytes, n, &cutoff))) return rc;
    if (ws_bytes < make_inplace_layout(n, key_bytes, cutoff).end) return BINAR_ERR_WORKSPACE_TOO_SMALL;
    Call c = blank_call();
    if ((rc = resolve_config(nullptr, key_bytes, val_bytes, c))) return rc;
    c.cutoff = cutoff;
    if (cfg && cfg->lookback_timeout_ns > 0) c.timeout_ns = cfg->lookback_timeout_ns;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0)
        return cudaMemsetAsync(d_ws, 0, sizeof(uint32_t), s) == cudaSuccess ? BINAR_OK : BINAR_ERR_CUDA;
    c.inplace = true;
    c.keys = d_keys;
    c.vals = val_bytes ? d_vals : nullptr;
    c.n = n;
    c.map = map;
    c.vb = val_bytes;
    c.ws = d_ws;
    c.stream = s;
    return dispatch(c, key_bytes);
}

int binar_strings_workspace_bytes(int64_t n, size_t *out) {
    if (!out || n < 0 || n > BINAR_MAX_BUCKET_KEYS) return BINAR_ERR_INVALID_ARG;
    *out = strings_workspace_bytes(n);
    return BINAR_OK;
}

int binar_sort_strings(const void *d_bytes, const int64_t *d_offsets, int64_t n, int64_t max_len,
                       uint32_t *d_order, void *d_ws, size_t ws_bytes, const binar_config *cfg,
                       void *stream) {
    if (n < 0 || n > BINAR_MAX_BUCKET_KEYS || max_len < 0 || max_len > BINAR_MAX_STRING_BYTES)
        return BINAR_ERR_INVALID_ARG;
    if (n > 0 && (!d_offsets || !d_order || (!d_bytes && max_len > 0)))
        return BINAR_ERR_INVALID_ARG;
    if (!d_ws || !aligned16(d_ws)) return BINAR_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_offsets) & 7) || (reinterpret_cast<uintptr_t>(d_order) & 3))
        return BINAR_ERR_INVALID_ARG;
    if (ws_bytes < strings_workspace_bytes(n)) return BINAR_ERR_WORKSPACE_TOO_SMALL;
    Call t = blank_call();
    int rc = resolve_config(cfg, 16, 4, t, kMinSortBits, n);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0)
        return cudaMemsetAsync(d_ws, 0, sizeof(uint32_t), s) == cudaSuccess ? BINAR_OK : BINAR_ERR_CUDA;
    return sort_strings(d_bytes, reinterpret_cast<const long long *>(d_offsets), n, max_len, d_order,
                        d_ws, t, s);
}

int binar_workspace_status(void *d_ws, void *stream, int *out_status) {
    if (!d_ws || !out_status) return BINAR_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, d_ws, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return BINAR_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BINAR_ERR_CUDA;
    if (cudaMemsetAsync(d_ws, 0, sizeof(v), s) != cudaSuccess) return BINAR_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BINAR_ERR_CUDA;
    *out_status = (int)v;
    return BINAR_OK;
}

const char *binar_status_string(int status) {
    switch (status) {
    case BINAR_OK: return "ok";
    case BINAR_ERR_INVALID_ARG: return "invalid argument";
    case BINAR_ERR_UNSUPPORTED: return "unsupported shape or option";
    case BINAR_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case BINAR_ERR_CUDA: return "CUDA runtime error";
    case BINAR_ERR_DEVICE_TIMEOUT: return "device look-back wait timed out";
    case BINAR_ERR_DEVICE_BOUNDS: return "device index out of bucket bounds";
    case BINAR_ERR_QUEUE_OVERFLOW: return "device work list overflow";
    default: return "unknown status";
    }
}

int binar_profile_start(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_prof.clear();
    g_events_used = 0;
    g_prof_on = true;
    return BINAR_OK;
}

int binar_profile_stop(binar_kernel_stat *out, int cap, int *count) {
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_prof_on = false;
        recs.swap(g_prof);
    }
    std::vector<binar_kernel_stat> stats;
    int rc = BINAR_OK;
    for (const auto &r : recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) {
            rc = BINAR_ERR_CUDA;
            continue;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            rc = BINAR_ERR_CUDA;
            continue;
        }
        binar_kernel_stat *hit = nullptr;
        for (auto &s : stats)
            if (r.name == s.name) hit = &s;
        if (!hit) {
            binar_kernel_stat s;
            std::memset(&s, 0, sizeof(s));
            std::strncpy(s.name, r.name.c_str(), sizeof(s.name) - 1);
            stats.push_back(s);
            hit = &stats.back();
        }
        hit->launches += 1;
        hit->total_ms += ms;
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_events_used = 0;
    }
    const int nout = (int)stats.size() < cap ? (int)stats.size() : cap;
    for (int i = 0; i < nout; i++) out[i] = stats[i];
    if (count) *count = (int)stats.size();
    return rc;
}

const char *binar_version(void) { return "0.1.0"; }

}  // extern "C"
