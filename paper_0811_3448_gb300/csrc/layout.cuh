// layout.cuh -- host-side declarations shared by the C ABI (binar.cu) and the
// per-key-width level loops (keys*.cu): workspace layout, the description of
// one call, profiling hooks.
#pragma once

#include <string>
#include <utility>

#include "binar_internal.cuh"

namespace binar {

// ---------------------------------------------------------------------------
// Host utilities implemented in binar.cu.
// ---------------------------------------------------------------------------
int device_sms();                                            // SMs of the current device
int kernel_ctas_per_sm(const void *fn, size_t smem);         // occupancy (cached per device)
bool profiling_on();
void profile_record(const std::string &name, cudaEvent_t a, cudaEvent_t b);
cudaEvent_t profile_event();

// Enqueues kernel<<<grid, block, smem, s>>>(args...) with programmatic stream
// serialization: the kernel may be scheduled while its predecessor in the
// stream drains, and waits for it with griddepcontrol.wait (pdl_entry) before
// touching memory.  This hides most of the launch latency between the
// dependent kernels of a call.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Launches `f` (which enqueues one kernel) bracketed by profiling events.
template <typename F>
int launch(const char *name, int index, cudaStream_t s, F &&f) {
    cudaEvent_t a = nullptr, b = nullptr;
    const bool prof = profiling_on();
    if (prof) {
        a = profile_event();
        cudaEventRecord(a, s);
    }
    f();
    if (cudaGetLastError() != cudaSuccess) return BINAR_ERR_CUDA;
    if (prof) {
        b = profile_event();
        cudaEventRecord(b, s);
        std::string nm(name);
        if (index >= 0) nm += "[" + std::to_string(index) + "]";
        profile_record(nm, a, b);
    }
    return BINAR_OK;
}

// ---------------------------------------------------------------------------
// Workspace layout.  Capacities are upper bounds for every configuration with
// a finisher cutoff of at least kMinCutoff:
//   buckets per level  <= n / (kMinCutoff + 1) + segments + 2  (live buckets exceed the cutoff)
//   tiles per level    <= n / tile + buckets                   (one ragged tile per bucket)
//   finisher jobs      <= levels * (19 n / kMinCutoff + 2 * buckets) + segments
//   copy jobs          <= levels * (n / kMinCutoff + buckets)
// ---------------------------------------------------------------------------
constexpr int kMinCutoff = 2048;

// keys per partition tile of tile variant tv (kernels.cuh PartShape), and the
// finisher's largest job (= the largest cutoff)
inline int tile_for(int kb, int vb, int tv = 0) {
    if (tv == 1) return kb == 4 ? 4096 : (kb == 8 ? 2048 : 1024);
    return kb == 4 ? (vb == 0 ? 7168 : 6144) : (kb == 8 ? 4096 : 2048);
}
inline int min_tile_for(int kb, int vb) {
    const int a = tile_for(kb, vb, 0), b = tile_for(kb, vb, 1);
    return a < b ? a : b;
}
// (kernels.cuh TileShape): 8192 / 4096 / 2048 keys for 4 / 8 / 16-byte keys
inline int finish_cap_for(int kb, int vb) {
    (void)vb;
    return kb == 4 ? 8192 : (kb == 8 ? 4096 : 2048);
}
// The cutoff of a call that sets none: the capacity, except for 4-byte keys
// in calls of at most 2^21 keys, whose sorts are latency-bound and ran faster
// with smaller jobs (a smaller finisher class: more CTAs per SM, fewer idle
// items): uniform uint32 keys, 64K: 84 -> 80 us, 256K: 86 -> 73 us, 2M: 160
// -> 149 us; 1M about equal.
inline int default_cutoff(int kb, int vb, long long n) {
    if (kb == 4 && n <= (1LL << 21)) {
        if (n <= (1LL << 17)) return 4096;
        if (n <= (3LL << 19)) return 6144;
        return 3072;
    }
    return finish_cap_for(kb, vb);
}
// partition levels of a sort that consumes `bits` key bits per pass
inline int levels_for(int kb, int bits = kBits) { return (8 * kb + bits - 1) / bits; }

struct Layout {
    size_t ctr, altk, altv, list[2], hist[2], andor[2], order[2], tilemap, cells, jobs, jobidx, jobs2, copies, total;
    uint32_t mcap, tcap, jcap, ccap;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline Layout make_layout(long long n, long long segs, int kb, int vb) {
    Layout L{};
    // capacities cover every tile variant and every bits per pass a sort accepts
    const long long T = min_tile_for(kb, vb), lv = levels_for(kb, kMinSortBits);
    const long long m = n / (kMinCutoff + 1) + segs + 2;
    const long long t = n / T + m + 2;
    // jobs of a level: own jobs (>= C/8 keys) and merged runs (two adjacent
    // runs hold > C keys) give 19n/C; every parent adds at most 2 around its
    // large children and 8 at its digit-group boundaries
    long long j = lv * (19 * (n / kMinCutoff) + 10 * m) + segs + 2;
    if (j > n + 2) j = n + 2;
    const long long c = lv * (n / kMinCutoff + m) + 2;
    L.mcap = (uint32_t)m;
    L.tcap = (uint32_t)t;
    L.jcap = (uint32_t)j;
    L.ccap = (uint32_t)c;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.ctr = take(sizeof(Counters));
    L.altk = take((size_t)n * kb);
    L.altv = take((size_t)n * vb);
    for (int s = 0; s < 2; s++) {
        L.list[s] = take((size_t)m * sizeof(Bucket));
        L.hist[s] = take((size_t)m * kRadix * sizeof(uint32_t));
        L.andor[s] = take((size_t)m * 2 * sizeof(uint4));
        L.order[s] = take((size_t)m * sizeof(uint32_t));
    }
    L.tilemap = take((size_t)t * sizeof(uint32_t));
    L.cells = take((size_t)t * kRadix * sizeof(uint32_t));
    L.jobs = take((size_t)j * sizeof(Job));
    L.jobidx = take((size_t)job_region(kMaxClasses, n, (unsigned long long)j) * sizeof(uint32_t));
    L.jobs2 = take((size_t)j * sizeof(Job));
    L.copies = take((size_t)c * sizeof(CopyJob));
    L.total = o;
    return L;
}

// Workspace of the in-place mode (1-bit exchange passes, kIpTile-key tiles):
// no second key / payload array and no look-back cells; per tile one marker
// bit per key, four counters and its first position and split point.  Capacities for the call's cutoff C: buckets
// of a level are disjoint and hold more than C keys; every bucket of every
// level yields at most two finisher jobs; reversed (copied) buckets are
// disjoint and larger than C.
struct InplaceLayout {
    Layout base;
    size_t mask, cnt, pre, bsum, total, first, tinfo, end;
    long long chunks;              // swap chunks per side (first[] entries per side)
};

inline InplaceLayout make_inplace_layout(long long n, int kb, int cutoff) {
    constexpr long long T = 4096;                 // kIpTile
    InplaceLayout L{};
    const long long lv = 8LL * kb;                // one bit per level
    const long long m = n / ((long long)cutoff + 1) + 2;
    const long long t = n / T + m + 2;
    long long j = 2 * lv * m + 2;
    if (j > n / 2 + 2) j = n / 2 + 2;
    const long long c = n / ((long long)cutoff + 1) + 2;
    Layout &B = L.base;
    B.mcap = (uint32_t)m;
    B.tcap = (uint32_t)t;
    B.jcap = (uint32_t)j;
    B.ccap = (uint32_t)c;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    B.ctr = take(sizeof(Counters));
    B.altk = take(0);
    B.altv = take(0);
    for (int s = 0; s < 2; s++) {
        B.list[s] = take((size_t)m * sizeof(Bucket));
        B.hist[s] = take((size_t)m * kRadix * sizeof(uint32_t));
        B.andor[s] = take((size_t)m * 2 * sizeof(uint4));
        B.order[s] = take((size_t)m * sizeof(uint32_t));
    }
    B.tilemap = take((size_t)t * sizeof(uint32_t));
    B.cells = take(0);
    B.jobs = take((size_t)j * sizeof(Job));
    B.jobidx = take((size_t)job_region(kMaxClasses, n, (unsigned long long)j) * sizeof(uint32_t));
    B.jobs2 = take((size_t)j * sizeof(Job));
    B.copies = take((size_t)c * sizeof(CopyJob));
    L.mask = take((size_t)t * (T / 32) * 4);
    L.cnt = take((size_t)t * 8);
    L.pre = take((size_t)t * 8);
    L.bsum = take((size_t)(t / (256 * 8) + 2) * 8);
    L.total = take(16);
    L.chunks = n / (2 * kIpChunk) + 2;            // kIpChunk ranks per chunk; misplaced <= n / 2
    L.first = take((size_t)L.chunks * 2 * 4);
    L.tinfo = take((size_t)t * 16);
    B.total = o;
    L.end = o;
    return L;
}

inline Ws carve(const Layout &L, void *base) {
    unsigned char *b = static_cast<unsigned char *>(base);
    Ws ws{};
    ws.ctr = reinterpret_cast<Counters *>(b + L.ctr);
    ws.alt_keys = b + L.altk;
    ws.alt_vals = b + L.altv;
    for (int s = 0; s < 2; s++) {
        ws.list[s] = reinterpret_cast<Bucket *>(b + L.list[s]);
        ws.hist[s] = reinterpret_cast<uint32_t *>(b + L.hist[s]);
        ws.andor[s] = reinterpret_cast<uint4 *>(b + L.andor[s]);
        ws.order[s] = reinterpret_cast<uint32_t *>(b + L.order[s]);
    }
    ws.tilemap = reinterpret_cast<uint32_t *>(b + L.tilemap);
    ws.cells = reinterpret_cast<uint32_t *>(b + L.cells);
    ws.jobs = reinterpret_cast<Job *>(b + L.jobs);
    ws.jobidx = reinterpret_cast<uint32_t *>(b + L.jobidx);
    ws.jobs2 = reinterpret_cast<Job *>(b + L.jobs2);
    ws.copies = reinterpret_cast<CopyJob *>(b + L.copies);
    ws.mcap = L.mcap;
    ws.tcap = L.tcap;
    ws.jcap = L.jcap;
    ws.ccap = L.ccap;
    return ws;
}

// ---------------------------------------------------------------------------
// One call.
// ---------------------------------------------------------------------------
struct Call {
    // sort mode: keys/vals are sorted in place; pass mode: in -> out
    void *keys, *vals;
    const void *keys_in, *vals_in;
    void *keys_out, *vals_out;
    long long *pass_offsets;
    int pass_pos;
    bool pass_mode;
    const Layout *layout;          // workspace layout to use instead of make_layout(), or nullptr
    const long long *offsets;      // segmented: device offsets, else nullptr
    long long num_segments;        // segmented: segments (an upper bound if num_segments_dev is set)
    const long long *num_segments_dev;   // segmented: device-side segment count, or nullptr
    long long n;
    int map, vb;
    int cutoff;
    int bits;                      // key bits per partition pass
    int tile_variant;              // 0 or 1 (PartShape TV)
    bool inplace;                  // unstable in-place mode (1-bit exchange passes)
    int ctas_per_sm;
    long long timeout_ns;
    int skip_publish_tile;
    void *ws;
    cudaStream_t stream;
};

}  // namespace binar
