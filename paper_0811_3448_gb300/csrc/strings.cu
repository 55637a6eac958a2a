// strings.cu -- keys longer than 16 bytes and byte strings of different
// lengths: the MSD recursion of binar sort carried past 128 bits.
//
// The paper sorts any data by the bits of its encoding, strings included, at
// a cost set by their average length ("The Other Universal Property",
// "Recursion Analysis").  Here a string is read in windows of 15 bytes; the
// window key of string s at level w is 16 bytes, compared as a big-endian bit
// string:
//
//     bytes 15w .. 15w+14 of s (zero past the end of s) | min(max(len - 15w, 0), 15)
//
// Ordering strings by their window keys, level after level, is the
// lexicographic order with a proper prefix first: the data bytes decide where
// they differ, and where they agree the last byte (the length left, clamped)
// puts the string that ends first before the one that goes on.  Two strings
// whose window keys agree with a length byte below 15 are equal.
//
// Level w sorts, stably, only the records still tied after levels 0 .. w-1
// (the "active" records) by their window key, inside the runs they are tied
// in (each run a segment of the existing 16-byte segmented sort).  After the
// sort every active record's output position is final unless it sits in a run
// of at least two equal window keys whose length byte is 15; only those runs
// go on to level w+1, compacted into new segments.  A run that leaves the
// active set skips every later window: the recursion stops per sub-array as
// soon as its keys differ or end (the base cases of "Evaluate for Recursive
// Base Case"), however long the common prefix of the rest.
//
// Every kernel reads its element counts from device memory, so a sort is one
// fixed sequence of launches on the caller's stream: nothing allocates or
// synchronises.
#include <cstring>

#include "kernels.cuh"
#include "layout.cuh"

namespace binar {
int run_call_k16(const Call &c);

namespace {

constexpr int kWin = 15;                 // data bytes per window key
constexpr int kScanItems = 8;            // run-marker scan: items per thread
constexpr int kScanTile = kThreads * kScanItems;
constexpr uint32_t kNoRun = 0xffffffffu;
constexpr unsigned long long kSlotMask = 0xffffffffull;   // slots < 2^32, segments above

// Where the strings are: variable-length strings (bytes + offsets) or n
// fixed-width keys of `width` bytes read as big-endian byte strings after the
// key map (unsigned / signed little-endian integers are read from their last
// byte; the sign bit of a signed key is inverted).
struct StrSrc {
    const unsigned char *bytes;
    const long long *offsets;    // n + 1, or nullptr for fixed-width keys
    int width;                   // fixed-width keys: bytes per key
    int map;                     // fixed-width keys: binar_key_map
};

// Device counters of the string levels (one 256-byte aligned header at the
// start of the workspace; status is the word binar_workspace_status reads).
struct StrCtr {
    uint32_t status;
    uint32_t pad;
    long long nact[2];           // active records of the current / next level
    long long nseg[2];           // segments (tied runs) of the current / next level
    unsigned long long alloc;    // next level: (segments << 32) | slots
    long long nruns;             // runs found at this level
};

struct StrWs {
    StrCtr *ctr;
    uint32_t *ord[2];            // active slot -> string index
    uint32_t *gpos[2];           // active slot -> output position
    long long *segoff[2];        // segment offsets into the active slots (nseg + 1)
    uint4 *key;                  // window keys of the active slots
    uint32_t *mark;              // run-start markers, then run index per slot
    uint32_t *bsum;              // per scan tile: run starts, then their exclusive prefix
    uint32_t *rstart;            // first slot of each run
    uint32_t *rbase;             // each run's first slot at the next level, or kNoRun
    void *inner;                 // workspace of the 16-byte segmented sort
    size_t inner_bytes;
};

struct StrLayout {
    size_t ctr, ord[2], gpos[2], segoff[2], key, mark, bsum, rstart, rbase, inner, total;
    size_t inner_bytes;
    Layout inner_layout;
};

StrLayout str_layout(long long n) {
    StrLayout L{};
    const long long segs = n / 2 + 2;    // tied runs hold at least two records
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.ctr = take(sizeof(StrCtr));
    for (int s = 0; s < 2; s++) {
        L.ord[s] = take((size_t)n * 4);
        L.gpos[s] = take((size_t)n * 4);
        L.segoff[s] = take((size_t)(segs + 1) * 8);
    }
    L.key = take((size_t)n * 16);
    L.mark = take((size_t)n * 4 + 4);
    L.bsum = take((size_t)(n / kScanTile + 2) * 4);
    L.rstart = take((size_t)(n + 1) * 4);
    L.rbase = take((size_t)(n + 1) * 4);
    L.inner_layout = make_layout(n, segs, 16, 4);
    L.inner_bytes = L.inner_layout.total;
    L.inner = take(L.inner_bytes);
    L.total = o;
    return L;
}

StrWs str_carve(const StrLayout &L, void *base) {
    unsigned char *b = static_cast<unsigned char *>(base);
    StrWs w{};
    w.ctr = reinterpret_cast<StrCtr *>(b + L.ctr);
    for (int s = 0; s < 2; s++) {
        w.ord[s] = reinterpret_cast<uint32_t *>(b + L.ord[s]);
        w.gpos[s] = reinterpret_cast<uint32_t *>(b + L.gpos[s]);
        w.segoff[s] = reinterpret_cast<long long *>(b + L.segoff[s]);
    }
    w.key = reinterpret_cast<uint4 *>(b + L.key);
    w.mark = reinterpret_cast<uint32_t *>(b + L.mark);
    w.bsum = reinterpret_cast<uint32_t *>(b + L.bsum);
    w.rstart = reinterpret_cast<uint32_t *>(b + L.rstart);
    w.rbase = reinterpret_cast<uint32_t *>(b + L.rbase);
    w.inner = b + L.inner;
    w.inner_bytes = L.inner_bytes;
    return w;
}

__device__ __forceinline__ void str_status(StrCtr *c, uint32_t code) {
    atomicCAS(&c->status, 0u, code);
}

// Byte j (0 = most significant) of string s and its length.
__device__ __forceinline__ long long str_len(const StrSrc &src, uint32_t s) {
    return src.offsets ? src.offsets[s + 1] - src.offsets[s] : (long long)src.width;
}
__device__ __forceinline__ uint32_t str_byte(const StrSrc &src, uint32_t s, long long j) {
    if (src.offsets) return src.bytes[src.offsets[s] + j];
    const unsigned char *k = src.bytes + (size_t)s * src.width;
    if (src.map == BINAR_MAP_BYTES_BE) return k[j];
    const uint32_t x = k[src.width - 1 - j];                // little-endian integer
    return (src.map == BINAR_MAP_SIGNED && j == 0) ? x ^ 0x80u : x;
}

// level 0: every record active, in input order, in the caller's segments
// (one segment [0, n) here); strings longer than max_len are an error.
__global__ void k_str_init(StrWs w, StrSrc src, long long n, long long max_len) {
    pdl_entry();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        w.ord[0][i] = (uint32_t)i;
        w.gpos[0][i] = (uint32_t)i;
        const long long len = str_len(src, (uint32_t)i);
        if (len < 0 || len > max_len) str_status(w.ctr, BINAR_ERR_INVALID_ARG);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        w.ctr->nact[0] = n;
        w.ctr->nseg[0] = 1;
        w.ctr->nact[1] = 0;
        w.ctr->nseg[1] = 0;
        w.ctr->alloc = 0;
        w.segoff[0][0] = 0;
        w.segoff[0][1] = n;
    }
}

// The window key of every active slot at level `lvl`: 15 data bytes from
// byte 15 * lvl on (zero past the end), then the clamped length left.
__global__ void k_str_window(StrWs w, StrSrc src, int cur, int lvl) {
    pdl_entry();
    const long long nact = w.ctr->nact[cur];
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long first = (long long)lvl * kWin;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nact; i += stride) {
        const uint32_t s = w.ord[cur][i];
        const long long len = str_len(src, s);
        long long left = len - first;
        left = left < 0 ? 0 : (left > kWin ? kWin : left);
        uint32_t b[16];
#pragma unroll
        for (int j = 0; j < kWin; j++) b[j] = j < left ? str_byte(src, s, first + j) : 0u;
        b[15] = (uint32_t)left;
        uint4 v;
        v.x = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
        v.y = b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24);
        v.z = b[8] | (b[9] << 8) | (b[10] << 16) | (b[11] << 24);
        v.w = b[12] | (b[13] << 8) | (b[14] << 16) | (b[15] << 24);
        w.key[i] = v;
    }
}

// After the level's sort: every active record's output position gets its
// string (final unless its run goes on); the inner sort's device status joins
// this call's; a slot is marked as a run start when its window key differs
// from the slot before it.
__global__ void k_str_emit(StrWs w, uint32_t *order, int cur) {
    pdl_entry();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t inner = *reinterpret_cast<const uint32_t *>(w.inner);
        if (inner) str_status(w.ctr, inner);
    }
    const long long nact = w.ctr->nact[cur];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nact; i += stride) {
        order[w.gpos[cur][i]] = w.ord[cur][i];
        const uint4 a = w.key[i];
        bool start = i == 0;
        if (!start) {
            const uint4 b = w.key[i - 1];
            start = a.x != b.x || a.y != b.y || a.z != b.z || a.w != b.w;
        }
        w.mark[i] = start ? 1u : 0u;
    }
}

// Every segment's first slot starts a run (equal keys in different segments
// are different runs).
__global__ void k_str_segstarts(StrWs w, int cur) {
    pdl_entry();
    const long long ns = w.ctr->nseg[cur], nact = w.ctr->nact[cur];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < ns; g += stride) {
        const long long at = w.segoff[cur][g];
        if (at >= 0 && at < nact) w.mark[at] = 1u;
    }
}

// Run numbering by an exclusive scan of the markers, in three passes over
// tiles of kScanTile slots: per-tile counts, one CTA scanning the counts, and
// per slot its run index (and the run's first slot).
__global__ void __launch_bounds__(kThreads) k_str_scan_count(StrWs w, int cur) {
    pdl_entry();
    __shared__ uint32_t red[kWarps];
    const long long nact = w.ctr->nact[cur];
    const long long ntiles = (nact + kScanTile - 1) / kScanTile;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const long long i = t * kScanTile + (long long)k * kThreads + threadIdx.x;
            if (i < nact) c += w.mark[i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t sum = 0;
            for (int i = 0; i < kWarps; i++) sum += red[i];
            w.bsum[t] = sum;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) k_str_scan_tiles(StrWs w, int cur) {
    pdl_entry();
    __shared__ uint32_t scratch[kWarps];
    const long long nact = w.ctr->nact[cur];
    const long long ntiles = (nact + kScanTile - 1) / kScanTile;
    uint32_t carry = 0;
    for (long long base = 0; base < ntiles; base += kThreads) {
        const long long t = base + threadIdx.x;
        const uint32_t v = t < ntiles ? w.bsum[t] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, scratch, &total);
        if (t < ntiles) w.bsum[t] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) w.ctr->nruns = carry;
}

__global__ void __launch_bounds__(kThreads) k_str_scan_apply(StrWs w, int cur) {
    pdl_entry();
    __shared__ uint32_t scratch[kWarps];
    const long long nact = w.ctr->nact[cur];
    const long long ntiles = (nact + kScanTile - 1) / kScanTile;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        // thread-contiguous items within the tile keep the scan in slot order
        const long long i0 = t * kScanTile + (long long)threadIdx.x * kScanItems;
        uint32_t m[kScanItems], c = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            m[k] = (i0 + k < nact) ? w.mark[i0 + k] : 0u;
            c += m[k];
        }
        uint32_t total;
        uint32_t run = w.bsum[t] + block_exclusive_scan(c, scratch, &total);
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const long long i = i0 + k;
            if (i < nact) {
                run += m[k];
                const uint32_t r = run - 1;          // run index of slot i
                if (m[k]) w.rstart[r] = (uint32_t)i;
                w.mark[i] = r;
            }
        }
    }
}

// Per run: a run of at least two equal window keys whose strings go on past
// this window (length byte 15) becomes a segment of the next level; its slots
// and its segment number come from one 64-bit counter (segments in the high
// half, slots in the low half: the slots of one level sum to at most n <
// 2^32), so segment offsets grow with the segment number.
__global__ void k_str_runs(StrWs w, int cur, int nxt) {
    pdl_entry();
    const long long nact = w.ctr->nact[cur], nruns = w.ctr->nruns;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nruns; r += stride) {
        const long long a = w.rstart[r];
        const long long b = r + 1 < nruns ? (long long)w.rstart[r + 1] : nact;
        const long long len = b - a;
        const bool goes_on = len >= 2 && (w.key[a].w >> 24) == (uint32_t)kWin;
        uint32_t base = kNoRun;
        if (goes_on) {
            const unsigned long long got =
                atomicAdd(&w.ctr->alloc, (1ull << 32) | (unsigned long long)len);
            base = (uint32_t)(got & kSlotMask);
            w.segoff[nxt][got >> 32] = (long long)(got & kSlotMask);
        }
        w.rbase[r] = base;
    }
}

// The slots of the runs that go on move, in order, to the next level.
__global__ void k_str_compact(StrWs w, int cur, int nxt) {
    pdl_entry();
    const long long nact = w.ctr->nact[cur];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nact; i += stride) {
        const uint32_t r = w.mark[i];
        const uint32_t base = w.rbase[r];
        if (base != kNoRun) {
            const long long j = (long long)base + (i - (long long)w.rstart[r]);
            w.ord[nxt][j] = w.ord[cur][i];
            w.gpos[nxt][j] = w.gpos[cur][i];
        }
    }
}

// Closes the level: the next level's counts and last segment offset.  After
// the last window no run can go on unless a string was longer than max_len.
__global__ void k_str_close(StrWs w, int nxt, int last) {
    pdl_entry();
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const unsigned long long a = w.ctr->alloc;
    const long long ns = (long long)(a >> 32), nact = (long long)(a & kSlotMask);
    w.ctr->nseg[nxt] = ns;
    w.ctr->nact[nxt] = nact;
    w.segoff[nxt][ns] = nact;
    w.ctr->alloc = 0;
    w.ctr->nseg[nxt ^ 1] = 0;
    w.ctr->nact[nxt ^ 1] = 0;
    if (last && ns > 0) str_status(w.ctr, BINAR_ERR_INVALID_ARG);
}

// Moves records into the sorted order: dst[i] = src[order[i]] for elements of
// `width` bytes (16-byte vectors when the width and both arrays allow).
__global__ void k_str_gather(const unsigned char *src, unsigned char *dst, const uint32_t *order,
                             long long n, int width) {
    pdl_entry();
    const long long stride = (long long)gridDim.x * blockDim.x;
    const bool vec = (width % 16) == 0 && ((reinterpret_cast<uintptr_t>(src) |
                                           reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    const int per = vec ? width / 16 : width;
    const long long total = n * per;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const long long i = e / per;
        const int part = (int)(e - i * per);
        const uint32_t s = order[i];
        if (vec)
            reinterpret_cast<uint4 *>(dst + i * width)[part] =
                reinterpret_cast<const uint4 *>(src + (size_t)s * width)[part];
        else
            dst[i * width + part] = src[(size_t)s * width + part];
    }
}

// Workspace of a sort of n keys wider than 16 bytes: the string levels, the
// permutation and one buffer for moving keys (and then payloads) into order.
struct WideLayout {
    StrLayout str;
    size_t order, tmp, total;
};

WideLayout wide_layout(long long n, int kb, int vb) {
    WideLayout L{};
    L.str = str_layout(n);
    L.order = align_up(L.str.total, 256);
    L.tmp = align_up(L.order + (size_t)n * 4, 256);
    const int eb = kb > vb ? kb : vb;
    L.total = align_up(L.tmp + (size_t)n * eb, 256);
    return L;
}

int ceil_grid(long long work, int cap) {
    long long g = (work + kThreads - 1) / kThreads;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

// The window levels: the order of n strings into `order`.
int run_strings(const StrSrc &src, long long n, long long max_len, uint32_t *order, void *ws,
                const Call &tuning, cudaStream_t st) {
    const StrLayout L = str_layout(n);
    const StrWs w = str_carve(L, ws);
    const int sms = device_sms();
    if (sms <= 0) return BINAR_ERR_CUDA;
    const int cap = sms * 4;
    const int g = ceil_grid(n, cap);
    const int levels = (int)(max_len / kWin) + 1;
    int rc;
    if (cudaMemsetAsync(w.ctr, 0, sizeof(StrCtr), st) != cudaSuccess) return BINAR_ERR_CUDA;
    if ((rc = launch("str_init", -1, st, [&] { launch_pdl(k_str_init, g, kThreads, 0, st, w, src, n, max_len); })))
        return rc;
    for (int lvl = 0; lvl < levels; lvl++) {
        const int cur = lvl & 1, nxt = cur ^ 1;
        if ((rc = launch("str_window", lvl, st, [&] { launch_pdl(k_str_window, g, kThreads, 0, st, w, src, cur, lvl); })))
            return rc;
        Call ic;
        std::memset(&ic, 0, sizeof(ic));
        ic.keys = w.key;
        ic.vals = w.ord[cur];
        ic.offsets = w.segoff[cur];
        ic.num_segments = lvl == 0 ? 1 : n / 2 + 2;
        ic.num_segments_dev = &w.ctr->nseg[cur];
        ic.layout = &L.inner_layout;
        ic.n = n;
        ic.map = BINAR_MAP_BYTES_BE;
        ic.vb = 4;
        ic.cutoff = tuning.cutoff;
        ic.bits = tuning.bits;
        ic.tile_variant = tuning.tile_variant;
        ic.ctas_per_sm = tuning.ctas_per_sm;
        ic.timeout_ns = tuning.timeout_ns;
        ic.skip_publish_tile = -1;
        ic.ws = w.inner;
        ic.stream = st;
        if ((rc = run_call_k16(ic))) return rc;
        if ((rc = launch("str_emit", lvl, st, [&] { launch_pdl(k_str_emit, g, kThreads, 0, st, w, order, cur); })))
            return rc;
        if ((rc = launch("str_segstarts", lvl, st, [&] { launch_pdl(k_str_segstarts, g, kThreads, 0, st, w, cur); })))
            return rc;
        const int sg = ceil_grid(n / kScanItems + 1, cap);
        if ((rc = launch("str_scan", lvl, st, [&] {
                 launch_pdl(k_str_scan_count, sg, kThreads, 0, st, w, cur);
                 launch_pdl(k_str_scan_tiles, 1, kThreads, 0, st, w, cur);
                 launch_pdl(k_str_scan_apply, sg, kThreads, 0, st, w, cur);
             })))
            return rc;
        if ((rc = launch("str_runs", lvl, st, [&] { launch_pdl(k_str_runs, g, kThreads, 0, st, w, cur, nxt); })))
            return rc;
        if ((rc = launch("str_compact", lvl, st, [&] { launch_pdl(k_str_compact, g, kThreads, 0, st, w, cur, nxt); })))
            return rc;
        if ((rc = launch("str_close", lvl, st, [&] {
                 launch_pdl(k_str_close, 1, 32, 0, st, w, nxt, lvl == levels - 1 ? 1 : 0);
             })))
            return rc;
    }
    return BINAR_OK;
}

}  // namespace

// Sorts n keys wider than 16 bytes (and their payloads) in place through the
// string levels: the order of the keys read as byte strings after the key
// map, then the keys and payloads moved into it.
int sort_wide(void *keys, void *vals, long long n, int kb, int map, int vb, void *ws,
              const Call &tuning, cudaStream_t st) {
    const WideLayout L = wide_layout(n, kb, vb);
    unsigned char *b = static_cast<unsigned char *>(ws);
    uint32_t *order = reinterpret_cast<uint32_t *>(b + L.order);
    unsigned char *tmp = b + L.tmp;
    StrSrc src{static_cast<const unsigned char *>(keys), nullptr, kb, map};
    int rc = run_strings(src, n, kb, order, ws, tuning, st);
    if (rc) return rc;
    const int cap = device_sms() * 4;
    auto move = [&](void *arr, int eb) -> int {
        const long long work = n * ((eb % 16) == 0 ? eb / 16 : eb);
        int r = launch("str_gather", -1, st, [&] {
            launch_pdl(k_str_gather, ceil_grid(work, cap), kThreads, 0, st,
                       static_cast<const unsigned char *>(arr), tmp, order, n, eb);
        });
        if (r) return r;
        if (cudaMemcpyAsync(arr, tmp, (size_t)n * eb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return BINAR_ERR_CUDA;
        return BINAR_OK;
    };
    if ((rc = move(keys, kb))) return rc;
    if (vb && (rc = move(vals, vb))) return rc;
    return BINAR_OK;
}

size_t wide_workspace_bytes(long long n, int kb, int vb) { return wide_layout(n, kb, vb).total; }
size_t strings_workspace_bytes(long long n) { return str_layout(n).total; }

int sort_strings(const void *bytes, const long long *offsets, long long n, long long max_len,
                 uint32_t *order, void *ws, const Call &tuning, cudaStream_t st) {
    StrSrc src{static_cast<const unsigned char *>(bytes), offsets, 0, BINAR_MAP_BYTES_BE};
    return run_strings(src, n, max_len, order, ws, tuning, st);
}

}  // namespace binar
