// binar_internal.cuh -- data structures shared by the host driver and the
// kernels of libbinar: key encodings, bucket/job descriptors, the workspace
// layout and small device helpers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/binar.h"

namespace binar {

// k: key bits consumed per partition pass.  The paper splits on one bit per
// pass ("Partition Array into Sub-arrays"); fusing k bits does the work of k
// of its passes in one read and one write of every live key.  k is chosen per
// call (Params::bits, at most kBits; 8 by default); every digit-indexed array
// holds kRadix = 2^kBits entries, of which a pass of k bits uses the first 2^k.
// kBits is also the window of the shared-memory LSD finisher.
constexpr int kBits = 8;
constexpr int kRadix = 1 << kBits;
constexpr int kMinSortBits = 4;      // smallest k a sort accepts (bounds the level count)
constexpr int kThreads = 256;        // threads of every tile kernel (one per digit)
constexpr int kWarps = kThreads / 32;

// ---------------------------------------------------------------------------
// Descriptors.  A Bucket is one live sub-array of the recursion: a contiguous
// range of the key array that still has to be split on bits pos .. w-1.
// ---------------------------------------------------------------------------
enum BucketFlags : uint8_t {
    kHasHist = 1,   // its digit histogram was computed by an earlier kernel
    kSkip = 2,      // no partition at this level (pass-through or finished)
};

struct Bucket {
    long long begin;       // first key index
    uint32_t len;          // keys in the bucket (> the finisher cutoff)
    uint32_t tile_start;   // first tile of the bucket in this level's tile space
    uint16_t pos;          // next bit position to split on (0 = most significant)
    uint8_t buf;           // 0: the caller's arrays, 1: the workspace arrays
    uint8_t flags;         // BucketFlags
    uint32_t pad;
};
static_assert(sizeof(Bucket) == 24, "Bucket layout");

// A bucket small enough to finish inside one CTA's shared memory: it is sorted
// on bits pos .. w-1 and written to the caller's arrays.
struct Job {
    long long begin;
    uint32_t len;
    uint16_t pos;          // == w: nothing left to sort, only move to buffer 0
    uint8_t buf;
    uint8_t pad;
};
static_assert(sizeof(Job) == 16, "Job layout");

// A finished bucket larger than the finisher cutoff that must still be moved:
// copied back from the workspace arrays to the caller's, or (kCopyReverse)
// reversed -- strictly decreasing keys -- into the caller's arrays, in place
// when it already sits there (kCopyInPlace).  A bucket whose keys are all
// equal (kCopyFill) gets its one key written, not read, and only its payloads
// copied.  The flags ride in the top bits of `begin` (key indices stay below
// 2^60).
struct CopyJob {
    long long begin;
    uint32_t len;
    uint32_t tile_start;
};
static_assert(sizeof(CopyJob) == 16, "CopyJob layout");
constexpr long long kCopyReverse = 1LL << 62;
constexpr long long kCopyInPlace = 1LL << 61;
constexpr long long kCopyFill = 1LL << 60;
constexpr long long kCopyBeginMask = (1LL << 60) - 1;

// Order flags of a bucket's adjacent key pairs (encoded keys).
constexpr uint32_t kHasDescent = 1;      // some key[i] > key[i+1]
constexpr uint32_t kHasNonDescent = 2;   // some key[i] <= key[i+1]

constexpr int kMaxClasses = 8;          // finisher size classes
constexpr int kIpChunk = 1024;          // in-place mode: exchanged pairs per swap work item

// Job indices are kept per finisher size class, each class in a region of
// its own: class 0 (jobs of up to 1024 keys) may hold every job (jcap), and
// every later class only jobs of more than 1024 keys -- disjoint key ranges,
// so at most n / 1025 + 1 of them.  Region c starts at job_region(c, ...).
__host__ __device__ inline unsigned long long job_region(int c, long long n, unsigned long long jcap) {
    return c == 0 ? 0ull : jcap + (unsigned long long)(c - 1) * (unsigned long long)(n / 1025 + 1);
}

struct Counters {
    uint32_t status;                  // first device error (binar_status), 0 = OK
    uint32_t njobs;                   // finisher jobs
    unsigned long long alloc[2];      // per list slot: (tiles << 32) | buckets
    unsigned long long copy_alloc;    // (tiles << 32) | copy jobs
    uint32_t ticket_hist, ticket_part, ticket_fin, ticket_copy;
    uint32_t ticket_prep;
    uint32_t njobs2;                  // finisher jobs left to the LSD path
    uint32_t ticket_fin2;
    uint32_t pad[5];
    uint32_t class_count[kMaxClasses];   // finisher jobs per size class
    uint32_t gbar[2];                 // grid barrier of the fused level tail (arrivals, generation)
    uint32_t unused[kMaxClasses - 2];
    uint32_t class_ticket[kMaxClasses];  // per-class work tickets
};
static_assert(sizeof(Counters) == 176, "Counters layout");

// Device view of the caller's workspace, carved by the host driver.
struct Ws {
    Counters *ctr;
    void *alt_keys;                // n * key_bytes
    void *alt_vals;                // n * val_bytes
    Bucket *list[2];               // two list slots: current level / next level
    uint32_t *hist[2];             // [bucket][kRadix]: counts, then exclusive prefix
    uint4 *andor[2];               // [bucket][2]: AND and OR of the encoded keys
    uint32_t *order[2];            // [bucket]: kHasDescent | kHasNonDescent over adjacent keys
    uint32_t *tilemap;             // [tile] -> bucket index in the current list
    uint32_t *cells;               // [tile][kRadix] look-back cells
    Job *jobs;
    uint32_t *jobidx;              // job indices grouped by size class
    Job *jobs2;                    // jobs the finisher's fast path hands to the LSD path
    CopyJob *copies;
    uint32_t mcap, tcap, jcap, ccap;   // capacities: buckets, tiles, jobs, copy jobs
};

// Per-call parameters shared by every kernel of one sort.
struct Params {
    void *keys;                    // caller's keys (buffer 0)
    void *vals;                    // caller's payloads (buffer 0) or nullptr
    long long n;
    int map;                       // binar_key_map
    int cutoff;                    // finisher cutoff C
    long long timeout_ns;
    int skip_publish_tile;         // test hook: level-0 tile that never publishes (-1 = none)
    int tile;                      // keys per partition tile (the call's tile variant)
    int bits;                      // k: key bits per partition pass, 1 .. kBits
    int inplace;                   // 1: children stay in the caller's arrays (in-place passes)
};

// ---------------------------------------------------------------------------
// Key encodings ("The Other Universal Property"): every supported key type is
// mapped to an unsigned bit string whose unsigned order is the key order.
// Keys stay in their raw form in memory; the map is applied when a digit is
// extracted.
// ---------------------------------------------------------------------------
struct U128 {
    uint64_t hi, lo;
};

template <int KB> struct KeyTraits;

template <> struct KeyTraits<4> {
    using Raw = uint32_t;
    using Bits = uint32_t;
    static constexpr int kW = 32;
    __device__ static __forceinline__ Bits encode(Raw x, int map) {
        switch (map) {
        case BINAR_MAP_SIGNED: return x ^ 0x80000000u;
        case BINAR_MAP_FLOAT: return (x & 0x80000000u) ? ~x : (x | 0x80000000u);
        case BINAR_MAP_BYTES_BE: return __byte_perm(x, 0, 0x0123);
        default: return x;
        }
    }
    __device__ static __forceinline__ uint32_t digit(Bits b, int pos) {
        return (b << pos) >> (32 - kBits);       // pos < 32
    }
    // nb (< 32) bits starting at bit position pos (0 = MSB); bits past the key read as 0
    __device__ static __forceinline__ uint32_t bits_at(Bits b, int pos, int nb) {
        return (b << pos) >> (32 - nb);
    }
    __device__ static __forceinline__ bool less(Bits a, Bits b) { return a < b; }
    __device__ static __forceinline__ Bits ones() { return 0xffffffffu; }
    __device__ static __forceinline__ Bits zero() { return 0u; }
    // first bit position (0 = MSB) where a and o differ, or kW if equal
    __device__ static __forceinline__ int first_diff(Bits a, Bits o) {
        return (a == o) ? kW : __clz(a ^ o);
    }
    __device__ static __forceinline__ uint4 pack(Bits b) { return make_uint4(b, 0, 0, 0); }
    __device__ static __forceinline__ Bits unpack(uint4 v) { return v.x; }
};

template <> struct KeyTraits<8> {
    using Raw = uint64_t;
    using Bits = uint64_t;
    static constexpr int kW = 64;
    __device__ static __forceinline__ uint64_t bswap64(uint64_t x) {
        uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
        return ((uint64_t)__byte_perm(lo, 0, 0x0123) << 32) | __byte_perm(hi, 0, 0x0123);
    }
    __device__ static __forceinline__ Bits encode(Raw x, int map) {
        const uint64_t s = 0x8000000000000000ull;
        switch (map) {
        case BINAR_MAP_SIGNED: return x ^ s;
        case BINAR_MAP_FLOAT: return (x & s) ? ~x : (x | s);
        case BINAR_MAP_BYTES_BE: return bswap64(x);
        default: return x;
        }
    }
    __device__ static __forceinline__ uint32_t digit(Bits b, int pos) {
        return (uint32_t)((b << pos) >> (64 - kBits));   // pos < 64
    }
    __device__ static __forceinline__ uint32_t bits_at(Bits b, int pos, int nb) {
        return (uint32_t)((b << pos) >> (64 - nb));
    }
    __device__ static __forceinline__ bool less(Bits a, Bits b) { return a < b; }
    __device__ static __forceinline__ Bits ones() { return ~0ull; }
    __device__ static __forceinline__ Bits zero() { return 0ull; }
    __device__ static __forceinline__ int first_diff(Bits a, Bits o) {
        return (a == o) ? kW : __clzll(a ^ o);
    }
    __device__ static __forceinline__ uint4 pack(Bits b) {
        return make_uint4((uint32_t)b, (uint32_t)(b >> 32), 0, 0);
    }
    __device__ static __forceinline__ Bits unpack(uint4 v) { return ((uint64_t)v.y << 32) | v.x; }
};

template <> struct KeyTraits<16> {
    using Raw = uint4;     // bytes 0..15 as four little-endian words x, y, z, w
    using Bits = U128;
    static constexpr int kW = 128;
    __device__ static __forceinline__ Bits encode(Raw x, int map) {
        Bits b;
        if (map == BINAR_MAP_BYTES_BE) {
            b.hi = ((uint64_t)__byte_perm(x.x, 0, 0x0123) << 32) | __byte_perm(x.y, 0, 0x0123);
            b.lo = ((uint64_t)__byte_perm(x.z, 0, 0x0123) << 32) | __byte_perm(x.w, 0, 0x0123);
        } else {   // little-endian 128-bit integer
            b.hi = ((uint64_t)x.w << 32) | x.z;
            b.lo = ((uint64_t)x.y << 32) | x.x;
            if (map == BINAR_MAP_SIGNED) b.hi ^= 0x8000000000000000ull;
        }
        return b;
    }
    __device__ static __forceinline__ uint32_t digit(Bits b, int pos) {
        uint64_t top;
        if (pos < 64) top = pos ? ((b.hi << pos) | (b.lo >> (64 - pos))) : b.hi;
        else top = b.lo << (pos - 64);
        return (uint32_t)(top >> (64 - kBits));
    }
    __device__ static __forceinline__ uint32_t bits_at(Bits b, int pos, int nb) {
        uint64_t top;
        if (pos < 64) top = pos ? ((b.hi << pos) | (b.lo >> (64 - pos))) : b.hi;
        else top = b.lo << (pos - 64);
        return (uint32_t)(top >> (64 - nb));
    }
    __device__ static __forceinline__ bool less(Bits a, Bits b) {
        return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
    }
    __device__ static __forceinline__ Bits ones() { return Bits{~0ull, ~0ull}; }
    __device__ static __forceinline__ Bits zero() { return Bits{0ull, 0ull}; }
    __device__ static __forceinline__ int first_diff(Bits a, Bits o) {
        uint64_t h = a.hi ^ o.hi, l = a.lo ^ o.lo;
        if (h) return __clzll(h);
        if (l) return 64 + __clzll(l);
        return kW;
    }
    __device__ static __forceinline__ uint4 pack(Bits b) {
        return make_uint4((uint32_t)b.lo, (uint32_t)(b.lo >> 32), (uint32_t)b.hi,
                          (uint32_t)(b.hi >> 32));
    }
    __device__ static __forceinline__ Bits unpack(uint4 v) {
        return Bits{((uint64_t)v.w << 32) | v.z, ((uint64_t)v.y << 32) | v.x};
    }
};

// Branch-free key encoders: built once per kernel from the runtime map, so the
// per-key encoding is a byte swap (selected) and one XOR with a mask.
template <int KB> struct Encoder;

template <> struct Encoder<4> {
    bool bswap;
    uint32_t fmask, smask;
    __device__ explicit Encoder(int map)
        : bswap(map == BINAR_MAP_BYTES_BE), fmask(map == BINAR_MAP_FLOAT ? ~0u : 0u),
          smask((map == BINAR_MAP_SIGNED || map == BINAR_MAP_FLOAT) ? 0x80000000u : 0u) {}
    __device__ __forceinline__ uint32_t operator()(uint32_t x) const {
        if (bswap) x = __byte_perm(x, 0, 0x0123);
        return x ^ (((uint32_t)((int32_t)x >> 31) & fmask) | smask);
    }
};

template <> struct Encoder<8> {
    bool bswap;
    uint64_t fmask, smask;
    __device__ explicit Encoder(int map)
        : bswap(map == BINAR_MAP_BYTES_BE), fmask(map == BINAR_MAP_FLOAT ? ~0ull : 0ull),
          smask((map == BINAR_MAP_SIGNED || map == BINAR_MAP_FLOAT) ? 0x8000000000000000ull : 0ull) {}
    __device__ __forceinline__ uint64_t operator()(uint64_t x) const {
        if (bswap) x = KeyTraits<8>::bswap64(x);
        return x ^ (((uint64_t)((int64_t)x >> 63) & fmask) | smask);
    }
};

template <> struct Encoder<16> {
    int map;
    __device__ explicit Encoder(int m) : map(m) {}
    __device__ __forceinline__ U128 operator()(uint4 x) const { return KeyTraits<16>::encode(x, map); }
};

// Inverses of the encoders (encoded bit string -> raw key).
template <int KB> struct Decoder;

template <> struct Decoder<4> {
    bool bswap;
    uint32_t fmask, smask;
    __device__ explicit Decoder(int map)
        : bswap(map == BINAR_MAP_BYTES_BE), fmask(map == BINAR_MAP_FLOAT ? ~0u : 0u),
          smask((map == BINAR_MAP_SIGNED || map == BINAR_MAP_FLOAT) ? 0x80000000u : 0u) {}
    __device__ __forceinline__ uint32_t operator()(uint32_t e) const {
        uint32_t x = e ^ (((uint32_t)((int32_t)~e >> 31) & fmask) | smask);
        return bswap ? __byte_perm(x, 0, 0x0123) : x;
    }
};

template <> struct Decoder<8> {
    bool bswap;
    uint64_t fmask, smask;
    __device__ explicit Decoder(int map)
        : bswap(map == BINAR_MAP_BYTES_BE), fmask(map == BINAR_MAP_FLOAT ? ~0ull : 0ull),
          smask((map == BINAR_MAP_SIGNED || map == BINAR_MAP_FLOAT) ? 0x8000000000000000ull : 0ull) {}
    __device__ __forceinline__ uint64_t operator()(uint64_t e) const {
        uint64_t x = e ^ (((uint64_t)((int64_t)~e >> 63) & fmask) | smask);
        return bswap ? KeyTraits<8>::bswap64(x) : x;
    }
};

template <> struct Decoder<16> {
    int map;
    __device__ explicit Decoder(int m) : map(m) {}
    __device__ __forceinline__ uint4 operator()(U128 e) const {
        uint4 x;
        if (map == BINAR_MAP_BYTES_BE) {
            x.x = __byte_perm((uint32_t)(e.hi >> 32), 0, 0x0123);
            x.y = __byte_perm((uint32_t)e.hi, 0, 0x0123);
            x.z = __byte_perm((uint32_t)(e.lo >> 32), 0, 0x0123);
            x.w = __byte_perm((uint32_t)e.lo, 0, 0x0123);
        } else {
            const uint64_t hi = map == BINAR_MAP_SIGNED ? e.hi ^ 0x8000000000000000ull : e.hi;
            x.x = (uint32_t)e.lo;
            x.y = (uint32_t)(e.lo >> 32);
            x.z = (uint32_t)hi;
            x.w = (uint32_t)(hi >> 32);
        }
        return x;
    }
};

__device__ __forceinline__ U128 operator&(U128 a, U128 b) { return U128{a.hi & b.hi, a.lo & b.lo}; }
__device__ __forceinline__ U128 operator|(U128 a, U128 b) { return U128{a.hi | b.hi, a.lo | b.lo}; }

template <int VB> struct ValTraits { using T = uint32_t; };
template <> struct ValTraits<8> { using T = uint64_t; };

// ---------------------------------------------------------------------------
// Device helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Programmatic dependent launch: every kernel of a call is launched with the
// programmatic-serialization attribute, so the next kernel in the stream may be
// scheduled while this one drains.  Its first act is to wait until its
// predecessor has completed and that grid's writes are visible
// (griddepcontrol.wait); it then allows its own successor to launch.  Nothing
// is read or written before the wait.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void set_status(Counters *c, uint32_t code) {
    atomicCAS(&c->status, 0u, code);
}

__device__ __forceinline__ bool has_error(const Counters *c) {
    return ld_relaxed(&c->status) != 0;
}

}  // namespace binar
