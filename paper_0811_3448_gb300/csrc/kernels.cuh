// kernels.cuh -- the CUDA kernels of libbinar (sm_103a).
//
// The paper's binar sort ("Operation of Algorithm") splits a sub-array on one
// bit, then recurses into the two parts.  Here every level of that recursion
// is run for all live sub-arrays ("buckets") at once and k = 8 bits at a time:
//
//   prep      builds the level's tile -> bucket map, clears its look-back cells
//             and histograms                         (bookkeeping of step 2)
//   hist      per bucket: digit counts at its bit position, and the AND / OR
//             of its encoded keys                     (bit extraction, step 3)
//   classify  per bucket: base case, pass-through or split; children become
//             next-level buckets, finisher jobs or copy jobs   (steps 1 and 4)
//   partition per tile: stable rank by digit, single-pass decoupled look-back
//             across the bucket's tiles, scatter through shared memory (step 3)
//   finish    per small bucket: the rest of the recursion in shared memory
//   copy      moves finished buckets that sit in the workspace back
#pragma once

#include "binar_internal.cuh"

namespace binar {

// Items per thread of the finisher's largest job: 8192 / 4096 / 2048 keys.
template <int KB> struct TileShape {
    static constexpr int kItems = KB == 4 ? 32 : (KB == 8 ? 16 : 8);
    static constexpr int kTile = kThreads * kItems;
};
// Items per thread of a partition / histogram tile -- 6144 keys for 4-byte
// keys with a payload, 7168 for 4-byte keys alone, 4096 for 8-byte keys, 2048
// for 16-byte keys -- and the resident partition CTAs per SM the register
// budget is sized for: 3 (measured against 4096 / 2048-key tiles at 4 CTAs/SM,
// the larger tiles spread the per-tile ticket, scan and look-back over more
// keys), 4 for keys without payload, whose tiles leave room for a fourth CTA
// (measured faster despite a few spilled registers; for 4-byte keys alone,
// 7168-key tiles measured faster than 3072 / 4096 at 5-8 CTAs/SM and than
// 6144 / 8192 at 4).  Every kernel of a call uses the same tile (Params::tile).
// TV selects one of two compiled tile shapes (the autotuner's tile choice):
// 0 is the shape above, 1 a tile of about two thirds or half its keys at one
// more resident CTA per SM (cheaper ragged tiles when buckets are small).
template <int KB, int VB, int TV = 0> struct PartShape {
    static constexpr int kItems = TV == 0 ? (KB == 4 ? (VB == 0 ? 28 : 24) : (KB == 8 ? 16 : 8))
                                          : (KB == 4 ? 16 : (KB == 8 ? 8 : 4));
    static constexpr int kTile = kThreads * kItems;
    static constexpr int kMinBlocks = TV == 0 ? ((VB == 0 && KB != 16) ? 4 : 3)
                                              : ((VB == 0 && KB != 16) ? 5 : 4);
};

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of one uint32 per thread (kThreads threads).
// `scratch` holds kWarps words.  Returns the exclusive prefix; *total gets the
// sum.  Contains two __syncthreads().
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *scratch,
                                                         uint32_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) scratch[w] = incl;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int i = 0; i < kWarps; i++) {
        uint32_t s = scratch[i];
        before += (i < w) ? s : 0u;
        all += s;
    }
    __syncthreads();
    *total = all;
    return before + incl - v;
}

// ---------------------------------------------------------------------------
// Tile ranking.  A tile of up to kThreads * ITEMS keys is held "warp-striped"
// with `iu` items per thread (iu <= ITEMS, uniform over the CTA): item j of
// lane l in warp w is tile element w*32*iu + j*32 + l, so the processing
// order (warp, item, lane) is the memory order.  Items with j >= iu or with an
// element index >= len are invalid and take no rank.
//
// Digits (< 256) and ranks (< 65536) are kept packed in registers: four digits
// or two ranks per 32-bit word.
// ---------------------------------------------------------------------------
template <int ITEMS>
struct Packed {
    uint32_t d[(ITEMS + 3) / 4];
    uint32_t r[(ITEMS + 1) / 2];
    __device__ __forceinline__ uint32_t dig(int j) const {
        return (d[j >> 2] >> ((j & 3) * 8)) & 0xffu;
    }
    __device__ __forceinline__ void set_dig(int j, uint32_t v) {   // in order of j
        if ((j & 3) == 0) d[j >> 2] = v;
        else d[j >> 2] |= v << ((j & 3) * 8);
    }
    __device__ __forceinline__ uint32_t rank(int j) const {
        return (r[j >> 1] >> ((j & 1) * 16)) & 0xffffu;
    }
    __device__ __forceinline__ void set_rank(int j, uint32_t v) {  // in order of j
        if ((j & 1) == 0) r[j >> 1] = v;
        else r[j >> 1] |= v << 16;
    }
    // adds v to rank j; the sum stays below 65536, so the other half is untouched
    __device__ __forceinline__ void add_rank(int j, uint32_t v) {
        r[j >> 1] += v << ((j & 1) * 16);
    }
};

__device__ __forceinline__ int striped(int iu, int j) {
    return (threadIdx.x >> 5) * 32 * iu + j * 32 + (threadIdx.x & 31);
}

// Shared memory of the ranking: per-warp digit counters and lane masks,
// per-digit tile counts (dcount) and their exclusive prefix (dstart).
struct RankSmemLite {
    uint32_t dcount[kRadix];
    uint32_t dstart[kRadix];
    uint32_t scratch[kWarps];
};
struct RankSmem : RankSmemLite {
    uint32_t wcnt[kWarps * kRadix];
    uint32_t wmask[kWarps * kRadix];
};
template <bool STABLE> struct RankSmemFor { using T = RankSmem; };
template <> struct RankSmemFor<false> { using T = RankSmemLite; };

// rank_stable: every valid item gets its position in the tile stably sorted
// by digit.  First per-warp digit counts (shared-memory atomics, order free),
// a per-digit exclusive scan across warps and across digits, then item by
// item a warp multisplit: lanes OR their bit into a per-warp digit mask, so
// each lane learns its same-digit peers and counts those below it; the
// highest peer advances the warp's counter.  A warp whose 32 lanes share one
// digit (sorted input) takes a shortcut without atomics.
template <int ITEMS>
__device__ __forceinline__ void rank_stable(Packed<ITEMS> &pk, int iu, int len, RankSmem &s) {
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const uint32_t lt = lanemask_lt();
    uint32_t *wc = s.wcnt + w * kRadix;
    uint32_t *wm = s.wmask + w * kRadix;
    for (int i = tid; i < kWarps * kRadix; i += kThreads) {
        s.wcnt[i] = 0;
        s.wmask[i] = 0;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        if (j < iu) {
            const bool valid = striped(iu, j) < len;
            const uint32_t d = pk.dig(j);
            const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
            if (__all_sync(0xffffffffu, valid && d == d0)) {
                if (lane == 0) atomicAdd(&wc[d0], 32u);
            } else if (valid) {
                atomicAdd(&wc[d], 1u);
            }
        }
    }
    __syncthreads();
    {
        const int d = tid;
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ww++) {
            const uint32_t c = s.wcnt[ww * kRadix + d];
            s.wcnt[ww * kRadix + d] = run;
            run += c;
        }
        s.dcount[d] = run;
        uint32_t total;
        const uint32_t start = block_exclusive_scan(run, s.scratch, &total);
        s.dstart[d] = start;
#pragma unroll
        for (int ww = 0; ww < kWarps; ww++) s.wcnt[ww * kRadix + d] += start;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        if (j < iu) {
            const bool valid = striped(iu, j) < len;
            const uint32_t d = pk.dig(j);
            const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
            uint32_t rk = 0;
            if (__all_sync(0xffffffffu, valid && d == d0)) {
                const uint32_t c = wc[d0];
                rk = c + lane;
                __syncwarp();
                if (lane == 0) wc[d0] = c + 32;
                __syncwarp();
            } else {
                if (valid) atomicOr(&wm[d], 1u << lane);
                __syncwarp();
                uint32_t peers = 0, c = 0;
                if (valid) {
                    peers = wm[d];
                    c = wc[d];
                    rk = c + __popc(peers & lt);
                }
                __syncwarp();
                if (valid && (peers >> lane) == 1u) {
                    wc[d] = c + __popc(peers);
                    wm[d] = 0;
                }
                __syncwarp();
            }
            pk.set_rank(j, rk);
        }
    }
}

// rank_stable_warp: the same stable ranking in one pass over the items.  Each
// warp ranks its own items (a contiguous run of the tile, in processing
// order) against per-warp digit counters -- peers found through the per-warp
// lane mask as above -- so no counting pass is needed; afterwards the warps'
// counts of every digit are scanned in warp order, offset by the digit's start
// in the tile, and each item adds its warp's offset for its digit.
// The per-warp lane masks must be zero on entry; they are left zero.
template <int ITEMS>
__device__ __forceinline__ void rank_stable_warp(Packed<ITEMS> &pk, int iu, int len, RankSmem &s) {
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const uint32_t lt = lanemask_lt();
    uint32_t *wc = s.wcnt + w * kRadix;
    uint32_t *wm = s.wmask + w * kRadix;
#pragma unroll
    for (int i = lane; i < kRadix; i += 32) wc[i] = 0;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        if (j < iu) {
            const bool valid = striped(iu, j) < len;
            const uint32_t d = pk.dig(j);
            const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
            uint32_t rk;
            if (__all_sync(0xffffffffu, valid && d == d0)) {
                const uint32_t c = wc[d0];
                rk = c + lane;
                __syncwarp();
                if (lane == 0) wc[d0] = c + 32;
                __syncwarp();
            } else {
                if (valid) atomicOr(&wm[d], 1u << lane);
                __syncwarp();
                uint32_t peers = 0, c = 0;
                if (valid) {
                    peers = wm[d];
                    c = wc[d];
                }
                rk = c + __popc(peers & lt);
                __syncwarp();
                if (valid && (peers >> lane) == 1u) {
                    wc[d] = c + __popc(peers);
                    wm[d] = 0;
                }
                __syncwarp();
            }
            pk.set_rank(j, rk);
        }
    }
    __syncthreads();
    {
        const int d = tid;
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ww++) {
            const uint32_t c = s.wcnt[ww * kRadix + d];
            s.wcnt[ww * kRadix + d] = run;
            run += c;
        }
        s.dcount[d] = run;
        uint32_t total;
        const uint32_t start = block_exclusive_scan(run, s.scratch, &total);
        s.dstart[d] = start;
#pragma unroll
        for (int ww = 0; ww < kWarps; ww++) s.wcnt[ww * kRadix + d] += start;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        if (j < iu) pk.add_rank(j, wc[pk.dig(j)]);
    }
}

// rank_unstable: positions grouped by digit, arbitrary order inside a digit.
// Enough for keys without payloads in an MSD pass (equal digits are split by
// later passes, equal keys are indistinguishable) and for the first window of
// an LSD sort of keys.  One block-wide counter per digit.
template <int ITEMS>
__device__ __forceinline__ void rank_unstable(Packed<ITEMS> &pk, int iu, int len, RankSmemLite &s) {
    const int tid = threadIdx.x, lane = tid & 31;
    s.dcount[tid] = 0;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        if (j < iu) {
            const bool valid = striped(iu, j) < len;
            const uint32_t d = pk.dig(j);
            const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
            uint32_t rk = 0;
            if (__all_sync(0xffffffffu, valid && d == d0)) {
                uint32_t c = 0;
                if (lane == 0) c = atomicAdd(&s.dcount[d0], 32u);
                rk = __shfl_sync(0xffffffffu, c, 0) + lane;
            } else if (valid) {
                rk = atomicAdd(&s.dcount[d], 1u);
            }
            pk.set_rank(j, rk);
        }
    }
    __syncthreads();
    uint32_t total;
    const uint32_t cnt = s.dcount[tid];
    const uint32_t start = block_exclusive_scan(cnt, s.scratch, &total);
    s.dstart[tid] = start;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        if (j < iu) pk.add_rank(j, s.dstart[pk.dig(j)]);
    }
}

template <int ITEMS>
__device__ __forceinline__ void rank_tile(Packed<ITEMS> &pk, int iu, int len, RankSmem &s) {
    rank_stable_warp<ITEMS>(pk, iu, len, s);
}
template <int ITEMS>
__device__ __forceinline__ void rank_tile(Packed<ITEMS> &pk, int iu, int len, RankSmemLite &s) {
    rank_unstable<ITEMS>(pk, iu, len, s);
}

// cp.async copies of 4, 8 or 16 bytes from global to shared memory (no
// registers), for the LSD finisher.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    if (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gmem_src),
                     "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Finisher size classes: a job of len keys is finished by the kernel whose
// capacity kThreads * IU is the smallest that holds it, so that every class
// kernel unrolls its loops with known bounds and sizes its shared memory and
// registers to its class.
// ---------------------------------------------------------------------------
template <int KB> struct FinishClasses;
// (Buckets after two 8-bit passes of a uniform input hold about n / 65536 keys:
// 4096 for 256M 4-byte keys, 2048 for 128M 8-byte keys; the classes 16 / 18
// and 8 / 9 let both halves of that spread run without idle items.)
template <> struct FinishClasses<4> {
    static constexpr int kCount = 7;
    __host__ __device__ static constexpr int iu(int c) {
        return c == 0 ? 4 : c == 1 ? 8 : c == 2 ? 12 : c == 3 ? 16 : c == 4 ? 18 : c == 5 ? 24 : 32;
    }
};
template <> struct FinishClasses<8> {
    static constexpr int kCount = 5;
    __host__ __device__ static constexpr int iu(int c) {
        return c == 0 ? 4 : c == 1 ? 8 : c == 2 ? 9 : c == 3 ? 12 : 16;
    }
};
template <> struct FinishClasses<16> {
    static constexpr int kCount = 2;
    __host__ __device__ static constexpr int iu(int c) { return c == 0 ? 4 : 8; }
};

static_assert(kThreads * FinishClasses<4>::iu(0) == 1024 && kThreads * FinishClasses<8>::iu(0) == 1024 &&
                  kThreads * FinishClasses<16>::iu(0) == 1024,
              "job_region: every class above 0 holds jobs of more than 1024 keys");

template <int KB>
__device__ __forceinline__ int finish_class(uint32_t len) {
    int c = 0;
    while (c + 1 < FinishClasses<KB>::kCount && (uint32_t)(kThreads * FinishClasses<KB>::iu(c)) < len) c++;
    return c;
}

// Appends a finisher job, counts it in its size class and lists its index in
// the class's region of jobidx (n: the call's keys, which bound the regions).
template <int KB>
__device__ __forceinline__ void push_job(const Ws &ws, const Job &j, long long n) {
    const uint32_t ji = atomicAdd(&ws.ctr->njobs, 1u);
    if (ji >= ws.jcap) {
        set_status(ws.ctr, BINAR_ERR_QUEUE_OVERFLOW);
        return;
    }
    ws.jobs[ji] = j;
    const int c = finish_class<KB>(j.len);
    const unsigned long long at = job_region(c, n, ws.jcap) + atomicAdd(&ws.ctr->class_count[c], 1u);
    if (at < job_region(c + 1, n, ws.jcap)) ws.jobidx[at] = ji;
    else set_status(ws.ctr, BINAR_ERR_QUEUE_OVERFLOW);
}

// ---------------------------------------------------------------------------
// init: resets the counters and seeds level 0 with the whole array, or the
// finisher with it when it is small.  One thread.
// ---------------------------------------------------------------------------
template <int KB>
__global__ void k_init(Ws ws, long long n, int cutoff, int pos0, uint32_t tiles0, int seed_list) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Counters *c = ws.ctr;
    uint32_t *cw = reinterpret_cast<uint32_t *>(c);
    for (int i = 0; i < (int)(sizeof(Counters) / 4); i++) cw[i] = 0;
    if (!seed_list) return;
    if (n > cutoff) {
        Bucket b;
        b.begin = 0;
        b.len = (uint32_t)n;
        b.tile_start = 0;
        b.pos = (uint16_t)pos0;
        b.buf = 0;
        b.flags = 0;
        b.pad = 0;
        ws.list[0][0] = b;
        c->alloc[0] = ((unsigned long long)tiles0 << 32) | 1ull;
    } else if (n >= 2) {
        Job j;
        j.begin = 0;
        j.len = (uint32_t)n;
        j.pos = (uint16_t)pos0;
        j.buf = 0;
        j.pad = 0;
        push_job<KB>(ws, j, n);
    }
}

// seed_segments: segment s = [offsets[s], offsets[s+1]) becomes a level-0
// bucket (more than `cutoff` keys), a finisher job (2..cutoff keys) or
// nothing (0 or 1 key).
// count_dev: if not null, the number of segments is read from device memory
// (at most num_segments), for callers whose segment count is known only on
// the device.
template <int KB>
__global__ void k_seed_segments(Ws ws, const long long *offsets, long long num_segments,
                                long long n, int cutoff, int tile, const long long *count_dev) {
    pdl_entry();
    if (count_dev) {
        const long long c = *count_dev;
        num_segments = c < num_segments ? (c > 0 ? c : 0) : num_segments;
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < num_segments;
         s += stride) {
        const long long a = offsets[s], b = offsets[s + 1];
        if (a < 0 || b < a || b > n || b - a > BINAR_MAX_BUCKET_KEYS) {
            set_status(ws.ctr, BINAR_ERR_INVALID_ARG);
            continue;
        }
        const long long len = b - a;
        if (len > cutoff) {
            const uint32_t tiles = (uint32_t)((len + tile - 1) / tile);
            const unsigned long long got =
                atomicAdd(&ws.ctr->alloc[0], ((unsigned long long)tiles << 32) | 1ull);
            const uint32_t bi = (uint32_t)got, t0 = (uint32_t)(got >> 32);
            if (bi >= ws.mcap || (unsigned long long)t0 + tiles > ws.tcap) {
                set_status(ws.ctr, BINAR_ERR_QUEUE_OVERFLOW);
                continue;
            }
            Bucket bk;
            bk.begin = a;
            bk.len = (uint32_t)len;
            bk.tile_start = t0;
            bk.pos = 0;
            bk.buf = 0;
            bk.flags = 0;
            bk.pad = 0;
            ws.list[0][bi] = bk;
        } else if (len >= 2) {
            Job j;
            j.begin = a;
            j.len = (uint32_t)len;
            j.pos = 0;
            j.buf = 0;
            j.pad = 0;
            push_job<KB>(ws, j, n);
        }
    }
}

// ---------------------------------------------------------------------------
// prep: for the level whose list sits in `slot`: tile map, cleared look-back
// cells, cleared histograms and AND/OR accumulators, reset tickets, and an
// empty list for the next level.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void prep_body(const Ws &ws, int slot) {
    if (has_error(ws.ctr)) return;
    const unsigned long long alloc = ws.ctr->alloc[slot];
    const uint32_t nb = (uint32_t)alloc, nt = (uint32_t)(alloc >> 32);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ws.ctr->ticket_hist = 0;
        ws.ctr->ticket_part = 0;
        ws.ctr->alloc[slot ^ 1] = 0;
    }
    if (nb == 0 || nb > ws.mcap || nt > ws.tcap) return;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    // cells: nt * kRadix words, as uint4 (none in the in-place mode, which
    // has no look-back)
    if (ws.cells) {
        uint4 *cells4 = reinterpret_cast<uint4 *>(ws.cells);
        const long long ncell4 = (long long)nt * kRadix / 4;
        for (long long i = gtid; i < ncell4; i += gstride) cells4[i] = make_uint4(0, 0, 0, 0);
    }
    uint4 *hist4 = reinterpret_cast<uint4 *>(ws.hist[slot]);
    const long long nhist4 = (long long)nb * kRadix / 4;
    for (long long i = gtid; i < nhist4; i += gstride) hist4[i] = make_uint4(0, 0, 0, 0);
    for (long long b = gtid; b < nb; b += gstride) {
        ws.andor[slot][2 * b] = make_uint4(~0u, ~0u, ~0u, ~0u);
        ws.andor[slot][2 * b + 1] = make_uint4(0, 0, 0, 0);
        ws.order[slot][b] = 0;
    }
    // tile map: CTA-per-bucket, threads stride over the bucket's tiles
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        const uint32_t t0 = ws.list[slot][b].tile_start;
        // number of tiles of this bucket = next bucket's start (or nt) - t0
        const uint32_t t1 = (b + 1 < nb) ? ws.list[slot][b + 1].tile_start : nt;
        for (uint32_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) ws.tilemap[t] = (uint32_t)b;
    }
}
static __global__ void k_prep(Ws ws, int slot) {
    pdl_entry();
    prep_body(ws, slot);
}

// ---------------------------------------------------------------------------
// hist: per bucket of the level, counts of the digit at the bucket's bit
// position and the AND / OR of its encoded keys.  Persistent CTAs take groups
// of `group` (1 .. kHistGroup) consecutive tiles by ticket, count into
// per-warp shared histograms, and flush to the bucket (global atomics) only
// when the bucket changes or the group ends.  Large calls take groups of
// kHistGroup (fewer flushes); small ones smaller groups, so that their few
// tiles spread over more CTAs (a small sort waits on its slowest CTA).
// ---------------------------------------------------------------------------
constexpr int kHistGroup = 8;

// The 16 / KB keys held in one 16-byte chunk (little-endian words).
template <int KB>
__device__ __forceinline__ void unpack_chunk(const uint4 &v, typename KeyTraits<KB>::Raw *r) {
    if constexpr (KB == 4) {
        r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    } else if constexpr (KB == 8) {
        r[0] = ((uint64_t)v.y << 32) | v.x;
        r[1] = ((uint64_t)v.w << 32) | v.z;
    } else {
        r[0] = v;
    }
}

// The next lane's raw key (full warp).
template <int KB>
__device__ __forceinline__ typename KeyTraits<KB>::Raw shfl_down_raw(typename KeyTraits<KB>::Raw x) {
    if constexpr (KB == 16) {
        return make_uint4(__shfl_down_sync(0xffffffffu, x.x, 1), __shfl_down_sync(0xffffffffu, x.y, 1),
                          __shfl_down_sync(0xffffffffu, x.z, 1), __shfl_down_sync(0xffffffffu, x.w, 1));
    } else {
        return __shfl_down_sync(0xffffffffu, x, 1);
    }
}

// A 16-byte load: through the read-only (non-coherent) path when the data
// cannot change while the kernel runs (NC), else an ordinary load (a kernel
// that also writes the keys, as the fused tail of small sorts does).
template <bool NC>
__device__ __forceinline__ uint4 load16(const uint4 *p) {
    if constexpr (NC) return __ldg(p);
    else return *p;
}

// IDENT: the key map is the identity (BINAR_MAP_UNSIGNED), known at compile time.
template <int KB, bool IDENT, bool NC>
__device__ __forceinline__ void hist_body(const Ws &ws, const Params &p, int slot, int group) {
    using KT = KeyTraits<KB>;
    using Raw = typename KT::Raw;
    using Bits = typename KT::Bits;
    const int T = p.tile;
    constexpr int PER = 16 / KB;
    __shared__ uint32_t sh[kWarps][kRadix];
    __shared__ uint4 sand[kWarps], sor[kWarps];
    __shared__ uint32_t sticket;
    if (has_error(ws.ctr)) return;
    const Encoder<KB> enc(IDENT ? (int)BINAR_MAP_UNSIGNED : p.map);
    const Bucket *list = slot ? ws.list[1] : ws.list[0];
    uint32_t *hist = slot ? ws.hist[1] : ws.hist[0];
    uint4 *andor = slot ? ws.andor[1] : ws.andor[0];
    uint32_t *order = slot ? ws.order[1] : ws.order[0];
    const unsigned long long alloc = slot ? ws.ctr->alloc[1] : ws.ctr->alloc[0];
    const uint32_t nt = (uint32_t)(alloc >> 32);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    uint32_t *wh = sh[w];
    for (int i = tid; i < kWarps * kRadix; i += kThreads) (&sh[0][0])[i] = 0;
    Bits a = KT::ones(), o = KT::zero();
    uint32_t ord = 0;   // order flags of the adjacent pairs this thread compared
    uint32_t cur_b = 0xffffffffu;   // bucket being accumulated (uniform across the CTA)

    // flush the accumulated counts, AND / OR and order flags into bucket cur_b
    auto flush = [&]() {
        const int od = __syncthreads_or((int)(ord & kHasDescent));
        const int on = __syncthreads_or((int)(ord & kHasNonDescent));
        if (tid == 0 && (od || on))
            atomicOr(&order[cur_b], (od ? kHasDescent : 0u) | (on ? kHasNonDescent : 0u));
        ord = 0;
        uint32_t c = 0;
#pragma unroll
        for (int ww = 0; ww < kWarps; ww++) {
            c += sh[ww][tid];
            sh[ww][tid] = 0;
        }
        if (c) atomicAdd(&hist[(size_t)cur_b * kRadix + tid], c);
        uint4 pa = KT::pack(a), po = KT::pack(o);
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            pa.x &= __shfl_xor_sync(0xffffffffu, pa.x, o2);
            pa.y &= __shfl_xor_sync(0xffffffffu, pa.y, o2);
            pa.z &= __shfl_xor_sync(0xffffffffu, pa.z, o2);
            pa.w &= __shfl_xor_sync(0xffffffffu, pa.w, o2);
            po.x |= __shfl_xor_sync(0xffffffffu, po.x, o2);
            po.y |= __shfl_xor_sync(0xffffffffu, po.y, o2);
            po.z |= __shfl_xor_sync(0xffffffffu, po.z, o2);
            po.w |= __shfl_xor_sync(0xffffffffu, po.w, o2);
        }
        if (lane == 0) {
            sand[w] = pa;
            sor[w] = po;
        }
        __syncthreads();
        if (tid == 0) {
            uint4 ra = sand[0], ro = sor[0];
            for (int i = 1; i < kWarps; i++) {
                ra.x &= sand[i].x; ra.y &= sand[i].y; ra.z &= sand[i].z; ra.w &= sand[i].w;
                ro.x |= sor[i].x; ro.y |= sor[i].y; ro.z |= sor[i].z; ro.w |= sor[i].w;
            }
            uint32_t *ga = reinterpret_cast<uint32_t *>(&andor[2 * cur_b]);
            uint32_t *go = reinterpret_cast<uint32_t *>(&andor[2 * cur_b + 1]);
            atomicAnd(ga + 0, ra.x); atomicAnd(ga + 1, ra.y);
            atomicAnd(ga + 2, ra.z); atomicAnd(ga + 3, ra.w);
            atomicOr(go + 0, ro.x); atomicOr(go + 1, ro.y);
            atomicOr(go + 2, ro.z); atomicOr(go + 3, ro.w);
        }
        a = KT::ones();
        o = KT::zero();
    };

    for (;;) {
        if (tid == 0) sticket = atomicAdd(&ws.ctr->ticket_hist, 1u);
        __syncthreads();
        const uint32_t g = sticket;
        __syncthreads();
        const uint32_t t0 = g * (uint32_t)group;
        if (t0 >= nt) break;
        const uint32_t t1 = min(t0 + (uint32_t)group, nt);
        for (uint32_t t = t0; t < t1;) {
            const uint32_t b = ws.tilemap[t];
            const Bucket bk = list[b];
            // the group's consecutive tiles of this bucket are one contiguous
            // range of keys, read in one loop (no partial round per tile)
            const uint32_t tcur = t;
            const uint32_t tend =
                min(t1, bk.tile_start + (uint32_t)(((long long)bk.len + T - 1) / T));
            t = tend > tcur ? tend : tcur + 1;
            if (bk.flags & (kHasHist | kSkip)) continue;
            if (b != cur_b) {
                if (cur_b != 0xffffffffu) flush();
                cur_b = b;
            }
            const long long tb = bk.begin + (long long)(tcur - bk.tile_start) * T;
            const int tlen = (int)min((long long)(t - tcur) * T, bk.begin + (long long)bk.len - tb);
            const Raw *src = reinterpret_cast<const Raw *>(bk.buf ? ws.alt_keys : p.keys) + tb;
            // 16-byte chunks from the boundary at or below src (every chunk holds
            // at least one key of the range); keys outside the range are skipped
            const uintptr_t a1 = reinterpret_cast<uintptr_t>(src);
            const uintptr_t a0 = a1 & ~(uintptr_t)15;
            const int shift = (int)((a1 - a0) / KB);
            const int nchunk = (int)((((a1 + (uintptr_t)tlen * KB + 15) & ~(uintptr_t)15) - a0) >> 4);
            const uint4 *c4 = reinterpret_cast<const uint4 *>(a0);
            // every key of the tile is compared with its successor in the
            // bucket (in the same chunk, in the next lane's chunk, or loaded
            // when that chunk is not the next lane's), so each adjacent pair of the bucket
            // is compared exactly once.  end_rel: the bucket's end, tile-relative.
            const int end_rel = (int)((long long)bk.len - (tb - bk.begin));
            constexpr int Q = 4;      // chunks in flight per thread
            for (int cb = tid - lane; cb < nchunk; cb += Q * kThreads) {     // warp-uniform
                Raw r[Q][PER];
#pragma unroll
                for (int q = 0; q < Q; q++) {
                    const int c = cb + q * kThreads + lane;
                    if (c < nchunk) {
                        unpack_chunk<KB>(load16<NC>(c4 + c), r[q]);
                    } else {
#pragma unroll
                        for (int e = 0; e < PER; e++) r[q][e] = Raw{};
                    }
                }
#pragma unroll
                for (int q = 0; q < Q; q++) {
                    const int c = cb + q * kThreads + lane;
                    // once this thread has seen both a descent and a non-descent
                    // the bucket's flags are settled and the comparisons stop
                    const bool look = ord != (kHasDescent | kHasNonDescent);
                    if (!__any_sync(0xffffffffu, look)) {
                        // flags settled for the whole warp: counts only
                        if (c >= nchunk) continue;
#pragma unroll
                        for (int e = 0; e < PER; e++) {
                            const int idx = c * PER + e - shift;
                            if (idx >= 0 && idx < tlen) {
                                const Bits x = enc(r[q][e]);
                                a = a & x;
                                o = o | x;
                                atomicAdd(&wh[KT::bits_at(x, bk.pos, p.bits)], 1u);
                            }
                        }
                        continue;
                    }
                    const bool has_after = look && (c + 1) * PER - shift < end_rel;
                    Raw rafter = shfl_down_raw<KB>(r[q][0]);
                    if (has_after && (lane == 31 || c + 1 >= nchunk)) {   // not in the next lane
                        Raw rn[PER];
                        unpack_chunk<KB>(load16<NC>(c4 + c + 1), rn);
                        rafter = rn[0];
                    }
                    if (c >= nchunk) continue;
#pragma unroll
                    for (int e = 0; e < PER; e++) {
                        const int idx = c * PER + e - shift;
                        if (idx >= 0 && idx < tlen) {
                            const Bits x = enc(r[q][e]);
                            a = a & x;
                            o = o | x;
                            atomicAdd(&wh[KT::bits_at(x, bk.pos, p.bits)], 1u);
                            if (!look) {
                            } else if (e + 1 < PER) {
                                if (idx + 1 < end_rel) {
                                    const Bits y = enc(r[q][e + 1 < PER ? e + 1 : e]);
                                    ord |= KT::less(y, x) ? kHasDescent : kHasNonDescent;
                                }
                            } else if (has_after) {
                                ord |= KT::less(enc(rafter), x) ? kHasDescent : kHasNonDescent;
                            }
                        }
                    }
                }
            }
        }
    }
    if (cur_b != 0xffffffffu) flush();
}
template <int KB, bool IDENT>
__global__ void __launch_bounds__(kThreads) k_hist(Ws ws, Params p, int slot, int group) {
    pdl_entry();
    hist_body<KB, IDENT, true>(ws, p, slot, group);
}

// ---------------------------------------------------------------------------
// classify: one CTA per bucket of the level ("Determine Recursive Call on
// Sub-arrays").  A bucket whose keys are all equal is finished (the base case
// "end of the bits").  A bucket whose digit is the same for every key passes
// through to the next level undivided, at the first bit where its keys differ
// (the paper's pass-through, with the skip-ahead of "Optimize the
// Algorithm").  Otherwise it is split: the exclusive prefix of its histogram
// replaces the counts (the partition kernel reads it), and every child
// becomes a next-level bucket (more than `cutoff` keys and bits left), a
// finisher job (at most `cutoff` keys, runs of small children merged), or is
// finished (all bits consumed; copied back if it sits in the workspace).
// ---------------------------------------------------------------------------
template <int KB>
__device__ __forceinline__ void classify_body(const Ws &ws, const Params &p, int slot, int last_level) {
    using KT = KeyTraits<KB>;
    using Bits = typename KT::Bits;
    constexpr int W = KT::kW;
    const int T = p.tile;
    __shared__ uint32_t scount[kRadix];
    __shared__ uint32_t sexcl[kRadix];
    __shared__ uint32_t scratch[kWarps];
    __shared__ unsigned long long sbase;
    __shared__ Job sjobs[kRadix];            // this parent's finisher jobs
    __shared__ CopyJob scopies[kRadix];      // and copy jobs (tile_start relative)
    __shared__ uint32_t snjobs, sncopies, scopy_tiles;
    __shared__ unsigned long long scopy_acc;
    __shared__ uint32_t sjob_base;
    __shared__ unsigned long long scopy_base;
    __shared__ uint32_t sclass[kMaxClasses];  // this parent's jobs per finisher class
    __shared__ uint32_t sclass_base[kMaxClasses];   // and their first slot in the class region
    if (has_error(ws.ctr)) return;
    const unsigned long long alloc = ws.ctr->alloc[slot];
    const uint32_t nb = (uint32_t)alloc;
    const int tid = threadIdx.x;
    const int next = slot ^ 1;
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        Bucket bk = ws.list[slot][b];
        const Bits a = KT::unpack(ws.andor[slot][2 * b]);
        const Bits o = KT::unpack(ws.andor[slot][2 * b + 1]);
        const int fd = KT::first_diff(a, o);
        const uint32_t cnt = ws.hist[slot][(size_t)b * kRadix + tid];
        const int nonzero = __syncthreads_count(cnt != 0);
        // already in order ("Optimize the Algorithm": stop on a sorted
        // sub-array): no adjacent descent -> finished as it stands; strictly
        // decreasing -> finished by a reversal (no equal keys, so stable)
        const uint32_t ord = ws.order[slot][b];
        const bool counted = !(bk.flags & kHasHist) && bk.len > 1 && ord != 0;
        const bool ascending = counted && !(ord & kHasDescent);
        const bool descending = counted && !(ord & kHasNonDescent);
        if (fd < W && (ascending || descending)) {
            if (tid == 0) {
                ws.list[slot][b].flags = bk.flags | kSkip;
                if (descending || bk.buf == 1) {
                    const uint32_t tiles = (uint32_t)(((long long)bk.len + T - 1) / T);
                    const unsigned long long got = atomicAdd(
                        &ws.ctr->copy_alloc, ((unsigned long long)tiles << 32) | 1ull);
                    const uint32_t ci = (uint32_t)got;
                    if (ci >= ws.ccap) {
                        set_status(ws.ctr, BINAR_ERR_QUEUE_OVERFLOW);
                    } else {
                        CopyJob cj;
                        cj.begin = bk.begin | (descending ? kCopyReverse : 0LL) |
                                   ((descending && bk.buf == 0) ? kCopyInPlace : 0LL);
                        cj.len = bk.len;
                        cj.tile_start = (uint32_t)(got >> 32);
                        ws.copies[ci] = cj;
                    }
                }
            }
            __syncthreads();
            continue;
        }
        if (fd >= W || nonzero <= 1) {
            // finished (all keys equal) or pass-through
            if (tid == 0) {
                ws.list[slot][b].flags = bk.flags | kSkip;
                if (fd >= W) {
                    if (bk.buf == 1) {
                        const uint32_t tiles = (uint32_t)(((long long)bk.len + T - 1) / T);
                        const unsigned long long got = atomicAdd(
                            &ws.ctr->copy_alloc, ((unsigned long long)tiles << 32) | 1ull);
                        const uint32_t ci = (uint32_t)got;
                        if (ci >= ws.ccap) {
                            set_status(ws.ctr, BINAR_ERR_QUEUE_OVERFLOW);
                        } else {
                            CopyJob cj;
                            cj.begin = bk.begin | kCopyFill;       // all keys equal
                            cj.len = bk.len;
                            cj.tile_start = (uint32_t)(got >> 32);
                            ws.copies[ci] = cj;
                        }
                    }
                } else if (last_level) {
                    set_status(ws.ctr, BINAR_ERR_QUEUE_OVERFLOW);  // cannot happen: fd >= w there
                } else {
                    const uint32_t tiles = (uint32_t)(((long long)bk.len + T - 1) / T);
                    const unsigned long long got =
                        atomicAdd(&ws.ctr->alloc[next], ((unsigned long long)tiles << 32) | 1ull);
                    const uint32_t bi = (uint32_t)got, t0 = (uint32_t)(got >> 32);
                    if (bi >= ws.mcap || (unsigned long long)t0 + tiles > ws.tcap) {
                        set_status(ws.ctr, BINAR_ERR_QUEUE_OVERFLOW);
                    } else {
                        Bucket nbk = bk;
                        nbk.pos = (uint16_t)fd;
                        nbk.tile_start = t0;
                        nbk.flags = 0;
                        ws.list[next][bi] = nbk;
                    }
                }
            }
            __syncthreads();
            continue;
        }
        // split
        uint32_t total;
        const uint32_t excl = block_exclusive_scan(cnt, scratch, &total);
        scount[tid] = cnt;
        sexcl[tid] = excl;
        ws.hist[slot][(size_t)b * kRadix + tid] = excl;
        const int cpos = bk.pos + p.bits;
        const int cbuf = p.inplace ? bk.buf : bk.buf ^ 1;
        const bool terminal = cpos >= W;
        const bool large = !terminal && cnt > (uint32_t)p.cutoff;
        const uint32_t tiles = large ? (cnt + T - 1) / T : 0;
        // reserve the large children in the next list, in digit order
        uint32_t nlarge, ntiles;
        const uint32_t li = block_exclusive_scan(large ? 1u : 0u, scratch, &nlarge);
        const uint32_t ti = block_exclusive_scan(tiles, scratch, &ntiles);
        if (tid == 0) {
            sbase = nlarge ? atomicAdd(&ws.ctr->alloc[next],
                                       ((unsigned long long)ntiles << 32) | nlarge)
                           : 0ull;
        }
        __syncthreads();
        if (large) {
            const uint32_t bi = (uint32_t)sbase + li;
            const uint32_t t0 = (uint32_t)(sbase >> 32) + ti;
            if (bi >= ws.mcap || (unsigned long long)t0 + tiles > ws.tcap) {
                set_status(ws.ctr, BINAR_ERR_QUEUE_OVERFLOW);
            } else {
                Bucket nbk;
                nbk.begin = bk.begin + excl;
                nbk.len = cnt;
                nbk.tile_start = t0;
                nbk.pos = (uint16_t)cpos;
                nbk.buf = (uint8_t)cbuf;
                nbk.flags = 0;
                nbk.pad = 0;
                ws.list[next][bi] = nbk;
            }
        }
        // small and finished children: runs of small children become merged
        // jobs.  Each warp walks one aligned group of 32 digits (lane 0, digit
        // order) and a run never crosses a group, so the keys of a merged job
        // share the top 3 bits of their digit and its 12-bit split still sees
        // at least 7 bits below the digit.  Jobs and copy jobs go to shared
        // lists (slots by shared atomics; a copy job's slot and tile offset
        // come from one 64-bit atomic, so both grow together), then the whole
        // CTA reserves and writes them.
        if (tid == 0) {
            snjobs = 0;
            scopy_acc = 0ull;
        }
        if (tid < kMaxClasses) sclass[tid] = 0;
        __syncthreads();
        {
            const uint32_t C = (uint32_t)p.cutoff;
            const uint32_t own = C / 8;       // a child this large is a job of its own
            auto emit = [&](long long begin, uint32_t len, uint32_t children) {
                if (len == 0) return;
                int jpos = terminal ? W : (children == 1 ? cpos : bk.pos);
                if (terminal && cbuf == 0) return;          // finished in place
                if (!terminal && len == 1 && cbuf == 0) return;
                Job j;
                j.begin = begin;
                j.len = len;
                j.pos = (uint16_t)jpos;
                j.buf = (uint8_t)cbuf;
                j.pad = 0;
                const uint32_t slot = atomicAdd(&snjobs, 1u);
                if (slot < (uint32_t)kRadix) sjobs[slot] = j;
                else set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
            };
            // finished and large: copy job if it sits in the workspace
            auto copy_child = [&](long long cb, uint32_t c) {
                if (cbuf != 1) return;
                const uint32_t tiles = (c + T - 1) / T;
                const unsigned long long got =
                    atomicAdd(&scopy_acc, ((unsigned long long)tiles << 32) | 1ull);
                const uint32_t slot = (uint32_t)got;
                CopyJob cj;
                cj.begin = cb | kCopyFill;      // every key bit consumed: all keys equal
                cj.len = c;
                cj.tile_start = (uint32_t)(got >> 32);
                if (slot < (uint32_t)kRadix) scopies[slot] = cj;
                else set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
            };
            const int d0 = (tid >> 5) * 32, lane = tid & 31;
            const uint32_t cl = scount[d0 + lane];
            const bool big_l = !terminal && cl > C, term_l = terminal && cl > C;
            // a child that would join a merged run (0 < c < own, not large)
            const bool small_l = cl > 0 && !big_l && !term_l && cl < own;
            if (!__any_sync(0xffffffffu, small_l)) {
                // no run to merge in this group: every lane handles its digit
                const long long cb = bk.begin + sexcl[d0 + lane];
                if (term_l) copy_child(cb, cl);
                else if (!big_l && cl > 0) emit(cb, cl, 1);
            } else if (lane == 0) {
                long long run_begin = -1;
                uint32_t run_len = 0, run_children = 0;
                for (int d = d0; d < d0 + 32; d++) {
                    const uint32_t c = scount[d];
                    if (c == 0) continue;
                    const long long cb = bk.begin + sexcl[d];
                    const bool big = !terminal && c > C;
                    if (terminal && c > C) {
                        emit(run_begin, run_len, run_children);
                        run_begin = -1; run_len = 0; run_children = 0;
                        copy_child(cb, c);
                        continue;
                    }
                    if (big) {
                        emit(run_begin, run_len, run_children);
                        run_begin = -1; run_len = 0; run_children = 0;
                        continue;
                    }
                    if (c >= own) {
                        emit(run_begin, run_len, run_children);
                        run_begin = -1; run_len = 0; run_children = 0;
                        emit(cb, c, 1);
                        continue;
                    }
                    if (run_begin >= 0 && run_len + c <= C) {
                        run_len += c;
                        run_children += 1;
                    } else {
                        emit(run_begin, run_len, run_children);
                        run_begin = cb;
                        run_len = c;
                        run_children = 1;
                    }
                }
                emit(run_begin, run_len, run_children);
            }
        }
        __syncthreads();
        if (tid == 0) {
            sncopies = (uint32_t)scopy_acc;
            scopy_tiles = (uint32_t)(scopy_acc >> 32);
            sjob_base = snjobs ? atomicAdd(&ws.ctr->njobs, snjobs) : 0u;
            scopy_base = sncopies ? atomicAdd(&ws.ctr->copy_alloc,
                                              ((unsigned long long)scopy_tiles << 32) | sncopies)
                                  : 0ull;
        }
        __syncthreads();
        int jcls = 0;
        uint32_t jslot = 0;
        const uint32_t ji = sjob_base + tid;
        const bool jvalid = tid < (int)snjobs && ji < ws.jcap;
        if (tid < (int)snjobs) {
            const Job j = sjobs[tid];
            if (jvalid) {
                ws.jobs[ji] = j;
                jcls = finish_class<KB>(j.len);
                jslot = atomicAdd(&sclass[jcls], 1u);
            } else {
                set_status(ws.ctr, BINAR_ERR_QUEUE_OVERFLOW);
            }
        }
        if (tid < (int)sncopies) {
            CopyJob cj = scopies[tid];
            const uint32_t ci = (uint32_t)scopy_base + tid;
            cj.tile_start += (uint32_t)(scopy_base >> 32);
            if (ci < ws.ccap) ws.copies[ci] = cj;
            else set_status(ws.ctr, BINAR_ERR_QUEUE_OVERFLOW);
        }
        __syncthreads();
        // one global atomic per class instead of one per job: this parent's
        // first slot in each class region (the same thread clears its entry
        // before the next parent's jobs are counted)
        if (tid < kMaxClasses && sclass[tid])
            sclass_base[tid] = atomicAdd(&ws.ctr->class_count[tid], sclass[tid]);
        __syncthreads();
        if (jvalid) {
            const unsigned long long at = job_region(jcls, p.n, ws.jcap) + sclass_base[jcls] + jslot;
            if (at < job_region(jcls + 1, p.n, ws.jcap)) ws.jobidx[at] = ji;
            else set_status(ws.ctr, BINAR_ERR_QUEUE_OVERFLOW);
        }
    }
}
template <int KB>
__global__ void __launch_bounds__(kThreads) k_classify(Ws ws, Params p, int slot, int last_level) {
    pdl_entry();
    classify_body<KB>(ws, p, slot, last_level);
}

// For binar_partition_pass: exclusive prefix of the single bucket's histogram
// (kept for the partition kernel) and the caller's group offsets.
// The caller's offsets array has 2^bits + 1 entries.
static __global__ void __launch_bounds__(kThreads) k_prefix_only(Ws ws, long long *offsets, long long n,
                                                                int bits) {
    pdl_entry();
    __shared__ uint32_t scratch[kWarps];
    const int tid = threadIdx.x;
    const uint32_t cnt = ws.hist[0][tid];
    uint32_t total;
    const uint32_t excl = block_exclusive_scan(cnt, scratch, &total);
    ws.hist[0][tid] = excl;
    if (offsets) {
        if (tid < (1 << bits)) offsets[tid] = excl;
        if (tid == 0) offsets[1 << bits] = n;
    }
}

// ---------------------------------------------------------------------------
// partition: one tile per ticket.  The tile's keys and payloads are copied
// into shared memory by the bulk-copy engine (the 16-byte chunks from the
// boundary at or below the tile's first element, completing on an mbarrier), the keys move to registers and are ranked
// by digit (digits and ranks packed in registers), and the tile is staged in
// shared memory in sorted order, in place: keys first, then payloads.  The
// tile is placed after its predecessors in the same bucket through a
// single-pass decoupled look-back: every tile publishes its per-digit count
// (AGGREGATE) as soon as it is ranked, and its inclusive prefix (INCLUSIVE)
// once known; a tile sums its predecessors' cells back to the first INCLUSIVE
// one, reading kLookbackWindow cells per round.  Finally the staged tile is
// written out in order, so that the global writes of every digit run are
// contiguous.
// Cell encoding: 0 = not ready, value+1 in bits 0..30, bit 31 = INCLUSIVE.
// ---------------------------------------------------------------------------
constexpr uint32_t kInclusive = 0x80000000u;
constexpr int kLookbackWindow = 8;

template <int KB, int VB, bool STABLE, int TV>
struct PartitionSmem {
    static constexpr int T = PartShape<KB, VB, TV>::kTile;
    typename RankSmemFor<STABLE>::T rank;
    int offs[kRadix];          // bucket-relative destination of digit d's run, minus its tile start
    uint32_t next_ticket;
    alignas(8) unsigned long long bar;     // mbarrier of the tile's bulk copies
    alignas(16) unsigned char keys[T * KB + 16];
    alignas(16) unsigned char vals[VB ? T * VB + 16 : 16];
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// The 16-byte aligned chunk range [*a0, *a0 + *bytes) that holds elements
// [0, len) of src (EB-byte elements, src aligned to EB); returns the index of
// src[0] in it.
template <int EB>
__device__ __forceinline__ int chunk_range(const void *src, int len, uintptr_t *a0, uint32_t *bytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(src);
    *a0 = a & ~(uintptr_t)15;
    const uintptr_t a1 = (a + (uintptr_t)len * EB + 15) & ~(uintptr_t)15;
    *bytes = (uint32_t)(a1 - *a0);
    return (int)((a - *a0) / EB);
}

// Tile loads by the bulk-copy (TMA) engine: one thread starts the copies of a
// tile, which complete on a shared-memory mbarrier; every thread then waits on
// the barrier's phase.  bulk_begin: the previous use of the destination
// (ordered by a __syncthreads before the call) comes before the async writes.
// Invalidates the barrier so that its shared memory can hold other data (the
// next level of the fused tail); every wait on it has ended (ordered by a
// __syncthreads before the call).
__device__ __forceinline__ void mbar_inval(void *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init(void *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bulk_begin(void *bar, uint32_t bytes) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, uintptr_t src, uint32_t bytes, void *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// A hint that brings [src, src + bytes) into L2 (16-byte aligned, a multiple
// of 16 bytes), without waiting.
__device__ __forceinline__ void l2_prefetch(uintptr_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Waits for phase `parity` of the barrier; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(void *bar, uint32_t parity, long long limit_ns) {
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (done) return true;
        if ((long long)(globaltimer_ns() - t0) > limit_ns) return false;
    }
}

// Sum of the counts of digit threadIdx.x over tiles first .. t-1 back to the
// nearest INCLUSIVE cell (tile `first`, the bucket's first tile, publishes
// INCLUSIVE at once).  A cell that stays 0 past the time limit sets
// BINAR_ERR_DEVICE_TIMEOUT and ends the walk.
__device__ __forceinline__ uint32_t lookback(const Ws &ws, const Params &p, uint32_t t,
                                             uint32_t first) {
    const int tid = threadIdx.x;
    uint32_t excl = 0;
    long long pt = (long long)t - 1;
    for (;;) {
        uint32_t x[kLookbackWindow];
#pragma unroll
        for (int i = 0; i < kLookbackWindow; i++)
            x[i] = (pt - i >= (long long)first)
                       ? ld_relaxed(ws.cells + (size_t)(pt - i) * kRadix + tid)
                       : (kInclusive | 1u);
#pragma unroll
        for (int i = 0; i < kLookbackWindow; i++) {
            if (x[i] == 0) {
                const uint32_t *pc = ws.cells + (size_t)(pt - i) * kRadix + tid;
                const unsigned long long t0 = globaltimer_ns();
                while ((x[i] = ld_relaxed(pc)) == 0) {
                    __nanosleep(32);
                    if ((long long)(globaltimer_ns() - t0) > p.timeout_ns) {
                        set_status(ws.ctr, BINAR_ERR_DEVICE_TIMEOUT);
                        x[i] = kInclusive | 1u;
                        break;
                    }
                }
            }
            excl += (x[i] & ~kInclusive) - 1;
            if (x[i] & kInclusive) return excl;
        }
        pt -= kLookbackWindow;
    }
}

// IDENT: the key map is the identity (BINAR_MAP_UNSIGNED), known at compile time.
template <int KB, int VB, bool STABLE, bool IDENT, int TV>
__device__ __forceinline__ void partition_body(const Ws &ws, const Params &p, int slot, int level,
                                               void *keys0, void *keys1, void *vals0, void *vals1) {
    using KT = KeyTraits<KB>;
    using Raw = typename KT::Raw;
    using V = typename ValTraits<VB>::T;
    constexpr int ITEMS = PartShape<KB, VB, TV>::kItems;
    constexpr int T = PartShape<KB, VB, TV>::kTile;
    // 4-byte keys with 4-byte payloads are staged as 8-byte records over the
    // key and payload arrays, which lie back to back
    constexpr bool KV8 = KB == 4 && VB == 4;
    using Smem = PartitionSmem<KB, VB, STABLE, TV>;
    static_assert(!KV8 || offsetof(Smem, vals) == offsetof(Smem, keys) + sizeof(Smem::keys),
                  "8-byte staging spans the key and payload arrays");
    static_assert(!KV8 || 8 * T <= sizeof(Smem::keys) + sizeof(Smem::vals), "8-byte staging fits");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &s = *reinterpret_cast<Smem *>(smem_raw);
    Raw *skeys = reinterpret_cast<Raw *>(s.keys);
    V *svals = reinterpret_cast<V *>(s.vals);
    if (has_error(ws.ctr)) return;
    if (p.tile != T) {            // the call's tiles must be this kernel's
        if (threadIdx.x == 0) set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
        return;
    }
    const Encoder<KB> enc(IDENT ? (int)BINAR_MAP_UNSIGNED : p.map);
    const Bucket *list = slot ? ws.list[1] : ws.list[0];
    const uint32_t *prefix = slot ? ws.hist[1] : ws.hist[0];
    const unsigned long long alloc = slot ? ws.ctr->alloc[1] : ws.ctr->alloc[0];
    const uint32_t nt = (uint32_t)(alloc >> 32);
    const int tid = threadIdx.x;
    if constexpr (STABLE) {
        for (int i = tid & 31; i < kRadix; i += 32) s.rank.wmask[(tid >> 5) * kRadix + i] = 0;
    }
    if (tid == 0) mbar_init(&s.bar);
    __syncthreads();
    uint32_t phase = 0;
    for (;;) {
        if (tid == 0) s.next_ticket = atomicAdd(&ws.ctr->ticket_part, 1u);
        __syncthreads();
        const uint32_t t = s.next_ticket;
        __syncthreads();
        if (t >= nt) break;
        const uint32_t b = ws.tilemap[t];
        const Bucket bk = list[b];
        if (bk.flags & kSkip) continue;
        const uint32_t ti = t - bk.tile_start;
        const long long tb = bk.begin + (long long)ti * T;
        const int tlen = (int)min((long long)T, (long long)bk.begin + (long long)bk.len - tb);
        const Raw *src = reinterpret_cast<const Raw *>(bk.buf ? keys1 : keys0) + tb;
        const V *vsrc = VB ? reinterpret_cast<const V *>(bk.buf ? vals1 : vals0) + tb : nullptr;
        Raw *dst = reinterpret_cast<Raw *>(bk.buf ? keys0 : keys1) + bk.begin;
        V *vdst = VB ? reinterpret_cast<V *>(bk.buf ? vals0 : vals1) + bk.begin : nullptr;

        // the tile's 16-byte chunks, by the bulk-copy engine
        uintptr_t ka0 = 0, va0 = 0;
        uint32_t kbytes = 0, vbytes = 0;
        const int ks = chunk_range<KB>(src, tlen, &ka0, &kbytes);
        const int vs = VB ? chunk_range<VB>(vsrc, tlen, &va0, &vbytes) : 0;
        if (tid == 0) {
            bulk_begin(&s.bar, kbytes + vbytes);
            bulk_load(s.keys, ka0, kbytes, &s.bar);
            if (VB) bulk_load(s.vals, va0, vbytes, &s.bar);
        }
        // tickets go out in order, so the tile one grid ahead is about to be
        // taken by some CTA: bring its bytes into the shared L2 now (3% off
        // the pass at 256M pairs)
        if (tid == 32 && t + gridDim.x < nt) {
            const uint32_t u = t + gridDim.x;
            const uint32_t bu = ws.tilemap[u];
            const Bucket bq = list[bu];
            if (!(bq.flags & kSkip)) {
                const long long ub = bq.begin + (long long)(u - bq.tile_start) * T;
                const int ulen = (int)min((long long)T, (long long)bq.begin + (long long)bq.len - ub);
                uintptr_t a0 = 0;
                uint32_t bytes = 0;
                chunk_range<KB>(reinterpret_cast<const Raw *>(bq.buf ? keys1 : keys0) + ub, ulen, &a0, &bytes);
                l2_prefetch(a0, bytes);
                if (VB) {
                    chunk_range<VB>(reinterpret_cast<const V *>(bq.buf ? vals1 : vals0) + ub, ulen, &a0, &bytes);
                    l2_prefetch(a0, bytes);
                }
            }
        }
        const bool landed = mbar_wait(&s.bar, phase, p.timeout_ns);
        if (__syncthreads_or(!landed)) {                  // uniform across the CTA
            if (tid == 0) set_status(ws.ctr, BINAR_ERR_DEVICE_TIMEOUT);
            if (!landed) mbar_wait(&s.bar, phase, p.timeout_ns);   // the copy in flight, bounded
            return;
        }
        phase ^= 1;

        Raw k[ITEMS];
        Packed<ITEMS> pk;
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            const int i = striped(ITEMS, j);
            k[j] = skeys[ks + i];
            pk.set_dig(j, i < tlen ? KT::bits_at(enc(k[j]), bk.pos, p.bits) : 0u);
        }
        rank_tile<ITEMS>(pk, ITEMS, tlen, s.rank);

        // publish this tile's counts
        const uint32_t cnt = s.rank.dcount[tid];
        uint32_t *cell = ws.cells + (size_t)t * kRadix + tid;
        const bool hooked = (level == 0 && (int)t == p.skip_publish_tile);
        if (!hooked) st_relaxed(cell, (ti == 0 ? kInclusive : 0u) | (cnt + 1));

        // stage the tile in sorted order, in place (its inputs are in registers)
        if constexpr (KV8) {
            // key and payload side by side, one 8-byte store per record into
            // the bytes of both arrays (every input is in registers after the
            // barrier)
            uint32_t v[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; j++) v[j] = svals[vs + striped(ITEMS, j)];
            __syncthreads();
            uint2 *skv = reinterpret_cast<uint2 *>(s.keys);
#pragma unroll
            for (int j = 0; j < ITEMS; j++) {
                const uint32_t r = pk.rank(j);
                if (striped(ITEMS, j) < tlen) {
                    if (r < (uint32_t)tlen) skv[r] = make_uint2(k[j], v[j]);
                    else set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < ITEMS; j++) {
                const int i = striped(ITEMS, j);
                if (i < tlen) {
                    const uint32_t r = pk.rank(j);
                    if (r < (uint32_t)tlen) skeys[r] = k[j];
                    else set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
                }
            }
            if (VB) {
                V v[ITEMS];
#pragma unroll
                for (int j = 0; j < ITEMS; j++) v[j] = svals[vs + striped(ITEMS, j)];
                __syncthreads();
#pragma unroll
                for (int j = 0; j < ITEMS; j++) {
                    const uint32_t r = pk.rank(j);
                    if (striped(ITEMS, j) < tlen && r < (uint32_t)tlen) svals[r] = v[j];
                }
            }
        }

        uint32_t excl = 0;
        if (ti > 0) {
            excl = lookback(ws, p, t, bk.tile_start);
            if (!hooked) st_relaxed(cell, kInclusive | (excl + cnt + 1));
        }
        s.offs[tid] = (int)(prefix[(size_t)b * kRadix + tid] + excl) - (int)s.rank.dstart[tid];
        __syncthreads();

        // write-out in sorted order: the digit runs are contiguous in memory
#pragma unroll 4
        for (int r = 0; r < ITEMS; r++) {
            const int i = r * kThreads + tid;
            if (i < tlen) {
                Raw kk;
                V vv{};
                if constexpr (KV8) {
                    const uint2 e = reinterpret_cast<const uint2 *>(s.keys)[i];
                    kk = e.x;
                    vv = e.y;
                } else {
                    kk = skeys[i];
                    if (VB) vv = svals[i];
                }
                const uint32_t at = (uint32_t)(s.offs[KT::bits_at(enc(kk), bk.pos, p.bits)] + i);
                if (at < bk.len) {
                    dst[at] = kk;
                    if (VB) vdst[at] = vv;
                } else {
                    set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
                }
            }
        }
        __syncthreads();
    }
}
template <int KB, int VB, bool STABLE, bool IDENT, int TV>
__global__ void __launch_bounds__(kThreads, PartShape<KB, VB, TV>::kMinBlocks)
    k_partition(Ws ws, Params p, int slot, int level, void *keys0, void *keys1, void *vals0,
                void *vals1) {
    pdl_entry();
    partition_body<KB, VB, STABLE, IDENT, TV>(ws, p, slot, level, keys0, keys1, vals0, vals1);
}

// ---------------------------------------------------------------------------
// finish: one small bucket (job) per ticket, sorted inside shared memory on
// bits pos .. w-1 -- the rest of the recursion for that sub-array.  Keys and
// payloads are staged in shared memory by the bulk-copy engine (one
// cp.async.bulk per array, completing on an mbarrier).
//
// Fast path: bits above the first bit f where the job's keys differ are equal
// (AND / OR of the encoded keys), so one MSD split on the 12 bits at f leaves
// runs of about len / 4096 keys.  The split uses one shared-memory atomic per
// key (unstable); the encoded keys are placed in split order, then every key
// counts the keys of its run that precede it in (encoded key, input position)
// order -- the stable order -- and is written straight to its final place.  If a run holds more than kFinishRun keys
// (heavy duplication) the job falls back to an LSD radix sort over 8-bit
// windows with stable passes (the last window starts at pos; windows whose
// bits are equal across the job are skipped; the first pass of a key-only
// sort may be unstable), which builds perm[sorted position] = input position.
// ---------------------------------------------------------------------------
constexpr int kFinishBits = 12;
constexpr int kFinishBins = 1 << kFinishBits;
constexpr int kFinishRun = 128;

// Split counters: 16-bit counts, two bins per word, in the first half of cs;
// after the scan cs[d] = start of bin d | count of bin d << 16 (counts and
// starts stay below the job size, < 65536).
struct FinishFastSmem {
    uint32_t cs[kFinishBins];
    uint32_t scratch[kWarps];
    uint32_t maxrun;
};

template <int KB, int VB, int IU>
struct FinishSmem {
    static constexpr int T = kThreads * IU;
    union {
        FinishFastSmem fast;
    } u;
    uint4 sand[kWarps], sor[kWarps];
    uint32_t next_ticket;
    Job next_job;
    alignas(8) unsigned long long bar;     // mbarrier of the job's bulk copies
    // the job's keys (16 bytes of chunk slack), reused for the packed words of
    // the in-run ranking, which read up to 3 words past the job's last one
    alignas(16) unsigned char keys[T * KB + 32];
    alignas(16) unsigned char vals[VB ? T * VB + 16 : 16];
    uint16_t perm[T];
};

// AND / OR of the job's encoded keys across the CTA (k-wide keys reduce only
// their live 32-bit words).
template <int KB>
__device__ __forceinline__ void block_and_or(typename KeyTraits<KB>::Bits &a,
                                             typename KeyTraits<KB>::Bits &o, uint4 *sand,
                                             uint4 *sor) {
    using KT = KeyTraits<KB>;
    constexpr int NW = KB / 4;
    uint4 pa = KT::pack(a), po = KT::pack(o);
    uint32_t *xa = &pa.x, *xo = &po.x;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
#pragma unroll
        for (int q = 0; q < NW; q++) {
            xa[q] &= __shfl_xor_sync(0xffffffffu, xa[q], o2);
            xo[q] |= __shfl_xor_sync(0xffffffffu, xo[q], o2);
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sand[w] = pa;
        sor[w] = po;
    }
    __syncthreads();
    uint4 ra = sand[0], ro = sor[0];
    for (int i = 1; i < kWarps; i++) {
        ra.x &= sand[i].x; ra.y &= sand[i].y; ra.z &= sand[i].z; ra.w &= sand[i].w;
        ro.x |= sor[i].x; ro.y |= sor[i].y; ro.z |= sor[i].z; ro.w |= sor[i].w;
    }
    a = KT::unpack(ra);
    o = KT::unpack(ro);
}

// The fast path for one job of len <= kThreads * IU keys staged in shared
// memory.  Returns false if the job's runs are too long (the job then goes to
// the LSD path untouched).
template <int KB, int VB, int IU>
__device__ __forceinline__ bool finish_fast(FinishSmem<KB, VB, IU> &s, const Ws &ws,
                                            const Encoder<KB> &enc, const Decoder<KB> &dec,
                                            const Job &job, int ks, int vs,
                                            typename KeyTraits<KB>::Raw *dst,
                                            typename ValTraits<VB>::T *vdst) {
    using KT = KeyTraits<KB>;
    using Raw = typename KT::Raw;
    using Bits = typename KT::Bits;
    using V = typename ValTraits<VB>::T;
    constexpr int W = KT::kW;
    Raw *skeys = reinterpret_cast<Raw *>(s.keys);
    V *svals = reinterpret_cast<V *>(s.vals);
    const int tid = threadIdx.x, lane = tid & 31;
    const int len = (int)job.len;
    FinishFastSmem &fs = s.u.fast;
    for (int i = tid; i < kFinishBins / 2; i += kThreads) fs.cs[i] = 0;
    if (tid == 0) fs.maxrun = 0;

    // encode once, in registers; AND / OR of the job
    Bits e[IU];
    Bits a = KT::ones(), o = KT::zero();
#pragma unroll
    for (int k = 0; k < IU; k++) {
        const int i = k * kThreads + tid;
        if (i < len) {
            e[k] = enc(skeys[ks + i]);
            a = a & e[k];
            o = o | e[k];
        }
    }
    block_and_or<KB>(a, o, s.sand, s.sor);
    const int f = KT::first_diff(a, o);
    if (f >= W) {
        // all keys equal: already in order
        if (job.buf == 1) {
            for (int i = tid; i < len; i += kThreads) {
                dst[i] = skeys[ks + i];
                if (VB) vdst[i] = svals[vs + i];
            }
        }
        return true;
    }

    // unstable 12-bit split at f: one shared-memory atomic per key
    uint32_t dr[IU];   // (digit << 16) | rank within the digit
#pragma unroll
    for (int k = 0; k < IU; k++) {
        const int i = k * kThreads + tid;
        const bool valid = i < len;
        const uint32_t d = valid ? KT::bits_at(e[k], f, kFinishBits) : 0u;
        const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
        const uint32_t sh = (d & 1) * 16;
        uint32_t r = 0;
        if (__all_sync(0xffffffffu, valid && d == d0)) {
            uint32_t c = 0;
            if (lane == 0) c = atomicAdd(&fs.cs[d0 >> 1], 32u << sh);
            r = ((__shfl_sync(0xffffffffu, c, 0) >> sh) & 0xffffu) + lane;
        } else if (valid) {
            r = (atomicAdd(&fs.cs[d >> 1], 1u << sh) >> sh) & 0xffffu;
        }
        dr[k] = (d << 16) | r;
    }
    __syncthreads();
    {
        constexpr int PW = kFinishBins / 2 / kThreads;   // words per thread
        uint32_t c[PW], sum = 0, mx = 0;
#pragma unroll
        for (int q = 0; q < PW; q++) {
            c[q] = fs.cs[tid * PW + q];
            const uint32_t lo = c[q] & 0xffffu, hi = c[q] >> 16;
            sum += lo + hi;
            mx = max(mx, max(lo, hi));
        }
        uint32_t total;
        uint32_t run = block_exclusive_scan(sum, fs.scratch, &total);   // all counts read
#pragma unroll
        for (int q = 0; q < PW; q++) {
            const uint32_t lo = c[q] & 0xffffu, hi = c[q] >> 16;
            fs.cs[2 * (tid * PW + q)] = run | (lo << 16);
            run += lo;
            fs.cs[2 * (tid * PW + q) + 1] = run | (hi << 16);
            run += hi;
        }
        if (mx > kFinishRun) atomicMax(&fs.maxrun, mx);
    }
    __syncthreads();
    if (fs.maxrun > (uint32_t)kFinishRun) return false;

    if constexpr (KB == 4 || KB == 8) {
        // Packed form: inside a run the keys agree on bits 0 .. f+11, so the
        // stable order of a run is the order of P = (e << (f + 12)) | input
        // position (only the position if the split reached the key's end).
        // P fits the key's width when the position needs at most f + 12 bits.
        const int sft = f + kFinishBits;
        const int nidx = 32 - __clz((uint32_t)(len - 1) | 1u);
        if (sft < W && nidx <= f) {
            // Jobs below the first levels (f >= the position's bits): the word
            // P = (key bits below f) << nidx | input position holds the whole
            // key below its common prefix, so it orders a run and also carries
            // the run's 12-bit digit (bits nidx + W - sft up): no digit array
            // to write at placement and read at ranking.
            Bits *sp = reinterpret_cast<Bits *>(s.keys);
            const int up = f - nidx;
#pragma unroll
            for (int k = 0; k < IU; k++) {
                const int i = k * kThreads + tid;
                if (i < len) {
                    const uint32_t d = dr[k] >> 16;
                    const uint32_t at = (fs.cs[d] & 0xffffu) + (dr[k] & 0xffffu);
                    if (at < (uint32_t)len) sp[at] = ((e[k] << f) >> up) | (Bits)i;
                    else set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
                }
            }
            __syncthreads();
            const Bits pre = a & (KT::ones() << (W - f));     // f >= nidx >= 1
            const Bits imask = ((Bits)1 << nidx) - 1;
            const int dsh = nidx + W - sft;
#pragma unroll 2
            for (int k = 0; k < IU; k++) {
                const int x = k * kThreads + tid;
                if (x < len) {
                    const Bits px = sp[x];
                    const uint32_t d = (uint32_t)(px >> dsh) & (uint32_t)(kFinishBins - 1);
                    const uint32_t bc = fs.cs[d];
                    const int b0 = (int)(bc & 0xffffu), m = (int)(bc >> 16);
                    int rank = 0;
#pragma unroll
                    for (int t = 0; t < 4; t++) {
                        const Bits py = sp[b0 + t];        // b0 + 3 <= len + 2: in the buffer
                        rank += (t < m && py < px) ? 1 : 0;
                    }
                    for (int y = b0 + 4; y < b0 + m; y++) rank += sp[y] < px ? 1 : 0;
                    uint32_t ix = (uint32_t)(px & imask);
                    if (ix >= (uint32_t)len) {
                        set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
                        ix = 0;
                    }
                    const int at = min(b0 + rank, len - 1);
                    dst[at] = dec(pre | (px >> nidx));
                    if (VB) vdst[at] = svals[vs + ix];
                }
            }
            return true;
        }
        if (sft >= W || nidx <= sft) {
            Bits *sp = reinterpret_cast<Bits *>(s.keys);
            uint16_t *sd = s.perm;
#pragma unroll
            for (int k = 0; k < IU; k++) {
                const int i = k * kThreads + tid;
                if (i < len) {
                    const uint32_t d = dr[k] >> 16;
                    const uint32_t at = (fs.cs[d] & 0xffffu) + (dr[k] & 0xffffu);
                    if (at < (uint32_t)len) {
                        sp[at] = (sft < W ? (e[k] << sft) : (Bits)0) | (Bits)i;
                        sd[at] = (uint16_t)d;
                    } else {
                        set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
                    }
                }
            }
            __syncthreads();
            // the bits above f are the job's common prefix
            const Bits pre = f ? (a & (KT::ones() << (W - f))) : (Bits)0;
            const Bits imask = ((Bits)1 << nidx) - 1;
            // no register arrays here: a loop unrolled twice keeps the code
            // small (fully unrolled, instruction fetch stalled the warps)
#pragma unroll 2
            for (int k = 0; k < IU; k++) {
                const int x = k * kThreads + tid;
                if (x < len) {
                    const Bits px = sp[x];
                    const uint32_t d = sd[x];
                    const uint32_t bc = fs.cs[d];
                    const int b0 = (int)(bc & 0xffffu), m = (int)(bc >> 16);
                    int rank = 0;
#pragma unroll
                    for (int t = 0; t < 4; t++) {
                        const Bits py = sp[b0 + t];        // b0 + 3 <= len + 2: in the buffer
                        rank += (t < m && py < px) ? 1 : 0;
                    }
                    for (int y = b0 + 4; y < b0 + m; y++) rank += sp[y] < px ? 1 : 0;
                    uint32_t ix = (uint32_t)(px & imask);
                    if (ix >= (uint32_t)len) {
                        set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
                        ix = 0;
                    }
                    const Bits ex = pre | (sft < W ? (((Bits)d << (W - sft)) | (px >> sft))
                                                   : ((Bits)d >> (sft - W)));
                    const int at = min(b0 + rank, len - 1);
                    dst[at] = dec(ex);
                    if (VB) vdst[at] = svals[vs + ix];
                }
            }
            return true;
        }
    }

    // place the encoded keys in split order (over the raw keys, all read), with
    // their input positions
    Bits *senc = reinterpret_cast<Bits *>(s.keys);
#pragma unroll
    for (int k = 0; k < IU; k++) {
        const int i = k * kThreads + tid;
        if (i < len) {
            const uint32_t at = (fs.cs[dr[k] >> 16] & 0xffffu) + (dr[k] & 0xffffu);
            if (at < (uint32_t)len) {
                senc[at] = e[k];
                s.perm[at] = (uint16_t)i;
            } else {
                set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
            }
        }
    }
    __syncthreads();
    // every key's place in its run: the run's keys that precede it in (encoded
    // key, input position) order; a fixed compare against the first four run
    // members, a loop for longer runs (rare); written straight to the output
#pragma unroll
    for (int k = 0; k < IU; k++) {
        const int x = k * kThreads + tid;
        if (x < len) {
            const Bits ex = senc[x];
            const uint32_t ix = s.perm[x];
            const uint32_t d = KT::bits_at(ex, f, kFinishBits);
            const uint32_t bc = fs.cs[d];
            const int b0 = (int)(bc & 0xffffu), m = (int)(bc >> 16);
            int rank = 0;
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const int y = min(b0 + t, len - 1);
                const Bits ey = senc[y];
                const uint32_t iy = s.perm[y];
                rank += ((t < m) && (KT::less(ey, ex) || (!KT::less(ex, ey) && iy < ix))) ? 1 : 0;
            }
            for (int y = b0 + 4; y < b0 + m; y++) {
                const Bits ey = senc[y];
                const uint32_t iy = s.perm[y];
                rank += (KT::less(ey, ex) || (!KT::less(ex, ey) && iy < ix)) ? 1 : 0;
            }
            const int at = min(b0 + rank, len - 1);
            dst[at] = dec(ex);
            if (VB) vdst[at] = svals[vs + ix];
        }
    }
    return true;
}

// IDENT: the key map is the identity (BINAR_MAP_UNSIGNED), known at compile time.
// Resident CTAs per SM the finisher's registers are sized for: 4 for keys
// without payload in classes of up to 16 items per thread (their shared memory
// leaves room; measured faster despite a few spilled registers), 3 up to 18
// items, 2 above.
template <int KB, int VB, int CLS, bool IDENT>
__global__ void __launch_bounds__(kThreads, (VB == 0 && FinishClasses<KB>::iu(CLS) <= 16)
                                                ? 4
                                                : (FinishClasses<KB>::iu(CLS) <= 18 ? 3 : 2))
    k_finish(Ws ws, Params p, void *keys0, void *keys1, void *vals0, void *vals1, int all_jobs) {
    pdl_entry();
    using KT = KeyTraits<KB>;
    using Raw = typename KT::Raw;
    using V = typename ValTraits<VB>::T;
    constexpr int IU = FinishClasses<KB>::iu(CLS);
    constexpr int W = KT::kW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &s = *reinterpret_cast<FinishSmem<KB, VB, IU> *>(smem_raw);
    Raw *skeys = reinterpret_cast<Raw *>(s.keys);
    V *svals = reinterpret_cast<V *>(s.vals);
    if (has_error(ws.ctr)) return;
    const Encoder<KB> enc(IDENT ? (int)BINAR_MAP_UNSIGNED : p.map);
    const Decoder<KB> dec(IDENT ? (int)BINAR_MAP_UNSIGNED : p.map);
    // all_jobs: this launch (of the smallest class that holds the call's
    // largest possible job) takes every job of the call straight from the
    // job list (small sorts: one launch instead of one per class); otherwise
    // the jobs of this class, listed in its region of jobidx
    const unsigned long long base = job_region(CLS, p.n, ws.jcap);
    const uint32_t count = all_jobs ? min(ws.ctr->njobs, ws.jcap) : ws.ctr->class_count[CLS];
    if (count == 0 || (!all_jobs && base + count > job_region(CLS + 1, p.n, ws.jcap))) return;
    const uint32_t *mine = all_jobs ? nullptr : ws.jobidx + base;
    const int tid = threadIdx.x;
    uint32_t phase = 0;
    if (tid == 0) {
        mbar_init(&s.bar);
        const uint32_t t = atomicAdd(&ws.ctr->class_ticket[CLS], 1u);
        s.next_ticket = t;
        if (t < count) s.next_job = ws.jobs[mine ? mine[t] : t];
    }
    for (;;) {
        __syncthreads();
        const uint32_t jt = s.next_ticket;
        if (jt >= count) break;
        const Job job = s.next_job;
        __syncthreads();
        const int len = (int)job.len;
        const Raw *src = reinterpret_cast<const Raw *>(job.buf ? keys1 : keys0) + job.begin;
        Raw *dst = reinterpret_cast<Raw *>(keys0) + job.begin;
        const V *vsrc = VB ? reinterpret_cast<const V *>(job.buf ? vals1 : vals0) + job.begin : nullptr;
        V *vdst = VB ? reinterpret_cast<V *>(vals0) + job.begin : nullptr;
        const bool trivial = job.pos >= W || len <= 1 || len > kThreads * IU;
        int ks = 0, vs = 0;
        if (!trivial) {   // the job's 16-byte chunks, by the bulk-copy engine
            uintptr_t ka0 = 0, va0 = 0;
            uint32_t kbytes = 0, vbytes = 0;
            ks = chunk_range<KB>(src, len, &ka0, &kbytes);
            if (VB) vs = chunk_range<VB>(vsrc, len, &va0, &vbytes);
            if (tid == 0) {
                bulk_begin(&s.bar, kbytes + vbytes);
                bulk_load(s.keys, ka0, kbytes, &s.bar);
                if (VB) bulk_load(s.vals, va0, vbytes, &s.bar);
            }
        }
        if (tid == 0) {   // the next job, while this one's data arrives
            const uint32_t t = atomicAdd(&ws.ctr->class_ticket[CLS], 1u);
            s.next_ticket = t;
            if (t < count) s.next_job = ws.jobs[mine ? mine[t] : t];
        }
        if (trivial) {
            if (len > kThreads * IU) {
                if (tid == 0) set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
            } else if (job.buf == 1) {
                for (int i = tid; i < len; i += kThreads) {
                    dst[i] = src[i];
                    if (VB) vdst[i] = vsrc[i];
                }
            }
            continue;
        }
        const bool landed = mbar_wait(&s.bar, phase, p.timeout_ns);
        if (__syncthreads_or(!landed)) {                  // uniform across the CTA
            if (tid == 0) set_status(ws.ctr, BINAR_ERR_DEVICE_TIMEOUT);
            if (!landed) mbar_wait(&s.bar, phase, p.timeout_ns);   // the copy in flight, bounded
            return;
        }
        phase ^= 1;
        if (!finish_fast<KB, VB, IU>(s, ws, enc, dec, job, ks, vs, dst, vdst) && tid == 0) {
            // runs too long for the fast path: the job goes to the LSD path
            const uint32_t ji = atomicAdd(&ws.ctr->njobs2, 1u);
            if (ji < ws.jcap) ws.jobs2[ji] = job;
            else set_status(ws.ctr, BINAR_ERR_QUEUE_OVERFLOW);
        }
    }
}

// ---------------------------------------------------------------------------
// finish_lsd: the jobs whose runs were too long for the fast path (heavy
// duplication), sorted by an LSD radix sort over 8-bit windows: the last
// window starts at pos and may overlap the one below it, windows whose bits
// are equal across the job are skipped, every pass is stable except the first
// one of a key-only sort.  The passes refine perm[sorted position] = input
// position over the keys and payloads staged in shared memory.
// ---------------------------------------------------------------------------
template <int KB, int VB>
struct FinishLsdSmem {
    static constexpr int T = TileShape<KB>::kTile;
    RankSmem rank;
    uint4 sand[kWarps], sor[kWarps];
    uint32_t ticket;
    alignas(16) unsigned char keys[T * KB];
    alignas(16) unsigned char vals[VB ? T * VB : 16];
    uint16_t perm[T];
};

template <int KB, int VB>
__global__ void __launch_bounds__(kThreads, 2)
    k_finish_lsd(Ws ws, Params p, void *keys0, void *keys1, void *vals0, void *vals1) {
    pdl_entry();
    using KT = KeyTraits<KB>;
    using Raw = typename KT::Raw;
    using Bits = typename KT::Bits;
    using V = typename ValTraits<VB>::T;
    constexpr int ITEMS = TileShape<KB>::kItems;
    constexpr int W = KT::kW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &s = *reinterpret_cast<FinishLsdSmem<KB, VB> *>(smem_raw);
    Raw *skeys = reinterpret_cast<Raw *>(s.keys);
    V *svals = reinterpret_cast<V *>(s.vals);
    if (has_error(ws.ctr)) return;
    const Encoder<KB> enc(p.map);
    const uint32_t njobs = min(ws.ctr->njobs2, ws.jcap);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (;;) {
        if (tid == 0) s.ticket = atomicAdd(&ws.ctr->ticket_fin2, 1u);
        __syncthreads();
        const uint32_t jt = s.ticket;
        __syncthreads();
        if (jt >= njobs) break;
        const Job job = ws.jobs2[jt];
        const int len = (int)job.len;
        const Raw *src = reinterpret_cast<const Raw *>(job.buf ? keys1 : keys0) + job.begin;
        Raw *dst = reinterpret_cast<Raw *>(keys0) + job.begin;
        const V *vsrc = VB ? reinterpret_cast<const V *>(job.buf ? vals1 : vals0) + job.begin : nullptr;
        V *vdst = VB ? reinterpret_cast<V *>(vals0) + job.begin : nullptr;
        for (int i = tid; i < len; i += kThreads) {
            cp_async<KB>(&skeys[i], &src[i]);
            if (VB) cp_async<VB ? VB : 4>(&svals[i], &vsrc[i]);
        }
        cp_async_wait_all();
        __syncthreads();
        Bits a = KT::ones(), o = KT::zero();
        for (int i = tid; i < len; i += kThreads) {
            const Bits x = enc(skeys[i]);
            a = a & x;
            o = o | x;
        }
        uint4 pa = KT::pack(a), po = KT::pack(o);
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            pa.x &= __shfl_xor_sync(0xffffffffu, pa.x, o2);
            pa.y &= __shfl_xor_sync(0xffffffffu, pa.y, o2);
            pa.z &= __shfl_xor_sync(0xffffffffu, pa.z, o2);
            pa.w &= __shfl_xor_sync(0xffffffffu, pa.w, o2);
            po.x |= __shfl_xor_sync(0xffffffffu, po.x, o2);
            po.y |= __shfl_xor_sync(0xffffffffu, po.y, o2);
            po.z |= __shfl_xor_sync(0xffffffffu, po.z, o2);
            po.w |= __shfl_xor_sync(0xffffffffu, po.w, o2);
        }
        if (lane == 0) {
            s.sand[w] = pa;
            s.sor[w] = po;
        }
        __syncthreads();
        uint4 ra = s.sand[0], ro = s.sor[0];
        for (int i = 1; i < kWarps; i++) {
            ra.x &= s.sand[i].x; ra.y &= s.sand[i].y; ra.z &= s.sand[i].z; ra.w &= s.sand[i].w;
            ro.x |= s.sor[i].x; ro.y |= s.sor[i].y; ro.z |= s.sor[i].z; ro.w |= s.sor[i].w;
        }
        const Bits diff_a = KT::unpack(ra), diff_o = KT::unpack(ro);
        const int iu = (len + kThreads - 1) / kThreads;
        int q = W - kBits;
        bool moved = false;
        Packed<ITEMS> pk;
        uint32_t src_pos[(ITEMS + 1) / 2];
        for (;;) {
            const int qq = q > (int)job.pos ? q : (int)job.pos;
            const bool varies = KT::digit(diff_a, qq) != KT::digit(diff_o, qq);
            if (varies) {
                __syncthreads();
#pragma unroll
                for (int j = 0; j < ITEMS; j++) {
                    if (j < iu) {
                        const int i = striped(iu, j);
                        uint32_t x = 0;
                        if (i < len) x = moved ? s.perm[i] : (uint32_t)i;
                        if (x >= (uint32_t)len) {
                            set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
                            x = 0;
                        }
                        if ((j & 1) == 0) src_pos[j >> 1] = x;
                        else src_pos[j >> 1] |= x << 16;
                        pk.set_dig(j, i < len ? KT::digit(enc(skeys[x]), qq) : 0u);
                    }
                }
                if (VB || moved) rank_stable<ITEMS>(pk, iu, len, s.rank);
                else rank_unstable<ITEMS>(pk, iu, len, s.rank);
#pragma unroll
                for (int j = 0; j < ITEMS; j++) {
                    if (j < iu && striped(iu, j) < len) {
                        const uint32_t r = pk.rank(j);
                        if (r < (uint32_t)len)
                            s.perm[r] = (uint16_t)(src_pos[j >> 1] >> ((j & 1) * 16));
                        else
                            set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
                    }
                }
                moved = true;
            }
            if (qq == (int)job.pos) break;
            q -= kBits;
        }
        __syncthreads();
        for (int x = tid; x < len; x += kThreads) {
            const int i = moved ? min((int)s.perm[x], len - 1) : x;
            dst[x] = skeys[i];
            if (VB) vdst[x] = svals[i];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// copy: finished buckets larger than the cutoff that sit in the workspace
// arrays go back to the caller's arrays.  Tiles by ticket; the job of a tile is
// found by binary search on tile_start (increasing with the job index).
// ---------------------------------------------------------------------------
// Copies count elements by the whole CTA: 16-byte vectors when source and
// destination share their alignment modulo 16 (after a scalar head up to the
// boundary), scalar otherwise and for the tail.
template <typename E>
__device__ __forceinline__ void copy_range(E *dst, const E *src, long long count) {
    const uintptr_t d = reinterpret_cast<uintptr_t>(dst), s = reinterpret_cast<uintptr_t>(src);
    long long head = count;
    if (((d ^ s) & 15) == 0) head = min(count, (long long)(((16 - (d & 15)) & 15) / sizeof(E)));
    for (long long i = threadIdx.x; i < head; i += kThreads) dst[i] = src[i];
    const long long nvec = (count - head) * (long long)sizeof(E) / 16;
    uint4 *dv = reinterpret_cast<uint4 *>(dst + head);
    const uint4 *sv = reinterpret_cast<const uint4 *>(src + head);
#pragma unroll 4
    for (long long v = threadIdx.x; v < nvec; v += kThreads) dv[v] = __ldg(sv + v);
    for (long long i = head + nvec * (16 / (long long)sizeof(E)) + threadIdx.x; i < count;
         i += kThreads)
        dst[i] = src[i];
}

// Writes `count` copies of v by the whole CTA: 16-byte vectors of v from the
// first 16-byte boundary (after a scalar head), scalar for the tail.
template <typename E>
__device__ __forceinline__ void fill_range(E *dst, const E &v, long long count) {
    static_assert(16 % sizeof(E) == 0, "element size divides 16");
    constexpr int PER = 16 / (int)sizeof(E);
    const uintptr_t d = reinterpret_cast<uintptr_t>(dst);
    const long long head = min(count, (long long)(((16 - (d & 15)) & 15) / sizeof(E)));
    for (long long i = threadIdx.x; i < head; i += kThreads) dst[i] = v;
    union {
        E e[PER];
        uint4 u;
    } w;
#pragma unroll
    for (int q = 0; q < PER; q++) w.e[q] = v;
    const long long nvec = (count - head) / PER;
    uint4 *dv = reinterpret_cast<uint4 *>(dst + head);
    for (long long i = threadIdx.x; i < nvec; i += kThreads) dv[i] = w.u;
    for (long long i = head + nvec * PER + threadIdx.x; i < count; i += kThreads) dst[i] = v;
}

// T: the call's tile (copy jobs are cut into tiles of the partition's size).
template <int KB, int VB>
__global__ void __launch_bounds__(kThreads) k_copy(Ws ws, int T, void *keys0, void *keys1,
                                                   void *vals0, void *vals1) {
    pdl_entry();
    using Raw = typename KeyTraits<KB>::Raw;
    using V = typename ValTraits<VB>::T;
    __shared__ uint32_t sticket;
    if (has_error(ws.ctr)) return;
    const unsigned long long ca = ws.ctr->copy_alloc;
    const uint32_t nj = min((uint32_t)ca, ws.ccap), nt = (uint32_t)(ca >> 32);
    for (;;) {
        if (threadIdx.x == 0) sticket = atomicAdd(&ws.ctr->ticket_copy, 1u);
        __syncthreads();
        const uint32_t t = sticket;
        __syncthreads();
        if (t >= nt || nj == 0) break;
        uint32_t lo = 0, hi = nj - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) / 2;
            if (ws.copies[mid].tile_start <= t) lo = mid;
            else hi = mid - 1;
        }
        const CopyJob cj = ws.copies[lo];
        const long long cb = cj.begin & kCopyBeginMask;
        const long long len = (long long)cj.len;
        const long long j0 = (long long)(t - cj.tile_start) * T;      // job-relative
        const long long j1 = min(j0 + T, len);
        const bool rev = (cj.begin & kCopyReverse) != 0;
        const bool inplace = (cj.begin & kCopyInPlace) != 0;
        const bool fill = (cj.begin & kCopyFill) != 0;
        Raw *dst = reinterpret_cast<Raw *>(keys0) + cb;
        V *vdst = VB ? reinterpret_cast<V *>(vals0) + cb : nullptr;
        if (!rev) {
            // from the workspace arrays, straight
            if (fill)      // all keys equal: the first one, written over the range
                fill_range<Raw>(dst + j0, reinterpret_cast<const Raw *>(keys1)[cb], j1 - j0);
            else
                copy_range<Raw>(dst + j0, reinterpret_cast<const Raw *>(keys1) + cb + j0, j1 - j0);
            if (VB) copy_range<V>(vdst + j0, reinterpret_cast<const V *>(vals1) + cb + j0, j1 - j0);
        } else if (!inplace) {
            // from the workspace arrays, reversed
            const Raw *src = reinterpret_cast<const Raw *>(keys1) + cb;
            const V *vsrc = VB ? reinterpret_cast<const V *>(vals1) + cb : nullptr;
            for (long long i = j0 + threadIdx.x; i < j1; i += kThreads) {
                dst[len - 1 - i] = src[i];
                if (VB) vdst[len - 1 - i] = vsrc[i];
            }
        } else {
            // reversed in place: the thread of position i < len-1-i swaps the pair
            for (long long i = j0 + threadIdx.x; i < j1; i += kThreads) {
                const long long k = len - 1 - i;
                if (i < k) {
                    const Raw x = dst[i];
                    dst[i] = dst[k];
                    dst[k] = x;
                    if (VB) {
                        const V y = vdst[i];
                        vdst[i] = vdst[k];
                        vdst[k] = y;
                    }
                }
            }
        }
    }
}

}  // namespace binar
