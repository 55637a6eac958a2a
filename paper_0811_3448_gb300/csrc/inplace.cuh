// inplace.cuh -- the in-place, unstable mode of libbinar: the paper's own
// form of the partition step ("Partition Array into Sub-arrays": one bit at
// a time, elements exchanged between the lower and the upper sub-array,
// nothing moved through a second array; "Space Analysis": the array plus a
// constant per call), run for every live sub-array ("bucket") of a level at
// once.
//
// For a bucket [lo, hi) split on bit `pos`, the histogram pass has counted
// its z keys with bit 0, so the split point mid = lo + z is known before any
// key moves.  A key is misplaced if its bit is 1 left of mid or 0 right of
// it; the two counts are equal.  The paper's exchange pairs a misplaced key
// of the lower part with one of the upper part; here the k-th misplaced key
// left of mid (in position order) is exchanged with the k-th misplaced key
// right of it:
//   count  per tile of kIpTile keys: one bit per key marking it misplaced
//          (warp ballots), and the tile's misplaced keys left / right of mid
//   scan   exclusive prefix of both counts over all tiles of the level, in
//          tile order; tiles are numbered bucket by bucket and every bucket
//          holds as many misplaced keys on each side, so the k-th misplaced
//          key on the left and on the right of the level (global ranks) lie
//          in the same bucket
//   swap   per chunk of kIpChunk ranks: the positions of those ranks on both
//          sides are read off the marker bits (never off the keys, which the
//          other chunks are exchanging meanwhile), then every pair is
//          exchanged by one thread, so no two threads touch one key
// Keys (and payloads) never leave the caller's arrays; the scratch is one
// bit per key and a few words per tile, per bucket and per finisher job.
#pragma once

#include "kernels.cuh"

namespace binar {

constexpr int kIpTile = 4096;                 // keys per tile of the in-place passes
constexpr int kIpWords = kIpTile / 32;        // marker words per tile (four per lane of a warp)
constexpr int kIpScanItems = 8;
constexpr int kIpScanTile = kThreads * kIpScanItems;   // tiles per scan block

struct IpWs {
    uint32_t *mask;              // [tile][kIpWords]: bit i set = key i of the tile is misplaced
    uint32_t *cnt;               // [tile][2]: misplaced keys left / right of the bucket's mid
    uint32_t *pre;               // [tile][2]: exclusive prefix of cnt over the level's tiles
    uint32_t *bsum;              // [scan block][2]
    unsigned long long *total;   // [2]: misplaced keys of the level, left / right
    uint32_t *first;             // [2][chunk]: the tile holding the chunk's first rank, per side
    long long chunk_cap;         // entries per side of `first`
    long long *tinfo;            // [tile][2]: the tile's first key position and its bucket's mid
};

// Bucket b's split point (its bit-0 keys come first): after classify, its
// histogram row holds the exclusive prefix, so entry 1 is the bit-0 count.
__device__ __forceinline__ long long ip_mid(const Ws &ws, int slot, uint32_t b, const Bucket &bk) {
    const uint32_t *h = slot ? ws.hist[1] : ws.hist[0];
    return bk.begin + (long long)h[(size_t)b * kRadix + 1];
}

// One warp per tile, no block barriers: the warp loads BATCH words' keys at
// once, ballots the misplaced bits, and lanes 0..BATCH-1 store the words.
template <int KB, bool IDENT>
__global__ void __launch_bounds__(kThreads) k_ip_count(Ws ws, Params p, int slot, IpWs ip) {
    pdl_entry();
    using KT = KeyTraits<KB>;
    using Raw = typename KT::Raw;
    constexpr int BATCH = KB == 16 ? 8 : 16;
    if (has_error(ws.ctr)) return;
    const Encoder<KB> enc(IDENT ? (int)BINAR_MAP_UNSIGNED : p.map);
    const Bucket *list = slot ? ws.list[1] : ws.list[0];
    const unsigned long long alloc = slot ? ws.ctr->alloc[1] : ws.ctr->alloc[0];
    const long long nt = (long long)(alloc >> 32);
    const int lane = threadIdx.x & 31;
    const Raw *keys = reinterpret_cast<const Raw *>(p.keys);
    const long long nw = (long long)gridDim.x * kWarps;
    for (long long t = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); t < nt; t += nw) {
        const uint32_t b = ws.tilemap[t];
        const Bucket bk = list[b];
        uint32_t cl = 0, cr = 0;
        long long tb = 0, mid = 0;
        uint32_t *mw = ip.mask + (size_t)t * kIpWords;
        if (!(bk.flags & kSkip)) {
            tb = bk.begin + (t - (long long)bk.tile_start) * kIpTile;
            const int tlen = (int)min((long long)kIpTile, bk.begin + (long long)bk.len - tb);
            mid = ip_mid(ws, slot, b, bk);
            for (int w0 = 0; w0 < kIpWords; w0 += BATCH) {
                Raw kx[BATCH];
#pragma unroll
                for (int q = 0; q < BATCH; q++) {
                    const int i = (w0 + q) * 32 + lane;
                    kx[q] = i < tlen ? keys[tb + i] : Raw{};
                }
                uint32_t mine = 0;
#pragma unroll
                for (int q = 0; q < BATCH; q++) {
                    const int i = (w0 + q) * 32 + lane;
                    const bool valid = i < tlen;
                    const bool left = valid && tb + i < mid;
                    const uint32_t bit = KT::bits_at(enc(kx[q]), bk.pos, 1);
                    const bool mis = valid && (left ? bit != 0 : bit == 0);
                    const uint32_t word = __ballot_sync(0xffffffffu, mis);
                    const uint32_t lw = __ballot_sync(0xffffffffu, left);
                    if (lane == q) mine = word;
                    cl += __popc(word & lw);
                    cr += __popc(word & ~lw);
                }
                if (lane < BATCH) mw[w0 + lane] = mine;
            }
        } else {
#pragma unroll
            for (int q = 0; q < kIpWords / 32; q++) mw[q * 32 + lane] = 0u;
        }
        if (lane == 0) {
            ip.cnt[2 * t] = cl;
            ip.cnt[2 * t + 1] = cr;
            ip.tinfo[2 * t] = tb;
            ip.tinfo[2 * t + 1] = mid;
        }
    }
}

// Exclusive scan of the (left, right) counts over the level's tiles, in three
// kernels: per-block sums, one CTA scanning them, per-tile prefixes.
static __global__ void __launch_bounds__(kThreads) k_ip_scan_sums(Ws ws, int slot, IpWs ip) {
    pdl_entry();
    __shared__ uint32_t red[2][kWarps];
    if (has_error(ws.ctr)) return;
    const unsigned long long alloc = slot ? ws.ctr->alloc[1] : ws.ctr->alloc[0];
    const long long nt = (long long)(alloc >> 32);
    const long long nblk = (nt + kIpScanTile - 1) / kIpScanTile;
    for (long long c = blockIdx.x; c < nblk; c += gridDim.x) {
        uint32_t a = 0, b = 0;
        for (int k = 0; k < kIpScanItems; k++) {
            const long long t = c * kIpScanTile + (long long)k * kThreads + threadIdx.x;
            if (t < nt) {
                a += ip.cnt[2 * t];
                b += ip.cnt[2 * t + 1];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = a;
            red[1][threadIdx.x >> 5] = b;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            uint32_t sum = 0;
            for (int i = 0; i < kWarps; i++) sum += red[threadIdx.x][i];
            ip.bsum[2 * c + threadIdx.x] = sum;
        }
        __syncthreads();
    }
}

static __global__ void __launch_bounds__(kThreads) k_ip_scan_blocks(Ws ws, int slot, IpWs ip) {
    pdl_entry();
    __shared__ uint32_t scratch[kWarps];
    if (has_error(ws.ctr)) return;
    const unsigned long long alloc = slot ? ws.ctr->alloc[1] : ws.ctr->alloc[0];
    const long long nt = (long long)(alloc >> 32);
    const long long nblk = (nt + kIpScanTile - 1) / kIpScanTile;
    for (int side = 0; side < 2; side++) {
        unsigned long long carry = 0;
        for (long long base = 0; base < nblk; base += kThreads) {
            const long long c = base + threadIdx.x;
            const uint32_t v = c < nblk ? ip.bsum[2 * c + side] : 0u;
            uint32_t total;
            const uint32_t ex = block_exclusive_scan(v, scratch, &total);
            if (c < nblk) ip.bsum[2 * c + side] = (uint32_t)carry + ex;
            carry += total;
        }
        if (threadIdx.x == 0) ip.total[side] = carry;
    }
}

static __global__ void __launch_bounds__(kThreads) k_ip_scan_apply(Ws ws, int slot, IpWs ip) {
    pdl_entry();
    __shared__ uint32_t scratch[kWarps];
    if (has_error(ws.ctr)) return;
    const unsigned long long alloc = slot ? ws.ctr->alloc[1] : ws.ctr->alloc[0];
    const long long nt = (long long)(alloc >> 32);
    const long long nblk = (nt + kIpScanTile - 1) / kIpScanTile;
    for (long long c = blockIdx.x; c < nblk; c += gridDim.x) {
        // thread-contiguous items keep the prefix in tile order
        const long long t0 = c * kIpScanTile + (long long)threadIdx.x * kIpScanItems;
        for (int side = 0; side < 2; side++) {
            uint32_t v[kIpScanItems], sum = 0;
#pragma unroll
            for (int k = 0; k < kIpScanItems; k++) {
                v[k] = (t0 + k < nt) ? ip.cnt[2 * (t0 + k) + side] : 0u;
                sum += v[k];
            }
            uint32_t total;
            uint32_t run = ip.bsum[2 * c + side] + block_exclusive_scan(sum, scratch, &total);
#pragma unroll
            for (int k = 0; k < kIpScanItems; k++) {
                if (t0 + k < nt) {
                    ip.pre[2 * (t0 + k) + side] = run;
                    // the tile holds ranks [run, run + v): it is the first tile
                    // of every swap chunk whose first rank falls there
                    for (uint32_t q = (run + kIpChunk - 1) / kIpChunk; v[k] && q * kIpChunk < run + v[k];
                         q++)
                        if ((long long)q < ip.chunk_cap) ip.first[side * ip.chunk_cap + q] = (uint32_t)(t0 + k);
                }
                run += v[k];
            }
        }
    }
}

// Exchanges the k-th misplaced key left of mid with the k-th right of it,
// chunk by chunk of ranks.  Positions are taken from the marker bits (a warp
// per tile, four words per lane); a chunk's positions start as -1 and a pair
// with a missing or foreign position is reported (BINAR_ERR_DEVICE_BOUNDS)
// and skipped.  Each thread loads its pairs before storing them.
template <int KB, int VB>
__global__ void __launch_bounds__(kThreads, 4) k_ip_swap(Ws ws, Params p, int slot, IpWs ip) {
    pdl_entry();
    using Raw = typename KeyTraits<KB>::Raw;
    using V = typename ValTraits<VB>::T;
    constexpr int PER = kIpChunk / kThreads;              // pairs per thread
    __shared__ int pos[2][kIpChunk];       // key positions (n < 2^31)
    __shared__ uint32_t sfirst;
    __shared__ uint32_t sscan[kWarps];
    if (has_error(ws.ctr)) return;
    const unsigned long long alloc = slot ? ws.ctr->alloc[1] : ws.ctr->alloc[0];
    const uint32_t nt = (uint32_t)(alloc >> 32);
    const unsigned long long mtot = ip.total[0];
    if (mtot != ip.total[1]) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
        return;
    }
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    Raw *keys = reinterpret_cast<Raw *>(p.keys);
    V *vals = VB ? reinterpret_cast<V *>(p.vals) : nullptr;
    const unsigned long long nchunks = (mtot + kIpChunk - 1) / kIpChunk;
    for (unsigned long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const unsigned long long lo = c * kIpChunk;
        const unsigned long long hi = min(lo + (unsigned long long)kIpChunk, mtot);
        for (int i = tid; i < 2 * kIpChunk; i += kThreads) (&pos[0][0])[i] = -1;
        for (int side = 0; side < 2; side++) {
            if (tid == 0) {              // the tile holding rank lo (recorded by the scan)
                const uint32_t f = (long long)c < ip.chunk_cap ? ip.first[side * ip.chunk_cap + c] : 0u;
                sfirst = f < nt ? f : 0u;
            }
            __syncthreads();
            // the tiles holding ranks [lo, hi) on this side, one at a time,
            // their 4096 marker bits spread over the CTA (16 per thread): a
            // block scan of the popcounts gives every bit its rank, and each
            // thread records the positions of its bits whose ranks are the
            // chunk's.  Tiles without marked keys on this side are passed over.
            for (uint32_t t = sfirst; t < nt; t++) {
                const unsigned long long r0 = ip.pre[2 * (size_t)t + side];    // uniform
                if (r0 >= hi) break;
                if (ip.cnt[2 * (size_t)t + side] == 0) continue;                // uniform
                const long long tb = ip.tinfo[2 * (size_t)t], mid = ip.tinfo[2 * (size_t)t + 1];
                const uint32_t word = ip.mask[(size_t)t * kIpWords + (tid >> 1)];
                uint32_t bits = (word >> ((tid & 1) * 16)) & 0xffffu;
                const long long wb = tb + (long long)tid * 16;
                const long long cut = mid - wb;             // bits below cut lie left of mid
                const uint32_t low = cut >= 16 ? 0xffffu : (cut <= 0 ? 0u : ((1u << cut) - 1u));
                bits &= side == 0 ? low : (~low & 0xffffu);
                uint32_t total;
                const uint32_t nb = (uint32_t)__popc(bits);
                unsigned long long r = r0 + block_exclusive_scan(nb, sscan, &total);
                if (r < hi && r + nb > lo) {
                    while (bits) {
                        const int j = __ffs(bits) - 1;
                        bits &= bits - 1;
                        if (r >= lo && r < hi) pos[side][r - lo] = (int)(wb + j);
                        r++;
                    }
                }
            }
            __syncthreads();
        }
        const int m = (int)(hi - lo);
        long long a[PER], z[PER];
        bool ok[PER];
#pragma unroll
        for (int q = 0; q < PER; q++) {
            const int j = q * kThreads + tid;
            ok[q] = false;
            if (j < m) {
                a[q] = pos[0][j];
                z[q] = pos[1][j];
                ok[q] = a[q] >= 0 && z[q] >= 0 && a[q] < p.n && z[q] < p.n && a[q] < z[q];
                if (!ok[q]) set_status(ws.ctr, BINAR_ERR_DEVICE_BOUNDS);
            }
        }
        Raw ka[PER], kz[PER];
        V va[PER], vz[PER];
#pragma unroll
        for (int q = 0; q < PER; q++) {
            if (ok[q]) {
                ka[q] = keys[a[q]];
                kz[q] = keys[z[q]];
                if (VB) {
                    va[q] = vals[a[q]];
                    vz[q] = vals[z[q]];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < PER; q++) {
            if (ok[q]) {
                keys[a[q]] = kz[q];
                keys[z[q]] = ka[q];
                if (VB) {
                    vals[a[q]] = vz[q];
                    vals[z[q]] = va[q];
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace binar
