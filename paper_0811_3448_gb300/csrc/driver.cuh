// driver.cuh -- host side of libbinar: workspace layout and the level loop
// that runs the recursion of binar sort as a fixed sequence of kernel
// launches ("Algorithm Variants": the recursion replaced by iteration, each
// level handling every live sub-array at once).  Everything is enqueued on the
// caller's stream; nothing allocates or synchronises.
#pragma once

#include <type_traits>
#include <utility>

#include "inplace.cuh"
#include "kernels.cuh"
#include "layout.cuh"
#include "tail.cuh"

namespace binar {

// Grids are persistent (occupancy x SMs) but never larger than the work a
// call of n keys can hold, so that small sorts do not launch idle CTAs.
inline int cap_grid(long long grid, long long work) {
    if (work < 1) work = 1;
    return (int)(grid < work ? grid : work);
}

// Tiles per histogram ticket for a level of at most `tiles` tiles on a
// persistent grid of `full` CTAs: kHistGroup once every CTA gets a group,
// fewer below that (down to one tile per ticket).
inline int hist_group(long long tiles, long long full) {
    const long long g = tiles / (full > 0 ? full : 1);
    return (int)(g < 1 ? 1 : (g > kHistGroup ? kHistGroup : g));
}

template <int KB, int VB, bool STABLE, int TV>
int launch_partition(const Call &c, const Ws &ws, const Params &p, int slot, int level,
                     void *k0, void *k1, void *v0, void *v1, long long max_tiles) {
    auto kfn = p.map == BINAR_MAP_UNSIGNED ? k_partition<KB, VB, STABLE, true, TV>
                                           : k_partition<KB, VB, STABLE, false, TV>;
    const size_t smem = sizeof(PartitionSmem<KB, VB, STABLE, TV>);
    int occ = kernel_ctas_per_sm((const void *)kfn, smem);
    if (c.ctas_per_sm > 0 && c.ctas_per_sm < occ) occ = c.ctas_per_sm;
    const int grid = cap_grid((long long)device_sms() * (occ > 0 ? occ : 1), max_tiles);
    return launch("partition", level, c.stream, [&] {
        launch_pdl(kfn, grid, kThreads, smem, c.stream, ws, p, slot, level, k0, k1, v0, v1);
    });
}

// Sorts of at most this many keys finish every job in one launch, of the
// smallest class that holds the largest job the call can have, instead of one
// launch per class (fewer launches; idle items in smaller jobs cost little at
// that size).
constexpr long long kOneFinishLaunchMaxN = 1LL << 21;

template <int KB, int VB, int CLS>
int launch_finish_class(const Call &c, const Ws &ws, const Params &p, void *k0, void *k1, void *v0,
                        void *v1, int all_jobs = 0) {
    constexpr int IU = FinishClasses<KB>::iu(CLS);
    // a job holds at most min(cutoff, n) keys: larger classes never get one
    const long long maxjob = c.cutoff < c.n ? c.cutoff : c.n;
    if (!all_jobs && CLS > 0 && (long long)kThreads * FinishClasses<KB>::iu(CLS > 0 ? CLS - 1 : 0) >= maxjob)
        return BINAR_OK;
    // the identity key map is compiled separately for 4- and 8-byte keys
    auto ffn = (KB != 16 && c.map == BINAR_MAP_UNSIGNED) ? k_finish<KB, VB, CLS, KB != 16>
                                                         : k_finish<KB, VB, CLS, false>;
    const size_t smem = sizeof(FinishSmem<KB, VB, IU>);
    const int occ = kernel_ctas_per_sm((const void *)ffn, smem);
    // jobs of this class hold more keys than the class below it can
    const long long lower = (CLS > 0 && !all_jobs) ? (long long)kThreads * FinishClasses<KB>::iu(CLS > 0 ? CLS - 1 : 0) : 1;
    // an unsegmented call of at most `cutoff` keys has at most one job
    const long long jobs_max = (all_jobs && !c.offsets && c.n <= c.cutoff) ? 1 : c.n / (lower + 1) + 1;
    const int grid = cap_grid((long long)device_sms() * (occ > 0 ? occ : 1), jobs_max);
    return launch("finish", CLS, c.stream, [&] {
        launch_pdl(ffn, grid, kThreads, smem, c.stream, ws, p, k0, k1, v0, v1, all_jobs);
    });
}

template <int KB, int VB, int... CLS>
int launch_finish_classes(const Call &c, const Ws &ws, const Params &p, void *k0, void *k1,
                          void *v0, void *v1, std::integer_sequence<int, CLS...>) {
    int rc = BINAR_OK;
    if (c.n <= kOneFinishLaunchMaxN) {
        // one launch, of the smallest class that holds min(cutoff, n) keys
        const long long maxjob = c.cutoff < c.n ? c.cutoff : c.n;
        bool launched = false;
        auto one = [&](auto cls) {
            constexpr int C = decltype(cls)::value;
            if (launched || (C + 1 < FinishClasses<KB>::kCount &&
                             (long long)kThreads * FinishClasses<KB>::iu(C) < maxjob))
                return;
            launched = true;
            rc = launch_finish_class<KB, VB, C>(c, ws, p, k0, k1, v0, v1, 1);
        };
        (one(std::integral_constant<int, CLS>{}), ...);
        return rc;
    }
    ((rc = rc ? rc : launch_finish_class<KB, VB, CLS>(c, ws, p, k0, k1, v0, v1)), ...);
    return rc;
}

// Sorts of at most this many keys with the default tile shape run the levels
// after the first as one cooperative launch (tail.cuh), which ends at the
// first level without a bucket.
constexpr long long kTailMaxN = 1LL << 21;
constexpr int kTailUnavailable = -1;

// Launches levels first .. levels-1 as one cooperative grid; kTailUnavailable
// (nothing enqueued) when the device cannot make that grid resident, so the
// caller enqueues the levels one kernel at a time.
template <int KB, int VB>
int launch_levels_tail(const Call &c, const Ws &ws, const Params &p, int first, int levels,
                       long long max_tiles, void *k0, void *k1, void *v0, void *v1) {
    auto fn = (KB != 16 && c.map == BINAR_MAP_UNSIGNED) ? k_levels_tail<KB, VB, KB != 16>
                                                        : k_levels_tail<KB, VB, false>;
    const size_t smem = sizeof(PartitionSmem<KB, VB, (VB > 0), 0>);
    const int occ = kernel_ctas_per_sm((const void *)fn, smem);
    const int sms = device_sms();
    if (occ < 1 || sms < 1) return kTailUnavailable;
    const int grid = cap_grid((long long)sms * occ, max_tiles);
    const int hgroup = hist_group(max_tiles, grid);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    bool refused = false;
    const int rc = launch("levels", first, c.stream, [&] {
        const cudaError_t e = cudaLaunchKernelEx(&cfg, fn, ws, p, first, levels, hgroup, k0, k1, v0, v1);
        if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
            cudaGetLastError();            // not an error of the call: one kernel per phase instead
            refused = true;
        }
    });
    return refused ? kTailUnavailable : rc;
}

// The in-place, unstable mode: one bit per level, keys exchanged across each
// bucket's split point inside the caller's arrays (inplace.cuh), buckets of
// at most `cutoff` keys finished in shared memory and written back in place.
template <int KB, int VB>
int run_inplace(const Call &c) {
    const int sms = device_sms();
    if (sms <= 0) return BINAR_ERR_CUDA;
    const InplaceLayout IL = make_inplace_layout(c.n, KB, c.cutoff);
    Ws ws = carve(IL.base, c.ws);
    ws.cells = nullptr;            // no look-back cells (and none allocated)
    ws.alt_keys = nullptr;         // no second array
    ws.alt_vals = nullptr;
    unsigned char *wb = static_cast<unsigned char *>(c.ws);
    IpWs ip;
    ip.mask = reinterpret_cast<uint32_t *>(wb + IL.mask);
    ip.cnt = reinterpret_cast<uint32_t *>(wb + IL.cnt);
    ip.pre = reinterpret_cast<uint32_t *>(wb + IL.pre);
    ip.bsum = reinterpret_cast<uint32_t *>(wb + IL.bsum);
    ip.total = reinterpret_cast<unsigned long long *>(wb + IL.total);
    ip.first = reinterpret_cast<uint32_t *>(wb + IL.first);
    ip.tinfo = reinterpret_cast<long long *>(wb + IL.tinfo);
    ip.chunk_cap = IL.chunks;
    Params p{};
    p.keys = c.keys;
    p.vals = c.vals;
    p.map = c.map;
    p.n = c.n;
    p.cutoff = c.cutoff;
    p.timeout_ns = c.timeout_ns;
    p.skip_publish_tile = -1;
    p.tile = kIpTile;
    p.bits = 1;
    p.inplace = 1;
    const int L = levels_for(KB, 1);
    const int small_grid = sms * 4;
    const long long max_buckets = c.n / ((long long)c.cutoff + 1) + 1;
    const long long max_tiles = c.n / kIpTile + max_buckets + 1;
    void *k0 = c.keys, *v0 = c.vals;
    int rc;
    if ((rc = launch("init", -1, c.stream, [&] {
             launch_pdl(k_init<KB>, 1, 1, 0, c.stream, ws, c.n, c.cutoff, 0,
                        (uint32_t)((c.n + kIpTile - 1) / kIpTile), 1);
         })))
        return rc;
    if (c.n > c.cutoff) {
        auto hfn = c.map == BINAR_MAP_UNSIGNED ? k_hist<KB, true> : k_hist<KB, false>;
        auto cfn = c.map == BINAR_MAP_UNSIGNED ? k_ip_count<KB, true> : k_ip_count<KB, false>;
        const int hocc = kernel_ctas_per_sm((const void *)hfn, 0);
        const long long hfull = (long long)sms * (hocc > 0 ? hocc : 1);
        const int hgroup = hist_group(max_tiles, hfull);
        const int hgrid = cap_grid(hfull, max_tiles / hgroup + 1);
        const int pgrid = cap_grid(small_grid, max_buckets > max_tiles / 4 ? max_buckets : max_tiles / 4);
        const int cgrid = cap_grid(small_grid, max_buckets);
        const int tgrid = cap_grid((long long)sms * 8, max_tiles / kWarps + 1);   // a warp per tile
        const int sgrid = cap_grid(small_grid, max_tiles / kIpScanTile + 1);
        const int wgrid = cap_grid((long long)sms * 8, c.n / (2LL * kIpChunk) + 1);
        for (int l = 0; l < L; l++) {
            const int slot = l & 1;
            if ((rc = launch("prep", l, c.stream, [&] {
                     launch_pdl(k_prep, pgrid, kThreads, 0, c.stream, ws, slot);
                 })))
                return rc;
            if ((rc = launch("hist", l, c.stream, [&] {
                     launch_pdl(hfn, hgrid, kThreads, 0, c.stream, ws, p, slot, hgroup);
                 })))
                return rc;
            if ((rc = launch("classify", l, c.stream, [&] {
                     launch_pdl(k_classify<KB>, cgrid, kThreads, 0, c.stream, ws, p, slot, l == L - 1);
                 })))
                return rc;
            if ((rc = launch("ip_count", l, c.stream, [&] {
                     launch_pdl(cfn, tgrid, kThreads, 0, c.stream, ws, p, slot, ip);
                 })))
                return rc;
            if ((rc = launch("ip_scan", l, c.stream, [&] {
                     launch_pdl(k_ip_scan_sums, sgrid, kThreads, 0, c.stream, ws, slot, ip);
                     launch_pdl(k_ip_scan_blocks, 1, kThreads, 0, c.stream, ws, slot, ip);
                     launch_pdl(k_ip_scan_apply, sgrid, kThreads, 0, c.stream, ws, slot, ip);
                 })))
                return rc;
            if ((rc = launch("ip_swap", l, c.stream, [&] {
                     launch_pdl(k_ip_swap<KB, VB>, wgrid, kThreads, 0, c.stream, ws, p, slot, ip);
                 })))
                return rc;
        }
    }
    if ((rc = launch_finish_classes<KB, VB>(c, ws, p, k0, k0, v0, v0,
                                             std::make_integer_sequence<int, FinishClasses<KB>::kCount>{})))
        return rc;
    auto lfn = k_finish_lsd<KB, VB>;
    const size_t lsmem = sizeof(FinishLsdSmem<KB, VB>);
    const int locc = kernel_ctas_per_sm((const void *)lfn, lsmem);
    if ((rc = launch("finish_lsd", -1, c.stream, [&] {
             launch_pdl(lfn, cap_grid((long long)sms * (locc > 0 ? locc : 1), c.n / 33 + 1), kThreads,
                        lsmem, c.stream, ws, p, k0, k0, v0, v0);
         })))
        return rc;
    return launch("copy", -1, c.stream, [&] {
        launch_pdl(k_copy<KB, VB>, cap_grid(small_grid, max_tiles), kThreads, 0, c.stream, ws, kIpTile,
                   k0, k0, v0, v0);
    });
}

template <int KB, int VB>
int run_call_vb(const Call &c) {
    if (c.inplace) return run_inplace<KB, VB>(c);
    constexpr int STABLE = VB > 0;
    const int tv = c.pass_mode ? 0 : c.tile_variant;      // a single pass uses tile shape 0
    const int T = tv ? PartShape<KB, VB, 1>::kTile : PartShape<KB, VB, 0>::kTile;
    const int bits = c.bits > 0 ? c.bits : kBits;
    const int L = levels_for(KB, bits);
    const int sms = device_sms();
    if (sms <= 0) return BINAR_ERR_CUDA;
    const Layout lay = c.layout ? *c.layout : make_layout(c.n, c.offsets ? c.num_segments : 1, KB, VB);
    const Ws ws = carve(lay, c.ws);
    Params p{};
    p.map = c.map;
    p.n = c.n;
    p.cutoff = c.cutoff;
    p.timeout_ns = c.timeout_ns;
    p.skip_publish_tile = c.skip_publish_tile;
    p.tile = T;
    p.bits = bits;
    const int small_grid = sms * 4;
    int rc;

    if (c.pass_mode) {
        p.keys = const_cast<void *>(c.keys_in);
        p.vals = const_cast<void *>(c.vals_in);
        const uint32_t tiles = (uint32_t)((c.n + T - 1) / T);
        if ((rc = launch("init", -1, c.stream, [&] {
                 launch_pdl(k_init<KB>, 1, 1, 0, c.stream, ws, c.n, 0, c.pass_pos, tiles, 1);
             })))
            return rc;
        if ((rc = launch("prep", 0, c.stream, [&] { launch_pdl(k_prep, small_grid, kThreads, 0, c.stream, ws, 0); })))
            return rc;
        {
            auto hfn = c.map == BINAR_MAP_UNSIGNED ? k_hist<KB, true> : k_hist<KB, false>;
            const int occ = kernel_ctas_per_sm((const void *)hfn, 0);
            const long long hfull = (long long)sms * (occ > 0 ? occ : 1);
            const int hgroup = hist_group(tiles, hfull);
            const int hg = cap_grid(hfull, tiles / hgroup + 1);
            if ((rc = launch("hist", 0, c.stream, [&] {
                     launch_pdl(hfn, hg, kThreads, 0, c.stream, ws, p, 0, hgroup);
                 })))
                return rc;
        }
        if ((rc = launch("prefix", -1, c.stream, [&] {
                 launch_pdl(k_prefix_only, 1, kThreads, 0, c.stream, ws, c.pass_offsets, c.n, bits);
             })))
            return rc;
        // the call's one partition is its level 0 (the test hook's level)
        return launch_partition<KB, VB, true, 0>(c, ws, p, 0, 0, const_cast<void *>(c.keys_in),
                                                 c.keys_out, const_cast<void *>(c.vals_in), c.vals_out,
                                                 tiles);
    }

    p.keys = c.keys;
    p.vals = c.vals;
    void *k0 = c.keys, *k1 = ws.alt_keys, *v0 = c.vals, *v1 = VB ? ws.alt_vals : nullptr;
    const bool seg = c.offsets != nullptr;
    const uint32_t tiles0 = (uint32_t)((c.n + T - 1) / T);
    // work bounds: every bucket of a level holds more than `cutoff` keys, and
    // has at most one partial tile
    const long long max_buckets = c.n / ((long long)c.cutoff + 1) + 1;
    const long long max_tiles = c.n / T + max_buckets + 1;
    if ((rc = launch("init", -1, c.stream, [&] {
             launch_pdl(k_init<KB>, 1, 1, 0, c.stream, ws, c.n, c.cutoff, 0, tiles0, seg ? 0 : 1);
         })))
        return rc;
    if (seg) {
        const long long S = c.num_segments;
        int grid = (int)((S + kThreads - 1) / kThreads);
        if (grid > small_grid) grid = small_grid;
        if (grid < 1) grid = 1;
        if ((rc = launch("seed", -1, c.stream, [&] {
                 launch_pdl(k_seed_segments<KB>, grid, kThreads, 0, c.stream, ws, c.offsets, S, c.n, c.cutoff, T,
                            c.num_segments_dev);
             })))
            return rc;
    }
    if (seg || c.n > c.cutoff) {
        auto hfn = c.map == BINAR_MAP_UNSIGNED ? k_hist<KB, true> : k_hist<KB, false>;
        const int hocc = kernel_ctas_per_sm((const void *)hfn, 0);
        const long long hfull = (long long)sms * (hocc > 0 ? hocc : 1);
        const int hgroup = hist_group(max_tiles, hfull);
        const int hgrid = cap_grid(hfull, max_tiles / hgroup + 1);
        const int pgrid = cap_grid(small_grid, max_buckets > max_tiles / 4 ? max_buckets : max_tiles / 4);
        const int cgrid = cap_grid(small_grid, max_buckets);
        for (int l = 0; l < L; l++) {
            const int slot = l & 1;
            if (l == 1 && tv == 0 && c.n <= kTailMaxN) {
                const int rt = launch_levels_tail<KB, VB>(c, ws, p, l, L, max_tiles, k0, k1, v0, v1);
                if (rt != kTailUnavailable) {
                    if (rt) return rt;
                    break;
                }
            }
            if ((rc = launch("prep", l, c.stream, [&] {
                     launch_pdl(k_prep, pgrid, kThreads, 0, c.stream, ws, slot);
                 })))
                return rc;
            if ((rc = launch("hist", l, c.stream, [&] {
                     launch_pdl(hfn, hgrid, kThreads, 0, c.stream, ws, p, slot, hgroup);
                 })))
                return rc;
            if ((rc = launch("classify", l, c.stream, [&] {
                     launch_pdl(k_classify<KB>, cgrid, kThreads, 0, c.stream, ws, p, slot, l == L - 1);
                 })))
                return rc;
            if ((rc = tv ? launch_partition<KB, VB, STABLE, 1>(c, ws, p, slot, l, k0, k1, v0, v1, max_tiles)
                         : launch_partition<KB, VB, STABLE, 0>(c, ws, p, slot, l, k0, k1, v0, v1, max_tiles)))
                return rc;
        }
    }
    {
        if ((rc = launch_finish_classes<KB, VB>(c, ws, p, k0, k1, v0, v1,
                                                 std::make_integer_sequence<int, FinishClasses<KB>::kCount>{})))
            return rc;
        auto lfn = k_finish_lsd<KB, VB>;
        const size_t lsmem = sizeof(FinishLsdSmem<KB, VB>);
        const int locc = kernel_ctas_per_sm((const void *)lfn, lsmem);
        if ((rc = launch("finish_lsd", -1, c.stream, [&] {
                 launch_pdl(lfn, cap_grid((long long)sms * (locc > 0 ? locc : 1), c.n / 33 + 1), kThreads,
                            lsmem, c.stream, ws, p, k0, k1, v0, v1);
             })))
            return rc;
    }
    return launch("copy", -1, c.stream, [&] {
        launch_pdl(k_copy<KB, VB>, cap_grid(small_grid, max_tiles), kThreads, 0, c.stream, ws, T, k0, k1,
                   v0, v1);
    });
}

}  // namespace binar
