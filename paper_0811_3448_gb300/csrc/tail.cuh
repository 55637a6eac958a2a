// tail.cuh -- levels 1.. of a small sort in one cooperative launch.
//
// A sort of a few million keys waits on launches: after level 0 the host
// enqueues prep, hist, classify and partition for every level the key width
// can need, although for most inputs of that size the buckets of level 0
// already fit the finisher and those launches find no work (about 1.75 us
// each).  Here the levels after the first run in one persistent grid, as the
// same device code (the kernels' bodies) with grid-wide barriers in place of
// kernel boundaries, and the loop ends at the first level without a bucket,
// so an empty tail costs one launch.  Level 0 and the finisher keep their own
// launches (and their occupancy).  A cooperative launch makes every CTA
// resident, so a barrier never waits on a CTA that has not started; every
// wait is bounded all the same.
#pragma once

#include "kernels.cuh"

namespace binar {

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier on ctr->gbar (arrivals, generation), both 0 when the call
// starts (init clears the counters).  The last CTA to arrive resets the count
// and bumps the generation; the others wait for the bump, at most limit_ns.
// The fences make every write before the barrier visible after it: to
// ordinary loads (the acquire drops stale L1 lines) and to the bulk-copy
// engine, which reads global memory through the async proxy.  Returns false,
// after recording BINAR_ERR_DEVICE_TIMEOUT, if the wait ran out.
__device__ __forceinline__ bool grid_sync(Counters *ctr, long long limit_ns) {
    uint32_t *gbar = ctr->gbar;
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __threadfence();
        const uint32_t gen = ld_acquire(&gbar[1]);      // read before arriving
        const uint32_t arrived = atomicAdd(&gbar[0], 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&gbar[0], 0u);
            __threadfence();
            st_release(&gbar[1], gen + 1);
        } else {
            const unsigned long long t0 = globaltimer_ns();
            while (ld_acquire(&gbar[1]) == gen) {
                if ((long long)(globaltimer_ns() - t0) > limit_ns) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    ok = __syncthreads_and(ok);
    if (!ok && threadIdx.x == 0) set_status(ctr, BINAR_ERR_DEVICE_TIMEOUT);
    return ok != 0;
}

// Levels first_level .. levels-1 of the call (driver.cuh run_call_vb's level
// loop, phase for phase), with the default tile shape.  The bucket count of
// a level is read after the barrier that ends the level before it (or after
// the previous kernel), so every CTA takes the same decision.
template <int KB, int VB, bool IDENT>
__global__ void __launch_bounds__(kThreads, 2)
    k_levels_tail(Ws ws, Params p, int first_level, int levels, int hgroup, void *k0, void *k1,
                  void *v0, void *v1) {
    constexpr bool STABLE = VB > 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Counters *ctr = ws.ctr;
    const long long lim = p.timeout_ns;
    for (int l = first_level; l < levels; l++) {
        const int slot = l & 1;
        if (has_error(ctr)) return;              // uniform after a barrier
        if (ld_acquire(reinterpret_cast<const uint32_t *>(&ctr->alloc[slot])) == 0u) return;
        prep_body(ws, slot);
        if (!grid_sync(ctr, lim)) return;
        hist_body<KB, IDENT, false>(ws, p, slot, hgroup);
        if (!grid_sync(ctr, lim)) return;
        classify_body<KB>(ws, p, slot, l == levels - 1 ? 1 : 0);
        if (!grid_sync(ctr, lim)) return;
        partition_body<KB, VB, STABLE, IDENT, 0>(ws, p, slot, l, k0, k1, v0, v1);
        // the partition's mbarrier before its shared memory serves the next
        // level (after an error a copy may still be in flight: left alone,
        // and the loop ends at the next check)
        if (threadIdx.x == 0 && !has_error(ctr))
            mbar_inval(&reinterpret_cast<PartitionSmem<KB, VB, STABLE, 0> *>(smem_raw)->bar);
        if (!grid_sync(ctr, lim)) return;
    }
}

}  // namespace binar
