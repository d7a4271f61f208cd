// fused.cu -- the batched form as one persistent launch over both ring
// degrees and both phases (forward transforms, then multiply-accumulate and
// inverse transforms) of every job.
//
// CTAs of Cfg<LB>::T threads (the tile of the larger degree 2^LB) take work
// units from one device counter in list order.  A unit of the larger degree
// runs on the whole CTA; a unit of the degree 2^(LB-1) runs up to two items,
// one per half of the CTA, each half on its own half of the shared memory
// (exactly the smaller tile's buffer) and with its own named barrier.  All
// forward units precede all multiply-accumulate units in the list; a forward
// item, once its stores are done, fences and counts itself in its job's
// fwd_done; a multiply-accumulate item first waits until fwd_done of its job
// reaches fwd_need.  It waits only on units claimed before it, by CTAs that
// are running and never wait themselves, so every wait ends; each is
// nevertheless bounded: after wait_limit polls the unit writes
// HE_ERR_TIMEOUT (and its index) to the status word and skips its work, and
// every CTA stops at its next claim.  The operands written inside the launch
// are read with coherent loads (ld.global.ca), never the read-only path;
// thread 0's acquire of the job counter, then the CTA barrier, orders them
// after the forward items' release.
#include <atomic>

#include "ntt_core.cuh"

namespace he {

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Poll job's forward counter until it reaches fwd_need; false if the limit
// ran out (status set) or another unit has already given up.
__device__ bool fused_wait(const FusedArgs &a, int job, int unit) {
    if (!HE_OBJ_OK(a.fwd_need + job) || !HE_OBJ_OK(a.fwd_done + job) || !HE_OBJ_OK(a.status + 1)) return false;
    const int need = a.fwd_need[job];
    long long polls = 0;
    while (ld_acquire(a.fwd_done + job) < need) {
        if (*(volatile int *)a.status != 0) return false;
        if (++polls > a.wait_limit) {
            if (atomicCAS(a.status, 0, HE_ERR_TIMEOUT) == 0) atomicExch(a.status + 1, unit);
            return false;
        }
        __nanosleep(256);
    }
    return true;
}

// the next unit index, or n_units (stop) once a unit has given up waiting;
// called by thread 0 only, so the whole CTA takes the same decision
__device__ __forceinline__ int fused_claim(const FusedArgs &a) {
    if (!HE_OBJ_OK(a.status) || !HE_OBJ_OK(a.counter)) return a.n_units;
    return *(volatile int *)a.status != 0 ? a.n_units : atomicAdd(a.counter, 1);
}

// a forward item's stores are complete in every thread of its group (the
// caller's barrier): make them visible device-wide, then count the item
__device__ __forceinline__ void fused_count(const FusedArgs &a, int job) {
    __threadfence();
    if (HE_OBJ_OK(a.fwd_done + job)) atomicAdd(a.fwd_done + job, 1);
}

// The four unit bodies are separate (not inlined) functions, so that each is
// register-allocated like the corresponding single-purpose kernel; inlined
// into one body they spilled kilobytes under the 64-register budget.
template <int LB, int MINB>
__device__ __noinline__ void fused_fwd_big(const FwdItem *ip, u64 *sm) {
    fwd_item<LB, false>(ip, sm, threadIdx.x);
}
template <int LB, int MINB>
__device__ __noinline__ void fused_mac_big(const MacItem *ip, u64 *sm) {
    mac_item<LB, MINB, false, CtaSync, true>(ip, sm, threadIdx.x);
}
// The half tiles run under the register budget of the whole CTA (twice their
// threads), so they take the accumulator groups and the forward quotient of
// that budget, not those of a CTA of their own size.
template <int LS, int MINB>
__device__ __noinline__ void fused_fwd_half(const FwdItem *ip, u64 *sm, int tau, int h) {
    fwd_item<LS, false, HalfSync, Cfg<LS + 1>::COARSE_FWD || MINB == 1>(ip, sm, tau, HalfSync{1 + h, Cfg<LS>::T});
}
template <int LS, int MINB>
__device__ __noinline__ void fused_mac_half(const MacItem *ip, u64 *sm, int tau, int h) {
    mac_item<LS, MINB, false, HalfSync, true, mac_group(Cfg<LS + 1>::T, MINB)>(ip, sm, tau,
                                                                               HalfSync{1 + h, Cfg<LS>::T});
}

template <int LB, int MINB>
__global__ void __launch_bounds__(Cfg<LB>::T, MINB) k_batch_fused(const __grid_constant__ FusedArgs a) {
    extern __shared__ u64 sm[];
    __shared__ int s_unit[2];
    __shared__ int s_go[2];
    constexpr int TS = Cfg<LB - 1>::T;            // threads of one half
    constexpr int HALF_WORDS = Cfg<LB - 1>::SMEM / 8;
    static_assert(2 * TS == Cfg<LB>::T && 2 * Cfg<LB - 1>::SMEM == Cfg<LB>::SMEM, "two half tiles fill the CTA");
    // thread 0 claims the next unit while the current one runs; the claims
    // alternate between two slots, so one barrier per unit publishes the
    // claim (and orders the previous unit's shared-memory use before this one's)
    // (a CTA holds a second unit only behind its current one; since every
    // forward unit precedes every multiply-accumulate unit, a forward unit
    // held that way waits only behind another forward unit, which never
    // waits, so no wait can depend on a unit held by a waiting CTA)
    if (threadIdx.x == 0) s_unit[0] = fused_claim(a);
    for (int iter = 0;; iter++) {
        __syncthreads();
        const int it = s_unit[iter & 1];
        if (it >= a.n_units) return;
        if (threadIdx.x == 0) s_unit[(iter + 1) & 1] = fused_claim(a);
        if (!HE_OBJ_OK(a.units + it)) continue;  // (checks build; uniform over the CTA)
        const FusedUnit u = a.units[it];
        if (u.big) {
            if (u.mac) {
                if (threadIdx.x == 0) s_go[0] = fused_wait(a, u.job[0], it);
                __syncthreads();
                if (s_go[0]) fused_mac_big<LB, MINB>(a.mac_big + u.item[0], sm);
            } else {
                fused_fwd_big<LB, MINB>(a.fwd_big + u.item[0], sm);
                __syncthreads();
                if (threadIdx.x == 0) fused_count(a, u.job[0]);
            }
        } else {
            const int h = threadIdx.x >= TS ? 1 : 0;
            const int tau = threadIdx.x - h * TS;
            const HalfSync hs{1 + h, TS};
            u64 *smh = sm + h * HALF_WORDS;
            const int item = h ? u.item[1] : u.item[0];
            const int job = h ? u.job[1] : u.job[0];
            if (item >= 0) {
                if (u.mac) {
                    if (tau == 0) s_go[h] = fused_wait(a, job, it);
                    hs.sync();
                    if (s_go[h]) fused_mac_half<LB - 1, MINB>(a.mac_small + item, smh, tau, h);
                } else {
                    fused_fwd_half<LB - 1, MINB>(a.fwd_small + item, smh, tau, h);
                    hs.sync();
                    if (tau == 0) fused_count(a, job);
                }
            }
        }
    }
}

// MINB: resident CTAs per SM the register budget is set for (1: 128
// registers per thread at the 512-thread tile, 2: 64).  The dynamic
// shared-memory attribute is per device and is set on the first launch on
// each device (before any graph capture of the batch, which the batch's
// autotuning or a first direct run precedes).
template <int LB, int MINB>
static int fused_attr() {
    static std::atomic<unsigned long long> attr_mask{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HE_ERR_CUDA;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_mask.load(std::memory_order_acquire) & bit)) {
        if (cudaFuncSetAttribute(k_batch_fused<LB, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 Cfg<LB>::SMEM) != cudaSuccess)
            return HE_ERR_CUDA;
        attr_mask.fetch_or(bit, std::memory_order_acq_rel);
    }
    return HE_OK;
}

template <int LB, int MINB>
static int fused_l(const FusedArgs &a, int grid, cudaStream_t st) {
    constexpr int smem = Cfg<LB>::SMEM;
    if (int rc = fused_attr<LB, MINB>()) return rc;
    k_batch_fused<LB, MINB><<<grid, Cfg<LB>::T, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? HE_OK : HE_ERR_CUDA;
}

int fused_set_attributes(int logN_big, int minb) {
#ifdef HE_CHECKS
    minb = 2;
#endif
    switch (logN_big * 2 + minb - 1) {
#ifndef HE_CHECKS
    case 24: return fused_attr<12, 1>();
#endif
    case 25: return fused_attr<12, 2>();
#ifndef HE_CHECKS
    case 26: return fused_attr<13, 1>();
#endif
    case 27: return fused_attr<13, 2>();
    }
    return HE_ERR_UNSUPPORTED_PARAMS;
}

int launch_fused(int logN_big, int minb, const FusedArgs &a, int grid, cudaStream_t st) {
    if (a.n_units <= 0) return HE_OK;
    if (grid <= 0 || minb < 1 || minb > 2) return HE_ERR_INVALID_ARG;
#ifdef HE_CHECKS
    // the bounds-checked build compiles one register budget (same bits)
    if (minb == 1) grid *= 2;
    minb = 2;
#endif
    switch (logN_big * 2 + minb - 1) {
#ifndef HE_CHECKS
    case 24: return fused_l<12, 1>(a, grid, st);
#endif
    case 25: return fused_l<12, 2>(a, grid, st);
#ifndef HE_CHECKS
    case 26: return fused_l<13, 1>(a, grid, st);
#endif
    case 27: return fused_l<13, 2>(a, grid, st);
    }
    return HE_ERR_UNSUPPORTED_PARAMS;
}

}  // namespace he

HE_CHECKS_UNIT(fused)
