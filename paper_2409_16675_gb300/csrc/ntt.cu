// ntt.cu -- negacyclic NTT kernels over RNS limbs: one CTA per limb polynomial
// (grid kernels), and the work-list kernels of the batched and served forms.
// The transforms themselves are in ntt_core.cuh.
#include <atomic>
#include <cstring>

#include "ntt_core.cuh"

namespace he {

// ---------------------------------------------------------------- grid kernels (one CTA per limb polynomial)
// Up to kMaxFwdJobs forward jobs over the same moduli in one grid: blocks
// [start[i], start[i+1]) belong to job i.  The job is selected with constant
// indices only, so the parameter block is never copied to local memory.
template <int LOGN, bool LAZY>
__global__ void __launch_bounds__(Cfg<LOGN>::T, Cfg<LOGN>::MINB) k_fwd(FwdJobs JS, const ModDev *__restrict__ mods) {
    extern __shared__ u64 sm[];
    constexpr int N = Cfg<LOGN>::N;
    const int tau = threadIdx.x;
    FwdJob J = JS.j[0];
    int base = 0;
#pragma unroll
    for (int i = 1; i < kMaxFwdJobs; i++)
        if (i < JS.n && (int)blockIdx.x >= JS.start[i]) { J = JS.j[i]; base = JS.start[i]; }
    const int local = (int)blockIdx.x - base;
    const int limb = local / J.n_polys;
    const int p = local - limb * J.n_polys;
    if (!HE_OBJ_OK(mods + J.mod_base + limb)) return;  // uniform over the CTA
    const ModDev M = mods[J.mod_base + limb];
    const void *src;
    if (J.kind == SRC_RNS)
        src = limb < J.split ? (const void *)((const u64 *)J.src + (long long)p * J.src_stride + (long long)limb * N)
                             : (const void *)((const u64 *)J.src2 + (long long)p * J.src2_stride +
                                              (long long)(limb - J.split) * N);
    else if (J.kind == SRC_I8)
        src = (const int8_t *)J.src + (long long)p * J.src_stride;
    else if (J.kind == SRC_U32)
        src = (const uint32_t *)J.src + (long long)p * J.src_stride;
    else
        src = (const u64 *)J.src + (long long)p * J.src_stride;
    u64 v[Cfg<LOGN>::R];
    fwd_load<LOGN>(J.kind, src, J.t, M, tau, v);
    fwd_transform_store<LOGN, LAZY>(v, sm, tau, M, J.dst + (long long)p * J.dst_stride + (long long)limb * N);
}

// Up to kMaxMacJobs multiply-accumulate jobs over the same moduli in one
// grid (blocks [start[i], start[i+1]) belong to job i).  The job block stays
// in the constant bank (__grid_constant__): fields are read through a
// block-uniform index, never copied to registers or local memory.
template <int LOGN, bool LAZY>
__global__ void __launch_bounds__(Cfg<LOGN>::T, Cfg<LOGN>::MINB)
    k_mac_intt(const __grid_constant__ MacJobs JS, const ModDev *__restrict__ mods) {
    extern __shared__ u64 sm[];
    constexpr int N = Cfg<LOGN>::N, T = Cfg<LOGN>::T;
    const int tau = threadIdx.x;
    int jj = 0;
#pragma unroll
    for (int i = 1; i < kMaxMacJobs; i++)
        if (i < JS.n && (int)blockIdx.x >= JS.start[i]) jj = i;
    const MacJob &J = JS.j[jj];
    const int local = (int)blockIdx.x - JS.start[jj];
    const int limb = local / J.n_out;
    const int o = local - limb * J.n_out;
    if (!HE_OBJ_OK(mods + J.mod_base + limb)) return;  // uniform over the CTA
    const ModDev M = mods[J.mod_base + limb];
    u64 v[Cfg<LOGN>::R];
    mac_accumulate<LOGN, mac_group(Cfg<LOGN>::T, Cfg<LOGN>::MINB)>(J.A, J.B, J.ta, J.tb, HE_LD(J.ptr + o),
                                                                   HE_LD(J.ptr + o + 1), limb, M, tau, v, sm);
    inv_transform<LOGN, LAZY>(v, sm, tau, M);
    // natural order: element j = k*T + tau
    const u64 q = M.q;
    u64 *out = J.out + (long long)o * J.out_stride + (long long)limb * N;
    const u64 *add = J.add ? J.add + (long long)o * J.add_stride + (long long)limb * N : nullptr;
    const int8_t *err = J.err ? J.err + (long long)o * J.err_stride : nullptr;
    const u64 *msg = (J.msg && (o % J.msg_div) == 0) ? J.msg + (long long)(o / J.msg_div) * J.msg_stride : nullptr;
    const u64 *s2 = J.s2 ? J.s2 + (long long)limb * N : nullptr;
    u64 g = 0, gs = 0, dl = 0, dls = 0;
    if (s2) {
        g = HE_LD(J.gmul + 2 * ((long long)o * J.n_limbs + limb));
        gs = HE_LD(J.gmul + 2 * ((long long)o * J.n_limbs + limb) + 1);
    }
    if (msg) { dl = HE_LD(J.E->delta_q + J.mod_base + limb); dls = HE_LD(J.E->delta_qs + J.mod_base + limb); }
    const u64 t = msg ? HE_LD(&J.E->t) : 0;
#pragma unroll
    for (int k = 0; k < Cfg<LOGN>::R; k++) {
        const int x = k * T + tau;
        const ulonglong2 zp = HE_LDG(M.z + x);
        u64 r = red1(shoup(v[k], zp.x, zp.y, q), q);
        if (err) {
            const int e = HE_LD(err + x);
            r = e >= 0 ? addm(r, (u64)e, q) : subm(r, (u64)(-e), q);
        }
        if (J.negate) r = r ? q - r : 0;
        if (s2) r = addm(r, red1(shoup(HE_LD(s2 + x), g, gs, q), q), q);
        if (msg) {
            u64 m = HE_LD(msg + x);
            m = m >= t ? m % t : m;
            r = addm(r, red1(shoup(m, dl, dls, q), q), q);
        }
        if (add) r = addm(r, HE_LD(add + x), q);
        HE_ST(out + x, r);
    }
}

// ---------------------------------------------------------------- persistent queue kernels
// Each CTA repeatedly takes the next item index of a launch (one atomic per
// item) until all `total` items are done; items live in `nseg` segments (an
// item array each, with the index of its first item) so a launch can cover
// several independently built work lists.  Items of one launch share the ring
// degree but may use any modulus of any context.  The counter must be zero
// at launch.
template <typename ITEM>
__device__ __forceinline__ const ITEM *next_item(const ItemSeg *segs, int nseg, int total, int *counter,
                                                 int *s_meta) {
    if (threadIdx.x == 0) {
        const int it = HE_OBJ_OK(counter) ? atomicAdd(counter, 1) : total;
        int sidx = 0;
        if (it < total) {
            int lo = 0, hi = nseg - 1;  // last segment whose begin <= it
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (HE_LD(&segs[mid].begin) <= it) lo = mid;
                else hi = mid - 1;
            }
            sidx = lo;
        }
        s_meta[0] = it;
        s_meta[1] = sidx;
    }
    __syncthreads();
    const int it = s_meta[0], sidx = s_meta[1];
    __syncthreads();
    if (it >= total) return nullptr;
    return (const ITEM *)HE_LD(&segs[sidx].items) + (it - HE_LD(&segs[sidx].begin));
}

// LAZY: every item's modulus is below 2^57 (checked by the host per launch)
template <int LOGN, int MINB, bool LAZY>
__global__ void __launch_bounds__(Cfg<LOGN>::T, MINB) k_fwd_queue(const ItemSeg *__restrict__ segs, int nseg,
                                                                  int total, int *counter) {
    extern __shared__ u64 sm[];
    __shared__ int s_meta[2];
    while (const FwdItem *ip = next_item<FwdItem>(segs, nseg, total, counter, s_meta))
        fwd_item<LOGN, LAZY>(ip, sm, threadIdx.x);
}

template <int LOGN, int MINB, bool LAZY>
__global__ void __launch_bounds__(Cfg<LOGN>::T, MINB) k_mac_queue(const ItemSeg *__restrict__ segs, int nseg,
                                                                  int total, int *counter) {
    extern __shared__ u64 sm[];
    __shared__ int s_meta[2];
    while (const MacItem *ip = next_item<MacItem>(segs, nseg, total, counter, s_meta))
        mac_item<LOGN, MINB, LAZY>(ip, sm, threadIdx.x);
}

// One CTA per item (no loop): CTA b takes item b of the segment table.  The
// hardware block scheduler then hands out items in list order (heaviest
// first), and each CTA has the register picture of the grid kernels.
template <typename ITEM>
__device__ __forceinline__ const ITEM *item_at(const ItemSeg *segs, int nseg, int it) {
    int lo = 0, hi = nseg - 1;  // last segment whose begin <= it
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (HE_LD(&segs[mid].begin) <= it) lo = mid;
        else hi = mid - 1;
    }
    return (const ITEM *)HE_LD(&segs[lo].items) + (it - HE_LD(&segs[lo].begin));
}

template <int LOGN, int MINB, bool LAZY>
__global__ void __launch_bounds__(Cfg<LOGN>::T, MINB) k_fwd_items(const ItemSeg *__restrict__ segs, int nseg) {
    extern __shared__ u64 sm[];
    fwd_item<LOGN, LAZY>(item_at<FwdItem>(segs, nseg, (int)blockIdx.x), sm, threadIdx.x);
}

template <int LOGN, int MINB, bool LAZY>
__global__ void __launch_bounds__(Cfg<LOGN>::T, MINB) k_mac_items(const ItemSeg *__restrict__ segs, int nseg) {
    extern __shared__ u64 sm[];
    mac_item<LOGN, MINB, LAZY>(item_at<MacItem>(segs, nseg, (int)blockIdx.x), sm, threadIdx.x);
}

// True the first time a call site runs on the current device: kernel
// attributes (the dynamic shared-memory limit) are per device, and several
// threads may launch (the request server's worker); setting them twice is
// harmless.
static bool first_on_device(std::atomic<unsigned long long> &mask) {
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (mask.load(std::memory_order_acquire) & bit) return false;
    mask.fetch_or(bit, std::memory_order_acq_rel);
    return true;
}

// true when every modulus of the launch is below 2^57 (no in-transform corrections)
static bool lazy_ok(const he_ctx *c, int mod_base, int n_limbs) {
    for (int i = 0; i < n_limbs; i++)
        if (c->h_mods[mod_base + i].q >= (1ull << 57)) return false;  // 57 q < 2^63
    return true;
}

bool ctx_lazy(const he_ctx *c) { return lazy_ok(c, 0, c->L); }

template <int LOGN>
static int fwd_t(he_ctx *c, const FwdJob *jobs, int n, cudaStream_t st) {
    const int smem = Cfg<LOGN>::SMEM;
    static std::atomic<unsigned long long> attr_mask{0};
    if (first_on_device(attr_mask)) {
        if constexpr (kAllVariants) cudaFuncSetAttribute(k_fwd<LOGN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_fwd<LOGN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    FwdJobs JS;
    memset(&JS, 0, sizeof JS);
    long long blocks = 0;
    double bytes = 0;
    const int N = Cfg<LOGN>::N;
    for (int i = 0; i < n; i++) {
        const FwdJob &j = jobs[i];
        if (j.n_limbs != jobs[0].n_limbs || j.mod_base != jobs[0].mod_base)
            return fail(c, HE_ERR_INVALID_ARG, "merged forward jobs must share their moduli");
        if (j.n_polys <= 0) continue;
        JS.start[JS.n] = (int)blocks;
        JS.j[JS.n++] = j;
        blocks += (long long)j.n_polys * j.n_limbs;
        const double src_bytes =
            j.kind == SRC_RNS ? 8.0 * j.n_limbs : (j.kind == SRC_I8 ? 1.0 : (j.kind == SRC_U32 ? 4.0 : 8.0));
        bytes += (double)j.n_polys * N * (src_bytes + 8.0 * j.n_limbs);
    }
    if (blocks == 0) return HE_OK;
    if (blocks > 0x7fffffffLL) return fail(c, HE_ERR_INVALID_ARG, "forward launch too large");
    const bool lazy = lazy_ok(c, jobs[0].mod_base, jobs[0].n_limbs);
    TraceScope ts(c, st, "ntt_fwd", bytes, (double)blocks * (N / 2) * LOGN);
    if constexpr (kAllVariants) {
        if (lazy) k_fwd<LOGN, true><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(JS, c->d_mods);
        else k_fwd<LOGN, false><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(JS, c->d_mods);
    } else {
        (void)lazy;
        k_fwd<LOGN, false><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(JS, c->d_mods);
    }
    return cuda_check(c, cudaGetLastError(), "k_fwd");
}

template <int LOGN>
static int mac_t(he_ctx *c, const MacJob *jobs, int n, cudaStream_t st) {
    const int smem = Cfg<LOGN>::SMEM;
    static std::atomic<unsigned long long> attr_mask{0};
    if (first_on_device(attr_mask)) {
        if constexpr (kAllVariants)
            cudaFuncSetAttribute(k_mac_intt<LOGN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_mac_intt<LOGN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    MacJobs JS;
    memset(&JS, 0, sizeof JS);
    long long blocks = 0;
    double bytes = 0, mm = 0;
    const int N = Cfg<LOGN>::N;
    for (int i = 0; i < n; i++) {
        const MacJob &j = jobs[i];
        if (j.n_limbs != jobs[0].n_limbs || j.mod_base != jobs[0].mod_base)
            return fail(c, HE_ERR_INVALID_ARG, "merged multiply-accumulate jobs must share their moduli");
        if (j.n_out <= 0) continue;
        JS.start[JS.n] = (int)blocks;
        JS.j[JS.n++] = j;
        const long long b = (long long)j.n_out * j.n_limbs;
        blocks += b;
        const double lb = 8.0 * N * j.n_limbs;  // one polynomial over all limbs
        bytes += lb * (j.n_out + j.n_dist_a + j.n_dist_b + (j.add ? j.n_out : 0));
        // modular products the kernel computes per output limb polynomial:
        // the inverse transform's butterflies, one Montgomery reduction ending
        // each coefficient's sum, the untwist, one product per term, and in
        // the epilogue Delta*m (outputs with a message) and g*s^2 (keygen)
        const double with_msg = (j.msg && j.msg_div > 0) ? (double)((j.n_out + j.msg_div - 1) / j.msg_div) : 0.0;
        mm += (double)b * ((N / 2) * LOGN + 2.0 * N) + (double)j.n_terms * N * j.n_limbs +
              with_msg * j.n_limbs * N + (j.s2 ? (double)b * N : 0.0);
    }
    if (blocks == 0) return HE_OK;
    if (blocks > 0x7fffffffLL) return fail(c, HE_ERR_INVALID_ARG, "multiply-accumulate launch too large");
    const bool lazy = lazy_ok(c, jobs[0].mod_base, jobs[0].n_limbs);
    TraceScope ts(c, st, "mac_intt", bytes, mm);
    if constexpr (kAllVariants) {
        if (lazy) k_mac_intt<LOGN, true><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(JS, c->d_mods);
        else k_mac_intt<LOGN, false><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(JS, c->d_mods);
    } else {
        (void)lazy;
        k_mac_intt<LOGN, false><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(JS, c->d_mods);
    }
    return cuda_check(c, cudaGetLastError(), "k_mac_intt");
}

int launch_fwd_multi(he_ctx *c, const FwdJob *jobs, int n, cudaStream_t st) {
    if (n < 1 || n > kMaxFwdJobs) return fail(c, HE_ERR_INVALID_ARG, "1 to 4 forward jobs per launch");
    switch (c->logN) {
    case 10: return fwd_t<10>(c, jobs, n, st);
    case 11: return fwd_t<11>(c, jobs, n, st);
    case 12: return fwd_t<12>(c, jobs, n, st);
    case 13: return fwd_t<13>(c, jobs, n, st);
    case 14: return fwd_t<14>(c, jobs, n, st);
    }
    return fail(c, HE_ERR_UNSUPPORTED_PARAMS, "unsupported N");
}

int launch_fwd(he_ctx *c, const FwdJob &j, cudaStream_t st) { return launch_fwd_multi(c, &j, 1, st); }

template <int LOGN, int MINB, bool LAZY>
static int queue_l(bool fwd, const ItemSeg *segs, int nseg, int total, int *counter, int grid, cudaStream_t st) {
    const int smem = Cfg<LOGN>::SMEM;
    static std::atomic<unsigned long long> attr_mask{0};
    if (first_on_device(attr_mask)) {
        cudaFuncSetAttribute(k_fwd_queue<LOGN, MINB, LAZY>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_mac_queue<LOGN, MINB, LAZY>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_fwd_items<LOGN, MINB, LAZY>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_mac_items<LOGN, MINB, LAZY>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    if (grid <= 0) {  // one CTA per item
        if (fwd) k_fwd_items<LOGN, MINB, LAZY><<<total, Cfg<LOGN>::T, smem, st>>>(segs, nseg);
        else k_mac_items<LOGN, MINB, LAZY><<<total, Cfg<LOGN>::T, smem, st>>>(segs, nseg);
    } else {
        if (fwd) k_fwd_queue<LOGN, MINB, LAZY><<<grid, Cfg<LOGN>::T, smem, st>>>(segs, nseg, total, counter);
        else k_mac_queue<LOGN, MINB, LAZY><<<grid, Cfg<LOGN>::T, smem, st>>>(segs, nseg, total, counter);
    }
    return cudaGetLastError() == cudaSuccess ? HE_OK : HE_ERR_CUDA;
}

template <int LOGN, int MINB>
static int queue_t(bool fwd, bool lazy, const ItemSeg *segs, int nseg, int total, int *counter, int grid,
                   cudaStream_t st) {
    if constexpr (kAllVariants)
        return lazy ? queue_l<LOGN, MINB, true>(fwd, segs, nseg, total, counter, grid, st)
                    : queue_l<LOGN, MINB, false>(fwd, segs, nseg, total, counter, grid, st);
    (void)lazy;
    return queue_l<LOGN, MINB, false>(fwd, segs, nseg, total, counter, grid, st);
}

int launch_queue(int logN, int minb, bool fwd, bool lazy, const ItemSeg *segs, int nseg, int total, int *counter,
                 int grid, cudaStream_t st) {
    if (total <= 0 || nseg <= 0) return HE_OK;
    if (!kAllVariants) minb = logN >= 14 ? 1 : 2;
    switch (logN * 2 + (minb >= 2 ? 1 : 0)) {
    case 20: if constexpr (kAllVariants) return queue_t<10, 1>(fwd, lazy, segs, nseg, total, counter, grid, st); break;
    case 21: return queue_t<10, 2>(fwd, lazy, segs, nseg, total, counter, grid, st);
    case 22: if constexpr (kAllVariants) return queue_t<11, 1>(fwd, lazy, segs, nseg, total, counter, grid, st); break;
    case 23: return queue_t<11, 2>(fwd, lazy, segs, nseg, total, counter, grid, st);
    case 24: if constexpr (kAllVariants) return queue_t<12, 1>(fwd, lazy, segs, nseg, total, counter, grid, st); break;
    case 25: return queue_t<12, 2>(fwd, lazy, segs, nseg, total, counter, grid, st);
    case 26: if constexpr (kAllVariants) return queue_t<13, 1>(fwd, lazy, segs, nseg, total, counter, grid, st); break;
    case 27: return queue_t<13, 2>(fwd, lazy, segs, nseg, total, counter, grid, st);
    case 28: return queue_t<14, 1>(fwd, lazy, segs, nseg, total, counter, grid, st);
    case 29: return queue_t<14, 1>(fwd, lazy, segs, nseg, total, counter, grid, st);
    }
    return HE_ERR_UNSUPPORTED_PARAMS;
}

int launch_mac_multi(he_ctx *c, const MacJob *jobs, int n, cudaStream_t st) {
    if (n < 1 || n > kMaxMacJobs) return fail(c, HE_ERR_INVALID_ARG, "1 to 8 multiply-accumulate jobs per launch");
    switch (c->logN) {
    case 10: return mac_t<10>(c, jobs, n, st);
    case 11: return mac_t<11>(c, jobs, n, st);
    case 12: return mac_t<12>(c, jobs, n, st);
    case 13: return mac_t<13>(c, jobs, n, st);
    case 14: return mac_t<14>(c, jobs, n, st);
    }
    return fail(c, HE_ERR_UNSUPPORTED_PARAMS, "unsupported N");
}

int launch_mac_intt(he_ctx *c, const MacJob &j, cudaStream_t st) { return launch_mac_multi(c, &j, 1, st); }

}  // namespace he

HE_CHECKS_UNIT(ntt)
