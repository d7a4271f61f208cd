// ntt.cu -- negacyclic NTT kernels over RNS limbs.
//
// The product in A_{N,q} = Z_q[x]/(x^N+1) (Section 2, Notations) is computed
// as NTT -> pointwise multiply-accumulate -> inverse NTT.  One CTA owns one
// limb polynomial; each of its N/R threads keeps R = 2^RB = 16 coefficients
// in registers and runs up to RB butterfly stages between exchanges through
// padded shared memory.  The forward
// transform is Cooley-Tukey with the psi twist merged into the twiddles
// (natural input, bit-reversed output); the inverse is a decimation-in-time
// Cooley-Tukey cyclic transform with omega^-1 on the bit-reversed input,
// followed by the untwist psi^-e N^-1 (times 2^64, which undoes the Montgomery
// reduction ending the multiply-accumulate).  Both use Harvey-style lazy
// butterflies with the approximate-quotient Shoup product built from 32-bit
// multiply-accumulates (twiddle product in [0, 4q) in the inverse and, for
// N <= 4096, in the forward transform: a coarser quotient from two high-half
// multiplies instead of two wide ones, measured 2.6% faster in the inverse;
// in [0, 3q) in the forward transform at N >= 8192, where the coarser one
// raised the spills under 64 registers and lost 1.8%); the butterfly adds 4q to
// the difference, so values grow by at most 4q per stage: with every modulus
// of a launch below 2^57 they stay below 57q < 2^63 through 14 stages and the
// LAZY variants make no correction inside the transform; otherwise X is
// brought below 4q before each butterfly and every value stays below
// 8q < 2^64.
//
// NTT-domain storage order (register-tile order): memory position
// k*(N/R) + tau holds the bit-reversed-order value of index R*tau + k, which
// is exactly what the last forward pass and the first inverse pass hold in
// registers, so both the forward store and the multiply-accumulate loads are
// coalesced.  This order never leaves the library.
#include <atomic>
#include <cstring>

#include "arith.cuh"

namespace he {

// Coefficients per 128-bit accumulator group of the multiply-accumulate: 4
// when the register budget is 64 per thread (resident threads per SM =
// 1024), else 8.
__host__ __device__ constexpr int mac_group(int threads, int minb) { return threads * minb >= 1024 ? 4 : 8; }

// Register tile: every thread holds R = 2^RB coefficients; passes of RB
// butterfly stages run in registers between shared-memory exchanges.  RB = 4
// at every ring degree: a 32-coefficient tile (RB = 5, two exchanges instead
// of three at N = 8192) made the forward transform 3% faster but halved the
// resident warps, and the multiply-accumulate kernels, which wait on their
// operand loads, lost 54%.
template <int LOGN>
struct Cfg {
    static constexpr int N = 1 << LOGN;
    static constexpr int RB = 4;
    static constexpr int R = 1 << RB;
    static constexpr int T = N / R;
    static constexpr int NP = (LOGN + RB - 1) / RB;
    static constexpr int RL = LOGN - RB * (NP - 1);
    static constexpr int SMEM = (N + N / R) * 8;
    // resident CTAs per SM the register budget targets (64 registers per
    // thread at N = 8192; N = 16384 runs one 1024-thread CTA per SM)
    static constexpr int MINB = LOGN >= 14 ? 1 : 2;
    // the forward transform takes the coarser Shoup quotient only where the
    // register budget leaves room for it (128 registers per thread)
    static constexpr bool COARSE_FWD = LOGN <= 12;
};

// one pad word per R elements: exchanges are conflict-free for every window
template <int RB>
__device__ __forceinline__ int padi(int j) { return j + (j >> RB); }
// element index of register k of thread tau when the RB-bit register window
// starts at bit lo
template <int RB>
__device__ __forceinline__ int jidx(int tau, int k, int lo) {
    return ((tau >> lo) << (lo + RB)) | (k << lo) | (tau & ((1 << lo) - 1));
}

// Forward pass: S stages on register bits S-1 .. 0 of the window starting at
// element bit lo (stage s0 + st acts on bit lo + S - 1 - st).  The twiddle of
// the pair whose lower element is j is the factor of group j >> (bit + 1) =
// h 2^gb + g at stage s, with g = k >> (kb + 1) (the gb = RB - 1 - kb
// register bits above kb) and h = tau >> lo; the table keeps it at 2^s +
// g 2^(s - gb) + h, so the loads of one g are contiguous across a warp
// (measured on the 26,624 digit transforms: 2.08 -> 1.80 ms).
template <int RB, int S, bool LAZY, bool COARSE>
__device__ __forceinline__ void fwd_pass(u64 (&v)[1 << RB], int tau, int lo, int s0, const ModDev &M) {
    static_assert(RB == kNttTileBits, "the forward table order follows the kernels' register tile");
    constexpr int R = 1 << RB;
    const u64 q4 = 2 * M.twoq, nq = M.nq;
#pragma unroll
    for (int st = 0; st < S; st++) {
        const int kb = S - 1 - st;
        const int s = s0 + st;
        const int gb = RB - 1 - kb;
        const int base = (1 << s) + (tau >> lo);
#pragma unroll
        for (int k = 0; k < R; k++) {
            if (k & (1 << kb)) continue;
            const int widx = base + ((k >> (kb + 1)) << (s - gb));
            const ulonglong2 Wp = __ldg(M.fw + widx);
            u64 X = v[k];
            const u64 Y = v[k | (1 << kb)];
            if (!LAZY) X = X >= q4 ? X - q4 : X;
            const u64 Tt = COARSE ? shoup4(Y, Wp.x, Wp.y, nq) : shoup3(Y, Wp.x, Wp.y, nq);
            v[k] = X + Tt;
            v[k | (1 << kb)] = X - Tt + q4;
        }
    }
}

// Decimation-in-time pass of the inverse: stages s0 .. s0+R-1 act on element
// bits lo+kb0 .. lo+kb0+R-1; the factor of the pair whose lower element is e
// is iw[2^s + (e mod 2^s)].
template <int RB, int S, int KB0, bool LAZY>
__device__ __forceinline__ void inv_pass(u64 (&v)[1 << RB], int tau, int lo, int s0, const ModDev &M) {
    constexpr int R = 1 << RB;
    const u64 q4 = 2 * M.twoq, nq = M.nq;
#pragma unroll
    for (int st = 0; st < S; st++) {
        const int kb = KB0 + st;
        const int s = s0 + st;
        const int base = (1 << s) + (tau & ((1 << lo) - 1));
#pragma unroll
        for (int k = 0; k < R; k++) {
            if (k & (1 << kb)) continue;
            const int widx = base + ((k & ((1 << kb) - 1)) << lo);
            const ulonglong2 Wp = __ldg(M.iw + widx);
            u64 X = v[k];
            if (!LAZY) X = X >= q4 ? X - q4 : X;
            const u64 Tt = shoup4(v[k | (1 << kb)], Wp.x, Wp.y, nq);
            v[k] = X + Tt;
            v[k | (1 << kb)] = X - Tt + q4;
        }
    }
}

// The element bits that a thread's warp index (tau >> 5) stands for when the
// register window starts at bit lo (tau holds the element bits below lo and
// those above lo + RB).  An exchange between two windows with the same mask
// moves data only within each warp, over shared-memory words no other warp
// touches, so a warp barrier orders it (measured on the 26,624 digit
// transforms: 1.80 -> 1.72 ms); otherwise it needs the CTA barrier.
template <int LOGN, int RB>
__host__ __device__ constexpr unsigned warp_bits(int lo) {
    unsigned m = 0;
    for (int i = 5; i < LOGN - RB; i++) m |= 1u << (i < lo ? i : i + RB);
    return m;
}

template <int LOGN, int RB>
__device__ __forceinline__ void exchange(u64 *sm, u64 (&v)[1 << RB], int tau, int lo_from, int lo_to) {
    const bool warp_local = warp_bits<LOGN, RB>(lo_from) == warp_bits<LOGN, RB>(lo_to);
#pragma unroll
    for (int k = 0; k < (1 << RB); k++) sm[padi<RB>(jidx<RB>(tau, k, lo_from))] = v[k];
    if (warp_local) __syncwarp();
    else __syncthreads();
#pragma unroll
    for (int k = 0; k < (1 << RB); k++) v[k] = sm[padi<RB>(jidx<RB>(tau, k, lo_to))];
    if (warp_local) __syncwarp();
    else __syncthreads();
}

// Work-list items: a launch whose moduli are not all below 2^57 is compiled
// without the lazy bound (LAZY = false), yet each item whose own modulus is
// below 2^57 still takes the lazy transform (the choice is uniform over a
// block).  Measured on 256 uneven jobs with 36-60-bit limbs: 24.18 -> 23.51 ms.
// The one-call grid kernels keep the launch-wide choice: there the second
// inlined transform raised the spills and the plain per-job launches lost 1%.
__device__ __forceinline__ bool lazy_mod(const ModDev &M) { return M.q < (1ull << 57); }

// ---------------------------------------------------------------- per-polynomial building blocks
// Load one limb polynomial into the first register window (bits [LOGN-4,
// LOGN): element k*T + tau, coalesced), reducing / lifting it into [0, q).
template <int LOGN>
__device__ __forceinline__ void fwd_load(int kind, const void *src, u64 t, const ModDev &M, int tau, u64 (&v)[Cfg<LOGN>::R]) {
    constexpr int T = Cfg<LOGN>::T, R = Cfg<LOGN>::R;
    switch (kind) {
    case SRC_RNS: {
        const u64 *s = (const u64 *)src;
#pragma unroll
        for (int k = 0; k < R; k++) v[k] = s[k * T + tau];
        break;
    }
    case SRC_T_LIFT: {
        const u64 *s = (const u64 *)src;
        const u64 half = (t - 1) / 2;
#pragma unroll
        for (int k = 0; k < R; k++) {
            u64 x = s[k * T + tau];
            x = x >= t ? x % t : x;
            v[k] = x <= half ? x : M.q - (t - x);
        }
        break;
    }
    case SRC_I8: {
        const int8_t *s = (const int8_t *)src;
#pragma unroll
        for (int k = 0; k < R; k++) {
            const int x = s[k * T + tau];
            v[k] = x >= 0 ? (u64)x : M.q - (u64)(-x);
        }
        break;
    }
    case SRC_U32: {
        const uint32_t *s = (const uint32_t *)src;
#pragma unroll
        for (int k = 0; k < R; k++) v[k] = s[k * T + tau];
        break;
    }
    default: {  // SRC_T_RAW
        const u64 *s = (const u64 *)src;
#pragma unroll
        for (int k = 0; k < R; k++) v[k] = reduce64(s[k * T + tau], M.q, M.one_s);
        break;
    }
    }
}

// Forward transform of a loaded polynomial and its store in register-tile
// order (position k*T + tau), fully reduced.
template <int LOGN, bool LAZY>
__device__ __forceinline__ void fwd_transform_store(u64 (&v)[Cfg<LOGN>::R], u64 *sm, int tau, const ModDev &M,
                                                    u64 *d) {
    constexpr int T = Cfg<LOGN>::T, NP = Cfg<LOGN>::NP, RL = Cfg<LOGN>::RL, RB = Cfg<LOGN>::RB, R = Cfg<LOGN>::R;
    int lo = LOGN - RB;
#pragma unroll
    for (int pass = 0; pass < NP - 1; pass++) {
        fwd_pass<RB, RB, LAZY, Cfg<LOGN>::COARSE_FWD>(v, tau, lo, RB * pass, M);
        const int lo_next = pass == NP - 2 ? 0 : lo - RB;
        exchange<LOGN, RB>(sm, v, tau, lo, lo_next);
        lo = lo_next;
    }
    fwd_pass<RB, RL, LAZY, Cfg<LOGN>::COARSE_FWD>(v, tau, 0, RB * (NP - 1), M);
#pragma unroll
    for (int k = 0; k < R; k++) d[k * T + tau] = reduce_small(v[k], M);  // from [0, 57q) or [0, 8q)
}

// sum over terms [t0, t1) of A[ta + limb] * B[tb + limb] in the NTT domain,
// in groups of CH coefficients (128-bit sums), times 2^-64 (a Montgomery
// reduction ends each sum; the untwist table carries the 2^64 back), fully
// reduced.  Every M.fold products the sum is folded exactly to below q, so
// the final sum stays below q (1 + (M.fold - 1) q) <= q 2^64.  The
// finished groups wait in shared memory (the exchange buffer is idle until
// the inverse transform), so the registers go to loads in flight: the term
// loop is unrolled by two.  Thread tau parks coefficient k in the slot its
// inverse transform's first exchange (from the window at bit 0) writes
// register k to, so no thread touches another's slots before that exchange
// and no CTA barrier is needed here.  The caller's shared buffer must be
// free on entry (no thread still reading a previous exchange).
template <int LOGN, int CH>
__device__ __forceinline__ void mac_accumulate(const u64 *__restrict__ A, const u64 *__restrict__ B,
                                               const int32_t *__restrict__ ta, const int32_t *__restrict__ tb, int t0,
                                               int t1, int limb, const ModDev &M, int tau, u64 (&v)[Cfg<LOGN>::R],
                                               u64 *sm) {
    constexpr int N = Cfg<LOGN>::N, T = Cfg<LOGN>::T, R = Cfg<LOGN>::R;
#pragma unroll 1
    for (int part = 0; part < R / CH; part++) {
        u64 lo[CH], hi[CH];
#pragma unroll
        for (int kk = 0; kk < CH; kk++) { lo[kk] = 0; hi[kk] = 0; }
        int cnt = 0;
#pragma unroll 2
        for (int tk = t0; tk < t1; tk++) {
            const u64 *a = A + ((long long)ta[tk] + limb) * N + part * CH * T + tau;
            const u64 *b = B + ((long long)tb[tk] + limb) * N + part * CH * T + tau;
#pragma unroll
            for (int kk = 0; kk < CH; kk++) {
                u64 pl, ph;
                mul128(a[kk * T], b[kk * T], pl, ph);
                lo[kk] += pl;
                hi[kk] += ph + (lo[kk] < pl);
            }
            if (++cnt == M.fold) {  // also keeps the 128-bit sum of products < 2^124 from overflowing
#pragma unroll
                for (int kk = 0; kk < CH; kk++) { lo[kk] = reduce128(lo[kk], hi[kk], M); hi[kk] = 0; }
                cnt = 0;
            }
        }
#pragma unroll
        for (int kk = 0; kk < CH; kk++)
            sm[padi<Cfg<LOGN>::RB>(jidx<Cfg<LOGN>::RB>(tau, part * CH + kk, 0))] = redc(lo[kk], hi[kk], M);
    }
#pragma unroll
    for (int k = 0; k < R; k++) v[k] = sm[padi<Cfg<LOGN>::RB>(jidx<Cfg<LOGN>::RB>(tau, k, 0))];
}

// Inverse transform: the register-tile bits [0, RB) first, then upward; the
// last window is the top RB bits [LOGN-RB, LOGN) holding the remaining RL
// stages, and leaves every thread with the natural-order elements k*T + tau
// (before the untwist / N^-1 scaling).
template <int LOGN, bool LAZY>
__device__ __forceinline__ void inv_transform(u64 (&v)[Cfg<LOGN>::R], u64 *sm, int tau, const ModDev &M) {
    constexpr int NP = Cfg<LOGN>::NP, RL = Cfg<LOGN>::RL, RB = Cfg<LOGN>::RB;
    inv_pass<RB, RB, 0, LAZY>(v, tau, 0, 0, M);
    if (LOGN == 13) {
        // windows at bits 0, 4, 5, 9: the single stage on bit 8 runs in the
        // window at bit 5, so the exchanges 0 -> 4 and 4 -> 5 stay within each
        // warp and only 5 -> 9 needs the CTA barrier (with windows 0, 4, 8, 9
        // two of the three would)
        exchange<LOGN, RB>(sm, v, tau, 0, RB);
        inv_pass<RB, RB, 0, LAZY>(v, tau, RB, RB, M);
        exchange<LOGN, RB>(sm, v, tau, RB, 2 * RB - 3);
        inv_pass<RB, 1, RB - 1, LAZY>(v, tau, 2 * RB - 3, 2 * RB, M);
        exchange<LOGN, RB>(sm, v, tau, 2 * RB - 3, LOGN - RB);
        inv_pass<RB, RB, 0, LAZY>(v, tau, LOGN - RB, LOGN - RB, M);
        return;
    }
    int lo = 0;
#pragma unroll
    for (int pass = 1; pass < NP - 1; pass++) {
        exchange<LOGN, RB>(sm, v, tau, lo, RB * pass);
        lo = RB * pass;
        inv_pass<RB, RB, 0, LAZY>(v, tau, lo, RB * pass, M);
    }
    exchange<LOGN, RB>(sm, v, tau, lo, LOGN - RB);
    inv_pass<RB, RL, RB - RL, LAZY>(v, tau, LOGN - RB, RB * (NP - 1), M);
}

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
    const ModDev M = mods[J.mod_base + limb];
    u64 v[Cfg<LOGN>::R];
    mac_accumulate<LOGN, mac_group(Cfg<LOGN>::T, Cfg<LOGN>::MINB)>(J.A, J.B, J.ta, J.tb, J.ptr[o], J.ptr[o + 1], limb, M, tau,
                                                                   v, sm);
    inv_transform<LOGN, LAZY>(v, sm, tau, M);
    // natural order: element j = k*T + tau
    const u64 q = M.q;
    u64 *out = J.out + (long long)o * J.out_stride + (long long)limb * N;
    const u64 *add = J.add ? J.add + (long long)o * J.add_stride + (long long)limb * N : nullptr;
    const int8_t *err = J.err ? J.err + (long long)o * J.err_stride : nullptr;
    const u64 *msg = (J.msg && (o % J.msg_div) == 0) ? J.msg + (long long)(o / J.msg_div) * J.msg_stride : nullptr;
    const u64 *s2 = J.s2 ? J.s2 + (long long)limb * N : nullptr;
    u64 g = 0, gs = 0, dl = 0, dls = 0;
    if (s2) { g = J.gmul[2 * ((long long)o * J.n_limbs + limb)]; gs = J.gmul[2 * ((long long)o * J.n_limbs + limb) + 1]; }
    if (msg) { dl = J.E->delta_q[J.mod_base + limb]; dls = J.E->delta_qs[J.mod_base + limb]; }
    const u64 t = msg ? J.E->t : 0;
#pragma unroll
    for (int k = 0; k < Cfg<LOGN>::R; k++) {
        const int x = k * T + tau;
        const ulonglong2 zp = __ldg(M.z + x);
        u64 r = red1(shoup(v[k], zp.x, zp.y, q), q);
        if (err) {
            const int e = err[x];
            r = e >= 0 ? addm(r, (u64)e, q) : subm(r, (u64)(-e), q);
        }
        if (J.negate) r = r ? q - r : 0;
        if (s2) r = addm(r, red1(shoup(s2[x], g, gs, q), q), q);
        if (msg) {
            u64 m = msg[x];
            m = m >= t ? m % t : m;
            r = addm(r, red1(shoup(m, dl, dls, q), q), q);
        }
        if (add) r = addm(r, add[x], q);
        out[x] = r;
    }
}

// ---------------------------------------------------------------- persistent queue kernels
// Each CTA repeatedly takes the next item index of a launch (one atomic per
// item) until all `total` items are done; items live in `nseg` segments (an
// item array each, with the index of its first item) so a launch can cover
// several independently built work lists.  Items of one launch share the ring
// degree but may use any modulus of any context.  The counter must be zero
// at launch.
// Multiply-accumulate, inverse transform and store of one item.  The item is
// read through its pointer where each field is needed (the output pointers
// only after the transform's barriers), so no field stays live in registers
// across the transform.
template <int LOGN, int MINB, bool LAZY>
__device__ __forceinline__ void mac_item(const MacItem *__restrict__ ip, u64 *sm, int tau) {
    constexpr int T = Cfg<LOGN>::T;
    const ModDev *__restrict__ mp = ip->mod;  // read-only: fields may be re-read rather than kept live
    const ModDev M = *mp;
    u64 v[Cfg<LOGN>::R];
    mac_accumulate<LOGN, mac_group(Cfg<LOGN>::T, MINB)>(ip->A, ip->B, ip->ta, ip->tb, ip->t0, ip->t1, ip->limb, M, tau,
                                                        v, sm);
    if (LAZY || lazy_mod(M)) inv_transform<LOGN, true>(v, sm, tau, M);
    else inv_transform<LOGN, false>(v, sm, tau, M);
    u64 *out = ip->out;
    const u64 *add = ip->add;
    const u64 q = M.q;
#pragma unroll
    for (int k = 0; k < Cfg<LOGN>::R; k++) {
        const int x = k * T + tau;
        const ulonglong2 zp = __ldg(M.z + x);
        u64 r = red1(shoup(v[k], zp.x, zp.y, q), q);
        if (add) r = addm(r, add[x], q);
        out[x] = r;
    }
}

template <int LOGN, bool LAZY>
__device__ __forceinline__ void fwd_item(const FwdItem *__restrict__ ip, u64 *sm, int tau) {
    const ModDev *__restrict__ mp = ip->mod;
    const ModDev M = *mp;
    u64 v[Cfg<LOGN>::R];
    fwd_load<LOGN>(ip->kind, ip->src, ip->t, M, tau, v);
    if (LAZY || lazy_mod(M)) fwd_transform_store<LOGN, true>(v, sm, tau, M, ip->dst);
    else fwd_transform_store<LOGN, false>(v, sm, tau, M, ip->dst);
}

template <typename ITEM>
__device__ __forceinline__ const ITEM *next_item(const ItemSeg *segs, int nseg, int total, int *counter,
                                                 int *s_meta) {
    if (threadIdx.x == 0) {
        const int it = atomicAdd(counter, 1);
        int sidx = 0;
        if (it < total) {
            int lo = 0, hi = nseg - 1;  // last segment whose begin <= it
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (segs[mid].begin <= it) lo = mid;
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
    return (const ITEM *)segs[sidx].items + (it - segs[sidx].begin);
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
        if (segs[mid].begin <= it) lo = mid;
        else hi = mid - 1;
    }
    return (const ITEM *)segs[lo].items + (it - segs[lo].begin);
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
        cudaFuncSetAttribute(k_fwd<LOGN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
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
    if (lazy) k_fwd<LOGN, true><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(JS, c->d_mods);
    else k_fwd<LOGN, false><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(JS, c->d_mods);
    return cuda_check(c, cudaGetLastError(), "k_fwd");
}

template <int LOGN>
static int mac_t(he_ctx *c, const MacJob *jobs, int n, cudaStream_t st) {
    const int smem = Cfg<LOGN>::SMEM;
    static std::atomic<unsigned long long> attr_mask{0};
    if (first_on_device(attr_mask)) {
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
        mm += (double)b * ((N / 2) * LOGN + 3.0 * N) + (double)j.n_terms * N * j.n_limbs;
    }
    if (blocks == 0) return HE_OK;
    if (blocks > 0x7fffffffLL) return fail(c, HE_ERR_INVALID_ARG, "multiply-accumulate launch too large");
    const bool lazy = lazy_ok(c, jobs[0].mod_base, jobs[0].n_limbs);
    TraceScope ts(c, st, "mac_intt", bytes, mm);
    if (lazy) k_mac_intt<LOGN, true><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(JS, c->d_mods);
    else k_mac_intt<LOGN, false><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(JS, c->d_mods);
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
    return lazy ? queue_l<LOGN, MINB, true>(fwd, segs, nseg, total, counter, grid, st)
                : queue_l<LOGN, MINB, false>(fwd, segs, nseg, total, counter, grid, st);
}

int launch_queue(int logN, int minb, bool fwd, bool lazy, const ItemSeg *segs, int nseg, int total, int *counter,
                 int grid, cudaStream_t st) {
    if (total <= 0 || nseg <= 0) return HE_OK;
    switch (logN * 2 + (minb >= 2 ? 1 : 0)) {
    case 20: return queue_t<10, 1>(fwd, lazy, segs, nseg, total, counter, grid, st);
    case 21: return queue_t<10, 2>(fwd, lazy, segs, nseg, total, counter, grid, st);
    case 22: return queue_t<11, 1>(fwd, lazy, segs, nseg, total, counter, grid, st);
    case 23: return queue_t<11, 2>(fwd, lazy, segs, nseg, total, counter, grid, st);
    case 24: return queue_t<12, 1>(fwd, lazy, segs, nseg, total, counter, grid, st);
    case 25: return queue_t<12, 2>(fwd, lazy, segs, nseg, total, counter, grid, st);
    case 26: return queue_t<13, 1>(fwd, lazy, segs, nseg, total, counter, grid, st);
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
