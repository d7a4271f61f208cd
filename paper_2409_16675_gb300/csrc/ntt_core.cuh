// ntt_core.cuh -- device building blocks of the negacyclic NTT kernels over RNS
// limbs (used by the grid and work-list kernels of ntt.cu and the fused
// batch kernel of fused.cu).
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
#pragma once
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
            const ulonglong2 Wp = HE_LDG(M.fw + widx);
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
            const ulonglong2 Wp = HE_LDG(M.iw + widx);
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

// Barrier of the threads that share one transform: the whole CTA, or one half
// of it (a named barrier) when a CTA runs two transforms of half the size.
struct CtaSync {
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct HalfSync {
    int id, nthreads;  // barrier 1 or 2 (0 is the CTA barrier); threads of the half
    __device__ __forceinline__ void sync() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
    }
};

template <int LOGN, int RB, class SYNC>
__device__ __forceinline__ void exchange(u64 *sm, u64 (&v)[1 << RB], int tau, int lo_from, int lo_to, const SYNC &sy) {
    const bool warp_local = warp_bits<LOGN, RB>(lo_from) == warp_bits<LOGN, RB>(lo_to);
#pragma unroll
    for (int k = 0; k < (1 << RB); k++) sm[padi<RB>(jidx<RB>(tau, k, lo_from))] = v[k];
    if (warp_local) __syncwarp();
    else sy.sync();
#pragma unroll
    for (int k = 0; k < (1 << RB); k++) v[k] = sm[padi<RB>(jidx<RB>(tau, k, lo_to))];
    if (warp_local) __syncwarp();
    else sy.sync();
}

// Work-list items: a launch whose moduli are not all below 2^57 is compiled
// without the lazy bound (LAZY = false), yet each item whose own modulus is
// below 2^57 still takes the lazy transform (the choice is uniform over a
// block).  Measured on 256 uneven jobs with 36-60-bit limbs: 24.18 -> 23.51 ms.
// The one-call grid kernels keep the launch-wide choice: there the second
// inlined transform raised the spills and the plain per-job launches lost 1%.
// The bounds-checked build compiles one variant of each kernel (the
// non-lazy transform, valid for every modulus below 2^61, and one register
// budget per ring degree); the variants give the same bits, so only speed
// differs, and its compile time stays a few minutes.
#ifdef HE_CHECKS
constexpr bool kAllVariants = false;
#else
constexpr bool kAllVariants = true;
#endif
__device__ __forceinline__ bool lazy_mod(const ModDev &M) { return kAllVariants && M.q < (1ull << 57); }

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
        for (int k = 0; k < R; k++) v[k] = HE_LD(s + k * T + tau);
        break;
    }
    case SRC_T_LIFT: {
        const u64 *s = (const u64 *)src;
        const u64 half = (t - 1) / 2;
#pragma unroll
        for (int k = 0; k < R; k++) {
            u64 x = HE_LD(s + k * T + tau);
            x = x >= t ? x % t : x;
            v[k] = x <= half ? x : M.q - (t - x);
        }
        break;
    }
    case SRC_I8: {
        const int8_t *s = (const int8_t *)src;
#pragma unroll
        for (int k = 0; k < R; k++) {
            const int x = HE_LD(s + k * T + tau);
            v[k] = x >= 0 ? (u64)x : M.q - (u64)(-x);
        }
        break;
    }
    case SRC_U32: {
        const uint32_t *s = (const uint32_t *)src;
#pragma unroll
        for (int k = 0; k < R; k++) v[k] = HE_LD(s + k * T + tau);
        break;
    }
    default: {  // SRC_T_RAW
        const u64 *s = (const u64 *)src;
#pragma unroll
        for (int k = 0; k < R; k++) v[k] = reduce64(HE_LD(s + k * T + tau), M.q, M.one_s);
        break;
    }
    }
}

// Forward transform of a loaded polynomial and its store in register-tile
// order (position k*T + tau), fully reduced.
// COARSE: the coarser Shoup quotient in the forward passes (where the
// register budget has room for it; see Cfg::COARSE_FWD).
template <int LOGN, bool LAZY, class SYNC = CtaSync, bool COARSE = Cfg<LOGN>::COARSE_FWD>
__device__ __forceinline__ void fwd_transform_store(u64 (&v)[Cfg<LOGN>::R], u64 *sm, int tau, const ModDev &M,
                                                    u64 *d, const SYNC &sy = SYNC()) {
    constexpr int T = Cfg<LOGN>::T, NP = Cfg<LOGN>::NP, RL = Cfg<LOGN>::RL, RB = Cfg<LOGN>::RB, R = Cfg<LOGN>::R;
    int lo = LOGN - RB;
#pragma unroll
    for (int pass = 0; pass < NP - 1; pass++) {
        fwd_pass<RB, RB, LAZY, COARSE>(v, tau, lo, RB * pass, M);
        const int lo_next = pass == NP - 2 ? 0 : lo - RB;
        exchange<LOGN, RB>(sm, v, tau, lo, lo_next, sy);
        lo = lo_next;
    }
    fwd_pass<RB, RL, LAZY, COARSE>(v, tau, 0, RB * (NP - 1), M);
#pragma unroll
    for (int k = 0; k < R; k++) HE_ST(d + k * T + tau, reduce_small(v[k], M));  // from [0, 57q) or [0, 8q)
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
// CG: load the operands with coherent, L1-cached loads (ld.global.ca), never
// through the non-coherent read-only path, for operands that other CTAs of
// the same launch write before this CTA's acquire (the fused batch kernel).
template <int LOGN, int CH, bool CG = false>
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
            const u64 *a = A + ((long long)HE_LD(ta + tk) + limb) * N + part * CH * T + tau;
            const u64 *b = B + ((long long)HE_LD(tb + tk) + limb) * N + part * CH * T + tau;
#pragma unroll
            for (int kk = 0; kk < CH; kk++) {
                u64 pl, ph;
                if (CG) mul128(HE_LDCA(a + kk * T), HE_LDCA(b + kk * T), pl, ph);
                else mul128(HE_LD(a + kk * T), HE_LD(b + kk * T), pl, ph);
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
template <int LOGN, bool LAZY, class SYNC = CtaSync>
__device__ __forceinline__ void inv_transform(u64 (&v)[Cfg<LOGN>::R], u64 *sm, int tau, const ModDev &M,
                                              const SYNC &sy = SYNC()) {
    constexpr int NP = Cfg<LOGN>::NP, RL = Cfg<LOGN>::RL, RB = Cfg<LOGN>::RB;
    inv_pass<RB, RB, 0, LAZY>(v, tau, 0, 0, M);
    if (LOGN == 13) {
        // windows at bits 0, 4, 5, 9: the single stage on bit 8 runs in the
        // window at bit 5, so the exchanges 0 -> 4 and 4 -> 5 stay within each
        // warp and only 5 -> 9 needs the CTA barrier (with windows 0, 4, 8, 9
        // two of the three would)
        exchange<LOGN, RB>(sm, v, tau, 0, RB, sy);
        inv_pass<RB, RB, 0, LAZY>(v, tau, RB, RB, M);
        exchange<LOGN, RB>(sm, v, tau, RB, 2 * RB - 3, sy);
        inv_pass<RB, 1, RB - 1, LAZY>(v, tau, 2 * RB - 3, 2 * RB, M);
        exchange<LOGN, RB>(sm, v, tau, 2 * RB - 3, LOGN - RB, sy);
        inv_pass<RB, RB, 0, LAZY>(v, tau, LOGN - RB, LOGN - RB, M);
        return;
    }
    int lo = 0;
#pragma unroll
    for (int pass = 1; pass < NP - 1; pass++) {
        exchange<LOGN, RB>(sm, v, tau, lo, RB * pass, sy);
        lo = RB * pass;
        inv_pass<RB, RB, 0, LAZY>(v, tau, lo, RB * pass, M);
    }
    exchange<LOGN, RB>(sm, v, tau, lo, LOGN - RB, sy);
    inv_pass<RB, RL, RB - RL, LAZY>(v, tau, LOGN - RB, RB * (NP - 1), M);
}

// ---------------------------------------------------------------- work items
// Multiply-accumulate, inverse transform and store of one item.  The item is
// read through its pointer where each field is needed (the output pointers
// only after the transform's barriers), so no field stays live in registers
// across the transform.
// CH: coefficients per accumulator group (by default the one the register
// budget of a CTA of this tile allows).
template <int LOGN, int MINB, bool LAZY, class SYNC = CtaSync, bool CG = false,
          int CH = mac_group(Cfg<LOGN>::T, MINB)>
__device__ __forceinline__ void mac_item(const MacItem *__restrict__ ip, u64 *sm, int tau, const SYNC &sy = SYNC()) {
    constexpr int T = Cfg<LOGN>::T;
    if (!HE_OBJ_OK(ip)) return;               // (checks build: the item lies in a registered allocation)
    const ModDev *__restrict__ mp = ip->mod;  // read-only: fields may be re-read rather than kept live
    if (!HE_OBJ_OK(mp)) return;
    const ModDev M = *mp;
    u64 v[Cfg<LOGN>::R];
    mac_accumulate<LOGN, CH, CG>(ip->A, ip->B, ip->ta, ip->tb, ip->t0, ip->t1, ip->limb, M, tau, v, sm);
    if (LAZY || lazy_mod(M)) inv_transform<LOGN, true>(v, sm, tau, M, sy);
    else inv_transform<LOGN, false>(v, sm, tau, M, sy);
    u64 *out = ip->out;
    const u64 *add = ip->add;
    const u64 q = M.q;
#pragma unroll
    for (int k = 0; k < Cfg<LOGN>::R; k++) {
        const int x = k * T + tau;
        const ulonglong2 zp = HE_LDG(M.z + x);
        u64 r = red1(shoup(v[k], zp.x, zp.y, q), q);
        if (add) r = addm(r, HE_LD(add + x), q);
        HE_ST(out + x, r);
    }
}

template <int LOGN, bool LAZY, class SYNC = CtaSync, bool COARSE = Cfg<LOGN>::COARSE_FWD>
__device__ __forceinline__ void fwd_item(const FwdItem *__restrict__ ip, u64 *sm, int tau, const SYNC &sy = SYNC()) {
    if (!HE_OBJ_OK(ip)) return;
    const ModDev *__restrict__ mp = ip->mod;
    if (!HE_OBJ_OK(mp)) return;
    const ModDev M = *mp;
    u64 v[Cfg<LOGN>::R];
    fwd_load<LOGN>(ip->kind, ip->src, ip->t, M, tau, v);
    if (LAZY || lazy_mod(M)) fwd_transform_store<LOGN, true, SYNC, COARSE>(v, sm, tau, M, ip->dst, sy);
    else fwd_transform_store<LOGN, false, SYNC, COARSE>(v, sm, tau, M, ip->dst, sy);
}

}  // namespace he
