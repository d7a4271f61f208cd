// keyswitch.cu -- the relinearisation key switch over small primes (Section 2,
// Motivation: CCMul needs relinearisation, Fig. 3(b)).
//
// For output o, component comp and limb i the key switch adds
// E_i = sum_j D_j rlk_{j,comp,i} to the rescaled d_comp, where D_j < 2^base are
// the digits of d2 and the product is in Z[x]/(x^N + 1).  Every coefficient
// of E_i is an integer of magnitude below ell N (2^base - 1)(q_i - 1), so it is
// fixed by its residues modulo a few primes p_k < 2^30 whose product P exceeds
// four times that bound (three primes for N = 8192, four 50-bit limbs,
// base 2^16).  The work then runs in the SM's native 32-bit arithmetic:
//   k_ks_fwd   digits (and, once per key, the key residues) to the NTT domain
//              modulo every p_k: ell * np transforms per output instead of
//              ell * L over the 50-bit limbs;
//   k_ks_mac   per (o, i, comp): for every p_k, sum_j of 32 x 32-bit products
//              in 64-bit registers (one wide multiply-add per term), one
//              Montgomery fold, the inverse transform mod p_k and the
//              untwist; the residues of the first np - 1 primes wait in a
//              global scratch that stays in L2 (each thread rereads its own
//              words), so shared memory holds only the exchange buffer and
//              three CTAs fit on an SM; then the mixed-radix (Garner) CRT gives
//              E_i mod q_i, which is added to d_comp and stored.
// The bits equal those of the key switch over the limbs (the sum is exact
// either way); contexts with a limb below 2^31 keep that one (four primes
// cover the sums of every other supported parameter set).
//
// 32-bit arithmetic: Shoup products a w - floor(a w' / 2^32) p lie in [0, 2p)
// for every 32-bit a (w' = floor(w 2^32 / p)); the butterflies keep Harvey's
// bounds (inputs below 4p, X brought below 2p, outputs below 4p < 2^32).
#include <atomic>
#include <cstring>

#include "ntt_core.cuh"

namespace he {

typedef uint32_t u32;

__device__ __forceinline__ u32 shoup32(u32 a, u32 w, u32 ws, u32 p) { return a * w - __umulhi(a, ws) * p; }
__device__ __forceinline__ u32 red32(u32 a, u32 p) { return a >= p ? a - p : a; }
// a 32-bit value below 2^32 taken into [0, 2p) (Shoup product by 1)
__device__ __forceinline__ u32 lift32(u32 a, const Mod32Dev &M) { return a - __umulhi(a, M.ones) * M.p; }

// Exact fold of a 64-bit sum T = h 2^32 + l: (h mod p)(2^32 mod p) + l, the
// same residue, below (p - 1)^2 + 2^32.
__device__ __forceinline__ u64 fold32(u64 T, const Mod32Dev &M) {
    const u32 h = red32(lift32((u32)(T >> 32), M), M.p);
    return (u64)h * M.r32 + (u32)T;
}

// Montgomery reduction of a 64-bit sum T: T 2^-32 mod p, in [0, p).  The high word
// is first brought below p, so T' = h 2^32 + l < p 2^32 and T' + m p (m = l
// (-p^-1) mod 2^32) is a multiple of 2^32 below 2p 2^32.
__device__ __forceinline__ u32 mont32(u64 T, const Mod32Dev &M) {
    u32 h = (u32)(T >> 32);
    const u32 l = (u32)T;
    if (h >= M.p) h = red32(lift32(h, M), M.p);
    const u32 m = l * M.pinv;
    const u64 s = ((((u64)h) << 32) | l) + (u64)m * M.p;
    return red32((u32)(s >> 32), M.p);
}

// Forward pass (as fwd_pass in ntt_core.cuh, the same permuted factor order).
template <int RB, int S>
__device__ __forceinline__ void fwd_pass32(u32 (&v)[1 << RB], int tau, int lo, int s0, const Mod32Dev &M) {
    constexpr int R = 1 << RB;
    const u32 p = M.p, p2 = M.twop;
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
            const uint2 W = HE_LDG(M.fw + widx);
            u32 X = v[k];
            X = X >= p2 ? X - p2 : X;
            const u32 T = shoup32(v[k | (1 << kb)], W.x, W.y, p);
            v[k] = X + T;
            v[k | (1 << kb)] = X - T + p2;
        }
    }
}

// Decimation-in-time pass of the inverse (as inv_pass in ntt_core.cuh).
template <int RB, int S, int KB0>
__device__ __forceinline__ void inv_pass32(u32 (&v)[1 << RB], int tau, int lo, int s0, const Mod32Dev &M) {
    constexpr int R = 1 << RB;
    const u32 p = M.p, p2 = M.twop;
#pragma unroll
    for (int st = 0; st < S; st++) {
        const int kb = KB0 + st;
        const int s = s0 + st;
        const int base = (1 << s) + (tau & ((1 << lo) - 1));
#pragma unroll
        for (int k = 0; k < R; k++) {
            if (k & (1 << kb)) continue;
            const int widx = base + ((k & ((1 << kb) - 1)) << lo);
            const uint2 W = HE_LDG(M.iw + widx);
            u32 X = v[k];
            X = X >= p2 ? X - p2 : X;
            const u32 T = shoup32(v[k | (1 << kb)], W.x, W.y, p);
            v[k] = X + T;
            v[k | (1 << kb)] = X - T + p2;
        }
    }
}

template <int LOGN, int RB>
__device__ __forceinline__ void exchange32(u32 *sm, u32 (&v)[1 << RB], int tau, int lo_from, int lo_to) {
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

// NTT-domain order of the 32-bit forms: register k of thread tau after the
// last forward pass (the register-tile element 16 tau + k of the transform)
// sits at word 4 ((k / 4) T + tau) + k % 4, so each thread stores and loads
// its coefficients four at a time (16-byte accesses, 512 contiguous bytes
// per warp); the multiply-accumulate reads both operands in this order and
// its inverse transform starts from the same register tile.
// Forward transform of loaded values (below 4p) and store, reduced into [0, p).
template <int LOGN>
__device__ __forceinline__ void fwd32_store(u32 (&v)[Cfg<LOGN>::R], u32 *sm, int tau, const Mod32Dev &M, u32 *d) {
    constexpr int T = Cfg<LOGN>::T, NP = Cfg<LOGN>::NP, RL = Cfg<LOGN>::RL, RB = Cfg<LOGN>::RB, R = Cfg<LOGN>::R;
    static_assert(R % 4 == 0, "four coefficients per 16-byte store");
    int lo = LOGN - RB;
#pragma unroll
    for (int pass = 0; pass < NP - 1; pass++) {
        fwd_pass32<RB, RB>(v, tau, lo, RB * pass, M);
        const int lo_next = pass == NP - 2 ? 0 : lo - RB;
        exchange32<LOGN, RB>(sm, v, tau, lo, lo_next);
        lo = lo_next;
    }
    fwd_pass32<RB, RL>(v, tau, 0, RB * (NP - 1), M);
    uint4 *d4 = (uint4 *)d + tau;
#pragma unroll
    for (int m = 0; m < R / 4; m++) {
        uint4 w;
        w.x = red32(red32(v[4 * m], M.twop), M.p);
        w.y = red32(red32(v[4 * m + 1], M.twop), M.p);
        w.z = red32(red32(v[4 * m + 2], M.twop), M.p);
        w.w = red32(red32(v[4 * m + 3], M.twop), M.p);
        HE_ST(d4 + m * T, w);
    }
}

// Inverse transform (the window schedule of inv_transform in ntt_core.cuh);
// leaves element k*T + tau of the natural order in v[k], below 4p.
template <int LOGN>
__device__ __forceinline__ void inv32(u32 (&v)[Cfg<LOGN>::R], u32 *sm, int tau, const Mod32Dev &M) {
    constexpr int NP = Cfg<LOGN>::NP, RL = Cfg<LOGN>::RL, RB = Cfg<LOGN>::RB;
    inv_pass32<RB, RB, 0>(v, tau, 0, 0, M);
    if (LOGN == 13) {
        exchange32<LOGN, RB>(sm, v, tau, 0, RB);
        inv_pass32<RB, RB, 0>(v, tau, RB, RB, M);
        exchange32<LOGN, RB>(sm, v, tau, RB, 2 * RB - 3);
        inv_pass32<RB, 1, RB - 1>(v, tau, 2 * RB - 3, 2 * RB, M);
        exchange32<LOGN, RB>(sm, v, tau, 2 * RB - 3, LOGN - RB);
        inv_pass32<RB, RB, 0>(v, tau, LOGN - RB, LOGN - RB, M);
        return;
    }
    int lo = 0;
#pragma unroll
    for (int pass = 1; pass < NP - 1; pass++) {
        exchange32<LOGN, RB>(sm, v, tau, lo, RB * pass);
        lo = RB * pass;
        inv_pass32<RB, RB, 0>(v, tau, lo, RB * pass, M);
    }
    exchange32<LOGN, RB>(sm, v, tau, lo, LOGN - RB);
    inv_pass32<RB, RL, RB - RL>(v, tau, LOGN - RB, RB * (NP - 1), M);
}

// One Garner digit: y_k = (((r_k - y_0) p_0^-1 - y_1) p_1^-1 - ...) p_{k-1}^-1
// mod p_k over the first k digits (y_m < p_m < 2 p_k: one subtraction brings
// each below p_k).
__device__ __forceinline__ u32 garner_step(u32 r, u32 p, const u32 *ginv, const u32 *ginvs, u32 y0, u32 y1, u32 y2,
                                           int k) {
    const u32 ys[3] = {y0, y1, y2};
    u32 t = r;
#pragma unroll
    for (int m = 0; m < 3; m++) {
        if (m < k) {
            const u32 ym = red32(ys[m], p);
            t = t >= ym ? t - ym : t + p - ym;
            t = red32(shoup32(t, ginv[m], ginvs[m], p), p);
        }
    }
    return t;
}

// ---------------------------------------------------------------- kernels
// Forward transforms modulo every small prime: blockIdx.x = p np + k for
// source polynomial p and prime k, so the np CTAs reading one source run side
// by side and all but the first find it in L2; u32 sources are digits
// (< 2^32, taken below 2p), u64 sources key residues (< 2^61, reduced mod p
// once per key).
template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T, (LOGN >= 14 ? 1 : 3))
    k_ks_fwd(const void *__restrict__ src, int u64_src, u32 *__restrict__ dst, const __grid_constant__ KsDev ks) {
    extern __shared__ u32 sm32[];
    constexpr int N = Cfg<LOGN>::N, T = Cfg<LOGN>::T, R = Cfg<LOGN>::R;
    const int tau = threadIdx.x;
    const int p = (int)blockIdx.x / ks.np, k = (int)blockIdx.x - p * ks.np;
    const Mod32Dev M = ks.m[k];
    u32 v[R];
    if (u64_src) {
        const u64 *s = (const u64 *)src + (long long)p * N + tau;
#pragma unroll
        for (int kk = 0; kk < R; kk++) v[kk] = (u32)(HE_LD(s + kk * T) % M.p);
    } else {
        const u32 *s = (const u32 *)src + (long long)p * N + tau;
#pragma unroll
        for (int kk = 0; kk < R; kk++) v[kk] = lift32(HE_LD(s + kk * T), M);
    }
    fwd32_store<LOGN>(v, sm32, tau, M, dst + ((long long)p * ks.np + k) * N);
}

struct KsMacArgs {
    const u32 *dig;    // [n_out][ell][np][N] NTT form
    const u32 *rlk32;  // [ell][2][L][np][N] NTT form
    const u64 *add;    // [n_out][2][L][N] coefficient form (rescaled d0, d1)
    u64 *out;          // [n_out][2][L][N]
    u32 *park;         // [n_out * L * 2][np - 1][N] residues of the first np - 1 primes
    int ell, L;
};

// One CTA per (output o, limb i, component comp): blockIdx.x = (o L + i) 2 +
// comp, so the 2L CTAs that read one output's digits run side by side.
// CH: coefficients per group of 64-bit sums.  Three resident CTAs per SM
// (40 registers) below N = 16384.
template <int LOGN, int CH>
__global__ void __launch_bounds__(Cfg<LOGN>::T, (LOGN >= 14 ? 1 : 3))
    k_ks_mac(const KsMacArgs a, const __grid_constant__ KsDev ks, const ModDev *__restrict__ mods) {
    extern __shared__ u32 sm32[];
    constexpr int N = Cfg<LOGN>::N, T = Cfg<LOGN>::T, R = Cfg<LOGN>::R;
    // residues of primes 0 .. np-2, [k][N]; each thread rereads only its own words
    u32 *park = a.park + (long long)blockIdx.x * (ks.np - 1) * N;
    const int tau = threadIdx.x;
    const int comp = blockIdx.x & 1, oi = blockIdx.x >> 1;
    const int L = a.L, ell = a.ell, np = ks.np;
    const int o = oi / L, i = oi - o * L;
    if (!HE_OBJ_OK(mods + i)) return;  // uniform over the CTA
    static_assert(CH % 4 == 0, "accumulator groups of whole 16-byte loads");
    const long long sA = (long long)np * N / 4, sB = 2LL * L * np * N / 4;  // 16-byte words between terms
    u32 v[R];
#pragma unroll 1
    for (int k = 0; k < np; k++) {
        const Mod32Dev M = ks.m[k];
        const uint4 *A = (const uint4 *)(a.dig + ((long long)o * ell * np + k) * N) + tau;
        const uint4 *B = (const uint4 *)(a.rlk32 + ((long long)(comp * L + i) * np + k) * N) + tau;
        // sum_j A_j B_j: one 32 x 32 -> 64-bit multiply-add per term, folded
        // exactly every ks.fold terms (ell is below it at the usual digit
        // bases) and Montgomery-reduced (times 2^-32) at the end; the term
        // loop is unrolled by two so that two terms' loads are in flight
#pragma unroll
        for (int part = 0; part < R / CH; part++) {
            u64 acc[CH];
#pragma unroll
            for (int kk = 0; kk < CH; kk++) acc[kk] = 0;
            int cnt = 0;
#pragma unroll 2
            for (int j = 0; j < ell; j++) {
                const uint4 *aj = A + j * sA + part * (CH / 4) * T;
                const uint4 *bj = B + j * sB + part * (CH / 4) * T;
#pragma unroll
                for (int g = 0; g < CH / 4; g++) {
                    const uint4 x = HE_LDG(aj + g * T), y = HE_LDG(bj + g * T);
                    acc[4 * g] += (u64)x.x * y.x;
                    acc[4 * g + 1] += (u64)x.y * y.y;
                    acc[4 * g + 2] += (u64)x.z * y.z;
                    acc[4 * g + 3] += (u64)x.w * y.w;
                }
                if (++cnt == ks.fold) {
#pragma unroll
                    for (int kk = 0; kk < CH; kk++) acc[kk] = fold32(acc[kk], M);
                    cnt = 0;
                }
            }
#pragma unroll
            for (int kk = 0; kk < CH; kk++) v[part * CH + kk] = mont32(acc[kk], M);
        }
        __syncthreads();  // no thread still reads the exchange buffer (previous prime's transform)
        inv32<LOGN>(v, sm32, tau, M);
        // untwist psi^-x N^-1 2^32: residue of E_i mod p_k at element x = kk T + tau
#pragma unroll
        for (int kk = 0; kk < R; kk++) {
            const int x = kk * T + tau;
            const uint2 z = HE_LDG(M.z + x);
            const u32 r = red32(shoup32(v[kk], z.x, z.y, M.p), M.p);
            if (k < np - 1) HE_ST(park + k * N + x, r);
            else v[kk] = r;
        }
    }
    // Garner CRT of the np residues, E_i mod q_i, plus d_comp
    const u64 q = mods[i].q, one_s = mods[i].one_s;
    const long long off = ((long long)(o * 2 + comp) * L + i) * N;
    const u64 *add = a.add + off;
    u64 *out = a.out + off;
    static_assert(kKsMaxPrimes == 4, "the CRT below is written out for up to four primes");
    const u32 p0 = ks.m[0].p, p1 = ks.m[1].p, p2 = ks.m[2].p, p3 = ks.m[3].p;
#pragma unroll
    for (int kk = 0; kk < R; kk++) {
        const int x = kk * T + tau;
        // residues r_k (the last prime's in v) and the mixed-radix digits y_k
        const u32 y0 = HE_LD(park + x);
        const u32 y1 = garner_step(np > 2 ? HE_LD(park + N + x) : v[kk], p1, ks.ginv[1], ks.ginvs[1], y0, 0, 0, 1);
        u32 y2 = 0, y3 = 0;
        if (np > 2)
            y2 = garner_step(np > 3 ? HE_LD(park + 2 * N + x) : v[kk], p2, ks.ginv[2], ks.ginvs[2], y0, y1, 0, 2);
        if (np > 3) y3 = garner_step(v[kk], p3, ks.ginv[3], ks.ginvs[3], y0, y1, y2, 3);
        // E' = y_0 + p_0 (y_1 + p_1 (y_2 + p_2 y_3)) mod q_i: the innermost
        // step is exact (below 2^60), the rest Shoup products
        u64 e;
        u32 ytop;
        if (np == 2) {
            e = reduce64((u64)y1 * p0 + y0, q, one_s);
            ytop = y1;
        } else if (np == 3) {
            e = reduce64((u64)y2 * p1 + y1, q, one_s);
            e = addm(red1(shoup(e, p0, ks.pq_s[i][0], q), q), (u64)y0, q);
            ytop = y2;
        } else {
            e = reduce64((u64)y3 * p2 + y2, q, one_s);
            e = addm(red1(shoup(e, p1, ks.pq_s[i][1], q), q), (u64)y1, q);
            e = addm(red1(shoup(e, p0, ks.pq_s[i][0], q), q), (u64)y0, q);
            ytop = y3;
        }
        if (ytop > ks.half_top) e = subm(e, ks.P_q[i], q);  // E < 0: E' - P
        HE_ST(out + x, addm(e, HE_LD(add + x), q));
    }
}

// ---------------------------------------------------------------- launchers
// True the first time a call site runs on the current device (kernel
// attributes are per device).
static bool ks_first_on_device(std::atomic<unsigned long long> &mask) {
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (mask.load(std::memory_order_acquire) & bit) return false;
    mask.fetch_or(bit, std::memory_order_acq_rel);
    return true;
}


template <int LOGN>
static int ks_fwd_t(he_ctx *c, const void *src, bool u64_src, int n_polys, u32 *dst, cudaStream_t st) {
    constexpr int N = Cfg<LOGN>::N;
    const int smem = (N + N / Cfg<LOGN>::R) * 4;
    static std::atomic<unsigned long long> attr_mask{0};
    if (ks_first_on_device(attr_mask))
        cudaFuncSetAttribute(k_ks_fwd<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int np = c->h_ks.np;
    const double bytes = (double)n_polys * N * ((u64_src ? 8.0 : 4.0) + 4.0 * np);
    TraceScope ts(c, st, "ks_fwd", bytes, (double)n_polys * np * (N / 2) * LOGN);
    if ((long long)n_polys * np > 0x7fffffffLL) return fail(c, HE_ERR_INVALID_ARG, "key-switch launch too large");
    k_ks_fwd<LOGN><<<(unsigned)(n_polys * np), Cfg<LOGN>::T, smem, st>>>(src, u64_src ? 1 : 0, dst, c->h_ks);
    return cuda_check(c, cudaGetLastError(), "k_ks_fwd");
}

template <int LOGN>
static int ks_mac_t(he_ctx *c, const u32 *dig, const u32 *rlk32, const u64 *add, int n_out, u64 *out, u32 *park,
                    cudaStream_t st) {
    constexpr int N = Cfg<LOGN>::N;
    constexpr int CH = 4;
    const int np = c->h_ks.np, L = c->L, ell = c->ell;
    const int smem = (N + N / Cfg<LOGN>::R) * 4;
    static std::atomic<unsigned long long> attr_mask{0};
    if (ks_first_on_device(attr_mask))
        cudaFuncSetAttribute(k_ks_mac<LOGN, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const long long blocks = (long long)n_out * L * 2;
    if (blocks > 0x7fffffffLL) return fail(c, HE_ERR_INVALID_ARG, "key-switch launch too large");
    // digits and key read once, addend read and output written once
    const double bytes = 4.0 * N * np * ell * ((double)n_out + 2.0 * L) + 16.0 * N * (double)blocks;
    // 32-bit modular products: terms, butterflies, untwist, Garner
    const double mm = (double)blocks * N * (np * (ell + (LOGN / 2.0) + 1.0) + np * (np - 1) / 2.0);
    TraceScope ts(c, st, "ks_mac", bytes, mm);
    KsMacArgs a;
    a.dig = dig; a.rlk32 = rlk32; a.add = add; a.out = out; a.park = park; a.ell = ell; a.L = L;
    k_ks_mac<LOGN, CH><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(a, c->h_ks, c->d_mods);
    return cuda_check(c, cudaGetLastError(), "k_ks_mac");
}

int launch_ks_fwd(he_ctx *c, const void *src, bool u64_src, int n_polys, uint32_t *dst, cudaStream_t st) {
    if (n_polys <= 0) return HE_OK;
    if (c->h_ks.np < 2) return fail(c, HE_ERR_INVALID_ARG, "no small-prime key switch in this context");
    switch (c->logN) {
    case 10: return ks_fwd_t<10>(c, src, u64_src, n_polys, dst, st);
    case 11: return ks_fwd_t<11>(c, src, u64_src, n_polys, dst, st);
    case 12: return ks_fwd_t<12>(c, src, u64_src, n_polys, dst, st);
    case 13: return ks_fwd_t<13>(c, src, u64_src, n_polys, dst, st);
    case 14: return ks_fwd_t<14>(c, src, u64_src, n_polys, dst, st);
    }
    return fail(c, HE_ERR_UNSUPPORTED_PARAMS, "unsupported N");
}

int launch_ks_mac(he_ctx *c, const uint32_t *dig, const uint32_t *rlk32, const u64 *add, int n_out, u64 *out,
                  uint32_t *park, cudaStream_t st) {
    if (n_out <= 0) return HE_OK;
    if (c->h_ks.np < 2) return fail(c, HE_ERR_INVALID_ARG, "no small-prime key switch in this context");
    switch (c->logN) {
    case 10: return ks_mac_t<10>(c, dig, rlk32, add, n_out, out, park, st);
    case 11: return ks_mac_t<11>(c, dig, rlk32, add, n_out, out, park, st);
    case 12: return ks_mac_t<12>(c, dig, rlk32, add, n_out, out, park, st);
    case 13: return ks_mac_t<13>(c, dig, rlk32, add, n_out, out, park, st);
    case 14: return ks_mac_t<14>(c, dig, rlk32, add, n_out, out, park, st);
    }
    return fail(c, HE_ERR_UNSUPPORTED_PARAMS, "unsupported N");
}

}  // namespace he

HE_CHECKS_UNIT(keyswitch)
