// ntt.cu -- negacyclic NTT kernels over RNS limbs.
//
// The product in A_{N,q} = Z_q[x]/(x^N+1) (Section 2, Notations) is computed
// as NTT -> pointwise multiply-accumulate -> inverse NTT.  One CTA owns one
// limb polynomial; each of its N/16 threads keeps 16 coefficients in
// registers and runs up to four butterfly stages (radix 16) between exchanges
// through padded shared memory.  The forward transform is Cooley-Tukey with
// the psi twist merged into the twiddles (bit-reversed output), the inverse is
// Gentleman-Sande; butterflies use Harvey's lazy reduction (values in [0,4q)
// forward, [0,2q) inverse) with Shoup products.
//
// NTT-domain storage order ("perm16"): memory position k*(N/16) + tau holds
// the bit-reversed-order value of index 16*tau + k, which is exactly what the
// last forward pass and the first inverse pass hold in registers, so both the
// forward store and the multiply-accumulate loads are coalesced.  This order
// never leaves the library.
#include "arith.cuh"

namespace he {

template <int LOGN>
struct Cfg {
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / 16;
    static constexpr int NP = (LOGN + 3) / 4;
    static constexpr int RL = LOGN - 4 * (NP - 1);
    static constexpr int SMEM = (N + N / 16) * 8;
};

__device__ __forceinline__ int padi(int j) { return j + (j >> 4); }
// element index of register k of thread tau when the 4-bit register window
// starts at bit lo
__device__ __forceinline__ int jidx(int tau, int k, int lo) {
    return ((tau >> lo) << (lo + 4)) | (k << lo) | (tau & ((1 << lo) - 1));
}

template <int LOGN, int R>
__device__ __forceinline__ void fwd_pass(u64 (&v)[16], int tau, int lo, int s0, const ModDev &M) {
    const u64 q = M.q, q2 = M.twoq;
#pragma unroll
    for (int st = 0; st < R; st++) {
        const int kb = R - 1 - st;
        const int s = s0 + st;
        const int base = (1 << s) + ((tau >> lo) << (3 - kb));
#pragma unroll
        for (int k = 0; k < 16; k++) {
            if (k & (1 << kb)) continue;
            const int widx = base + (k >> (kb + 1));
            const u64 W = __ldg(M.fw + widx), Ws = __ldg(M.fws + widx);
            u64 X = v[k];
            const u64 Y = v[k | (1 << kb)];
            X = X >= q2 ? X - q2 : X;
            const u64 Tt = shoup(Y, W, Ws, q);
            v[k] = X + Tt;
            v[k | (1 << kb)] = X - Tt + q2;
        }
    }
}

template <int LOGN, int R>
__device__ __forceinline__ void inv_pass(u64 (&v)[16], int tau, int lo, int s_top, const ModDev &M) {
    const u64 q = M.q, q2 = M.twoq;
#pragma unroll
    for (int st = 0; st < R; st++) {
        const int kb = st;
        const int s = s_top - st;
        const int base = (1 << s) + ((tau >> lo) << (3 - kb));
#pragma unroll
        for (int k = 0; k < 16; k++) {
            if (k & (1 << kb)) continue;
            const int widx = base + (k >> (kb + 1));
            const u64 W = __ldg(M.iw + widx), Ws = __ldg(M.iws + widx);
            const u64 X = v[k], Y = v[k | (1 << kb)];
            u64 S = X + Y;
            S = S >= q2 ? S - q2 : S;
            v[k] = S;
            v[k | (1 << kb)] = shoup(X - Y + q2, W, Ws, q);
        }
    }
}

__device__ __forceinline__ void exchange(u64 *sm, u64 (&v)[16], int tau, int lo_from, int lo_to) {
#pragma unroll
    for (int k = 0; k < 16; k++) sm[padi(jidx(tau, k, lo_from))] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = sm[padi(jidx(tau, k, lo_to))];
    __syncthreads();
}

template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T) k_fwd(FwdJob J, const ModDev *__restrict__ mods) {
    extern __shared__ u64 sm[];
    constexpr int N = Cfg<LOGN>::N, T = Cfg<LOGN>::T, NP = Cfg<LOGN>::NP, RL = Cfg<LOGN>::RL;
    const int tau = threadIdx.x;
    const int limb = blockIdx.x / J.n_polys;
    const int p = blockIdx.x - limb * J.n_polys;
    const ModDev M = mods[J.mod_base + limb];
    u64 v[16];
    // first window: bits [LOGN-4, LOGN): element j = k*T + tau (coalesced)
    switch (J.kind) {
    case SRC_RNS: {
        const u64 *s = limb < J.split
            ? (const u64 *)J.src + (long long)p * J.src_stride + (long long)limb * N
            : (const u64 *)J.src2 + (long long)p * J.src2_stride + (long long)(limb - J.split) * N;
#pragma unroll
        for (int k = 0; k < 16; k++) v[k] = s[k * T + tau];
        break;
    }
    case SRC_T_LIFT: {
        const u64 *s = (const u64 *)J.src + (long long)p * J.src_stride;
        const u64 t = J.t, half = (J.t - 1) / 2;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            u64 x = s[k * T + tau];
            x = x >= t ? x % t : x;
            v[k] = x <= half ? x : M.q - (t - x);
        }
        break;
    }
    case SRC_I8: {
        const int8_t *s = (const int8_t *)J.src + (long long)p * J.src_stride;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const int x = s[k * T + tau];
            v[k] = x >= 0 ? (u64)x : M.q - (u64)(-x);
        }
        break;
    }
    case SRC_U32: {
        const uint32_t *s = (const uint32_t *)J.src + (long long)p * J.src_stride;
#pragma unroll
        for (int k = 0; k < 16; k++) v[k] = s[k * T + tau];
        break;
    }
    default: {  // SRC_T_RAW
        const u64 *s = (const u64 *)J.src + (long long)p * J.src_stride;
#pragma unroll
        for (int k = 0; k < 16; k++) v[k] = reduce64(s[k * T + tau], M.q, M.one_s);
        break;
    }
    }
    int lo = LOGN - 4;
    for (int pass = 0; pass < NP - 1; pass++) {
        fwd_pass<LOGN, 4>(v, tau, lo, 4 * pass, M);
        const int lo_next = pass == NP - 2 ? 0 : lo - 4;
        exchange(sm, v, tau, lo, lo_next);
        lo = lo_next;
    }
    fwd_pass<LOGN, RL>(v, tau, 0, 4 * (NP - 1), M);
    u64 *d = J.dst + (long long)p * J.dst_stride + (long long)limb * N;
    const u64 q = M.q, q2 = M.twoq;
#pragma unroll
    for (int k = 0; k < 16; k++) {
        u64 x = v[k];
        x = x >= q2 ? x - q2 : x;
        d[k * T + tau] = red1(x, q);
    }
}

template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T) k_mac_intt(MacJob J, const ModDev *__restrict__ mods) {
    extern __shared__ u64 sm[];
    constexpr int N = Cfg<LOGN>::N, T = Cfg<LOGN>::T, NP = Cfg<LOGN>::NP, RL = Cfg<LOGN>::RL;
    const int tau = threadIdx.x;
    const int limb = blockIdx.x / J.n_out;
    const int o = blockIdx.x - limb * J.n_out;
    const ModDev M = mods[J.mod_base + limb];
    u64 v[16];
    {
        u64 lo[16], hi[16];
#pragma unroll
        for (int k = 0; k < 16; k++) { lo[k] = 0; hi[k] = 0; }
        const int t0 = J.ptr[o], t1 = J.ptr[o + 1];
        int cnt = 0;
        for (int tk = t0; tk < t1; tk++) {
            const u64 *a = J.A + ((long long)J.ta[tk] + limb) * N;
            const u64 *b = J.B + ((long long)J.tb[tk] + limb) * N;
#pragma unroll
            for (int k = 0; k < 16; k++) {
                u64 pl, ph;
                mul128(a[k * T + tau], b[k * T + tau], pl, ph);
                lo[k] += pl;
                hi[k] += ph + (lo[k] < pl);
            }
            if (++cnt == 15) {  // products < 2^124: fold before the 128-bit sum can overflow
#pragma unroll
                for (int k = 0; k < 16; k++) { lo[k] = reduce128(lo[k], hi[k], M); hi[k] = 0; }
                cnt = 0;
            }
        }
#pragma unroll
        for (int k = 0; k < 16; k++) v[k] = reduce128(lo[k], hi[k], M);
    }
    inv_pass<LOGN, RL>(v, tau, 0, LOGN - 1, M);
    int lo = 0;
    for (int pass = NP - 2; pass >= 0; pass--) {
        const int lo_next = LOGN - 4 * (pass + 1);
        exchange(sm, v, tau, lo, lo_next);
        lo = lo_next;
        inv_pass<LOGN, 4>(v, tau, lo, 4 * pass + 3, M);
    }
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
    for (int k = 0; k < 16; k++) {
        const int x = k * T + tau;
        u64 r = red1(shoup(v[k], M.ninv, M.ninvs, q), q);
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

template <int LOGN>
static int fwd_t(he_ctx *c, const FwdJob &j, cudaStream_t st) {
    const int smem = Cfg<LOGN>::SMEM;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_fwd<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr_set = true;
    }
    const long long blocks = (long long)j.n_polys * j.n_limbs;
    if (blocks == 0) return HE_OK;
    const int N = Cfg<LOGN>::N;
    const double src_bytes = j.kind == SRC_RNS ? 8.0 * j.n_limbs : (j.kind == SRC_I8 ? 1.0 : (j.kind == SRC_U32 ? 4.0 : 8.0));
    TraceScope ts(c, st, "ntt_fwd", (double)j.n_polys * N * (src_bytes + 8.0 * j.n_limbs),
                  (double)blocks * (N / 2) * LOGN);
    k_fwd<LOGN><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(j, c->d_mods);
    return cuda_check(c, cudaGetLastError(), "k_fwd");
}

template <int LOGN>
static int mac_t(he_ctx *c, const MacJob &j, cudaStream_t st) {
    const int smem = Cfg<LOGN>::SMEM;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_mac_intt<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr_set = true;
    }
    const long long blocks = (long long)j.n_out * j.n_limbs;
    if (blocks == 0) return HE_OK;
    const int N = Cfg<LOGN>::N;
    const double lb = 8.0 * N * j.n_limbs;  // one polynomial over all limbs
    double bytes = lb * (j.n_out + j.n_dist_a + j.n_dist_b + (j.add ? j.n_out : 0));
    double mm = (double)blocks * ((N / 2) * LOGN + 3.0 * N) + (double)j.n_terms * N * j.n_limbs;
    TraceScope ts(c, st, "mac_intt", bytes, mm);
    k_mac_intt<LOGN><<<(unsigned)blocks, Cfg<LOGN>::T, smem, st>>>(j, c->d_mods);
    return cuda_check(c, cudaGetLastError(), "k_mac_intt");
}

int launch_fwd(he_ctx *c, const FwdJob &j, cudaStream_t st) {
    switch (c->logN) {
    case 10: return fwd_t<10>(c, j, st);
    case 11: return fwd_t<11>(c, j, st);
    case 12: return fwd_t<12>(c, j, st);
    case 13: return fwd_t<13>(c, j, st);
    case 14: return fwd_t<14>(c, j, st);
    }
    return fail(c, HE_ERR_UNSUPPORTED_PARAMS, "unsupported N");
}

int launch_mac_intt(he_ctx *c, const MacJob &j, cudaStream_t st) {
    switch (c->logN) {
    case 10: return mac_t<10>(c, j, st);
    case 11: return mac_t<11>(c, j, st);
    case 12: return mac_t<12>(c, j, st);
    case 13: return mac_t<13>(c, j, st);
    case 14: return mac_t<14>(c, j, st);
    }
    return fail(c, HE_ERR_UNSUPPORTED_PARAMS, "unsupported N");
}

}  // namespace he
