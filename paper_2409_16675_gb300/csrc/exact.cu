// exact.cu -- per-coefficient kernels that need all RNS limbs at once:
// sampling, the exact base extension Q -> Q u B, the exact BFV rescaling
// floor((t d + floor(q/2)) / q) with digit decomposition, exact decryption,
// and the encoding / decoding gathers.
//
// Exactness: a base conversion needs the CRT overflow count v = floor(sum_i
// y_i / m_i) of its value; it is taken from a fixed-point estimate of that
// sum, and wherever the estimate could be off (the sum within 64 ulps of an
// integer, or of one half for a centred lift) the value is instead rebuilt as
// a multi-word integer (sum of y_i * (M/m_i), overflow multiples of M
// subtracted) and reduced directly, so no step is an approximation.  The
// rescaling uses the identity
//   floor((t d + h) / q) = (t d + h - r) / q,  r = [t d + h]_q, h = floor(q/2),
// whose right side is an exact division, evaluated modulo each auxiliary
// prime and brought back to Q by a second exact CRT (the quotient is smaller
// than B/2 by construction of B).
#include "arith.cuh"

namespace he {

// ---------------------------------------------------------------- sampling
// one ChaCha block (8 words) of a sample job: thread gid of the job
__device__ __forceinline__ void sample_block(int kind, uint64_t seed, uint32_t tag, uint32_t idx0, int n_limbs, int N,
                                             void *out, long long gid, const ModDev *__restrict__ mods,
                                             const ExactDev *__restrict__ E, int eta) {
    if (kind == SAMPLE_UNIFORM_Q) {
        // 4 coefficients per ChaCha block (two words each)
        const int per = N / 4;
        const int b = (int)(gid % per);
        const long long ol = gid / per;
        const int limb = (int)(ol % n_limbs);
        const long long obj = ol / n_limbs;
        u64 w[8];
        chacha_block8(seed, tag, idx0 + (uint32_t)obj, (uint32_t)limb, (uint32_t)b, w);
        if (!HE_OBJ_OK(mods + limb)) return;
        const ModDev M = mods[limb];
        u64 *o = (u64 *)out + (obj * n_limbs + limb) * N + 4 * b;
#pragma unroll
        for (int j = 0; j < 4; j++) HE_ST(o + j, reduce128(w[2 * j], w[2 * j + 1], M));
        return;
    }
    const int per = N / 8;
    const int b = (int)(gid % per);
    const long long obj = gid / per;
    u64 w[8];
    chacha_block8(seed, tag, idx0 + (uint32_t)obj, 0u, (uint32_t)b, w);
    if (kind == SAMPLE_UNIFORM_T) {
        if (!HE_OBJ_OK(E)) return;
        u64 *o = (u64 *)out + obj * N + 8 * b;
#pragma unroll
        for (int j = 0; j < 8; j++) HE_ST(o + j, reduce64(w[j], E->t, E->one_ts));
        return;
    }
    int8_t r[8];
    if (kind == SAMPLE_TERNARY) {
#pragma unroll
        for (int j = 0; j < 8; j++) r[j] = (int8_t)((int)__umul64hi(w[j], 3ull) - 1);
    } else {
        const u64 mask = (eta >= 64) ? ~0ull : ((1ull << eta) - 1);
#pragma unroll
        for (int j = 0; j < 8; j++) r[j] = (int8_t)(__popcll(w[j] & mask) - __popcll((w[j] >> eta) & mask));
    }
    int8_t *o = (int8_t *)out + obj * N + 8 * b;
    u64 packed = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) packed |= (u64)(uint8_t)r[j] << (8 * j);
    HE_ST((u64 *)o, packed);
}

__global__ void k_sample(int kind, uint64_t seed, uint32_t tag, uint32_t idx0, int n_limbs, int N, void *out,
                         long long total_blocks, const ModDev *__restrict__ mods, const ExactDev *__restrict__ E,
                         int eta) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid < total_blocks) sample_block(kind, seed, tag, idx0, n_limbs, N, out, gid, mods, E, eta);
}

// Sample jobs of one launch: blocks [start[i], start[i+1]) belong to job i,
// whose threads cover total[i] ChaCha blocks.
struct SampleJobs {
    int n;
    SampleJob j[kMaxSampleJobs];
    long long total[kMaxSampleJobs];
    int start[kMaxSampleJobs + 1];
};

__global__ void k_sample_multi(const __grid_constant__ SampleJobs JS, int N, const ModDev *__restrict__ mods,
                               const ExactDev *__restrict__ E, int eta) {
    int i = 0;
#pragma unroll
    for (int k = 1; k < kMaxSampleJobs; k++)
        if (k < JS.n && (int)blockIdx.x >= JS.start[k]) i = k;
    const long long gid = (long long)((int)blockIdx.x - JS.start[i]) * blockDim.x + threadIdx.x;
    if (gid >= JS.total[i]) return;
    const SampleJob &J = JS.j[i];
    sample_block(J.kind, J.seed, J.tag, J.idx0, J.n_limbs, N, J.out, gid, mods, E, eta);
}

int launch_sample(he_ctx *c, int kind, uint64_t seed, uint32_t tag, uint32_t idx0, int n_obj, int n_limbs,
                  void *out, cudaStream_t st) {
    const int N = c->N;
    long long total = kind == SAMPLE_UNIFORM_Q ? (long long)n_obj * n_limbs * (N / 4) : (long long)n_obj * (N / 8);
    if (!total) return HE_OK;
    TraceScope ts(c, st, "sample", kind == SAMPLE_UNIFORM_Q ? 32.0 * total : (kind == SAMPLE_UNIFORM_T ? 64.0 * total : 8.0 * total), 0);
    k_sample<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(kind, seed, tag, idx0, n_limbs, N, out, total,
                                                               c->d_mods, c->d_exact, c->P.eta);
    return cuda_check(c, cudaGetLastError(), "k_sample");
}

int launch_sample_multi(he_ctx *c, const SampleJob *jobs, int n, cudaStream_t st) {
    if (n < 0 || n > kMaxSampleJobs) return fail(c, HE_ERR_INVALID_ARG, "sample job count");
    const int N = c->N;
    SampleJobs JS;
    memset(&JS, 0, sizeof JS);
    long long blocks = 0;
    double bytes = 0;
    int m = 0;
    for (int i = 0; i < n; i++) {
        const SampleJob &J = jobs[i];
        const long long total = J.kind == SAMPLE_UNIFORM_Q ? (long long)J.n_obj * J.n_limbs * (N / 4)
                                                           : (long long)J.n_obj * (N / 8);
        if (total <= 0) continue;
        JS.j[m] = J;
        JS.total[m] = total;
        JS.start[m] = (int)blocks;
        blocks += (total + 127) / 128;
        bytes += J.kind == SAMPLE_UNIFORM_Q ? 32.0 * total : (J.kind == SAMPLE_UNIFORM_T ? 64.0 * total : 8.0 * total);
        m++;
    }
    if (!m) return HE_OK;
    if (blocks > 0x7fffffffLL) return fail(c, HE_ERR_INVALID_ARG, "sample launch too large");
    JS.n = m;
    JS.start[m] = (int)blocks;
    TraceScope ts(c, st, "sample", bytes, 0);
    k_sample_multi<<<(unsigned)blocks, 128, 0, st>>>(JS, N, c->d_mods, c->d_exact, c->P.eta);
    return cuda_check(c, cudaGetLastError(), "k_sample_multi");
}

// ---------------------------------------------------------------- exact CRT kernels
// Template parameters: LM, KM bound the runtime limb counts L and K (loops are
// unrolled to the bound with guards so every array stays in registers); MW
// bounds the words of a multi-word CRT sum (exact fallback path, digits).

// centred lift of each coefficient (residues mod Q) to the auxiliary primes
template <int LM, int KM, int MW>
__global__ void __launch_bounds__(128) k_base_extend(const u64 *__restrict__ src, long long n_polys, int L, int K,
                                                     int N, u64 *__restrict__ dst, const ModDev *__restrict__ mods,
                                                     const ExactDev *__restrict__ E) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n_polys * N) return;
    if (!HE_OBJ_OK(E) || !HE_SPAN_OK(mods, L + K)) return;
    const int x = (int)(gid % N);
    const long long p = gid / N;
    const CrtDev &Q = E->Q;
    u64 y[LM];
#pragma unroll
    for (int i = 0; i < LM; i++)
        if (i < L) y[i] = crt_y(Q, i, HE_LD(src + (p * L + i) * N + x));
    int v;
    u64 fr;
    if (crt_overflow<LM>(E->Qc, y, L, v, fr) && half_certain(fr)) {
        const u64 k = (u64)v + (fr >= (1ull << 57));
#pragma unroll
        for (int j = 0; j < KM; j++)
            if (j < K) HE_ST(dst + (p * K + j) * N + x, conv_to_m<LM>(y, L, E->QhatBm[j], k, E->Q_b[j], E->Q_bs[j], mods[L + j]));
        return;
    }
    u64 X[MW];
    crt_compose<MW>(Q, y, X);
    const bool neg = mw_greater<MW>(X, Q.Mhalf, Q.W);
    for (int j = 0; j < K; j++) {
        const ModDev &M = mods[L + j];
        u64 a = mw_mod<MW>(X, Q.W, M.q, M.r64, M.r64s, M.one_s);
        if (neg) a = subm(a, E->Q_b[j], M.q);
        HE_ST(dst + (p * K + j) * N + x, a);
    }
}

// d: [n_out][3][L+K][N] exact tensor products (coefficient form).
// dq: [n_out][2][L][N] rescaled d0, d1; digits: [n_out][ell][N] of rescaled d2.
// The smallest size class is held to 64 registers (eight 128-thread CTAs per
// SM, a few bytes spilled): measured faster than 66 registers and seven CTAs.
template <int LM, int KM, int MW>
__global__ void __launch_bounds__(128, (LM <= 4 ? 8 : 1)) k_scale_round(const u64 *__restrict__ d, int n_out, int L, int K, int N,
                                                     int ell, int base_log2, u64 *__restrict__ dq,
                                                     uint32_t *__restrict__ digits, const ModDev *__restrict__ mods,
                                                     const ExactDev *__restrict__ E) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)n_out * 3 * N) return;
    if (!HE_OBJ_OK(E) || !HE_SPAN_OK(mods, L + K)) return;
    const int x = (int)(gid % N);
    const int j = (int)((gid / N) % 3);
    const long long o = gid / (3LL * N);
    const int LK = L + K;
    const u64 *src = d + ((o * 3 + j) * LK) * N + x;
    const CrtDev &Q = E->Q, &B = E->B;
    // r = [t d + floor(q/2)]_q as residues y (CRT form): y_i = d_i (t inv_i)
    // + floor(q/2) inv_i mod q_i
    u64 y[LM];
#pragma unroll
    for (int i = 0; i < LM; i++)
        if (i < L) {
            const u64 qi = mods[i].q;
            y[i] = addm(red1(shoup(HE_LD(src + (long long)i * N), E->f_tq[i], E->f_tqs[i], qi), qi), E->f_hq[i], qi);
        }
    // r c_k mod b_k (c_k = q^-1 (B/b_k)^-1 mod b_k folded into the conversion)
    u64 rc[KM];
    int v;
    u64 fr;
    if (crt_overflow<LM>(E->Qc, y, L, v, fr)) {
#pragma unroll
        for (int k = 0; k < KM; k++)
            if (k < K)
                rc[k] = conv_to_m<LM>(y, L, E->QhatBcm[k], (u64)v, E->Q_bc[k], E->Q_bcs[k], mods[L + k]);
    } else {
        u64 R[MW];
        crt_compose<MW>(Q, y, R);
#pragma unroll
        for (int k = 0; k < KM; k++)
            if (k < K) {
                const ModDev &M = mods[L + k];
                const u64 rb = mw_mod<MW>(R, Q.W, M.q, M.r64, M.r64s, M.one_s);
                rc[k] = red1(shoup(rb, E->f_cb[k], E->f_cbs[k], M.q), M.q);
            }
    }
    // F = (t d + h - r) / q modulo each aux prime, as CRT residues over B:
    // yb_k = (t d + h - r) c_k mod b_k
    u64 yb[KM];
#pragma unroll
    for (int k = 0; k < KM; k++)
        if (k < K) {
            const u64 b = mods[L + k].q;
            const u64 td = red1(shoup(HE_LD(src + (long long)(L + k) * N), E->f_tb[k], E->f_tbs[k], b), b);
            yb[k] = subm(addm(td, E->f_hb[k], b), rc[k], b);
        }
    // centred F mod q_i; for the digit component (j = 2) directly its CRT
    // residue F inv_i mod q_i (the constants carry the inv_i factor)
    const bool dig = j == 2;
    const u64(*H)[MAXP] = dig ? E->BhatQim : E->BhatQm;
    const u64 *Bq = dig ? E->B_qi : E->B_q;
    const u64 *Bqs = dig ? E->B_qis : E->B_qs;
    u64 f[LM];
    if (crt_overflow<KM>(E->Bc, yb, K, v, fr) && half_certain(fr)) {
        const u64 k = (u64)v + (fr >= (1ull << 57));
#pragma unroll
        for (int i = 0; i < LM; i++)
            if (i < L) f[i] = conv_to_m<KM>(yb, K, H[i], k, Bq[i], Bqs[i], mods[i]);
    } else {
        u64 F[MW];
        crt_compose<MW>(B, yb, F);
        const bool neg = mw_greater<MW>(F, B.Mhalf, B.W);
#pragma unroll
        for (int i = 0; i < LM; i++)
            if (i < L) {
                const ModDev &M = mods[i];
                u64 a = mw_mod<MW>(F, B.W, M.q, M.r64, M.r64s, M.one_s);
                if (neg) a = subm(a, E->B_q[i], M.q);
                f[i] = dig ? crt_y(Q, i, a) : a;
            }
    }
    if (!dig) {
        u64 *out = dq + ((o * 2 + j) * L) * N + x;
#pragma unroll
        for (int i = 0; i < LM; i++)
            if (i < L) HE_ST(out + (long long)i * N, f[i]);
        return;
    }
    // digits of [F]_q in [0, q): exact multi-word value
#pragma unroll
    for (int i = 0; i < LM; i++)
        if (i < L) y[i] = f[i];
    u64 X[MW];
    crt_compose<MW>(Q, y, X);
    const u64 dmask = (1ull << base_log2) - 1;
    uint32_t *dg = digits + (o * ell) * N + x;
    if (base_log2 == 16) {  // the paper's base: four whole digits per word, no straddling
#pragma unroll
        for (int k = 0; k < MW; k++)
#pragma unroll
            for (int s4 = 0; s4 < 4; s4++)
                if (4 * k + s4 < ell) HE_ST(dg + (long long)(4 * k + s4) * N, (uint32_t)((X[k] >> (16 * s4)) & 0xffff));
        return;
    }
    for (int dd = 0; dd < ell; dd++) {
        const int bit = dd * base_log2;
        const int w = bit >> 6, sh = bit & 63;
        u64 val = 0;
#pragma unroll
        for (int k = 0; k < MW; k++) {
            if (k == w) val = X[k] >> sh;
            if (k == w + 1 && sh + base_log2 > 64) val |= X[k] << (64 - sh);
        }
        HE_ST(dg + (long long)dd * N, (uint32_t)(val & dmask));
    }
}

// x: [n][L][N] = c0 + c1 s; m = floor((t x + floor(q/2)) / q) mod t
//    = (floor(q/2) - [t x + floor(q/2)]_q) * q^-1 mod t
template <int LM, int KM, int MW>
__global__ void __launch_bounds__(128) k_decrypt_exact(const u64 *__restrict__ xs, int n, int L, int N,
                                                       u64 *__restrict__ m, const ModDev *__restrict__ mods,
                                                       const ExactDev *__restrict__ E) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)n * N) return;
    if (!HE_OBJ_OK(E) || !HE_SPAN_OK(mods, L)) return;
    const int x = (int)(gid % N);
    const long long k = gid / N;
    const CrtDev &Q = E->Q;
    u64 y[LM];
#pragma unroll
    for (int i = 0; i < LM; i++)
        if (i < L) {
            const u64 qi = mods[i].q;
            y[i] = addm(red1(shoup(HE_LD(xs + (k * L + i) * N + x), E->f_tq[i], E->f_tqs[i], qi), qi), E->f_hq[i], qi);
        }
    const u64 t = E->t;
    u64 rt;
    int v;
    u64 fr;
    if (crt_overflow<LM>(E->Qc, y, L, v, fr)) {
        rt = conv_to<LM>(y, L, E->Qhat_t, E->Qhat_ts, (u64)v, E->Q_t, E->Q_ts, t);
    } else {
        u64 R[MW];
        crt_compose<MW>(Q, y, R);
        rt = mw_mod<MW>(R, Q.W, t, E->r64_t, E->r64_ts, E->one_ts);
    }
    HE_ST(m + k * N + x, red1(shoup(subm(E->Qhalf_t, rt, t), E->Qinv_t, E->Qinv_ts, t), t));
}

// kernel size class of a context: limb bounds and multi-word capacity
static int size_class(he_ctx *c) {
    const int W = c->h_exact.Q.W > c->h_exact.B.W ? c->h_exact.Q.W : c->h_exact.B.W;
    if (c->L <= 4 && c->K <= 4 && W <= 6) return 0;
    if (c->L <= 8 && c->K <= 8 && W <= 10) return 1;
    return 2;
}

#define HE_DISPATCH_EXACT(KER, ...)                                                   \
    switch (size_class(c)) {                                                           \
    case 0: KER<4, 4, 6><<<g, 128, 0, st>>>(__VA_ARGS__); break;                      \
    case 1: KER<8, 8, 10><<<g, 128, 0, st>>>(__VA_ARGS__); break;                     \
    default: KER<16, 24, 18><<<g, 128, 0, st>>>(__VA_ARGS__); break;                  \
    }

int launch_base_extend(he_ctx *c, const u64 *src, long long n_polys, u64 *dst_aux, cudaStream_t st) {
    const long long total = n_polys * c->N;
    if (!total) return HE_OK;
    const unsigned g = (unsigned)((total + 127) / 128);
    TraceScope ts(c, st, "base_extend", 8.0 * total * (c->L + c->K), 0);
    HE_DISPATCH_EXACT(k_base_extend, src, n_polys, c->L, c->K, c->N, dst_aux, c->d_mods, c->d_exact)
    return cuda_check(c, cudaGetLastError(), "k_base_extend");
}

int launch_scale_round(he_ctx *c, const u64 *d, int n_out, u64 *dq, uint32_t *digits, cudaStream_t st) {
    const long long total = (long long)n_out * 3 * c->N;
    if (!total) return HE_OK;
    const unsigned g = (unsigned)((total + 127) / 128);
    const int b = c->P.base_log2;
    TraceScope ts(c, st, "scale_round", 8.0 * total * (c->L + c->K) + 8.0 * n_out * 2 * c->L * c->N +
                  4.0 * n_out * c->ell * c->N, 0);
    HE_DISPATCH_EXACT(k_scale_round, d, n_out, c->L, c->K, c->N, c->ell, b, dq, digits, c->d_mods, c->d_exact)
    return cuda_check(c, cudaGetLastError(), "k_scale_round");
}

int launch_decrypt_exact(he_ctx *c, const u64 *x, int n, u64 *m, cudaStream_t st) {
    const long long total = (long long)n * c->N;
    if (!total) return HE_OK;
    const unsigned g = (unsigned)((total + 127) / 128);
    TraceScope ts(c, st, "decrypt_exact", 8.0 * total * (c->L + 1), 0);
    HE_DISPATCH_EXACT(k_decrypt_exact, x, n, c->L, c->N, m, c->d_mods, c->d_exact)
    return cuda_check(c, cudaGetLastError(), "k_decrypt_exact");
}

// ---------------------------------------------------------------- encode / decode
__device__ __forceinline__ u64 to_t(const void *tensor, int dtype, long long i, u64 t) {
    long long v;
    if (dtype == HE_DTYPE_U8) v = HE_LD((const uint8_t *)tensor + i);
    else if (dtype == HE_DTYPE_I8) v = HE_LD((const int8_t *)tensor + i);
    else v = HE_LD((const long long *)tensor + i);
    if (v >= 0) return (u64)v % t;
    const u64 r = (u64)(-(v + 1)) % t;  // -(v+1) >= 0, no overflow
    return t - 1 - r;
}

// input role: out[(b*out_batch_polys + p)*N + x] = x_b[map[p*N + x]] mod t
__global__ void k_encode_input(const int32_t *__restrict__ map, int n_polys, int N, const void *tensor, int dtype,
                               long long tensor_stride, int batch, long long out_batch_polys, u64 *__restrict__ out,
                               u64 t) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per = (long long)n_polys * N;
    if (gid >= per * batch) return;
    const long long b = gid / per;
    const long long r = gid - b * per;
    const int idx = HE_LD(map + r);
    HE_ST(out + b * out_batch_polys * N + r, idx >= 0 ? to_t(tensor, dtype, b * tensor_stride + idx, t) : 0);
}

// kernel role: out[(mg*G + g)*N + x] = w[map[(mg*G + g)*N + x]] mod t (absolute index into w)
__global__ void k_encode_kernel(const int32_t *__restrict__ map, int G, int M, int N, const void *tensor, int dtype,
                                long long per_m, u64 *__restrict__ out, u64 t) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)G * N * M) return;
    (void)per_m;
    const int idx = HE_LD(map + gid);
    HE_ST(out + gid, idx >= 0 ? to_t(tensor, dtype, idx, t) : 0);
}

// out[(b*M + m)*HW + i] = centred((pt - sub)[b*polys*N + map[m*HW + i]] mod t),
// polys = MG*T product polynomials per image
__global__ void k_decode(const int32_t *__restrict__ map, int HW, int M, int polys, int N, int batch,
                         const u64 *__restrict__ pt, const u64 *__restrict__ sub, long long *__restrict__ out, u64 t) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)batch * M * HW) return;
    const long long mi = gid % ((long long)M * HW);
    const long long b = gid / ((long long)M * HW);
    const long long src = b * polys * N + HE_LD(map + mi);
    u64 v = HE_LD(pt + src);
    v = v >= t ? v % t : v;
    if (sub) {
        u64 s = HE_LD(sub + src);
        s = s >= t ? s % t : s;
        v = v >= s ? v - s : v + t - s;
    }
    HE_ST(out + gid, v > (t - 1) / 2 ? (long long)v - (long long)t : (long long)v);
}

// inverse of k_decode: out[b*polys*N + map[m*HW + i]] = values[(b*M + m)*HW + i] mod t
// (out zeroed by the caller; every (m, i) owns a distinct coefficient)
__global__ void k_encode_output(const int32_t *__restrict__ map, int HW, int M, int polys, int N, int batch,
                                const long long *__restrict__ values, u64 *__restrict__ out, u64 t) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)batch * M * HW) return;
    const long long mi = gid % ((long long)M * HW);
    const long long b = gid / ((long long)M * HW);
    const long long v = HE_LD(values + gid);
    HE_ST(out + b * polys * N + HE_LD(map + mi), v >= 0 ? (u64)v % t : t - 1 - (u64)(-(v + 1)) % t);
}

// ciphertext addition (CCAdd): out = a + b mod q_limb over n polynomials of L limbs
__global__ void k_ct_add(const u64 *__restrict__ a, const u64 *__restrict__ b, long long total, int N, int L,
                         u64 *__restrict__ out, const ModDev *__restrict__ mods) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    if (!HE_SPAN_OK(mods, L)) return;
    const u64 q = mods[(gid / N) % L].q;
    HE_ST(out + gid, addm(HE_LD(a + gid), HE_LD(b + gid), q));
}

__global__ void k_pt_sub(const u64 *__restrict__ a, const u64 *__restrict__ b, long long n, u64 *__restrict__ out,
                         u64 t) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n) return;
    u64 x = HE_LD(a + gid), y = HE_LD(b + gid);
    x = x >= t ? x % t : x;
    y = y >= t ? y % t : y;
    HE_ST(out + gid, x >= y ? x - y : x + t - y);
}

__global__ void k_copy_sk(const int8_t *__restrict__ s8, long long *__restrict__ sk, int N) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid < N) HE_ST(sk + gid, (long long)HE_LD(s8 + gid));
}

int launch_encode(he_ctx *c, const int32_t *map, int n_polys, int map_polys, const void *tensor, int dtype,
                  long long tensor_stride, int batch, long long out_batch_polys, u64 *out, cudaStream_t st) {
    (void)map_polys;
    const long long total = (long long)n_polys * c->N * batch;
    if (!total) return HE_OK;
    k_encode_input<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(map, n_polys, c->N, tensor, dtype, tensor_stride,
                                                                     batch, out_batch_polys, out, c->P.t);
    return cuda_check(c, cudaGetLastError(), "k_encode_input");
}

int launch_encode_kernel(he_ctx *c, const int32_t *map, int G, int M, const void *tensor, int dtype, long long per_m,
                         u64 *out, cudaStream_t st) {
    const long long total = (long long)G * M * c->N;
    if (!total) return HE_OK;
    k_encode_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(map, G, M, c->N, tensor, dtype, per_m, out,
                                                                      c->P.t);
    return cuda_check(c, cudaGetLastError(), "k_encode_kernel");
}

int launch_decode(he_ctx *c, const int32_t *map, int HW, int M, int polys, int batch, const u64 *pt, const u64 *sub,
                  int64_t *out, cudaStream_t st) {
    const long long total = (long long)batch * M * HW;
    if (!total) return HE_OK;
    k_decode<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(map, HW, M, polys, c->N, batch, pt, sub,
                                                               (long long *)out, c->P.t);
    return cuda_check(c, cudaGetLastError(), "k_decode");
}

int launch_encode_output(he_ctx *c, const int32_t *map, int HW, int M, int polys, int batch, const int64_t *values,
                         u64 *out, cudaStream_t st) {
    const long long total = (long long)batch * M * HW;
    const int rc = cuda_check(c, cudaMemsetAsync(out, 0, (size_t)batch * polys * c->N * 8, st), "output encode clear");
    if (rc || !total) return rc;
    k_encode_output<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(map, HW, M, polys, c->N, batch,
                                                                      (const long long *)values, out, c->P.t);
    return cuda_check(c, cudaGetLastError(), "k_encode_output");
}

int launch_ct_add(he_ctx *c, const u64 *a, const u64 *b, long long n_polys, u64 *out, cudaStream_t st) {
    const long long total = n_polys * c->L * c->N;
    if (!total) return HE_OK;
    k_ct_add<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a, b, total, c->N, c->L, out, c->d_mods);
    return cuda_check(c, cudaGetLastError(), "k_ct_add");
}

int launch_pt_sub(he_ctx *c, const u64 *a, const u64 *b, long long n, u64 *out, cudaStream_t st) {
    if (!n) return HE_OK;
    k_pt_sub<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n, out, c->P.t);
    return cuda_check(c, cudaGetLastError(), "k_pt_sub");
}

// import checks: a ternary secret key (as int8 for the forward transform) and
// residues below their limb modulus; a violation sets *bad (never traps)
__global__ void k_import_sk(const long long *__restrict__ sk, int N, int8_t *__restrict__ s8, int *bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const long long v = HE_LD(sk + i);
    if ((v < -1 || v > 1) && HE_OBJ_OK(bad)) atomicOr(bad, 1);
    HE_ST(s8 + i, (int8_t)(v < -1 ? -1 : (v > 1 ? 1 : v)));
}
__global__ void k_check_residues(const u64 *__restrict__ a, long long total, int N, int L,
                                 const ModDev *__restrict__ mods, int *bad) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    if (!HE_SPAN_OK(mods, L) || !HE_OBJ_OK(bad)) return;
    if (HE_LD(a + gid) >= mods[(gid / N) % L].q) atomicOr(bad, 2);
}

int launch_import_sk(he_ctx *c, const int64_t *sk, int8_t *s8, int *bad, cudaStream_t st) {
    k_import_sk<<<(c->N + 255) / 256, 256, 0, st>>>((const long long *)sk, c->N, s8, bad);
    return cuda_check(c, cudaGetLastError(), "k_import_sk");
}
int launch_check_residues(he_ctx *c, const u64 *a, long long n_polys, int *bad, cudaStream_t st) {
    const long long total = n_polys * c->L * c->N;
    if (!total) return HE_OK;
    k_check_residues<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a, total, c->N, c->L, c->d_mods, bad);
    return cuda_check(c, cudaGetLastError(), "k_check_residues");
}

int launch_copy_sk(he_ctx *c, const int8_t *s8, u64 *sk, cudaStream_t st) {
    k_copy_sk<<<(c->N + 255) / 256, 256, 0, st>>>(s8, (long long *)sk, c->N);
    return cuda_check(c, cudaGetLastError(), "k_copy_sk");
}

}  // namespace he

HE_CHECKS_UNIT(exact)
