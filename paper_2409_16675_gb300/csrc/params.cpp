// params.cpp -- host-side parameter generation for a context: limb primes,
// auxiliary primes of the tensor-product basis, NTT twiddle tables, and the
// CRT / rescaling constants used by the exact kernels.  Runs once per
// he_setup; everything it computes is uploaded to the device.
#include <cstring>
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace he {

typedef unsigned __int128 u128;

static u64 mulmod(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }
static u64 powmod(u64 a, u64 e, u64 m) {
    u64 r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod(r, a, m);
        a = mulmod(a, a, m);
        e >>= 1;
    }
    return r;
}
// modular inverse by the extended Euclidean algorithm; 0 if none
static u64 invmod(u64 a, u64 m) {
    __int128 t = 0, nt = 1, r = m, nr = a % m;
    while (nr) {
        __int128 qq = r / nr, tmp;
        tmp = t - qq * nt; t = nt; nt = tmp;
        tmp = r - qq * nr; r = nr; nr = tmp;
    }
    if (r != 1) return 0;
    if (t < 0) t += m;
    return (u64)t;
}
// strong probable-prime test to the first 12 prime bases: deterministic for
// all 64-bit inputs
static bool is_prime(u64 n) {
    if (n < 2) return false;
    static const u64 small[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : small) {
        if (n % p == 0) return n == p;
    }
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) { d >>= 1; s++; }
    for (u64 a : small) {
        u64 x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int r = 1; r < s && witness; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}
static u64 shoup_c(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

// ---------------------------------------------------------------- multi-word
struct Big {
    std::vector<u64> w;  // little endian
    static Big of(u64 v) { Big b; b.w.push_back(v); return b; }
    void trim() { while (w.size() > 1 && w.back() == 0) w.pop_back(); }
    Big mul(u64 m) const {
        Big r;
        u64 carry = 0;
        for (u64 x : w) {
            u128 p = (u128)x * m + carry;
            r.w.push_back((u64)p);
            carry = (u64)(p >> 64);
        }
        r.w.push_back(carry);
        r.trim();
        return r;
    }
    // quotient by a single word, remainder in *rem
    Big div(u64 d, u64 *rem) const {
        Big r;
        r.w.assign(w.size(), 0);
        u128 cur = 0;
        for (size_t i = w.size(); i-- > 0;) {
            cur = (cur << 64) | w[i];
            r.w[i] = (u64)(cur / d);
            cur %= d;
        }
        if (rem) *rem = (u64)cur;
        r.trim();
        return r;
    }
    u64 mod(u64 d) const { u64 r; div(d, &r); return r; }
    Big shr1() const {
        Big r = *this;
        for (size_t i = 0; i < r.w.size(); i++) {
            r.w[i] >>= 1;
            if (i + 1 < r.w.size()) r.w[i] |= r.w[i + 1] << 63;
        }
        r.trim();
        return r;
    }
    int bits() const {
        for (size_t i = w.size(); i-- > 0;)
            if (w[i]) return (int)(64 * i) + 64 - __builtin_clzll(w[i]);
        return 0;
    }
};

static Big product(const std::vector<u64> &m) {
    Big b = Big::of(1);
    for (u64 x : m) b = b.mul(x);
    return b;
}

static bool fill_crt(CrtDev &C, const std::vector<u64> &m, std::string &err) {
    if ((int)m.size() > MAXP) { err = "too many primes in one CRT basis"; return false; }
    memset(&C, 0, sizeof C);
    C.n = (int)m.size();
    Big M = product(m);
    int nb = 0;
    while ((1 << nb) < C.n) nb++;
    C.W = (M.bits() + nb + 63) / 64;
    if (C.W < 1) C.W = 1;
    if (C.W > MAXW) { err = "modulus too large"; return false; }
    for (int i = 0; i < C.n; i++) {
        C.m[i] = m[i];
        u64 r;
        Big hat = M.div(m[i], &r);
        for (size_t k = 0; k < hat.w.size() && (int)k < MAXW; k++) C.hat[i][k] = hat.w[k];
        C.Wh = std::max(C.Wh, std::min((int)hat.w.size(), C.W));
        C.inv[i] = invmod(hat.mod(m[i]), m[i]);
        C.invs[i] = shoup_c(C.inv[i], m[i]);
    }
    for (size_t k = 0; k < M.w.size() && (int)k < MAXW; k++) C.M[k] = M.w[k];
    Big h = M.shr1();
    for (size_t k = 0; k < h.w.size() && (int)k < MAXW; k++) C.Mhalf[k] = h.w[k];
    return true;
}

static int bitrev(int x, int n) {
    int r = 0;
    for (int i = 0; i < n; i++) r |= ((x >> i) & 1) << (n - 1 - i);
    return r;
}

// a primitive 2N-th root of unity mod q (q prime, q = 1 mod 2N)
static u64 root_2n(u64 q, int N) {
    for (u64 g = 2; g < 1000000; g++) {
        u64 psi = powmod(g, (q - 1) / (2 * (u64)N), q);
        if (powmod(psi, (u64)N, q) == q - 1) return psi;
    }
    return 0;
}

static bool add_modulus(he_ctx *c, u64 q, std::string &err) {
    const int N = c->N, logN = c->logN;
    u64 psi = root_2n(q, N);
    if (!psi) { err = "no primitive 2N-th root"; return false; }
    u64 psiinv = invmod(psi, q);
    const u64 ninv = invmod((u64)N, q);
    const u64 r64 = (u64)(((u128)1 << 64) % q);
    // interleaved (value, Shoup companion) pairs: fw [N], iw [N], z [N]; the
    // untwist z_k = psi^-k N^-1 2^64 also undoes the 2^-64 of the Montgomery
    // reduction that ends the multiply-accumulate
    std::vector<u64> tab(6 * (size_t)N, 0);
    u64 *fw = tab.data(), *iw = fw + 2 * N, *zt = iw + 2 * N;
    // powers psi^e and psi^-e for e in [0, 2N)
    std::vector<u64> pw(2 * N), ipw(2 * N);
    pw[0] = ipw[0] = 1;
    for (int e = 1; e < 2 * N; e++) { pw[e] = mulmod(pw[e - 1], psi, q); ipw[e] = mulmod(ipw[e - 1], psiinv, q); }
    for (int k = 0; k < N; k++) {
        zt[2 * k] = mulmod(mulmod(ipw[k], ninv, q), r64, q);
        zt[2 * k + 1] = shoup_c(zt[2 * k], q);
    }
    // forward factors psi^bitrev(2^s + i), each stage's groups permuted to the
    // order its register pass reads them: passes of RB stages from the top
    // bit down, the last pass holding the remaining RL stages; in a pass, the
    // stage at position st acts on register bit kb = S - 1 - st and its group
    // index is i = h 2^gb + g with g the gb = RB - 1 - kb register bits above
    // kb and h = the thread's bits above the register window
    {
        const int RB = kNttTileBits, NP = (logN + RB - 1) / RB, RL = logN - RB * (NP - 1);
        for (int pass = 0; pass < NP; pass++) {
            const int S = pass == NP - 1 ? RL : RB;
            for (int st = 0; st < S; st++) {
                const int s = RB * pass + st, gb = RB - 1 - (S - 1 - st);
                for (int i = 0; i < (1 << s); i++) {
                    const int g = i & ((1 << gb) - 1), h = i >> gb;
                    const size_t pos = (size_t)(1 << s) + ((size_t)g << (s - gb)) + h;
                    fw[2 * pos] = pw[bitrev((1 << s) + i, logN)];
                    fw[2 * pos + 1] = shoup_c(fw[2 * pos], q);
                }
            }
        }
    }
    // inverse stage s: omega^-(k 2^(n-1-s)) = psi^-(k 2^(n-s)) for k < 2^s
    for (int s = 0; s < logN; s++)
        for (int k = 0; k < (1 << s); k++) {
            const u64 e = ((u64)k << (logN - s)) % (2 * (u64)N);
            const size_t i = (size_t)(1 << s) + k;
            iw[2 * i] = ipw[e];
            iw[2 * i + 1] = shoup_c(iw[2 * i], q);
        }
    void *d = nullptr;
    if (he::dev_alloc((void **)&d, tab.size() * 8) != cudaSuccess) { err = "cudaMalloc twiddles"; return false; }
    c->allocs.push_back(d);
    if (cudaMemcpy(d, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) { err = "upload twiddles"; return false; }
    ModDev M;
    memset(&M, 0, sizeof M);
    M.q = q;
    M.twoq = 2 * q;
    M.r64 = (u64)(((u128)1 << 64) % q);
    M.r64s = shoup_c(M.r64, q);
    M.one_s = (u64)(((u128)1 << 64) / q);
    M.ninv = ninv;
    M.ninvs = shoup_c(M.ninv, q);
    M.fw = (const ulonglong2 *)d;
    M.iw = M.fw + N;
    M.z = M.iw + N;
    M.nq = 0 - q;
    {
        u64 x = q;  // q^-1 mod 2^64 by Newton's iteration (3, 6, ..., 96 correct bits)
        for (int it = 0; it < 5; it++) x *= 2 - q * x;
        M.qinv = x;
        const u64 f = ~0ull / q + 1;
        M.fold = (int)(f < 15 ? f : 15);
    }
    {
        int bq = 0;
        while (bq < 64 && (q >> bq)) bq++;
        M.qsh = bq + 6 > 32 ? bq + 6 - 32 : 0;
        const double d = std::ldexp(1.0, M.qsh) / (double)q;
        float f = (float)d;
        while ((double)f > d * (1.0 - 1e-12)) f = std::nextafter(f, 0.0f);  // round down, with margin
        M.qf = f;
    }
    c->h_mods.push_back(M);
    return true;
}

// largest unused prime below 2^bits with p = 1 mod 2N
static u64 next_prime_below(int bits, int N, const std::vector<u64> &used) {
    const u64 step = 2 * (u64)N;
    u64 p = (((u64)1 << bits) - 2) / step * step + 1;
    for (; p > step; p -= step) {
        if (std::find(used.begin(), used.end(), p) != used.end()) continue;
        if (is_prime(p)) return p;
    }
    return 0;
}

// Limb primes of a parameter set: the explicit q[] (checked), or for each
// prime_bits[i] the largest unused prime below 2^bits with q = 1 mod 2N.
static int limb_primes(const he_params &P, int N, std::vector<u64> &out, std::string &err) {
    out.clear();
    const bool explicit_q = P.q[0] != 0;
    for (int i = 0; i < P.L; i++) {
        u64 q = explicit_q ? P.q[i] : 0;
        if (explicit_q) {
            if (!is_prime(q) || q % (2 * (u64)N) != 1 || q >= ((u64)1 << 61) ||
                std::find(out.begin(), out.end(), q) != out.end()) {
                err = "explicit q must be distinct primes < 2^61 with q = 1 mod 2N";
                return HE_ERR_UNSUPPORTED_PARAMS;
            }
        } else {
            if (P.prime_bits[i] < 20 || P.prime_bits[i] > 61) { err = "prime_bits out of [20, 61]"; return HE_ERR_UNSUPPORTED_PARAMS; }
            q = next_prime_below(P.prime_bits[i], N, out);
            if (!q) { err = "no prime of that size"; return HE_ERR_UNSUPPORTED_PARAMS; }
        }
        out.push_back(q);
    }
    return HE_OK;
}

// The small primes of the relinearisation key switch for limbs q, plaintext
// modulus t, degree N and ell digits of base_log2 bits: the largest primes
// below 2^30 with p = 1 mod 2N (none of them a limb or t), as many as make
// P = prod p_k exceed 4 ell N (2^base - 1)(max q_i - 1), the bound on four
// times any |E_i|.  Empty (the key switch runs over the limbs) when that
// takes more than kKsMaxPrimes or when a limb is below 2^31 (the CRT adds the
// residues y_k < 2^30 mod q_i).
static std::vector<u64> ks_select(const std::vector<u64> &q, u64 t, int N, int ell, int base_log2) {
    u64 qmax = 0;
    for (u64 qi : q) {
        if (qi < ((u64)1 << 31)) return {};
        qmax = std::max(qmax, qi);
    }
    const u64 dmax = base_log2 >= 32 ? 0xffffffffull : (((u64)1 << base_log2) - 1);
    const Big bound = product({4, (u64)ell, (u64)N, dmax, qmax - 1});
    std::vector<u64> used = q, ps;
    used.push_back(t);
    while (ps.size() < 2 || product(ps).bits() - 1 < bound.bits()) {  // P >= 2^(bits(P) - 1)
        if ((int)ps.size() == kKsMaxPrimes) return {};
        const u64 p = next_prime_below(30, N, used);
        if (!p || p < ((u64)1 << 29)) return {};
        used.push_back(p);
        ps.push_back(p);
    }
    return ps;
}

int build_tables(he_ctx *c, std::string &err) {
    he_params &P = c->P;
    const int N = P.N;
    if (N < 1024 || N > 16384 || (N & (N - 1))) { err = "N must be a power of two in [1024, 16384]"; return HE_ERR_UNSUPPORTED_PARAMS; }
    if (P.L < 1 || P.L > HE_MAX_LIMBS) { err = "L out of range"; return HE_ERR_INVALID_ARG; }
    if (P.t < 2 || P.t >= ((u64)1 << 61)) { err = "t out of range"; return HE_ERR_UNSUPPORTED_PARAMS; }
    if (P.base_log2 == 0) P.base_log2 = 16;
    if (P.eta == 0) P.eta = 21;
    if (P.max_ccmul_group == 0) P.max_ccmul_group = 64;
    if (P.base_log2 < 1 || P.base_log2 > 32) { err = "base_log2 out of range"; return HE_ERR_INVALID_ARG; }
    if (P.eta < 1 || P.eta > 32) { err = "eta out of range"; return HE_ERR_INVALID_ARG; }
    if (P.max_ccmul_group < 1) { err = "max_ccmul_group out of range"; return HE_ERR_INVALID_ARG; }
    if (!(P.max_ccmul_scratch_bytes >= 0)) { err = "max_ccmul_scratch_bytes out of range"; return HE_ERR_INVALID_ARG; }
    if (!(P.max_table_cache_bytes >= 0)) { err = "max_table_cache_bytes out of range"; return HE_ERR_INVALID_ARG; }
    c->N = N;
    c->logN = 0;
    while ((1 << c->logN) < N) c->logN++;
    c->L = P.L;
    // limb primes
    {
        const int rc = limb_primes(P, N, c->q, err);
        if (rc) return rc;
    }
    for (int i = 0; i < P.L; i++) P.q[i] = c->q[i];
    for (u64 q : c->q)
        if (std::__gcd(q, (u64)P.t) != 1) { err = "t must be coprime to q"; return HE_ERR_UNSUPPORTED_PARAMS; }
    Big Q = product(c->q);
    c->ell = (Q.bits() + P.base_log2 - 1) / P.base_log2;
    // auxiliary basis: 61-bit primes until B > group * N * t * Q * 2
    int gbits = 0;
    while ((1LL << gbits) < P.max_ccmul_group) gbits++;
    const int need = gbits + c->logN + Big::of(P.t).bits() + Q.bits() + 1;
    std::vector<u64> used = c->q;
    c->aux.clear();
    while (true) {
        Big B = product(c->aux);
        if (!c->aux.empty() && B.bits() - 1 >= need) break;
        u64 p = next_prime_below(61, N, used);
        if (!p) { err = "aux primes exhausted"; return HE_ERR_UNSUPPORTED_PARAMS; }
        used.push_back(p);
        c->aux.push_back(p);
        if ((int)c->aux.size() > 24) { err = "aux basis too large"; return HE_ERR_UNSUPPORTED_PARAMS; }
    }
    if (std::find(c->q.begin(), c->q.end(), P.t) != c->q.end()) { err = "t equals a limb prime"; return HE_ERR_UNSUPPORTED_PARAMS; }
    c->K = (int)c->aux.size();
    c->h_mods.clear();
    for (u64 q : c->q)
        if (!add_modulus(c, q, err)) return HE_ERR_CUDA;
    for (u64 q : c->aux)
        if (!add_modulus(c, q, err)) return HE_ERR_CUDA;
    c->t_mod = -1;
    if (is_prime(P.t) && P.t % (2 * (u64)N) == 1) {
        if (!add_modulus(c, P.t, err)) return HE_ERR_CUDA;
        c->t_mod = c->L + c->K;
    }
    c->n_mods = (int)c->h_mods.size();
    if (c->n_mods > MAX_MODS) { err = "too many moduli"; return HE_ERR_UNSUPPORTED_PARAMS; }
    // exact-kernel constants
    ExactDev &E = c->h_exact;
    memset(&E, 0, sizeof E);
    if (!fill_crt(E.Q, c->q, err) || !fill_crt(E.B, c->aux, err)) return HE_ERR_UNSUPPORTED_PARAMS;
    Big Qh = Q.shr1();
    Big Bp = product(c->aux);
    const u64 t = P.t;
    u64 rem;
    Big delta = Q.div(t, &rem);
    for (int j = 0; j < c->K; j++) {
        const u64 b = c->aux[j];
        E.Q_b[j] = Q.mod(b);
        E.Qhalf_b[j] = Qh.mod(b);
        E.Qinv_b[j] = invmod(E.Q_b[j], b);
        E.Qinv_bs[j] = shoup_c(E.Qinv_b[j], b);
        E.t_b[j] = t % b;
        E.t_bs[j] = shoup_c(E.t_b[j], b);
    }
    for (int i = 0; i < c->L; i++) {
        const u64 q = c->q[i];
        E.B_q[i] = Bp.mod(q);
        E.Qhalf_q[i] = Qh.mod(q);
        E.t_q[i] = t % q;
        E.t_qs[i] = shoup_c(E.t_q[i], q);
        E.delta_q[i] = delta.mod(q);
        E.delta_qs[i] = shoup_c(E.delta_q[i], q);
    }
    auto fill_conv = [](ConvDev &C, const std::vector<u64> &m) {
        for (size_t i = 0; i < m.size(); i++) {
            int sh = __builtin_clzll(m[i]);
            u64 mp = m[i] << sh;  // in [2^63, 2^64)
            C.sh[i] = (u64)sh;
            C.c[i] = (u64)((((u128)1) << 127) / mp);
        }
    };
    fill_conv(E.Qc, c->q);
    fill_conv(E.Bc, c->aux);
    for (int j = 0; j < c->K; j++) {
        const u64 b = c->aux[j];
        for (int i = 0; i < c->L; i++) {
            u64 r;
            E.QhatB[j][i] = Q.div(c->q[i], &r).mod(b);
            E.QhatBm[j][i] = mulmod(E.QhatB[j][i], (u64)(((u128)1 << 64) % b), b);
        }
        E.Q_bs[j] = shoup_c(E.Q_b[j], b);
    }
    for (int i = 0; i < c->L; i++) {
        const u64 q = c->q[i];
        for (int j = 0; j < c->K; j++) {
            u64 r;
            E.BhatQ[i][j] = Bp.div(c->aux[j], &r).mod(q);
            E.BhatQm[i][j] = mulmod(E.BhatQ[i][j], (u64)(((u128)1 << 64) % q), q);
        }
        E.B_qs[i] = shoup_c(E.B_q[i], q);
        u64 r;
        E.Qhat_t[i] = Q.div(q, &r).mod(t);
        E.Qhat_ts[i] = shoup_c(E.Qhat_t[i], t);
    }
    E.Q_t = Q.mod(t);
    E.Q_ts = shoup_c(E.Q_t, t);
    E.t = t;
    E.Qhalf_t = Qh.mod(t);
    E.Qinv_t = invmod(Q.mod(t), t);
    if (!E.Qinv_t && t > 1) { err = "q not invertible mod t"; return HE_ERR_UNSUPPORTED_PARAMS; }
    E.Qinv_ts = shoup_c(E.Qinv_t, t);
    // folded constants of the rescaling
    for (int i = 0; i < c->L; i++) {
        const u64 q = c->q[i], inv = E.Q.inv[i];
        E.f_tq[i] = mulmod(E.t_q[i], inv, q);
        E.f_tqs[i] = shoup_c(E.f_tq[i], q);
        E.f_hq[i] = mulmod(E.Qhalf_q[i], inv, q);
        for (int j = 0; j < c->K; j++) {
            E.BhatQi[i][j] = mulmod(E.BhatQ[i][j], inv, q);
            E.BhatQim[i][j] = mulmod(E.BhatQi[i][j], (u64)(((u128)1 << 64) % q), q);
        }
        E.B_qi[i] = mulmod(E.B_q[i], inv, q);
        E.B_qis[i] = shoup_c(E.B_qi[i], q);
    }
    for (int j = 0; j < c->K; j++) {
        const u64 b = c->aux[j], cj = mulmod(E.Qinv_b[j], E.B.inv[j], b);
        E.f_cb[j] = cj;
        E.f_cbs[j] = shoup_c(cj, b);
        E.f_tb[j] = mulmod(E.t_b[j], cj, b);
        E.f_tbs[j] = shoup_c(E.f_tb[j], b);
        E.f_hb[j] = mulmod(E.Qhalf_b[j], cj, b);
        for (int i = 0; i < c->L; i++) {
            E.QhatBc[j][i] = mulmod(E.QhatB[j][i], cj, b);
            E.QhatBcm[j][i] = mulmod(E.QhatBc[j][i], (u64)(((u128)1 << 64) % b), b);
        }
        E.Q_bc[j] = mulmod(E.Q_b[j], cj, b);
        E.Q_bcs[j] = shoup_c(E.Q_bc[j], b);
    }
    E.r64_t = (u64)(((u128)1 << 64) % t);
    E.r64_ts = shoup_c(E.r64_t, t);
    E.one_ts = (u64)(((u128)1 << 64) / t);
    // upload
    if (he::dev_alloc((void **)&c->d_mods, sizeof(ModDev) * c->n_mods) != cudaSuccess ||
        he::dev_alloc((void **)&c->d_exact, sizeof(ExactDev)) != cudaSuccess) {
        err = "cudaMalloc tables";
        return HE_ERR_OOM;
    }
    if (cudaMemcpy(c->d_mods, c->h_mods.data(), sizeof(ModDev) * c->n_mods, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_exact, &E, sizeof(ExactDev), cudaMemcpyHostToDevice) != cudaSuccess) {
        err = "upload tables";
        return HE_ERR_CUDA;
    }
    return build_ks(c, err);
}

// Tables of one small prime p < 2^30 of the key switch: the same three tables
// as add_modulus (forward factors in the register pass order, inverse
// factors, untwist), as (value, floor(value 2^32 / p)) pairs of 32-bit words;
// the untwist carries 2^32 for the Montgomery fold of the sums.
static bool add_ks_prime(he_ctx *c, u64 p, Mod32Dev &M, std::string &err) {
    const int N = c->N, logN = c->logN;
    const u64 psi = root_2n(p, N);
    if (!psi) { err = "no primitive 2N-th root"; return false; }
    const u64 psiinv = invmod(psi, p), ninv = invmod((u64)N, p), r32 = ((u64)1 << 32) % p;
    auto comp = [&](u64 w) { return (uint32_t)((w << 32) / p); };
    std::vector<uint32_t> tab(6 * (size_t)N, 0);
    uint32_t *fw = tab.data(), *iw = fw + 2 * N, *zt = iw + 2 * N;
    std::vector<u64> pw(2 * N), ipw(2 * N);
    pw[0] = ipw[0] = 1;
    for (int e = 1; e < 2 * N; e++) { pw[e] = mulmod(pw[e - 1], psi, p); ipw[e] = mulmod(ipw[e - 1], psiinv, p); }
    for (int k = 0; k < N; k++) {
        const u64 z = mulmod(mulmod(ipw[k], ninv, p), r32, p);
        zt[2 * k] = (uint32_t)z;
        zt[2 * k + 1] = comp(z);
    }
    const int RB = kNttTileBits, NP = (logN + RB - 1) / RB, RL = logN - RB * (NP - 1);
    for (int pass = 0; pass < NP; pass++) {
        const int S = pass == NP - 1 ? RL : RB;
        for (int st = 0; st < S; st++) {
            const int s = RB * pass + st, gb = RB - 1 - (S - 1 - st);
            for (int i = 0; i < (1 << s); i++) {
                const int g = i & ((1 << gb) - 1), h = i >> gb;
                const size_t pos = (size_t)(1 << s) + ((size_t)g << (s - gb)) + h;
                const u64 w = pw[bitrev((1 << s) + i, logN)];
                fw[2 * pos] = (uint32_t)w;
                fw[2 * pos + 1] = comp(w);
            }
        }
    }
    for (int s = 0; s < logN; s++)
        for (int k = 0; k < (1 << s); k++) {
            const u64 w = ipw[((u64)k << (logN - s)) % (2 * (u64)N)];
            const size_t i = (size_t)(1 << s) + k;
            iw[2 * i] = (uint32_t)w;
            iw[2 * i + 1] = comp(w);
        }
    void *d = nullptr;
    if (he::dev_alloc(&d, tab.size() * 4) != cudaSuccess) { err = "cudaMalloc key-switch tables"; return false; }
    c->allocs.push_back(d);
    if (cudaMemcpy(d, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        err = "upload key-switch tables";
        return false;
    }
    M.p = (uint32_t)p;
    M.twop = (uint32_t)(2 * p);
    u64 x = p;  // p^-1 mod 2^64 (Newton), then -p^-1 mod 2^32
    for (int it = 0; it < 5; it++) x *= 2 - p * x;
    M.pinv = (uint32_t)(0 - x);
    M.ones = (uint32_t)((((u64)1) << 32) / p);
    M.r32 = (uint32_t)r32;
    M.fw = (const uint2 *)d;
    M.iw = M.fw + N;
    M.z = M.iw + N;
    return true;
}

// Tables and CRT constants of the context's key-switch primes (ks_select;
// np = 0 when it chooses none).
int build_ks(he_ctx *c, std::string &err) {
    KsDev &K = c->h_ks;
    memset(&K, 0, sizeof K);
    const std::vector<u64> ps = ks_select(c->q, c->P.t, c->N, c->ell, c->P.base_log2);
    if (ps.empty()) return HE_OK;
    const int np = (int)ps.size();
    for (int k = 0; k < np; k++)
        if (!add_ks_prime(c, ps[k], K.m[k], err)) return HE_ERR_CUDA;
    // a 64-bit sum of products below (p - 1)^2 is folded to (h mod p)(2^32
    // mod p) + l < (p - 1)^2 + 2^32 every `fold` products, so it stays below
    // 2^64 with fold more products added
    u128 f = ~(u64)0;
    for (u64 p : ps) {
        const u128 sq = (u128)(p - 1) * (p - 1);
        f = std::min<u128>(f, ((u128)(~(u64)0) - sq - ((u128)1 << 32)) / sq);
    }
    K.fold = (int)std::min<u128>(f, 64);
    for (int k = 0; k < np; k++)
        for (int m = 0; m < k; m++) {
            const u64 v = invmod(ps[m] % ps[k], ps[k]);
            K.ginv[k][m] = (uint32_t)v;
            K.ginvs[k][m] = (uint32_t)((v << 32) / ps[k]);
        }
    K.half_top = (uint32_t)(ps[np - 1] >> 1);
    for (int i = 0; i < c->L; i++) {
        const u64 q = c->q[i];
        u64 P = 1;
        for (int m = 0; m < np; m++) {
            K.pq_s[i][m] = shoup_c(ps[m], q);
            P = mulmod(P, ps[m], q);
        }
        K.P_q[i] = P;
        K.P_qs[i] = shoup_c(P, q);
    }
    K.np = np;
    return HE_OK;
}

// 2^(base*j) mod q_i with Shoup companions, [ell][L][2]
std::vector<u64> relin_multipliers(const he_ctx *c) {
    std::vector<u64> g((size_t)c->ell * c->L * 2);
    for (int j = 0; j < c->ell; j++)
        for (int i = 0; i < c->L; i++) {
            u64 v = powmod(2, (u64)c->P.base_log2 * (u64)j, c->q[i]);
            g[((size_t)j * c->L + i) * 2] = v;
            g[((size_t)j * c->L + i) * 2 + 1] = shoup_c(v, c->q[i]);
        }
    return g;
}

}  // namespace he

extern "C" int he_ks_primes(const he_params *params, uint64_t *primes, int32_t *np) {
    if (!params || !primes || !np) return HE_ERR_INVALID_ARG;
    *np = 0;
    const int N = params->N;
    if (N < 1024 || N > 16384 || (N & (N - 1))) return HE_ERR_UNSUPPORTED_PARAMS;
    if (params->L < 1 || params->L > HE_MAX_LIMBS) return HE_ERR_INVALID_ARG;
    const int base = params->base_log2 ? params->base_log2 : 16;
    if (base < 1 || base > 32) return HE_ERR_INVALID_ARG;
    std::vector<u64> q;
    std::string err;
    const int rc = he::limb_primes(*params, N, q, err);
    if (rc) return rc;
    const int ell = (he::product(q).bits() + base - 1) / base;
    const std::vector<u64> ps = he::ks_select(q, params->t, N, ell, base);
    for (size_t k = 0; k < ps.size(); k++) primes[k] = ps[k];
    *np = (int32_t)ps.size();
    return HE_OK;
}
