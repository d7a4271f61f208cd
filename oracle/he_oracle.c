/*
 * he_oracle.c -- plain, slow CPU reference for the RLWE/BFV linear-layer path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only tests, the package smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code with the CUDA path.
 *
 * Every routine follows the mathematical definition as directly as possible:
 *   - ring A_{N,q} = Z_q[x]/(x^N+1) (Section 2, Notations), products by a
 *     textbook negacyclic NTT (twist by psi, cyclic radix-2 with an explicit
 *     bit-reversal, untwist), pinned by tests against a schoolbook product;
 *   - BFV encryption / decryption eps(p,pk), sigma(c,sk) (Section 2, HE) with
 *     Delta = floor(q/t) and decryption floor((t*x + floor(q/2))/q) mod t done
 *     with an explicit big integer;
 *   - CPMul (c0*p, c1*p) and CCAdd (Section 2, Motivation / Fig. 3);
 *   - CCMul: exact integer tensor product of the centred lifts, exact
 *     rounding floor((t*d + floor(q/2))/q) mod q, then relinearisation with
 *     base-2^k digits (Section 2, Motivation / Fig. 3(b));
 *   - PPMul: negacyclic product mod t (Section 3.2, online phase).
 * Randomness: ChaCha20 block function (RFC 8439, section 2.3) used as a
 * counter-based generator; the sampling conventions are stated at each
 * sampler.  Parity unpinned for the samplers: the paper fixes no generator,
 * so the mapping from stream words to samples -- and with it the exact bits
 * of keys, ciphertexts and masks -- is a convention both sides implement from
 * its written definition; the block function itself is pinned by the RFC test
 * vector and the sample distributions by statistics tests.
 *
 * Integer products that exceed 64 bits use unsigned __int128 with the '%'
 * operator; big integers are fixed-width two's-complement arrays of 32-bit
 * words and use schoolbook / bit-serial algorithms only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* 64-bit modular helpers                                              */
/* ------------------------------------------------------------------ */
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)(((u128)a * b) % m); }
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t m) { u128 s = (u128)a + b; return (uint64_t)(s % m); }
static uint64_t submod(uint64_t a, uint64_t b, uint64_t m) { return a >= b ? a - b : a + (m - b); }
static uint64_t powmod(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m; a %= m;
    while (e) { if (e & 1) r = mulmod(r, a, m); a = mulmod(a, a, m); e >>= 1; }
    return r;
}
static uint64_t invmod(uint64_t a, uint64_t p) { return powmod(a, p - 2, p); } /* p prime */
/* signed integer v mapped to [0, m) */
static uint64_t smod(int64_t v, uint64_t m) {
    if (v >= 0) return (uint64_t)v % m;
    uint64_t r = (uint64_t)(-(v + 1)) % m; /* avoids overflow at INT64_MIN */
    r = (r + 1) % m;
    return r == 0 ? 0 : m - r;
}

/* Deterministic Miller-Rabin for 64-bit n with the first twelve primes as
 * bases (correct for all n < 3.3e24, Sorenson & Webster 2015). */
int orc_is_prime(uint64_t n) {
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) { if (n == bases[i]) return 1; if (n % bases[i] == 0) return 0; }
    uint64_t d = n - 1; int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int r = 1; r < s; r++) { x = mulmod(x, x, n); if (x == n - 1) { comp = 0; break; } }
        if (comp) return 0;
    }
    return 1;
}

/* For each requested bit size b (in order), the largest prime p < 2^b with
 * p = 1 mod 2N that is not excluded and not already chosen.  Returns 0 on
 * success, -1 if none exists. */
int orc_gen_primes(int N, const int *bits, int L, const uint64_t *excl, int n_excl, uint64_t *out) {
    uint64_t step = 2 * (uint64_t)N;
    for (int i = 0; i < L; i++) {
        if (bits[i] < 2 || bits[i] > 62) return -1;
        uint64_t top = (uint64_t)1 << bits[i];
        uint64_t p = ((top - 2) / step) * step + 1; /* largest candidate < 2^b that is 1 mod 2N */
        int found = 0;
        for (; p > step; p -= step) {
            int used = 0;
            for (int j = 0; j < i; j++) if (out[j] == p) used = 1;
            for (int j = 0; j < n_excl; j++) if (excl[j] == p) used = 1;
            if (used) continue;
            if (orc_is_prime(p)) { found = 1; break; }
        }
        if (!found) return -1;
        out[i] = p;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* ChaCha20 (RFC 8439, section 2.3)                                     */
/* ------------------------------------------------------------------ */
static uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }
static void qround(uint32_t *s, int a, int b, int c, int d) {
    s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 16);
    s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 12);
    s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 8);
    s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 7);
}
void orc_chacha20_block(const uint32_t key[8], uint32_t counter, const uint32_t nonce[3], uint32_t out[16]) {
    uint32_t init[16];
    init[0] = 0x61707865u; init[1] = 0x3320646eu; init[2] = 0x79622d32u; init[3] = 0x6b206574u;
    for (int i = 0; i < 8; i++) init[4 + i] = key[i];
    init[12] = counter; init[13] = nonce[0]; init[14] = nonce[1]; init[15] = nonce[2];
    uint32_t s[16];
    memcpy(s, init, sizeof s);
    for (int i = 0; i < 10; i++) {
        qround(s, 0, 4, 8, 12); qround(s, 1, 5, 9, 13); qround(s, 2, 6, 10, 14); qround(s, 3, 7, 11, 15);
        qround(s, 0, 5, 10, 15); qround(s, 1, 6, 11, 12); qround(s, 2, 7, 8, 13); qround(s, 3, 4, 9, 14);
    }
    for (int i = 0; i < 16; i++) out[i] = s[i] + init[i];
}

/* Stream convention: key = (seed low 32, seed high 32, 0 x 6), nonce =
 * (tag, idx, limb), block counter = w / 8; 64-bit word w is state words
 * 2(w%8) (low half) and 2(w%8)+1 (high half) of that block. */
void orc_stream_words(uint64_t seed, uint32_t tag, uint32_t idx, uint32_t limb,
                      uint64_t first, uint64_t n, uint64_t *out) {
    uint32_t key[8] = {(uint32_t)seed, (uint32_t)(seed >> 32), 0, 0, 0, 0, 0, 0};
    uint32_t nonce[3] = {tag, idx, limb};
    uint32_t blk[16];
    uint64_t cur = UINT64_MAX;
    for (uint64_t k = 0; k < n; k++) {
        uint64_t w = first + k;
        if (w / 8 != cur) { cur = w / 8; orc_chacha20_block(key, (uint32_t)cur, nonce, blk); }
        int j = (int)(w % 8);
        out[k] = (uint64_t)blk[2 * j] | ((uint64_t)blk[2 * j + 1] << 32);
    }
}

/* uniform mod q: coefficient k = (word(2k+1) * 2^64 + word(2k)) mod q */
void orc_sample_uniform(uint64_t seed, uint32_t tag, uint32_t idx, uint32_t limb, uint64_t q, int N, uint64_t *out) {
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * 2 * (size_t)N);
    orc_stream_words(seed, tag, idx, limb, 0, 2 * (uint64_t)N, w);
    for (int k = 0; k < N; k++) {
        u128 v = ((u128)w[2 * k + 1] << 64) | w[2 * k];
        out[k] = (uint64_t)(v % q);
    }
    free(w);
}
/* ternary: floor(word * 3 / 2^64) - 1 in {-1,0,1}; stream limb field 0 */
void orc_sample_ternary(uint64_t seed, uint32_t tag, uint32_t idx, int N, int64_t *out) {
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    orc_stream_words(seed, tag, idx, 0, 0, (uint64_t)N, w);
    for (int k = 0; k < N; k++) out[k] = (int64_t)(uint64_t)(((u128)w[k] * 3) >> 64) - 1;
    free(w);
}
/* centred binomial: popcount(low eta bits) - popcount(next eta bits) */
void orc_sample_cbd(uint64_t seed, uint32_t tag, uint32_t idx, int eta, int N, int64_t *out) {
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    orc_stream_words(seed, tag, idx, 0, 0, (uint64_t)N, w);
    uint64_t mask = ((uint64_t)1 << eta) - 1;
    for (int k = 0; k < N; k++) {
        int a = 0, b = 0;
        for (int i = 0; i < eta; i++) { a += (int)((w[k] >> i) & 1); b += (int)((w[k] >> (eta + i)) & 1); }
        (void)mask;
        out[k] = a - b;
    }
    free(w);
}
/* uniform mod t: word mod t */
void orc_sample_uniform_t(uint64_t seed, uint32_t tag, uint32_t idx, uint64_t t, int N, uint64_t *out) {
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    orc_stream_words(seed, tag, idx, 0, 0, (uint64_t)N, w);
    for (int k = 0; k < N; k++) out[k] = w[k] % t;
    free(w);
}

/* ------------------------------------------------------------------ */
/* Negacyclic product in Z_p[x]/(x^N+1), p prime, p = 1 mod 2N          */
/* ------------------------------------------------------------------ */
/* a primitive 2N-th root of unity: g^((p-1)/2N) with the smallest g >= 2
 * for which the result has psi^N = -1 */
static uint64_t find_psi(uint64_t p, int N) {
    for (uint64_t g = 2;; g++) {
        uint64_t psi = powmod(g, (p - 1) / (2 * (uint64_t)N), p);
        if (powmod(psi, (uint64_t)N, p) == p - 1) return psi;
    }
}
static void bitrev_permute(uint64_t *a, int N) {
    for (int i = 1, j = 0; i < N; i++) {
        int bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}
/* textbook iterative radix-2 cyclic DFT: A[k] = sum_i a[i] w^(ik) */
static void cyclic_dft(uint64_t *a, int N, uint64_t w, uint64_t p) {
    bitrev_permute(a, N);
    for (int len = 2; len <= N; len <<= 1) {
        uint64_t wl = powmod(w, (uint64_t)(N / len), p);
        for (int i = 0; i < N; i += len) {
            uint64_t ww = 1;
            for (int j = 0; j < len / 2; j++) {
                uint64_t u = a[i + j], v = mulmod(a[i + j + len / 2], ww, p);
                a[i + j] = addmod(u, v, p);
                a[i + j + len / 2] = submod(u, v, p);
                ww = mulmod(ww, wl, p);
            }
        }
    }
}
/* c = a*b in Z_p[x]/(x^N+1); inputs in [0,p).  c may alias a or b. */
void orc_polymul(const uint64_t *a, const uint64_t *b, uint64_t *c, int N, uint64_t p) {
    uint64_t psi = find_psi(p, N), w = mulmod(psi, psi, p);
    uint64_t *fa = (uint64_t *)malloc(8 * (size_t)N), *fb = (uint64_t *)malloc(8 * (size_t)N);
    uint64_t pw = 1;
    for (int i = 0; i < N; i++) { fa[i] = mulmod(a[i] % p, pw, p); fb[i] = mulmod(b[i] % p, pw, p); pw = mulmod(pw, psi, p); }
    cyclic_dft(fa, N, w, p);
    cyclic_dft(fb, N, w, p);
    for (int i = 0; i < N; i++) fa[i] = mulmod(fa[i], fb[i], p);
    cyclic_dft(fa, N, invmod(w, p), p);
    uint64_t ninv = invmod((uint64_t)N, p), psiinv = invmod(psi, p);
    pw = ninv;
    for (int i = 0; i < N; i++) { c[i] = mulmod(fa[i], pw, p); pw = mulmod(pw, psiinv, p); }
    free(fa); free(fb);
}

/* ------------------------------------------------------------------ */
/* Fixed-width big integers (two's complement, 32-bit words)            */
/* ------------------------------------------------------------------ */
#define BW 44 /* 1408 bits: enough for t * (tensor products of 480-bit moduli) */
typedef struct { uint32_t w[BW]; } big;

static void big_zero(big *a) { memset(a, 0, sizeof *a); }
static void big_from_u64(big *a, uint64_t v) { big_zero(a); a->w[0] = (uint32_t)v; a->w[1] = (uint32_t)(v >> 32); }
static int big_is_neg(const big *a) { return (a->w[BW - 1] >> 31) & 1; }
static void big_add(big *r, const big *a, const big *b) {
    uint64_t c = 0;
    for (int i = 0; i < BW; i++) { c += (uint64_t)a->w[i] + b->w[i]; r->w[i] = (uint32_t)c; c >>= 32; }
}
static void big_sub(big *r, const big *a, const big *b) {
    int64_t br = 0;
    for (int i = 0; i < BW; i++) {
        int64_t d = (int64_t)a->w[i] - b->w[i] - br;
        br = d < 0; r->w[i] = (uint32_t)(d + (br ? ((int64_t)1 << 32) : 0));
    }
}
static void big_neg(big *r, const big *a) { big z; big_zero(&z); big_sub(r, &z, a); }
/* r = a * m (m < 2^64); a may be negative (the product is taken mod 2^(32 BW),
 * which is the two's-complement product whenever it fits) */
static void big_mul_u64(big *r, const big *a, uint64_t m) {
    big out; big_zero(&out);
    uint32_t ml = (uint32_t)m, mh = (uint32_t)(m >> 32);
    for (int part = 0; part < 2; part++) {
        uint64_t mm = part ? mh : ml, c = 0;
        for (int i = 0; i + part < BW; i++) {
            c += (uint64_t)out.w[i + part] + (uint64_t)a->w[i] * mm;
            out.w[i + part] = (uint32_t)c; c >>= 32;
        }
    }
    *r = out;
}
/* signed compare */
static int big_cmp(const big *a, const big *b) {
    int na = big_is_neg(a), nb = big_is_neg(b);
    if (na != nb) return na ? -1 : 1;
    for (int i = BW - 1; i >= 0; i--) if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
    return 0;
}
static int big_nwords(const big *a) { /* a >= 0: index of the top non-zero word + 1 */
    for (int i = BW - 1; i >= 0; i--) if (a->w[i]) return i + 1;
    return 0;
}
static int big_bitlen(const big *a) { /* a >= 0 */
    int n = big_nwords(a);
    if (!n) return 0;
    int b = 31; while (!((a->w[n - 1] >> b) & 1)) b--;
    return 32 * (n - 1) + b + 1;
}
static int big_bit(const big *a, int i) { return (a->w[i / 32] >> (i % 32)) & 1; }
/* non-negative a mod m (m < 2^64), Horner over 32-bit words */
static uint64_t big_mod_u64(const big *a, uint64_t m) {
    u128 r = 0;
    for (int i = big_nwords(a) - 1; i >= 0; i--) r = ((r << 32) | a->w[i]) % m;
    return (uint64_t)r;
}
/* signed a mod m in [0,m) */
static uint64_t big_smod_u64(const big *a, uint64_t m) {
    if (!big_is_neg(a)) return big_mod_u64(a, m);
    big p; big_neg(&p, a);
    uint64_t r = big_mod_u64(&p, m);
    return r == 0 ? 0 : m - r;
}
/* floor(num / den) for den > 0, num of either sign: restoring bit-serial long
 * division of |num| (remainder kept below 2*den, so only the low words of den
 * plus one are touched), then the floor correction for negative num. */
static void big_floordiv(big *quo, const big *num, const big *den) {
    int neg = big_is_neg(num);
    big n; if (neg) big_neg(&n, num); else n = *num;
    int W = big_nwords(den) + 1;
    if (W > BW) W = BW;
    uint32_t r[BW], d[BW];
    memset(r, 0, sizeof r);
    for (int i = 0; i < W; i++) d[i] = den->w[i];
    big q; big_zero(&q);
    for (int i = big_bitlen(&n) - 1; i >= 0; i--) {
        /* r = 2 r + bit */
        uint32_t carry = (uint32_t)big_bit(&n, i);
        for (int k = 0; k < W; k++) { uint32_t nc = r[k] >> 31; r[k] = (r[k] << 1) | carry; carry = nc; }
        /* if r >= d: r -= d, quotient bit set */
        int ge = 1;
        for (int k = W - 1; k >= 0; k--) if (r[k] != d[k]) { ge = r[k] > d[k]; break; }
        if (ge) {
            int64_t br = 0;
            for (int k = 0; k < W; k++) {
                int64_t x = (int64_t)r[k] - d[k] - br;
                br = x < 0; r[k] = (uint32_t)(x + (br ? ((int64_t)1 << 32) : 0));
            }
            q.w[i / 32] |= 1u << (i % 32);
        }
    }
    if (neg) {
        int rz = 1; for (int k = 0; k < W; k++) if (r[k]) rz = 0;
        big_neg(&q, &q);
        if (!rz) { big one; big_from_u64(&one, 1); big_sub(&q, &q, &one); }
    }
    *quo = q;
}

/* CRT basis: moduli m[0..k), M = prod m, Mhat_i = M/m_i, and
 * (Mhat_i)^-1 mod m_i. */
typedef struct {
    int k;
    uint64_t m[32];
    big M, Mhalf; /* Mhalf = floor(M/2) */
    big Mhat[32];
    uint64_t Mhat_inv[32];
} crt_basis;

static void crt_init(crt_basis *B, const uint64_t *m, int k) {
    B->k = k;
    big_from_u64(&B->M, 1);
    for (int i = 0; i < k; i++) { B->m[i] = m[i]; big_mul_u64(&B->M, &B->M, m[i]); }
    for (int i = 0; i < k; i++) {
        big_from_u64(&B->Mhat[i], 1);
        for (int j = 0; j < k; j++) if (j != i) big_mul_u64(&B->Mhat[i], &B->Mhat[i], m[j]);
        B->Mhat_inv[i] = invmod(big_mod_u64(&B->Mhat[i], m[i]), m[i]);
    }
    big two; big_from_u64(&two, 2);
    big_floordiv(&B->Mhalf, &B->M, &two);
}
/* X in [0, M) with X = r_i mod m_i */
static void crt_reconstruct(const crt_basis *B, const uint64_t *r, big *X) {
    big acc, t; big_zero(&acc);
    for (int i = 0; i < B->k; i++) {
        uint64_t y = mulmod(r[i] % B->m[i], B->Mhat_inv[i], B->m[i]);
        big_mul_u64(&t, &B->Mhat[i], y);
        big_add(&acc, &acc, &t);
    }
    while (big_cmp(&acc, &B->M) >= 0) big_sub(&acc, &acc, &B->M);
    *X = acc;
}
/* centred representative in (-M/2, M/2] */
static void crt_reconstruct_centred(const crt_basis *B, const uint64_t *r, big *X) {
    crt_reconstruct(B, r, X);
    if (big_cmp(X, &B->Mhalf) > 0) big_sub(X, X, &B->M);
}

/* ------------------------------------------------------------------ */
/* Parameter block passed from Python                                   */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t N, L;
    uint64_t q[16];
    uint64_t t;
    int32_t base_log2; /* relinearisation digit size */
    int32_t eta;       /* CBD parameter */
} orc_params;

/* domain tags of the random streams */
enum { TAG_SK = 1, TAG_PK_A = 2, TAG_PK_E = 3, TAG_ENC_U = 4, TAG_ENC_E1 = 5, TAG_ENC_E2 = 6,
       TAG_RLK_A = 7, TAG_RLK_E = 8, TAG_MASK = 9 };

typedef struct {
    const orc_params *P;
    crt_basis Q;
    big qhalf;          /* floor(q/2) */
    big delta;          /* floor(q/t) */
    int ell;            /* number of relinearisation digits */
} ctx_t;

static void ctx_init(ctx_t *c, const orc_params *P) {
    c->P = P;
    crt_init(&c->Q, P->q, P->L);
    c->qhalf = c->Q.Mhalf;
    big tb; big_from_u64(&tb, P->t);
    big_floordiv(&c->delta, &c->Q.M, &tb);
    int bl = big_bitlen(&c->Q.M);
    c->ell = (bl + P->base_log2 - 1) / P->base_log2;
}

int orc_num_digits(const orc_params *P) { ctx_t c; ctx_init(&c, P); return c.ell; }

/* small signed poly -> RNS poly */
static void small_to_rns(const int64_t *v, const orc_params *P, uint64_t *out /*[L][N]*/) {
    for (int i = 0; i < P->L; i++)
        for (int k = 0; k < P->N; k++) out[(size_t)i * P->N + k] = smod(v[k], P->q[i]);
}

/* out = a*b in R_q (RNS, [L][N] each) */
static void rns_mul(const orc_params *P, const uint64_t *a, const uint64_t *b, uint64_t *out) {
    for (int i = 0; i < P->L; i++)
        orc_polymul(a + (size_t)i * P->N, b + (size_t)i * P->N, out + (size_t)i * P->N, P->N, P->q[i]);
}

/* ------------------------------------------------------------------ */
/* Key generation (Section 2, HE; relinearisation key implied by Fig. 3b) */
/* ------------------------------------------------------------------ */
/* sk: int64[N] ternary; pk: [2][L][N] = (b, a), b = -(a s + e);
 * rlk (optional): [ell][2][L][N] with rlk_j = (-(a_j s + e_j) + 2^(base*j) s^2, a_j). */
int orc_keygen(const orc_params *P, uint64_t seed, int64_t *sk, uint64_t *pk, uint64_t *rlk) {
    ctx_t c; ctx_init(&c, P);
    int N = P->N, L = P->L;
    size_t LN = (size_t)L * N;
    orc_sample_ternary(seed, TAG_SK, 0, N, sk);
    uint64_t *s = malloc(8 * LN), *a = malloc(8 * LN), *e = malloc(8 * LN), *as = malloc(8 * LN);
    int64_t *es = malloc(8 * (size_t)N);
    small_to_rns(sk, P, s);
    for (int i = 0; i < L; i++) orc_sample_uniform(seed, TAG_PK_A, 0, (uint32_t)i, P->q[i], N, a + (size_t)i * N);
    orc_sample_cbd(seed, TAG_PK_E, 0, P->eta, N, es);
    small_to_rns(es, P, e);
    rns_mul(P, a, s, as);
    for (int i = 0; i < L; i++)
        for (int k = 0; k < N; k++) {
            size_t o = (size_t)i * N + k;
            pk[o] = submod(0, addmod(as[o], e[o], P->q[i]), P->q[i]);
            pk[LN + o] = a[o];
        }
    if (rlk) {
        uint64_t *s2 = malloc(8 * LN);
        rns_mul(P, s, s, s2);
        for (int j = 0; j < c.ell; j++) {
            uint64_t *r0 = rlk + (size_t)j * 2 * LN, *r1 = r0 + LN;
            for (int i = 0; i < L; i++) orc_sample_uniform(seed, TAG_RLK_A, (uint32_t)j, (uint32_t)i, P->q[i], N, r1 + (size_t)i * N);
            orc_sample_cbd(seed, TAG_RLK_E, (uint32_t)j, P->eta, N, es);
            small_to_rns(es, P, e);
            rns_mul(P, r1, s, as);
            for (int i = 0; i < L; i++) {
                /* 2^(base*j) mod q_i */
                uint64_t g = powmod(2, (uint64_t)P->base_log2 * (uint64_t)j, P->q[i]);
                for (int k = 0; k < N; k++) {
                    size_t o = (size_t)i * N + k;
                    uint64_t v = submod(0, addmod(as[o], e[o], P->q[i]), P->q[i]);
                    r0[o] = addmod(v, mulmod(g, s2[o], P->q[i]), P->q[i]);
                }
            }
        }
        free(s2);
    }
    free(s); free(a); free(e); free(as); free(es);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Encryption / decryption (Section 2, HE)                              */
/* ------------------------------------------------------------------ */
/* ct_k = (b u + e1 + Delta m, a u + e2), u/e1/e2 drawn with object index
 * idx; m: [N] in [0,t). */
int orc_encrypt(const orc_params *P, const uint64_t *pk, const uint64_t *m, uint64_t seed, uint32_t idx, uint64_t *ct) {
    ctx_t c; ctx_init(&c, P);
    int N = P->N, L = P->L;
    size_t LN = (size_t)L * N;
    int64_t *u = malloc(8 * (size_t)N), *e1 = malloc(8 * (size_t)N), *e2 = malloc(8 * (size_t)N);
    uint64_t *ur = malloc(8 * LN), *bu = malloc(8 * LN), *au = malloc(8 * LN);
    orc_sample_ternary(seed, TAG_ENC_U, idx, N, u);
    orc_sample_cbd(seed, TAG_ENC_E1, idx, P->eta, N, e1);
    orc_sample_cbd(seed, TAG_ENC_E2, idx, P->eta, N, e2);
    small_to_rns(u, P, ur);
    rns_mul(P, pk, ur, bu);
    rns_mul(P, pk + LN, ur, au);
    for (int i = 0; i < L; i++) {
        uint64_t qi = P->q[i], di = big_mod_u64(&c.delta, qi);
        for (int k = 0; k < N; k++) {
            size_t o = (size_t)i * N + k;
            uint64_t v = addmod(bu[o], smod(e1[k], qi), qi);
            ct[o] = addmod(v, mulmod(di, m[k] % P->t % qi, qi), qi);
            ct[LN + o] = addmod(au[o], smod(e2[k], qi), qi);
        }
    }
    free(u); free(e1); free(e2); free(ur); free(bu); free(au);
    return 0;
}

/* x = [c0 + c1 s]_q in [0,q) (exact), m = floor((t x + floor(q/2)) / q) mod t */
int orc_decrypt(const orc_params *P, const int64_t *sk, const uint64_t *ct, uint64_t *m) {
    ctx_t c; ctx_init(&c, P);
    int N = P->N, L = P->L;
    size_t LN = (size_t)L * N;
    uint64_t *s = malloc(8 * LN), *c1s = malloc(8 * LN);
    small_to_rns(sk, P, s);
    rns_mul(P, ct + LN, s, c1s);
    uint64_t r[32];
    big X, num, quo;
    for (int k = 0; k < N; k++) {
        for (int i = 0; i < L; i++) r[i] = addmod(ct[(size_t)i * N + k], c1s[(size_t)i * N + k], P->q[i]);
        crt_reconstruct(&c.Q, r, &X);
        big_mul_u64(&num, &X, P->t);
        big_add(&num, &num, &c.qhalf);
        big_floordiv(&quo, &num, &c.Q.M);
        m[k] = big_mod_u64(&quo, P->t);
    }
    free(s); free(c1s);
    return 0;
}

/* x = [c0 + c1 s]_q, centred, as doubles of log2|x| are not needed: return
 * the decryption noise infinity norm in bits (floor(log2(max |x - Delta m|)))
 * for the noise-budget tests. */
int orc_noise_bits(const orc_params *P, const int64_t *sk, const uint64_t *ct, const uint64_t *m) {
    ctx_t c; ctx_init(&c, P);
    int N = P->N, L = P->L;
    size_t LN = (size_t)L * N;
    uint64_t *s = malloc(8 * LN), *c1s = malloc(8 * LN);
    small_to_rns(sk, P, s);
    rns_mul(P, ct + LN, s, c1s);
    uint64_t r[32];
    int worst = 0;
    big X, dm;
    for (int k = 0; k < N; k++) {
        for (int i = 0; i < L; i++) r[i] = addmod(ct[(size_t)i * N + k], c1s[(size_t)i * N + k], P->q[i]);
        crt_reconstruct(&c.Q, r, &X);
        big_mul_u64(&dm, &c.delta, m[k] % P->t);
        big_sub(&X, &X, &dm);
        /* centre mod q */
        while (big_cmp(&X, &c.qhalf) > 0) big_sub(&X, &X, &c.Q.M);
        big lo; big_neg(&lo, &c.qhalf);
        while (big_cmp(&X, &lo) < 0) big_add(&X, &X, &c.Q.M);
        if (big_is_neg(&X)) big_neg(&X, &X);
        int b = big_bitlen(&X);
        if (b > worst) worst = b;
    }
    free(s); free(c1s);
    return worst;
}

/* ------------------------------------------------------------------ */
/* CPMul + CCAdd: out_o = sum_{terms of o} ct[g] * pt[p] (+ add_o)      */
/* ------------------------------------------------------------------ */
/* pt values in [0,t) are centre-lifted: v <= (t-1)/2 -> v, else v - t.
 * term_ptr[n_out+1] (CSR), term_ct / term_pt: indices; ct: [n_ct][2][L][N];
 * pt: [n_pt][N]; add: [n_out][2][L][N] or NULL; out: [n_out][2][L][N]. */
int orc_cpmul_terms(const orc_params *P, const uint64_t *ct, const uint64_t *pt,
                    const int32_t *term_ptr, const int32_t *term_ct, const int32_t *term_pt, int n_out,
                    const uint64_t *add, uint64_t *out) {
    int N = P->N, L = P->L;
    size_t LN = (size_t)L * N;
    uint64_t *pl = malloc(8 * (size_t)N), *prod = malloc(8 * (size_t)N);
    for (int o = 0; o < n_out; o++) {
        uint64_t *dst = out + (size_t)o * 2 * LN;
        if (add) memcpy(dst, add + (size_t)o * 2 * LN, 8 * 2 * LN);
        else memset(dst, 0, 8 * 2 * LN);
        for (int k = term_ptr[o]; k < term_ptr[o + 1]; k++) {
            const uint64_t *c = ct + (size_t)term_ct[k] * 2 * LN;
            const uint64_t *p = pt + (size_t)term_pt[k] * N;
            for (int i = 0; i < L; i++) {
                uint64_t qi = P->q[i];
                for (int x = 0; x < N; x++) {
                    uint64_t v = p[x] % P->t;
                    int64_t sv = v <= (P->t - 1) / 2 ? (int64_t)v : (int64_t)v - (int64_t)P->t;
                    pl[x] = smod(sv, qi);
                }
                for (int comp = 0; comp < 2; comp++) {
                    orc_polymul(c + comp * LN + (size_t)i * N, pl, prod, N, qi);
                    uint64_t *d = dst + comp * LN + (size_t)i * N;
                    for (int x = 0; x < N; x++) d[x] = addmod(d[x], prod[x], qi);
                }
            }
        }
    }
    free(pl); free(prod);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Exact integer negacyclic products of centred lifts (for CCMul)       */
/* ------------------------------------------------------------------ */
/* An auxiliary prime set A, independent of any GPU choice: the largest
 * 61-bit primes = 1 mod 2N, as many as needed so that prod(A) > 2^need. */
static int aux_primes(int N, int need_bits, uint64_t *out) {
    int k = need_bits / 60 + 2;
    if (k > 32) return -1;
    int bits[32];
    for (int i = 0; i < k; i++) bits[i] = 61;
    if (orc_gen_primes(N, bits, k, NULL, 0, out)) return -1;
    return k;
}

/* Centred big-integer lift of one RNS polynomial, reduced mod each aux prime:
 * res[j][x] = lift(c)[x] mod A_j. */
static void lift_to_aux(const ctx_t *c, const uint64_t *poly /*[L][N]*/, const uint64_t *A, int nA, uint64_t *res) {
    int N = c->P->N, L = c->P->L;
    uint64_t r[32];
    big X;
    for (int x = 0; x < N; x++) {
        for (int i = 0; i < L; i++) r[i] = poly[(size_t)i * N + x];
        crt_reconstruct_centred(&c->Q, r, &X);
        for (int j = 0; j < nA; j++) res[(size_t)j * N + x] = big_smod_u64(&X, A[j]);
    }
}

/* CCMul with exact rounding and relinearisation.
 * For each output o, with pairs k in [o*group, (o+1)*group):
 *   d0 = sum a0*b0, d1 = sum (a0*b1 + a1*b0), d2 = sum a1*b1  (exact integers
 *   of the centred lifts), d_j <- floor((t d_j + floor(q/2)) / q) mod q,
 *   then (c0, c1) = (d0, d1) + sum_j D_j rlk_j with D_j the base-2^base
 *   digits of d2 in [0,q).
 * ct_a: [n_a][2][L][N], ct_b: [n_b][2][L][N], pair_a/pair_b: [n_pairs]
 * indices, rlk: [ell][2][L][N] (coefficient form), out: [n_pairs/group][2][L][N]. */
int orc_ccmul(const orc_params *P, const uint64_t *rlk, const uint64_t *ct_a, const uint64_t *ct_b,
              const int32_t *pair_a, const int32_t *pair_b, int n_pairs, int group, uint64_t *out) {
    ctx_t c; ctx_init(&c, P);
    int N = P->N, L = P->L;
    size_t LN = (size_t)L * N;
    if (group < 1 || n_pairs % group) return -1;
    int qbits = big_bitlen(&c.Q.M);
    int need = 2 * qbits + 20 + 40; /* > log2(group * 2N * (q/2)^2) + sign, generous */
    uint64_t A[32];
    int nA = aux_primes(N, need, A);
    if (nA < 0) return -1;
    crt_basis AB; crt_init(&AB, A, nA);
    size_t AN = (size_t)nA * N;
    uint64_t *la0 = malloc(8 * AN), *la1 = malloc(8 * AN), *lb0 = malloc(8 * AN), *lb1 = malloc(8 * AN);
    uint64_t *d[3], *tmp = malloc(8 * (size_t)N);
    for (int j = 0; j < 3; j++) d[j] = malloc(8 * AN);
    uint64_t *dq[3];
    for (int j = 0; j < 3; j++) dq[j] = malloc(8 * LN);
    uint64_t *digit = malloc(8 * (size_t)c.ell * N), *dr = malloc(8 * LN), *pr = malloc(8 * LN);
    uint64_t r[32];
    big D, num, quo, X;
    for (int o = 0; o < n_pairs / group; o++) {
        for (int j = 0; j < 3; j++) memset(d[j], 0, 8 * AN);
        for (int k = o * group; k < (o + 1) * group; k++) {
            const uint64_t *a = ct_a + (size_t)pair_a[k] * 2 * LN, *b = ct_b + (size_t)pair_b[k] * 2 * LN;
            lift_to_aux(&c, a, A, nA, la0);
            lift_to_aux(&c, a + LN, A, nA, la1);
            lift_to_aux(&c, b, A, nA, lb0);
            lift_to_aux(&c, b + LN, A, nA, lb1);
            for (int j = 0; j < nA; j++) {
                size_t off = (size_t)j * N;
                orc_polymul(la0 + off, lb0 + off, tmp, N, A[j]);
                for (int x = 0; x < N; x++) d[0][off + x] = addmod(d[0][off + x], tmp[x], A[j]);
                orc_polymul(la0 + off, lb1 + off, tmp, N, A[j]);
                for (int x = 0; x < N; x++) d[1][off + x] = addmod(d[1][off + x], tmp[x], A[j]);
                orc_polymul(la1 + off, lb0 + off, tmp, N, A[j]);
                for (int x = 0; x < N; x++) d[1][off + x] = addmod(d[1][off + x], tmp[x], A[j]);
                orc_polymul(la1 + off, lb1 + off, tmp, N, A[j]);
                for (int x = 0; x < N; x++) d[2][off + x] = addmod(d[2][off + x], tmp[x], A[j]);
            }
        }
        /* exact rounding of every coefficient */
        for (int j = 0; j < 3; j++)
            for (int x = 0; x < N; x++) {
                for (int i = 0; i < nA; i++) r[i] = d[j][(size_t)i * N + x];
                crt_reconstruct_centred(&AB, r, &D);
                big_mul_u64(&num, &D, P->t);
                big_add(&num, &num, &c.qhalf);
                big_floordiv(&quo, &num, &c.Q.M);
                for (int i = 0; i < L; i++) dq[j][(size_t)i * N + x] = big_smod_u64(&quo, P->q[i]);
            }
        /* digits of d2 in [0,q) */
        for (int x = 0; x < N; x++) {
            for (int i = 0; i < L; i++) r[i] = dq[2][(size_t)i * N + x];
            crt_reconstruct(&c.Q, r, &X);
            for (int j = 0; j < c.ell; j++) {
                uint64_t v = 0;
                for (int b = 0; b < P->base_log2; b++) {
                    int bi = j * P->base_log2 + b;
                    if (bi < 32 * BW) v |= (uint64_t)big_bit(&X, bi) << b;
                }
                digit[(size_t)j * N + x] = v;
            }
        }
        uint64_t *dst = out + (size_t)o * 2 * LN;
        memcpy(dst, dq[0], 8 * LN);
        memcpy(dst + LN, dq[1], 8 * LN);
        for (int j = 0; j < c.ell; j++) {
            for (int i = 0; i < L; i++)
                for (int x = 0; x < N; x++) dr[(size_t)i * N + x] = digit[(size_t)j * N + x] % P->q[i];
            for (int comp = 0; comp < 2; comp++) {
                rns_mul(P, dr, rlk + ((size_t)j * 2 + comp) * LN, pr);
                for (int i = 0; i < L; i++)
                    for (int x = 0; x < N; x++) {
                        size_t oo = (size_t)i * N + x;
                        dst[comp * LN + oo] = addmod(dst[comp * LN + oo], pr[oo], P->q[i]);
                    }
            }
        }
    }
    free(la0); free(la1); free(lb0); free(lb1); free(tmp);
    for (int j = 0; j < 3; j++) { free(d[j]); free(dq[j]); }
    free(digit); free(dr); free(pr);
    (void)quo; (void)num;
    return 0;
}

/* ------------------------------------------------------------------ */
/* PPMul: negacyclic product mod t of values in [0,t)                   */
/* ------------------------------------------------------------------ */
/* out_o = sum_{terms} a[ia] * b[ib] mod t, computed as the exact integer
 * product of the [0,t) representatives (via two 61-bit aux primes), then
 * reduced mod t; t needs no NTT structure. a: [n_a][N], b: [n_b][N]. */
int orc_ppmul_terms(const orc_params *P, const uint64_t *a, const uint64_t *b,
                    const int32_t *term_ptr, const int32_t *term_a, const int32_t *term_b, int n_out, uint64_t *out) {
    int N = P->N;
    uint64_t A[32];
    int nA = aux_primes(N, 2 * 64 + 20, A);
    if (nA < 0) return -1;
    crt_basis AB; crt_init(&AB, A, nA);
    uint64_t *acc = malloc(8 * (size_t)nA * N), *ta = malloc(8 * (size_t)N), *tb = malloc(8 * (size_t)N), *tp = malloc(8 * (size_t)N);
    uint64_t r[32];
    big X;
    for (int o = 0; o < n_out; o++) {
        memset(acc, 0, 8 * (size_t)nA * N);
        for (int k = term_ptr[o]; k < term_ptr[o + 1]; k++)
            for (int j = 0; j < nA; j++) {
                for (int x = 0; x < N; x++) { ta[x] = a[(size_t)term_a[k] * N + x] % P->t; tb[x] = b[(size_t)term_b[k] * N + x] % P->t; }
                orc_polymul(ta, tb, tp, N, A[j]);
                for (int x = 0; x < N; x++) acc[(size_t)j * N + x] = addmod(acc[(size_t)j * N + x], tp[x], A[j]);
            }
        for (int x = 0; x < N; x++) {
            for (int j = 0; j < nA; j++) r[j] = acc[(size_t)j * N + x];
            crt_reconstruct_centred(&AB, r, &X);
            out[(size_t)o * N + x] = big_smod_u64(&X, P->t);
        }
    }
    free(acc); free(ta); free(tb); free(tp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Small exported helpers used by the tests                             */
/* ------------------------------------------------------------------ */
/* exact integer rounding of one value given as decimal-free words:
 * num = sum w[i] 2^(32 i) (two's complement, nw words), returns
 * floor((t*num + floor(q/2))/q) mod q_i for each limb. */
int orc_round_scalar(const orc_params *P, const uint32_t *w, int nw, uint64_t *out) {
    ctx_t c; ctx_init(&c, P);
    big D, num, quo;
    big_zero(&D);
    for (int i = 0; i < nw && i < BW; i++) D.w[i] = w[i];
    if (nw < BW && (w[nw - 1] >> 31)) for (int i = nw; i < BW; i++) D.w[i] = 0xffffffffu;
    big_mul_u64(&num, &D, P->t);
    big_add(&num, &num, &c.qhalf);
    big_floordiv(&quo, &num, &c.Q.M);
    for (int i = 0; i < P->L; i++) out[i] = big_smod_u64(&quo, P->q[i]);
    return 0;
}
