// arith.cuh -- device arithmetic: Shoup / Harvey modular products, lazy
// butterflies, multi-word CRT, ChaCha20.
//
// Modular products follow V. Shoup's precomputed-quotient method as used for
// NTTs by D. Harvey, "Faster arithmetic for number-theoretic transforms"
// (J. Symbolic Computation, 2014): for w < q < 2^62 and w' = floor(w 2^64 / q),
// a*w - floor(a w' / 2^64)*q lies in [0, 2q) for every 64-bit a.
#pragma once
#include "internal.h"
#include "checks.cuh"

namespace he {

__device__ __forceinline__ u64 shoup(u64 a, u64 w, u64 ws, u64 q) {
    u64 qh = __umul64hi(a, ws);
    return a * w - qh * q;  // [0, 2q)
}
// Shoup product built only from 32-bit multiply-accumulates (mul/mad.wide.u32
// and mad.lo.u32), the cheapest integer-multiply forms of the SM.  The
// quotient h = a1 s1 + floor((a1 s0 + a0 s1) / 2^32) is floor((a w' - a0 s0)
// / 2^64), at most 1 below the exact floor(a w' / 2^64); the remainder is
// a w + h (2^64 - q) mod 2^64.  Result in [0, 3q) for every 64-bit a.
// nq = 2^64 - q.
__device__ __forceinline__ u64 shoup3(u64 a, u64 w, u64 ws, u64 nq) {
    u64 r;
    asm("{\n\t"
        ".reg .u32 a0, a1, s0, s1, w0, w1, n0, n1, t0, t1, u0, u1, h0, h1, c, l0, l1, z;\n\t"
        ".reg .u64 t, tl, u, x, h, l;\n\t"
        "mov.b64 {a0, a1}, %1;\n\t"
        "mov.b64 {w0, w1}, %2;\n\t"
        "mov.b64 {s0, s1}, %3;\n\t"
        "mov.b64 {n0, n1}, %4;\n\t"
        "mul.wide.u32 t, a0, s1;\n\t"
        "mov.b64 {t0, t1}, t;\n\t"
        "cvt.u64.u32 tl, t0;\n\t"
        "mad.wide.u32 u, a1, s0, tl;\n\t"
        "mov.b64 {u0, u1}, u;\n\t"
        "add.cc.u32 c, u1, t1;\n\t"
        "addc.u32 z, 0, 0;\n\t"
        "mov.b64 x, {c, z};\n\t"
        "mad.wide.u32 h, a1, s1, x;\n\t"
        "mov.b64 {h0, h1}, h;\n\t"
        "mul.wide.u32 l, a0, w0;\n\t"
        "mad.wide.u32 l, h0, n0, l;\n\t"
        "mul.lo.u32 c, a0, w1;\n\t"
        "mad.lo.u32 c, a1, w0, c;\n\t"
        "mad.lo.u32 c, h0, n1, c;\n\t"
        "mad.lo.u32 c, h1, n0, c;\n\t"
        "mov.b64 {l0, l1}, l;\n\t"
        "add.u32 l1, l1, c;\n\t"
        "mov.b64 %0, {l0, l1};\n\t"
        "}"
        : "=l"(r)
        : "l"(a), "l"(w), "l"(ws), "l"(nq));
    return r;
}
// The same Shoup product for a multiplier k < 2^32 (a CRT overflow count):
// floor(k w' / 2^64) = floor((k w'_1 + floor(k w'_0 / 2^32)) / 2^32) with
// w' = w'_1 2^32 + w'_0, and that quotient is below k, so every partial
// product is 32 x 32 bits.  Bit-identical to shoup(k, w, ws, q).
__device__ __forceinline__ u64 shoup_small(uint32_t k, u64 w, u64 ws, u64 q) {
    const u64 qh = ((u64)k * (uint32_t)(ws >> 32) + __umulhi(k, (uint32_t)ws)) >> 32;
    return (u64)k * w - (u64)(uint32_t)qh * q;  // [0, 2q)
}
// The same product with a coarser quotient: h = a1 s1 + floor(a0 s1 / 2^32)
// + floor(a1 s0 / 2^32), two high-half multiplies instead of two wide ones.
// The three dropped fractions sum to below 3, so h is at most 2 below
// floor(a w' / 2^64) and the result lies in [0, 4q) for every 64-bit a.
__device__ __forceinline__ u64 shoup4(u64 a, u64 w, u64 ws, u64 nq) {
    u64 r;
    asm("{\n\t"
        ".reg .u32 a0, a1, s0, s1, w0, w1, n0, n1, t1, c, z, h0, h1, l0, l1;\n\t"
        ".reg .u64 x, h, l;\n\t"
        "mov.b64 {a0, a1}, %1;\n\t"
        "mov.b64 {w0, w1}, %2;\n\t"
        "mov.b64 {s0, s1}, %3;\n\t"
        "mov.b64 {n0, n1}, %4;\n\t"
        "mul.hi.u32 t1, a0, s1;\n\t"
        "mad.hi.cc.u32 c, a1, s0, t1;\n\t"
        "addc.u32 z, 0, 0;\n\t"
        "mov.b64 x, {c, z};\n\t"
        "mad.wide.u32 h, a1, s1, x;\n\t"
        "mov.b64 {h0, h1}, h;\n\t"
        "mul.wide.u32 l, a0, w0;\n\t"
        "mad.wide.u32 l, h0, n0, l;\n\t"
        "mul.lo.u32 c, a0, w1;\n\t"
        "mad.lo.u32 c, a1, w0, c;\n\t"
        "mad.lo.u32 c, h0, n1, c;\n\t"
        "mad.lo.u32 c, h1, n0, c;\n\t"
        "mov.b64 {l0, l1}, l;\n\t"
        "add.u32 l1, l1, c;\n\t"
        "mov.b64 %0, {l0, l1};\n\t"
        "}"
        : "=l"(r)
        : "l"(a), "l"(w), "l"(ws), "l"(nq));
    return r;
}
__device__ __forceinline__ u64 red1(u64 a, u64 q) { return a >= q ? a - q : a; }
__device__ __forceinline__ u64 addm(u64 a, u64 b, u64 q) { return red1(a + b, q); }   // a,b < q
__device__ __forceinline__ u64 subm(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }
// full product a*b mod q for a,b < q via the 128-bit value
__device__ __forceinline__ void mul128(u64 a, u64 b, u64 &lo, u64 &hi) {
    lo = a * b;
    hi = __umul64hi(a, b);
}
// (hi 2^64 + lo) mod q, fully reduced, any hi, lo < 2^64
__device__ __forceinline__ u64 reduce128(u64 lo, u64 hi, const ModDev &M) {
    u64 a = shoup(hi, M.r64, M.r64s, M.q);   // hi * 2^64 mod q, [0, 2q)
    u64 b = shoup(lo, 1, M.one_s, M.q);      // lo mod q, [0, 2q)
    u64 r = a + b;                           // [0, 4q)
    r = r >= M.twoq ? r - M.twoq : r;
    return red1(r, M.q);
}
// Montgomery reduction (P. L. Montgomery, Math. Comp. 44 (1985)) of
// T = hi 2^64 + lo < q 2^64: returns T 2^-64 mod q, fully reduced.  With
// m = lo q^-1 mod 2^64 the low word of m q equals lo, so T - m q =
// (hi - mulhi(m, q)) 2^64 exactly, and hi - mulhi(m, q) lies in (-q, q).
__device__ __forceinline__ u64 redc(u64 lo, u64 hi, const ModDev &M) {
    const u64 mh = __umul64hi(lo * M.qinv, M.q);
    return hi >= mh ? hi - mh : hi - mh + M.q;
}
// x mod q for x < 64 q, fully reduced, from a single-precision quotient
// estimate: every rounding is toward zero and qf <= 2^qsh / q, so the
// estimate never exceeds floor(x / q); its relative error (< 2^-21) and the
// dropped low bits (< 2^qsh, at most 2^-25 q) keep it at least floor(x/q) - 1
// below 64, so one conditional subtraction finishes.  The conversions run on
// the conversion unit, leaving the integer multiply pipe two multiplies.
__device__ __forceinline__ u64 reduce_small(u64 x, const ModDev &M) {
    const uint32_t xh = (uint32_t)(x >> M.qsh);
    const uint32_t k = __float2uint_rz(__fmul_rz(__uint2float_rz(xh), M.qf));
    return red1(x - (u64)k * M.q, M.q);
}
// a (< 2^64) mod q given r64-style constants, fully reduced
__device__ __forceinline__ u64 reduce64(u64 a, u64 q, u64 one_s) { return red1(shoup(a, 1, one_s, q), q); }

// ---------------------------------------------------------------- multi-word
// Little-endian arrays of 64-bit words, compile-time capacity MW, runtime
// used length W <= MW.  Loops are unrolled to MW with guards so the arrays
// stay in registers.

// X = sum_i y_i hat_i then reduced into [0, M); returns the number of M
// subtracted (the CRT overflow count v).
template <int MW, int NM>
__device__ __forceinline__ int crt_compose(const CrtDev &B, const u64 (&y)[NM], u64 (&X)[MW]) {
#pragma unroll
    for (int k = 0; k < MW; k++) X[k] = 0;
#pragma unroll
    for (int i = 0; i < NM; i++) {
        if (i >= B.n) break;
        u64 carry = 0;
#pragma unroll
        for (int k = 0; k < MW; k++) {
            if (k < B.Wh) {  // words of hat_i
                u64 lo, hi;
                mul128(y[i], B.hat[i][k], lo, hi);
                u64 s = X[k] + lo;
                hi += (s < lo);
                s += carry;
                hi += (s < carry);
                X[k] = s;
                carry = hi;
            } else if (k < B.W) {  // carry into the words above
                const u64 s = X[k] + carry;
                carry = s < carry;
                X[k] = s;
            }
        }
    }
    int v = 0;
    for (int it = 0; it < B.n; it++) {
        // X >= M ?
        bool ge = true, decided = false;
#pragma unroll
        for (int k = MW - 1; k >= 0; k--) {
            if (k < B.W && !decided && X[k] != B.M[k]) { ge = X[k] > B.M[k]; decided = true; }
        }
        if (!ge) break;
        u64 br = 0;
#pragma unroll
        for (int k = 0; k < MW; k++) {
            if (k < B.W) {
                u64 d = X[k] - B.M[k];
                u64 b1 = X[k] < B.M[k];
                u64 d2 = d - br;
                u64 b2 = d < br;
                X[k] = d2;
                br = b1 | b2;
            }
        }
        v++;
    }
    return v;
}

// residues r_i (< m_i) -> y_i = r_i * inv_i mod m_i
__device__ __forceinline__ u64 crt_y(const CrtDev &B, int i, u64 r) {
    return red1(shoup(r, B.inv[i], B.invs[i], B.m[i]), B.m[i]);
}

template <int MW>
__device__ __forceinline__ bool mw_greater(const u64 (&X)[MW], const u64 *Y, int W) {
    bool gt = false, decided = false;
#pragma unroll
    for (int k = MW - 1; k >= 0; k--) {
        if (k < W && !decided && X[k] != Y[k]) { gt = X[k] > Y[k]; decided = true; }
    }
    return gt;
}

// X mod p by Horner over 64-bit words: r <- r 2^64 + w
template <int MW>
__device__ __forceinline__ u64 mw_mod(const u64 (&X)[MW], int W, u64 p, u64 r64, u64 r64s, u64 one_s) {
    u64 r = 0;
#pragma unroll
    for (int k = MW - 1; k >= 0; k--) {
        if (k < W) {
            u64 a = shoup(r, r64, r64s, p);        // r 2^64 mod p, [0, 2p)
            u64 b = shoup(X[k], 1, one_s, p);      // [0, 2p)
            u64 s = a + b;                         // [0, 4p)
            s = s >= 2 * p ? s - 2 * p : s;
            r = red1(s, p);
        }
    }
    return r;
}

// ---------------------------------------------------------------- fast exact base conversion
// Overflow count v = floor(sum_i y_i / m_i) of a CRT sum from a 58-bit
// fixed-point estimate S (an underestimate of the true sum by < 1.07 n ulps).
// Returns false when S's fraction is within 64 ulps of the next integer, the
// only case in which the estimate could be off; callers then take the exact
// multi-word path.
template <int NM>
__device__ __forceinline__ bool crt_overflow(const ConvDev &C, const u64 (&y)[NM], int n, int &v, u64 &frac) {
    u64 S = 0;
#pragma unroll
    for (int i = 0; i < NM; i++)
        if (i < n) S += __umul64hi(y[i] << C.sh[i], C.c[i]) >> 5;
    v = (int)(S >> 58);
    frac = S & ((1ull << 58) - 1);
    return frac <= (1ull << 58) - 64;
}
// the centring decision X > M/2 is certain when the fraction is not within 64
// ulps below one half
__device__ __forceinline__ bool half_certain(u64 frac) {
    const u64 half = 1ull << 57;
    return frac >= half || frac + 64 <= half;
}
// (sum_i y_i h_i - k M) mod p, fully reduced; h, hs: constants (M/m_i) mod p
template <int NM>
__device__ __forceinline__ u64 conv_to(const u64 (&y)[NM], int n, const u64 *h, const u64 *hs, u64 k, u64 Mp, u64 Mps,
                                       u64 p) {
    u64 acc = 0;
    const u64 p2 = 2 * p;
#pragma unroll
    for (int i = 0; i < NM; i++)
        if (i < n) {
            acc += shoup(y[i], h[i], hs[i], p);
            acc = acc >= p2 ? acc - p2 : acc;
        }
    acc = red1(acc, p);
    return subm(acc, red1(shoup_small((uint32_t)k, Mp, Mps, p), p), p);
}

// The same conversion with the constants in Montgomery form (hm_i = h_i 2^64
// mod p): products summed in 128 bits, eight at a time (every y_i < 2^61 and
// hm_i < p, so eight products stay below 2^64 p), each sum ended by one
// Montgomery reduction, which removes the 2^64 again.  P is p's table entry.
template <int NM>
__device__ __forceinline__ u64 conv_to_m(const u64 (&y)[NM], int n, const u64 *hm, u64 k, u64 Mp, u64 Mps,
                                         const ModDev &P) {
    const u64 p = P.q;
    u64 acc = 0;
#pragma unroll
    for (int c0 = 0; c0 < NM; c0 += 8) {
        u64 lo = 0, hi = 0;
#pragma unroll
        for (int i = c0; i < c0 + 8 && i < NM; i++)
            if (i < n) {
                u64 pl, ph;
                mul128(y[i], hm[i], pl, ph);
                lo += pl;
                hi += ph + (lo < pl);
            }
        acc = addm(acc, redc(lo, hi, P), p);
    }
    return subm(acc, red1(shoup_small((uint32_t)k, Mp, Mps, p), p), p);
}

// ---------------------------------------------------------------- ChaCha20
// Block function of RFC 8439 (section 2.3): 20 rounds over the 4x4 state of
// constants, 256-bit key, 32-bit counter and 96-bit nonce, then the input
// state added back.
__device__ __forceinline__ uint32_t rotl(uint32_t x, int r) { return __funnelshift_l(x, x, r); }
#define HE_QR(a, b, c, d)                                        \
    a += b; d ^= a; d = rotl(d, 16); c += d; b ^= c; b = rotl(b, 12); \
    a += b; d ^= a; d = rotl(d, 8);  c += d; b ^= c; b = rotl(b, 7);

// Stream of 64-bit words of (seed, tag, idx, limb): key = (seed lo, seed hi,
// 0 x 6), nonce = (tag, idx, limb), block counter = word / 8; word w is state
// words 2(w%8) (low half) and 2(w%8)+1 (high half).
__device__ __forceinline__ void chacha_block8(uint64_t seed, uint32_t tag, uint32_t idx, uint32_t limb,
                                              uint32_t counter, u64 (&out)[8]) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint32_t x0 = 0x61707865u, x1 = 0x3320646eu, x2 = 0x79622d32u, x3 = 0x6b206574u;
    uint32_t x4 = k0, x5 = k1, x6 = 0, x7 = 0, x8 = 0, x9 = 0, x10 = 0, x11 = 0;
    uint32_t x12 = counter, x13 = tag, x14 = idx, x15 = limb;
#pragma unroll
    for (int i = 0; i < 10; i++) {
        HE_QR(x0, x4, x8, x12) HE_QR(x1, x5, x9, x13) HE_QR(x2, x6, x10, x14) HE_QR(x3, x7, x11, x15)
        HE_QR(x0, x5, x10, x15) HE_QR(x1, x6, x11, x12) HE_QR(x2, x7, x8, x13) HE_QR(x3, x4, x9, x14)
    }
    x0 += 0x61707865u; x1 += 0x3320646eu; x2 += 0x79622d32u; x3 += 0x6b206574u;
    x4 += k0; x5 += k1;
    x12 += counter; x13 += tag; x14 += idx; x15 += limb;
    out[0] = (u64)x0 | ((u64)x1 << 32);
    out[1] = (u64)x2 | ((u64)x3 << 32);
    out[2] = (u64)x4 | ((u64)x5 << 32);
    out[3] = (u64)x6 | ((u64)x7 << 32);
    out[4] = (u64)x8 | ((u64)x9 << 32);
    out[5] = (u64)x10 | ((u64)x11 << 32);
    out[6] = (u64)x12 | ((u64)x13 << 32);
    out[7] = (u64)x14 | ((u64)x15 << 32);
}
#undef HE_QR

}  // namespace he
