"""The output ranges that the device arithmetic's comments claim, checked on
the host with exact integers: the two Shoup products of the NTT butterflies
(finer quotient: [0, 3q); coarser: [0, 4q)), the 32-bit form of the Shoup
product for small multipliers (the same quotient as the 64-bit one), and the
Montgomery reduction that ends the multiply-accumulate together with its
fold interval.  Each model follows the 32-bit partial products of the
corresponding inline-PTX or C routine step by step; the assertions are the
ranges and congruences that the lazy-butterfly growth bounds rely on."""
import random

import pytest

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1


def primes_near(bits, count, rng):
    from oracle import he
    out = []
    for b in bits:
        out += he.gen_primes(1 << 10, [b])[:1]
    while len(out) < count:
        out.append(out[rng.randrange(len(out))])
    return out


def split(x):
    return x & M32, x >> 32


def shoup_w(w, q):
    return (w << 64) // q


def shoup_fine(a, w, ws, q):
    """h = a1 s1 + floor((a0 s1 + a1 s0 + ...) / 2^32) as the forward
    butterfly forms it: a0 s1 (wide), its low half added to a1 s0 (wide), the
    high halves summed with carry, then a1 s1 (wide) plus that sum."""
    a0, a1 = split(a)
    s0, s1 = split(ws)
    t = a0 * s1
    u = a1 * s0 + (t & M32)
    c = (u >> 32) + (t >> 32)
    h = a1 * s1 + c
    return (a * w + h * ((1 << 64) - q)) & M64


def shoup_coarse(a, w, ws, q):
    """h = a1 s1 + floor(a0 s1 / 2^32) + floor(a1 s0 / 2^32)."""
    a0, a1 = split(a)
    s0, s1 = split(ws)
    h = a1 * s1 + ((a0 * s1) >> 32) + ((a1 * s0) >> 32)
    return (a * w + h * ((1 << 64) - q)) & M64


def cases(rng, q, n=400):
    yield M64, q - 1
    yield M64, 1
    yield 0, q - 1
    # the largest butterfly input: 57q - 1 under the lazy bound (q < 2^57),
    # else 8q - 1
    yield (57 * q - 1 if q < (1 << 57) else 8 * q - 1), q - 1
    for _ in range(n):
        yield rng.randrange(1 << 64), rng.randrange(q)


@pytest.mark.parametrize("bits", [20, 36, 50, 57, 60, 61])
def test_butterfly_products(bits):
    rng = random.Random(bits)
    q = primes_near([bits], 1, rng)[0]
    for a, w in cases(rng, q):
        ws = shoup_w(w, q)
        r3 = shoup_fine(a, w, ws, q)
        r4 = shoup_coarse(a, w, ws, q)
        assert r3 % q == a * w % q and r3 < 3 * q
        assert r4 % q == a * w % q and r4 < 4 * q


@pytest.mark.parametrize("bits", [20, 50, 61])
def test_small_multiplier_quotient(bits):
    """The quotient of the overflow-count product equals the 64-bit one."""
    rng = random.Random(100 + bits)
    p = primes_near([bits], 1, rng)[0]
    for _ in range(500):
        k = rng.randrange(1 << 32) if rng.random() < 0.5 else rng.randrange(64)
        w = rng.randrange(p)
        ws = shoup_w(w, p)
        qh = (k * (ws >> 32) + ((k * (ws & M32)) >> 32)) >> 32
        assert qh == (k * ws) >> 64 and qh < (1 << 32)
        r = (k * w - qh * p) & M64
        assert r % p == k * w % p and r < 2 * p


def redc(lo, hi, q, qinv):
    mh = (((lo * qinv) & M64) * q) >> 64
    return hi - mh if hi >= mh else hi - mh + q


@pytest.mark.parametrize("bits", [20, 36, 50, 57, 60, 61])
def test_montgomery_end_of_the_sum(bits):
    """With the fold interval f = min(15, floor((2^64-1)/q) + 1), a sum of
    at most f-1 products of residues after a fold (value below q) stays below
    q 2^64, and the reduction returns T 2^-64 mod q, fully reduced."""
    rng = random.Random(200 + bits)
    q = primes_near([bits], 1, rng)[0]
    qinv = pow(q, -1, 1 << 64)
    fold = min(15, M64 // q + 1)
    assert (fold - 1) * q + 1 <= (1 << 64)
    rinv = pow(1 << 64, -1, q)
    worst = (q - 1) + (fold - 1) * (q - 1) ** 2
    assert worst < q << 64
    for _ in range(300):
        terms = rng.randrange(fold)
        T = rng.randrange(q) + sum(rng.randrange(q) * rng.randrange(q) for _ in range(terms))
        if rng.random() < 0.1:
            T = worst
        r = redc(T & M64, T >> 64, q, qinv)
        assert 0 <= r < q and r == T * rinv % q


def test_montgomery_conversion_chunk():
    """Eight products y_i hm_i with y_i < 2^61 and hm_i < p stay below 2^64 p,
    the precondition of the conversion's Montgomery reduction."""
    for p in (1 << 20, (1 << 50) - 27, (1 << 61) - 1):
        assert 8 * ((1 << 61) - 1) * (p - 1) < (1 << 64) * p


@pytest.mark.parametrize("bits", [20, 36, 50, 60, 61])
def test_crt_overflow_estimate(bits):
    """The overflow-count estimate: with m' = m << sh in [2^63, 2^64) and
    c = floor(2^127 / m'), each term floor(floor((y << sh) c / 2^64) / 2^5)
    is below y / m * 2^58 by less than 1.07 (so n terms by < 1.07 n < 64
    ulps: the fallback window)."""
    from fractions import Fraction
    rng = random.Random(300 + bits)
    m = primes_near([bits], 1, rng)[0]
    sh = 64 - m.bit_length()
    mp = m << sh
    assert (1 << 63) <= mp < (1 << 64)
    c = (1 << 127) // mp
    for y in [0, 1, m - 1, m // 2, m // 2 + 1] + [rng.randrange(m) for _ in range(500)]:
        term = (((y << sh) * c) >> 64) >> 5
        err = Fraction(y, m) * (1 << 58) - term
        assert 0 <= err < Fraction(107, 100)


# ---------------------------------------------------------------- single-precision quotient
def f32_round_down_constant(qsh, q):
    """qf as the context builds it: 2^qsh / q in double precision, converted
    to single precision (round to nearest), then stepped down while it is not
    below that double by a relative margin of 1e-12."""
    import math

    import numpy as np
    d = math.ldexp(1.0, qsh) / float(q)
    f = np.float32(d)
    while float(f) > d * (1.0 - 1e-12):
        f = np.nextafter(f, np.float32(0.0))
    return f


def rz24(v):
    """A non-negative rational rounded toward zero to 24 significant bits
    (single precision, no overflow or subnormals in this range)."""
    from fractions import Fraction
    if v == 0:
        return Fraction(0)
    e = v.numerator.bit_length() - v.denominator.bit_length()
    # 2^e <= v < 2^(e+2): find e with 2^23 <= v / 2^(e-23) < 2^24
    while Fraction(2) ** e > v:
        e -= 1
    while Fraction(2) ** (e + 1) <= v:
        e += 1
    scale = Fraction(2) ** (e - 23)
    return Fraction(int(v / scale)) * scale


def reduce_small_model(x, q, qsh, qf):
    """The device routine step by step: xh = x >> qsh (32 bits), k =
    float2uint_rz(fmul_rz(uint2float_rz(xh), qf)); returns x - k q before
    its one conditional subtraction."""
    from fractions import Fraction
    xh = x >> qsh
    assert xh < (1 << 32)
    a = rz24(Fraction(xh))                         # __uint2float_rz
    p = rz24(a * Fraction(float(qf)))              # __fmul_rz (qf is exact in a double)
    k = int(p)                                     # __float2uint_rz
    return x - k * q


def reduce_small_moduli(rng):
    """Every modulus size the forward transform reduces against: plaintext
    moduli from 17 bits (t = 65537) and RNS / auxiliary primes up to 61 bits,
    at both ends of each bit length, plus the primes the library generates."""
    from oracle import he
    qs = {65537, 1032193}
    for b in range(17, 63):
        qs.add((1 << (b - 1)) + 1)
        qs.add((1 << b) - 1)
        qs.add(rng.randrange(1 << (b - 1), 1 << b) | 1)
    for N in (1024, 8192, 16384):
        for b in (36, 40, 50, 60, 61):
            qs.update(he.gen_primes(N, [b]))
    return sorted(qs)


def test_single_precision_quotient_of_the_final_reduction():
    """The forward transform's final reduction of x < 64 q takes its quotient
    from a round-toward-zero single-precision estimate: it never exceeds
    floor(x / q) and is at most one below, so x - k q lies in [0, 2q) and one
    conditional subtraction finishes.  Checked on the boundaries k q - 1,
    k q and k q + q - 1 for every k < 64, the largest x, and random x, for
    moduli of every bit length from 17 to 62."""
    rng = random.Random(4242)
    for q in reduce_small_moduli(rng):
        bq = q.bit_length()
        qsh = bq + 6 - 32 if bq + 6 > 32 else 0
        qf = f32_round_down_constant(qsh, q)
        xs = {64 * q - 1}
        for k in range(64):
            xs.update({k * q, k * q + q - 1})
            if k:
                xs.add(k * q - 1)
        xs.update(rng.randrange(64 * q) for _ in range(40))
        for x in xs:
            r = reduce_small_model(x, q, qsh, qf)
            assert 0 <= r < 2 * q, (q, x, r)
