"""Pins of the oracle's ring layer: primes, the negacyclic product, ChaCha20
and the samplers (no GPU)."""
import numpy as np
import pytest
import sympy

from oracle import he
from tests.bruteforce import negacyclic_mod
from tests.conftest import read_golden


@pytest.mark.parametrize("N,bits", [(4096, 36), (8192, 50), (16384, 60), (64, 30)])
def test_gen_primes_are_largest(N, bits):
    ps = he.gen_primes(N, [bits] * 3)
    assert ps == sorted(ps, reverse=True)
    for p in ps:
        assert sympy.isprime(p) and p % (2 * N) == 1 and p < 2 ** bits
    # nothing skipped: every candidate = 1 mod 2N between ps[-1] and 2^bits is one of ps or composite
    c = ((2 ** bits - 2) // (2 * N)) * (2 * N) + 1
    while c >= ps[-1]:
        assert (c in ps) == sympy.isprime(c)
        c -= 2 * N


def test_primes_of_the_workload_rings():
    # the 3 x 36-bit and 4 x 50-bit moduli used by the synthetic layers
    assert he.gen_primes(4096, [36] * 3) == [68719403009, 68719230977, 68719206401]
    assert he.gen_primes(8192, [50] * 4) == [1125899906826241, 1125899906629633,
                                             1125899905744897, 1125899905351681]


def test_is_prime_matches_sympy():
    rng = np.random.default_rng(1)
    for n in list(rng.integers(2, 2 ** 62, size=300, dtype=np.int64)) + [2, 3, 4, 561, 2 ** 61 - 1, 3215031751]:
        assert he.is_prime(int(n)) == sympy.isprime(int(n))


@pytest.mark.parametrize("N", [8, 16, 32, 64])
@pytest.mark.parametrize("bits", [20, 36, 50, 60])
def test_polymul_equals_schoolbook(N, bits):
    q = he.gen_primes(N, [bits])[0]
    rng = np.random.default_rng(N * bits)
    for _ in range(3):
        a = rng.integers(0, q, N, dtype=np.uint64)
        b = rng.integers(0, q, N, dtype=np.uint64)
        got = he.polymul(a, b, q)
        assert [int(v) for v in got] == negacyclic_mod(a, b, q)


def test_polymul_monomial_is_negacyclic_shift():
    # x^k * b = (-b[N-k..N-1], b[0..N-k-1]) shifted: closed form of the ring
    N, q = 256, he.gen_primes(256, [50])[0]
    rng = np.random.default_rng(3)
    b = rng.integers(0, q, N, dtype=np.uint64)
    for k in (0, 1, 77, 255):
        a = np.zeros(N, dtype=np.uint64)
        a[k] = 1
        got = [int(v) for v in he.polymul(a, b, q)]
        want = [0] * N
        for j in range(N):
            if j + k < N:
                want[j + k] = int(b[j])
            else:
                want[j + k - N] = (q - int(b[j])) % q
        assert got == want


def test_polymul_large_N_inverse_identity():
    # (a * x^N-... ) use the unit x: x^(2N) = 1 so x^k * x^(2N-k) = 1
    N, q = 8192, he.gen_primes(8192, [50])[0]
    a = np.zeros(N, dtype=np.uint64)
    b = np.zeros(N, dtype=np.uint64)
    a[5] = 1
    b[N - 5] = q - 1          # -x^(N-5), and x^5 * (-x^(N-5)) = -x^N = 1
    got = he.polymul(a, b, q)
    want = np.zeros(N, dtype=np.uint64)
    want[0] = 1
    assert np.array_equal(got, want)


def test_chacha20_rfc8439_vector():
    g = read_golden("chacha20_rfc8439_2_3_2.txt")
    kb = bytes.fromhex(g["key"][0])
    nb = bytes.fromhex(g["nonce"][0])
    key = [int.from_bytes(kb[4 * i:4 * i + 4], "little") for i in range(8)]
    nonce = [int.from_bytes(nb[4 * i:4 * i + 4], "little") for i in range(3)]
    out = he.chacha20_block(key, int(g["counter"][0]), nonce)
    assert out.tobytes().hex() == g["block"][0]


def test_stream_word_layout():
    # word w = block (w // 8), 32-bit state words 2(w%8) (low) and 2(w%8)+1 (high)
    seed = 0x123456789ABCDEF
    words = he.stream_words(seed, 4, 7, 2, 0, 24)
    key = [seed & 0xFFFFFFFF, seed >> 32, 0, 0, 0, 0, 0, 0]
    for blk in range(3):
        st = he.chacha20_block(key, blk, [4, 7, 2])
        for j in range(8):
            assert int(words[8 * blk + j]) == int(st[2 * j]) | (int(st[2 * j + 1]) << 32)
    assert np.array_equal(he.stream_words(seed, 4, 7, 2, 5, 10), words[5:15])


def test_samplers_distribution():
    N = 1 << 16
    tern = he.sample_ternary(11, 1, 0, N)
    assert set(np.unique(tern)) <= {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs(np.mean(tern == v) - 1 / 3) < 0.01
    e = he.sample_cbd(11, 3, 0, 21, N)
    assert e.min() >= -21 and e.max() <= 21
    assert abs(e.mean()) < 0.05 and abs(e.var() - 10.5) < 0.3   # CBD(21): variance eta/2
    q = 1125899906826241
    u = he.sample_uniform(11, 2, 0, 1, q, N)
    assert int(u.max()) < q and abs(u.astype(np.float64).mean() / q - 0.5) < 0.01
    w = he.stream_words(11, 2, 0, 1, 0, 4)
    assert int(u[0]) == ((int(w[1]) << 64) | int(w[0])) % q
    assert int(u[1]) == ((int(w[3]) << 64) | int(w[2])) % q


def test_samplers_follow_the_stream_convention():
    """Each sample is the written function of its stream word (limb field 0
    for the small samplers): ternary floor(3 w / 2^64) - 1; CBD(eta)
    popcount of the low eta bits minus popcount of the next eta bits;
    uniform mod t: w mod t; uniform mod q: (w_{2k+1} 2^64 + w_{2k}) mod q."""
    N = 64
    w = [int(v) for v in he.stream_words(5, 4, 9, 0, 0, N)]
    assert [int(v) for v in he.sample_ternary(5, 4, 9, N)] == [(3 * x >> 64) - 1 for x in w]
    for eta in (3, 21):
        m = (1 << eta) - 1
        want = [bin(x & m).count("1") - bin((x >> eta) & m).count("1") for x in w]
        assert [int(v) for v in he.sample_cbd(5, 4, 9, eta, N)] == want
    t = 1032193
    got = np.zeros(N, dtype=np.uint64)
    he._clib.lib().orc_sample_uniform_t(5, 4, 9, t, N, he._u64(got))
    assert [int(v) for v in got] == [x % t for x in w]
    q = 1125899906826241
    w2 = [int(v) for v in he.stream_words(5, 4, 9, 3, 0, 2 * N)]
    assert [int(v) for v in he.sample_uniform(5, 4, 9, 3, q, N)] == [
        ((w2[2 * k + 1] << 64) | w2[2 * k]) % q for k in range(N)]
