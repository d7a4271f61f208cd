"""Pins of the oracle's BFV layer against homomorphic identities, key
relations and big-integer brute force on tiny rings (no GPU)."""
import numpy as np
import pytest

from oracle import he
from tests.bruteforce import centred, crt, negacyclic_int, negacyclic_mod, round_tq


def small_params(N=16, bits=(50, 50, 50, 50), t=65537):
    return he.Params(N, he.gen_primes(N, list(bits)), t)


def rns_to_int(P, poly):
    """[L][N] residues -> list of N integers in [0, q)."""
    return [crt([int(poly[i][k]) for i in range(P.L)], P.q) for k in range(P.N)]


def test_keygen_relations():
    P = small_params(32)
    K = he.keygen(P, 5, True)
    s = [int(v) for v in K.sk]
    assert set(s) <= {-1, 0, 1}
    Q = P.Q
    b, a = rns_to_int(P, K.pk[0]), rns_to_int(P, K.pk[1])
    # b + a s = -e, e a small CBD error
    e = [centred((bb + v) % Q, Q) for bb, v in zip(b, negacyclic_int(a, s))]
    assert max(abs(v) for v in e) <= 21 and any(e)
    s2 = negacyclic_int(s, s)
    for j in range(P.ell):
        r0, r1 = rns_to_int(P, K.rlk[j][0]), rns_to_int(P, K.rlk[j][1])
        # rlk_j0 + rlk_j1 s - 2^(16 j) s^2 = -e_j
        ej = [centred((x + y - (1 << (16 * j)) * z) % Q, Q) for x, y, z in zip(r0, negacyclic_int(r1, s), s2)]
        assert max(abs(v) for v in ej) <= 21


def test_keys_equal_their_definition_from_the_streams():
    """Every key polynomial equals its definition (Section 2, HE; Fig. 3(b)
    for rlk), evaluated with schoolbook products on the samples the stream
    convention names: s = ternary(seed, sk, 0); a_i = uniform(seed, pk_a, 0,
    limb i); e = CBD(seed, pk_e, 0); b = -(a s + e).  rlk_j: a_j from
    (seed, rlk_a, j, limb), e_j from (seed, rlk_e, j), r0 = -(a_j s + e_j) +
    2^(16 j) s^2."""
    P = small_params(16, (40, 41, 42), 65537)
    seed = 31
    K = he.keygen(P, seed, True)
    N = P.N
    s = he.sample_ternary(seed, he.TAG_SK, 0, N)
    assert [int(v) for v in K.sk] == [int(v) for v in s]
    e = he.sample_cbd(seed, he.TAG_PK_E, 0, P.eta, N)
    for i, qi in enumerate(P.q):
        a = he.sample_uniform(seed, he.TAG_PK_A, 0, i, qi, N)
        assert [int(v) for v in K.pk[1, i]] == [int(v) for v in a]
        as_ = negacyclic_int([int(v) for v in a], [int(v) for v in s])
        assert [int(v) for v in K.pk[0, i]] == [(-(x + int(y))) % qi for x, y in zip(as_, e)]
    s2 = negacyclic_int([int(v) for v in s], [int(v) for v in s])
    for j in range(P.ell):
        ej = he.sample_cbd(seed, he.TAG_RLK_E, j, P.eta, N)
        for i, qi in enumerate(P.q):
            aj = he.sample_uniform(seed, he.TAG_RLK_A, j, i, qi, N)
            assert [int(v) for v in K.rlk[j, 1, i]] == [int(v) for v in aj]
            ajs = negacyclic_int([int(v) for v in aj], [int(v) for v in s])
            want = [(-(x + int(y)) + (1 << (P.base_log2 * j)) * z) % qi for x, y, z in zip(ajs, ej, s2)]
            assert [int(v) for v in K.rlk[j, 0, i]] == want


def test_encryption_equals_its_definition_from_the_streams():
    """ct = (b u + e1 + Delta m, a u + e2) bit for bit, with Delta =
    floor(Q/t), u = ternary(seed, enc_u, k), e1 = CBD(seed, enc_e1, k), e2 =
    CBD(seed, enc_e2, k) for ciphertext k (first + position), by schoolbook
    products: a dropped or swapped term, a wrong sign or a wrong Delta fails."""
    P = small_params(16, (36, 37, 38), 65537)
    K = he.keygen(P, 8, False)
    N, t = P.N, P.t
    delta = P.Q // t
    rng = np.random.default_rng(4)
    m = rng.integers(0, t, (2, N), dtype=np.uint64)
    seed, first = 55, 3
    ct = he.encrypt(P, K, m, seed, first)
    for k in range(2):
        idx = first + k
        u = [int(v) for v in he.sample_ternary(seed, he.TAG_ENC_U, idx, N)]
        e1 = he.sample_cbd(seed, he.TAG_ENC_E1, idx, P.eta, N)
        e2 = he.sample_cbd(seed, he.TAG_ENC_E2, idx, P.eta, N)
        for i, qi in enumerate(P.q):
            bu = negacyclic_int([int(v) for v in K.pk[0, i]], u)
            au = negacyclic_int([int(v) for v in K.pk[1, i]], u)
            want0 = [(x + int(y) + delta * int(mm)) % qi for x, y, mm in zip(bu, e1, m[k])]
            want1 = [(x + int(y)) % qi for x, y in zip(au, e2)]
            assert [int(v) for v in ct[k, 0, i]] == want0
            assert [int(v) for v in ct[k, 1, i]] == want1


@pytest.mark.parametrize("N,bits,t", [(16, (36, 36, 36), 65537), (64, (50,) * 4, 1032193), (4096, (36,) * 3, 65537)])
def test_encrypt_decrypt_roundtrip(N, bits, t):
    P = he.Params(N, he.gen_primes(N, list(bits)), t)
    K = he.keygen(P, 9, False)
    rng = np.random.default_rng(N)
    m = rng.integers(0, t, (3, N), dtype=np.uint64)
    ct = he.encrypt(P, K, m, 77)
    assert np.array_equal(he.decrypt(P, K, ct), m)
    # fresh noise |e1 + e u + e2 s| is far below Delta/2
    assert he.noise_bits(P, K, ct[0], m[0]) < 20


def test_decrypt_rounding_boundaries():
    # ct = (x, 0) decrypts to floor((t x + floor(q/2)) / q) mod t
    P = small_params(16, (36, 36, 36), 65537)
    K = he.keygen(P, 1, False)
    Q, t = P.Q, P.t
    xs = [0, 1, Q - 1, Q // 2, Q // 2 + 1, Q // (2 * t), Q // (2 * t) + 1, (Q // t) * 5 + Q // (2 * t)]
    for x in xs:
        ct = np.zeros((2, P.L, P.N), dtype=np.uint64)
        for i, qi in enumerate(P.q):
            ct[0, i, 3] = x % qi
        m = he.decrypt(P, K, ct)[0]
        assert int(m[3]) == ((t * x + Q // 2) // Q) % t
        assert int(m[0]) == 0


def test_cpmul_ccadd_identity():
    P = small_params(64, (50,) * 4, 1032193)
    K = he.keygen(P, 3, False)
    rng = np.random.default_rng(4)
    t = P.t
    m = rng.integers(0, t, (3, P.N), dtype=np.uint64)
    pt = rng.integers(0, t, (2, P.N), dtype=np.uint64)
    ct = he.encrypt(P, K, m, 8)
    # out0 = ct0 * pt0 + ct1 * pt1 ; out1 = ct2 * pt0 + add(=ct0)
    out = he.cpmul_terms(P, ct, pt, [[(0, 0), (1, 1)], [(2, 0)]],
                         add=np.stack([np.zeros_like(ct[0]), ct[0]]))
    dec = he.decrypt(P, K, out)
    want0 = [(x + y) % t for x, y in zip(negacyclic_mod(m[0], pt[0], t), negacyclic_mod(m[1], pt[1], t))]
    want1 = [(x + int(y)) % t for x, y in zip(negacyclic_mod(m[2], pt[0], t), m[0])]
    assert [int(v) for v in dec[0]] == want0
    assert [int(v) for v in dec[1]] == want1


def test_cpmul_centred_lift_of_plaintext():
    # pt = t-1 is the constant -1: ct * pt must decrypt to -m and the
    # ciphertext must equal the negation of ct (centred lift, not t-1)
    P = small_params(16, (36, 36, 36), 65537)
    K = he.keygen(P, 3, False)
    m = np.arange(16, dtype=np.uint64)
    ct = he.encrypt(P, K, m, 2)
    pt = np.zeros((1, 16), dtype=np.uint64)
    pt[0, 0] = P.t - 1
    out = he.cpmul_terms(P, ct, pt, [[(0, 0)]])
    for i, qi in enumerate(P.q):
        assert np.array_equal(out[0, :, i], (np.uint64(qi) - ct[0, :, i]) % np.uint64(qi))


def ccmul_bruteforce(P, K, a, b, group_pairs):
    """Exact CCMul of the definition with Python integers and schoolbook products."""
    Q, t = P.Q, P.t
    N, L = P.N, P.L
    d = [[0] * N for _ in range(3)]
    for (ca, cb) in group_pairs:
        a0 = [centred(v, Q) for v in rns_to_int(P, ca[0])]
        a1 = [centred(v, Q) for v in rns_to_int(P, ca[1])]
        b0 = [centred(v, Q) for v in rns_to_int(P, cb[0])]
        b1 = [centred(v, Q) for v in rns_to_int(P, cb[1])]
        for k, v in enumerate(negacyclic_int(a0, b0)):
            d[0][k] += v
        for k, (v, w) in enumerate(zip(negacyclic_int(a0, b1), negacyclic_int(a1, b0))):
            d[1][k] += v + w
        for k, v in enumerate(negacyclic_int(a1, b1)):
            d[2][k] += v
    r = [[round_tq(v, t, Q) % Q for v in dj] for dj in d]
    c0, c1 = r[0][:], r[1][:]
    B = 1 << P.base_log2
    for j in range(P.ell):
        dig = [(v >> (P.base_log2 * j)) % B for v in r[2]]
        k0 = rns_to_int(P, K.rlk[j][0])
        k1 = rns_to_int(P, K.rlk[j][1])
        for k, v in enumerate(negacyclic_int(dig, k0)):
            c0[k] = (c0[k] + v) % Q
        for k, v in enumerate(negacyclic_int(dig, k1)):
            c1[k] = (c1[k] + v) % Q
    out = np.zeros((2, L, N), dtype=np.uint64)
    for i, qi in enumerate(P.q):
        out[0, i] = [v % qi for v in c0]
        out[1, i] = [v % qi for v in c1]
    return out


@pytest.mark.parametrize("bits,t", [((36, 36, 36), 65537), ((50,) * 4, 1032193), ((60, 60), 17)])
def test_ccmul_bits_equal_bruteforce(bits, t):
    P = he.Params(8, he.gen_primes(8, list(bits)), t)
    K = he.keygen(P, 21, True)
    rng = np.random.default_rng(2)
    m = rng.integers(0, t, (4, 8), dtype=np.uint64)
    ct = he.encrypt(P, K, m, 5)
    got = he.ccmul(P, K, ct, ct, [(0, 1), (2, 3)], group=2)
    want = ccmul_bruteforce(P, K, ct, ct, [(ct[0], ct[1]), (ct[2], ct[3])])
    assert np.array_equal(got[0], want)
    got1 = he.ccmul(P, K, ct, ct, [(1, 3)], group=1)
    assert np.array_equal(got1[0], ccmul_bruteforce(P, K, ct, ct, [(ct[1], ct[3])]))


@pytest.mark.parametrize("bits,t", [((36, 36, 36), 65537), ((50,) * 4, 1032193), ((60, 60), 17)])
def test_ccmul_bits_equal_bruteforce_at_rounding_boundaries(bits, t):
    """CCMul of a = (1, 1) with b = (b0, b1) gives d0 = b0, d1 = b0 + b1,
    d2 = b1 exactly.  The coefficients of b are chosen where the rounding is
    delicate: within a few units of Q/2 (the centred lift), with
    [t d + floor(Q/2)]_Q within a few units of Q, and with the rounded
    quotient equal to -1 and 0.  The result equals the big-integer brute force."""
    P = he.Params(8, he.gen_primes(8, list(bits)), t)
    K = he.keygen(P, 23, True)
    Q = P.Q
    h = Q // 2
    tinv = pow(t, -1, Q)
    near_q = [((Q - 1 - j - h) * tinv) % Q for j in range(2)]
    neg_f = [(-((h + t - 1) // t) - j) % Q for j in (1, 2)]
    b0 = [h - 1, h, h + 1, h + 2] + near_q + neg_f[:2]
    b1 = neg_f[::-1] + [h + 1, h] + near_q[::-1] + [Q - 1, 0]
    for v in neg_f:
        vc = v if v <= h else v - Q
        assert (t * vc + h) // Q == -1
    one = np.zeros((P.L, 8), dtype=np.uint64)
    one[:, 0] = 1
    a = np.stack([one, one])[None]
    b = np.zeros((1, 2, P.L, 8), dtype=np.uint64)
    for i, qi in enumerate(P.q):
        b[0, 0, i] = [v % qi for v in b0[:8]]
        b[0, 1, i] = [v % qi for v in b1[:8]]
    got = he.ccmul(P, K, a, b, [(0, 0)], group=1)
    assert np.array_equal(got[0], ccmul_bruteforce(P, K, a, b, [(a[0], b[0])]))


@pytest.mark.parametrize("N,bits,t", [(64, (50,) * 4, 1032193), (1024, (36,) * 3, 65537)])
def test_ccmul_decrypts_to_product(N, bits, t):
    P = he.Params(N, he.gen_primes(N, list(bits)), t)
    K = he.keygen(P, 4, True)
    rng = np.random.default_rng(N + 1)
    m = rng.integers(0, t, (4, N), dtype=np.uint64)
    ct = he.encrypt(P, K, m, 6)
    out = he.ccmul(P, K, ct[:2], ct[2:], [(0, 0), (1, 1)], group=2)
    dec = he.decrypt(P, K, out)[0]
    want = [(x + y) % t for x, y in zip(negacyclic_mod(m[0], m[2], t), negacyclic_mod(m[1], m[3], t))]
    assert [int(v) for v in dec] == want


def test_round_scalar_against_floor_division():
    P = small_params(16, (50,) * 4, 1032193)
    Q, t = P.Q, P.t
    rng = np.random.default_rng(7)
    vals = [0, 1, -1, Q, -Q, Q // 2, -(Q // 2), Q * Q, -(Q * Q) + 12345]
    vals += [int(rng.integers(1, 2 ** 62)) * int(rng.integers(1, 2 ** 62)) * (1 if i % 2 else -1) * Q // 7
             for i in range(20)]
    for v in vals:
        want = round_tq(v, t, Q)
        assert he.round_scalar(P, v) == [want % qi for qi in P.q]


def test_ppmul_equals_schoolbook_mod_t():
    N = 64
    for t in (65537, 1032193, 1099511480321, 255):
        P = he.Params(N, he.gen_primes(N, [50]), t)
        rng = np.random.default_rng(t % 1000)
        a = rng.integers(0, t, (2, N), dtype=np.uint64)
        b = rng.integers(0, t, (2, N), dtype=np.uint64)
        got = he.ppmul_terms(P, a, b, [[(0, 0), (1, 1)]])[0]
        want = [(x + y) % t for x, y in zip(negacyclic_mod(a[0], b[0], t), negacyclic_mod(a[1], b[1], t))]
        assert [int(v) for v in got] == want
        # crossed indices: a transposed operand index fails
        got = he.ppmul_terms(P, a, b, [[(0, 1)], [(1, 0)]])
        assert [int(v) for v in got[0]] == negacyclic_mod(a[0], b[1], t)
        assert [int(v) for v in got[1]] == negacyclic_mod(a[1], b[0], t)


@pytest.mark.parametrize("N,bits,t", [(64, (40, 41), 257), (1024, (50, 50, 50), 65537)])
def test_symmetric_encryption_round_trip_and_compression(N, bits, t):
    """Seed-compressed secret-key encryption: the expanded ciphertext
    decrypts to the message with fresh-encryption noise, c1 is exactly the
    seeded uniform stream (so only c0 and the seed need to travel), and the
    noise c0 + c1 s - Delta m equals -e."""
    P = he.Params(N, he.gen_primes(N, list(bits)), t)
    keys = he.keygen(P, 5, False)
    m = np.random.default_rng(3).integers(0, t, (3, N), dtype=np.uint64)
    c0 = he.encrypt_symmetric(P, keys, m, seed=99)
    ct = he.expand_symmetric(P, 99, c0)
    assert c0.nbytes * 2 == ct.nbytes
    assert np.array_equal(he.decrypt(P, keys, ct), m)
    assert max(he.noise_bits(P, keys, ct[k], m[k]) for k in range(3)) <= 5   # |e| <= eta = 21
    for i, q in enumerate(P.q):
        assert np.array_equal(ct[1, 1, i], he.sample_uniform(99, he.TAG_SYM_A, 1, i, q, N))
    # exactly: c0 + c1 s - Delta m = -e, e the CBD samples of (seed, SYM_E, k)
    if N <= 64:
        Q, delta = P.Q, P.Q // t
        sk = [int(v) for v in keys.sk]
        for k in range(3):
            e = he.sample_cbd(99, he.TAG_SYM_E, k, P.eta, N)
            c0i = rns_to_int(P, ct[k, 0])
            c1s = negacyclic_int(rns_to_int(P, ct[k, 1]), sk)
            x = [centred((a + b - delta * int(mm)) % Q, Q) for a, b, mm in zip(c0i, c1s, m[k])]
            assert x == [-int(v) for v in e]
    # a sub-batch starting at `first` equals the same positions of the whole batch
    c0_sub = he.encrypt_symmetric(P, keys, m[1:], seed=99, first=1)
    assert np.array_equal(c0_sub, c0[1:])
    assert np.array_equal(he.expand_symmetric(P, 99, c0_sub, first=1), ct[1:])
    # a different seed gives a different ciphertext of the same message
    ct2 = he.expand_symmetric(P, 98, he.encrypt_symmetric(P, keys, m, seed=98))
    assert not np.array_equal(ct2, ct) and np.array_equal(he.decrypt(P, keys, ct2), m)
