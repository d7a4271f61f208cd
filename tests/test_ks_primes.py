"""The small primes of the relinearisation key switch (host only, no GPU).

The key switch adds E_i = sum_j D_j rlk_{j,i} (a product in Z[x]/(x^N + 1))
to each limb.  Its coefficients are integers with |E| <= ell N (2^base - 1)
(q_i - 1), and the library takes them modulo primes p < 2^30 and maps them
back with a CRT that is exact when P = prod p > 4 max|E| (the sign is read
from the top mixed-radix digit).  Random parity inputs almost never come near
that worst case, so the prime choice is pinned here on its own, against the
oracle's limb primes and the bound computed with Python integers:
  - each p is prime, p = 1 mod 2N, 2^29 < p < 2^30, none a limb or t;
  - P exceeds four times the bound, and the primes are the largest candidates;
  - no primes exactly when a limb is below 2^31;
  - four primes suffice at the largest supported bound (N = 16384, sixteen
    61-bit limbs, base 2^32).
"""
import pytest

from oracle import he
from paper_2409_16675_gb300 import native as nv

CASES = [  # (N, prime bits, t, base_log2, expected number of primes)
    (8192, (50, 50, 50, 50), 1032193, 16, 3),        # the layer ring
    (4096, (36, 36, 36), 65537, 16, 3),
    (1024, (40, 45), 65537, 16, 3),
    (2048, (50, 50, 50), 1099511480321, 16, 3),
    (16384, (60, 60, 55), 65537, 16, 4),
    (16384, (50, 50), 65537, 16, 3),
    (8192, (50, 50, 50, 50), 65537, 32, 4),
    (4096, (50, 50, 50, 50, 50), 65537, 16, 3),
    (4096, (30, 50, 50), 65537, 16, 0),              # a limb below 2^31
    (8192, (31, 40), 65537, 16, 0),
    (16384, (61,) * 16, 65537, 32, 4),               # the largest bound
    (1024, (61,) * 16, 65537, 1, 3),                 # 976 one-bit digits
    (1024, (32, 32), 65537, 8, 2),                   # two primes suffice
    (1024, (50,) * 9, 65537, 32, 4),
]


def bound(N, q, base):
    ell = -(-he.Params(N, q, 2).Q.bit_length() // base)
    return ell * N * (2 ** base - 1) * (max(q) - 1)


@pytest.mark.parametrize("N,bits,t,base,want", CASES)
def test_key_switch_primes(N, bits, t, base, want):
    q = he.gen_primes(N, list(bits))
    ps = nv.he_ks_primes(nv.make_params(N, prime_bits=bits, t=t, base_log2=base))
    assert len(ps) == want
    if min(q) < 2 ** 31:
        assert ps == []
        return
    assert 2 <= len(ps) <= 4 and len(set(ps)) == len(ps)
    for p in ps:
        assert he.is_prime(p) and p % (2 * N) == 1 and 2 ** 29 < p < 2 ** 30
        assert p not in q and p != t
    P = 1
    for p in ps:
        P *= p
    assert P > 4 * bound(N, q, base)
    # the largest candidates below 2^30, in descending order
    assert ps == sorted(ps, reverse=True)
    c = (2 ** 30 - 2) // (2 * N) * (2 * N) + 1
    while c > ps[-1]:
        if he.is_prime(c) and c not in q and c != t:
            assert c in ps
        c -= 2 * N
    # one prime fewer would leave at most one bit of margin to spare
    if len(ps) > 2:
        assert P // ps[-1] < 2 * 2 ** (4 * bound(N, q, base)).bit_length()


def test_exactness_condition_is_tight_enough_to_matter():
    """The CRT reads the sign of E from the top digit: with P > 4|E| a
    non-negative E gives a top digit below p/4 + 1 and a negative one a top
    digit of at least 3p/4 - 1, so the threshold p/2 separates them.  Checked
    here on the extreme values of the layer ring's bound with Python integers
    (mixed-radix digits of E mod P)."""
    N, bits = 8192, (50, 50, 50, 50)
    q = he.gen_primes(N, list(bits))
    ps = nv.he_ks_primes(nv.make_params(N, prime_bits=bits, t=1032193, base_log2=16))
    P = 1
    for p in ps:
        P *= p
    B = bound(N, q, 16)
    below = P // ps[-1]
    for E in (0, 1, B, -1, -B, B // 3, -(B // 7)):
        top = (E % P) // below
        assert (top > ps[-1] // 2) == (E < 0)
