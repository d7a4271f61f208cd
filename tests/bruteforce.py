"""Brute-force helpers for the oracle pins: Python big integers and
O(N^2) schoolbook products only, no NTT and no CRT, so that a mistake in the
oracle's transform or big-integer code cannot cancel out."""
from __future__ import annotations


def negacyclic_int(a, b):
    """Exact integer product in Z[x]/(x^N+1) (schoolbook)."""
    N = len(a)
    c = [0] * N
    for i, ai in enumerate(a):
        if ai == 0:
            continue
        for j, bj in enumerate(b):
            k = i + j
            if k < N:
                c[k] += ai * bj
            else:
                c[k - N] -= ai * bj
    return c


def negacyclic_mod(a, b, m):
    return [v % m for v in negacyclic_int([int(x) for x in a], [int(x) for x in b])]


def crt(residues, moduli):
    """Integer in [0, prod m) with the given residues (Python big ints)."""
    M = 1
    for m in moduli:
        M *= m
    x = 0
    for r, m in zip(residues, moduli):
        Mi = M // m
        x += int(r) * Mi * pow(Mi, -1, m)
    return x % M


def centred(x, M):
    return x - M if x > M // 2 else x


def round_tq(d, t, q):
    """floor((t d + floor(q/2)) / q), Python floor division (any sign of d)."""
    return (t * d + q // 2) // q
