"""An independent pin of the plan search (Section 3.3, window constraints;
Eq. 1-2): the product counts the oracle's search chooses equal the minimum
over every layout that is empirically correct.

The brute force here shares nothing with oracle/packing.py's geometry.  For a
correlated layout it places each channel of an output tile's input window by
Eq. 1 (row stride O = the largest tile extent + h - 1, the reading both sides
take) at channel offset c*S, the kernel channel by Eq. 2 at (C_n - 1 - c)*S,
and tries every channel stride S: a layout counts as feasible when, for
random data, the schoolbook negacyclic product of every tile decodes to the
direct zero-padded convolution at the positions the definition gives
(u*O + v + (C_n - 1)*S for output (a, b)).  For the conventional packing it
places the zero-padded square window row-major and the reversed kernel at
offset O = (C_n-1) H_n W_n + (h-1) W_n + h - 1, and checks the same way.  The
minimum of ceil(C / C_n) * tiles over the feasible layouts is compared with
the oracle plan's G * T (one output channel, so no output packing)."""
import itertools

import numpy as np
import pytest

from oracle import packing

P = 65521  # random data mod a prime: a wrong layout matches every checked output with negligible probability


def negacyclic(a, b, N):
    """Schoolbook negacyclic product mod P (int64: products < 2^32, sums of
    at most N < 2^10 of them)."""
    full = np.convolve(a, b)
    out = full[:N].copy()
    out[:len(full) - N] -= full[N:]
    return out % P


def conv_direct(x, w, pad):
    C, H, W = x.shape
    h = w.shape[-1]
    xp = np.zeros((C, H + 2 * pad, W + 2 * pad), dtype=np.int64)
    xp[:, pad:pad + H, pad:pad + W] = x
    Ho, Wo = H + 2 * pad - h + 1, W + 2 * pad - h + 1
    y = np.zeros((Ho, Wo), dtype=np.int64)
    for a in range(Ho):
        for b in range(Wo):
            y[a, b] = (xp[:, a:a + h, b:b + h] * w).sum() % P
    return y


def tiles_of(Ho, Wo, th, tw):
    return [(a0, min(Ho, a0 + th), b0, min(Wo, b0 + tw))
            for a0 in range(0, Ho, th) for b0 in range(0, Wo, tw)]


def corr_feasible(N, C, H, W, h, pad, th, tw, Cn, S, x, w, y):
    """Every tile of every channel group decodes correctly under the layout."""
    Ho, Wo = H + 2 * pad - h + 1, W + 2 * pad - h + 1
    tl = tiles_of(Ho, Wo, th, tw)
    # input window of a tile: rows [a0 - pad, a1 - pad + h - 1) clipped to the image
    wins = [(max(0, a0 - pad), min(H, a1 - pad + h - 1), max(0, b0 - pad), min(W, b1 - pad + h - 1))
            for (a0, a1, b0, b1) in tl]
    O = max(max(r1 - r0, s1 - s0) for (r0, r1, s0, s1) in wins) + h - 1
    for g0 in range(0, C, Cn):
        chans = list(range(g0, min(C, g0 + Cn)))
        kp = np.zeros(N, dtype=np.int64)
        for ci, c in enumerate(chans):
            for k in range(h):
                for l in range(h):
                    pos = (Cn - 1 - ci) * S + (h - 1 - k) * O + (h - 1 - l)
                    if pos >= N:
                        return False
                    kp[pos] = (kp[pos] + w[c, k, l]) % P
        part = conv_direct(x[chans], w[chans], pad)
        for (a0, a1, b0, b1), (r0, r1, s0, s1) in zip(tl, wins):
            xp = np.zeros(N, dtype=np.int64)
            for ci, c in enumerate(chans):
                for i in range(r0, r1):
                    for j in range(s0, s1):
                        pos = ci * S + (i - r0) * O + (j - s0)
                        if pos >= N:
                            return False
                        xp[pos] = (xp[pos] + x[c, i, j]) % P
            prod = negacyclic(xp, kp, N)
            for a in range(a0, a1):
                for b in range(b0, b1):
                    pos = (Cn - 1) * S + (a - pad - r0 + h - 1) * O + (b - pad - s0 + h - 1)
                    if pos >= N or (prod[pos] - part[a, b]) % P:
                        return False
    return True


def corr_bruteforce(N, C, H, W, h, pad, rng):
    x = rng.integers(0, P, (C, H, W))
    w = rng.integers(0, P, (C, h, h))
    Ho, Wo = H + 2 * pad - h + 1, W + 2 * pad - h + 1
    best = None
    for th, tw in itertools.product(range(1, Ho + 1), range(1, Wo + 1)):
        T = len(tiles_of(Ho, Wo, th, tw))
        for Cn in range(1, C + 1):
            cnt = -(-C // Cn) * T
            if best is not None and cnt >= best:
                continue
            if any(corr_feasible(N, C, H, W, h, pad, th, tw, Cn, S, x, w, None) for S in range(1, N + 1)):
                best = cnt
    return best


def conv_feasible(N, C, H, W, h, pad, s, Cn, x, w):
    Hp, Wp = H + 2 * pad, W + 2 * pad
    Hn, Wn = min(s, Hp), min(s, Wp)
    th, tw = Hn - h + 1, Wn - h + 1
    Ho, Wo = Hp - h + 1, Wp - h + 1
    xpad = np.zeros((C, Hp, Wp), dtype=np.int64)
    xpad[:, pad:pad + H, pad:pad + W] = x
    Oc = (Cn - 1) * Hn * Wn + (h - 1) * Wn + h - 1
    for g0 in range(0, C, Cn):
        chans = list(range(g0, min(C, g0 + Cn)))
        kp = np.zeros(N, dtype=np.int64)
        for ci, c in enumerate(chans):
            for k in range(h):
                for l in range(h):
                    pos = Oc - ci * Hn * Wn - k * Wn - l
                    if not 0 <= pos < N:
                        return False
                    kp[pos] = (kp[pos] + w[c, k, l]) % P
        part = conv_direct(x[chans], w[chans], pad)
        for (a0, a1, b0, b1) in tiles_of(Ho, Wo, th, tw):
            xp = np.zeros(N, dtype=np.int64)
            for ci, c in enumerate(chans):
                for i in range(Hn):
                    for j in range(Wn):
                        r, q = a0 + i, b0 + j
                        if r < Hp and q < Wp:
                            pos = ci * Hn * Wn + i * Wn + j
                            if pos >= N:
                                return False
                            xp[pos] = (xp[pos] + xpad[c, r, q]) % P
            prod = negacyclic(xp, kp, N)
            for a in range(a0, a1):
                for b in range(b0, b1):
                    pos = Oc + (a - a0) * Wn + (b - b0)
                    if pos >= N or (prod[pos] - part[a, b]) % P:
                        return False
    return True


def conv_bruteforce(N, C, H, W, h, pad, rng):
    x = rng.integers(0, P, (C, H, W))
    w = rng.integers(0, P, (C, h, h))
    Hp, Wp = H + 2 * pad, W + 2 * pad
    Ho, Wo = Hp - h + 1, Wp - h + 1
    best = None
    for s in range(h, max(Hp, Wp) + 1):
        Hn, Wn = min(s, Hp), min(s, Wp)
        T = len(tiles_of(Ho, Wo, Hn - h + 1, Wn - h + 1))
        for Cn in range(1, C + 1):
            cnt = -(-C // Cn) * T
            if best is not None and cnt >= best:
                continue
            if conv_feasible(N, C, H, W, h, pad, s, Cn, x, w):
                best = cnt
    return best


CASES = [(16, 1, 2, 2, 2, 1), (32, 2, 4, 4, 3, 1), (64, 3, 5, 4, 3, 1), (64, 2, 6, 6, 3, 0), (128, 3, 6, 5, 3, 2),
         (64, 1, 7, 7, 3, 1), (128, 2, 8, 8, 5, 2), (32, 3, 3, 3, 1, 0)]


@pytest.mark.parametrize("N,C,H,W,h,pad", CASES)
def test_correlated_plan_is_the_bruteforce_minimum(N, C, H, W, h, pad):
    rng = np.random.default_rng(N * 31 + C * 7 + H + 100 * h + pad)
    want = corr_bruteforce(N, C, H, W, h, pad, rng)
    p = packing.make_plan("corr", N, C, H, W, 1, h, pad)
    assert want is not None and p.G * p.T == want, (p.G, p.T, want)


@pytest.mark.parametrize("N,C,H,W,h,pad", CASES)
def test_conventional_plan_is_the_bruteforce_minimum(N, C, H, W, h, pad):
    rng = np.random.default_rng(N * 37 + C * 11 + H + 100 * h + pad)
    want = conv_bruteforce(N, C, H, W, h, pad, rng)
    p = packing.make_plan("conv", N, C, H, W, 1, h, pad)
    assert want is not None and p.G * p.T == want, (p.G, p.T, want)


# ---------------------------------------------------------------- output packing (R14)
def corr_outpack_feasible(N, C, H, W, h, pad, th, tw, Cn, S, Mn, Sout, x, ws):
    """Mn kernels share one polynomial, kernel m at offset m*Sout: every
    kernel's outputs decode correctly for every tile and channel group."""
    Ho, Wo = H + 2 * pad - h + 1, W + 2 * pad - h + 1
    tl = tiles_of(Ho, Wo, th, tw)
    wins = [(max(0, a0 - pad), min(H, a1 - pad + h - 1), max(0, b0 - pad), min(W, b1 - pad + h - 1))
            for (a0, a1, b0, b1) in tl]
    O = max(max(r1 - r0, s1 - s0) for (r0, r1, s0, s1) in wins) + h - 1
    for g0 in range(0, C, Cn):
        chans = list(range(g0, min(C, g0 + Cn)))
        kp = np.zeros(N, dtype=np.int64)
        for m in range(Mn):
            for ci, c in enumerate(chans):
                for k in range(h):
                    for l in range(h):
                        pos = m * Sout + (Cn - 1 - ci) * S + (h - 1 - k) * O + (h - 1 - l)
                        if pos >= N:
                            return False
                        kp[pos] = (kp[pos] + ws[m][c, k, l]) % P
        parts = [conv_direct(x[chans], ws[m][chans], pad) for m in range(Mn)]
        for (a0, a1, b0, b1), (r0, r1, s0, s1) in zip(tl, wins):
            xp = np.zeros(N, dtype=np.int64)
            for ci, c in enumerate(chans):
                for i in range(r0, r1):
                    for j in range(s0, s1):
                        pos = ci * S + (i - r0) * O + (j - s0)
                        if pos >= N:
                            return False
                        xp[pos] = (xp[pos] + x[c, i, j]) % P
            prod = negacyclic(xp, kp, N)
            for m in range(Mn):
                for a in range(a0, a1):
                    for b in range(b0, b1):
                        pos = m * Sout + (Cn - 1) * S + (a - pad - r0 + h - 1) * O + (b - pad - s0 + h - 1)
                        if pos >= N or (prod[pos] - parts[m][a, b]) % P:
                            return False
    return True


def corr_outpack_bruteforce(N, C, H, W, M, h, pad, rng):
    x = rng.integers(0, P, (C, H, W))
    ws = [rng.integers(0, P, (C, h, h)) for _ in range(M)]
    Ho, Wo = H + 2 * pad - h + 1, W + 2 * pad - h + 1
    best = None
    for th, tw in itertools.product(range(1, Ho + 1), range(1, Wo + 1)):
        T = len(tiles_of(Ho, Wo, th, tw))
        for Cn in range(1, C + 1):
            G = -(-C // Cn)
            if best is not None and G * T >= best:
                continue
            for S in range(1, N + 1):
                if not corr_feasible(N, C, H, W, h, pad, th, tw, Cn, S, x, ws[0], None):
                    continue
                for Mn in range(M, 0, -1):
                    cnt = -(-M // Mn) * G * T
                    if best is not None and cnt >= best:
                        continue
                    if any(corr_outpack_feasible(N, C, H, W, h, pad, th, tw, Cn, S, Mn, So, x, ws)
                           for So in range(1, N)):
                        best = cnt
    return best


@pytest.mark.parametrize("N,C,H,W,h,pad", [(32, 1, 3, 3, 2, 1), (64, 2, 3, 4, 3, 1), (64, 1, 4, 4, 3, 0),
                                            (128, 2, 4, 4, 3, 2)])
def test_correlated_output_packing_is_the_bruteforce_minimum(N, C, H, W, h, pad):
    """With M = 3 output channels: the oracle plan's M_G G T equals the
    minimum over every correctly decoding layout with M_n kernels per
    polynomial at any stride S_out (and any tile size, C_n and S)."""
    M = 3
    rng = np.random.default_rng(N * 41 + C * 13 + H + 100 * h + pad)
    want = corr_outpack_bruteforce(N, C, H, W, M, h, pad, rng)
    p = packing.make_plan("corr", N, C, H, W, M, h, pad)
    assert want is not None and p.MG * p.G * p.T == want, (p.MG, p.G, p.T, want)
