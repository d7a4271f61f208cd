"""Polynomial packing for convolution (test infrastructure).

Two encodings of a stride-1, zero-padded 2-D convolution into products in
A_{N,t} = Z_t[x]/(x^N+1):

* conventional ("conv"), the row-major packing the paper builds on (Section 3.3,
  left half of Fig. 7; Section 3.1): the input is zero-padded to H' x W' and
  packed row-major, the kernel is packed reversed, output (a, b) is read at
  coefficient O + a W_n + b.  Cut into C_n x H_n x W_n windows when it does not
  fit.
* correlated ("corr"), Eq. 1 and Eq. 2 of Section 3.3: x^[iO+j] = x[i,j],
  w^[(h-1-i)O + (h-1-j)] = w[i,j], O = max(W, H) + h - 1; no coefficient is
  spent on padding.  Partition windows per Section 3.3 ("For large input ...").

Readings where the paper is silent or garbled:
  R1  conventional windows are square with side s, clipped to the padded
      image (H_n = min(s, H'), W_n = min(s, W')); this is the only reading that
      gives the toy example's 4 products at a degree cap of 8.
  R2  conventional channel blocks: C_n channels per polynomial at stride
      H_n W_n, kernel offset O = (C_n-1) H_n W_n + (h-1) W_n + h - 1.
  R3  correlated channel blocks: channel c at offset c S, kernel channel c at
      (C_n-1-c) S, S the smallest stride that keeps the cross-channel terms
      off the requested outputs; C_n ranges over every count up to the
      largest for which the requested outputs stay below N and no wrapped
      term reaches them (fewer channels can leave room for output packing).
  R4  correlated windows are chosen over output tiles th x tw; a tile covering
      output rows [a0, a1) encodes input rows [a0-p, a1-p+h-1) clipped to the
      image; O uses the largest tile extent.
  R5  window objective: minimise the polynomial products per image
      ceil(M / M_n) G T, then the input polynomials G T, then G, then prefer
      larger windows; the paper's printed objective is garbled (floors, and
      W_w + h - 1 where W_w - h + 1 is meant).
  R6  output packing (the FC layers follow Cheetah, which packs several
      matrix rows per polynomial): M_n kernels share one polynomial at stride
      S_out, kernel m at offset (m mod M_n) S_out; S_out is the smallest
      stride that keeps the other kernels' products off each kernel's
      requested outputs, and M_n the largest count for which every requested
      output stays below N and no wrapped term reaches one.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Plan:
    encoding: str
    N: int
    C: int
    H: int
    W: int
    M: int
    h: int
    pad: int
    Cn: int
    G: int
    th: int          # output rows per tile
    tw: int          # output cols per tile
    Th: int
    Tw: int
    # conventional window
    Hn: int = 0
    Wn: int = 0
    Ooff: int = 0    # conventional kernel offset O
    # correlated
    O: int = 0
    S: int = 0
    # output packing
    Mn: int = 1
    Sout: int = 0
    tiles: list = field(default_factory=list)   # (a0, a1, b0, b1, r0, r1, s0, s1) per tile
    depthwise: bool = False   # output channel m reads input channel m only

    @property
    def T(self):
        return self.Th * self.Tw

    @property
    def MG(self):
        return -(-self.M // self.Mn)

    @property
    def Ho(self):
        return self.H + 2 * self.pad - self.h + 1

    @property
    def Wo(self):
        return self.W + 2 * self.pad - self.h + 1

    def key(self):
        return (self.encoding, self.N, self.C, self.H, self.W, self.M, self.h, self.pad, self.Cn, self.G,
                self.th, self.tw, self.Th, self.Tw, self.Hn, self.Wn, self.Ooff, self.O, self.S, self.Mn, self.Sout,
                self.depthwise)

    def pair_used(self, mg, g):
        """Whether kernel polynomial mg meets channel group g in a product:
        always, except in a depthwise plan, where the Mn outputs of mg (all in
        one channel group: Mn divides Cn, or there is one group) meet only
        that group."""
        return (not self.depthwise) or g == (mg * self.Mn) // self.Cn

    @property
    def products(self):
        """Polynomial products per image."""
        return self.MG * self.T * (1 if self.depthwise else self.G)


def _out_packing(M, N, ranges, depthwise_cn=0):
    """(M_n, S_out) for product spans given as (r_lo, r_hi, D) per tile: r_lo, r_hi
    the lowest and highest requested coefficient of one kernel's product,
    D its highest possible degree (before any wrap).  For a depthwise layer
    with several channel groups (depthwise_cn = C_n) M_n is the largest
    fitting divisor of C_n, so that a kernel polynomial's outputs lie in one
    channel group (with a single group any M_n does)."""
    Sout = max(max(rhi, D - rlo) for (rlo, rhi, D) in ranges) + 1
    def fits(k):
        for (rlo, rhi, D) in ranges:
            if (k - 1) * Sout + rhi >= N:
                return False
            tot = (k - 1) * Sout + D
            if not (tot < N or tot - N < rlo):
                return False
        return True
    k = 1
    while k < M and fits(k + 1):
        k += 1
    if depthwise_cn:
        while depthwise_cn % k:
            k -= 1
        return k, Sout
    G = -(-M // k)
    return -(-M // G), Sout


def _check_shape(C, H, W, M, h, pad):
    if min(C, H, W, M, h) < 1 or pad < 0 or pad > h - 1:
        raise ValueError("bad conv shape")
    if H + 2 * pad - h + 1 < 1 or W + 2 * pad - h + 1 < 1:
        raise ValueError("empty output")


def _conv_ranges(Cn, Hn, Wn, h, th_list):
    """requested (r_lo, r_hi) and max degree D of a conventional window product;
    th_list: (rows, cols) of output per tile"""
    O = (Cn - 1) * Hn * Wn + (h - 1) * Wn + h - 1
    D = Cn * Hn * Wn - 1 + O
    return [(O, O + (a - 1) * Wn + (b - 1), D) for (a, b) in th_list]


def plan_conventional(N, C, H, W, M, h, pad, depthwise=False) -> Plan:
    _check_shape(C, H, W, M, h, pad)
    Hp, Wp = H + 2 * pad, W + 2 * pad
    Ho, Wo = Hp - h + 1, Wp - h + 1
    best = None
    for G in range(1, C + 1):
        Cn = -(-C // G)
        if -(-C // Cn) != G:
            continue
        for s in range(h, max(Hp, Wp) + 1):
            Hn, Wn = min(s, Hp), min(s, Wp)
            if Cn * Hn * Wn > N:
                continue
            th, tw = Hn - h + 1, Wn - h + 1
            Th, Tw = -(-Ho // th), -(-Wo // tw)
            sizes = {(min(th, Ho - i * th), min(tw, Wo - j * tw)) for i in range(Th) for j in range(Tw)}
            Mn, Sout = _out_packing(M, N, _conv_ranges(Cn, Hn, Wn, h, sizes), Cn if depthwise and G > 1 else 0)
            MG = -(-M // Mn)
            key = (MG * (1 if depthwise else G) * Th * Tw, G * Th * Tw, G, -Hn, -Wn)
            if best is None or key < best[0]:
                best = (key, (Cn, G, Hn, Wn, th, tw, Th, Tw, Mn, Sout))
    if best is None:
        raise ValueError("plan does not fit")
    Cn, G, Hn, Wn, th, tw, Th, Tw, Mn, Sout = best[1]
    p = Plan("conv", N, C, H, W, M, h, pad, Cn, G, th, tw, Th, Tw, Hn=Hn, Wn=Wn,
             Ooff=(Cn - 1) * Hn * Wn + (h - 1) * Wn + h - 1, Mn=Mn, Sout=Sout, depthwise=depthwise)
    for ti in range(Th):
        for tj in range(Tw):
            a0, b0 = ti * th, tj * tw
            p.tiles.append((a0, min(Ho, a0 + th), b0, min(Wo, b0 + tw), a0, a0 + Hn, b0, b0 + Wn))
    return p


def _corr_tiles(H, W, h, pad, th, tw):
    Ho, Wo = H + 2 * pad - h + 1, W + 2 * pad - h + 1
    tiles = []
    for ti in range(-(-Ho // th)):
        for tj in range(-(-Wo // tw)):
            a0, b0 = ti * th, tj * tw
            a1, b1 = min(Ho, a0 + th), min(Wo, b0 + tw)
            r0, r1 = max(0, a0 - pad), min(H, a1 - pad + h - 1)
            s0, s1 = max(0, b0 - pad), min(W, b1 - pad + h - 1)
            tiles.append((a0, a1, b0, b1, r0, r1, s0, s1))
    return tiles


def _corr_geometry(tiles, h, pad):
    """O, S and per-tile (r_lo, r_hi, D1) for a list of correlated tiles."""
    Hmax = max(t[5] - t[4] for t in tiles)
    Wmax = max(t[7] - t[6] for t in tiles)
    O = max(Wmax, Hmax) + h - 1
    geo = []
    for (a0, a1, b0, b1, r0, r1, s0, s1) in tiles:
        ulo, uhi = a0 - pad - r0 + h - 1, a1 - 1 - pad - r0 + h - 1
        vlo, vhi = b0 - pad - s0 + h - 1, b1 - 1 - pad - s0 + h - 1
        D1 = (r1 - r0 + h - 2) * O + (s1 - s0 + h - 2)
        geo.append((ulo * O + vlo, uhi * O + vhi, D1))
    S = max(max(rhi, D1 - rlo) for (rlo, rhi, D1) in geo) + 1
    return O, S, geo


def _corr_fits(c, S, geo, N):
    for (rlo, rhi, D1) in geo:
        if (c - 1) * S + rhi >= N:
            return False
        D = 2 * (c - 1) * S + D1
        if not (D < N or D - N < (c - 1) * S + rlo):
            return False
    return True


def plan_correlated(N, C, H, W, M, h, pad, depthwise=False) -> Plan:
    _check_shape(C, H, W, M, h, pad)
    Ho, Wo = H + 2 * pad - h + 1, W + 2 * pad - h + 1
    best = None
    for th in range(1, Ho + 1):
        for tw in range(1, Wo + 1):
            tiles = _corr_tiles(H, W, h, pad, th, tw)
            O, S, geo = _corr_geometry(tiles, h, pad)
            if not _corr_fits(1, S, geo, N):
                continue
            cmax = 1
            while cmax < C and _corr_fits(cmax + 1, S, geo, N):
                cmax += 1
            T = len(tiles)
            # every channel count up to the largest that fits (R3): fewer
            # channels per polynomial can leave room for more kernels (R6)
            seen = set()
            for ct in range(cmax, 0, -1):
                G = -(-C // ct)
                if G in seen:
                    continue
                seen.add(G)
                Cn = -(-C // G)
                ranges = [((Cn - 1) * S + rlo, (Cn - 1) * S + rhi, 2 * (Cn - 1) * S + D1) for (rlo, rhi, D1) in geo]
                Mn, Sout = _out_packing(M, N, ranges, Cn if depthwise and G > 1 else 0)
                MG = -(-M // Mn)
                key = (MG * (1 if depthwise else G) * T, G * T, G, -th, -tw)
                if best is None or key < best[0]:
                    best = (key, (Cn, G, th, tw, O, S, tiles, Mn, Sout))
    if best is None:
        raise ValueError("plan does not fit")
    Cn, G, th, tw, O, S, tiles, Mn, Sout = best[1]
    return Plan("corr", N, C, H, W, M, h, pad, Cn, G, th, tw, -(-Ho // th), -(-Wo // tw), O=O, S=S, Mn=Mn,
                Sout=Sout, tiles=tiles, depthwise=depthwise)


def make_plan(encoding, N, C, H, W, M, h, pad, depthwise=False) -> Plan:
    """depthwise: output channel m reads input channel m only (M = C; the
    weights are diagonal in the channel indices, as the gamma of a batch
    norm): the search minimises MG * T, the products actually needed."""
    if depthwise and M != C:
        raise ValueError("a depthwise layer has M = C")
    if encoding == "conv":
        return plan_conventional(N, C, H, W, M, h, pad, depthwise)
    if encoding == "corr":
        return plan_correlated(N, C, H, W, M, h, pad, depthwise)
    raise ValueError(encoding)


# ------------------------------------------------------------------ maps
def input_slots(p: Plan, t: int, g: int):
    """(coefficient, channel, row, col) of every input value of poly (tile t, group g)."""
    a0, a1, b0, b1, r0, r1, s0, s1 = p.tiles[t]
    out = []
    for cl in range(p.Cn):
        c = g * p.Cn + cl
        if c >= p.C:
            break
        if p.encoding == "conv":
            for i in range(p.Hn):
                for j in range(p.Wn):
                    r, s = r0 + i - p.pad, s0 + j - p.pad
                    if 0 <= r < p.H and 0 <= s < p.W:
                        out.append((cl * p.Hn * p.Wn + i * p.Wn + j, c, r, s))
        else:
            for i in range(r0, r1):
                for j in range(s0, s1):
                    out.append((cl * p.S + (i - r0) * p.O + (j - s0), c, i, j))
    return out


def kernel_slots(p: Plan, g: int):
    """(coefficient, channel, k, l) of every weight of the kernel of one output
    channel in group g, before its output-packing offset (m mod M_n) S_out."""
    out = []
    for cl in range(p.Cn):
        c = g * p.Cn + cl
        if c >= p.C:
            break
        for k in range(p.h):
            for l in range(p.h):
                if p.encoding == "conv":
                    out.append((p.Ooff - cl * p.Hn * p.Wn - k * p.Wn - l, c, k, l))
                else:
                    out.append(((p.Cn - 1 - cl) * p.S + (p.h - 1 - k) * p.O + (p.h - 1 - l), c, k, l))
    return out


def output_slots(p: Plan, t: int):
    """(coefficient, a, b) of every output of the product poly of tile t."""
    a0, a1, b0, b1, r0, r1, s0, s1 = p.tiles[t]
    out = []
    for a in range(a0, a1):
        for b in range(b0, b1):
            if p.encoding == "conv":
                out.append((p.Ooff + (a - a0) * p.Wn + (b - b0), a, b))
            else:
                u = a - p.pad - r0 + p.h - 1
                v = b - p.pad - s0 + p.h - 1
                out.append(((p.Cn - 1) * p.S + u * p.O + v, a, b))
    return out


def encode_input(p: Plan, x, t_mod) -> np.ndarray:
    """x: [C, H, W] integers -> [T][G][N] uint64 mod t."""
    x = np.asarray(x)
    out = np.zeros((p.T, p.G, p.N), dtype=np.uint64)
    for t in range(p.T):
        for g in range(p.G):
            for (k, c, i, j) in input_slots(p, t, g):
                out[t, g, k] = int(x[c, i, j]) % t_mod
    return out


def encode_kernel(p: Plan, w, t_mod) -> np.ndarray:
    """w: [M, C, h, h] integers -> [MG][G][N] uint64 mod t; output channel m
    sits in polynomial m // M_n at offset (m mod M_n) S_out."""
    w = np.asarray(w)
    out = np.zeros((p.MG, p.G, p.N), dtype=np.uint64)
    for g in range(p.G):
        slots = kernel_slots(p, g)
        for m in range(p.M):
            off = (m % p.Mn) * p.Sout
            for (k, c, a, b) in slots:
                out[m // p.Mn, g, k + off] = int(w[m, c, a, b]) % t_mod
    return out


def decode(p: Plan, polys, t_mod) -> np.ndarray:
    """polys: [MG][T][N] mod t -> int64 [M, Ho, Wo], centred (v > t/2 -> v - t)."""
    polys = np.asarray(polys)
    out = np.zeros((p.M, p.Ho, p.Wo), dtype=np.int64)
    for t in range(p.T):
        for (k, a, b) in output_slots(p, t):
            for m in range(p.M):
                v = int(polys[m // p.Mn, t, k + (m % p.Mn) * p.Sout])
                out[m, a, b] = v - t_mod if v > (t_mod - 1) // 2 else v
    return out


def encode_output(p: Plan, values, t_mod) -> np.ndarray:
    """values: [M, Ho, Wo] integers -> [MG][T][N] uint64 mod t holding each
    value where decode reads that output (zero elsewhere): a per-output
    plaintext such as a bias, placed on the layer's product positions."""
    values = np.asarray(values)
    out = np.zeros((p.MG, p.T, p.N), dtype=np.uint64)
    for t in range(p.T):
        for (k, a, b) in output_slots(p, t):
            for m in range(p.M):
                out[m // p.Mn, t, k + (m % p.Mn) * p.Sout] = int(values[m, a, b]) % t_mod
    return out


def product_terms(p: Plan):
    """Term lists of the polynomial products: output (mg, t) = sum_g in(t,g) *
    ker(mg,g).  Returns, per output o = mg*T + t, the list of (input poly
    index t*G+g, kernel poly index mg*G+g)."""
    terms = []
    for mg in range(p.MG):
        for t in range(p.T):
            terms.append([(t * p.G + g, mg * p.G + g) for g in range(p.G) if p.pair_used(mg, g)])
    return terms
