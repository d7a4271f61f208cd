"""Multiplication counts of padded convolution under several readings of the
paper's comparison (test infrastructure; counting only, no arithmetic of the
method).

Section 4's kernel/input-size ablation (Fig. 8) compares the polynomial
products of the correlation-aware packing (Section 3.3, Eq. 1-2) with those
of the conventional packing it builds on, at C = M = 3: a 5x5 kernel over
inputs 8x8 .. 64x64 (about 4x fewer at 64x64), then kernels of growing size
over a 64x64 input (about 5.1x fewer for the largest).  The figure itself is
missing from the source, and so are N, the padding and the exact baseline.
This module counts products per image under each combination of:

  conventional side
    windows    "square": square windows of side s clipped to the padded
               image (the reading that reproduces the toy example's 4
               products at a degree cap of 8); "rect": any H_n x W_n.
    channels   "blocks": C_n channels per polynomial at stride H_n W_n;
               "one": one channel per polynomial.
    out_pack   several kernels per polynomial (output packing) or one.
  correlated side
    O_rule     "tile": O = max(tile input rows, tile input cols) + h - 1, the
               paper's O_w of the partition window; "literal": O = max(W, H)
               + h - 1 of the whole image, as printed with Eq. 1-2.
    channels   "blocks" (channel c at offset c S) or "one".
    out_pack   as above.
  shared: N, and the padding ("same" p = (h-1)/2, "valid" p = 0, "full"
  p = h - 1).

Every count is M_G G T, the polynomial products per image, from an
exhaustive search over windows minimising it (ties do not matter for a
count).  Each configuration's window must satisfy the same no-wrap rules as
the plans in packing.py: every requested output coefficient below N, and no
wrapped term (x^N = -1) landing on one.
"""
from __future__ import annotations

from . import packing

PADS = ("same", "valid", "full")


def pad_of(mode: str, h: int) -> int:
    return {"same": (h - 1) // 2, "valid": 0, "full": h - 1}[mode]


def conventional_count(N, C, H, W, M, h, pad, windows="square", channels="blocks", out_pack=True):
    """Fewest products per image of the row-major packing of the zero-padded
    input (kernel reversed at offset O = (C_n-1) H_n W_n + (h-1) W_n + h - 1,
    output (a, b) at O + a W_n + b); None if no window fits."""
    Hp, Wp = H + 2 * pad, W + 2 * pad
    Ho, Wo = Hp - h + 1, Wp - h + 1
    if Ho < 1 or Wo < 1:
        return None
    if windows == "square":
        shapes = [(min(s, Hp), min(s, Wp)) for s in range(h, max(Hp, Wp) + 1)]
    else:
        shapes = [(a, b) for a in range(h, Hp + 1) for b in range(h, Wp + 1)]
    groups = range(1, C + 1) if channels == "blocks" else [C]
    best = None
    for G in groups:
        Cn = -(-C // G)
        if -(-C // Cn) != G:
            continue
        for (Hn, Wn) in set(shapes):
            if Cn * Hn * Wn > N:
                continue
            th, tw = Hn - h + 1, Wn - h + 1
            Th, Tw = -(-Ho // th), -(-Wo // tw)
            T = Th * Tw
            if best is not None and G * T >= best:
                continue    # at least one kernel polynomial: cannot beat the best
            if out_pack:
                sizes = {(min(th, Ho - i * th), min(tw, Wo - j * tw)) for i in range(Th) for j in range(Tw)}
                Mn, _ = packing._out_packing(M, N, packing._conv_ranges(Cn, Hn, Wn, h, sizes))
            else:
                Mn = 1
            cnt = -(-M // Mn) * G * T
            if best is None or cnt < best:
                best = cnt
    return best


def correlated_count(N, C, H, W, M, h, pad, O_rule="tile", channels="blocks", out_pack=True):
    """Fewest products per image of the correlated packing (Eq. 1-2) over
    output tiles th x tw; None if no tile fits."""
    Ho, Wo = H + 2 * pad - h + 1, W + 2 * pad - h + 1
    if Ho < 1 or Wo < 1:
        return None
    best = None
    # large tiles first, so that the bound below prunes early
    for th in range(Ho, 0, -1):
        for tw in range(Wo, 0, -1):
            T = -(-Ho // th) * -(-Wo // tw)
            if best is not None and T >= best:
                continue    # at least one product per tile: cannot beat the best
            tiles = packing._corr_tiles(H, W, h, pad, th, tw)
            O, S, geo = _geometry(tiles, H, W, h, pad, O_rule)
            if not packing._corr_fits(1, S, geo, N):
                continue
            cmax = 1
            if channels == "blocks":
                while cmax < C and packing._corr_fits(cmax + 1, S, geo, N):
                    cmax += 1
            G = -(-C // cmax)
            Cn = -(-C // G)
            if out_pack:
                ranges = [((Cn - 1) * S + lo, (Cn - 1) * S + hi, 2 * (Cn - 1) * S + D1) for (lo, hi, D1) in geo]
                Mn, _ = packing._out_packing(M, N, ranges)
            else:
                Mn = 1
            cnt = -(-M // Mn) * G * T
            if best is None or cnt < best:
                best = cnt
    return best


def _geometry(tiles, H, W, h, pad, O_rule):
    """O, the channel stride S and per-tile (r_lo, r_hi, D1) as in
    packing._corr_geometry, with O taken per the reading."""
    if O_rule == "tile":
        return packing._corr_geometry(tiles, h, pad)
    O = max(W, H) + h - 1
    geo = []
    for (a0, a1, b0, b1, r0, r1, s0, s1) in tiles:
        ulo, uhi = a0 - pad - r0 + h - 1, a1 - 1 - pad - r0 + h - 1
        vlo, vhi = b0 - pad - s0 + h - 1, b1 - 1 - pad - s0 + h - 1
        D1 = (r1 - r0 + h - 2) * O + (s1 - s0 + h - 2)
        geo.append((ulo * O + vlo, uhi * O + vhi, D1))
    S = max(max(rhi, D1 - rlo) for (rlo, rhi, D1) in geo) + 1
    return O, S, geo


CONV_READINGS = {
    # name: (windows, channels, out_pack)
    "library": ("square", "blocks", True),
    "square_no_outpack": ("square", "blocks", False),
    "cheetah_rect": ("rect", "blocks", False),
    "square_one_channel": ("square", "one", False),
    "rect_one_channel": ("rect", "one", False),
}
CORR_READINGS = {
    # name: (O_rule, channels, out_pack)
    "library": ("tile", "blocks", True),
    "tile_no_outpack": ("tile", "blocks", False),
    "literal_O": ("literal", "blocks", True),
    "literal_O_no_outpack": ("literal", "blocks", False),
    "tile_one_channel": ("tile", "one", False),
}


def correlated_capacity(H, W, h, pad, O_rule="tile"):
    """The smallest number of coefficients at which one channel of the
    correlated packing (Eq. 1-2) fits one polynomial with all its requested
    outputs: the toy example's "degree cap" reading (capacity 9, degree <= 8,
    for its 2x2 input and kernel with padding 1)."""
    lo, hi = 1, (H + 2 * h) * (max(H, W) + 2 * h) * 2
    while lo < hi:
        mid = (lo + hi) // 2
        if correlated_count(mid, 1, H, W, 1, h, pad, O_rule, "one", False) == 1:
            hi = mid
        else:
            lo = mid + 1
    return lo


def ratio(N, C, H, M, h, padmode, conv_reading, corr_reading):
    """conventional / correlated products per image for an H x H input."""
    p = pad_of(padmode, h)
    a = conventional_count(N, C, H, H, M, h, p, *CONV_READINGS[conv_reading])
    b = correlated_count(N, C, H, H, M, h, p, *CORR_READINGS[corr_reading])
    if a is None or b is None:
        return None, a, b
    return a / b, a, b
