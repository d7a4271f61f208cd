"""CryptoTrain-P linear layer on the oracle (test infrastructure).

Section 3.2: offline, the client draws masks r^x, r^w, encrypts them and the
server computes [r^x r^w] by CCMul (with relinearisation); online, the server
computes c = [x](w - r^w) + [w](x - r^x) + [r^x r^w] by two CPMuls and CCAdds
and p = (x - r^x)(w - r^w) by PPMul; the client recovers Dec(c) - p = x w.
With channel groups the products are summed over the G groups of an output.

Reading: masks are uniform over all N coefficients of R_t (the paper's
"R^n" is undefined).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import he, packing


@dataclass
class LayerRun:
    plan: packing.Plan
    keys: he.Keys
    x_polys: np.ndarray      # [T*G][N]
    w_polys: np.ndarray      # [MG*G][N]
    r_x: np.ndarray
    r_w: np.ndarray
    ct_x: np.ndarray
    ct_w: np.ndarray
    ct_rx: np.ndarray
    ct_rw: np.ndarray
    rr: np.ndarray           # [B*MG*T][2][L][N] precomputed [r^x r^w]
    out: np.ndarray          # [B*MG*T][2][L][N] online result c
    p: np.ndarray            # [B*MG*T][N] PPMul result
    y: np.ndarray            # decoded [M, Ho, Wo]


def precompute_pairs(plan, batch=1):
    """CCMul pairs (rx index, rw index), consecutive per output (b, m, t) in
    that order (G per output; one in a depthwise plan); rx index
    (b*T + t)*G + g, rw index m*G + g."""
    pairs = []
    for b in range(batch):
        for m in range(plan.MG):
            for t in range(plan.T):
                for g in range(plan.G):
                    if plan.pair_used(m, g):
                        pairs.append(((b * plan.T + t) * plan.G + g, m * plan.G + g))
    return pairs


def ccmul_group(plan):
    """Pairs summed into one CCMul output."""
    return 1 if plan.depthwise else plan.G


def online_terms(plan, batch=1):
    """CPMul terms over ct = [ct_x ; ct_w] and pt = [(w - r^w) ; (x - r^x)],
    output order (b, m, t)."""
    TG, MG = plan.T * plan.G, plan.MG * plan.G
    terms = []
    for b in range(batch):
        for m in range(plan.MG):
            for t in range(plan.T):
                tl = []
                for g in range(plan.G):
                    if not plan.pair_used(m, g):
                        continue
                    xi = (b * plan.T + t) * plan.G + g
                    tl.append((xi, m * plan.G + g))
                    tl.append((batch * TG + m * plan.G + g, MG + xi))
                terms.append(tl)
    return terms


def ppmul_terms(plan, batch=1):
    terms = []
    for b in range(batch):
        for m in range(plan.MG):
            for t in range(plan.T):
                terms.append([((b * plan.T + t) * plan.G + g, m * plan.G + g) for g in range(plan.G)
                              if plan.pair_used(m, g)])
    return terms


def run_layer(P: he.Params, plan, x, w, seeds, keys=None, first_image: int = 0, bias=None) -> LayerRun:
    """x: [C,H,W] or [B,C,H,W] ints, w: [M,C,h,h] ints; seeds:
    workloads.ProtocolSeeds.  Every random object of the batch is drawn from
    one stream per kind, object index = position in the flattened batch.
    first_image: the batch position of x's first image, so that images of a
    large batch can be recomputed one at a time (the weight-side objects do
    not depend on it).
    bias: optional per-output-channel integers [M] (a batch-norm beta): each
    image's encode_output of the bias broadcast over [M, Ho, Wo] is encrypted
    on the enc_w stream after the kernel polynomials (row k of image b is
    object MG*G + b*MG*T + k) and added to the precomputed [r^x r^w] (CCAdd),
    so the layer decodes to conv + bias."""
    t = P.t
    x = np.asarray(x)
    if x.ndim == 3:
        x = x[None]
    B = x.shape[0]
    if keys is None:
        keys = he.keygen(P, seeds.keys, True)
    xp = np.concatenate([packing.encode_input(plan, x[b], t).reshape(-1, P.N) for b in range(B)])
    wp = packing.encode_kernel(plan, w, t).reshape(-1, P.N)
    first = first_image * plan.T * plan.G
    r_x = he.sample_masks(P, seeds.mask_x, xp.shape[0], first)
    r_w = he.sample_masks(P, seeds.mask_w, wp.shape[0])
    ct_x = he.encrypt(P, keys, xp, seeds.enc_x, first)
    ct_w = he.encrypt(P, keys, wp, seeds.enc_w)
    ct_rx = he.encrypt(P, keys, r_x, seeds.enc_rx, first)
    ct_rw = he.encrypt(P, keys, r_w, seeds.enc_rw)
    # offline: [r^x r^w] summed over channel groups
    rr = he.ccmul(P, keys, ct_rx, ct_rw, precompute_pairs(plan, B), ccmul_group(plan))
    if bias is not None:
        nw = plan.MG * plan.G
        bv = np.broadcast_to(np.asarray(bias, dtype=np.int64)[:, None, None], (plan.M, plan.Ho, plan.Wo))
        no = plan.MG * plan.T
        for b in range(B):
            bp = packing.encode_output(plan, bv, t).reshape(-1, P.N)
            cb = he.encrypt(P, keys, bp, seeds.enc_w, nw + (first_image + b) * no)
            for o in range(no):
                for comp in range(2):
                    for i, q in enumerate(P.q):
                        row = rr[b * no + o, comp, i]
                        rr[b * no + o, comp, i] = [(int(u) + int(v)) % q for u, v in zip(row, cb[o, comp, i])]
    # online
    tt = np.uint64(t)
    wm = (wp + (tt - r_w)) % tt
    xm = (xp + (tt - r_x)) % tt
    ct_all = np.concatenate([ct_x, ct_w])
    pt_all = np.concatenate([wm, xm])
    out = he.cpmul_terms(P, ct_all, pt_all, online_terms(plan, B), add=rr)
    p = he.ppmul_terms(P, xm, wm, ppmul_terms(plan, B))
    dec = he.decrypt(P, keys, out)
    z = (dec + (tt - p)) % tt
    zz = z.reshape(B, plan.MG, plan.T, P.N)
    y = np.stack([packing.decode(plan, zz[b], t) for b in range(B)])
    if B == 1:
        y = y[0]
    return LayerRun(plan, keys, xp, wp, r_x, r_w, ct_x, ct_w, ct_rx, ct_rw, rr, out, p, y)


@dataclass
class LayerRunB:
    plan: packing.Plan
    keys: he.Keys
    x_polys: np.ndarray
    w_polys: np.ndarray
    ct_x: np.ndarray
    ct_w: np.ndarray
    out: np.ndarray          # [B*MG*T][2][L][N] relinearised [x][w]
    y: np.ndarray


def run_layer_b(P: he.Params, plan, x, w, seeds, keys=None) -> LayerRunB:
    """CryptoTrain-B linear layer (Section 3.1): encrypt x and w, multiply the
    ciphertexts (CCMul with relinearisation; the G channel groups of an output
    summed before the rounding), decrypt and decode.  Object indices as in
    run_layer (enc_x, enc_w streams)."""
    t = P.t
    x = np.asarray(x)
    if x.ndim == 3:
        x = x[None]
    B = x.shape[0]
    if keys is None:
        keys = he.keygen(P, seeds.keys, True)
    xp = np.concatenate([packing.encode_input(plan, x[b], t).reshape(-1, P.N) for b in range(B)])
    wp = packing.encode_kernel(plan, w, t).reshape(-1, P.N)
    ct_x = he.encrypt(P, keys, xp, seeds.enc_x)
    ct_w = he.encrypt(P, keys, wp, seeds.enc_w)
    out = he.ccmul(P, keys, ct_x, ct_w, precompute_pairs(plan, B), ccmul_group(plan))
    dec = he.decrypt(P, keys, out).reshape(B, plan.MG, plan.T, P.N)
    y = np.stack([packing.decode(plan, dec[b], t) for b in range(B)])
    if B == 1:
        y = y[0]
    return LayerRunB(plan, keys, xp, wp, ct_x, ct_w, out, y)


def conv_reference(x, w, pad):
    """Direct integer cross-correlation (what a CNN layer computes), used as
    the brute-force check of the whole protocol: y[m,a,b] = sum_{c,k,l}
    x[c, a+k-pad, b+l-pad] w[m,c,k,l]."""
    x = np.asarray(x, dtype=np.int64)
    w = np.asarray(w, dtype=np.int64)
    C, H, W = x.shape
    M, _, h, _ = w.shape
    xp = np.zeros((C, H + 2 * pad, W + 2 * pad), dtype=np.int64)
    xp[:, pad:pad + H, pad:pad + W] = x
    Ho, Wo = H + 2 * pad - h + 1, W + 2 * pad - h + 1
    y = np.zeros((M, Ho, Wo), dtype=np.int64)
    for k in range(h):
        for l in range(h):
            y += np.einsum("mc,cab->mab", w[:, :, k, l], xp[:, k:k + Ho, l:l + Wo])
    return y
