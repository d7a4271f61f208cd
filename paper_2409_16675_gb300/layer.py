"""CryptoTrain-P homomorphic linear layer on the GPU, composed from the C ABI.

Section 3.2: offline, [r^x r^w] is computed by CCMul with relinearisation;
online, c = [x](w - r^w) + [w](x - r^x) + [r^x r^w] (two CPMuls and CCAdds in
one fused launch), p = (x - r^x)(w - r^w) (PPMul), and the client recovers
Dec(c) - p = x w, decoded to the convolution output.  Every step is a call
into libcryptotrain.so; this module only allocates buffers and sequences the
calls.

Batch convention: a batch of B images shares the weights and their mask r^w;
every random object of one kind is drawn from one seed with object index equal
to its position in the flattened batch.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import native as nv
from .workloads import RingSpec, ConvShape, ProtocolSeeds

ENC = {"conv": nv.HE_ENC_CONVENTIONAL, "corr": nv.HE_ENC_CORRELATED}


class Context:
    """A he_ctx for one ring."""

    def __init__(self, spec: RingSpec, device: int = 0, max_ccmul_group: int = 64, max_ccmul_scratch_bytes: float = 0,
                 max_table_cache_bytes: float = 0):
        self.spec = spec
        self.params = nv.make_params(spec.N, prime_bits=spec.prime_bits, t=spec.t, base_log2=spec.base_log2,
                                     eta=spec.eta, max_ccmul_group=max_ccmul_group, device=device,
                                     max_ccmul_scratch_bytes=max_ccmul_scratch_bytes,
                                     max_table_cache_bytes=max_table_cache_bytes)
        self.h = nv.he_setup(self.params)
        self.info = nv.he_ctx_query(self.h)
        self.N, self.L, self.t = spec.N, spec.L, spec.t
        self.q = [self.info.q[i] for i in range(self.L)]
        self.ell = self.info.ell
        self.device = torch.device("cuda", device)

    def close(self):
        if self.h:
            nv.he_ctx_destroy(self.h)
            self.h = None

    def u64(self, *shape):
        return torch.empty(shape, dtype=torch.uint64, device=self.device)

    def ct(self, n):
        return self.u64(n, 2, self.L, self.N)


class Keys:
    def __init__(self, ctx: Context, seed: int, with_relin: bool = True):
        self.ctx = ctx
        self.h = nv.he_keygen(ctx.h, seed, with_relin)

    def export(self, which):
        c = self.ctx
        shape = {nv.HE_KEY_SK: (c.N,), nv.HE_KEY_PK: (2, c.L, c.N), nv.HE_KEY_RLK: (c.ell, 2, c.L, c.N)}[which]
        out = torch.empty(shape, dtype=torch.int64 if which == nv.HE_KEY_SK else torch.uint64, device=c.device)
        nv.he_keys_export(c.h, self.h, which, out)
        return out

    def close(self):
        if self.h:
            nv.he_keys_destroy(self.h)
            self.h = None


class Plan:
    def __init__(self, ctx: Context, shape: ConvShape, encoding: str, depthwise: bool = False):
        """depthwise: output channel m reads input channel m only (M = C, weights
        diagonal in the channel indices); only the needed products run."""
        self.ctx, self.shape, self.encoding, self.depthwise = ctx, shape, encoding, depthwise
        enc = ENC[encoding] | (nv.HE_PLAN_DEPTHWISE if depthwise else 0)
        self.h = nv.he_conv_plan(ctx.h, shape.C, shape.H, shape.W, shape.M, shape.h, shape.pad, enc)
        self.info = nv.he_plan_query(self.h)
        self.T, self.G, self.MG = self.info.T, self.info.G, self.info.MG

    @property
    def products(self):
        """Polynomial products per image."""
        return self.MG * self.T * (1 if self.depthwise else self.G)

    def encode_input(self, x, batch, out):
        f = nv.he_encode_conventional if self.encoding == "conv" else nv.he_encode_correlated
        f(self.ctx.h, self.h, nv.HE_ROLE_INPUT, x, batch, out)

    def encode_kernel(self, w, out):
        f = nv.he_encode_conventional if self.encoding == "conv" else nv.he_encode_correlated
        f(self.ctx.h, self.h, nv.HE_ROLE_KERNEL, w, 1, out)

    def close(self):
        if self.h:
            nv.he_plan_destroy(self.h)
            self.h = None


@dataclass
class LayerBuffers:
    xp: torch.Tensor
    wp: torch.Tensor
    r_x: torch.Tensor
    r_w: torch.Tensor
    ct_x: torch.Tensor
    ct_w: torch.Tensor
    ct_rx: torch.Tensor
    ct_rw: torch.Tensor
    rr: torch.Tensor
    xm: torch.Tensor
    wm: torch.Tensor
    out: torch.Tensor
    p: torch.Tensor
    dec: torch.Tensor
    y: torch.Tensor


class PLayer:
    """One CryptoTrain-P linear layer over a batch of B images."""

    def __init__(self, ctx: Context, keys: Keys, plan: Plan, batch: int, with_bias: bool = False):
        """with_bias: the layer adds a per-output-channel bias (a batch-norm
        beta): its per-image plaintexts sit on the product positions
        (he_encode_output), are encrypted on the weights' stream after the
        kernel polynomials and are added to [r^x r^w] offline."""
        self.ctx, self.keys, self.plan, self.B = ctx, keys, plan, batch
        c, s = ctx, plan.shape
        nx, nw, no = batch * plan.T * plan.G, plan.MG * plan.G, batch * plan.MG * plan.T
        self.nx, self.nw, self.no = nx, nw, no
        self.with_bias = with_bias
        nb = no if with_bias else 0
        self.wp_all, self.ct_w_all = c.u64(nw + nb, c.N), c.ct(nw + nb)   # kernel rows, then bias rows
        self.buf = LayerBuffers(
            xp=c.u64(nx, c.N), wp=self.wp_all[:nw], r_x=c.u64(nx, c.N), r_w=c.u64(nw, c.N),
            ct_x=c.ct(nx), ct_w=self.ct_w_all[:nw], ct_rx=c.ct(nx), ct_rw=c.ct(nw), rr=c.ct(no),
            xm=c.u64(nx, c.N), wm=c.u64(nw, c.N), out=c.ct(no), p=c.u64(no, c.N), dec=c.u64(no, c.N),
            y=torch.empty((batch, s.M, plan.info.Ho, plan.info.Wo), dtype=torch.int64, device=c.device))

    def client_prepare(self, x, w, seeds: ProtocolSeeds, bias=None):
        """Client side: encode, draw masks, encrypt x, w (and the bias) and
        the masks.  bias: int64 [M] when the layer was built with_bias."""
        c, b = self.ctx, self.buf
        self.plan.encode_input(x, self.B, b.xp)
        self.plan.encode_kernel(w, b.wp)
        nwb = self.nw
        if self.with_bias:
            info = self.plan.info
            vals = bias.to(device=c.device, dtype=torch.int64).reshape(1, -1, 1, 1).expand(
                self.B, self.plan.shape.M, info.Ho, info.Wo).contiguous()
            nv.he_encode_output(c.h, self.plan.h, self.B, vals, self.wp_all[self.nw:])
            nwb += self.no
        nv.he_sample_masks(c.h, seeds.mask_x, self.nx, b.r_x)
        nv.he_sample_masks(c.h, seeds.mask_w, self.nw, b.r_w)
        nv.he_encrypt_many(c.h, self.keys.h, [(b.xp, self.nx, seeds.enc_x, b.ct_x),
                                               (self.wp_all, nwb, seeds.enc_w, self.ct_w_all),
                                               (b.r_x, self.nx, seeds.enc_rx, b.ct_rx),
                                               (b.r_w, self.nw, seeds.enc_rw, b.ct_rw)])
        nv.he_pt_sub(c.h, b.xp, b.r_x, self.nx * c.N, b.xm)
        nv.he_pt_sub(c.h, b.wp, b.r_w, self.nw * c.N, b.wm)

    def offline(self):
        """Server, preprocessing: [r^x r^w] by CCMul + relinearisation."""
        b = self.buf
        nv.he_ccmul_conv_precompute(self.ctx.h, self.keys.h, self.plan.h, self.B, b.ct_rx, b.ct_rw, b.rr)
        if self.with_bias:   # CCAdd of the encrypted bias into [r^x r^w]
            nv.he_ct_add(self.ctx.h, b.rr, self.ct_w_all[self.nw:], self.no, b.rr)

    def online(self):
        """Server, online: c = [x](w - r^w) + [w](x - r^x) + [r^x r^w]; p = PPMul."""
        b, c = self.buf, self.ctx
        nv.he_cpmul_conv(c.h, self.plan.h, self.B, b.ct_x, b.wm, b.ct_w, b.xm, b.rr, b.out)
        nv.he_ppmul_conv(c.h, self.plan.h, self.B, b.xm, b.wm, b.p)

    def client_finish(self):
        """Client: Dec(c) - p, decoded to [B, M, Ho, Wo]."""
        b, c = self.buf, self.ctx
        nv.he_decrypt(c.h, self.keys.h, b.out, self.no, b.dec)
        nv.he_decode(c.h, self.plan.h, self.B, b.dec, b.p, b.y)
        return b.y

    def step(self, x, w, seeds: ProtocolSeeds, bias=None):
        self.client_prepare(x, w, seeds, bias)
        self.offline()
        self.online()
        return self.client_finish()


def batch_norm_weights(gamma):
    """The batch-norm scale as a 1x1 convolution: int [C] -> diagonal [C, C, 1, 1]
    (output channel c sees only input channel c, with weight gamma_c)."""
    C = gamma.shape[0]
    w = torch.zeros((C, C, 1, 1), dtype=gamma.dtype, device=gamma.device)
    idx = torch.arange(C, device=gamma.device)
    w[idx, idx, 0, 0] = gamma
    return w


class BLayer:
    """One CryptoTrain-B linear layer over a batch of B images (Section 3.1,
    the baseline protocol that CryptoTrain-P improves on): the client encrypts
    x and w; the server multiplies the two ciphertexts online (CCMul with
    relinearisation, the products of a kernel's channel groups summed before
    the one rounding); the client decrypts and decodes x w directly."""

    def __init__(self, ctx: Context, keys: Keys, plan: Plan, batch: int):
        self.ctx, self.keys, self.plan, self.B = ctx, keys, plan, batch
        c, s = ctx, plan.shape
        nx, nw, no = batch * plan.T * plan.G, plan.MG * plan.G, batch * plan.MG * plan.T
        self.nx, self.nw, self.no = nx, nw, no
        self.xp, self.wp = c.u64(nx, c.N), c.u64(nw, c.N)
        self.ct_x, self.ct_w, self.out = c.ct(nx), c.ct(nw), c.ct(no)
        self.dec = c.u64(no, c.N)
        self.y = torch.empty((batch, s.M, plan.info.Ho, plan.info.Wo), dtype=torch.int64, device=c.device)

    def client_prepare(self, x, w, seeds: ProtocolSeeds):
        """Client: encode and encrypt x and w."""
        c = self.ctx
        self.plan.encode_input(x, self.B, self.xp)
        self.plan.encode_kernel(w, self.wp)
        nv.he_encrypt_many(c.h, self.keys.h, [(self.xp, self.nx, seeds.enc_x, self.ct_x),
                                              (self.wp, self.nw, seeds.enc_w, self.ct_w)])

    def online(self):
        """Server, online: [x][w] by CCMul + relinearisation."""
        nv.he_ccmul_conv_precompute(self.ctx.h, self.keys.h, self.plan.h, self.B, self.ct_x, self.ct_w, self.out)

    def client_finish(self):
        """Client: Dec([x][w]) decoded to [B, M, Ho, Wo]."""
        c = self.ctx
        nv.he_decrypt(c.h, self.keys.h, self.out, self.no, self.dec)
        nv.he_decode(c.h, self.plan.h, self.B, self.dec, None, self.y)
        return self.y

    def step(self, x, w, seeds: ProtocolSeeds):
        self.client_prepare(x, w, seeds)
        self.online()
        return self.client_finish()
