"""One training step of a small CNN's homomorphic linear layers on the GPU.

Section 2 (Neural Network Training) and Section 3: every linear operation of
the forward pass and of backpropagation (input gradient and weight gradient)
is a CryptoTrain-P linear layer (offline CCMul-Precompute, online CPMul +
CCAdd, PPMul, client decryption).  The non-linear layers (ReLU, max pooling,
which the paper runs as OT protocols on secret shares) are simulated in
plaintext on the decrypted results, as are the re-quantisation of
activations to uint8 and of gradients to int8 and the loss gradient.

Network (the 512-input fully connected layer fixes the shapes):
  conv1 1->16 3x3 pad 1 on 28x28 -> ReLU -> max-pool 2 (14x14)
  conv2 16->32 3x3 pad 0 (12x12) -> ReLU -> max-pool 3 (4x4) -> FC 512->10.
Backward: FC input and weight gradients, conv2 input and weight gradients,
conv1 weight gradient (the first layer's input gradient is not needed).

Each linear operation is a convolution over the library's plan:
  input gradient   dX = conv(dY, flip(w)^T) with padding h-1-p
  weight gradient  dW[m, c] = conv over the batch used as channels:
                   input x[:, c] ([C][B, H, W]), kernel dY[:, m] ([M][B, Ho, Wo])
  fully connected  a 1x1 convolution with C input channels.
For every operation the plan with fewer polynomial products is used (both
encodings give the same exact result).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import layer
from .workloads import ConvShape, ProtocolSeeds, protocol_seeds


@dataclass(frozen=True)
class CNNSpec:
    H0: int = 28
    c1: int = 16
    c2: int = 32
    pool1: int = 2
    pool2: int = 3
    n_out: int = 10
    # re-quantisation shifts (plaintext simulation of the non-linear side)
    s1: int = 7
    s2: int = 11
    s3: int = 9
    sg: int = 6

    @property
    def H1(self):  # after pool1
        return self.H0 // self.pool1

    @property
    def H2(self):  # conv2 output (valid)
        return self.H1 - 2

    @property
    def H3(self):  # after pool2
        return self.H2 // self.pool2

    @property
    def fc_in(self):
        return self.c2 * self.H3 * self.H3


def op_shapes(s: CNNSpec, B: int):
    """(name, ConvShape, images per call) of the eight linear operations."""
    return [
        ("conv1_fwd", ConvShape(1, s.H0, s.H0, s.c1, 3, 1), B),
        ("conv2_fwd", ConvShape(s.c1, s.H1, s.H1, s.c2, 3, 0), B),
        ("fc_fwd", ConvShape(s.fc_in, 1, 1, s.n_out, 1, 0), B),
        ("fc_dx", ConvShape(s.n_out, 1, 1, s.fc_in, 1, 0), B),
        ("fc_dw", ConvShape(B, 1, 1, s.n_out, 1, 0), s.fc_in),
        ("conv2_dx", ConvShape(s.c2, s.H2, s.H2, s.c1, 3, 2), B),
        ("conv2_dw", ConvShape(B, s.H1, s.H1, s.c2, s.H2, 0), s.c1),
        ("conv1_dw", ConvShape(B, s.H0, s.H0, s.c1, s.H0, 1), 1),
    ]


def _maxpool(y, k):
    """non-overlapping k x k max pooling with the argmax (for the backward)."""
    B, C, H, W = y.shape
    Ho, Wo = H // k, W // k
    v = y[:, :, :Ho * k, :Wo * k].reshape(B, C, Ho, k, Wo, k).permute(0, 1, 2, 4, 3, 5).reshape(B, C, Ho, Wo, k * k)
    m, idx = v.max(dim=-1)
    return m, idx


def _maxpool_back(g, idx, k, H, W):
    B, C, Ho, Wo = g.shape
    z = torch.zeros((B, C, Ho, Wo, k * k), dtype=g.dtype, device=g.device)
    z.scatter_(-1, idx.unsqueeze(-1), g.unsqueeze(-1))
    z = z.reshape(B, C, Ho, Wo, k, k).permute(0, 1, 2, 4, 3, 5).reshape(B, C, Ho * k, Wo * k)
    out = torch.zeros((B, C, H, W), dtype=g.dtype, device=g.device)
    out[:, :, :Ho * k, :Wo * k] = z
    return out


def _u8(y, s):
    return torch.clamp(y >> s, 0, 255).to(torch.uint8)


def _i8(g, s):
    return torch.clamp(g >> s, -127, 127).to(torch.int8)


@dataclass
class OpRecord:
    name: str
    x: torch.Tensor        # input fed to the layer
    w: torch.Tensor        # kernel fed to the layer
    y: torch.Tensor        # decoded output
    seeds: ProtocolSeeds
    plan: layer.Plan
    player: layer.PLayer


@dataclass
class StepResult:
    y1: torch.Tensor
    y2: torch.Tensor
    y3: torch.Tensor
    dx3: torch.Tensor
    dw3: torch.Tensor
    dx2: torch.Tensor
    dw2: torch.Tensor
    dw1: torch.Tensor
    ops: dict = field(default_factory=dict)


class HETrainer:
    """The eight CryptoTrain-P linear operations of one training step."""

    def __init__(self, ctx: layer.Context, keys: layer.Keys, B: int, spec: CNNSpec = CNNSpec(),
                 encoding: str = "auto"):
        self.ctx, self.keys, self.B, self.spec = ctx, keys, B, spec
        self.plans, self.layers = {}, {}
        for name, shape, imgs in op_shapes(spec, B):
            if encoding == "auto":
                cands = [layer.Plan(ctx, shape, e) for e in ("corr", "conv")]
                cost = [p.MG * p.G * p.T for p in cands]
                best = 0 if cost[0] <= cost[1] else 1
                cands[1 - best].close()
                plan = cands[best]
            else:
                plan = layer.Plan(ctx, shape, encoding)
            self.plans[name] = plan
            self.layers[name] = layer.PLayer(ctx, keys, plan, imgs)

    def products(self):
        return {n: p.MG * p.G * p.T * self.layers[n].B for n, p in self.plans.items()}

    def _op(self, name, x, w, seed, rec):
        seeds = protocol_seeds(seed)
        y = self.layers[name].step(x.contiguous(), w.contiguous(), seeds)
        if rec is not None:
            rec[name] = OpRecord(name, x.contiguous(), w.contiguous(), y, seeds, self.plans[name], self.layers[name])
        return y

    def step(self, x0, w1, w2, w3, labels, seed: int, record: bool = False) -> StepResult:
        """x0: uint8 [B,1,H0,H0]; w1 int8 [c1,1,3,3]; w2 int8 [c2,c1,3,3];
        w3 int8 [n_out, fc_in]; labels int64 [B]."""
        s, B = self.spec, self.B
        rec = {} if record else None
        # ---- forward
        y1 = self._op("conv1_fwd", x0, w1, seed + 1, rec).clone()
        p1, i1 = _maxpool(torch.relu(y1), s.pool1)
        x1 = _u8(p1, s.s1)
        y2 = self._op("conv2_fwd", x1, w2, seed + 2, rec).clone()
        p2, i2 = _maxpool(torch.relu(y2), s.pool2)
        x2 = _u8(p2, s.s2)
        xf = x2.reshape(B, s.fc_in, 1, 1)
        y3 = self._op("fc_fwd", xf, w3.reshape(s.n_out, s.fc_in, 1, 1), seed + 3, rec).clone()
        # ---- loss gradient (plaintext): scaled logits minus a one-hot target
        logits = y3.reshape(B, s.n_out) >> s.s3
        target = torch.nn.functional.one_hot(labels, s.n_out).to(torch.int64) * 64
        g3 = torch.clamp(logits - target, -127, 127).to(torch.int8)
        # ---- backward
        dx3 = self._op("fc_dx", g3.reshape(B, s.n_out, 1, 1), w3.t().reshape(s.fc_in, s.n_out, 1, 1),
                       seed + 4, rec).clone()
        dw3 = self._op("fc_dw", x2.reshape(B, s.fc_in).t().reshape(s.fc_in, B, 1, 1),
                       g3.t().reshape(s.n_out, B, 1, 1), seed + 5, rec).clone()
        dw3 = dw3.reshape(s.fc_in, s.n_out).t()
        g2p = dx3.reshape(B, s.c2, s.H3, s.H3)
        g2 = _maxpool_back(g2p, i2, s.pool2, s.H2, s.H2) * (y2 > 0)
        g2 = _i8(g2, s.sg)
        w2f = torch.flip(w2, dims=(2, 3)).transpose(0, 1)
        dx2 = self._op("conv2_dx", g2, w2f, seed + 6, rec).clone()
        dw2 = self._op("conv2_dw", x1.transpose(0, 1), g2.transpose(0, 1), seed + 7, rec).clone()
        dw2 = dw2.transpose(0, 1)
        g1 = _maxpool_back(dx2, i1, s.pool1, s.H0, s.H0) * (y1 > 0)
        g1 = _i8(g1, s.sg)
        dw1 = self._op("conv1_dw", x0.transpose(0, 1), g1.transpose(0, 1), seed + 8, rec).clone()
        dw1 = dw1.transpose(0, 1)
        return StepResult(y1, y2, y3, dx3, dw3, dx2, dw2, dw1, rec or {})

    def close(self):
        for p in self.plans.values():
            p.close()
