"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This module holds only input *generators* and workload descriptions (ring
sizes, prime bit sizes, plaintext modulus, tensor shapes, seeds).  It contains
none of the homomorphic arithmetic: prime search, keys, encodings and products
are computed separately by the CUDA library and by the CPU oracle.

The paper trains on MNIST, CIFAR-10 and Tiny-ImageNet (Section 4, Datasets and
models); none of them is available here, so every tensor is a seeded uniform
stand-in with the same shape and value range: uint8 activations in [0, 255]
and int8 weights in [-8, 7].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 0x240916675


@dataclass(frozen=True)
class RingSpec:
    """RLWE/BFV ring: degree N, one prime bit size per RNS limb, plaintext
    modulus t, relinearisation digit size (bits) and CBD parameter eta."""

    N: int
    prime_bits: tuple
    t: int
    base_log2: int = 16
    eta: int = 21

    @property
    def L(self) -> int:
        return len(self.prime_bits)


@dataclass(frozen=True)
class ConvShape:
    """2-D convolution, stride 1: C input channels of H x W, M output channels,
    square h x h kernel, zero padding p on every side."""

    C: int
    H: int
    W: int
    M: int
    h: int
    pad: int = 0

    @property
    def Ho(self) -> int:
        return self.H + 2 * self.pad - self.h + 1

    @property
    def Wo(self) -> int:
        return self.W + 2 * self.pad - self.h + 1


# Ring parameters of the synthetic CNN layers.
# 4096 / 3 x 36-bit / t = 65537: a single plain encrypted conv layer.
RING_SMALL = RingSpec(4096, (36, 36, 36), 65537)
# 8192 / 4 x 50-bit / t = largest 20-bit prime = 1 mod 16384.
RING_MID = RingSpec(8192, (50, 50, 50, 50), 1032193)
# Same ring with a 40-bit t so that training-step gradient sums stay exact.
RING_TRAIN = RingSpec(8192, (50, 50, 50, 50), 1099511480321)


@dataclass(frozen=True)
class LayerWorkload:
    name: str
    ring: RingSpec
    shape: ConvShape
    encoding: str          # "conv" (row-major, Cheetah-style) or "corr" (correlated)
    seed: int
    extra: dict = field(default_factory=dict)


# one 1x28x28 image, 4 output channels, 3x3, valid, row-major encoding, CPMul only
CONV_SMALL = LayerWorkload("conv1x28x28_m4_k3_valid_N4096", RING_SMALL,
                           ConvShape(1, 28, 28, 4, 3, 0), "conv", MASTER_SEED + 1)
# one 3x32x32 image, 16 output channels, 3x3, same padding, correlated encoding,
# offline CCMul-Precompute + online CPMul
CONV_MID = LayerWorkload("conv3x32x32_m16_k3_same_N8192", RING_MID,
                         ConvShape(3, 32, 32, 16, 3, 1), "corr", MASTER_SEED + 2)


def rng(seed: int) -> np.random.Generator:
    """NumPy Philox stream for tensor inputs."""
    return np.random.Generator(np.random.Philox(seed))


def activations(seed: int, shape) -> np.ndarray:
    """uint8 activations, uniform in [0, 255]."""
    return rng(seed).integers(0, 256, size=shape, dtype=np.uint8)


def weights(seed: int, shape) -> np.ndarray:
    """int8 weights, uniform in [-8, 7]."""
    return rng(seed).integers(-8, 8, size=shape, dtype=np.int8)


def layer_inputs(w: LayerWorkload, batch: int = 1):
    """x: uint8 [batch, C, H, W]; w: int8 [M, C, h, h]."""
    s = w.shape
    x = activations(w.seed, (batch, s.C, s.H, s.W))
    k = weights(w.seed + 1000, (s.M, s.C, s.h, s.h))
    return x, k


def uniform_mod(seed: int, shape, modulus: int) -> np.ndarray:
    """uint64 values uniform in [0, modulus) (test messages / plaintexts)."""
    return rng(seed).integers(0, modulus, size=shape, dtype=np.uint64)


@dataclass(frozen=True)
class ProtocolSeeds:
    """Seeds of every random object of one CryptoTrain-P linear layer: keys,
    the encryptions of x, w and the two masks, and the masks themselves."""

    keys: int
    enc_x: int
    enc_w: int
    mask_x: int
    mask_w: int
    enc_rx: int
    enc_rw: int


def protocol_seeds(seed: int) -> ProtocolSeeds:
    return ProtocolSeeds(seed * 7 + 1, seed * 7 + 2, seed * 7 + 3, seed * 7 + 4, seed * 7 + 5,
                         seed * 7 + 6, seed * 7 + 7)


@dataclass(frozen=True)
class BatchJob:
    """One ct x pt convolution job of the batched form."""

    ring: RingSpec
    shape: ConvShape
    encoding: str
    seed: int


def batched_jobs(seed: int = MASTER_SEED + 4, n_jobs: int = 256, channels=(3, 16, 32, 64, 128),
                 sizes=(8, 16, 32), kernels=(1, 3, 5), degrees=(4096, 8192), limbs=(2, 5), bits=(36, 60)):
    """Uneven CNN-layer jobs: C and M uniform over `channels`, H = W uniform over
    `sizes`, kernel uniform over `kernels` with same padding (h-1)/2, N uniform
    over `degrees`, L uniform in `limbs`, each limb's prime size uniform in
    `bits`, encoding conventional or correlated with equal probability,
    t = 65537."""
    r = rng(seed)
    jobs = []
    for j in range(n_jobs):
        C = int(r.choice(channels))
        M = int(r.choice(channels))
        H = int(r.choice(sizes))
        h = int(r.choice(kernels))
        N = int(r.choice(degrees))
        L = int(r.integers(limbs[0], limbs[1] + 1))
        pb = tuple(int(b) for b in r.integers(bits[0], bits[1] + 1, size=L))
        enc = "corr" if r.integers(0, 2) else "conv"
        jobs.append(BatchJob(RingSpec(N, pb, 65537), ConvShape(C, H, H, M, h, (h - 1) // 2), enc, seed * 1000 + j))
    return jobs


def served_clients(seed: int = MASTER_SEED + 5, n_clients: int = 64):
    """Clients of the served form: each owns one layer drawn as in the batched
    form (channels {3,16,32,64,128}, spatial {8,16,32}, kernel {1,3,5}, both
    encodings) on its own ring: N uniform over {4096, 8192, 16384}, 2-8 limbs
    whose prime sizes are uniform in [36, 60] bits, t = 65537."""
    return batched_jobs(seed=seed, n_jobs=n_clients, degrees=(4096, 8192, 16384), limbs=(2, 8), bits=(36, 60))


def poisson_arrivals(seed: int, rate: float, seconds: float, n_clients: int):
    """Open-loop arrivals: exponential inter-arrival times of mean 1/rate over
    `seconds`, each arrival from a client drawn uniformly; returns (times,
    clients) as numpy arrays."""
    r = rng(seed)
    n = int(rate * seconds * 1.5) + 16
    t = np.cumsum(r.exponential(1.0 / rate, size=n))
    t = t[t < seconds]
    return t, r.integers(0, n_clients, size=len(t))
