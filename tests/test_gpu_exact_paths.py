"""The exact multi-word paths of the CRT kernels, bit for bit against the
oracle.

The base extension, the exact rescaling floor((t d + floor(q/2)) / q) of the
tensor product and the exact decryption take the CRT overflow count from a
fixed-point estimate of sum_i y_i / m_i and fall back to a multi-word
reconstruction only when that sum's fraction lies within a few ulps (2^-52
or less) of an integer or of one half.  Random ciphertexts almost never land
there, so these tests craft coefficients that do:

* a coefficient within a few units of Q/2 (the centring decision of the base
  extension Q -> B);
* d with [t d + floor(Q/2)]_Q within a few units of Q (the remainder r of the
  rescaling);
* d whose rounded quotient F is a small negative number (F / B within 2^-200
  of 0 from below, i.e. the CRT fraction over B within a few ulps of 1);
* ciphertexts whose [t x + floor(Q/2)]_Q lies within a few units of Q (the
  exact decryption).

The CCMul operands are a = (1, 1) and b = (b0, b1) with crafted b0, b1, so
that d0 = b0, d1 = b0 + b1, d2 = b1 exactly (a product by the constant
polynomial 1), and the digits of the rescaled d2 go through the relinearised
output as well.  Every crafted case is checked to lie in its window by exact
rational arithmetic before the GPU runs.
"""
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import he  # noqa: E402
from paper_2409_16675_gb300 import layer, native as nv, workloads as wl  # noqa: E402

RINGS = {
    "n8192_4x50": wl.RING_MID,
    "n4096_3x36": wl.RING_SMALL,
    "n2048_6x60": wl.RingSpec(2048, (60,) * 6, 65537),
    "n2048_t40": wl.RingSpec(2048, (50, 50, 50), 1099511480321),
    "n1024_12x40": wl.RingSpec(1024, (40,) * 12, 65537),  # the largest kernel size class (L > 8)
}
WINDOW = Fraction(1, 2 ** 50)


def to_np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def residues(values, q, N, rng):
    """[L][N] residues: the given integers (in [0, Q)) in the first
    coefficients, uniform elements of Z_Q after them."""
    out = np.zeros((len(q), N), dtype=np.uint64)
    for i, qi in enumerate(q):
        out[i] = rng.integers(0, qi, N, dtype=np.uint64)
        for k, v in enumerate(values):
            out[i, k] = v % qi
    return out


def frac_dist(x, y):
    """distance of the rational x from the nearest point y + k (k integer)"""
    f = (x - y) % 1
    return min(f, 1 - f)


def crafted(Q, t, aux_B):
    """(b0 values, b1 values, decryption values), each an integer in [0, Q)."""
    h = Q // 2
    tinv = pow(t, -1, Q)
    half = [h - 2, h - 1, h, h + 1, h + 2, h + 3]
    for v in half:  # centring decision: v / Q within the window of 1/2
        assert frac_dist(Fraction(v, Q), Fraction(1, 2)) < WINDOW
    near_q = [((Q - 1 - j - h) * tinv) % Q for j in range(4)]
    for v in near_q:  # remainder of the rescaling within a few units of Q
        assert Q - 8 <= (t * (v if v <= h else v - Q) + h) % Q < Q
    neg_f = []
    for j in range(4):
        xc = -((h + t - 1) // t) - j
        assert (t * xc + h) // Q == -1  # rounded quotient F = -1
        neg_f.append(xc % Q)
    # F = -1 over B: fraction 1 - 1/B
    assert 1 - Fraction(aux_B - 1, aux_B) < WINDOW
    small = [0, 1, Q - 1, 2, Q - 2]
    b0 = half + near_q + neg_f + small
    b1 = neg_f[::-1] + near_q[::-1] + small + half
    dec = near_q + [((Q - j - h) * tinv) % Q for j in range(1, 4)] + [(j * tinv - h * tinv) % Q for j in range(3)]
    return b0, b1, dec


@pytest.mark.parametrize("name", list(RINGS))
def test_ccmul_exact_fallbacks(name):
    spec = RINGS[name]
    c = layer.Context(spec)
    P = he.Params.from_spec(spec)
    Q = 1
    for qi in c.q:
        Q *= int(qi)
    B = 1
    for j in range(c.info.n_aux):
        B *= int(c.info.aux[j])
    b0, b1, _ = crafted(Q, c.t, B)
    rng = np.random.default_rng(41)
    one = np.zeros((len(c.q), c.N), dtype=np.uint64)
    one[:, 0] = 1
    a = np.stack([one, one])[None]                                  # (1, 1)
    b = np.stack([residues(b0, c.q, c.N, rng), residues(b1, c.q, c.N, rng)])[None]
    k = layer.Keys(c, 5, True)
    ok = he.keygen(P, 5, True)
    out = c.ct(1)
    nv.he_ccmul_precompute(c.h, k.h, cuda(a), 1, cuda(b), 1, [(0, 0)], 1, out)
    want = he.ccmul(P, ok, a, b, [(0, 0)], 1)
    assert np.array_equal(to_np(out), want)
    k.close()
    c.close()


@pytest.mark.parametrize("name", list(RINGS))
def test_decrypt_exact_fallback(name):
    spec = RINGS[name]
    c = layer.Context(spec)
    P = he.Params.from_spec(spec)
    Q = 1
    for qi in c.q:
        Q *= int(qi)
    _, _, dec = crafted(Q, c.t, 2 ** 64)
    h = Q // 2
    for v in dec[:7]:  # [t x + h]_Q within a few units of Q
        assert Q - 8 <= (c.t * v + h) % Q < Q
    rng = np.random.default_rng(43)
    ct = np.stack([residues(dec, c.q, c.N, rng), np.zeros((len(c.q), c.N), dtype=np.uint64)])[None]
    k = layer.Keys(c, 6, False)
    ok = he.keygen(P, 6, False)
    out = c.u64(1, c.N)
    nv.he_decrypt(c.h, k.h, cuda(ct), 1, out)
    want = he.decrypt(P, ok, ct)
    assert np.array_equal(to_np(out), want)
    k.close()
    c.close()
