"""The homomorphic linear layers of one CNN training step (forward, input
gradient, weight gradient) on the GPU: every decoded result equals the exact
integer computation at full size (batch 64, N = 8192, four 50-bit limbs,
40-bit t), and every ciphertext equals the oracle's bit for bit on a small
network."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import he, packing, protocol  # noqa: E402
from paper_2409_16675_gb300 import layer, training, workloads as wl  # noqa: E402


def inputs(spec, B, seed):
    rng = np.random.default_rng(seed)
    x0 = rng.integers(0, 256, (B, 1, spec.H0, spec.H0), dtype=np.uint8)
    w1 = rng.integers(-8, 8, (spec.c1, 1, 3, 3), dtype=np.int8)
    w2 = rng.integers(-8, 8, (spec.c2, spec.c1, 3, 3), dtype=np.int8)
    w3 = rng.integers(-8, 8, (spec.n_out, spec.fc_in), dtype=np.int8)
    lab = rng.integers(0, spec.n_out, (B,), dtype=np.int64)
    return [torch.from_numpy(a).cuda() for a in (x0, w1, w2, w3, lab)]


def conv_int(x, w, pad):
    """exact int64 cross-correlation over a batch (numpy)."""
    x = x.cpu().numpy().astype(np.int64)
    w = w.cpu().numpy().astype(np.int64)
    return np.stack([protocol.conv_reference(x[b], w, pad) for b in range(x.shape[0])])


def test_training_step_full_size_equals_integer_computation():
    spec = training.CNNSpec()
    B = 64
    ctx = layer.Context(wl.RING_TRAIN)
    keys = layer.Keys(ctx, 31, True)
    tr = training.HETrainer(ctx, keys, B, spec)
    x0, w1, w2, w3, lab = inputs(spec, B, 5)
    r = tr.step(x0, w1, w2, w3, lab, seed=1000, record=True)
    torch.cuda.synchronize()
    ops = r.ops
    # every operation's decoded output is the exact integer convolution of what it was fed
    for name, rec in ops.items():
        want = conv_int(rec.x, rec.w, rec.plan.shape.pad)
        assert np.array_equal(rec.y.cpu().numpy(), want), name
    # and the plaintext glue is the network's backpropagation
    y1 = conv_int(x0, w1, 1)
    assert np.array_equal(r.y1.cpu().numpy(), y1)
    assert r.dw1.shape == (spec.c1, 1, 3, 3) and r.dw2.shape == (spec.c2, spec.c1, 3, 3)
    assert r.dw3.shape == (spec.n_out, spec.fc_in)
    g3 = ops["fc_dx"].x.reshape(B, spec.n_out).cpu().numpy().astype(np.int64)
    x2 = ops["fc_fwd"].x.reshape(B, spec.fc_in).cpu().numpy().astype(np.int64)
    assert np.array_equal(r.dw3.cpu().numpy(), g3.T @ x2)
    assert np.array_equal(r.dx3.reshape(B, spec.fc_in).cpu().numpy(),
                          g3 @ w3.cpu().numpy().astype(np.int64))
    tr.close()
    keys.close()
    ctx.close()


def test_training_ops_bits_equal_oracle_small_network():
    spec = training.CNNSpec(H0=10, c1=2, c2=3, pool1=2, pool2=2, n_out=3, s1=4, s2=5, s3=3, sg=2)
    B = 2
    ring = wl.RingSpec(1024, (50, 50, 50, 50), 1099511480321)
    ctx = layer.Context(ring)
    keys = layer.Keys(ctx, 17, True)
    tr = training.HETrainer(ctx, keys, B, spec)
    x0, w1, w2, w3, lab = inputs(spec, B, 9)
    r = tr.step(x0, w1, w2, w3, lab, seed=77, record=True)
    torch.cuda.synchronize()
    P = he.Params(ring.N, ctx.q, ring.t)
    okeys = he.keygen(P, 17, True)
    for name, rec in r.ops.items():
        s = rec.plan.shape
        op = packing.make_plan(rec.plan.encoding, ring.N, s.C, s.H, s.W, s.M, s.h, s.pad)
        ref = protocol.run_layer(P, op, rec.x.cpu().numpy(), rec.w.cpu().numpy(), rec.seeds, keys=okeys)
        assert np.array_equal(rec.player.buf.out.cpu().numpy(), ref.out), name
        y = rec.y.cpu().numpy()
        assert np.array_equal(y if y.shape[0] > 1 else y[0], ref.y), name
    tr.close()
    keys.close()
    ctx.close()
