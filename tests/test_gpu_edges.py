"""Edge cases of the boundary on the GPU: zero-sized calls leave every buffer
untouched; degenerate layer shapes (a 1x1 image, a kernel as large as the
image, single channels) and the largest ring of the served workload
(N = 16384, eight 60-bit limbs) are bit-exact against the oracle and decode
to the exact convolution."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import he, packing, protocol  # noqa: E402
from paper_2409_16675_gb300 import layer, native as nv, workloads as wl  # noqa: E402

SENT = 0x5A5A5A5A5A5A5A5A


def to_np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def sentinel(t):
    t.view(torch.int64).fill_(SENT)
    return t


def untouched(t):
    return bool((to_np(t.view(torch.int64)) == SENT).all())


def test_zero_sized_calls_touch_nothing():
    c = layer.Context(wl.RingSpec(1024, (40, 40), 65537))
    k = layer.Keys(c, 3, True)
    plan = layer.Plan(c, wl.ConvShape(2, 6, 6, 3, 3, 1), "corr")
    ct, pt, out_ct, out_pt = c.ct(2), c.u64(2, c.N), sentinel(c.ct(2)), sentinel(c.u64(2, c.N))
    y = sentinel(torch.empty((1, 3, 6, 6), dtype=torch.int64, device="cuda"))
    x = torch.zeros((1, 2, 6, 6), dtype=torch.uint8, device="cuda")
    nv.he_encrypt(c.h, k.h, pt, 0, 1, out_ct)
    nv.he_encrypt_many(c.h, k.h, [(pt, 0, 1, out_ct), (pt, 0, 2, out_ct)])
    nv.he_encrypt_symmetric(c.h, k.h, pt, 0, 1, out_ct)
    nv.he_expand_symmetric(c.h, 1, 0, ct, out_ct)
    nv.he_decrypt(c.h, k.h, ct, 0, out_pt)
    nv.he_sample_masks(c.h, 1, 0, out_pt)
    nv.he_pt_sub(c.h, pt, pt, 0, out_pt)
    nv.he_ct_add(c.h, ct, ct, 0, out_ct)
    nv.he_cpmul_conv(c.h, plan.h, 0, ct, pt, ct, pt, ct, out_ct)
    nv.he_ccmul_conv_precompute(c.h, k.h, plan.h, 0, ct, ct, out_ct)
    nv.he_ccmul_precompute(c.h, k.h, ct, 1, ct, 1, [], 1, out_ct)
    nv.he_ppmul_conv(c.h, plan.h, 0, pt, pt, out_pt)
    nv.he_decode(c.h, plan.h, 0, pt, None, y)
    nv.he_encode_correlated(c.h, plan.h, nv.HE_ROLE_INPUT, x, 0, out_pt)
    nv.he_encode_output(c.h, plan.h, 0, y, out_pt)
    assert untouched(out_ct) and untouched(out_pt) and untouched(y)
    k.close()
    plan.close()
    c.close()


DEGENERATE = [
    wl.ConvShape(1, 1, 1, 1, 1, 0),     # a 1x1 image, a 1x1 kernel
    wl.ConvShape(3, 5, 5, 2, 5, 0),     # kernel as large as the image: one output
    wl.ConvShape(1, 7, 3, 1, 3, 1),     # one channel in and out, a narrow image
    wl.ConvShape(4, 2, 9, 5, 1, 0),     # two rows, many output channels
]


@pytest.mark.parametrize("enc", ["corr", "conv"])
@pytest.mark.parametrize("shape", DEGENERATE, ids=lambda s: "%dx%dx%d_m%d_k%d_p%d" % (s.C, s.H, s.W, s.M, s.h, s.pad))
def test_degenerate_layers(enc, shape):
    spec = wl.RingSpec(1024, (40, 40, 40), 65537)
    c = layer.Context(spec)
    seeds = wl.protocol_seeds(shape.C * 100 + shape.H * 10 + shape.h)
    x = wl.activations(11, (2, shape.C, shape.H, shape.W))
    w = wl.weights(12, (shape.M, shape.C, shape.h, shape.h))
    keys = layer.Keys(c, seeds.keys, True)
    plan = layer.Plan(c, shape, enc)
    pl = layer.PLayer(c, keys, plan, 2)
    y = to_np(pl.step(torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda(), seeds))
    op = packing.make_plan(enc, c.N, shape.C, shape.H, shape.W, shape.M, shape.h, shape.pad)
    ref = protocol.run_layer(he.Params.from_spec(spec), op, x, w, seeds)
    assert np.array_equal(to_np(pl.buf.rr), ref.rr)
    assert np.array_equal(to_np(pl.buf.out), ref.out)
    for b in range(2):
        assert np.array_equal(y[b], protocol.conv_reference(x[b], w, shape.pad))
    keys.close()
    plan.close()
    c.close()


def test_largest_served_ring():
    """N = 16384 with eight 60-bit limbs (480 bits, the largest ring of the
    served workload): keys, encryption, one CCMul with relinearisation and a
    small layer, bit-exact against the oracle."""
    spec = wl.RingSpec(16384, (60,) * 8, 65537)
    c = layer.Context(spec)
    P = he.Params.from_spec(spec)
    assert [int(q) for q in c.q] == [int(q) for q in P.q]
    seeds = wl.protocol_seeds(808)
    keys = layer.Keys(c, seeds.keys, True)
    ok = he.keygen(P, seeds.keys, True)
    pk = to_np(keys.export(nv.HE_KEY_PK))
    assert np.array_equal(pk, ok.pk)
    shape = wl.ConvShape(1, 8, 8, 2, 3, 1)
    x = wl.activations(809, (1, 1, 8, 8))
    w = wl.weights(810, (2, 1, 3, 3))
    plan = layer.Plan(c, shape, "corr")
    pl = layer.PLayer(c, keys, plan, 1)
    y = to_np(pl.step(torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda(), seeds))
    op = packing.make_plan("corr", c.N, 1, 8, 8, 2, 3, 1)
    ref = protocol.run_layer(P, op, x, w, seeds, keys=ok)
    assert np.array_equal(to_np(pl.buf.ct_x), ref.ct_x)
    assert np.array_equal(to_np(pl.buf.rr), ref.rr)
    assert np.array_equal(to_np(pl.buf.out), ref.out)
    assert np.array_equal(y[0], protocol.conv_reference(x[0], w, 1))
    keys.close()
    plan.close()
    c.close()


def test_keys_and_plans_of_another_context_are_refused():
    """Keys carry the parameter fingerprint of their context and plans their
    ring degree: every call given foreign ones fails before any device work,
    and the output buffers stay untouched."""
    a = layer.Context(wl.RingSpec(1024, (40, 40), 65537))
    b = layer.Context(wl.RingSpec(1024, (40, 45), 65537))   # same N and L, other primes
    c = layer.Context(wl.RingSpec(2048, (40, 40), 65537))   # another ring degree
    assert nv.he_ctx_fingerprint(a.h) != nv.he_ctx_fingerprint(b.h)
    ka = layer.Keys(a, 3, True)
    pa = layer.Plan(a, wl.ConvShape(2, 6, 6, 3, 3, 1), "corr")
    for ctx in (b, c):
        pt = ctx.u64(1, ctx.N)
        pt.zero_()
        out_ct = sentinel(ctx.ct(1))
        out_pt = sentinel(ctx.u64(1, ctx.N))
        calls = [
            lambda: nv.he_encrypt(ctx.h, ka.h, pt, 1, 1, out_ct),
            lambda: nv.he_encrypt_symmetric(ctx.h, ka.h, pt, 1, 1, out_ct),
            lambda: nv.he_decrypt(ctx.h, ka.h, out_ct, 1, out_pt),
            lambda: nv.he_ccmul_precompute(ctx.h, ka.h, out_ct, 1, out_ct, 1, [(0, 0)], 1, out_ct),
        ]
        if ctx is c:
            calls += [
                lambda: nv.he_cpmul_conv(ctx.h, pa.h, 1, out_ct, pt, None, None, None, out_ct),
                lambda: nv.he_ppmul_conv(ctx.h, pa.h, 1, pt, pt, out_pt),
                lambda: nv.he_encode_correlated(ctx.h, pa.h, nv.HE_ROLE_INPUT,
                                                torch.zeros((1, 2, 6, 6), dtype=torch.uint8, device="cuda"), 1, out_pt),
            ]
        for call in calls:
            with pytest.raises(nv.HEError):
                call()
        assert untouched(out_ct) and untouched(out_pt)
    # the same objects still work on their own context
    ct = a.ct(1)
    m = torch.zeros((1, a.N), dtype=torch.uint64, device="cuda")
    nv.he_encrypt(a.h, ka.h, m, 1, 1, ct)
    back = a.u64(1, a.N)
    nv.he_decrypt(a.h, ka.h, ct, 1, back)
    assert not to_np(back.view(torch.int64)).any()
    ka.close()
    pa.close()
    for ctx in (a, b, c):
        ctx.close()
