"""GPU parity: every entry point of libcryptotrain.so against the CPU oracle,
bit for bit (exact integer arithmetic, identical seeds)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import he, packing, protocol  # noqa: E402
from paper_2409_16675_gb300 import layer, native as nv, workloads as wl  # noqa: E402

RINGS = {
    "n4096": wl.RING_SMALL,
    "n8192": wl.RING_MID,
    "n1024": wl.RingSpec(1024, (40, 45), 65537),
    "n16384": wl.RingSpec(16384, (60, 60, 55), 65537),
    "n2048_t40": wl.RingSpec(2048, (50, 50, 50), 1099511480321),
    # base-2^32 digits: four small primes in the key switch
    "n8192_b32": wl.RingSpec(8192, (50, 50, 50, 50), 65537, 32),
    # N = 16384 with three small primes (the 1024-thread kernels)
    "n16384_np3": wl.RingSpec(16384, (50, 50), 65537),
    # 16 digits: the key switch's 64-bit sums are folded once (every 14 terms)
    "n4096_l5": wl.RingSpec(4096, (50, 50, 50, 50, 50), 65537),
    # a limb below 2^31: the key switch runs over the limbs
    "n4096_q30": wl.RingSpec(4096, (30, 50, 50), 65537),
    # base-2^8 digits of a 64-bit q: two small primes suffice
    "n1024_np2": wl.RingSpec(1024, (32, 32), 65537, 8),
    # four small primes and 15 digits: the sums are folded at the last term
    "n1024_b32_l9": wl.RingSpec(1024, (50,) * 9, 65537, 32),
}
_CTX = {}


def ctx_for(name):
    if name not in _CTX:
        c = layer.Context(RINGS[name])
        _CTX[name] = c
    return _CTX[name]


def oparams(c):
    return he.Params(c.N, c.q, c.t, c.spec.base_log2, c.spec.eta)


def to_np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name", list(RINGS))
def test_primes_match_oracle(name):
    c = ctx_for(name)
    assert c.q == he.gen_primes(c.N, list(c.spec.prime_bits))
    for p in [c.info.aux[j] for j in range(c.info.n_aux)]:
        assert he.is_prime(p) and p % (2 * c.N) == 1 and p not in c.q


@pytest.mark.parametrize("name", ["n4096", "n8192", "n1024", "n16384"])
def test_keygen_bits(name):
    c = ctx_for(name)
    k = layer.Keys(c, 1234, True)
    ok = he.keygen(oparams(c), 1234, True)
    assert np.array_equal(to_np(k.export(nv.HE_KEY_SK)), ok.sk)
    assert np.array_equal(to_np(k.export(nv.HE_KEY_PK)), ok.pk)
    assert np.array_equal(to_np(k.export(nv.HE_KEY_RLK)), ok.rlk)
    k.close()


@pytest.mark.parametrize("name", list(RINGS))
def test_encrypt_decrypt_bits(name):
    c = ctx_for(name)
    P = oparams(c)
    k = layer.Keys(c, 77, False)
    ok = he.keygen(P, 77, False)
    n = 3
    m = wl.uniform_mod(5, (n, c.N), c.t)
    m[0, :5] = [0, 1, c.t - 1, c.t // 2, c.t // 2 + 1]
    ct = c.ct(n)
    nv.he_encrypt(c.h, k.h, cuda(m), n, 99, ct)
    oct_ = he.encrypt(P, ok, m, 99)
    assert np.array_equal(to_np(ct), oct_)
    out = c.u64(n, c.N)
    nv.he_decrypt(c.h, k.h, cuda(oct_), n, out)
    assert np.array_equal(to_np(out), m)
    k.close()


def test_encrypt_many_equals_separate_calls():
    """he_encrypt_many shares the launches of several groups (own seeds and
    counts, one of them empty) and gives the bits of separate he_encrypt calls."""
    c = ctx_for("n4096")
    keys = layer.Keys(c, 77, False)
    counts, seeds = [3, 0, 2, 5], [101, 102, 103, 104]
    pts = [cuda(wl.uniform_mod(200 + g, (max(n, 1), c.N), c.t)) for g, n in enumerate(counts)]
    many = [c.ct(max(n, 1)).zero_() for n in counts]
    nv.he_encrypt_many(c.h, keys.h, [(pts[g], counts[g], seeds[g], many[g]) for g in range(4)])
    for g in range(4):
        if counts[g] == 0:
            assert not to_np(many[g]).any()     # an empty group writes nothing
            continue
        one = c.ct(counts[g])
        nv.he_encrypt(c.h, keys.h, pts[g], counts[g], seeds[g], one)
        assert np.array_equal(to_np(many[g]), to_np(one))
    with pytest.raises(nv.HEError):
        nv.he_encrypt_many(c.h, keys.h, [(pts[0], 3, 1, many[0])] * 5)   # at most 4 groups
    keys.close()


@pytest.mark.parametrize("name", ["n4096", "n8192", "n16384"])
def test_symmetric_encryption_bits(name):
    """Seed-compressed secret-key encryption: c0 and the expanded ciphertext
    equal the oracle's bit for bit and decrypt to the message."""
    c = ctx_for(name)
    P = oparams(c)
    keys = layer.Keys(c, 31, False)
    okeys = he.keygen(P, 31, False)
    n, seed = 3, 4242
    m = wl.uniform_mod(55, (n, c.N), c.t)
    c0 = c.u64(n, c.L, c.N)
    nv.he_encrypt_symmetric(c.h, keys.h, cuda(m), n, seed, c0)
    ct = c.ct(n)
    nv.he_expand_symmetric(c.h, seed, n, c0, ct)
    ref_c0 = he.encrypt_symmetric(P, okeys, m, seed)
    assert np.array_equal(to_np(c0), ref_c0)
    assert np.array_equal(to_np(ct), he.expand_symmetric(P, seed, ref_c0))
    dec = c.u64(n, c.N)
    nv.he_decrypt(c.h, keys.h, ct, n, dec)
    assert np.array_equal(to_np(dec), m)
    keys.close()


def test_decrypt_rounding_edges():
    # ciphertexts (x, 0) with x at the rounding boundaries of floor((t x + q/2)/q)
    c = ctx_for("n4096")
    P = oparams(c)
    k = layer.Keys(c, 3, False)
    ok = he.keygen(P, 3, False)
    Q, t = P.Q, P.t
    xs = [0, 1, Q - 1, Q // 2, Q // 2 + 1, Q // (2 * t), Q // (2 * t) + 1, (Q // t) * 7 + Q // (2 * t) + 1]
    rng = np.random.default_rng(0)
    xs += [int(v) for v in rng.integers(0, 2 ** 62, 50)] + [Q - int(v) for v in rng.integers(1, 2 ** 40, 20)]
    ct = np.zeros((1, 2, P.L, P.N), dtype=np.uint64)
    for j, x in enumerate(xs):
        for i, qi in enumerate(P.q):
            ct[0, 0, i, j] = x % qi
    out = c.u64(1, c.N)
    nv.he_decrypt(c.h, k.h, cuda(ct), 1, out)
    assert np.array_equal(to_np(out), he.decrypt(P, ok, ct))
    k.close()


@pytest.mark.parametrize("name", ["n8192", "n1024", "n16384", "n2048_t40"])
def test_masks_bits(name):
    c = ctx_for(name)
    out = c.u64(4, c.N)
    nv.he_sample_masks(c.h, 2024, 4, out)
    assert np.array_equal(to_np(out), he.sample_masks(oparams(c), 2024, 4))


SHAPES = [
    # (C, H, W, M, h, pad) -- several tiles / groups at small N, ragged tails,
    # packed output channels (small images, fully connected shapes)
    (3, 12, 11, 2, 3, 1),
    (5, 20, 17, 3, 3, 2),
    (2, 7, 9, 2, 5, 4),
    (4, 1, 1, 3, 1, 0),
    (1, 28, 28, 4, 3, 0),
    (40, 1, 1, 37, 1, 0),
    (3, 4, 5, 11, 3, 1),
]


@pytest.mark.parametrize("enc", ["conv", "corr"])
@pytest.mark.parametrize("shape", SHAPES)
def test_plan_and_encoding_match_oracle(enc, shape):
    c = ctx_for("n1024")
    C, H, W, M, h, pad = shape
    pl = layer.Plan(c, wl.ConvShape(*shape), enc)
    op = packing.make_plan(enc, c.N, C, H, W, M, h, pad)
    i = pl.info
    assert (i.Cn, i.G, i.th, i.tw, i.Th, i.Tw, i.T) == (op.Cn, op.G, op.th, op.tw, op.Th, op.Tw, op.T)
    assert (i.Mn, i.MG) == (op.Mn, op.MG) and (op.Mn == 1 or i.Sout == op.Sout)
    if enc == "conv":
        assert (i.Hn, i.Wn, i.Ooff) == (op.Hn, op.Wn, op.Ooff)
    else:
        assert (i.O, i.S) == (op.O, op.S)
    B = 2
    x = wl.activations(11, (B, C, H, W))
    w = wl.weights(12, (M, C, h, h))
    xp = c.u64(B * op.T * op.G, c.N)
    wp = c.u64(op.MG * op.G, c.N)
    pl.encode_input(cuda(x), B, xp)
    pl.encode_kernel(cuda(w), wp)
    want_x = np.concatenate([packing.encode_input(op, x[b], c.t).reshape(-1, c.N) for b in range(B)])
    assert np.array_equal(to_np(xp), want_x)
    assert np.array_equal(to_np(wp), packing.encode_kernel(op, w, c.t).reshape(-1, c.N))
    # decode: random polys, with a subtracted operand
    rng = np.random.default_rng(1)
    z = rng.integers(0, c.t, (B, op.MG, op.T, c.N), dtype=np.uint64)
    s = rng.integers(0, c.t, (B, op.MG, op.T, c.N), dtype=np.uint64)
    y = torch.empty((B, M, op.Ho, op.Wo), dtype=torch.int64, device="cuda")
    nv.he_decode(c.h, pl.h, B, cuda(z), cuda(s), y)
    tt = np.uint64(c.t)
    want = np.stack([packing.decode(op, (z[b] + tt - s[b]) % tt, c.t) for b in range(B)])
    assert np.array_equal(to_np(y), want)
    pl.close()


@pytest.mark.parametrize("name", ["n1024", "n8192"])
@pytest.mark.parametrize("families", ["x", "w", "both"])
def test_cpmul_conv_bits(name, families):
    c = ctx_for(name)
    P = oparams(c)
    k = layer.Keys(c, 5, False)
    ok = he.keygen(P, 5, False)
    shape = wl.ConvShape(5, 20, 17, 3, 3, 2) if c.N == 1024 else wl.ConvShape(16, 32, 32, 4, 3, 1)
    pl = layer.Plan(c, shape, "corr")
    T, G, M, B = pl.T, pl.G, pl.MG, 2
    nx, nw = B * T * G, M * G
    rng = np.random.default_rng(3)
    mx = rng.integers(0, c.t, (nx, c.N), dtype=np.uint64)
    mw = rng.integers(0, c.t, (nw, c.N), dtype=np.uint64)
    ptw = rng.integers(0, c.t, (nw, c.N), dtype=np.uint64)
    ptx = rng.integers(0, c.t, (nx, c.N), dtype=np.uint64)
    ptw[0, :3] = [c.t - 1, (c.t - 1) // 2, (c.t + 1) // 2]
    ctx_ = he.encrypt(P, ok, mx, 1)
    ctw = he.encrypt(P, ok, mw, 2)
    add = he.encrypt(P, ok, rng.integers(0, c.t, (B * M * T, c.N), dtype=np.uint64), 3)
    use_x, use_w = families in ("x", "both"), families in ("w", "both")
    out = c.ct(B * M * T)
    nv.he_cpmul_conv(c.h, pl.h, B, cuda(ctx_) if use_x else None, cuda(ptw) if use_x else None,
                     cuda(ctw) if use_w else None, cuda(ptx) if use_w else None, cuda(add), out)
    terms = []
    for b in range(B):
        for m in range(M):
            for t in range(T):
                tl = []
                for g in range(G):
                    xi = (b * T + t) * G + g
                    if use_x:
                        tl.append((xi, m * G + g))
                    if use_w:
                        tl.append((nx + m * G + g, nw + xi))
                terms.append(tl)
    want = he.cpmul_terms(P, np.concatenate([ctx_, ctw]), np.concatenate([ptw, ptx]), terms, add=add)
    assert np.array_equal(to_np(out), want)
    k.close()
    pl.close()


# small primes of the relinearisation key switch per ring (0: over the limbs,
# which a limb below 2^31 forces)
KS_PRIMES = {"n1024": 3, "n4096": 3, "n8192": 3, "n2048_t40": 3, "n16384": 4, "n8192_b32": 4, "n16384_np3": 3,
             "n4096_l5": 3, "n4096_q30": 0, "n1024_np2": 2, "n1024_b32_l9": 4}


@pytest.mark.parametrize("name,group", [("n1024", 1), ("n1024", 3), ("n4096", 2), ("n8192", 1), ("n2048_t40", 2),
                                        ("n16384", 1), ("n8192_b32", 2), ("n16384_np3", 1), ("n4096_l5", 2),
                                        ("n4096_q30", 1), ("n1024_np2", 2), ("n1024_b32_l9", 1)])
def test_ccmul_bits(name, group):
    """CCMul with relinearisation equals the oracle bit for bit on every key
    switch: two, three and four small primes at N = 1024 to 16384 (sums
    folded at 15 and 16 digits), and over the limbs where a limb is below
    2^31."""
    c = ctx_for(name)
    assert nv.he_ctx_query(c.h).ks_primes == KS_PRIMES[name]
    P = oparams(c)
    k = layer.Keys(c, 8, True)
    ok = he.keygen(P, 8, True)
    rng = np.random.default_rng(group)
    a = he.encrypt(P, ok, rng.integers(0, c.t, (3, c.N), dtype=np.uint64), 4)
    b = he.encrypt(P, ok, rng.integers(0, c.t, (4, c.N), dtype=np.uint64), 5)
    pairs = [(0, 1), (2, 3), (1, 0), (2, 2), (0, 0), (1, 3)][: 2 * group]
    out = c.ct(len(pairs) // group)
    nv.he_ccmul_precompute(c.h, k.h, cuda(a), 3, cuda(b), 4, pairs, group, out)
    want = he.ccmul(P, ok, a, b, pairs, group)
    assert np.array_equal(to_np(out), want)
    k.close()


@pytest.mark.parametrize("name", ["n8192", "n8192_b32", "n16384"])
def test_ccmul_key_switch_near_its_bound(name):
    """With a relinearisation key whose every coefficient is q_i - 1 (imported
    on both sides), coefficient N - 1 of sum_j D_j rlk_j is (q_i - 1) times
    the sum of all digits and coefficient 0 about minus that: with random
    ciphertexts about half the worst-case magnitude, of both signs.  The key
    switch over three or four small primes still equals the oracle bit for
    bit."""
    c = ctx_for(name)
    P = oparams(c)
    ok = he.keygen(P, 21, True)
    rlk = np.empty_like(ok.rlk)
    for i, qi in enumerate(c.q):
        rlk[:, :, i, :] = qi - 1
    keys = he.Keys(ok.sk, ok.pk, rlk)
    kh = nv.he_keys_import(c.h, cuda(ok.sk), cuda(ok.pk), cuda(rlk))
    rng = np.random.default_rng(23)
    a = he.encrypt(P, ok, rng.integers(0, c.t, (2, c.N), dtype=np.uint64), 24)
    b = he.encrypt(P, ok, rng.integers(0, c.t, (2, c.N), dtype=np.uint64), 25)
    pairs = [(0, 1), (1, 0)]
    out = c.ct(2)
    nv.he_ccmul_precompute(c.h, kh, cuda(a), 2, cuda(b), 2, pairs, 1, out)
    assert np.array_equal(to_np(out), he.ccmul(P, keys, a, b, pairs, 1))
    nv.he_keys_destroy(kh)


def test_ccmul_in_chunks_gives_the_same_bits():
    """A CCMul-Precompute whose scratch exceeds the context's budget runs in
    chunks of outputs; a budget of one output per chunk gives the bits of the
    single-chunk call (a 3x16x16 -> 6 layer at N = 4096, batch 2)."""
    c = ctx_for("n4096")
    small = layer.Context(c.spec, max_ccmul_scratch_bytes=1.0)
    shape = wl.ConvShape(3, 16, 16, 6, 3, 1)
    outs = []
    for ctx in (c, small):
        keys = layer.Keys(ctx, 12, True)
        plan = layer.Plan(ctx, shape, "corr")
        pl = layer.PLayer(ctx, keys, plan, 2)
        x = torch.from_numpy(wl.activations(13, (2, 3, 16, 16))).cuda()
        w = torch.from_numpy(wl.weights(14, (6, 3, 3, 3))).cuda()
        pl.client_prepare(x, w, wl.protocol_seeds(15))
        pl.offline()
        outs.append(to_np(pl.buf.rr))
        assert pl.no > 1
        keys.close()
        plan.close()
    assert np.array_equal(outs[0], outs[1])
    small.close()


def test_table_cache_budget_gives_the_same_bits():
    """A context whose term-table cache budget is one byte drops its cached
    tables (after a device synchronisation) at the start of every call; two
    layer steps on it give the bits of the same steps on a default context."""
    c = ctx_for("n4096")
    tiny = layer.Context(c.spec, max_table_cache_bytes=1.0)
    shape = wl.ConvShape(3, 16, 16, 6, 3, 1)
    outs = []
    for ctx in (c, tiny):
        keys = layer.Keys(ctx, 16, True)
        plan = layer.Plan(ctx, shape, "conv")
        pl = layer.PLayer(ctx, keys, plan, 2)
        x = torch.from_numpy(wl.activations(17, (2, 3, 16, 16))).cuda()
        w = torch.from_numpy(wl.weights(18, (6, 3, 3, 3))).cuda()
        for step in range(2):
            y = pl.step(x, w, wl.protocol_seeds(19 + step))
            outs.append((to_np(pl.buf.rr), to_np(pl.buf.out), to_np(y)))
        keys.close()
        plan.close()
    for a, b in zip(outs[:2], outs[2:]):
        for u, v in zip(a, b):
            assert np.array_equal(u, v)
    tiny.close()


@pytest.mark.parametrize("name", ["n1024", "n8192", "n2048_t40"])
def test_ppmul_bits(name):
    c = ctx_for(name)
    P = oparams(c)
    pl = layer.Plan(c, wl.ConvShape(3, 12, 11, 2, 3, 1) if c.N < 4096 else wl.ConvShape(3, 32, 32, 3, 3, 1), "conv")
    T, G, M, B = pl.T, pl.G, pl.MG, 2
    rng = np.random.default_rng(9)
    px = rng.integers(0, c.t, (B * T * G, c.N), dtype=np.uint64)
    pw = rng.integers(0, c.t, (M * G, c.N), dtype=np.uint64)
    out = c.u64(B * M * T, c.N)
    nv.he_ppmul_conv(c.h, pl.h, B, cuda(px), cuda(pw), out)
    terms = [[((b * T + t) * G + g, m * G + g) for g in range(G)] for b in range(B) for m in range(M) for t in range(T)]
    assert np.array_equal(to_np(out), he.ppmul_terms(P, px, pw, terms))
    pl.close()


def run_layer_both(name, shape, enc, B, seed):
    c = ctx_for(name)
    seeds = wl.protocol_seeds(seed)
    x = wl.activations(seed, (B, shape.C, shape.H, shape.W))
    w = wl.weights(seed + 1, (shape.M, shape.C, shape.h, shape.h))
    keys = layer.Keys(c, seeds.keys, True)
    plan = layer.Plan(c, shape, enc)
    pl = layer.PLayer(c, keys, plan, B)
    y = pl.step(cuda(x), cuda(w), seeds)
    torch.cuda.synchronize()
    op = packing.make_plan(enc, c.N, shape.C, shape.H, shape.W, shape.M, shape.h, shape.pad)
    ref = protocol.run_layer(oparams(c), op, x, w, seeds)
    return c, pl, y, ref, x, w, (keys, plan)


@pytest.mark.parametrize("enc", ["conv", "corr"])
def test_layer_conv_1x28x28_n4096_end_to_end(enc):
    """The 1x28x28 -> 4 channel 3x3 valid layer at N = 4096, 3 x 36-bit limbs."""
    c, pl, y, ref, x, w, hs = run_layer_both("n4096", wl.CONV_SMALL.shape, enc, 1, wl.CONV_SMALL.seed)
    b = pl.buf
    assert np.array_equal(to_np(b.ct_x), ref.ct_x)
    assert np.array_equal(to_np(b.ct_rw), ref.ct_rw)
    assert np.array_equal(to_np(b.rr), ref.rr)
    assert np.array_equal(to_np(b.out), ref.out)
    assert np.array_equal(to_np(b.p), ref.p)
    assert np.array_equal(to_np(y)[0], ref.y)
    assert np.array_equal(ref.y, protocol.conv_reference(x[0], w, 0))
    for h in hs:
        h.close()


@pytest.mark.parametrize("enc", ["corr", "conv"])
def test_layer_conv_3x32x32_n8192_end_to_end(enc):
    """The 3x32x32 -> 16 channel 3x3 same layer at N = 8192, 4 x 50-bit limbs,
    20-bit t: offline CCMul-Precompute + online CPMul, full size."""
    c, pl, y, ref, x, w, hs = run_layer_both("n8192", wl.CONV_MID.shape, enc, 1, wl.CONV_MID.seed)
    b = pl.buf
    assert np.array_equal(to_np(b.rr), ref.rr)
    assert np.array_equal(to_np(b.out), ref.out)
    assert np.array_equal(to_np(y)[0], ref.y)
    assert np.array_equal(ref.y, protocol.conv_reference(x[0], w, 1))
    for h in hs:
        h.close()


def test_layer_bench_configuration_batch64_sampled():
    """The benchmark's launch configuration: the 3x32x32 -> 16 layer at N = 8192
    with batch 64 and the seeds of its first timed step.  Every image decodes
    to the exact convolution; the ciphertext bits of images 0 and 63 (input
    encryptions, precomputed [r^x r^w], online result) equal the oracle's,
    which recomputes those images one at a time at their batch positions."""
    w_ = wl.CONV_MID
    s, B = w_.shape, 64
    c = ctx_for("n8192")
    seeds = wl.protocol_seeds(w_.seed)
    keys = layer.Keys(c, seeds.keys, True)
    plan = layer.Plan(c, s, w_.encoding)
    pl = layer.PLayer(c, keys, plan, B)
    x, k = wl.layer_inputs(w_, B)
    y = to_np(pl.step(cuda(x), cuda(k), seeds))
    for b in range(B):
        assert np.array_equal(y[b], protocol.conv_reference(x[b], k, s.pad)), b
    P = oparams(c)
    okeys = he.keygen(P, seeds.keys, True)
    op = packing.make_plan(w_.encoding, c.N, s.C, s.H, s.W, s.M, s.h, s.pad)
    nx, no = plan.T * plan.G, plan.MG * plan.T
    ct_x, rr, out = to_np(pl.buf.ct_x), to_np(pl.buf.rr), to_np(pl.buf.out)
    for b in (0, B - 1):
        ref = protocol.run_layer(P, op, x[b], k, seeds, keys=okeys, first_image=b)
        assert np.array_equal(ct_x[b * nx:(b + 1) * nx], ref.ct_x)
        assert np.array_equal(rr[b * no:(b + 1) * no], ref.rr)
        assert np.array_equal(out[b * no:(b + 1) * no], ref.out)
        assert np.array_equal(y[b], ref.y)
    keys.close()
    plan.close()


@pytest.mark.parametrize("name,shape_of,enc", [("n4096", wl.CONV_SMALL, "conv"), ("n8192", wl.CONV_MID, "corr")])
def test_layer_b_protocol_bits(name, shape_of, enc):
    """CryptoTrain-B (Section 3.1): the online [x][w] CCMul of the GPU equals
    the oracle's bit for bit, and decodes to the exact convolution."""
    c = ctx_for(name)
    s = shape_of.shape
    seeds = wl.protocol_seeds(shape_of.seed + 5)
    x = wl.activations(shape_of.seed + 6, (1, s.C, s.H, s.W))
    w = wl.weights(shape_of.seed + 7, (s.M, s.C, s.h, s.h))
    keys = layer.Keys(c, seeds.keys, True)
    plan = layer.Plan(c, s, enc)
    bl = layer.BLayer(c, keys, plan, 1)
    y = to_np(bl.step(cuda(x), cuda(w), seeds))
    op = packing.make_plan(enc, c.N, s.C, s.H, s.W, s.M, s.h, s.pad)
    ref = protocol.run_layer_b(oparams(c), op, x, w, seeds)
    assert np.array_equal(to_np(bl.ct_x), ref.ct_x)
    assert np.array_equal(to_np(bl.out), ref.out)
    assert np.array_equal(y[0], ref.y)
    assert np.array_equal(ref.y, protocol.conv_reference(x[0], w, s.pad))
    keys.close()
    plan.close()


@pytest.mark.parametrize("enc,depthwise", [("corr", False), ("conv", False), ("corr", True), ("conv", True)])
def test_batch_norm_layer_bits(enc, depthwise):
    """The batch-norm linear protocol as a CryptoTrain-P layer: the diagonal
    1x1 kernel gamma and the bias beta added to [r^x r^gamma] offline, under
    the dense and the depthwise plan.  Bits of the precomputed and online
    ciphertexts equal the oracle's; every image decodes to gamma_c x_c + beta_c
    (16 channels of 16x16, batch 2, N = 8192)."""
    c = ctx_for("n8192")
    C, H, B = 16, 16, 2
    shape = wl.ConvShape(C, H, H, C, 1, 0)
    seeds = wl.protocol_seeds(606)
    x = wl.activations(607, (B, C, H, H))
    gamma = torch.from_numpy(wl.weights(608, (C,)).astype(np.int64))
    beta = torch.from_numpy(wl.rng(609).integers(-1000, 1000, C))
    w = layer.batch_norm_weights(gamma)
    keys = layer.Keys(c, seeds.keys, True)
    plan = layer.Plan(c, shape, enc, depthwise=depthwise)
    pl = layer.PLayer(c, keys, plan, B, with_bias=True)
    y = to_np(pl.step(cuda(x), w.cuda(), seeds, beta))
    op = packing.make_plan(enc, c.N, C, H, H, C, 1, 0, depthwise=depthwise)
    assert plan.products == op.products
    ref = protocol.run_layer(oparams(c), op, x, w.numpy(), seeds, bias=beta.numpy())
    assert np.array_equal(to_np(pl.buf.rr), ref.rr)
    assert np.array_equal(to_np(pl.buf.out), ref.out)
    g, bt = gamma.numpy()[:, None, None], beta.numpy()[:, None, None]
    for b in range(B):
        assert np.array_equal(y[b], ref.y[b])
        assert np.array_equal(y[b], g * x[b].astype(np.int64) + bt)
    keys.close()
    plan.close()


def test_depthwise_convolution_bits():
    """A depthwise 3x3 convolution (each channel with its own kernel) under the
    depthwise plan at N = 4096: bit-exact against the oracle, decoded to the
    per-channel convolution."""
    c = ctx_for("n4096")
    C, H = 12, 20
    shape = wl.ConvShape(C, H, H, C, 3, 1)
    seeds = wl.protocol_seeds(707)
    x = wl.activations(708, (1, C, H, H))
    kern = wl.weights(709, (C, 3, 3)).astype(np.int64)
    w = np.zeros((C, C, 3, 3), dtype=np.int64)
    for ch in range(C):
        w[ch, ch] = kern[ch]
    keys = layer.Keys(c, seeds.keys, True)
    plan = layer.Plan(c, shape, "corr", depthwise=True)
    pl = layer.PLayer(c, keys, plan, 1)
    y = to_np(pl.step(cuda(x), cuda(w), seeds))
    op = packing.make_plan("corr", c.N, C, H, H, C, 3, 1, depthwise=True)
    ref = protocol.run_layer(oparams(c), op, x, w, seeds)
    assert np.array_equal(to_np(pl.buf.rr), ref.rr)
    assert np.array_equal(to_np(pl.buf.out), ref.out)
    assert np.array_equal(y[0], protocol.conv_reference(x[0], w, 1))
    keys.close()
    plan.close()


def test_layer_alexnet_shaped_first_layer():
    """An AlexNet-shaped first layer on a 64x64x3 input with an 11x11 kernel
    (same padding, 16 of its output channels) at N = 8192: bit-exact against
    the oracle and decoded to the exact convolution."""
    c = ctx_for("n8192")
    shape = wl.ConvShape(3, 64, 64, 16, 11, 5)
    c2, pl, y, ref, x, w, hs = run_layer_both("n8192", shape, "corr", 1, 4711)
    assert pl.plan.T * pl.plan.G * pl.plan.MG == 48
    assert np.array_equal(to_np(pl.buf.rr), ref.rr)
    assert np.array_equal(to_np(pl.buf.out), ref.out)
    assert np.array_equal(to_np(y)[0], protocol.conv_reference(x[0], w, 5))
    for h in hs:
        h.close()


def test_layer_batched_ragged_tiles():
    """batch 3, several tiles and channel groups with ragged tails at N = 1024."""
    shape = wl.ConvShape(8, 24, 17, 3, 3, 2)
    c, pl, y, ref, x, w, hs = run_layer_both("n1024", shape, "corr", 3, 41)
    assert pl.plan.T > 1 and pl.plan.G > 1
    assert np.array_equal(to_np(pl.buf.out), ref.out)
    yy = to_np(y)
    for b in range(3):
        assert np.array_equal(yy[b], protocol.conv_reference(x[b], w, 2))
    for h in hs:
        h.close()


def test_errors_are_reported_not_raised_on_device():
    c = ctx_for("n1024")
    with pytest.raises(nv.HEError) as e:
        nv.he_conv_plan(c.h, 1, 40, 40, 2, 40, 0, nv.HE_ENC_CORRELATED)   # a 40x40 kernel cannot fit N = 1024
    assert e.value.code == -3
    with pytest.raises(nv.HEError):
        nv.he_conv_plan(c.h, 3, 8, 8, 2, 3, 3, nv.HE_ENC_CORRELATED)      # pad > h - 1
    with pytest.raises(nv.HEError):
        nv.he_setup(nv.make_params(3000, prime_bits=[40], t=65537))       # N not a power of two
    k = layer.Keys(c, 1, False)
    a = c.ct(1)
    with pytest.raises(nv.HEError):
        nv.he_ccmul_precompute(c.h, k.h, a, 1, a, 1, [(0, 0)], 1, c.ct(1))  # no relin key
    # zero-sized calls are no-ops
    nv.he_encrypt(c.h, k.h, c.u64(1, c.N), 0, 1, a)
    nv.he_decrypt(c.h, k.h, a, 0, c.u64(1, c.N))
    k.close()
    torch.cuda.synchronize()


def test_checkpoint_resume(tmp_path):
    """Checkpoint / resume of a serving process: keys exported in coefficient
    form and the precomputed [r^x r^w] saved with the context fingerprint;
    a fresh context resumes them (he_keys_import recomputes the NTT forms)
    and the online layer gives the same bits as before.  A context with other
    parameters is refused, and so are keys that are not valid residues."""
    from paper_2409_16675_gb300 import checkpoint
    spec = wl.RING_SMALL
    c1 = layer.Context(spec)
    seeds = wl.protocol_seeds(515)
    keys = layer.Keys(c1, seeds.keys, True)
    shape = wl.ConvShape(3, 12, 12, 4, 3, 1)
    plan = layer.Plan(c1, shape, "corr")
    pl = layer.PLayer(c1, keys, plan, 2)
    x = torch.from_numpy(wl.activations(516, (2, 3, 12, 12))).cuda()
    w = torch.from_numpy(wl.weights(517, (4, 3, 3, 3))).cuda()
    pl.client_prepare(x, w, seeds)
    pl.offline()
    pl.online()
    want = to_np(pl.buf.out)
    path = str(tmp_path / "state")
    checkpoint.save(path, c1, keys, {"rr": pl.buf.rr, "ct_x": pl.buf.ct_x, "ct_w": pl.buf.ct_w,
                                     "xm": pl.buf.xm, "wm": pl.buf.wm})
    # resume on a new context of the same ring
    c2 = layer.Context(spec)
    keys2, t = checkpoint.load(path, c2)
    for which in (nv.HE_KEY_SK, nv.HE_KEY_PK, nv.HE_KEY_RLK):
        assert torch.equal(keys2.export(which), keys.export(which))
    plan2 = layer.Plan(c2, shape, "corr")
    out = c2.ct(pl.no)
    nv.he_cpmul_conv(c2.h, plan2.h, 2, t["ct_x"], t["wm"], t["ct_w"], t["xm"], t["rr"], out)
    assert np.array_equal(to_np(out), want)
    # the resumed keys encrypt, relinearise and decrypt like the originals
    m = cuda(wl.uniform_mod(518, (2, c2.N), c2.t))
    a, b = c1.ct(2), c2.ct(2)
    nv.he_encrypt(c1.h, keys.h, m, 2, 99, a)
    nv.he_encrypt(c2.h, keys2.h, m, 2, 99, b)
    assert torch.equal(a, b)
    pa, pb = c1.ct(1), c2.ct(1)
    nv.he_ccmul_precompute(c1.h, keys.h, a, 2, a, 2, [(0, 1)], 1, pa)
    nv.he_ccmul_precompute(c2.h, keys2.h, b, 2, b, 2, [(0, 1)], 1, pb)
    assert torch.equal(pa, pb)
    # other parameters: refused
    c3 = layer.Context(wl.RingSpec(4096, (36, 36, 40), 65537))
    with pytest.raises(ValueError):
        checkpoint.load(path, c3)
    # a key residue outside its limb: refused on the device, no fault
    bad_pk = keys.export(nv.HE_KEY_PK).clone()
    bad_pk[0, 0, 0] = c1.q[0]
    with pytest.raises(nv.HEError):
        nv.he_keys_import(c1.h, keys.export(nv.HE_KEY_SK), bad_pk, None)
    for h in (keys, keys2, plan, plan2):
        h.close()
    for cc in (c1, c2, c3):
        cc.close()


def test_determinism_same_seeds_same_bits():
    """Same seeds, same bits: the whole layer step (keys, encryptions,
    CCMul-Precompute, online, PPMul, decryption) repeated five times on the
    benchmark's layer (batch 8) gives identical ciphertexts and outputs --
    no result depends on the order in which CTAs or streams run."""
    w_ = wl.CONV_MID
    c = ctx_for("n8192")
    seeds = wl.protocol_seeds(w_.seed)
    x, k = wl.layer_inputs(w_, 8)
    runs = []
    for _ in range(5):
        keys = layer.Keys(c, seeds.keys, True)
        plan = layer.Plan(c, w_.shape, w_.encoding)
        pl = layer.PLayer(c, keys, plan, 8)
        y = pl.step(cuda(x), cuda(k), seeds)
        runs.append([to_np(t) for t in (pl.buf.ct_x, pl.buf.rr, pl.buf.out, pl.buf.p, y)])
        keys.close()
        plan.close()
    for r in runs[1:]:
        for a, b in zip(r, runs[0]):
            assert np.array_equal(a, b)
