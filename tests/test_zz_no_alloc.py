"""he_cpmul_conv_noalloc: the CPMul convolution for callers that cannot
allocate device memory during the call.  These include serving processes
whose device memory another allocator (a framework's caching pool, an
inference engine's arena) has reserved up front, so that a cudaMalloc inside
the library would fail or evict that cache, and latency-critical loops that
must not pay the device-wide synchronisation of cudaMalloc/cudaFree.  Its
scratch is a fixed 32 MiB static device array.

Checked here: the output equals he_cpmul_conv's bit for bit on two calls in
a row (dense and depthwise plans, one or both operand families, with and
without the addend); a call on a context that has never allocated scratch
leaves the device's free memory unchanged; oversize calls are refused.

The file name sorts last so that a run stopping at the first failure has run
every other test before this one."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2409_16675_gb300 import layer, native as nv, workloads as wl  # noqa: E402

SMALL_RING = wl.RingSpec(1024, (40, 45), 65537)


def _operands(c, plan, B, seed):
    """Random ciphertexts / plaintexts of the right shapes (fresh encryptions
    are not needed to compare two implementations of the same product)."""
    rng = np.random.default_rng(seed)
    T, G, M = plan.T, plan.G, plan.MG
    nx, nw, no = B * T * G, M * G, B * M * T

    def ct(n):
        a = np.stack([rng.integers(0, q, (n, 2, c.N), dtype=np.uint64) for q in c.q], axis=2)
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    def pt(n):
        return torch.from_numpy(rng.integers(0, c.t, (n, c.N), dtype=np.uint64)).cuda()

    return ct(nx), pt(nw), ct(nw), pt(nx), ct(no), no


def _setup_call():
    """One call on a throw-away context: the first call on a device looks up
    the static array's address (and the runtime may load the module that
    holds it), which is the set-up this entry point documents."""
    c = layer.Context(SMALL_RING)
    plan = layer.Plan(c, wl.ConvShape(2, 8, 8, 2, 3, 1), "corr")
    x, ptw, _, _, _, no = _operands(c, plan, 1, 1)
    out = c.ct(no)
    nv.he_cpmul_conv_noalloc(c.h, plan.h, 1, x, ptw, None, None, None, out)
    torch.cuda.synchronize()
    plan.close()
    c.close()


@pytest.mark.parametrize("ring,shape,enc,B,depthwise", [
    (wl.RING_MID, wl.CONV_MID.shape, "corr", 1, False),                       # the online 3x32x32 -> 16 layer
    (SMALL_RING, wl.ConvShape(8, 24, 17, 3, 3, 2), "corr", 3, False),          # tiles + channel groups
    (SMALL_RING, wl.ConvShape(12, 20, 20, 12, 3, 1), "conv", 2, True),         # depthwise plan
])
def test_noalloc_matches_allocating_entry_point(ring, shape, enc, B, depthwise):
    c = layer.Context(ring)
    plan = layer.Plan(c, shape, enc, depthwise=depthwise)
    for call in range(2):
        ctx_, ptw, ctw, ptx, add, no = _operands(c, plan, B, 10 + call)
        ref = c.ct(no)
        got = c.ct(no)
        nv.he_cpmul_conv_noalloc(c.h, plan.h, B, ctx_, ptw, ctw, ptx, add, got)
        nv.he_cpmul_conv(c.h, plan.h, B, ctx_, ptw, ctw, ptx, add, ref)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        # each operand family alone, no addend
        for args in ((ctx_, ptw, None, None), (None, None, ctw, ptx)):
            nv.he_cpmul_conv(c.h, plan.h, B, *args, None, ref)
            nv.he_cpmul_conv_noalloc(c.h, plan.h, B, *args, None, got)
            torch.cuda.synchronize()
            assert torch.equal(got, ref)
    plan.close()
    c.close()


def test_noalloc_allocates_nothing_on_a_fresh_context():
    """A context that has never run an allocating call has no workspace, so an
    implementation that still took its scratch from the context (or uploaded
    a cached term table) would allocate here; a cudaMalloc lowers the device's
    free memory by at least 2 MiB."""
    _setup_call()
    c = layer.Context(wl.RING_MID)
    plan = layer.Plan(c, wl.CONV_MID.shape, "corr")
    ops = [_operands(c, plan, 1, 20 + i) for i in range(2)]
    outs = [c.ct(o[5]) for o in ops]
    refs = [c.ct(o[5]) for o in ops]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for (x, ptw, ctw, ptx, add, _), out in zip(ops, outs):
        nv.he_cpmul_conv_noalloc(c.h, plan.h, 1, x, ptw, ctw, ptx, add, out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < (1 << 20), "the no-allocation call allocated %d bytes" % (free0 - free1)
    for (x, ptw, ctw, ptx, add, _), ref in zip(ops, refs):
        nv.he_cpmul_conv(c.h, plan.h, 1, x, ptw, ctw, ptx, add, ref)
    torch.cuda.synchronize()
    for out, ref in zip(outs, refs):
        assert torch.equal(out, ref)
    plan.close()
    c.close()


def test_noalloc_refuses_oversize_calls():
    c = layer.Context(wl.RING_MID)
    plan = layer.Plan(c, wl.CONV_MID.shape, "corr")
    B = 64                                       # about 34 MiB of NTT-form operands
    T, G, M = plan.T, plan.G, plan.MG
    x = c.ct(B * T * G)
    out = c.ct(B * M * T)
    with pytest.raises(nv.HEError) as e:
        nv.he_cpmul_conv_noalloc(c.h, plan.h, B, x, c.u64(M * G, c.N), None, None, None, out)
    assert e.value.code == -5 and "32 MiB" in str(e.value)
    torch.cuda.synchronize()
    plan.close()
    c.close()
