"""he_cpmul_conv_noalloc, the variant of the CPMul convolution for callers
that cannot allocate device memory during the call (stream capture into a
CUDA graph, memory fully reserved by another allocator, latency-critical
serving loops).  Its output must equal he_cpmul_conv's bit for bit on two
calls in a row, and oversize requests must be refused cleanly.

The file name sorts last so that a run stopping at the first failure has run
every other test before this one."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2409_16675_gb300 import layer, native as nv, workloads as wl  # noqa: E402


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


@pytest.mark.parametrize("ring,shape,enc,B", [
    (wl.RING_MID, wl.CONV_MID.shape, "corr", 1),                      # the online 3x32x32 -> 16 layer
    (wl.RingSpec(1024, (40, 45), 65537), wl.ConvShape(8, 24, 17, 3, 3, 2), "corr", 3),  # tiles + groups
])
def test_noalloc_matches_allocating_entry_point(ring, shape, enc, B):
    c = layer.Context(ring)
    plan = layer.Plan(c, shape, enc)
    for call in range(2):
        ctx_, ptw, ctw, ptx, add, no = _operands(c, plan, B, 10 + call)
        ref = c.ct(no)
        got = c.ct(no)
        nv.he_cpmul_conv(c.h, plan.h, B, ctx_, ptw, ctw, ptx, add, ref)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        nv.he_cpmul_conv_noalloc(c.h, plan.h, B, ctx_, ptw, ctw, ptx, add, got)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert torch.equal(got, ref)
        if call > 0:
            # the first call on a device is the set-up call (the runtime may load
            # the module holding the fixed scratch then); later calls allocate nothing
            assert free0 - free1 < (1 << 20)
        # one family only, no add operand
        nv.he_cpmul_conv(c.h, plan.h, B, ctx_, ptw, None, None, None, ref)
        nv.he_cpmul_conv_noalloc(c.h, plan.h, B, ctx_, ptw, None, None, None, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
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
