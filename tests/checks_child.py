"""Run in a child process by tests/test_gpu_checks.py with
CRYPTOTRAIN_LIB=checks: exercises the bounds-checked build of the library.

1. A small CryptoTrain-P layer step gives the oracle's ciphertexts and
   decoded output with no violation reported.
2. With the last coefficient of a CPMul output left out of the checked
   ranges (valid memory, so nothing can fault), the call returns
   HE_ERR_INVALID_ARG naming the store, that coefficient keeps its old value
   (the store was skipped), and every other output word equals the unchecked
   result.
3. With the exclusion cleared the same call succeeds again; so do the
   no-allocation entry point and a small batch (work-list kernels).
Prints "checks ok" at the end."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

from oracle import he, packing, protocol  # noqa: E402
from paper_2409_16675_gb300 import layer, native as nv, workloads as wl  # noqa: E402


def main():
    assert nv.LIB_NAME == "libcryptotrain_checks.so" and nv.he_checks_enabled()
    # 1. a small layer against the oracle
    spec = wl.RingSpec(1024, (36, 36, 36), 65537)
    shape = wl.ConvShape(2, 9, 8, 3, 3, 1)
    x = wl.activations(7, (1, shape.C, shape.H, shape.W))
    w = wl.weights(8, (shape.M, shape.C, shape.h, shape.h))
    seeds = wl.protocol_seeds(5)
    ctx = layer.Context(spec)
    keys = layer.Keys(ctx, seeds.keys, True)
    plan = layer.Plan(ctx, shape, "corr")
    pl = layer.PLayer(ctx, keys, plan, 1)
    y = pl.step(torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda(), seeds)
    torch.cuda.synchronize()
    P = he.Params(spec.N, ctx.q, spec.t)
    ref = protocol.run_layer(P, packing.make_plan("corr", spec.N, shape.C, shape.H, shape.W, shape.M, shape.h,
                                                  shape.pad), x, w, seeds)
    assert np.array_equal(pl.buf.out.cpu().numpy(), ref.out)
    assert np.array_equal(y.cpu().numpy()[0], ref.y)

    # 2. a skipped store is reported
    b = pl.buf
    want = b.out.clone()
    out = torch.full_like(b.out.view(torch.int64), 7).view(torch.uint64)
    last = out.view(-1)[-1:]
    nv.he_checks_test_exclude(last, 8)
    try:
        nv.he_cpmul_conv(ctx.h, plan.h, 1, b.ct_x, b.wm, b.ct_w, b.xm, b.rr, out)
        raise AssertionError("the excluded store was not reported")
    except nv.HEError as e:
        assert e.code == -1, e.code
    msg = nv.he_checks_last_error()
    assert "out-of-range device access" in msg and "ntt" in msg, msg
    flat, wflat = out.view(torch.int64).view(-1), want.view(torch.int64).view(-1)
    assert int(flat[-1]) == 7
    assert torch.equal(flat[:-1], wflat[:-1])

    # 3. cleared: the same call, the no-allocation variant and a batch
    nv.he_checks_test_exclude(None, 0)
    nv.he_cpmul_conv(ctx.h, plan.h, 1, b.ct_x, b.wm, b.ct_w, b.xm, b.rr, out)
    torch.cuda.synchronize()
    assert torch.equal(out, want)
    out.zero_()
    nv.he_cpmul_conv_noalloc(ctx.h, plan.h, 1, b.ct_x, b.wm, b.ct_w, b.xm, b.rr, out)
    torch.cuda.synchronize()
    assert torch.equal(out, want)
    bt = nv.he_batch_create(0)
    nv.he_batch_add_cpmul2(bt, ctx.h, plan.h, 1, b.ct_x, b.wm, b.ct_w, b.xm, b.rr, out)
    nv.he_batch_prepare(bt)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out.zero_()
        nv.he_batch_run(bt, nv.HE_BATCH_PERSISTENT)
        nv.he_batch_status(bt)
    torch.cuda.synchronize()
    assert torch.equal(out, want)
    nv.he_batch_destroy(bt)
    for o in (plan, keys, ctx):
        o.close()
    print("checks ok")


if __name__ == "__main__":
    main()
