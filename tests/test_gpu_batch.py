"""Batched form: many ct x pt convolution jobs of uneven shapes, ring degrees,
limb counts and primes.  The plain, persistent and graph forms give identical
bits, a job's result is the same alone and in the mix, and the results equal
the oracle's."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import he, packing  # noqa: E402
from paper_2409_16675_gb300 import layer, native as nv, workloads as wl  # noqa: E402


def make_inputs(ctx, plan, B, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    T, G, MG = plan.T, plan.G, plan.MG
    ct = torch.empty((B * T * G, 2, ctx.L, ctx.N), dtype=torch.int64, device="cuda")
    for i, q in enumerate(ctx.q):
        ct[:, :, i, :] = torch.randint(0, q, (B * T * G, 2, ctx.N), generator=g, device="cuda", dtype=torch.int64)
    pt = torch.randint(0, ctx.t, (MG * G, ctx.N), generator=g, device="cuda", dtype=torch.int64)
    return ct.view(torch.uint64), pt.view(torch.uint64)


def build(jobs, B=1):
    ctxs, items = {}, []
    for j in jobs:
        key = (j.ring.N, j.ring.prime_bits)
        if key not in ctxs:
            ctxs[key] = layer.Context(j.ring)
        c = ctxs[key]
        p = layer.Plan(c, j.shape, j.encoding)
        ct, pt = make_inputs(c, p, B, j.seed)
        out = c.ct(B * p.MG * p.T)
        items.append((c, p, ct, pt, out))
    return ctxs, items


def test_batch_forms_identical_and_equal_alone():
    jobs = wl.batched_jobs(seed=123, n_jobs=14, channels=(3, 5, 16), sizes=(6, 8, 12), kernels=(1, 3, 5))
    ctxs, items = build(jobs, B=2)
    b = nv.he_batch_create(0)
    for (c, p, ct, pt, out) in items:
        nv.he_batch_add_cpmul(b, c.h, p.h, 2, ct, pt, None, out)
    nv.he_batch_prepare(b)
    s = torch.cuda.Stream()
    results = {}
    with torch.cuda.stream(s):
        for mode in (nv.HE_BATCH_PLAIN, nv.HE_BATCH_PERSISTENT, nv.HE_BATCH_GRAPH, nv.HE_BATCH_GRAPH):
            for it in items:
                it[4].zero_()
            nv.he_batch_run(b, mode)
            s.synchronize()
            results.setdefault(mode, []).append([it[4].clone() for it in items])
        tuning = nv.he_batch_autotune(b)
        nv.he_batch_run(b, nv.HE_BATCH_PERSISTENT)
        s.synchronize()
        tuned = [it[4].clone() for it in items]
    assert tuning and all(t["ms"] > 0 for t in tuning)
    ref = results[nv.HE_BATCH_PLAIN][0]
    for mode, runs in results.items():
        for run in runs:
            for a, r in zip(run, ref):
                assert torch.equal(a, r), mode
    for a, r in zip(tuned, ref):
        assert torch.equal(a, r)
    # a job alone equals the same job inside the batch
    for (c, p, ct, pt, out), r in zip(items, ref):
        alone = c.ct(out.shape[0])
        nv.he_cpmul_conv(c.h, p.h, 2, ct, pt, None, None, None, alone)
        torch.cuda.synchronize()
        assert torch.equal(alone, r)
    nv.he_batch_destroy(b)
    # two jobs against the oracle
    for (c, p, ct, pt, out), r in list(zip(items, ref))[:2]:
        P = he.Params(c.N, c.q, c.t)
        op = packing.make_plan(p.encoding, c.N, *[getattr(p.shape, k) for k in ("C", "H", "W", "M", "h", "pad")])
        T, G, MG = op.T, op.G, op.MG
        terms = [[((bb * T + t) * G + g, m * G + g) for g in range(G)]
                 for bb in range(2) for m in range(MG) for t in range(T)]
        want = he.cpmul_terms(P, ct.cpu().numpy(), pt.cpu().numpy(), terms)
        assert np.array_equal(r.cpu().numpy(), want)
    for c in ctxs.values():
        c.close()


def test_every_launch_configuration_gives_the_same_bits():
    """The work-list launch of each ring degree in every configuration the
    autotuner can choose (register budget 1 or 2 CTAs per SM; persistent with
    1..4 CTAs per SM, or one CTA per item) gives the plain form's bits, and
    out-of-range tunings are refused."""
    jobs = wl.batched_jobs(seed=321, n_jobs=8, channels=(3, 16), sizes=(8, 12), kernels=(1, 3), degrees=(4096, 8192))
    ctxs, items = build(jobs, B=1)
    b = nv.he_batch_create(0)
    for (c, p, ct, pt, out) in items:
        nv.he_batch_add_cpmul(b, c.h, p.h, 1, ct, pt, None, out)
    nv.he_batch_prepare(b)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        nv.he_batch_run(b, nv.HE_BATCH_PLAIN)
        s.synchronize()
        ref = [it[4].clone() for it in items]
        degrees = sorted({c.N.bit_length() - 1 for c in ctxs.values()})
        for regs in (1, 2):
            for grid in range(0, 5):
                for it in items:
                    it[4].zero_()
                nv.he_batch_set_tuning(b, [dict(logN=d, regs_ctas_per_sm=regs, grid_ctas_per_sm=grid) for d in degrees])
                nv.he_batch_run(b, nv.HE_BATCH_GRAPH if grid % 2 else nv.HE_BATCH_PERSISTENT)
                s.synchronize()
                for it, r in zip(items, ref):
                    assert torch.equal(it[4], r), (regs, grid)
    with pytest.raises(nv.HEError):
        nv.he_batch_set_tuning(b, [dict(logN=12, regs_ctas_per_sm=3, grid_ctas_per_sm=0)])
    with pytest.raises(nv.HEError):
        nv.he_batch_set_tuning(b, [dict(logN=15, regs_ctas_per_sm=1, grid_ctas_per_sm=0)])
    nv.he_batch_destroy(b)
    for c in ctxs.values():
        c.close()


def test_full_config4_batch_sampled_against_the_oracle():
    """The real 256-job batch of the batched form (C, M in {3..128}, spatial
    {8, 16, 32}, kernels {1, 3, 5}, N in {4096, 8192}, 2-5 limbs of 36-60
    bits, both encodings), one image per job, replayed from its CUDA graph in
    the launch configuration the autotuner picks: for every 16th job, the
    first and the last output ciphertext (all limbs, both components) equal
    the oracle's sum of ciphertext x plaintext products."""
    jobs = wl.batched_jobs()
    ctxs, items = build(jobs, B=1)
    b = nv.he_batch_create(0)
    for (c, p, ct, pt, out) in items:
        nv.he_batch_add_cpmul(b, c.h, p.h, 1, ct, pt, None, out)
    nv.he_batch_prepare(b)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        nv.he_batch_autotune(b)
        for it in items:
            it[4].zero_()
        nv.he_batch_run(b, nv.HE_BATCH_GRAPH)
        s.synchronize()
    nv.he_batch_destroy(b)
    checked = set()
    for (c, p, ct, pt, out) in items[::16]:
        T, G, MG = p.T, p.G, p.MG
        terms = [[(t * G + g, m * G + g) for g in range(G)] for m in range(MG) for t in range(T)]
        sel = sorted({0, len(terms) - 1})
        want = he.cpmul_terms(he.Params(c.N, c.q, c.t), ct.cpu().numpy(), pt.cpu().numpy(), [terms[o] for o in sel])
        got = out.cpu().numpy()[sel]
        assert np.array_equal(got, want), (c.N, c.L, p.shape, p.encoding)
        checked.add((c.N, c.L, p.encoding))
    assert {n for (n, _, _) in checked} == {4096, 8192} and {e for (_, _, e) in checked} == {"conv", "corr"}
    for (c, p, ct, pt, out) in items:
        p.close()
    for c in ctxs.values():
        c.close()


def _mixed_batch(seed=123, n_jobs=14):
    jobs = wl.batched_jobs(seed=seed, n_jobs=n_jobs, channels=(3, 5, 16), sizes=(6, 8, 12), kernels=(1, 3, 5),
                           degrees=(4096, 8192))
    ctxs, items = build(jobs, B=2)
    b = nv.he_batch_create(0)
    for (c, p, ct, pt, out) in items:
        nv.he_batch_add_cpmul(b, c.h, p.h, 2, ct, pt, None, out)
    nv.he_batch_prepare(b)
    return ctxs, items, b


def test_fused_one_launch_form_bits():
    """The whole batch (N = 4096 and 8192 jobs, both phases) in one persistent
    launch, at both register budgets and replayed from a CUDA graph, gives
    the plain form's bits on every run, and its status stays clear."""
    ctxs, items, b = _mixed_batch()
    info = nv.he_batch_query(b)
    assert info["fused_supported"] == 1 and info["n_units"] > 0
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        nv.he_batch_run(b, nv.HE_BATCH_PLAIN)
        s.synchronize()
        ref = [it[4].clone() for it in items]
        for regs in (1, 2):
            nv.he_batch_set_fused(b, True, regs)
            for mode in (nv.HE_BATCH_FUSED, nv.HE_BATCH_FUSED, nv.HE_BATCH_GRAPH, nv.HE_BATCH_GRAPH):
                for it in items:
                    it[4].zero_()
                nv.he_batch_run(b, mode)
                nv.he_batch_status(b)
                for it, r in zip(items, ref):
                    assert torch.equal(it[4], r), (regs, mode)
        tuning = nv.he_batch_autotune(b)
        info = nv.he_batch_query(b)
        assert tuning and info["fused_ms"] > 0 and info["per_degree_ms"] > 0
        for it in items:
            it[4].zero_()
        nv.he_batch_run(b, nv.HE_BATCH_GRAPH)
        nv.he_batch_status(b)
        for it, r in zip(items, ref):
            assert torch.equal(it[4], r)
    nv.he_batch_destroy(b)
    for c in ctxs.values():
        c.close()


def test_fused_wait_limit_gives_up_and_recovers():
    """A job whose forward count is held one short (a host-side hold: its
    multiply-accumulate units can never start) makes those units run out of a
    short wait limit: the run reports HE_ERR_TIMEOUT, the held job's outputs
    are never written, and after the hold is released the same batch runs to
    the plain form's bits."""
    ctxs, items, b = _mixed_batch(seed=77, n_jobs=6)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        nv.he_batch_run(b, nv.HE_BATCH_PLAIN)
        s.synchronize()
        ref = [it[4].clone() for it in items]
        for it in items:
            it[4].zero_()
        nv.he_batch_set_wait_limit(b, 2000)
        nv.he_batch_test_hold_job(b, 0, True)
        nv.he_batch_run(b, nv.HE_BATCH_FUSED)
        with pytest.raises(nv.HEError) as e:
            nv.he_batch_status(b)
        assert e.value.code == -6 and "gave up" in str(e.value)
        assert not bool(items[0][4].view(torch.int64).any())
        nv.he_batch_status(b)                     # the status was cleared by the read
        nv.he_batch_test_hold_job(b, 0, False)
        nv.he_batch_set_wait_limit(b, 1 << 22)
        nv.he_batch_run(b, nv.HE_BATCH_FUSED)
        nv.he_batch_status(b)
        for it, r in zip(items, ref):
            assert torch.equal(it[4], r)
    nv.he_batch_destroy(b)
    for c in ctxs.values():
        c.close()
