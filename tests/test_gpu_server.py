"""Served form: continuous batching of CryptoTrain-P online layers from several
clients (each with its own ring, keys and resident precomputed products).
Every result is bit-identical to the same request run alone, decodes to the
exact convolution, equals the oracle's ciphertexts on every client ring, and
admission respects the HBM budget."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import he, protocol  # noqa: E402
from paper_2409_16675_gb300 import layer, native as nv, workloads as wl  # noqa: E402

CLIENTS = [
    (wl.RingSpec(4096, (40, 45, 50), 65537), wl.ConvShape(3, 12, 12, 5, 3, 1), "corr"),
    (wl.RingSpec(8192, (50, 50, 50, 50), 1032193), wl.ConvShape(16, 8, 8, 16, 3, 1), "conv"),
    (wl.RingSpec(16384, (60, 55), 65537), wl.ConvShape(5, 16, 16, 7, 5, 2), "corr"),
]


def setup_clients(B=2):
    out = []
    for i, (ring, shape, enc) in enumerate(CLIENTS):
        ctx = layer.Context(ring)
        keys = layer.Keys(ctx, 100 + i, True)
        plan = layer.Plan(ctx, shape, enc)
        pl = layer.PLayer(ctx, keys, plan, B)
        x = torch.from_numpy(wl.activations(10 + i, (B, shape.C, shape.H, shape.W))).cuda()
        w = torch.from_numpy(wl.weights(20 + i, (shape.M, shape.C, shape.h, shape.h))).cuda()
        seeds = wl.protocol_seeds(30 + i)
        pl.client_prepare(x, w, seeds)
        pl.offline()                      # [r^x r^w] resident on the device
        pl.online()                       # reference: the request run alone
        torch.cuda.synchronize()
        out.append((ctx, keys, plan, pl, x, w))
    return out


def test_server_results_equal_alone_and_decode():
    clients = setup_clients()
    srv = nv.he_server_create(0, hbm_budget_bytes=4e9, max_group=8, max_inflight=3, n_streams=3)
    outs, ids = [], []
    for rep in range(3):                 # several requests per client, interleaved
        for (ctx, keys, plan, pl, x, w) in clients:
            b = pl.buf
            o = torch.zeros_like(b.out)
            ids.append(nv.he_server_submit(srv, ctx.h, plan.h, pl.B, b.ct_x, b.wm, b.ct_w, b.xm, b.rr, o))
            outs.append((pl, o))
    nv.he_server_wait_all(srv, 120.0)
    st = nv.he_server_stats(srv)
    assert st["completed"] == len(ids) and st["p50_us"] > 0 and st["p99_us"] >= st["p50_us"]
    for rid in ids:
        done, lat = nv.he_server_poll(srv, rid)
        assert done and lat > 0
    for pl, o in outs:
        assert torch.equal(o, pl.buf.out)           # same bits as the request alone
    # one served result per client ring against the oracle's CPMul + CCAdd at
    # the ciphertext level: out[b][m][t] = sum_g [x][b][t][g] (w - r^w)[m][g]
    # + [w][m][g] (x - r^x)[b][t][g] + [r^x r^w][b][m][t]
    for (ctx, keys, plan, pl, x, w), (pl2, o) in zip(clients, outs[:len(clients)]):
        b = pl.buf
        T, G, MG, B = plan.T, plan.G, plan.MG, pl.B
        nx, nw = B * T * G, MG * G
        terms = [[((bb * T + t) * G + g, m * G + g) for g in range(G)] +
                 [(nx + m * G + g, nw + (bb * T + t) * G + g) for g in range(G)]
                 for bb in range(B) for m in range(MG) for t in range(T)]
        ct = torch.cat([b.ct_x, b.ct_w]).cpu().numpy()
        pt = torch.cat([b.wm, b.xm]).cpu().numpy()
        want = he.cpmul_terms(he.Params(ctx.N, ctx.q, ctx.t), ct, pt, terms, add=b.rr.cpu().numpy())
        assert np.array_equal(o.cpu().numpy(), want), ctx.N
    # decode one result per client: the exact convolution
    for (ctx, keys, plan, pl, x, w), (pl2, o) in zip(clients, outs[:len(clients)]):
        pl.buf.out.copy_(o)
        y = pl.client_finish().cpu().numpy()
        xs, ws = x.cpu().numpy(), w.cpu().numpy()
        for bb in range(pl.B):
            assert np.array_equal(y[bb], protocol.conv_reference(xs[bb], ws, plan.shape.pad))
    nv.he_server_destroy(srv)


def test_server_admission_under_a_small_budget():
    clients = setup_clients()
    need = [nv.he_server_request_bytes(c.h, p.h, l.B) for (c, k, p, l, _, _) in clients]
    # a budget that holds only about one request at a time (plus item lists)
    budget = 1.3 * max(need) + (1 << 20)
    srv = nv.he_server_create(0, hbm_budget_bytes=budget, max_group=4, max_inflight=2, n_streams=2)
    outs = []
    for rep in range(3):
        for (c, k, p, l, _, _) in clients:
            o = torch.zeros_like(l.buf.out)
            nv.he_server_submit(srv, c.h, p.h, l.B, l.buf.ct_x, l.buf.wm, l.buf.ct_w, l.buf.xm, l.buf.rr, o)
            outs.append((l, o))
    # a request that could never fit is refused at submission (sizes are
    # checked before any buffer is touched)
    ctx, keys, plan, pl, x, w = clients[2]
    with pytest.raises(nv.HEError) as e:
        nv.he_server_submit(srv, ctx.h, plan.h, 4096, pl.buf.ct_x, pl.buf.wm, pl.buf.ct_w, pl.buf.xm, pl.buf.rr,
                            torch.zeros_like(pl.buf.out))
    assert e.value.code == -5
    nv.he_server_wait_all(srv, 120.0)
    st = nv.he_server_stats(srv)
    assert st["completed"] == len(outs) and st["arena_peak_bytes"] <= st["arena_bytes"]
    for l, o in outs:
        assert torch.equal(o, l.buf.out)
    nv.he_server_destroy(srv)


def test_cancel_waiting_requests():
    """Requests still waiting for admission can be withdrawn: with room for
    one request at a time, the later submissions are cancelled, their output
    buffers are never touched, and every request that was not cancelled
    completes with the bits of the request run alone."""
    clients = setup_clients()
    need = [nv.he_server_request_bytes(c.h, p.h, l.B) for (c, k, p, l, _, _) in clients]
    srv = nv.he_server_create(0, hbm_budget_bytes=1.3 * max(need) + (1 << 20), max_group=1, max_inflight=1,
                              n_streams=1)
    subs = []
    for rep in range(4):
        for (c, k, p, l, _, _) in clients:
            o = torch.full_like(l.buf.out.view(torch.int64), 7).view(torch.uint64)
            rid = nv.he_server_submit(srv, c.h, p.h, l.B, l.buf.ct_x, l.buf.wm, l.buf.ct_w, l.buf.xm, l.buf.rr, o)
            subs.append((rid, l, o))
    cancelled = {rid for (rid, l, o) in subs[-6:] if nv.he_server_cancel(srv, rid)}
    assert cancelled, "nothing was still waiting"
    nv.he_server_wait_all(srv, 120.0)
    st = nv.he_server_stats(srv)
    assert st["completed"] == len(subs) - len(cancelled)
    for rid, l, o in subs:
        done, lat = nv.he_server_poll(srv, rid)
        assert done
        if rid in cancelled:
            assert lat < 0 and bool((o.view(torch.int64) == 7).all())
            assert not nv.he_server_cancel(srv, rid)        # cancelling twice reports nothing
        else:
            assert torch.equal(o, l.buf.out)
    assert not nv.he_server_cancel(srv, subs[0][0])      # long finished
    nv.he_server_destroy(srv)
