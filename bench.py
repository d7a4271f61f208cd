"""Benchmark: encrypted CryptoTrain-P conv layers per second on GB300.

Workload (one step): a batch of B images through the 3x32x32 -> 16-channel
3x3 same-padded conv layer, correlated encoding, ring N = 8192 with four
50-bit RNS limbs and t = 1032193.  A step is one pass of the whole hot path:
encode x and w, draw the masks, encrypt x, w and the masks, the offline
CCMul-Precompute ([r^x r^w] with relinearisation), the online fused CPMul +
CCAdd, PPMul, decryption and decoding.  Keys are generated once, before the
timed region (they stay resident on the device).

value: layers (images) per second over all ranks; e2e: the same through the
public API with the input tensors copied from pinned host memory and the
decoded output copied back inside the timed region.

The default line also carries the metric's other parts, each measured for a
few seconds: the batched form against the plain per-job launch (vs_plain),
the served form with p50/p99 latency (serve), this layer under both
encodings (conv_vs_corr) and the plain N = 4096 conventional layer (config1);
and the CPU oracle on every host core (cpu_baseline, with the single-core
rate beside it).

--impl reference times the CPU oracle on the host cores: each step is one
whole image of the layer per core, one single-threaded oracle process per
core.  Under torchrun every rank runs its own batch (weak scaling,
no data-path collective); only the timing uses collectives.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes (read + write) per launch of the k_mac_intt family in this
# workload, averaged over its launches in one ncu capture of this command
# (dram__bytes_read.sum + dram__bytes_write.sum); None once the kernel changes.
MAC_INTT_TRAFFIC = 305.1e6

METRIC = "Encrypted conv layers/s & NTT HBM GB/s (% of peak) vs plain launch; p50/p99 latency"
UNIT = "layers/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="layer", choices=["layer", "train", "batched", "serve", "plancount", "protocols", "alexnet"],
                    help="layer: the 3x32x32 -> 16 CryptoTrain-P layer (default); "
                         "train: one CNN training step's eight linear operations, batch 64; "
                         "batched: 256 uneven ct x pt convolution jobs, plain vs persistent vs graph; "
                         "serve: 64 clients, Poisson arrivals swept over --rates, p50/p99 latency; "
                         "plancount: polynomial products of both packings over input and kernel sizes (no GPU); "
                         "protocols: CryptoTrain-B vs CryptoTrain-P on the same layer (online server time, step); "
                         "alexnet: AlexNet-shaped first convolution and batch norm (64x64x3 input)")
    ap.add_argument("--rates", default="10,30,100,300,1000,2000,6000", help="serve: arrival rates (req/s)")
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="serve: measured seconds per rate")
    ap.add_argument("--serve-warmup", type=float, default=1.0, help="serve: warm-up seconds per rate")
    ap.add_argument("--hbm-budget-gb", type=float, default=150.0, help="serve: admission budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="layer: skip the batched, served, both-encodings and config-1 sub-objects")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples every period_ms (10 ms by default)
    while running.  The serving sweep samples every 100 ms: its windows last
    seconds, and each query takes driver locks that the request server's
    worker also needs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_ms=10):
        self.index = index
        self.period_ms = period_ms
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = sorted(float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit())
        mx = max((float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 5 + i and s[5 + i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(self.samples)}


# ---------------------------------------------------------------- CPU oracle on the host cores
# One image of the layer per task: the whole CryptoTrain-P layer through the
# oracle (encode, masks, 4 encryptions, CCMul-Precompute, CPMul, PPMul,
# decrypt, decode), keys generated once per worker outside the timing.  A
# process pool (spawn start method: the parent may hold a CUDA context) runs
# one task per host core at a time; each worker is single-threaded.
_ORC = {}


def _oracle_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    from oracle import he, packing
    from paper_2409_16675_gb300 import workloads as wl
    w = wl.CONV_MID
    s = w.shape
    P = he.Params.from_spec(w.ring)
    _ORC.update(P=P, keys=he.keygen(P, 1, True), w=w,
                plan=packing.make_plan(w.encoding, P.N, s.C, s.H, s.W, s.M, s.h, s.pad),
                inputs=wl.layer_inputs(w, 8))


def _oracle_image(i):
    from oracle import protocol
    from paper_2409_16675_gb300 import workloads as wl
    x, k = _ORC["inputs"]
    t0 = time.perf_counter()
    protocol.run_layer(_ORC["P"], _ORC["plan"], x[i % len(x)], k, wl.protocol_seeds(_ORC["w"].seed + i),
                       keys=_ORC["keys"])
    return time.perf_counter() - t0


class OraclePool:
    """nproc single-threaded oracle workers; step() runs one image per worker
    and returns (wall seconds, per-image seconds)."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = cores or os.cpu_count() or 1
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init)
        self.next = 0

    def step(self):
        idx = list(range(self.next, self.next + self.cores))
        self.next += self.cores
        t0 = time.perf_counter()
        per = self.pool.map(_oracle_image, idx, chunksize=1)
        return time.perf_counter() - t0, per

    def close(self):
        self.pool.terminate()
        self.pool.join()


ORACLE_SAMPLE = ("one 3x32x32 image per host core per step, all 16 output channels (the whole CryptoTrain-P "
                 "layer: encode, masks, 4 encryptions, CCMul-Precompute, CPMul, PPMul, decrypt, decode), "
                 "one single-threaded oracle process per core; keygen once per process, outside the timing")


def cpu_oracle_baseline():
    """One pool step (one image per core, about 10 s): all-core layers/s, and
    the single-core rate from the same run's per-image times."""
    pool = OraclePool()
    try:
        pool.step()                      # warm-up (imports, tables, first-touch)
        wall, per = pool.step()
    finally:
        pool.close()
    single = len(per) / sum(per)
    return {"value": pool.cores / wall, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": ORACLE_SAMPLE + "; one warm-up step, then one timed step",
            "nproc": os.cpu_count(), "single_core": {"value": single, "unit": UNIT, "cores": 1,
                                                     "ms_per_layer": 1000.0 / single}}


def run_reference(args):
    from paper_2409_16675_gb300 import dist as hd
    ws, rank, _ = hd.world()
    if rank != 0:
        return
    from paper_2409_16675_gb300 import workloads as wl
    pool = OraclePool()
    t_start = time.perf_counter()
    try:
        for _ in range(args.warmup):
            pool.step()
        walls, per = [], []
        for _ in range(args.steps):
            wt, pt = pool.step()
            walls.append(wt)
            per += pt
    finally:
        pool.close()
    total = sum(walls)
    val = pool.cores * args.steps / total
    w = wl.CONV_MID
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": w.name, "batch": pool.cores, "N": w.ring.N, "L": w.ring.L, "t": w.ring.t,
                       "encoding": w.encoding, "images_per_step": pool.cores},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                             "sample": ORACLE_SAMPLE, "nproc": os.cpu_count(),
                             "single_core": {"value": len(per) / sum(per), "unit": UNIT, "cores": 1}},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "consistency": {"timed_s": total, "wall_s_incl_warmup_and_pool": time.perf_counter() - t_start,
                            "extrapolated": False}}
    print(json.dumps(line), flush=True)


def _timed(fn, steps, warmup, stream):
    """ms per call of fn: warm-up calls, then steps calls between CUDA events
    on the launching stream."""
    import torch
    for _ in range(max(1, warmup)):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def config1_measure(steps, warmup, batch=64):
    """Config 1: the plain single encrypted conv layer, conventional encoding,
    CPMul only.  N = 4096, 3 x 36-bit limbs, t = 65537; one 1x28x28 uint8
    image, 4 int8 3x3 kernels, valid.  A step: encode x and w, encrypt x,
    he_cpmul_conv ([x] times the encoded kernels), decrypt, decode.  Timed at
    batch 1 (the latency of one layer) and at `batch` images per call; the
    decoded outputs are checked against a float64 convolution (exact here:
    |values| <= 255 * 8 * 9)."""
    import torch

    from paper_2409_16675_gb300 import layer, native as nv, workloads as wl

    w_ = wl.CONV_SMALL
    s = w_.shape
    ctx = layer.Context(w_.ring)
    keys = layer.Keys(ctx, w_.seed * 7 + 1, False)
    plan = layer.Plan(ctx, s, w_.encoding)
    st = torch.cuda.current_stream()
    x_h, k_h = wl.layer_inputs(w_, batch)
    x_all, k = torch.from_numpy(x_h).cuda(), torch.from_numpy(k_h).cuda()
    out = {}
    exact = True
    for B in (1, batch):
        x = x_all[:B].contiguous()
        nx, nw, no = B * plan.T * plan.G, plan.MG * plan.G, B * plan.MG * plan.T
        xp, wp, ct_x, ct_o, dec = ctx.u64(nx, ctx.N), ctx.u64(nw, ctx.N), ctx.ct(nx), ctx.ct(no), ctx.u64(no, ctx.N)
        y = torch.empty((B, s.M, plan.info.Ho, plan.info.Wo), dtype=torch.int64, device="cuda")

        def step():
            plan.encode_input(x, B, xp)
            plan.encode_kernel(k, wp)
            nv.he_encrypt(ctx.h, keys.h, xp, nx, 1234, ct_x)
            nv.he_cpmul_conv(ctx.h, plan.h, B, ct_x, wp, None, None, None, ct_o)
            nv.he_decrypt(ctx.h, keys.h, ct_o, no, dec)
            nv.he_decode(ctx.h, plan.h, B, dec, None, y)

        ms = _timed(step, steps, warmup, st)
        ref = torch.nn.functional.conv2d(x.double(), k.double(), padding=s.pad).round().long()
        exact = exact and bool(torch.equal(y, ref))
        out["batch%d" % B] = {"ms_per_step": ms, "layers_per_s": B / (ms / 1000.0)}
    plan.close()
    keys.close()
    ctx.close()
    return {"workload": w_.name, **out, "products_per_image": plan.products,
            "decoded_equals_integer_conv": exact, "steps": steps, "warmup": warmup}


def conv_vs_corr_measure(steps, warmup, batch=64):
    """Config 2 under both encodings: the whole CryptoTrain-P layer step
    (3x32x32 -> 16, 3x3 same, N = 8192, 4 x 50-bit, batch `batch`) with the
    conventional and with the correlated packing; both decode to the same
    integer convolution."""
    import torch

    from paper_2409_16675_gb300 import layer, workloads as wl

    w_ = wl.CONV_MID
    ctx = layer.Context(w_.ring)
    keys = layer.Keys(ctx, w_.seed * 7 + 1, True)
    x_h, k_h = wl.layer_inputs(w_, batch)
    x, k = torch.from_numpy(x_h).cuda(), torch.from_numpy(k_h).cuda()
    seeds = wl.protocol_seeds(w_.seed)
    st = torch.cuda.current_stream()
    res, ys = {}, {}
    for enc in ("conv", "corr"):
        plan = layer.Plan(ctx, w_.shape, enc)
        pl = layer.PLayer(ctx, keys, plan, batch)
        ms = _timed(lambda: pl.step(x, k, seeds), steps, warmup, st)
        ys[enc] = pl.buf.y.clone()
        res[enc] = {"ms_per_step": ms, "layers_per_s": batch / (ms / 1000.0), "products_per_image": plan.products,
                    "input_polys_per_image": plan.T * plan.G}
        del pl
        plan.close()
    keys.close()
    ctx.close()
    return {"workload": w_.name, "batch": batch, **res,
            "corr_speedup": res["conv"]["ms_per_step"] / res["corr"]["ms_per_step"],
            "same_decoded_outputs": bool(torch.equal(ys["conv"], ys["corr"])), "steps": steps, "warmup": warmup}


def run_gpu(args):
    import torch

    from paper_2409_16675_gb300 import dist as hd
    ws, rank, local = hd.world()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_2409_16675_gb300 import layer, native as nv, workloads as wl

    w = wl.CONV_MID
    s = w.shape
    B = args.batch
    ctx = layer.Context(w.ring, device=local)
    keys = layer.Keys(ctx, hd.rank_seed(w.seed * 7 + 1, rank), True)
    plan = layer.Plan(ctx, s, w.encoding)
    pl = layer.PLayer(ctx, keys, plan, B)
    x_h, k_h = wl.layer_inputs(w, B)
    x_h = x_h.copy()
    x_h[0, 0, 0, 0] = rank % 256
    x = torch.from_numpy(x_h).cuda()
    k = torch.from_numpy(k_h).cuda()
    stream = torch.cuda.current_stream()

    def step(i):
        return pl.step(x, k, wl.protocol_seeds(hd.rank_seed(w.seed + 17 * i, rank)))

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    def barrier():
        hd.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed regions: the first (no per-launch events)
    # gives the value; the second, the same K steps with the library's launch
    # trace on (a CUDA event pair around every launch), gives the per-kernel
    # times of the roofline
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tv0, tv1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for i in range(args.steps):
            step(args.warmup + i)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        nv.he_trace_enable(ctx.h, True)
        barrier()
        tv0.record(stream)
        for i in range(args.steps):
            step(args.warmup + args.steps + i)
        tv1.record(stream)
        torch.cuda.synchronize()
        barrier()
        nv.he_trace_enable(ctx.h, False)
    trace = nv.he_trace_read(ctx.h)
    ms = hd.reduce_max(ev0.elapsed_time(ev1), device="cuda")
    ms_traced = hd.reduce_max(tv0.elapsed_time(tv1), device="cuda")
    ms_step = ms / args.steps
    value = hd.whole_job_rate(B * args.steps, ws, ms / 1000.0)

    # ---- end to end through the API with host buffers: every step copies its
    # inputs from pinned host memory and its decoded output back.  The copies
    # run on a second stream, overlapped with the neighbouring steps' kernels
    # (two sets of layer buffers alternate; events order each copy after the
    # step it feeds or drains), and the timed region ends once the last
    # output copy has landed.
    pls = [pl, layer.PLayer(ctx, keys, plan, B)]
    xp = torch.from_numpy(x_h).pin_memory()
    kp = torch.from_numpy(k_h).pin_memory()
    yps = [torch.empty(pl.buf.y.shape, dtype=torch.int64).pin_memory() for _ in range(2)]
    xds, kds = [torch.empty_like(x) for _ in range(2)], [torch.empty_like(k) for _ in range(2)]
    cs = torch.cuda.Stream()
    in_ev = [torch.cuda.Event() for _ in range(2)]
    out_ev = [torch.cuda.Event() for _ in range(2)]
    back_ev = [torch.cuda.Event() for _ in range(2)]

    def e2e_step(i):
        j = i % 2
        with torch.cuda.stream(cs):
            xds[j].copy_(xp, non_blocking=True)
            kds[j].copy_(kp, non_blocking=True)
            in_ev[j].record(cs)
        stream.wait_event(in_ev[j])
        stream.wait_event(back_ev[j])        # this buffer set's previous output has been copied out
        y = pls[j].step(xds[j], kds[j], wl.protocol_seeds(hd.rank_seed(w.seed + 31 * i, rank)))
        out_ev[j].record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(out_ev[j])
            yps[j].copy_(y, non_blocking=True)
            back_ev[j].record(cs)

    for i in range(max(1, args.warmup)):
        e2e_step(i)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        e2e_step(1000 + i)
    for ev in back_ev:
        stream.wait_event(ev)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ems = hd.reduce_max(e0.elapsed_time(e1), device="cuda")
    e2e_value = hd.whole_job_rate(B * args.steps, ws, ems / 1000.0)
    yp = yps[0]

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    # ---- roofline of the dominant kernel family
    peak, peak_kind = peaks()
    clocks = clk.summary()
    # kernel families (the part of a trace name before the call site's role)
    fam = {}
    for k, (n, t, b_, m_) in trace.items():
        f = fam.setdefault(k.split(".")[0], [0, 0.0, 0.0, 0.0])
        f[0] += n; f[1] += t; f[2] += b_; f[3] += m_
    name, (launches, tot_ms, byt, mm) = max(fam.items(), key=lambda kv: kv[1][1])
    gbs = byt / (tot_ms / 1000.0) / 1e9
    # The NTT / multiply-accumulate kernels are bound by the integer multiply
    # pipe, not by HBM: peak = SMs x 64 IMAD lanes per cycle x SM clock / 10
    # (the 32-bit multiplies of one 64-bit Shoup modular product); achieved =
    # algorithmic modular products (butterflies, untwist/scaling products, MAC
    # terms) per second over the kernel's event-timed launches.
    # The key-switch families (ks_*) count 32-bit modular products: a Shoup
    # product there is one high-half multiply (half rate, two lane slots) and
    # two low multiplies, so their peak is the same lane rate / 4.
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clocks.get("sm_max_mhz") or 2070.0
    per_product = 4 if name.startswith("ks_") else 10
    alu_peak = sms * 64 * mhz * 1e6 / per_product / 1e12
    alu = mm / (tot_ms / 1000.0) / 1e12
    roof = {"kernel": name, "bound": "alu", "achieved": alu, "peak": alu_peak,
            "unit": "Tmodmul32/s" if per_product == 4 else "Tmodmul/s",
            "frac": alu / alu_peak,
            "peak_source": "derived: %d SMs x 64 IMAD lanes/cycle x %.0f MHz / %d IMAD per %d-bit modular product"
                           % (sms, mhz, per_product, 32 if per_product == 4 else 64),
            "traffic": MAC_INTT_TRAFFIC if name == "mac_intt" else None,
            "launches": launches, "avg_launch_us": 1000.0 * tot_ms / launches,
            "timed_region": "the same K steps again with a CUDA event pair around every launch: %.3f ms per step"
                            % (ms_traced / args.steps),
            "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                    "peak_source": peak_kind + " (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured" else peak_kind}}
    total_ms = sum(u[1] for u in trace.values())
    kernels = {k: {"launches": v[0], "ms": v[1], "share": v[1] / total_ms,
                   "GB/s": v[2] / (v[1] / 1000.0) / 1e9 if v[1] else None,
                   ("Tmodmul32/s" if k.startswith("ks_") else "Tmodmul/s"):
                       v[3] / (v[1] / 1000.0) / 1e12 if v[1] else None}
               for k, v in sorted(trace.items(), key=lambda kv: -kv[1][1])}
    families = {k: {"launches": v[0], "ms": v[1], "share": v[1] / total_ms} for k, v in fam.items()}
    launches_total = sum(v[0] for v in trace.values())
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": w.name, "batch": B, "N": w.ring.N, "L": w.ring.L, "t": w.ring.t,
                       "encoding": w.encoding, "parallelism": "independent batches per GPU" if ws > 1 else "1 GPU",
                       "l2": "inputs larger than L2 (working set of one step > 129 MB)"},
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(x_h.nbytes + k_h.nbytes),
                    "d2h_bytes_per_step": int(yp.numel() * 8),
                    "copies": "pinned host <-> device on a second stream, overlapped with the neighbouring steps; "
                              "the timed region ends after the last output copy"},
            "gpu_launches": int(launches_total),
            "roofline": roof,
            "kernels": kernels, "families": families}
    if ws == 1 and not args.no_extras:
        # the metric's other parts, each bounded to seconds: the batched form
        # against the plain per-job launch (config 4), the served form with
        # p50/p99 (config 5), both encodings of this layer (config 2) and the
        # plain N = 4096 conventional layer (config 1)
        line["vs_plain"] = batched_measure(5, 2)
        line["serve"] = serve_measure([300.0, 1000.0, 2000.0], 2.0, 0.5, args.hbm_budget_gb)
        line["conv_vs_corr"] = conv_vs_corr_measure(10, 2)
        line["config1"] = config1_measure(20, 3)
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_oracle_baseline()
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def run_train(args):
    """Training steps per second: the eight homomorphic linear operations of one
    step of the 1x28x28 CNN (conv 1->16, conv 16->32, FC 512->10; forward,
    input and weight gradients), batch 64, N = 8192, 4 x 50-bit limbs, 40-bit t,
    with the OT non-linear layers simulated in plaintext."""
    import numpy as np
    import torch

    from paper_2409_16675_gb300 import layer, training, workloads as wl

    B = 64
    spec = training.CNNSpec()
    ctx = layer.Context(wl.RING_TRAIN)
    keys = layer.Keys(ctx, 7, True)
    tr = training.HETrainer(ctx, keys, B, spec)
    rng = np.random.default_rng(wl.MASTER_SEED + 3)
    x0 = torch.from_numpy(rng.integers(0, 256, (B, 1, 28, 28), dtype=np.uint8)).cuda()
    w1 = torch.from_numpy(rng.integers(-8, 8, (spec.c1, 1, 3, 3), dtype=np.int8)).cuda()
    w2 = torch.from_numpy(rng.integers(-8, 8, (spec.c2, spec.c1, 3, 3), dtype=np.int8)).cuda()
    w3 = torch.from_numpy(rng.integers(-8, 8, (spec.n_out, spec.fc_in), dtype=np.int8)).cuda()
    lab = torch.from_numpy(rng.integers(0, 10, (B,), dtype=np.int64)).cuda()
    for i in range(args.warmup):
        tr.step(x0, w1, w2, w3, lab, seed=100 * i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record()
        for i in range(args.steps):
            tr.step(x0, w1, w2, w3, lab, seed=100 * (args.warmup + i))
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"metric": "encrypted CNN training steps/s (linear layers, batch 64)", "value": 1000.0 / ms,
                      "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms, "higher_is_better": True, "dtype": "u64", "data": "synthetic",
                      "config": {"workload": "cnn_train_step_b64_N8192", "batch": B,
                                 "products_per_step": tr.products()},
                      "clocks": clk.summary()}), flush=True)
    tr.close()


def batched_measure(steps, warmup, sample_every=16):
    """Config 4: 256 ct x pt convolution jobs of uneven shapes (channels
    {3,16,32,64,128}, spatial {8,16,32}, kernel {1,3,5}), N in {4096, 8192},
    2-5 limbs of 36-60 bits, both encodings.  ms per batch as one call per job
    (plain), as per-degree work-list launches (persistent), as one persistent
    launch for the whole batch (fused), and replayed from a CUDA graph of the
    faster of the last two, after the autotuner has picked the launch
    configuration; every sample_every-th job's output compared across the
    modes."""
    import torch

    from paper_2409_16675_gb300 import layer, native as nv, workloads as wl

    t_setup = time.perf_counter()
    jobs = wl.batched_jobs()
    ctxs, items = {}, []
    for j in jobs:
        key = (j.ring.N, j.ring.prime_bits)
        if key not in ctxs:
            ctxs[key] = layer.Context(j.ring)
        c = ctxs[key]
        p = layer.Plan(c, j.shape, j.encoding)
        g = torch.Generator(device="cuda").manual_seed(j.seed)
        nx, nw = p.T * p.G, p.MG * p.G
        ct = torch.empty((nx, 2, c.L, c.N), dtype=torch.int64, device="cuda")
        for i, q in enumerate(c.q):
            ct[:, :, i, :] = torch.randint(0, q, (nx, 2, c.N), generator=g, device="cuda", dtype=torch.int64)
        pt = torch.randint(0, c.t, (nw, c.N), generator=g, device="cuda", dtype=torch.int64)
        items.append((c, p, ct.view(torch.uint64), pt.view(torch.uint64), c.ct(p.MG * p.T)))
    b = nv.he_batch_create(0)
    for (c, p, ct, pt, out) in items:
        nv.he_batch_add_cpmul(b, c.h, p.h, 1, ct, pt, None, out)
    nv.he_batch_prepare(b)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    s = torch.cuda.Stream()
    res, outs = {}, {}
    with torch.cuda.stream(s):
        t0 = time.perf_counter()
        tuning = nv.he_batch_autotune(b)
        tune_s = time.perf_counter() - t0
        info = nv.he_batch_query(b)
        modes = [("plain", nv.HE_BATCH_PLAIN), ("persistent", nv.HE_BATCH_PERSISTENT)]
        if info["fused_supported"]:
            modes.append(("fused", nv.HE_BATCH_FUSED))
        modes.append(("graph", nv.HE_BATCH_GRAPH))
        for name, mode in modes:
            for it in items:
                it[4].zero_()
            for _ in range(max(1, warmup)):
                nv.he_batch_run(b, mode)
            s.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(steps):
                nv.he_batch_run(b, mode)
            e1.record(s)
            s.synchronize()
            res[name] = e0.elapsed_time(e1) / steps
            nv.he_batch_status(b)
            outs[name] = [it[4].clone() for it in items[::sample_every]]
    same = all(torch.equal(a, r) for m in outs for a, r in zip(outs[m], outs["plain"]))
    nv.he_batch_destroy(b)
    for (c, p, ct, pt, out) in items:
        p.close()
    for c in ctxs.values():
        c.close()
    return {"jobs": len(jobs), "ms_per_batch": res,
            "jobs_per_s": {k: len(jobs) / (v / 1000.0) for k, v in res.items()},
            "speedup_vs_plain": {k: res["plain"] / v for k, v in res.items()},
            "identical_results": bool(same), "compared_jobs": len(outs["plain"]), "autotune": tuning,
            "one_launch": {"graph_uses_it": bool(info["graph_fused"]), "regs_ctas_per_sm": info["fused_regs_ctas_per_sm"],
                           "units": info["n_units"], "autotune_ms": info["fused_ms"],
                           "per_degree_autotune_ms": info["per_degree_ms"]},
            "contexts": len(ctxs), "steps": steps, "warmup": warmup, "setup_s": setup_s, "autotune_s": tune_s}


def run_batched(args):
    r = batched_measure(args.steps, args.warmup)
    print(json.dumps({"metric": "batched ct x pt conv jobs/s (256 uneven jobs)", "unit": "jobs/s",
                      "value": r["jobs_per_s"]["graph"], "higher_is_better": True,
                      "steps": args.steps, "warmup": args.warmup, "dtype": "u64", "data": "synthetic",
                      **r, "config": {"workload": "256 uneven conv jobs, N 4096/8192, 2-5 limbs of 36-60 bits"}}),
          flush=True)


def serve_measure(rates, seconds, warmup_s, budget_gb):
    """Served form: 64 clients, each with its own ring (N in {4096, 8192,
    16384}, 2-8 limbs of 36-60 bits), keys, plan and layer (shapes as in the
    batched form), whose encrypted inputs, masked plaintexts and precomputed
    [r^x r^w] stay resident on the device.  One request is the online phase
    of one CryptoTrain-P layer (two CPMuls and the precomputed add, one
    image).  Requests arrive open-loop as a Poisson process at each rate; a
    client holds at most DEPTH requests in flight (one output buffer each) and
    an arrival that finds all of them busy is shed.  Reported per rate: layers
    per second (completions over the span from first submission to last
    completion), p50/p99 latency (submission to completion), shed arrivals;
    plus the saturated throughput of the server against one he_cpmul_conv
    call per request on one stream (the plain launch), and whether every
    sampled result equals the request run alone."""
    import numpy as np
    import torch

    from paper_2409_16675_gb300 import layer, native as nv, workloads as wl

    DEPTH = 4
    t0 = time.perf_counter()
    clients = []
    for j in wl.served_clients():
        s = j.shape
        ctx = layer.Context(j.ring)
        keys = layer.Keys(ctx, j.seed, True)
        plan = layer.Plan(ctx, s, j.encoding)
        pl = layer.PLayer(ctx, keys, plan, 1)
        x = torch.from_numpy(wl.activations(j.seed + 1, (1, s.C, s.H, s.W))).cuda()
        w = torch.from_numpy(wl.weights(j.seed + 2, (s.M, s.C, s.h, s.h))).cuda()
        pl.client_prepare(x, w, wl.protocol_seeds(j.seed))
        pl.offline()                          # [r^x r^w], resident
        pl.online()                           # the request alone: pl.buf.out
        clients.append((ctx, keys, plan, pl, [torch.empty_like(pl.buf.out) for _ in range(DEPTH)]))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    resident = torch.cuda.memory_allocated()

    def submit(srv, ci, slot):
        ctx, keys, plan, pl, outs = clients[ci]
        b = pl.buf
        return nv.he_server_submit(srv, ctx.h, plan.h, 1, b.ct_x, b.wm, b.ct_w, b.xm, b.rr, outs[slot])

    # plain launch: one he_cpmul_conv per request, one stream
    reps = 3
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        for _ in range(2):
            for (ctx, keys, plan, pl, outs) in clients:
                b = pl.buf
                nv.he_cpmul_conv(ctx.h, plan.h, 1, b.ct_x, b.wm, b.ct_w, b.xm, b.rr, outs[0])
        st.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            for (ctx, keys, plan, pl, outs) in clients:
                b = pl.buf
                nv.he_cpmul_conv(ctx.h, plan.h, 1, b.ct_x, b.wm, b.ct_w, b.xm, b.rr, outs[0])
        e1.record(st)
        st.synchronize()
    plain_lps = reps * len(clients) / (e0.elapsed_time(e1) / 1000.0)

    srv = nv.he_server_create(0, hbm_budget_bytes=budget_gb * 1e9, max_group=64, max_inflight=4,
                              n_streams=4, poll_us=20)
    # saturation: every client submits DEPTH requests at once
    for rep in range(2):
        nv.he_server_reset_stats(srv)
        for slot in range(DEPTH):
            for ci in range(len(clients)):
                submit(srv, ci, slot)
        nv.he_server_wait_all(srv, 600.0)
        sat = nv.he_server_stats(srv)
    sat_lps = sat["completed"] / sat["span_s"]
    same = all(torch.equal(outs[k], pl.buf.out) for (_, _, _, pl, outs) in clients for k in range(DEPTH))

    sweep = []
    gpu = int(os.environ.get("LOCAL_RANK", "0"))
    with ClockSampler(gpu, 100) as clk:
        for ri, rate in enumerate(rates):
            times, who = wl.poisson_arrivals(wl.MASTER_SEED + 50 + ri, rate, warmup_s + seconds, len(clients))
            inflight = [[] for _ in clients]          # (request id, slot)
            shed, lag, measured = 0, [], False
            start = time.perf_counter()
            for tt, ci in zip(times, who):
                if not measured and tt >= warmup_s:
                    nv.he_server_reset_stats(srv)
                    measured = True
                while True:
                    dt = start + tt - time.perf_counter()
                    if dt <= 0:
                        break
                    if dt > 2e-4:
                        time.sleep(dt - 1e-4)
                inflight[ci] = [(r, k) for (r, k) in inflight[ci] if not nv.he_server_poll(srv, r)[0]]
                if len(inflight[ci]) >= DEPTH:
                    if measured:
                        shed += 1
                    continue
                busy = {k for _, k in inflight[ci]}
                slot = next(k for k in range(DEPTH) if k not in busy)
                inflight[ci].append((submit(srv, ci, int(slot)), slot))
                if measured:
                    lag.append(time.perf_counter() - (start + tt))
            nv.he_server_wait_all(srv, 600.0)
            r = nv.he_server_stats(srv)
            same = same and all(torch.equal(outs[k], pl.buf.out)
                                for (_, _, _, pl, outs) in clients[:: 7] for k in range(DEPTH))
            sweep.append({"rate": rate, "completed": r["completed"], "shed": shed,
                          "layers_per_s": r["completed"] / r["span_s"] if r["span_s"] > 0 else 0.0,
                          "p50_ms": r["p50_us"] / 1e3, "p99_ms": r["p99_us"] / 1e3, "max_ms": r["max_us"] / 1e3,
                          "groups": r["groups"], "arena_peak_gb": r["arena_peak_bytes"] / 1e9,
                          "submit_lag_p99_ms": float(np.percentile(lag, 99)) * 1e3 if lag else None})
    nv.he_server_destroy(srv)
    for (ctx, keys, plan, pl, outs) in clients:
        keys.close()
        plan.close()
        ctx.close()
    return {"saturated_layers_per_s": sat_lps, "plain_launch_layers_per_s": plain_lps,
            "speedup_vs_plain": sat_lps / plain_lps,
            "saturation": {"requests": sat["completed"], "p50_ms": sat["p50_us"] / 1e3,
                           "p99_ms": sat["p99_us"] / 1e3, "groups": sat["groups"]},
            "sweep": sweep, "identical_results": bool(same), "clocks": clk.summary(),
            "setup_s": setup_s, "resident_gb": resident / 1e9,
            "config": {"workload": "64 clients, N 4096/8192/16384, 2-8 limbs of 36-60 bits, batched-form shapes, "
                                   "one image per request",
                       "hbm_budget_gb": budget_gb, "seconds_per_rate": seconds, "warmup_s_per_rate": warmup_s,
                       "max_requests_per_client": DEPTH}}


def run_serve(args):
    """Served form (config 5), see serve_measure."""
    r = serve_measure([float(x) for x in args.rates.split(",")], args.serve_seconds, args.serve_warmup,
                      args.hbm_budget_gb)
    print(json.dumps({
        "metric": "served CryptoTrain-P layers/s with p50/p99 latency (64 clients, Poisson arrivals)",
        "unit": "layers/s", "value": r["saturated_layers_per_s"], "higher_is_better": True, "n_gpus": 1,
        "dtype": "u64", "data": "synthetic", **r}), flush=True)


def run_plancount(args):
    """Multiply-count sweep of Section 3.3 / Fig. 8: polynomial products per
    image (MG * G * T) of the conventional and the correlated packing for a
    C = 3 input of H x H, kernels h x h with same and valid padding, M = 3
    output channels, at N = 2048, 4096, 8192.  Host-only plan search."""
    from paper_2409_16675_gb300 import native as nv
    rows, best = [], None
    for N in (2048, 4096, 8192):
        for H in (8, 16, 32, 64):
            for h in (1, 3, 5, 7, 9, 11):
                if h > H:
                    continue
                for pad in sorted({0, h // 2}):
                    cnt = {}
                    for name, enc in (("conv", nv.HE_ENC_CONVENTIONAL), ("corr", nv.HE_ENC_CORRELATED)):
                        try:
                            i = nv.he_plan_search(N, 3, H, H, 3, h, pad, enc)
                            cnt[name] = i.MG * i.G * i.T
                        except nv.HEError:
                            cnt[name] = None
                    r = (cnt["conv"] / cnt["corr"]) if cnt["conv"] and cnt["corr"] else None
                    rows.append({"N": N, "H": H, "h": h, "pad": pad, "conventional": cnt["conv"],
                                 "correlated": cnt["corr"], "ratio": r})
                    if r is not None and (best is None or r > best["ratio"]):
                        best = rows[-1]
    print(json.dumps({"metric": "polynomial products per image, conventional vs correlated packing (Fig. 8 sweep)",
                      "unit": "products", "value": best["ratio"] if best else None, "max_ratio_at": best,
                      "rows": rows, "data": "plan search only",
                      "config": {"workload": "C=3, M=3, H in {8,16,32,64}, h in {1..11}, N in {2048,4096,8192}"}}),
          flush=True)


def run_protocols(args):
    """CryptoTrain-B (Section 3.1) against CryptoTrain-P (Section 3.2) on the
    3x32x32 -> 16 layer at N = 8192, batch 64: the server's online work (B: the
    [x][w] CCMul with relinearisation; P: the fused two-CPMul + CCAdd and the
    PPMul), the offline work of P (CCMul-Precompute), and whole steps.  The
    paper reports CCMul at about 7x a CPMul on its CPU (Section 3.2)."""
    import torch

    from paper_2409_16675_gb300 import layer, native as nv, workloads as wl

    w_ = wl.CONV_MID
    B = args.batch
    ctx = layer.Context(w_.ring)
    keys = layer.Keys(ctx, w_.seed * 7 + 1, True)
    plan = layer.Plan(ctx, w_.shape, w_.encoding)
    pl, bl = layer.PLayer(ctx, keys, plan, B), layer.BLayer(ctx, keys, plan, B)
    x_h, k_h = wl.layer_inputs(w_, B)
    x, k = torch.from_numpy(x_h).cuda(), torch.from_numpy(k_h).cuda()
    seeds = wl.protocol_seeds(w_.seed)
    st = torch.cuda.current_stream()

    def timed(fn, reps):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    pl.client_prepare(x, k, seeds)
    bl.client_prepare(x, k, seeds)
    reps = max(3, args.steps)
    p_offline = timed(pl.offline, reps)
    p_online = timed(pl.online, reps)
    b_online = timed(bl.online, reps)
    p_step = timed(lambda: pl.step(x, k, seeds), reps)
    b_step = timed(lambda: bl.step(x, k, seeds), reps)
    same = bool(torch.equal(pl.client_finish(), bl.client_finish()))
    print(json.dumps({
        "metric": "CryptoTrain-B vs CryptoTrain-P linear layer (3x32x32 -> 16, N=8192, batch %d)" % B,
        "unit": "ms", "value": b_online / p_online, "higher_is_better": False, "n_gpus": 1, "dtype": "u64",
        "data": "synthetic", "steps": reps, "warmup": args.warmup,
        "online_ms": {"B_ccmul": b_online, "P_cpmul_ppmul": p_online}, "P_offline_ms": p_offline,
        "step_ms": {"B": b_step, "P": p_step}, "online_ratio_B_over_P": b_online / p_online,
        "layers_per_s": {"B": B / (b_step / 1000.0), "P": B / (p_step / 1000.0)},
        "same_decoded_outputs": same,
        "config": {"workload": w_.name, "batch": B, "N": w_.ring.N, "L": w_.ring.L, "t": w_.ring.t}}), flush=True)


def run_alexnet(args):
    """AlexNet-shaped layers on a 64x64x3 (Tiny-ImageNet-sized) input as
    CryptoTrain-P layers, whole steps (encode, masks, encryptions, offline
    CCMul-Precompute, online, PPMul, decryption, decoding): the first
    convolution 3 -> 64 with an 11x11 kernel (same padding, stride 1) and a
    batch norm over its 64 channels (diagonal 1x1 kernel and bias, under the
    depthwise plan: one product per kernel polynomial and tile).  Ring
    N = 8192 with 4 x 50-bit limbs and a 40-bit t (no wrap of the sums);
    batch at most 16."""
    import torch

    from paper_2409_16675_gb300 import layer, workloads as wl

    B = min(args.batch, 16)
    ctx = layer.Context(wl.RING_TRAIN)
    keys = layer.Keys(ctx, 77, True)
    out = {}
    specs = [("conv1_3x64x64_64_k11", wl.ConvShape(3, 64, 64, 64, 11, 5), False),
             ("bn1_64x64x64", wl.ConvShape(64, 64, 64, 64, 1, 0), True)]
    for name, shape, bn in specs:
        cands = [layer.Plan(ctx, shape, e, depthwise=bn) for e in ("corr", "conv")]
        plan = min(cands, key=lambda p: p.products)
        pl = layer.PLayer(ctx, keys, plan, B, with_bias=bn)
        x = torch.from_numpy(wl.activations(5, (B, shape.C, shape.H, shape.W))).cuda()
        if bn:
            gamma = torch.from_numpy(wl.weights(6, (shape.C,)).astype("int64")).cuda()
            w, beta = layer.batch_norm_weights(gamma), torch.arange(shape.C, device="cuda") - 32
        else:
            w, beta = torch.from_numpy(wl.weights(6, (shape.M, shape.C, shape.h, shape.h))).cuda(), None
        seeds = wl.protocol_seeds(9)
        for _ in range(max(1, args.warmup)):
            pl.step(x, w, seeds, beta)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(1, args.steps)
        e0.record()
        for _ in range(reps):
            pl.step(x, w, seeds, beta)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms_per_step": ms, "images_per_s": B / (ms / 1000.0), "encoding": plan.encoding,
                     "depthwise": plan.depthwise, "products_per_image": plan.products}
        for p in cands:
            p.close()
    print(json.dumps({"metric": "AlexNet-shaped CryptoTrain-P layers, images/s (batch %d)" % B, "unit": "images/s",
                      "value": out["conv1_3x64x64_64_k11"]["images_per_s"], "higher_is_better": True, "n_gpus": 1,
                      "dtype": "u64", "data": "synthetic", "layers": out, "steps": args.steps, "warmup": args.warmup,
                      "config": {"workload": "64x64x3 input, conv 11x11 -> 64, batch norm 64; N=8192, 4x50-bit, 40-bit t",
                                 "batch": B}}), flush=True)


def main():
    args = parse()
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    if args.workload == "plancount":
        run_plancount(args)
        return
    if args.workload == "protocols":
        run_protocols(args)
        return
    if args.workload == "alexnet":
        run_alexnet(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "train":
        run_train(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
