"""Thin Python binding of the C ABI in include/cryptotrain.h.

Argument marshalling only: every function has the name of its C entry point,
takes PyTorch CUDA tensors (or None for NULL), passes their device pointers
and the current CUDA stream, and raises HEError on a negative status.  All
computation happens in libcryptotrain.so; there is no fallback of any kind:
importing this module without the built library raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# CRYPTOTRAIN_LIB=checks selects the bounds-checked debug build of the same
# library (libcryptotrain_checks.so, built by build.build_checks()).
LIB_NAME = "libcryptotrain_checks.so" if os.environ.get("CRYPTOTRAIN_LIB") == "checks" else "libcryptotrain.so"
LIB_PATH = os.path.join(_HERE, LIB_NAME)

HE_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "UNSUPPORTED_PARAMS", -3: "PLAN_DOES_NOT_FIT", -4: "OOM",
          -5: "BUDGET_EXCEEDED", -6: "TIMEOUT", -7: "CUDA"}
HE_MAX_LIMBS = 16
HE_ENC_CONVENTIONAL, HE_ENC_CORRELATED = 0, 1
HE_ROLE_INPUT, HE_ROLE_KERNEL = 0, 1
HE_DTYPE_U8, HE_DTYPE_I8, HE_DTYPE_I64 = 0, 1, 2
HE_PLAN_DEPTHWISE = 16
HE_KEY_SK, HE_KEY_PK, HE_KEY_RLK = 0, 1, 2
HE_BATCH_PLAIN, HE_BATCH_PERSISTENT, HE_BATCH_GRAPH, HE_BATCH_FUSED = 0, 1, 2, 3


class HEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class he_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("L", ctypes.c_int32), ("prime_bits", ctypes.c_int32 * HE_MAX_LIMBS),
                ("q", ctypes.c_uint64 * HE_MAX_LIMBS), ("t", ctypes.c_uint64), ("base_log2", ctypes.c_int32),
                ("eta", ctypes.c_int32), ("max_ccmul_group", ctypes.c_int32), ("device", ctypes.c_int32),
                ("max_ccmul_scratch_bytes", ctypes.c_double), ("max_table_cache_bytes", ctypes.c_double)]


class he_ctx_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("L", ctypes.c_int32), ("q", ctypes.c_uint64 * HE_MAX_LIMBS),
                ("t", ctypes.c_uint64), ("ell", ctypes.c_int32), ("n_aux", ctypes.c_int32),
                ("aux", ctypes.c_uint64 * 24), ("ppmul_ok", ctypes.c_int32),
                ("ks_primes", ctypes.c_int32)]


class he_conv_shape(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("C", "H", "W", "M", "h", "pad")]


class he_trace_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("modmuls", ctypes.c_double)]


class he_batch_info(ctypes.Structure):
    _fields_ = [("fused_supported", ctypes.c_int32), ("graph_fused", ctypes.c_int32),
                ("fused_regs_ctas_per_sm", ctypes.c_int32), ("n_units", ctypes.c_int32),
                ("fused_ms", ctypes.c_float), ("per_degree_ms", ctypes.c_float)]


class he_batch_tuning(ctypes.Structure):
    _fields_ = [("logN", ctypes.c_int32), ("regs_ctas_per_sm", ctypes.c_int32), ("grid_ctas_per_sm", ctypes.c_int32),
                ("ms", ctypes.c_float), ("fwd_items", ctypes.c_int32), ("mac_items", ctypes.c_int32)]


class he_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_double), ("max_group", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("n_streams", ctypes.c_int32), ("poll_us", ctypes.c_int32)]


class he_server_report(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("images", ctypes.c_int64),
                ("groups", ctypes.c_int64), ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double), ("span_s", ctypes.c_double),
                ("arena_peak_bytes", ctypes.c_double), ("arena_bytes", ctypes.c_double)]


class he_plan_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("encoding", "Cn", "G", "th", "tw", "Th", "Tw", "T", "Hn", "Wn",
                                              "Ooff", "O", "S", "Ho", "Wo", "Mn", "Sout", "MG", "depthwise")]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("%s is not built (run __graft_entry__.build()); "
                          "there is no fallback implementation" % LIB_NAME)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "he_setup": [ctypes.POINTER(he_params), pp],
        "he_ctx_destroy": [vp],
        "he_ctx_query": [vp, ctypes.POINTER(he_ctx_info)],
        "he_last_error": [vp, ctypes.c_char_p, i32],
        "he_keygen": [vp, u64, i32, pp, vp],
        "he_keys_destroy": [vp],
        "he_keys_export": [vp, vp, i32, vp, vp],
        "he_encrypt": [vp, vp, vp, i32, u64, vp, vp],
        "he_decrypt": [vp, vp, vp, i32, vp, vp],
        "he_sample_masks": [vp, u64, i32, vp, vp],
        "he_pt_sub": [vp, vp, vp, i64, vp, vp],
        "he_conv_plan": [vp, ctypes.POINTER(he_conv_shape), i32, pp],
        "he_plan_destroy": [vp],
        "he_plan_query": [vp, ctypes.POINTER(he_plan_info)],
        "he_plan_search": [i32, ctypes.POINTER(he_conv_shape), i32, ctypes.POINTER(he_plan_info)],
        "he_ks_primes": [ctypes.POINTER(he_params), ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(i32)],
        "he_encode_conventional": [vp, vp, i32, vp, i32, i32, vp, vp],
        "he_encode_correlated": [vp, vp, i32, vp, i32, i32, vp, vp],
        "he_cpmul_conv": [vp, vp, i32, vp, vp, vp, vp, vp, vp, vp],
        "he_keys_import": [vp, vp, vp, vp, pp, vp],
        "he_ctx_fingerprint": [vp, ctypes.POINTER(u64)],
        "he_encrypt_symmetric": [vp, vp, vp, i32, u64, vp, vp],
        "he_expand_symmetric": [vp, u64, i32, vp, vp, vp],
        "he_encrypt_many": [vp, vp, i32, ctypes.POINTER(vp), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint64),
                            ctypes.POINTER(vp), vp],
        "he_cpmul_conv_noalloc": [vp, vp, i32, vp, vp, vp, vp, vp, vp, vp],
        "he_ccmul_precompute": [vp, vp, vp, i32, vp, i32, vp, vp, i32, i32, vp, vp],
        "he_ccmul_conv_precompute": [vp, vp, vp, i32, vp, vp, vp, vp],
        "he_ppmul_conv": [vp, vp, i32, vp, vp, vp, vp],
        "he_decode": [vp, vp, i32, vp, vp, vp, vp],
        "he_encode_output": [vp, vp, i32, vp, vp, vp],
        "he_ct_add": [vp, vp, vp, i32, vp, vp],
        "he_batch_create": [i32, pp],
        "he_batch_destroy": [vp],
        "he_batch_last_error": [vp, ctypes.c_char_p, i32],
        "he_batch_add_cpmul": [vp, vp, vp, i32, vp, vp, vp, vp],
        "he_batch_prepare": [vp],
        "he_batch_run": [vp, i32, vp],
        "he_batch_autotune": [vp, vp, ctypes.POINTER(he_batch_tuning), i32, ctypes.POINTER(i32)],
        "he_batch_add_cpmul2": [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp],
        "he_batch_set_tuning": [vp, ctypes.POINTER(he_batch_tuning), i32],
        "he_batch_query": [vp, ctypes.POINTER(he_batch_info)],
        "he_batch_set_fused": [vp, i32, i32],
        "he_batch_status": [vp, vp],
        "he_batch_set_wait_limit": [vp, ctypes.c_int64],
        "he_batch_test_hold_job": [vp, i32, i32],
        "he_checks_enabled": [],
        "he_checks_last_error": [ctypes.c_char_p, i32],
        "he_checks_test_exclude": [vp, ctypes.c_int64],
        "he_server_create": [ctypes.POINTER(he_server_config), pp],
        "he_server_submit": [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(i64)],
        "he_server_poll": [vp, i64, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)],
        "he_server_cancel": [vp, i64, ctypes.POINTER(i32)],
        "he_server_wait_all": [vp, ctypes.c_double],
        "he_server_request_bytes": [vp, vp, i32, i32, i32, ctypes.POINTER(ctypes.c_double)],
        "he_server_stats": [vp, ctypes.POINTER(he_server_report)],
        "he_server_reset_stats": [vp],
        "he_server_destroy": [vp],
        "he_trace_enable": [vp, i32],
        "he_trace_read": [vp, ctypes.POINTER(he_trace_entry), i32, ctypes.POINTER(i32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    return lib


lib = _load()


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_cuda:
            raise ValueError("device tensor expected")
        if not t.is_contiguous():
            raise ValueError("contiguous tensor expected")
        return ctypes.c_void_p(t.data_ptr())
    return t


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def last_error(ctx=None) -> str:
    buf = ctypes.create_string_buffer(512)
    lib.he_last_error(ctx, buf, 512)
    return buf.value.decode()


def _check(rc, ctx=None):
    if rc != HE_OK:
        msg = last_error(ctx)
        if not msg and LIB_NAME == "libcryptotrain_checks.so":
            msg = he_checks_last_error()
        raise HEError(rc, msg)


def make_params(N, L=None, prime_bits=None, q=None, t=65537, base_log2=16, eta=21, max_ccmul_group=64, device=0,
                max_ccmul_scratch_bytes=0.0, max_table_cache_bytes=0.0):
    p = he_params()
    p.N = N
    if q:
        p.L = len(q)
        for i, v in enumerate(q):
            p.q[i] = v
    else:
        p.L = len(prime_bits)
        for i, b in enumerate(prime_bits):
            p.prime_bits[i] = b
    p.t, p.base_log2, p.eta, p.max_ccmul_group, p.device = t, base_log2, eta, max_ccmul_group, device
    p.max_ccmul_scratch_bytes = float(max_ccmul_scratch_bytes)
    p.max_table_cache_bytes = float(max_table_cache_bytes)
    return p


# ---------------------------------------------------------------- entry points
def he_setup(params: he_params):
    h = ctypes.c_void_p()
    _check(lib.he_setup(ctypes.byref(params), ctypes.byref(h)))
    return h


def he_ctx_destroy(ctx):
    _check(lib.he_ctx_destroy(ctx))


def he_ctx_query(ctx) -> he_ctx_info:
    info = he_ctx_info()
    _check(lib.he_ctx_query(ctx, ctypes.byref(info)), ctx)
    return info


def he_keygen(ctx, seed: int, with_relin: bool = True):
    h = ctypes.c_void_p()
    _check(lib.he_keygen(ctx, seed, int(with_relin), ctypes.byref(h), _stream()), ctx)
    return h


def he_keys_destroy(keys):
    _check(lib.he_keys_destroy(keys))


def he_keys_export(ctx, keys, which: int, dst: torch.Tensor):
    _check(lib.he_keys_export(ctx, keys, which, _ptr(dst), _stream()), ctx)


def he_encrypt(ctx, keys, pt: torch.Tensor, n: int, seed: int, ct: torch.Tensor):
    _check(lib.he_encrypt(ctx, keys, _ptr(pt), n, seed, _ptr(ct), _stream()), ctx)


def he_encrypt_many(ctx, keys, groups):
    """groups: up to 4 tuples (pt [n][N], n, seed, ct [n][2][L][N])."""
    k = len(groups)
    pts = (ctypes.c_void_p * k)(*[_ptr(g[0]) for g in groups])
    counts = (ctypes.c_int32 * k)(*[int(g[1]) for g in groups])
    seeds = (ctypes.c_uint64 * k)(*[int(g[2]) for g in groups])
    cts = (ctypes.c_void_p * k)(*[_ptr(g[3]) for g in groups])
    _check(lib.he_encrypt_many(ctx, keys, k, pts, counts, seeds, cts, _stream()), ctx)


def he_encrypt_symmetric(ctx, keys, pt, n: int, seed: int, c0):
    _check(lib.he_encrypt_symmetric(ctx, keys, _ptr(pt), n, seed, _ptr(c0), _stream()), ctx)


def he_expand_symmetric(ctx, seed: int, n: int, c0, ct):
    _check(lib.he_expand_symmetric(ctx, seed, n, _ptr(c0), _ptr(ct), _stream()), ctx)


def he_keys_import(ctx, sk, pk, rlk=None):
    h = ctypes.c_void_p()
    _check(lib.he_keys_import(ctx, _ptr(sk), _ptr(pk), _ptr(rlk), ctypes.byref(h), _stream()), ctx)
    return h


def he_ctx_fingerprint(ctx) -> int:
    v = ctypes.c_uint64()
    _check(lib.he_ctx_fingerprint(ctx, ctypes.byref(v)), ctx)
    return v.value


def he_decrypt(ctx, keys, ct: torch.Tensor, n: int, pt: torch.Tensor):
    _check(lib.he_decrypt(ctx, keys, _ptr(ct), n, _ptr(pt), _stream()), ctx)


def he_sample_masks(ctx, seed: int, n: int, out: torch.Tensor):
    _check(lib.he_sample_masks(ctx, seed, n, _ptr(out), _stream()), ctx)


def he_pt_sub(ctx, a, b, n: int, out):
    _check(lib.he_pt_sub(ctx, _ptr(a), _ptr(b), n, _ptr(out), _stream()), ctx)


def he_conv_plan(ctx, C, H, W, M, h, pad, encoding):
    s = he_conv_shape(C, H, W, M, h, pad)
    p = ctypes.c_void_p()
    _check(lib.he_conv_plan(ctx, ctypes.byref(s), encoding, ctypes.byref(p)), ctx)
    return p


def he_plan_search(N, C, H, W, M, h, pad, encoding) -> "he_plan_info":
    """Plan search without a context or a GPU (host only)."""
    s = he_conv_shape(C, H, W, M, h, pad)
    info = he_plan_info()
    _check(lib.he_plan_search(N, ctypes.byref(s), encoding, ctypes.byref(info)))
    return info


def he_ks_primes(params) -> list:
    """Small primes of the relinearisation key switch for these parameters
    (host only); [] when the key switch runs over the limbs."""
    arr = (ctypes.c_uint64 * 4)()
    n = ctypes.c_int32()
    _check(lib.he_ks_primes(ctypes.byref(params), arr, ctypes.byref(n)))
    return [int(arr[k]) for k in range(n.value)]


def he_plan_destroy(plan):
    _check(lib.he_plan_destroy(plan))


def he_plan_query(plan) -> he_plan_info:
    info = he_plan_info()
    _check(lib.he_plan_query(plan, ctypes.byref(info)))
    return info


def _dtype_code(t: torch.Tensor) -> int:
    return {torch.uint8: HE_DTYPE_U8, torch.int8: HE_DTYPE_I8, torch.int64: HE_DTYPE_I64}[t.dtype]


def he_encode_conventional(ctx, plan, role, tensor, batch, polys):
    _check(lib.he_encode_conventional(ctx, plan, role, _ptr(tensor), _dtype_code(tensor), batch, _ptr(polys),
                                      _stream()), ctx)


def he_encode_correlated(ctx, plan, role, tensor, batch, polys):
    _check(lib.he_encode_correlated(ctx, plan, role, _ptr(tensor), _dtype_code(tensor), batch, _ptr(polys),
                                    _stream()), ctx)


def he_cpmul_conv(ctx, plan, batch, ct_x, pt_w, ct_w, pt_x, ct_add, ct_out):
    _check(lib.he_cpmul_conv(ctx, plan, batch, _ptr(ct_x), _ptr(pt_w), _ptr(ct_w), _ptr(pt_x), _ptr(ct_add),
                             _ptr(ct_out), _stream()), ctx)


def he_cpmul_conv_noalloc(ctx, plan, batch, ct_x, pt_w, ct_w, pt_x, ct_add, ct_out):
    """he_cpmul_conv without any device allocation (fixed 32 MiB library scratch)."""
    _check(lib.he_cpmul_conv_noalloc(ctx, plan, batch, _ptr(ct_x), _ptr(pt_w), _ptr(ct_w), _ptr(pt_x),
                                     _ptr(ct_add), _ptr(ct_out), _stream()), ctx)


def he_ccmul_precompute(ctx, keys, ct_a, n_a, ct_b, n_b, pairs, group, ct_out):
    n = len(pairs)
    pa = (ctypes.c_int32 * max(n, 1))(*[p[0] for p in pairs])
    pb = (ctypes.c_int32 * max(n, 1))(*[p[1] for p in pairs])
    _check(lib.he_ccmul_precompute(ctx, keys, _ptr(ct_a), n_a, _ptr(ct_b), n_b, pa, pb, n, group, _ptr(ct_out),
                                   _stream()), ctx)


def he_ccmul_conv_precompute(ctx, keys, plan, batch, ct_rx, ct_rw, ct_out):
    _check(lib.he_ccmul_conv_precompute(ctx, keys, plan, batch, _ptr(ct_rx), _ptr(ct_rw), _ptr(ct_out), _stream()),
           ctx)


def he_ppmul_conv(ctx, plan, batch, pt_x, pt_w, out):
    _check(lib.he_ppmul_conv(ctx, plan, batch, _ptr(pt_x), _ptr(pt_w), _ptr(out), _stream()), ctx)


def he_decode(ctx, plan, batch, pt, sub, out):
    _check(lib.he_decode(ctx, plan, batch, _ptr(pt), _ptr(sub), _ptr(out), _stream()), ctx)


def he_encode_output(ctx, plan, batch, values, polys):
    _check(lib.he_encode_output(ctx, plan, batch, _ptr(values), _ptr(polys), _stream()), ctx)


def he_ct_add(ctx, a, b, n, out):
    _check(lib.he_ct_add(ctx, _ptr(a), _ptr(b), n, _ptr(out), _stream()), ctx)


def he_trace_enable(ctx, on: bool):
    _check(lib.he_trace_enable(ctx, int(on)), ctx)


def he_trace_read(ctx) -> dict:
    """{kernel family: (launches, total_ms, algorithmic bytes, modular products)}"""
    arr = (he_trace_entry * 64)()
    n = ctypes.c_int32()
    _check(lib.he_trace_read(ctx, arr, 64, ctypes.byref(n)), ctx)
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms, arr[i].bytes, arr[i].modmuls)
            for i in range(min(n.value, 64))}


def _bcheck(rc, b):
    if rc < 0:
        buf = ctypes.create_string_buffer(512)
        lib.he_batch_last_error(b, buf, 512)
        raise HEError(rc, buf.value.decode())
    return rc


def he_batch_create(device=0):
    h = ctypes.c_void_p()
    _check(lib.he_batch_create(device, ctypes.byref(h)))
    return h


def he_batch_destroy(b):
    _check(lib.he_batch_destroy(b))


def he_batch_add_cpmul(b, ctx, plan, n_images, ct_x, pt_w, ct_add, ct_out) -> int:
    return _bcheck(lib.he_batch_add_cpmul(b, ctx, plan, n_images, _ptr(ct_x), _ptr(pt_w), _ptr(ct_add),
                                          _ptr(ct_out)), b)


def he_batch_prepare(b):
    _bcheck(lib.he_batch_prepare(b), b)


def he_batch_run(b, mode):
    _bcheck(lib.he_batch_run(b, mode, _stream()), b)


def he_batch_set_tuning(b, tunings):
    """tunings: dicts with logN, regs_ctas_per_sm, grid_ctas_per_sm."""
    arr = (he_batch_tuning * len(tunings))()
    for i, t in enumerate(tunings):
        arr[i].logN, arr[i].regs_ctas_per_sm, arr[i].grid_ctas_per_sm = t["logN"], t["regs_ctas_per_sm"], t["grid_ctas_per_sm"]
    _bcheck(lib.he_batch_set_tuning(b, arr, len(tunings)), b)


def he_batch_autotune(b):
    arr = (he_batch_tuning * 8)()
    n = ctypes.c_int32()
    _bcheck(lib.he_batch_autotune(b, _stream(), arr, 8, ctypes.byref(n)), b)
    return [dict(logN=arr[i].logN, regs_ctas_per_sm=arr[i].regs_ctas_per_sm, grid_ctas_per_sm=arr[i].grid_ctas_per_sm,
                 ms=arr[i].ms, fwd_items=arr[i].fwd_items, mac_items=arr[i].mac_items) for i in range(min(n.value, 8))]


def he_batch_query(b) -> dict:
    info = he_batch_info()
    _bcheck(lib.he_batch_query(b, ctypes.byref(info)), b)
    return {f: getattr(info, f) for f, _ in he_batch_info._fields_}


def he_batch_set_fused(b, graph_fused, regs_ctas_per_sm=0):
    _bcheck(lib.he_batch_set_fused(b, int(graph_fused), regs_ctas_per_sm), b)


def he_batch_status(b):
    """Synchronise the current stream and raise HEError (HE_ERR_TIMEOUT) if a
    fused run gave up waiting; clears the status."""
    _bcheck(lib.he_batch_status(b, _stream()), b)


def he_batch_set_wait_limit(b, polls):
    _bcheck(lib.he_batch_set_wait_limit(b, int(polls)), b)


def he_batch_test_hold_job(b, job, hold):
    _bcheck(lib.he_batch_test_hold_job(b, job, int(hold)), b)


def he_checks_enabled() -> bool:
    return lib.he_checks_enabled() == 1


def he_checks_last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    lib.he_checks_last_error(buf, 512)
    return buf.value.decode()


def he_checks_test_exclude(t, nbytes):
    """Leave [t.data_ptr(), + nbytes) out of the checked ranges (None: clear)."""
    _check(lib.he_checks_test_exclude(_ptr(t) if t is not None else None, int(nbytes)))


def he_batch_last_error(b) -> str:
    buf = ctypes.create_string_buffer(512)
    lib.he_batch_last_error(b, buf, 512)
    return buf.value.decode()


def he_last_error(ctx=None) -> str:
    return last_error(ctx)


def he_batch_add_cpmul2(b, ctx, plan, n_images, ct_x, pt_w, ct_w, pt_x, ct_add, ct_out) -> int:
    return _bcheck(lib.he_batch_add_cpmul2(b, ctx, plan, n_images, _ptr(ct_x), _ptr(pt_w), _ptr(ct_w), _ptr(pt_x),
                                           _ptr(ct_add), _ptr(ct_out)), b)


def he_server_create(device=0, hbm_budget_bytes=150e9, max_group=64, max_inflight=4, n_streams=4, poll_us=20):
    cfg = he_server_config(device, float(hbm_budget_bytes), max_group, max_inflight, n_streams, poll_us)
    h = ctypes.c_void_p()
    _check(lib.he_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def he_server_submit(s, ctx, plan, n_images, ct_x, pt_w, ct_w, pt_x, ct_add, ct_out) -> int:
    rid = ctypes.c_int64()
    _check(lib.he_server_submit(s, ctx, plan, n_images, _ptr(ct_x), _ptr(pt_w), _ptr(ct_w), _ptr(pt_x), _ptr(ct_add),
                                _ptr(ct_out), ctypes.byref(rid)))
    return rid.value


def he_server_poll(s, rid):
    done = ctypes.c_int32()
    lat = ctypes.c_double()
    _check(lib.he_server_poll(s, rid, ctypes.byref(done), ctypes.byref(lat)))
    return bool(done.value), lat.value


def he_server_cancel(s, rid) -> bool:
    c = ctypes.c_int32()
    _check(lib.he_server_cancel(s, rid, ctypes.byref(c)))
    return bool(c.value)


def he_server_wait_all(s, timeout_s=600.0):
    _check(lib.he_server_wait_all(s, timeout_s))


def he_server_stats(s) -> dict:
    st = he_server_report()
    _check(lib.he_server_stats(s, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in he_server_report._fields_}


def he_server_reset_stats(s):
    _check(lib.he_server_reset_stats(s))


def he_server_destroy(s):
    _check(lib.he_server_destroy(s))


def he_server_request_bytes(ctx, plan, n_images, has_x=True, has_w=True) -> float:
    b = ctypes.c_double()
    _check(lib.he_server_request_bytes(ctx, plan, n_images, int(has_x), int(has_w), ctypes.byref(b)), ctx)
    return b.value
