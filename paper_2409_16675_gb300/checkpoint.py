"""Checkpoint / resume of a serving process's resident state: keys in
coefficient form and named device tensors (the precomputed [r^x r^w], encoded
weights, ...) as raw uint64 / int64 arrays in one NumPy archive, with the
context's parameter fingerprint.  Resuming checks the fingerprint against the
new context, imports the keys (their NTT forms are recomputed on the device)
and puts the tensors back on the device.  Only argument marshalling here:
every device step is a library call.
"""
from __future__ import annotations

import numpy as np
import torch

from . import native as nv


def save(path: str, ctx, keys, tensors: dict | None = None) -> None:
    """ctx: layer.Context, keys: layer.Keys; tensors: name -> device tensor."""
    sk = keys.export(nv.HE_KEY_SK)
    pk = keys.export(nv.HE_KEY_PK)
    arrays = {"fingerprint": np.array([nv.he_ctx_fingerprint(ctx.h)], dtype=np.uint64),
              "sk": sk.cpu().numpy(), "pk": pk.view(torch.int64).cpu().numpy().view(np.uint64)}
    try:
        rlk = keys.export(nv.HE_KEY_RLK)
        arrays["rlk"] = rlk.view(torch.int64).cpu().numpy().view(np.uint64)
    except nv.HEError:
        pass  # keys without relinearisation
    for name, t in (tensors or {}).items():
        if name in arrays or name.startswith("dtype:"):
            raise ValueError("reserved name: " + name)
        arrays[name] = t.view(torch.int64).cpu().numpy()
        arrays["dtype:" + name] = np.array([str(t.dtype)])
    np.savez(path, **arrays)


def load(path: str, ctx):
    """-> (keys handle wrapper, {name: device tensor}); raises ValueError when
    the checkpoint was written for a context with other parameters."""
    from .layer import Keys
    z = np.load(path if path.endswith(".npz") else path + ".npz")
    if int(z["fingerprint"][0]) != nv.he_ctx_fingerprint(ctx.h):
        raise ValueError("checkpoint written for a context with other parameters")
    dev = ctx.device
    sk = torch.from_numpy(z["sk"]).to(dev)
    pk = torch.from_numpy(z["pk"].view(np.int64)).to(dev).view(torch.uint64)
    rlk = torch.from_numpy(z["rlk"].view(np.int64)).to(dev).view(torch.uint64) if "rlk" in z else None
    keys = Keys.__new__(Keys)
    keys.ctx = ctx
    keys.h = nv.he_keys_import(ctx.h, sk, pk, rlk)
    tensors = {}
    for name in z.files:
        if name in ("fingerprint", "sk", "pk", "rlk") or name.startswith("dtype:"):
            continue
        dt = getattr(torch, str(z["dtype:" + name][0]).split(".")[-1])
        tensors[name] = torch.from_numpy(z[name]).to(dev).view(dt)
    return keys, tensors
