"""Build and load the oracle's C core with ctypes (test infrastructure)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "he_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# A prebuilt oracle library to load instead of liboracle.so: the mutation
# test (tests/test_oracle_mutants.py) points it at deliberately broken builds
# of he_oracle.c to show that the pins fail on them.
_OVERRIDE = os.environ.get("ORACLE_LIB_OVERRIDE")
_lib = None


def build(force: bool = False) -> str:
    """Compile he_oracle.c into liboracle.so with gcc (portable C11, no
    architecture flags, so the same source builds on x86-64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("L", ctypes.c_int32), ("q", ctypes.c_uint64 * 16),
                ("t", ctypes.c_uint64), ("base_log2", ctypes.c_int32), ("eta", ctypes.c_int32)]


def lib():
    global _lib
    if _lib is None:
        if _OVERRIDE:
            _lib = ctypes.CDLL(_OVERRIDE)
        else:
            build()
            _lib = ctypes.CDLL(_LIB)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        P = ctypes.POINTER(OrcParams)
        sig = {
            "orc_is_prime": (ctypes.c_int, [ctypes.c_uint64]),
            "orc_gen_primes": (ctypes.c_int, [ctypes.c_int, i32p, ctypes.c_int, u64p, ctypes.c_int, u64p]),
            "orc_chacha20_block": (None, [u32p, ctypes.c_uint32, u32p, u32p]),
            "orc_stream_words": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint64, ctypes.c_uint64, u64p]),
            "orc_sample_uniform": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_uint64, ctypes.c_int, u64p]),
            "orc_sample_ternary": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, i64p]),
            "orc_sample_cbd": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                      ctypes.c_int, i64p]),
            "orc_sample_uniform_t": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                            ctypes.c_int, u64p]),
            "orc_polymul": (None, [u64p, u64p, u64p, ctypes.c_int, ctypes.c_uint64]),
            "orc_num_digits": (ctypes.c_int, [P]),
            "orc_keygen": (ctypes.c_int, [P, ctypes.c_uint64, i64p, u64p, u64p]),
            "orc_encrypt": (ctypes.c_int, [P, u64p, u64p, ctypes.c_uint64, ctypes.c_uint32, u64p]),
            "orc_decrypt": (ctypes.c_int, [P, i64p, u64p, u64p]),
            "orc_noise_bits": (ctypes.c_int, [P, i64p, u64p, u64p]),
            "orc_cpmul_terms": (ctypes.c_int, [P, u64p, u64p, i32p, i32p, i32p, ctypes.c_int, u64p, u64p]),
            "orc_ccmul": (ctypes.c_int, [P, u64p, u64p, u64p, i32p, i32p, ctypes.c_int, ctypes.c_int, u64p]),
            "orc_ppmul_terms": (ctypes.c_int, [P, u64p, u64p, i32p, i32p, i32p, ctypes.c_int, u64p]),
            "orc_round_scalar": (ctypes.c_int, [P, u32p, ctypes.c_int, u64p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
