"""The C ABI library builds, loads and exports every entry point that
include/cryptotrain.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:int|const char \*|void)\s+(he_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("he_setup", "he_keygen", "he_encrypt", "he_decrypt", "he_encode_conventional",
                     "he_encode_correlated", "he_cpmul_conv", "he_ccmul_precompute", "he_ppmul_conv", "he_decode"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2409_16675_gb300", "libcryptotrain.so"))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_header():
    from paper_2409_16675_gb300 import native
    for n in declared_functions():
        if n == "he_last_error":
            continue
        assert hasattr(native, n), n


def test_setup_rejects_bad_params_without_touching_a_gpu():
    # argument validation happens before any CUDA call: N = 3000 is not a power of two
    from paper_2409_16675_gb300 import native
    h = ctypes.c_void_p()
    rc = native.lib.he_setup(None, ctypes.byref(h))
    assert rc == -1
