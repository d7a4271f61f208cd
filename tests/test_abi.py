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


def test_binding_structs_match_the_header_layout(tmp_path):
    """sizeof and every field offset of the header's public structs, printed
    by a C program compiled against include/cryptotrain.h, equal those of the
    ctypes mirrors in the binding."""
    import shutil
    import subprocess
    from paper_2409_16675_gb300 import native
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda_inc = "/usr/local/cuda/include"
    if not cc or not os.path.isdir(cuda_inc):
        import pytest
        pytest.skip("needs gcc and the CUDA headers")
    structs = [native.he_params, native.he_ctx_info, native.he_conv_shape, native.he_plan_info,
               native.he_batch_tuning, native.he_server_config, native.he_server_report, native.he_trace_entry]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cryptotrain.h"', "int main(void) {"]
    for S in structs:
        n = S.__name__
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (n, n))
        for f in S._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (n, f[0], n, f[0]))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, str(src), "-o", str(exe), "-I", os.path.join(ROOT, "include"), "-I", cuda_inc], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for S in structs:
        n = S.__name__
        assert int(got[n + " sizeof"]) == ctypes.sizeof(S), n
        for f in S._fields_:
            assert int(got["%s %s" % (n, f[0])]) == getattr(S, f[0]).offset, (n, f[0])
