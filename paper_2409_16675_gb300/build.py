"""Build the in-tree CUDA library libcryptotrain.so for sm_103a (GB300).

Every translation unit under csrc/ is compiled in parallel with nvcc (one
-gencode, sm_103a only) and linked into one shared library with the CUDA
runtime linked statically, so the library only needs the driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libcryptotrain.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["params.cpp", "plan.cpp", "ntt.cu", "fused.cu", "exact.cu", "keyswitch.cu", "capi.cu", "batch.cu", "server.cu",
           "noalloc.cu"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    cmd = [nvcc(), "-c", path, "-o", obj, "-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-lineinfo",
           "-I", os.path.join(HERE, "..", "include")] + ARCH
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    if verbose and src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(HERE, "..", "include", "cryptotrain.h"))
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(f) for f in srcs + hdrs)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


# ---------------------------------------------------------------- bounds-checked debug build
# libcryptotrain_checks.so: the same sources compiled with -DHE_CHECKS (every
# kernel access checked against the registered device ranges, violations
# recorded instead of trapping) plus checks.cpp, and every entry point of
# include/cryptotrain.h wrapped: the library's own definitions are renamed
# he_X -> he_X_core by a forced include, and generated wrappers he_X register
# the allocations holding the call's device pointers, run he_X_core, then
# return HE_ERR_INVALID_ARG if any kernel recorded a violation.
LIB_CHECKS = os.path.join(HERE, "libcryptotrain_checks.so")
BUILD_CHECKS = os.path.join(HERE, "_build_checks")
HEADER = os.path.join(HERE, "..", "include", "cryptotrain.h")
# entry points taking host arrays of device pointers: parameter -> element count
_POINTER_ARRAYS = {"he_encrypt_many": {"pts": "n_groups", "cts": "n_groups"}}


def _entry_points():
    """(name, [(param text, param name)]) of every int he_* declaration, except
    the checks build's own calls."""
    import re
    with open(HEADER) as f:
        s = f.read()
    s = re.sub(r"/\*.*?\*/", "", s, flags=re.S)
    s = re.sub(r"//[^\n]*", "", s)
    out = []
    for name, params in re.findall(r"\bint\s+(he_\w+)\s*\(([^;{]*?)\)\s*;", s):
        if name.startswith("he_checks_"):
            continue
        ps = [" ".join(p.split()) for p in params.split(",")]
        if ps == ["void"]:
            ps = []
        out.append((name, [(p, re.findall(r"\w+", p)[-1]) for p in ps]))
    return out


def _generate_checks_sources():
    os.makedirs(BUILD_CHECKS, exist_ok=True)
    eps = _entry_points()
    rename = "".join("#define %s %s_core\n" % (n, n) for n, _ in eps)
    lines = ['// generated by build.py: checked wrappers of the entry points (bounds-checked build)',
             '#include <cuda_runtime.h>', '#include "cryptotrain.h"',
             'void *he_checks_call_begin();', 'void he_checks_call_arg(void *cc, const void *p);',
             'void he_checks_call_ready(void *cc);', 'int he_checks_call_end(void *cc, int rc);', 'extern "C" {']
    for name, params in eps:
        decl = ", ".join(p for p, _ in params) or "void"
        lines.append("int %s_core(%s);" % (name, decl))
        lines.append("int %s(%s) {" % (name, decl))
        lines.append("    void *cc = he_checks_call_begin();")
        arrays = _POINTER_ARRAYS.get(name, {})
        for p, pn in params:
            if pn in arrays:
                lines.append("    for (int i = 0; %s && i < %s; i++) he_checks_call_arg(cc, (const void *)%s[i]);"
                             % (pn, arrays[pn], pn))
            elif "*" in p:
                lines.append("    he_checks_call_arg(cc, (const void *)%s);" % pn)
        lines.append("    he_checks_call_ready(cc);")
        lines.append("    return he_checks_call_end(cc, %s_core(%s));" % (name, ", ".join(pn for _, pn in params)))
        lines.append("}")
    lines.append('}  // extern "C"')
    rp, ap = os.path.join(BUILD_CHECKS, "rename.h"), os.path.join(BUILD_CHECKS, "checks_api.cu")
    for path, text in ((rp, rename), (ap, "\n".join(lines) + "\n")):
        old = open(path).read() if os.path.exists(path) else None
        if old != text:
            with open(path, "w") as f:
                f.write(text)
    return rp, ap


def _compile_checks(src: str, rename: str) -> str:
    name = os.path.splitext(os.path.basename(src))[0]
    obj = os.path.join(BUILD_CHECKS, name + ".o")
    cmd = [nvcc(), "-c", src, "-o", obj, "-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-lineinfo", "-DHE_CHECKS",
           "-I", os.path.join(HERE, "..", "include"), "-I", CSRC] + ARCH
    if os.path.basename(src) != "checks_api.cu":
        cmd += ["-include", rename]
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s (checks build):\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj


def build_checks(force: bool = False) -> str:
    rename, api = _generate_checks_sources()
    srcs = [os.path.join(CSRC, s) for s in SOURCES + ["checks.cpp"]] + [api]
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))] + [HEADER, rename]
    if not force and os.path.exists(LIB_CHECKS):
        if os.path.getmtime(LIB_CHECKS) >= max(os.path.getmtime(f) for f in srcs + hdrs):
            return LIB_CHECKS
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile_checks(s, rename), srcs))
    tmp = LIB_CHECKS + ".%d.tmp" % os.getpid()
    r = subprocess.run([nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"], capture_output=True,
                       text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed (checks build):\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB_CHECKS)
    return LIB_CHECKS


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
    if "--checks" in sys.argv:
        print(build_checks(force="--force" in sys.argv))
