"""The pins catch plausible mistakes in the oracle.

Each case below plants one mistake in a copy of the oracle. In the C core
(he_oracle.c) the mistakes include a wrong root of unity, a dropped rounding
term, a dropped or swapped product term, an off-by-one digit, a wrong sign,
a missing centred lift, a transposed operand, a wrong rotation, skipped
prime candidates, truncating instead of floor division, an uncentred lift
before the tensor product and a too small auxiliary basis. In the Python packing and protocol modules they include a
kernel not reversed, a wrong channel order, a missing output offset, a wrong
index sign, ignored padding, a dropped wrap check, an uncentred or
misplaced decode, wrong mask signs, and a dropped error or wrong stream
index in the seed-compressed encryption.

The broken copy is built apart and the oracle's pin modules run against it
in a subprocess: the C library is loaded through the oracle loader's
override, and the Python package comes from a copied tree. Every case must
make some pin fail, and a control build of the unmodified sources must pass
them all. Nothing here touches the committed oracle or its library."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "he_oracle.c")
PINS = [os.path.join(ROOT, "tests", "test_oracle_he.py"), os.path.join(ROOT, "tests", "test_oracle_ring.py")]

MUTANTS = {
    "ntt_twist_by_omega": [("pw = mulmod(pw, psi, p); }", "pw = mulmod(pw, w, p); }")],
    "ntt_no_untwist": [("c[i] = mulmod(fa[i], pw, p); pw = mulmod(pw, psiinv, p);",
                        "c[i] = mulmod(fa[i], ninv, p); pw = mulmod(pw, psiinv, p);")],
    "primes_skip_candidates": [("for (; p > step; p -= step) {", "for (; p > step; p -= 2 * step) {")],
    "chacha_rotation": [("s[b] = rotl32(s[b], 12);", "s[b] = rotl32(s[b], 11);")],
    "ternary_mapping": [("(((u128)w[k] * 3) >> 64) - 1", "(w[k] % 3) - 1")],
    "cbd_sign": [("out[k] = a - b;", "out[k] = b - a;")],
    "pk_sign": [("pk[o] = submod(0, addmod(as[o], e[o], P->q[i]), P->q[i]);",
                 "pk[o] = addmod(as[o], e[o], P->q[i]);")],
    "rlk_power_off_by_one": [("powmod(2, (uint64_t)P->base_log2 * (uint64_t)j, P->q[i])",
                              "powmod(2, (uint64_t)P->base_log2 * (uint64_t)(j + 1), P->q[i])")],
    "encrypt_drops_e1": [("uint64_t v = addmod(bu[o], smod(e1[k], qi), qi);", "uint64_t v = bu[o];")],
    "encrypt_e1_e2_swapped": [("smod(e1[k], qi)", "smod(E2PLACE[k], qi)"),
                              ("smod(e2[k], qi)", "smod(e1[k], qi)"), ("E2PLACE", "e2")],
    "delta_plus_one": [("uint64_t qi = P->q[i], di = big_mod_u64(&c.delta, qi);",
                        "uint64_t qi = P->q[i], di = (big_mod_u64(&c.delta, qi) + 1) % qi;")],
    "decrypt_floor": [("big_mul_u64(&num, &X, P->t);\n        big_add(&num, &num, &c.qhalf);\n",
                       "big_mul_u64(&num, &X, P->t);\n")],
    "cpmul_no_centred_lift": [("int64_t sv = v <= (P->t - 1) / 2 ? (int64_t)v : (int64_t)v - (int64_t)P->t;",
                               "int64_t sv = (int64_t)v;")],
    "ccmul_floor": [("big_mul_u64(&num, &D, P->t);\n                big_add(&num, &num, &c.qhalf);\n",
                     "big_mul_u64(&num, &D, P->t);\n")],
    "tensor_drops_a1b0": [("orc_polymul(la1 + off, lb0 + off, tmp, N, A[j]);\n"
                           "                for (int x = 0; x < N; x++) d[1][off + x] = addmod(d[1][off + x], tmp[x], A[j]);\n",
                           "")],
    "digit_shift_off_by_one": [("int bi = j * P->base_log2 + b;", "int bi = (j + 1) * P->base_log2 + b;")],
    "relin_components_swapped": [("rlk + ((size_t)j * 2 + comp) * LN", "rlk + ((size_t)j * 2 + (1 - comp)) * LN")],
    "ppmul_transposed_index": [("tb[x] = b[(size_t)term_b[k] * N + x] % P->t;",
                                "tb[x] = b[(size_t)term_a[k] * N + x] % P->t;")],
    "floordiv_truncates": [("if (!rz) { big one; big_from_u64(&one, 1); big_sub(&q, &q, &one); }", "(void)rz;")],
    "ccmul_lift_not_centred": [("crt_reconstruct_centred(&c->Q, r, &X);\n        for (int j = 0; j < nA; j++) res",
                                "crt_reconstruct(&c->Q, r, &X);\n        for (int j = 0; j < nA; j++) res")],
    "ccmul_aux_basis_too_small": [("int k = need_bits / 60 + 2;", "int k = need_bits / 60 - 2;")],
}


# mistakes planted in the oracle's Python modules (file, [(old, new), ...])
PY_MUTANTS = {
    "corr_kernel_not_reversed": ("packing.py", [
        ("(p.Cn - 1 - cl) * p.S + (p.h - 1 - k) * p.O + (p.h - 1 - l), c, k, l)",
         "(p.Cn - 1 - cl) * p.S + k * p.O + l, c, k, l)")]),
    "corr_channel_order": ("packing.py", [
        ("(p.Cn - 1 - cl) * p.S + (p.h - 1 - k) * p.O", "cl * p.S + (p.h - 1 - k) * p.O")]),
    "corr_output_offset": ("packing.py", [("u = a - p.pad - r0 + p.h - 1", "u = a - p.pad - r0")]),
    "conv_kernel_column_sign": ("packing.py", [
        ("p.Ooff - cl * p.Hn * p.Wn - k * p.Wn - l, c, k, l)", "p.Ooff - cl * p.Hn * p.Wn - k * p.Wn + l, c, k, l)")]),
    "conv_input_ignores_padding": ("packing.py", [
        ("r, s = r0 + i - p.pad, s0 + j - p.pad", "r, s = r0 + i, s0 + j")]),
    "corr_no_wrap_check": ("packing.py", [("if not (D < N or D - N < (c - 1) * S + rlo):", "if False:")]),
    "decode_no_centring": ("packing.py", [
        ("out[m, a, b] = v - t_mod if v > (t_mod - 1) // 2 else v", "out[m, a, b] = v")]),
    "decode_output_packing_offset": ("packing.py", [
        ("v = int(polys[m // p.Mn, t, k + (m % p.Mn) * p.Sout])", "v = int(polys[m // p.Mn, t, k + (m // p.Mn) * p.Sout])")]),
    "protocol_mask_sign": ("protocol.py", [("wm = (wp + (tt - r_w)) % tt", "wm = (wp + r_w) % tt")]),
    "protocol_input_mask_sign": ("protocol.py", [("xm = (xp + (tt - r_x)) % tt", "xm = (xp + r_x) % tt")]),
    "symmetric_drops_e": ("he.py", [("(-(int(x) + int(ee)) + d * mm) % q", "(-int(x) + d * mm) % q")]),
    "symmetric_wrong_stream": ("he.py", [("a = sample_uniform(seed, TAG_SYM_A, first + k, i, q, P.N)",
                                          "a = sample_uniform(seed, TAG_SYM_A, k, i, q, P.N)")]),
}
PY_PINS = {"packing.py": "tests/test_oracle_packing.py", "protocol.py": "tests/test_oracle_packing.py",
           "he.py": "tests/test_oracle_he.py"}


def build_py_variant(tmp_path, name, fname, edits):
    """A tree whose oracle package is a copy with one module edited; the
    tests and the input generators are links to the repository's."""
    d = tmp_path / name
    d.mkdir()
    shutil.copytree(os.path.join(ROOT, "oracle"), d / "oracle",
                    ignore=shutil.ignore_patterns("__pycache__", "*.tmp"))
    path = d / "oracle" / fname
    src = path.read_text()
    for old, new in edits:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    path.write_text(src)
    for link in ("tests", "paper_2409_16675_gb300"):
        os.symlink(os.path.join(ROOT, link), d / link)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d / "pytest.ini")
    return str(d)


def run_py_pins(tree, pins="tests/test_oracle_packing.py"):
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu",
                        "--basetemp", os.path.join(tree, "pt"), pins],
                       cwd=tree, capture_output=True, text=True, timeout=300)
    return r.returncode, r.stdout[-2000:]


def build_variant(tmp_path, name, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    d = tmp_path / name
    d.mkdir()
    (d / "he_oracle.c").write_text(src)
    lib = d / "liboracle.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", str(lib), str(d / "he_oracle.c")],
                   check=True, capture_output=True)
    return str(lib)


def run_pins(lib):
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu",
                        "--basetemp", os.path.join(os.path.dirname(lib), "pt")] + PINS,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def gcc():
    if not shutil.which("gcc"):
        pytest.skip("needs gcc")


def test_control_build_passes_every_pin(tmp_path, gcc):
    rc, out = run_pins(build_variant(tmp_path, "control", []))
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(tmp_path, gcc, name):
    rc, out = run_pins(build_variant(tmp_path, name, MUTANTS[name]))
    assert rc == 1, "no pin caught mutant %s:\n%s" % (name, out)


def test_python_control_tree_passes_the_packing_pins(tmp_path, gcc):
    rc, out = run_py_pins(build_py_variant(tmp_path, "py_control", "packing.py", []))
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_planted_packing_or_protocol_mistake_fails_a_pin(tmp_path, gcc, name):
    fname, edits = PY_MUTANTS[name]
    rc, out = run_py_pins(build_py_variant(tmp_path, name, fname, edits), PY_PINS[fname])
    assert rc == 1, "no pin caught mutant %s:\n%s" % (name, out)
