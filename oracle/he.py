"""BFV-style RLWE operations of the oracle (test infrastructure).

Follows Section 2 (HE: eps(p, pk), sigma(c, sk); Notations: A_{N,p} =
Z_p[x]/(x^N+1); Motivation / Fig. 3: CPMul (c0 p, c1 p), CCMul tensor product
(c0 c0', c0 c1' + c1 c0', c1 c1') and relinearisation) and Section 3.2 (PPMul,
CCAdd).  The arithmetic lives in he_oracle.c; this module only marshals numpy
arrays.

Layouts: ciphertext uint64 [2][L][N] (coefficient form, limb i in [0, q_i)),
plaintext uint64 [N] in [0, t), secret key int64 [N] in {-1, 0, 1}, public key
uint64 [2][L][N] = (b, a), relinearisation key uint64 [ell][2][L][N].

Parameter readings (the paper states none): Delta = floor(q / t); ternary
secret; centred-binomial errors with eta = 21; relinearisation digits of
base_log2 bits, ell = ceil(bitlen(q) / base_log2); pt operands centre-lifted
before CPMul.

Parity unpinned for the random objects (keys, encryption randomness, masks,
the symmetric-encryption a and e): the paper fixes no generator, so their
exact bits follow this project's stream convention (ChaCha20, pinned to RFC
8439; words to samples as stated at each sampler).  Given that convention,
the tests pin every sampler to its written function of the stream words, and
the keys and ciphertexts to their definitions evaluated by schoolbook
products on those samples.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _clib

TAG_SK, TAG_PK_A, TAG_PK_E, TAG_ENC_U, TAG_ENC_E1, TAG_ENC_E2, TAG_RLK_A, TAG_RLK_E, TAG_MASK = range(1, 10)
TAG_SYM_A, TAG_SYM_E = 10, 11


def _u64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _i64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _i32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _u32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def gen_primes(N: int, bits, exclude=()) -> list:
    """Largest primes below 2^b, = 1 mod 2N, one per entry of ``bits``."""
    L = len(bits)
    b = np.asarray(bits, dtype=np.int32)
    ex = np.asarray(list(exclude) or [0], dtype=np.uint64)
    out = np.zeros(L, dtype=np.uint64)
    rc = _clib.lib().orc_gen_primes(N, _i32(b), L, _u64(ex), len(exclude), _u64(out))
    if rc:
        raise ValueError("no such primes")
    return [int(v) for v in out]


def is_prime(n: int) -> bool:
    return bool(_clib.lib().orc_is_prime(n))


@dataclass
class Params:
    N: int
    q: list
    t: int
    base_log2: int = 16
    eta: int = 21

    @property
    def L(self):
        return len(self.q)

    @property
    def Q(self):
        r = 1
        for p in self.q:
            r *= p
        return r

    @property
    def delta(self):
        return self.Q // self.t

    @classmethod
    def from_spec(cls, spec) -> "Params":
        return cls(spec.N, gen_primes(spec.N, spec.prime_bits), spec.t, spec.base_log2, spec.eta)

    def c(self) -> _clib.OrcParams:
        p = _clib.OrcParams()
        p.N, p.L, p.t, p.base_log2, p.eta = self.N, self.L, self.t, self.base_log2, self.eta
        for i, v in enumerate(self.q):
            p.q[i] = v
        return p

    @property
    def ell(self) -> int:
        return _clib.lib().orc_num_digits(ctypes.byref(self.c()))


# ---------------------------------------------------------------- randomness
def chacha20_block(key_words, counter, nonce_words):
    k = np.asarray(key_words, dtype=np.uint32)
    n = np.asarray(nonce_words, dtype=np.uint32)
    out = np.zeros(16, dtype=np.uint32)
    _clib.lib().orc_chacha20_block(_u32(k), counter, _u32(n), _u32(out))
    return out


def stream_words(seed, tag, idx, limb, first, n):
    out = np.zeros(n, dtype=np.uint64)
    _clib.lib().orc_stream_words(seed, tag, idx, limb, first, n, _u64(out))
    return out


def sample_ternary(seed, tag, idx, N):
    out = np.zeros(N, dtype=np.int64)
    _clib.lib().orc_sample_ternary(seed, tag, idx, N, _i64(out))
    return out


def sample_cbd(seed, tag, idx, eta, N):
    out = np.zeros(N, dtype=np.int64)
    _clib.lib().orc_sample_cbd(seed, tag, idx, eta, N, _i64(out))
    return out


def sample_uniform(seed, tag, idx, limb, q, N):
    out = np.zeros(N, dtype=np.uint64)
    _clib.lib().orc_sample_uniform(seed, tag, idx, limb, q, N, _u64(out))
    return out


def sample_masks(P: Params, seed: int, n: int, first: int = 0) -> np.ndarray:
    """n uniform polynomials mod t; row k uses stream (seed, MASK, first + k)."""
    out = np.zeros((n, P.N), dtype=np.uint64)
    for k in range(n):
        _clib.lib().orc_sample_uniform_t(seed, TAG_MASK, first + k, P.t, P.N, _u64(out[k]))
    return out


# ---------------------------------------------------------------- ring
def polymul(a, b, q):
    """Negacyclic product in Z_q[x]/(x^N+1), q = 1 mod 2N prime."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    c = np.zeros_like(a)
    _clib.lib().orc_polymul(_u64(a), _u64(b), _u64(c), a.shape[0], q)
    return c


# ---------------------------------------------------------------- keys
@dataclass
class Keys:
    sk: np.ndarray
    pk: np.ndarray
    rlk: np.ndarray | None


def keygen(P: Params, seed: int, with_relin: bool = True) -> Keys:
    sk = np.zeros(P.N, dtype=np.int64)
    pk = np.zeros((2, P.L, P.N), dtype=np.uint64)
    rlk = np.zeros((P.ell, 2, P.L, P.N), dtype=np.uint64) if with_relin else None
    pc = P.c()
    _clib.lib().orc_keygen(ctypes.byref(pc), seed, _i64(sk), _u64(pk),
                           _u64(rlk) if rlk is not None else None)
    return Keys(sk, pk, rlk)


def encrypt(P: Params, keys: Keys, m, seed: int, first: int = 0) -> np.ndarray:
    """m: [n][N] in [0, t) -> [n][2][L][N]; row k is encrypted with object
    index first + k (its position in a larger flattened batch)."""
    m = np.ascontiguousarray(np.atleast_2d(m), dtype=np.uint64)
    ct = np.zeros((m.shape[0], 2, P.L, P.N), dtype=np.uint64)
    pc = P.c()
    for k in range(m.shape[0]):
        _clib.lib().orc_encrypt(ctypes.byref(pc), _u64(keys.pk), _u64(m[k]), seed, first + k, _u64(ct[k]))
    return ct


def encrypt_symmetric(P: Params, keys: Keys, m, seed: int, first: int = 0) -> np.ndarray:
    """Seed-compressed secret-key encryption: c0_k = -(a_k s + e_k) + Delta m_k
    with a_k uniform mod q from streams (seed, SYM_A, first + k, limb) and e_k
    CBD from (seed, SYM_E, first + k); returns c0 [n][L][N] (the ciphertext
    is (c0_k, a_k), see expand_symmetric).  Written from the definitions with
    the oracle's samplers and polymul, limb by limb."""
    m = np.atleast_2d(np.asarray(m, dtype=np.uint64))
    Q = 1
    for q in P.q:
        Q *= q
    delta = Q // P.t
    out = np.zeros((m.shape[0], P.L, P.N), dtype=np.uint64)
    for k in range(m.shape[0]):
        e = sample_cbd(seed, TAG_SYM_E, first + k, P.eta, P.N).astype(object)
        mk = [int(v) % P.t for v in m[k]]
        for i, q in enumerate(P.q):
            a = sample_uniform(seed, TAG_SYM_A, first + k, i, q, P.N)
            s_i = np.array([int(v) % q for v in keys.sk], dtype=np.uint64)
            a_s = polymul(a, s_i, q)
            d = delta % q
            out[k, i] = [(-(int(x) + int(ee)) + d * mm) % q for x, ee, mm in zip(a_s, e, mk)]
    return out


def expand_symmetric(P: Params, seed: int, c0, first: int = 0) -> np.ndarray:
    """(seed, c0 [n][L][N]) -> ct [n][2][L][N] with ct_k = (c0_k, a_k)."""
    c0 = np.asarray(c0, dtype=np.uint64).reshape(-1, P.L, P.N)
    ct = np.zeros((c0.shape[0], 2, P.L, P.N), dtype=np.uint64)
    for k in range(c0.shape[0]):
        ct[k, 0] = c0[k]
        for i, q in enumerate(P.q):
            ct[k, 1, i] = sample_uniform(seed, TAG_SYM_A, first + k, i, q, P.N)
    return ct


def decrypt(P: Params, keys: Keys, ct) -> np.ndarray:
    ct = np.ascontiguousarray(ct, dtype=np.uint64).reshape(-1, 2, P.L, P.N)
    out = np.zeros((ct.shape[0], P.N), dtype=np.uint64)
    pc = P.c()
    for k in range(ct.shape[0]):
        _clib.lib().orc_decrypt(ctypes.byref(pc), _i64(keys.sk), _u64(ct[k]), _u64(out[k]))
    return out


def noise_bits(P: Params, keys: Keys, ct, m) -> int:
    """bit length of the largest |[c0 + c1 s]_q - Delta m| over all coefficients."""
    ct = np.ascontiguousarray(ct, dtype=np.uint64).reshape(2, P.L, P.N)
    m = np.ascontiguousarray(m, dtype=np.uint64)
    return _clib.lib().orc_noise_bits(ctypes.byref(P.c()), _i64(keys.sk), _u64(ct), _u64(m))


# ---------------------------------------------------------------- products
def _csr(terms_per_out):
    ptr = [0]
    a, b = [], []
    for terms in terms_per_out:
        for (i, j) in terms:
            a.append(i)
            b.append(j)
        ptr.append(len(a))
    return (np.asarray(ptr, dtype=np.int32), np.asarray(a or [0], dtype=np.int32),
            np.asarray(b or [0], dtype=np.int32))


def cpmul_terms(P: Params, ct, pt, terms_per_out, add=None) -> np.ndarray:
    """out_o = sum_{(g, p) in terms_o} ct[g] * lift(pt[p]) (+ add_o): CPMul and CCAdd."""
    ct = np.ascontiguousarray(ct, dtype=np.uint64)
    pt = np.ascontiguousarray(pt, dtype=np.uint64)
    n_out = len(terms_per_out)
    ptr, ta, tb = _csr(terms_per_out)
    out = np.zeros((n_out, 2, P.L, P.N), dtype=np.uint64)
    addp = None
    if add is not None:
        add = np.ascontiguousarray(add, dtype=np.uint64)
        addp = _u64(add)
    _clib.lib().orc_cpmul_terms(ctypes.byref(P.c()), _u64(ct), _u64(pt), _i32(ptr), _i32(ta), _i32(tb),
                                n_out, addp, _u64(out))
    return out


def ccmul(P: Params, keys: Keys, ct_a, ct_b, pairs, group: int = 1) -> np.ndarray:
    """CCMul with exact rounding and relinearisation; consecutive groups of
    ``group`` pairs are summed before rounding."""
    ct_a = np.ascontiguousarray(ct_a, dtype=np.uint64)
    ct_b = np.ascontiguousarray(ct_b, dtype=np.uint64)
    pa = np.asarray([p[0] for p in pairs], dtype=np.int32)
    pb = np.asarray([p[1] for p in pairs], dtype=np.int32)
    n_out = len(pairs) // group
    out = np.zeros((n_out, 2, P.L, P.N), dtype=np.uint64)
    rc = _clib.lib().orc_ccmul(ctypes.byref(P.c()), _u64(keys.rlk), _u64(ct_a), _u64(ct_b), _i32(pa), _i32(pb),
                               len(pairs), group, _u64(out))
    if rc:
        raise ValueError("orc_ccmul failed")
    return out


def ppmul_terms(P: Params, a, b, terms_per_out) -> np.ndarray:
    """PPMul: out_o = sum a[i] * b[j] mod t (negacyclic)."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    ptr, ta, tb = _csr(terms_per_out)
    out = np.zeros((len(terms_per_out), P.N), dtype=np.uint64)
    _clib.lib().orc_ppmul_terms(ctypes.byref(P.c()), _u64(a), _u64(b), _i32(ptr), _i32(ta), _i32(tb),
                                len(terms_per_out), _u64(out))
    return out


def round_scalar(P: Params, value: int) -> list:
    """floor((t * value + floor(q/2)) / q) mod q_i for one signed integer."""
    nw = 40
    words = np.asarray([(value >> (32 * i)) & 0xFFFFFFFF for i in range(nw)], dtype=np.uint32)
    out = np.zeros(P.L, dtype=np.uint64)
    _clib.lib().orc_round_scalar(ctypes.byref(P.c()), _u32(words), nw, _u64(out))
    return [int(v) for v in out]
