"""Plain CPU oracle for full-RNS CKKS HE Mul -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library never does,
and this package never imports the product.  The only module both sides use is
``seeded_inputs`` (seeded synthetic messages and level draws), which holds none
of the method's arithmetic.

The arithmetic lives in ``oracle.c`` (uint64 residues, ``unsigned __int128``
products, plain ``%`` reductions) and follows "HEAAN Demystified"
(arXiv 2003.04510): NTT = Algo 3 with Algo 4's butterfly, iNTT as described
beneath Algo 4, the HE Mul flow of Fig. 2 in its full-RNS form (Sec. 7,
Table 11), encryption/decryption and rescale of Sec. 3.1.  Encoding and
decoding (``oracle.encoding``) use numpy's FFT as a library primitive.

Functions whose only pin is the decryption bound are marked "parity unpinned"
in their docstrings; every other function is pinned by a closed form or a brute
force check in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no vector flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u64, i64, i32, dbl = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        P = ctypes.c_void_p
        sig = {
            "or_mulmod": (u64, [u64, u64, u64]),
            "or_addmod": (u64, [u64, u64, u64]),
            "or_submod": (u64, [u64, u64, u64]),
            "or_powmod": (u64, [u64, u64, u64]),
            "or_invmod": (u64, [u64, u64]),
            "or_is_prime": (i32, [u64]),
            "or_gen_primes": (i32, [i32, i32, i32, P, i32, P]),
            "or_min_psi": (u64, [u64, i32]),
            "or_ntt": (None, [P, i32, u64, u64]),
            "or_intt": (None, [P, i32, u64, u64]),
            "or_butterfly_count": (u64, []),
            "or_reset_butterfly_count": (None, []),
            "or_splitmix64": (u64, [u64, u64]),
            "or_sample_gauss": (None, [u64, u64, dbl, i64, P]),
            "or_sample_zo": (None, [u64, u64, i64, P]),
            "or_sample_uniform": (None, [u64, u64, u64, i64, P]),
            "or_keygen_sk": (None, [i32, i32, u64, P]),
            "or_keygen_pk": (None, [i32, i32, P, P, dbl, P, u64, P]),
            "or_keygen_evk": (None, [i32, i32, i32, i32, P, P, P, P, dbl, P, u64, P]),
            "or_encrypt": (None, [i32, i32, P, P, dbl, P, P, i32, u64, P]),
            "or_decrypt": (None, [i32, P, P, P, P, i32, P]),
            "or_tensor": (None, [i32, i32, P, P, P, P, P, P]),
            "or_modup_digit": (None, [i32, i32, i32, i32, P, P, i32, P, P]),
            "or_inner_product": (None, [i32, i32, i32, i32, i32, P, P, P, P, P]),
            "or_moddown": (None, [i32, i32, i32, P, P, P, P, P, P]),
            "or_keyswitch": (None, [i32, i32, i32, i32, i32, P, P, P, P, P, P, P, P, P]),
            "or_he_mul": (None, [i32, i32, i32, i32, i32, P, P, P, P, P, P, P, P]),
            "or_rescale": (None, [i32, i32, P, P, P, P]),
            "or_he_mul_rescale_pq": (None, [i32, i32, i32, i32, i32, P, P, P, P, P, P, P, P]),
            "or_automorphism": (None, [P, i32, u64, u64, P]),
            "or_keygen_rot": (None, [i32, i32, i32, i32, P, P, P, P, dbl, P, u64, u64, P]),
            "or_rotate": (None, [i32, i32, i32, i32, i32, P, P, P, P, P, u64, P, P]),
            "or_add": (None, [i32, i32, P, P, P, P]),
            "or_sub": (None, [i32, i32, P, P, P, P]),
            "or_plain_ntt": (None, [i32, i32, P, P, P, P]),
            "or_mul_plain": (None, [i32, i32, P, P, P, P]),
            "or_add_plain": (None, [i32, i32, P, P, P, P]),
            "or_seeded_a": (u64, [u64, i32, u64, u64]),
            "or_keygen_evk_seeded": (None, [i32, i32, i32, i32, P, P, P, P, dbl, P, u64, P]),
            "or_nr_polymul": (None, [i32, i32, P, P, P, i32, P, i32, P, i32, P]),
            "or_nr_he_mul": (None, [i32, i32, i32, i32, i32, P, P, P, P, P, P]),
            "or_nr_rescale": (None, [i32, i32, i32, P, P]),
            "or_nr_keygen": (None, [i32, i32, i32, P, P, dbl, P, u64, P, P]),
            "or_nr_encrypt": (None, [i32, i32, i32, i32, P, P, dbl, P, P, u64, P]),
            "or_nr_decrypt": (None, [i32, i32, i32, P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


# --------------------------------------------------------------------------
# Parameters (reading c-1: largest NTT-friendly primes, descending; smallest
# primitive 2N-th root; specials exclude the ciphertext primes).
# --------------------------------------------------------------------------
@dataclass
class Params:
    logN: int
    L: int
    K: int
    alpha: int
    q_bits: int
    p_bits: int
    h: int = 64
    sigma: float = 3.2
    q: np.ndarray = field(default=None, repr=False)
    p: np.ndarray = field(default=None, repr=False)
    psi_q: np.ndarray = field(default=None, repr=False)
    psi_p: np.ndarray = field(default=None, repr=False)

    @property
    def N(self) -> int:
        return 1 << self.logN

    @property
    def dnum(self) -> int:
        return -(-self.L // self.alpha)

    def beta(self, l: int) -> int:
        return -(-l // self.alpha)

    def digit(self, j: int, l: int) -> range:
        return range(j * self.alpha, min((j + 1) * self.alpha, l))

    @property
    def ext(self) -> list[int]:
        """Moduli in ext order: K special primes first, then the L ciphertext primes."""
        return [int(x) for x in self.p] + [int(x) for x in self.q]


_param_cache: dict = {}


def make_params(logN, L, K, alpha, q_bits, p_bits, h=64, sigma=3.2) -> Params:
    key = (logN, L, K, alpha, q_bits, p_bits, h, sigma)
    if key in _param_cache:
        return _param_cache[key]
    lb = lib()
    q = np.zeros(L, dtype=np.uint64)
    if lb.or_gen_primes(logN, q_bits, L, None, 0, _p(q)) != 0:
        raise ValueError("not enough ciphertext primes")
    p = np.zeros(max(K, 1), dtype=np.uint64)
    if lb.or_gen_primes(logN, p_bits, K, _p(q), L, _p(p)) != 0:
        raise ValueError("not enough special primes")
    p = p[:K].copy()
    psi_q = np.array([lb.or_min_psi(int(x), logN) for x in q], dtype=np.uint64)
    psi_p = np.array([lb.or_min_psi(int(x), logN) for x in p], dtype=np.uint64)
    prm = Params(logN, L, K, alpha, q_bits, p_bits, h, sigma, q, p, psi_q, psi_p)
    _param_cache[key] = prm
    return prm


# Workload presets (the configurations the build is measured on).
PRESETS = {
    # N=2^12, 3 x 50-bit limbs + one 51-bit special prime, one limb per digit
    "n12": dict(logN=12, L=3, K=1, alpha=1, q_bits=50, p_bits=51, h=64, scale_bits=40),
    # N=2^15 serving preset: 16 limbs + 8 specials, alpha 8
    "n15": dict(logN=15, L=16, K=8, alpha=8, q_bits=54, p_bits=55, h=192, scale_bits=50),
    # N=2^16, 24 x 54-bit limbs + 8 x 55-bit specials, dnum 3
    "n16": dict(logN=16, L=24, K=8, alpha=8, q_bits=54, p_bits=55, h=192, scale_bits=50),
    # N=2^17, 44 x 54-bit limbs + 12 x 54-bit specials, dnum 4
    "n17": dict(logN=17, L=44, K=12, alpha=11, q_bits=54, p_bits=54, h=192, scale_bits=50),
}


def preset(name: str) -> Params:
    d = dict(PRESETS[name])
    d.pop("scale_bits")
    return make_params(**d)


# --------------------------------------------------------------------------
# Thin wrappers (allocation + argument marshalling only).
# --------------------------------------------------------------------------
def ntt(a, q: int, psi: int, logN: int) -> np.ndarray:
    out = _u64(a).copy()
    lib().or_ntt(_p(out), logN, q, psi)
    return out


def intt(a, q: int, psi: int, logN: int) -> np.ndarray:
    out = _u64(a).copy()
    lib().or_intt(_p(out), logN, q, psi)
    return out


def keygen_sk(prm: Params, seed: int) -> np.ndarray:
    s = np.zeros(prm.N, dtype=np.int64)
    lib().or_keygen_sk(prm.logN, prm.h, seed, _p(s))
    return s


def keygen_pk(prm: Params, sk: np.ndarray, seed: int) -> np.ndarray:
    pk = np.zeros((2, prm.L, prm.N), dtype=np.uint64)
    lib().or_keygen_pk(prm.logN, prm.L, _p(prm.q), _p(prm.psi_q), prm.sigma, _p(sk), seed, _p(pk))
    return pk


def keygen_evk(prm: Params, sk: np.ndarray, seed: int) -> np.ndarray:
    evk = np.zeros((prm.dnum, 2, prm.K + prm.L, prm.N), dtype=np.uint64)
    lib().or_keygen_evk(prm.logN, prm.L, prm.K, prm.alpha, _p(prm.q), _p(prm.psi_q), _p(prm.p),
                        _p(prm.psi_p), prm.sigma, _p(sk), seed, _p(evk))
    return evk


def keygen_evk_seeded(prm: Params, sk: np.ndarray, seed: int) -> np.ndarray:
    """Evaluation key whose a halves come from the per-element counter sampler
    (seeded_a); the full [dnum][2][K+L][N] key, b halves first."""
    evk = np.zeros((prm.dnum, 2, prm.K + prm.L, prm.N), dtype=np.uint64)
    lib().or_keygen_evk_seeded(prm.logN, prm.L, prm.K, prm.alpha, _p(prm.q), _p(prm.psi_q), _p(prm.p),
                               _p(prm.psi_p), prm.sigma, _p(sk), seed, _p(evk))
    return evk


def seeded_a(seed: int, j: int, idx: int, t: int) -> int:
    return int(lib().or_seeded_a(seed, j, idx, t))


def encrypt_poly(prm: Params, pk: np.ndarray, pt: np.ndarray, level: int, seed: int) -> np.ndarray:
    pt = np.ascontiguousarray(pt, dtype=np.int64)
    ct = np.zeros((2, level, prm.N), dtype=np.uint64)
    lib().or_encrypt(prm.logN, prm.L, _p(prm.q), _p(prm.psi_q), prm.sigma, _p(_u64(pk)), _p(pt),
                     level, seed, _p(ct))
    return ct


def decrypt_residues(prm: Params, sk: np.ndarray, ct: np.ndarray, level: int) -> np.ndarray:
    m = np.zeros((level, prm.N), dtype=np.uint64)
    lib().or_decrypt(prm.logN, _p(prm.q), _p(prm.psi_q), _p(np.ascontiguousarray(sk, dtype=np.int64)),
                     _p(_u64(ct)), level, _p(m))
    return m


def tensor(prm: Params, ct1, ct2, level: int):
    ct1, ct2 = _u64(ct1), _u64(ct2)
    d = np.zeros((3, level, prm.N), dtype=np.uint64)
    lib().or_tensor(prm.logN, level, _p(prm.q), _p(ct1), _p(ct2), _p(d[0]), _p(d[1]), _p(d[2]))
    return d


def modup_digit(prm: Params, x, level: int, j: int) -> np.ndarray:
    U = np.zeros((prm.K + level, prm.N), dtype=np.uint64)
    lib().or_modup_digit(prm.logN, level, prm.K, prm.alpha, _p(prm.q), _p(prm.p), j, _p(_u64(x)), _p(U))
    return U


def inner_product(prm: Params, U, evk, level: int) -> np.ndarray:
    KS = np.zeros((2, prm.K + level, prm.N), dtype=np.uint64)
    lib().or_inner_product(prm.logN, level, prm.L, prm.K, prm.alpha, _p(prm.q), _p(prm.p),
                           _p(_u64(U)), _p(_u64(evk)), _p(KS))
    return KS


def moddown(prm: Params, X, level: int) -> np.ndarray:
    out = np.zeros((level, prm.N), dtype=np.uint64)
    lib().or_moddown(prm.logN, level, prm.K, _p(prm.q), _p(prm.psi_q), _p(prm.p), _p(prm.psi_p),
                     _p(_u64(X)), _p(out))
    return out


def keyswitch(prm: Params, d2, evk, level: int, want_intermediates: bool = False):
    E, beta = prm.K + level, prm.beta(level)
    ks = np.zeros((2, level, prm.N), dtype=np.uint64)
    U = np.zeros((beta, E, prm.N), dtype=np.uint64) if want_intermediates else None
    KS = np.zeros((2, E, prm.N), dtype=np.uint64) if want_intermediates else None
    lib().or_keyswitch(prm.logN, level, prm.L, prm.K, prm.alpha, _p(prm.q), _p(prm.psi_q), _p(prm.p),
                       _p(prm.psi_p), _p(_u64(d2)), _p(_u64(evk)), _p(ks),
                       _p(U) if U is not None else None, _p(KS) if KS is not None else None)
    if want_intermediates:
        return ks, U, KS
    return ks


def he_mul(prm: Params, ct1, ct2, evk, level: int) -> np.ndarray:
    out = np.zeros((2, level, prm.N), dtype=np.uint64)
    lib().or_he_mul(prm.logN, level, prm.L, prm.K, prm.alpha, _p(prm.q), _p(prm.psi_q), _p(prm.p),
                    _p(prm.psi_p), _p(_u64(ct1)), _p(_u64(ct2)), _p(_u64(evk)), _p(out))
    return out


def he_mul_rescale_pq(prm: Params, ct1, ct2, evk, level: int) -> np.ndarray:
    """HE Mul with ModDown and rescale as one division by P q_{l-1} (one floor
    instead of two); [2][level-1][N] NTT domain."""
    out = np.zeros((2, level - 1, prm.N), dtype=np.uint64)
    lib().or_he_mul_rescale_pq(prm.logN, level, prm.L, prm.K, prm.alpha, _p(prm.q), _p(prm.psi_q), _p(prm.p),
                               _p(prm.psi_p), _p(_u64(ct1)), _p(_u64(ct2)), _p(_u64(evk)), _p(out))
    return out


def rescale(prm: Params, ct, level: int) -> np.ndarray:
    out = np.zeros((2, level - 1, prm.N), dtype=np.uint64)
    lib().or_rescale(prm.logN, level, _p(prm.q), _p(prm.psi_q), _p(_u64(ct)), _p(out))
    return out


# --------------------------------------------------------------------------
# Rotation (NEXT-1): Galois automorphisms and key switching with rotation keys.
# --------------------------------------------------------------------------
def galois_elt(prm: Params, steps: int) -> int:
    """g = 5^steps mod 2N: kappa_g moves slot k+steps to slot k (steps may be negative)."""
    return pow(5, steps % (prm.N // 2), 2 * prm.N)


def conj_elt(prm: Params) -> int:
    """g = 2N - 1: kappa_g conjugates every slot."""
    return 2 * prm.N - 1


def automorphism(a, q: int, g: int, logN: int) -> np.ndarray:
    """a(X) -> a(X^g) mod (X^N + 1, q), coefficient form."""
    a = _u64(a)
    out = np.zeros_like(a)
    lib().or_automorphism(_p(a), logN, q, g, _p(out))
    return out


def keygen_rot(prm: Params, sk: np.ndarray, g: int, seed: int) -> np.ndarray:
    rk = np.zeros((prm.dnum, 2, prm.K + prm.L, prm.N), dtype=np.uint64)
    lib().or_keygen_rot(prm.logN, prm.L, prm.K, prm.alpha, _p(prm.q), _p(prm.psi_q), _p(prm.p),
                        _p(prm.psi_p), prm.sigma, _p(np.ascontiguousarray(sk, dtype=np.int64)), g, seed, _p(rk))
    return rk


def rotate(prm: Params, ct, g: int, rk, level: int) -> np.ndarray:
    out = np.zeros((2, level, prm.N), dtype=np.uint64)
    lib().or_rotate(prm.logN, level, prm.L, prm.K, prm.alpha, _p(prm.q), _p(prm.psi_q), _p(prm.p),
                    _p(prm.psi_p), _p(_u64(ct)), g, _p(_u64(rk)), _p(out))
    return out


# --------------------------------------------------------------------------
# HE Add / Sub (Sec. 3.2) and plaintext operations (NEXT-4).
# --------------------------------------------------------------------------
def add(prm: Params, ct1, ct2, level: int) -> np.ndarray:
    out = np.zeros((2, level, prm.N), dtype=np.uint64)
    lib().or_add(prm.logN, level, _p(prm.q), _p(_u64(ct1)), _p(_u64(ct2)), _p(out))
    return out


def sub(prm: Params, ct1, ct2, level: int) -> np.ndarray:
    out = np.zeros((2, level, prm.N), dtype=np.uint64)
    lib().or_sub(prm.logN, level, _p(prm.q), _p(_u64(ct1)), _p(_u64(ct2)), _p(out))
    return out


def plain_ntt(prm: Params, coeffs, level: int) -> np.ndarray:
    pt = np.zeros((level, prm.N), dtype=np.uint64)
    lib().or_plain_ntt(prm.logN, level, _p(prm.q), _p(prm.psi_q), _p(np.ascontiguousarray(coeffs, dtype=np.int64)),
                       _p(pt))
    return pt


def mul_plain(prm: Params, ct, pt, level: int) -> np.ndarray:
    out = np.zeros((2, level, prm.N), dtype=np.uint64)
    lib().or_mul_plain(prm.logN, level, _p(prm.q), _p(_u64(ct)), _p(_u64(pt)), _p(out))
    return out


def add_plain(prm: Params, ct, pt, level: int) -> np.ndarray:
    out = np.zeros((2, level, prm.N), dtype=np.uint64)
    lib().or_add_plain(prm.logN, level, _p(prm.q), _p(_u64(ct)), _p(_u64(pt)), _p(out))
    return out


# --------------------------------------------------------------------------
# Big-integer helpers for decryption (Python ints are the big integers).
# --------------------------------------------------------------------------
def crt_centered(residues: np.ndarray, moduli) -> list[int]:
    """CRT-reconstruct each column of residues[l][N] and centre it in (-Q/2, Q/2]."""
    moduli = [int(m) for m in moduli]
    Q = 1
    for m in moduli:
        Q *= m
    coefs = []
    for m in moduli:
        Qh = Q // m
        coefs.append(Qh * pow(Qh % m, -1, m))
    l, N = residues.shape
    cols = [residues[i].tolist() for i in range(l)]
    out = []
    for n in range(N):
        v = 0
        for i in range(l):
            v += cols[i][n] * coefs[i]
        v %= Q
        if v > Q // 2:
            v -= Q
        out.append(v)
    return out


def decrypt(prm: Params, sk, ct, level: int, scale: float) -> np.ndarray:
    """Decrypt and decode to N/2 complex slots (Sec. 3.1 decryption relation)."""
    from .encoding import decode
    m = decrypt_residues(prm, sk, ct, level)
    coeffs = crt_centered(m, prm.q[:level])
    return decode(np.array([float(c) for c in coeffs]) / scale, prm.logN)


# --------------------------------------------------------------------------
# NEXT-2: the paper's non-RNS HEAAN HE Mul (BigInt coefficients modulo powers
# of two; CRT / NTT / iCRT polynomial products).  Word-major BigInt arrays:
# a[w][n] = word w of coefficient n, little-endian, ceil(k/64) words.
# --------------------------------------------------------------------------
@dataclass
class NrParams:
    logN: int
    logQ: int         # top modulus Q = 2^logQ (fresh ciphertexts at logq = logQ)
    logp: int         # rescaling factor p = 2^logp (= the scaling factor Delta)
    np1: int          # primes of a ciphertext x ciphertext product (region 1)
    np2: int          # primes of a ciphertext x evaluation-key product (region 2)
    h: int = 64
    sigma: float = 3.2
    primes: np.ndarray = field(default=None, repr=False)
    psis: np.ndarray = field(default=None, repr=False)

    @property
    def N(self) -> int:
        return 1 << self.logN


def nwords(k: int) -> int:
    return (k + 63) // 64


def nr_params(logN: int, logQ: int, logp: int, prime_bits: int = 57, h: int = 64) -> NrParams:
    """np from the product bounds: P > 4 N 2^(2 logQ) (region 1 and key
    generation) and P > 4 N 2^(3 logQ) (region 2); primes are the largest
    prime_bits-bit primes = 1 mod 2N, descending, with their smallest roots."""
    import math
    cand = np.zeros(96, dtype=np.uint64)
    rc = lib().or_gen_primes(logN, prime_bits, len(cand), None, 0, _p(cand))
    assert rc == 0

    def count(bits):  # fewest leading primes whose product exceeds 2^bits
        tot = 0.0
        for i, q in enumerate(cand):
            tot += math.log2(int(q))
            if tot > bits:
                return i + 1
        raise ValueError("not enough primes")

    np1 = count(2 * logQ + logN + 2)
    np2 = count(3 * logQ + logN + 2)
    primes = np.ascontiguousarray(cand[:np2])
    psis = np.array([lib().or_min_psi(int(q), logN) for q in primes], dtype=np.uint64)
    return NrParams(logN, logQ, logp, np1, np2, h, 3.2, primes, psis)


def nr_polymul(prm: NrParams, A, wa: int, B, wb: int, kout: int, small=None, np_: int = None) -> np.ndarray:
    out = np.zeros((nwords(kout), prm.N), dtype=np.uint64)
    npr = np_ or prm.np2
    lib().or_nr_polymul(prm.logN, npr, _p(prm.primes), _p(prm.psis), _p(_u64(A)), wa,
                        _p(_u64(B)) if B is not None else None, wb,
                        _p(np.ascontiguousarray(small, dtype=np.int64)) if small is not None else None, kout, _p(out))
    return out


def nr_keygen(prm: NrParams, sk, seed: int):
    pk = np.zeros((2, nwords(prm.logQ), prm.N), dtype=np.uint64)
    evk = np.zeros((2, nwords(2 * prm.logQ), prm.N), dtype=np.uint64)
    lib().or_nr_keygen(prm.logN, prm.logQ, prm.np1, _p(prm.primes), _p(prm.psis), prm.sigma,
                       _p(np.ascontiguousarray(sk, dtype=np.int64)), seed, _p(pk), _p(evk))
    return pk, evk


def nr_encrypt(prm: NrParams, pk, pt, logq: int, seed: int) -> np.ndarray:
    ct = np.zeros((2, nwords(logq), prm.N), dtype=np.uint64)
    lib().or_nr_encrypt(prm.logN, logq, prm.logQ, prm.np1, _p(prm.primes), _p(prm.psis), prm.sigma, _p(_u64(pk)),
                        _p(np.ascontiguousarray(pt, dtype=np.int64)), seed, _p(ct))
    return ct


def nr_decrypt_coeffs(prm: NrParams, sk, ct, logq: int) -> np.ndarray:
    m = np.zeros(prm.N, dtype=np.float64)
    lib().or_nr_decrypt(prm.logN, logq, prm.np1, _p(prm.primes), _p(prm.psis),
                        _p(np.ascontiguousarray(sk, dtype=np.int64)), _p(_u64(ct)), _p(m))
    return m


def nr_decrypt(prm: NrParams, sk, ct, logq: int, scale: float) -> np.ndarray:
    from .encoding import decode
    return decode(nr_decrypt_coeffs(prm, sk, ct, logq) / scale, prm.logN)


def nr_he_mul(prm: NrParams, ct1, ct2, evk, logq: int) -> np.ndarray:
    out = np.zeros((2, nwords(logq), prm.N), dtype=np.uint64)
    lib().or_nr_he_mul(prm.logN, logq, prm.logQ, prm.np1, prm.np2, _p(prm.primes), _p(prm.psis), _p(_u64(ct1)),
                       _p(_u64(ct2)), _p(_u64(evk)), _p(out))
    return out


def nr_rescale(prm: NrParams, ct, logq: int) -> np.ndarray:
    out = np.zeros((2, nwords(logq - prm.logp), prm.N), dtype=np.uint64)
    lib().or_nr_rescale(prm.logN, logq, prm.logp, _p(_u64(ct)), _p(out))
    return out


def words_to_ints(a: np.ndarray, k: int) -> list[int]:
    """Word-major [W][N] -> Python ints (unsigned, < 2^k)."""
    W, N = a.shape
    out = []
    for n in range(N):
        v = 0
        for w in range(W - 1, -1, -1):
            v = (v << 64) | int(a[w, n])
        out.append(v % (1 << k))
    return out


def ints_to_words(vals, k: int) -> np.ndarray:
    W = nwords(k)
    a = np.zeros((W, len(vals)), dtype=np.uint64)
    for n, v in enumerate(vals):
        v %= 1 << k
        for w in range(W):
            a[w, n] = (v >> (64 * w)) & ((1 << 64) - 1)
    return a
