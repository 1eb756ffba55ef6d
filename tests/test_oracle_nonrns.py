"""Pins for the oracle's non-RNS HEAAN HE Mul (the paper's own algorithm).

Every BigInt polynomial product (CRT, NTT, element-wise product, iNTT, exact
iCRT) is checked against the schoolbook negacyclic product with Python
integers at N = 16; the HE Mul against an independent Python re-statement of
Fig. 2 with big integers; the keys by their defining relations; and the whole
scheme by decryption of an HE Mul followed by a rescale.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle.encoding import encode

from test_oracle_scheme import negacyclic_int

LOGN, LOGQ, LOGP = 4, 120, 20


@pytest.fixture(scope="module")
def prm():
    return oracle.nr_params(LOGN, LOGQ, LOGP)


def _rand_words(rng, k, N):
    return oracle.ints_to_words([int(rng.integers(0, 1 << 62)) << 60 ^ int(rng.integers(0, 1 << 62)) << 3
                                 ^ int(rng.integers(0, 1 << 62)) << 120 ^ int(rng.integers(0, 1 << 62)) << 180
                                 for _ in range(N)], k)


def _mod(vals, k):
    return [v % (1 << k) for v in vals]


@pytest.mark.parametrize("ka,kb,kout,region", [(120, 120, 120, 1), (100, 120, 57, 1), (120, 240, 240, 2),
                                              (64, 240, 130, 2), (240, 0, 240, 1)])
def test_polymul_is_the_schoolbook_product(prm, ka, kb, kout, region):
    rng = np.random.default_rng(ka + kb + kout)
    N = prm.N
    A = _rand_words(rng, ka, N)
    a = oracle.words_to_ints(A, ka)
    npr = prm.np1 if region == 1 else prm.np2
    if kb:
        B = _rand_words(rng, kb, N)
        b = oracle.words_to_ints(B, kb)
        C = oracle.nr_polymul(prm, A, oracle.nwords(ka), B, oracle.nwords(kb), kout, np_=npr)
    else:  # a small signed polynomial
        b = [int(v) for v in rng.integers(-3, 4, size=N)]
        C = oracle.nr_polymul(prm, A, oracle.nwords(ka), None, 0, kout, small=np.array(b), np_=npr)
    assert oracle.words_to_ints(C, kout) == _mod(negacyclic_int(a, b), kout)


def _py_he_mul(c1, c2, evk, logq, logQ):
    """Fig. 2 with Python integers: region 1 mod q, region 2 mod qQ, rounding division by Q."""
    q, qQ, Q = 1 << logq, 1 << (logq + logQ), 1 << logQ
    b1, a1 = c1
    b2, a2 = c2
    d0 = [v % q for v in negacyclic_int(b1, b2)]
    d1 = [(u + v) % q for u, v in zip(negacyclic_int(a1, b2), negacyclic_int(a2, b1))]
    d2 = [v % q for v in negacyclic_int(a1, a2)]
    out = []
    for h, d in ((0, d0), (1, d1)):
        k = [v % qQ for v in negacyclic_int(d2, evk[h])]
        ks = [((v + (Q >> 1)) >> logQ) % q for v in k]
        out.append([(x + y) % q for x, y in zip(d, ks)])
    return out


@pytest.mark.parametrize("logq", [120, 100])
def test_he_mul_matches_big_integer_restatement(prm, logq):
    rng = np.random.default_rng(logq)
    N = prm.N
    c1 = np.stack([_rand_words(rng, logq, N) for _ in range(2)])
    c2 = np.stack([_rand_words(rng, logq, N) for _ in range(2)])
    evk = np.stack([_rand_words(rng, 2 * LOGQ, N) for _ in range(2)])
    got = oracle.nr_he_mul(prm, c1, c2, evk, logq)
    want = _py_he_mul([oracle.words_to_ints(c1[h], logq) for h in range(2)],
                      [oracle.words_to_ints(c2[h], logq) for h in range(2)],
                      [oracle.words_to_ints(evk[h], 2 * LOGQ) for h in range(2)], logq, LOGQ)
    assert [oracle.words_to_ints(got[h], logq) for h in range(2)] == want
    # rescale: round(c / p) mod q / p
    rs = oracle.nr_rescale(prm, got, logq)
    for h in range(2):
        want_rs = [((v + (1 << (LOGP - 1))) >> LOGP) % (1 << (logq - LOGP)) for v in want[h]]
        assert oracle.words_to_ints(rs[h], logq - LOGP) == want_rs


def test_key_relations(prm):
    sk = oracle.keygen_sk(oracle.make_params(LOGN, 1, 1, 1, 50, 51, h=4), 9)
    pk, evk = oracle.nr_keygen(prm, sk, 9)
    s = [int(v) for v in sk]
    Q, QQ = 1 << LOGQ, 1 << (2 * LOGQ)
    pb, pa = oracle.words_to_ints(pk[0], LOGQ), oracle.words_to_ints(pk[1], LOGQ)
    e = [(b - v) % Q for b, v in zip(pb, negacyclic_int(pa, s))]
    e = [v if v < Q // 2 else v - Q for v in e]
    assert max(abs(v) for v in e) <= 19 and any(e)
    eb, ea = oracle.words_to_ints(evk[0], 2 * LOGQ), oracle.words_to_ints(evk[1], 2 * LOGQ)
    s2 = negacyclic_int(s, s)
    e = [(b - v - Q * t) % QQ for b, v, t in zip(eb, negacyclic_int(ea, s), s2)]
    e = [v if v < QQ // 2 else v - QQ for v in e]
    assert max(abs(v) for v in e) <= 19 and any(e)


def test_he_mul_rescale_decrypts():
    """Encrypt, HE Mul, rescale, decrypt: m1*m2 at N = 2^10, log Q = 300, log p = 30."""
    prm = oracle.nr_params(10, 300, 30)
    sk = oracle.keygen_sk(oracle.make_params(10, 1, 1, 1, 50, 51, h=64), 31)
    pk, evk = oracle.nr_keygen(prm, sk, 31)
    sc = 2.0 ** prm.logp
    m1, m2 = si.messages(prm.N // 2, 32), si.messages(prm.N // 2, 33)
    c1 = oracle.nr_encrypt(prm, pk, encode(m1, prm.logN, sc), prm.logQ, 34)
    c2 = oracle.nr_encrypt(prm, pk, encode(m2, prm.logN, sc), prm.logQ, 35)
    # Delta = 2^30: the fresh noise (v e + e0 - e1 s, about sqrt(N) sigma sqrt(h) per slot)
    # is near 2^-17 of a unit; HE Mul and rescale keep the same order
    assert np.abs(oracle.nr_decrypt(prm, sk, c1, prm.logQ, sc) - m1).max() < 2.0 ** -12
    c3 = oracle.nr_he_mul(prm, c1, c2, evk, prm.logQ)
    assert np.abs(oracle.nr_decrypt(prm, sk, c3, prm.logQ, sc * sc) - m1 * m2).max() < 2.0 ** -12
    c4 = oracle.nr_rescale(prm, c3, prm.logQ)
    err = np.abs(oracle.nr_decrypt(prm, sk, c4, prm.logQ - prm.logp, sc) - m1 * m2).max()
    assert 2.0 ** -30 < err < 2.0 ** -12
