"""Pins for the oracle's HE Add / Sub (Sec. 3.2) and plaintext operations, and
for a multiplication chain with rescale at every level (Sec. 3.1's log q
bookkeeping: each HE Mul + rescale drops one prime).

Exact pins use the decryption relation b - a*s in coefficient form: addition
is linear in it, a plaintext product multiplies it by the plaintext
polynomial (schoolbook negacyclic product with Python integers).
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle.encoding import encode

from test_oracle_scheme import negacyclic_int, tiny


def _rand_ct(prm, l, seed):
    rng = np.random.default_rng(seed)
    return np.stack([np.stack([rng.integers(0, int(prm.q[i]), size=prm.N, dtype=np.uint64) for i in range(l)])
                     for _ in range(2)])


@pytest.mark.parametrize("l", [5, 2])
def test_add_sub_are_linear_in_the_decryption(l):
    prm = tiny()
    sk = oracle.keygen_sk(prm, 3)
    c1, c2 = _rand_ct(prm, l, 1), _rand_ct(prm, l, 2)
    d1, d2 = oracle.decrypt_residues(prm, sk, c1, l), oracle.decrypt_residues(prm, sk, c2, l)
    da = oracle.decrypt_residues(prm, sk, oracle.add(prm, c1, c2, l), l)
    ds = oracle.decrypt_residues(prm, sk, oracle.sub(prm, c1, c2, l), l)
    for i in range(l):
        q = int(prm.q[i])
        assert da[i].tolist() == [(int(x) + int(y)) % q for x, y in zip(d1[i], d2[i])]
        assert ds[i].tolist() == [(int(x) - int(y)) % q for x, y in zip(d1[i], d2[i])]
    assert np.array_equal(oracle.sub(prm, oracle.add(prm, c1, c2, l), c2, l), c1)
    # the largest residues: the sum wraps exactly once
    top = np.stack([np.stack([np.full(prm.N, int(prm.q[i]) - 1, dtype=np.uint64) for i in range(l)])] * 2)
    s = oracle.add(prm, top, top, l)
    assert all((s[h, i] == np.uint64(int(prm.q[i]) - 2)).all() for h in range(2) for i in range(l))


@pytest.mark.parametrize("l", [5, 3])
def test_plaintext_product_and_sum_exact(l):
    prm = tiny()
    sk = oracle.keygen_sk(prm, 4)
    c = _rand_ct(prm, l, 9)
    rng = np.random.default_rng(l)
    t = rng.integers(-(1 << 40), 1 << 40, size=prm.N, dtype=np.int64)
    t[0], t[1] = -(1 << 62), (1 << 62) - 1
    pt = oracle.plain_ntt(prm, t, l)
    dc = oracle.decrypt_residues(prm, sk, c, l)
    dm = oracle.decrypt_residues(prm, sk, oracle.mul_plain(prm, c, pt, l), l)
    dp = oracle.decrypt_residues(prm, sk, oracle.add_plain(prm, c, pt, l), l)
    tl = [int(v) for v in t]
    for i in range(l):
        q = int(prm.q[i])
        want = [v % q for v in negacyclic_int([int(x) for x in dc[i]], tl)]
        assert dm[i].tolist() == want
        assert dp[i].tolist() == [(int(x) + v) % q for x, v in zip(dc[i], tl)]
    # multiplying by the constant 1 is the identity, by X a negacyclic shift
    one = np.zeros(prm.N, dtype=np.int64)
    one[0] = 1
    assert np.array_equal(oracle.mul_plain(prm, c, oracle.plain_ntt(prm, one, l), l), c)
    x = np.zeros(prm.N, dtype=np.int64)
    x[1] = 1
    dx = oracle.decrypt_residues(prm, sk, oracle.mul_plain(prm, c, oracle.plain_ntt(prm, x, l), l), l)
    for i in range(l):
        q = int(prm.q[i])
        assert dx[i].tolist() == [(-int(dc[i][-1])) % q] + [int(v) for v in dc[i][:-1]]


def _n12():
    prm = oracle.preset("n12")
    sc = 2.0 ** oracle.PRESETS["n12"]["scale_bits"]
    ks, s1, s2 = si.SEEDS["n12"]
    sk = oracle.keygen_sk(prm, ks)
    pk = oracle.keygen_pk(prm, sk, ks)
    return prm, sc, sk, pk, s1, s2


def test_add_and_plaintext_ops_decrypt_n12():
    prm, sc, sk, pk, s1, s2 = _n12()
    m1, m2 = si.messages(prm.N // 2, s1), si.messages(prm.N // 2, s2)
    c1 = oracle.encrypt_poly(prm, pk, encode(m1, prm.logN, sc), prm.L, s1)
    c2 = oracle.encrypt_poly(prm, pk, encode(m2, prm.logN, sc), prm.L, s2)
    L = prm.L
    assert np.abs(oracle.decrypt(prm, sk, oracle.add(prm, c1, c2, L), L, sc) - (m1 + m2)).max() < 2.0 ** -19
    assert np.abs(oracle.decrypt(prm, sk, oracle.sub(prm, c1, c2, L), L, sc) - (m1 - m2)).max() < 2.0 ** -19
    pt = oracle.plain_ntt(prm, encode(m2, prm.logN, sc), L)
    prod = oracle.rescale(prm, oracle.mul_plain(prm, c1, pt, L), L)
    z = oracle.decrypt(prm, sk, prod, L - 1, sc * sc / int(prm.q[L - 1]))
    assert 0 < np.abs(z - m1 * m2).max() < 2.0 ** -14
    z = oracle.decrypt(prm, sk, oracle.add_plain(prm, c1, pt, L), L, sc)
    assert np.abs(z - (m1 + m2)).max() < 2.0 ** -19


def test_squaring_chain_descends_the_levels_n12():
    """Encode at scale q_{L-1}; each HE Mul + rescale keeps the scale near the
    prime size (Delta^2 / q_{l-1}) and drops one prime, down to level 1."""
    prm, _, sk, pk, s1, _ = _n12()
    evk = oracle.keygen_evk(prm, sk, si.SEEDS["n12"][0])
    m = 0.5 * si.messages(prm.N // 2, s1)
    L = prm.L
    scale = float(int(prm.q[L - 1]))
    ct = oracle.encrypt_poly(prm, pk, encode(m, prm.logN, scale), L, s1)
    want = m
    for l in range(L, 1, -1):
        ct = oracle.rescale(prm, oracle.he_mul(prm, ct, ct, evk, l), l)
        scale = scale * scale / int(prm.q[l - 1])
        want = want * want
        z = oracle.decrypt(prm, sk, ct, l - 1, scale)
        assert np.abs(z - want).max() < 2.0 ** -12, l
