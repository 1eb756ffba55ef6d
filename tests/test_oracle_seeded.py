"""Pins for the seeded evaluation key (a halves from a per-element counter
sampler, so a device can regenerate them instead of reading them).

The sampler is pinned against its definition evaluated with Python integers
over the SplitMix64 words (SplitMix64 itself is pinned by the golden vectors),
by range and uniformity statistics, and the key by its defining relation and by
decryption of an HE Mul that uses it.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle.encoding import encode

from test_oracle_scheme import negacyclic_int, tiny

ST_SEED_A = 144


def test_sampler_closed_form():
    L = oracle.lib()
    for seed, j, idx, t in ((1, 0, 0, 97), (2024, 3, 12345, (1 << 54) - 33), (7, 11, 1 << 20, (1 << 57) - 111),
                            (0, 0, 5, 3)):
        S = L.or_splitmix64(seed, ST_SEED_A + j)          # stream state = word (ST + j) of the seed's generator
        w1, w2 = L.or_splitmix64(S, 2 * idx), L.or_splitmix64(S, 2 * idx + 1)
        want = ((w1 << 64) + w2) * t >> 128
        assert oracle.seeded_a(seed, j, idx, t) == want


def test_sampler_range_and_uniformity():
    t = (1 << 54) - 33
    v = np.array([oracle.seeded_a(99, 2, i, t) for i in range(40000)], dtype=np.float64)
    assert v.min() >= 0 and v.max() < t
    assert abs(v.mean() / t - 0.5) < 0.01
    hist = np.histogram(v / t, bins=16, range=(0, 1))[0]
    chi2 = float(((hist - 2500.0) ** 2 / 2500.0).sum())
    assert chi2 < 45.0  # 15 degrees of freedom: p ~ 1e-4
    # different digits and seeds give different streams
    assert oracle.seeded_a(99, 3, 0, t) != oracle.seeded_a(99, 2, 0, t)
    assert oracle.seeded_a(98, 2, 0, t) != oracle.seeded_a(99, 2, 0, t)


def test_seeded_key_relation():
    """b_j - a_j*s - [i in I_j] P*s^2 is one small error polynomial, a_j the sampler's."""
    prm = tiny()
    s = oracle.keygen_sk(prm, 5)
    evk = oracle.keygen_evk_seeded(prm, s, 5)
    s_int = [int(v) for v in s]
    s2 = negacyclic_int(s_int, s_int)
    P = 1
    for v in prm.p:
        P *= int(v)
    for j in range(prm.dnum):
        I = list(prm.digit(j, prm.L))
        errs = []
        for x, t in enumerate(prm.ext):
            assert [int(v) for v in evk[j, 1, x]] == [oracle.seeded_a(5, j, x * prm.N + n, t) for n in range(prm.N)]
            psi = int(prm.psi_p[x]) if x < prm.K else int(prm.psi_q[x - prm.K])
            S = oracle.ntt(np.array([v % t for v in s_int], dtype=np.uint64), t, psi, prm.logN)
            diff = [(int(b) - int(a) * int(sv)) % t for b, a, sv in zip(evk[j, 0, x], evk[j, 1, x], S)]
            dc = oracle.intt(np.array(diff, dtype=np.uint64), t, psi, prm.logN).tolist()
            if x >= prm.K and (x - prm.K) in I:
                dc = [(v - (P % t) * (c % t)) % t for v, c in zip(dc, s2)]
            ec = [v if v < t // 2 else v - t for v in dc]
            assert max(abs(v) for v in ec) <= 19
            errs.append(ec)
        assert all(e == errs[0] for e in errs) and any(errs[0])
    # the same error streams as the plain key: only the a halves differ
    plain = oracle.keygen_evk(prm, s, 5)
    assert not np.array_equal(plain[:, 1], evk[:, 1])


def test_he_mul_with_seeded_key_decrypts_n12():
    prm = oracle.preset("n12")
    sc = 2.0 ** oracle.PRESETS["n12"]["scale_bits"]
    ks, s1, s2 = si.SEEDS["n12"]
    sk = oracle.keygen_sk(prm, ks)
    pk = oracle.keygen_pk(prm, sk, ks)
    evk = oracle.keygen_evk_seeded(prm, sk, ks)
    m1, m2 = si.messages(prm.N // 2, s1), si.messages(prm.N // 2, s2)
    c1 = oracle.encrypt_poly(prm, pk, encode(m1, prm.logN, sc), prm.L, s1)
    c2 = oracle.encrypt_poly(prm, pk, encode(m2, prm.logN, sc), prm.L, s2)
    L = prm.L
    c3 = oracle.rescale(prm, oracle.he_mul(prm, c1, c2, evk, L), L)
    z = oracle.decrypt(prm, sk, c3, L - 1, sc * sc / int(prm.q[L - 1]))
    assert 2.0 ** -40 < np.abs(z - m1 * m2).max() < 2.0 ** -14
