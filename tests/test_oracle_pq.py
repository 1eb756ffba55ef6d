"""Pins for the oracle's single-division HE Mul + rescale (ModDown and rescale
as one division by M = P q_{l-1}).

The closed form is checked with Python integers, independently of the
oracle's conversion: Y = P d + KS is rebuilt from the tensor product (written
out here) and the key-switch intermediate KS, its CRT value taken over P Q_l,
and every output coefficient must be floor(Y / M) - floor(sum_j y_j / b_j) mod
q_i.  The result is also compared with HE Mul followed by a rescale (two
floors: the two differ by a small integer per coefficient) and decrypted.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle.encoding import encode

from test_oracle_scheme import crt, ppsi, qpsi, rand_ct, tiny, to_coeff


def _rand_evk(prm, seed):
    rng = np.random.default_rng(seed)
    return np.stack([np.stack([np.stack([rng.integers(0, int(t), size=prm.N, dtype=np.uint64) for t in prm.ext])
                               for _ in range(2)]) for _ in range(prm.dnum)])


def _tensor(prm, c1, c2, l):
    """d0 = b1 b2, d1 = a1 b2 + a2 b1 element-wise mod q_i (NTT domain), Python ints."""
    d = np.zeros((2, l, prm.N), dtype=np.uint64)
    for i in range(l):
        q = int(prm.q[i])
        for n in range(prm.N):
            b1, a1, b2, a2 = (int(c1[0, i, n]), int(c1[1, i, n]), int(c2[0, i, n]), int(c2[1, i, n]))
            d[0, i, n] = b1 * b2 % q
            d[1, i, n] = (a1 * b2 + a2 * b1) % q
    return d


@pytest.mark.parametrize("l", [5, 3, 2])
def test_single_division_closed_form(l):
    prm = tiny()
    c1, c2 = rand_ct(prm, l, 70 + l), rand_ct(prm, l, 80 + l)
    evk = _rand_evk(prm, 90 + l)
    out = oracle.he_mul_rescale_pq(prm, c1, c2, evk, l)
    assert out.shape == (2, l - 1, prm.N)
    _, _, KS = oracle.keyswitch(prm, oracle.tensor(prm, c1, c2, l)[2], evk, l, want_intermediates=True)
    d = _tensor(prm, c1, c2, l)
    ps = [int(v) for v in prm.p]
    qs = [int(v) for v in prm.q[:l]]
    P = 1
    for v in ps:
        P *= v
    B = ps + [qs[l - 1]]
    M = P * qs[l - 1]
    for h in range(2):
        # Y = P d + KS over the ext basis (specials first), NTT domain
        Y = np.zeros((prm.K + l, prm.N), dtype=np.uint64)
        Y[: prm.K] = KS[h, : prm.K]
        for i in range(l):
            Y[prm.K + i] = [(P * int(x) + int(k)) % qs[i] for x, k in zip(d[h, i], KS[h, prm.K + i])]
        yc = to_coeff(prm, Y, ppsi(prm) + qpsi(prm, l))
        oc = to_coeff(prm, out[h], qpsi(prm, l - 1))
        for n in range(prm.N):
            Yv, _ = crt(yc[:, n], ps + qs)
            u = Fraction(0)
            for b in B:
                Mh = M // b
                u += Fraction((Yv % b) * pow(Mh % b, -1, b) % b, b)
            want = Yv // M - (u.numerator // u.denominator)
            for i in range(l - 1):
                assert int(oc[i, n]) == want % qs[i], (h, n, i)


@pytest.mark.parametrize("l", [5, 2])
def test_single_division_is_near_the_two_floor_result(l):
    """Both approximate Y / (P q_{l-1}); per coefficient they differ by a small
    integer (the conversions' overflow terms, at most K + 1, and the inner floor)."""
    prm = tiny()
    c1, c2 = rand_ct(prm, l, 60 + l), rand_ct(prm, l, 65 + l)
    evk = _rand_evk(prm, 67 + l)
    pq = oracle.he_mul_rescale_pq(prm, c1, c2, evk, l)
    two = oracle.rescale(prm, oracle.he_mul(prm, c1, c2, evk, l), l)
    qs = [int(v) for v in prm.q[: l - 1]]
    Q = 1
    for v in qs:
        Q *= v
    diffs = set()
    for h in range(2):
        a = to_coeff(prm, pq[h], qpsi(prm, l - 1))
        b = to_coeff(prm, two[h], qpsi(prm, l - 1))
        for n in range(prm.N):
            x, _ = crt(a[:, n], qs)
            y, _ = crt(b[:, n], qs)
            dlt = (x - y) % Q
            dlt = dlt - Q if dlt > Q // 2 else dlt
            assert abs(dlt) <= prm.K + 2
            diffs.add(dlt)
    assert len(diffs) > 1  # not the same bits


def test_single_division_decrypts_n12():
    prm = oracle.preset("n12")
    sc = 2.0 ** oracle.PRESETS["n12"]["scale_bits"]
    ks, s1, s2 = si.SEEDS["n12"]
    sk = oracle.keygen_sk(prm, ks)
    pk = oracle.keygen_pk(prm, sk, ks)
    evk = oracle.keygen_evk(prm, sk, ks)
    m1, m2 = si.messages(prm.N // 2, s1), si.messages(prm.N // 2, s2)
    L = prm.L
    c1 = oracle.encrypt_poly(prm, pk, encode(m1, prm.logN, sc), L, s1)
    c2 = oracle.encrypt_poly(prm, pk, encode(m2, prm.logN, sc), L, s2)
    c3 = oracle.he_mul_rescale_pq(prm, c1, c2, evk, L)
    z = oracle.decrypt(prm, sk, c3, L - 1, sc * sc / int(prm.q[L - 1]))
    # n12 has K = 1: the conversion's overflow term adds at most 2 per
    # coefficient, within the two-floor bound's margin
    assert 2.0 ** -40 < np.abs(z - m1 * m2).max() < 2.0 ** -14
